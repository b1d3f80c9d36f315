"""Treecode parameter choice (degree n, MAC theta, leaf size N_L) under an
error bar: the selection rule on the host, and on the device a choice whose
fields stay within the bar of the direct sums (Eqs. of the singularity-
subtracted Yukawa and Coulomb convolutions, summed in full by the oracle)."""
import math

import numpy as np
import pytest

from paper_2003_01833_gb300.autotune import Trial, autotune, rel_errors, report, select


def _t(n, th, nl, ms, err, seg=8192):
    return Trial(n, th, nl, seg, 1.0, ms, err, 0)


def test_select_takes_fastest_within_tol():
    trials = [_t(8, 0.5, 2000, 5.0, 1e-8), _t(6, 0.8, 2000, 1.0, 3e-6), _t(8, 0.7, 2000, 2.0, 4e-7),
              _t(6, 0.7, 1000, 1.5, 9e-7)]
    best = select(trials, 1e-6)
    assert (best.degree, best.theta, best.leaf_size) == (6, 0.7, 1000)
    assert select(trials, 1e-7).conv_ms == 5.0


def test_select_rejects_nonfinite_and_returns_none():
    trials = [_t(6, 0.8, 2000, 0.5, math.nan), _t(6, 0.8, 1000, 0.4, math.inf), _t(8, 0.7, 2000, 2.0, 2e-6)]
    assert select(trials, 1e-6) is None
    assert select(trials, 1e-5).conv_ms == 2.0
    assert select([], 1.0) is None


def test_select_bar_is_inclusive():
    assert select([_t(6, 0.7, 2000, 1.0, 1e-6)], 1e-6) is not None


def test_select_across_segment_lengths():
    trials = [_t(8, 0.7, 2000, 2.0, 4e-7, 8192), _t(8, 0.7, 2000, 1.8, 4.1e-7, 16384),
              _t(8, 0.7, 2000, 2.2, 4e-7, 4096)]
    assert select(trials, 1e-6).segment == 16384


def test_grid_for_large_meshes_uses_a_narrower_grid_and_fp32c_reference():
    import paper_2003_01833_gb300.tagi as T
    from paper_2003_01833_gb300.autotune import grid_for

    small, big = grid_for(300_000), grid_for(1_700_000)
    assert small == {"segments": (4096, 8192, 16384)}
    assert big["prec_ref"] == T.TAGI_FP32C and len(big["degrees"]) * len(big["thetas"]) * \
        len(big["leaf_sizes"]) * len(big["segments"]) == 24


def test_rel_errors_plain_and_weighted():
    """An error at a point of tiny quadrature weight (a mesh point next to a
    nucleus) dominates the plain norm and vanishes from the weighted one;
    the largest field decides."""
    ref = [np.ones(4), 2 * np.ones(4)]
    w = np.array([1e-12, 1.0, 1.0, 1.0])
    rows = [np.array([1 + 1e-3, 1, 1, 1]), 2 * np.ones(4)]
    l2, wt = rel_errors(rows, ref, w)
    assert l2 == pytest.approx(1e-3 / 2)
    assert wt == pytest.approx(1e-3 * math.sqrt(1e-12 / 3), rel=1e-9)
    rows = [np.ones(4), 2 * np.ones(4) + np.array([0, 4e-6, 0, 0])]
    l2, wt = rel_errors(rows, ref, w)
    assert l2 == pytest.approx(4e-6 / 4) and wt == pytest.approx(4e-6 / (2 * math.sqrt(3)))


def test_unknown_norm_is_rejected_before_any_work():
    with pytest.raises(ValueError):
        autotune(None, None, None, None, norm="max")


def test_report_is_json_ready():
    import json

    trials = [_t(8, 0.7, 2000, 2.0, 4e-7)]
    out = report(select(trials, 1e-6), trials, (8, 0.4, 2000), 1e-6)
    s = json.loads(json.dumps(out))
    assert s["best"]["theta"] == 0.7 and s["reference"]["theta"] == 0.4 and len(s["trials"]) == 1
    assert s["norm"] == "l2"
    assert json.loads(json.dumps(report(None, [], (8, 0.4, 2000), 1e-6)))["best"] is None


@pytest.mark.gpu
def test_choice_meets_the_bar_against_direct_sums():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g

    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2003_01833_gb300.tagi as T
    from paper_2003_01833_gb300 import autotune as A
    from paper_2003_01833_gb300 import workloads as W

    wl = W.hydrogen_adaptive(seed=1)
    m = wl.mesh
    rng = np.random.default_rng(3)
    r = np.sqrt(np.sum(m.xyz**2, axis=0))
    f = np.stack([wl.f[0], np.exp(-1.5 * r) * (1 + 0.1 * np.cos(m.xyz[1]))])
    k = [float(wl.k[0]), 1.7]
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    tol = 1e-6
    best, trials, ref = A.autotune(dev(m.xyz), dev(m.w), dev(f), k, rho=dev(wl.rho), tol=tol, degrees=(6, 8),
                                   thetas=(0.6, 0.8), leaf_sizes=(1000, 2000), segments=(4096, 16384))
    print({(t.degree, t.theta, t.leaf_size, t.segment): (round(t.conv_ms, 3), f"{t.err_l2:.1e}",
                                                         f"{t.err_weighted:.1e}") for t in trials})
    assert len(trials) == 16 and best is not None and best.max_rel_err <= tol
    # the segment length regroups the float32 sums only: the two lengths of
    # one (n, theta, N_L) agree to float32 accumulation
    by = {}
    for t in trials:
        by.setdefault((t.degree, t.theta, t.leaf_size), []).append(t.err_l2)
    assert all(abs(a - b) <= 1e-7 for a, b in by.values())
    assert all(t.max_rel_err == t.err_l2 and math.isfinite(t.err_weighted) for t in trials)
    assert all(t.conv_ms >= best.conv_ms for t in trials if t.ok(tol))
    # the chosen configuration against the oracle's direct sums on sampled targets
    tg = np.sort(rng.choice(wl.n, size=3000, replace=False))
    with T.Tree(dev(m.xyz), dev(m.w), theta=best.theta, degree=best.degree, leaf_size=best.leaf_size,
                segment=best.segment, prec=T.TAGI_FP32C) as tr:
        u = torch.empty((2, wl.n), dtype=torch.float64, device="cuda")
        vh = torch.empty(wl.n, dtype=torch.float64, device="cuda")
        T.tagi_fields_conv(tr.handle, dev(f), k, u, rho=dev(wl.rho), vh=vh)
        u, vh = u.cpu().numpy(), vh.cpu().numpy()
    for o in range(2):
        d = oracle.direct_yukawa(m.xyz, m.w, f[o], k[o], targets=tg)
        e = np.linalg.norm(u[o][tg] - d) / np.linalg.norm(d)
        assert e < 2 * tol, (o, e)
    d = oracle.direct_coulomb(m.xyz, m.w, wl.rho, targets=tg)
    assert np.linalg.norm(vh[tg] - d) / np.linalg.norm(d) < 2 * tol

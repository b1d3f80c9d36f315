"""The learned warm start on the device (tagi_mlp_*) against the oracle
(oracle/mlp.py), and measured by the SCF iteration.

- Features: bit-exact bfloat16 encodings (both sides form them in float64,
  in the same operation order, and round once, ties to even).
- Forward: the device computes each point in float32 (products of bfloat16
  operands, fmaf chains of 8 and 32 terms, tanhf); the oracle in float64.
  Bound: |dy| <= 1e-4 (1 + |y|) per point, derived from about 80 float32
  roundings of relative size 6e-8 on sums of magnitude <= 10 in these
  networks; the median must sit near float32 resolution (<= 1e-6).
- Gradient: float32 per point, float64 over points; relative L2 1e-4.
- Adam: float64 on both sides: one step from a given gradient to 1e-14.
- Training: 40 full-batch steps follow the oracle's loss curve to 1e-3.
- Warm start: psi = s (1 + y) normalised, to 1e-5 relative.
- SCF measure: trained on three H2 geometries, the predicted start for a fourth
  is closer to the converged orbital than the superposition start, and the
  SCF from it converges to the same energy in no more Green iterations.
"""
import numpy as np
import pytest

import oracle.mlp as M
from paper_2003_01833_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g

    g.build()
    import paper_2003_01833_gb300.tagi as T

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return T


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def as_values(feat):
    """int16 tensor of bfloat16 encodings -> float64 host values."""
    u = feat.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def _points(seed, n):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.normal(size=(3, n)) * 2.5)


def _params(seed):
    rng = np.random.default_rng(seed)
    p = W.mlp_init(seed)
    p[256:288] = rng.normal(size=32) * 0.3  # b1
    p[1312:1344] = rng.normal(size=32) * 0.3  # b2
    p[-1] = 0.1
    return p


def test_features_bit_exact(T):
    nuc = np.array([[-0.7, 0.0, 0.0], [0.7, 0.0, 0.0], [0.3, 2.1, -0.4]])
    xyz = _points(0, 40001)
    xyz[:, :3] = nuc.T  # points on the nuclei
    xyz[:, 3] = 0.0     # the midpoint of the first two
    f = as_values(T.tagi_mlp_features(dev(xyz), nuc))
    np.testing.assert_array_equal(f, M.features(xyz, nuc))
    wl = W.hydrogen_molecule(1.4, tol_m=1e-5)
    f = as_values(T.tagi_mlp_features(dev(wl.mesh.xyz), wl.meta["nuclei"]))
    np.testing.assert_array_equal(f, M.features(wl.mesh.xyz, wl.meta["nuclei"]))


def test_ordered_features_bit_exact(T):
    nuc = np.array([[-1.06581, 0.0, 0.0], [1.06581, 0.0, 0.0]])
    xyz = _points(21, 30011)
    xyz[:, :2] = nuc.T
    f = as_values(T.tagi_mlp_features(dev(xyz), nuc, ordered=True))
    np.testing.assert_array_equal(f, M.features(xyz, nuc, ordered=True))
    z = [5.7, 7.7]  # Slater 1s exponents of C and O
    f = as_values(T.tagi_mlp_features(dev(xyz), nuc, ordered=True, scale=z))
    np.testing.assert_array_equal(f, M.features(xyz, nuc, ordered=True, scale=z))
    nuc3 = np.array([[-0.7, 0.0, 0.0], [0.7, 0.0, 0.0], [0.3, 2.1, -0.4]])
    z3 = [1.0, 2.5, 4.0]
    f = as_values(T.tagi_mlp_features(dev(xyz), nuc3, scale=z3))
    np.testing.assert_array_equal(f, M.features(xyz, nuc3, scale=z3))


def test_forward_against_oracle(T):
    nuc = np.array([[-0.7, 0.0, 0.0], [0.7, 0.0, 0.0]])
    xyz = _points(1, 100003)
    feat = T.tagi_mlp_features(dev(xyz), nuc)
    x = as_values(feat)
    for seed in (2, 3):
        p = _params(seed)
        with T.Mlp(p) as m:
            y = m.forward(feat).cpu().numpy().astype(np.float64)
            np.testing.assert_array_equal(m.params(), p)
        ref = M.forward(p, x)[0]
        d = np.abs(y - ref)
        print("forward: max", d.max(), "median", np.median(d))
        assert np.all(d <= 1e-4 * (1.0 + np.abs(ref)))
        assert np.median(d) <= 1e-6


def _train_data(T, seed, n):
    rng = np.random.default_rng(seed)
    nuc = np.array([[-0.75, 0.0, 0.0], [0.75, 0.0, 0.0]])
    xyz = _points(seed, n)
    feat = T.tagi_mlp_features(dev(xyz), nuc)
    x = as_values(feat)
    r = np.sqrt(((xyz.T - nuc[0]) ** 2).sum(1)) + np.sqrt(((xyz.T - nuc[1]) ** 2).sum(1))
    t = (0.3 * np.tanh(r - 2.0) + 0.05 * rng.normal(size=n)).astype(np.float32)
    wt = (rng.uniform(0.5, 1.5, size=n) / n).astype(np.float32)
    return feat, x, t, wt


def test_gradient_and_adam_against_oracle(T):
    feat, x, t, wt = _train_data(T, 4, 50001)
    p = _params(5)
    with T.Mlp(p) as m:
        L, g = m.gradient(feat, dev(t, torch.float32), dev(wt, torch.float32))
        Lo, go = M.loss_grad(p, x, t.astype(np.float64), wt.astype(np.float64))
        print("gradient: rel L2", np.linalg.norm(g - go) / np.linalg.norm(go), "loss", L, Lo)
        assert abs(L - Lo) <= 1e-5 * Lo
        assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
        # one Adam step applies the device gradient exactly as the oracle's update
        m.train_step(feat, dev(t, torch.float32), dev(wt, torch.float32), lr=1e-3)
        q = m.params()
    qo, _, _ = M.adam_step(p, np.zeros_like(p), np.zeros_like(p), g, 1, 1e-3)
    np.testing.assert_allclose(q, qo, rtol=1e-14, atol=1e-17)


def test_training_follows_the_oracle(T):
    feat, x, t, wt = _train_data(T, 6, 20011)
    p0 = _params(7)
    steps, lr = 40, 3e-3
    tt, ww = dev(t, torch.float32), dev(wt, torch.float32)
    with T.Mlp(p0) as m:
        losses = [m.train_step(feat, tt, ww, lr, want_loss=True) for _ in range(steps)]
        p = m.params()
    po, lo = M.train(p0, x, t.astype(np.float64), wt.astype(np.float64), steps, lr)
    print("training: loss", losses[0], "->", losses[-1], "oracle", lo[0], "->", lo[-1])
    np.testing.assert_allclose(losses, lo, rtol=1e-3)
    assert np.linalg.norm(p - po) <= 1e-3 * np.linalg.norm(po)
    assert losses[-1] < 0.5 * losses[0]


def test_warm_start_against_oracle(T):
    wl = W.hydrogen_molecule(1.3, tol_m=1e-5)
    p = _params(8) * 0.5
    feat = T.tagi_mlp_features(dev(wl.mesh.xyz), wl.meta["nuclei"])
    with T.Mlp(p) as m:
        psi = m.warm_start(feat, dev(wl.psi[0]), dev(wl.mesh.w)).cpu().numpy()
    ref = M.warm_start(p, as_values(feat), wl.psi[0], wl.mesh.w)
    assert np.linalg.norm(psi - ref) <= 1e-5 * np.linalg.norm(ref)
    assert abs(np.sum(psi * psi * wl.mesh.w) - 1.0) < 1e-12


def test_predicted_start_is_measured_by_the_scf(T):
    from paper_2003_01833_gb300 import warmstart as WS

    records = WS.generate([1.2, 1.4, 1.6, 1.5], log=print)
    orb, eig, info = WS.train(records, [0, 1, 2], steps=1500, log=print)
    rows = WS.evaluate(orb, eig, records, [3], R_range=info["R_range"], log=print)
    orb.close()
    eig.close()
    r = rows[0]
    assert r["used_prediction"] and r["converged"]
    assert r["orbital_error"]["predicted"] < 0.5 * r["orbital_error"]["superposition"]
    assert abs(r["eps"]["predicted"] - r["eps"]["converged"]) < 0.01
    assert r["green_iterations"]["predicted"] <= r["green_iterations"]["superposition"]
    assert abs(r["e_total"]["predicted"] - r["e_total"]["superposition"]) < 1e-5


# ------------------------------------------ H = 64 on the tensor cores
def _params64(seed):
    rng = np.random.default_rng(seed)
    p = W.mlp_init(seed, hidden=64)
    H, F = 64, 8
    p[H * F:H * F + H] = rng.normal(size=H) * 0.3  # b1
    o2 = H * F + H + H * H
    p[o2:o2 + H] = rng.normal(size=H) * 0.3  # b2
    p[-1] = 0.1
    return p


def _rows_ok(d, ref, rate):
    """Per-point bound: float32 tensor-core sums and float32 tanh against
    float64.  A point whose float32 activation lies within float32 rounding
    of a bfloat16 rounding boundary can round to the neighbouring bfloat16
    value (a rate of about 1e-5 per activation, so a few tenths of a percent
    of the points); those may differ by up to 1e-2 (1 + |y|)."""
    tight = d <= 2e-5 * (1.0 + np.abs(ref))
    return np.mean(~tight) <= rate and np.all(d <= 1e-2 * (1.0 + np.abs(ref)))


def test_forward_h64_tensor_cores_against_oracle(T):
    nuc = np.array([[-0.7, 0.0, 0.0], [0.7, 0.0, 0.0]])
    xyz = _points(11, 100003)
    feat = T.tagi_mlp_features(dev(xyz), nuc)
    x = as_values(feat)
    for seed in (12, 13):
        p = _params64(seed)
        with T.Mlp(p, hidden=64) as m:
            y = m.forward(feat).cpu().numpy().astype(np.float64)
            np.testing.assert_array_equal(m.params(), p)
        ref = M.forward_tc(p, x, 64)[0]
        d = np.abs(y - ref)
        print("forward H=64: max", d.max(), "median", np.median(d), "beyond 2e-5:",
              np.mean(d > 2e-5 * (1 + np.abs(ref))))
        assert _rows_ok(d, ref, 5e-3)
        assert np.median(d) <= 1e-6


def test_gradient_h64_tensor_cores_against_oracle(T):
    feat, x, t, wt = _train_data(T, 14, 50001)
    p = _params64(15)
    with T.Mlp(p, hidden=64) as m:
        L, g = m.gradient(feat, dev(t, torch.float32), dev(wt, torch.float32))
        Lo, go = M.loss_grad_tc(p, x, t.astype(np.float64), wt.astype(np.float64), 64)
        rel = np.linalg.norm(g - go) / np.linalg.norm(go)
        print("gradient H=64: rel L2", rel, "loss", L, Lo)
        assert abs(L - Lo) <= 1e-5 * Lo
        assert rel <= 2e-3
        m.train_step(feat, dev(t, torch.float32), dev(wt, torch.float32), lr=1e-3)
        q = m.params()
    qo, _, _ = M.adam_step(p, np.zeros_like(p), np.zeros_like(p), g, 1, 1e-3)
    np.testing.assert_allclose(q, qo, rtol=1e-14, atol=1e-17)


def test_training_h64_follows_the_oracle(T):
    feat, x, t, wt = _train_data(T, 16, 20011)
    p0 = _params64(17)
    steps, lr = 40, 3e-3
    tt, ww = dev(t, torch.float32), dev(wt, torch.float32)
    with T.Mlp(p0, hidden=64) as m:
        losses = [m.train_step(feat, tt, ww, lr, want_loss=True) for _ in range(steps)]
        p = m.params()
    po, lo = M.train(p0, x, t.astype(np.float64), wt.astype(np.float64), steps, lr, H=64, tc=True)
    print("training H=64: loss", losses[0], "->", losses[-1], "oracle", lo[0], "->", lo[-1])
    np.testing.assert_allclose(losses, lo, rtol=1e-2)
    assert np.linalg.norm(p - po) <= 1e-2 * np.linalg.norm(po)
    assert losses[-1] < 0.5 * losses[0]


def test_warm_start_h64_against_oracle(T):
    wl = W.hydrogen_molecule(1.3, tol_m=1e-5)
    p = _params64(18) * 0.5
    feat = T.tagi_mlp_features(dev(wl.mesh.xyz), wl.meta["nuclei"])
    with T.Mlp(p, hidden=64) as m:
        psi = m.warm_start(feat, dev(wl.psi[0]), dev(wl.mesh.w)).cpu().numpy()
    ref = M.warm_start(p, as_values(feat), wl.psi[0], wl.mesh.w, H=64, tc=True)
    assert np.linalg.norm(psi - ref) <= 1e-4 * np.linalg.norm(ref)
    assert abs(np.sum(psi * psi * wl.mesh.w) - 1.0) < 1e-12

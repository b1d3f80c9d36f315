"""Green Iteration to convergence with Anderson mixing of eigenpairs
(tagi_green_iterate: Algorithm 2, Section 4.3) against the oracle's loop,
through the C ABI.

Float64 path: the same step decisions (which orbital converged at which
step) and the same iterates to rounding order, with and without mixing.
Tolerances: eps 1e-10 Ha, psi 1e-9 of its largest value (each step takes
a few hundred float64 sums; the Anderson normal equations add a factor of
their condition number, bounded here by testing at most 6 mixed steps).
FP32C path: converges to the float64 fixed point within the FP32C step
tolerance (eps 2e-6 Ha).
"""
import numpy as np
import pytest

import oracle
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _norm(v, w):
    return v / np.sqrt(np.sum(v * v * w))


@pytest.fixture(scope="module")
def hcase():
    """Hydrogen on the 36,000-point adaptive mesh: 1s and 2s starts."""
    wl = W.hydrogen_adaptive()
    w = wl.mesh.w
    r = np.sqrt(np.sum(wl.mesh.xyz**2, axis=0))
    p0 = _norm(np.exp(-r), w)
    p1 = (2.0 - r) * np.exp(-0.5 * r)
    p1 = _norm(p1 - np.sum(p1 * p0 * w) * p0, w)
    return wl, np.stack([p0, p1]), np.array([-0.5, -0.125]), oracle.Tree(wl.mesh.xyz, 2000)


def _gpu_loop(T, wl, psi0, eps0, vshift, prec, **kw):
    with T.Tree(dev(wl.mesh.xyz), dev(wl.mesh.w), theta=0.7, degree=6, leaf_size=2000, prec=prec) as tr:
        psi = dev(psi0)
        out = T.tagi_green_iterate(tr.handle, dev(wl.veff), vshift, psi, eps0, **kw)
        out["psi"] = psi.cpu().numpy()
    return out


@pytest.mark.parametrize("store_output", [False, True])
def test_plain_loop_matches_oracle_with_a_convergence_event(T, hcase, store_output):
    """A convergence event of orbital 0; the converged orbital keeps its step
    input (Algorithm 2) or, with store_output, its step output."""
    wl, psi0, eps0, otree = hcase
    w = wl.mesh.w
    free = oracle.green_iterate(otree, 0.7, 6, w, wl.veff, -0.5, psi0, eps0, tol_gi=0.0, max_iter=8, mix_tol=0.0)
    tr = free["trace"]
    # a tolerance between two steps of orbital 0, far from every residual of
    # both orbitals, so rounding cannot move a convergence decision
    def ok(k):
        t = np.sqrt(tr[k - 1, 0] * tr[k, 0])
        return tr[k, 0] < 0.8 * tr[k - 1, 0] and tr[k, 0] < tr[:k, 0].min() and np.all(tr[:, 1] > 1.2 * t)

    k = next(k for k in range(2, 7) if ok(k))
    tol = float(np.sqrt(tr[k - 1, 0] * tr[k, 0]))
    ref = oracle.green_iterate(otree, 0.7, 6, w, wl.veff, -0.5, psi0, eps0, tol_gi=tol, max_iter=8, mix_tol=0.0,
                               store_output=store_output)
    assert ref["iters"][0] == k + 1 and ref["iters"][1] == -1
    out = _gpu_loop(T, wl, psi0, eps0, -0.5, T.TAGI_FP64, tol_gi=tol, max_iter=8, mix_tol=0.0,
                    store_output=store_output)
    np.testing.assert_array_equal(out["iters"], ref["iters"])
    assert out["steps"] == ref["steps"] and out["field_steps"] == ref["field_steps"]
    assert out["n_converged"] == 1
    assert np.abs(out["eps"] - ref["eps"]).max() < 1e-10
    for o in range(2):
        assert np.abs(out["psi"][o] - ref["psi"][o]).max() < 1e-9 * np.abs(ref["psi"][o]).max()
    np.testing.assert_allclose(out["resid"], ref["resid"], rtol=1e-6)


@pytest.mark.parametrize("history", [0, 3])
def test_mixed_loop_matches_oracle(T, hcase, history):
    wl, psi0, eps0, otree = hcase
    w = wl.mesh.w
    ref = oracle.green_iterate(otree, 0.7, 6, w, wl.veff, -0.5, psi0, eps0, tol_gi=0.0, max_iter=6, beta=0.5,
                               history=history)
    out = _gpu_loop(T, wl, psi0, eps0, -0.5, T.TAGI_FP64, tol_gi=0.0, max_iter=6, beta=0.5, history=history)
    assert out["steps"] == 6 and np.all(out["iters"] == -1)
    assert np.abs(out["eps"] - ref["eps"]).max() < 1e-10
    for o in range(2):
        assert np.abs(out["psi"][o] - ref["psi"][o]).max() < 1e-9 * np.abs(ref["psi"][o]).max()


def test_fp32c_loop_reaches_the_fp64_fixed_point(T, hcase):
    """From psi = e^{-0.7 r}, eps = -0.4, mixing on: both precisions
    converge, to one eigenvalue within the FP32C tolerance, near -0.5 Ha."""
    wl, _, _, _ = hcase
    w = wl.mesh.w
    r = np.sqrt(np.sum(wl.mesh.xyz**2, axis=0))
    psi0 = _norm(np.exp(-0.7 * r), w)[None]
    kw = dict(tol_gi=1e-5, max_iter=40, beta=0.5, history=5)
    a = _gpu_loop(T, wl, psi0, np.array([-0.4]), 0.0, T.TAGI_FP64, **kw)
    b = _gpu_loop(T, wl, psi0, np.array([-0.4]), 0.0, T.TAGI_FP32C, **kw)
    assert a["n_converged"] == 1 and b["n_converged"] == 1
    assert abs(a["iters"][0] - b["iters"][0]) <= 1
    assert abs(a["eps"][0] - b["eps"][0]) < 2e-6
    assert abs(a["eps"][0] + 0.5) < 5e-3


def test_loop_reports_loss_of_decay(T):
    """On the uniform 8^3 mesh with V_shift = 0, mixing drives eps + V_shift
    to >= 0 (the oracle's loop stops there too); the library returns
    TAGI_ERR_INVALID_ARG with the last completed step in psi."""
    wl = W.hydrogen_1s(seed=0, ncell=8)
    w = wl.mesh.w
    x = wl.mesh.xyz.T
    r = np.sqrt(np.sum((x - np.array(wl.meta["nucleus"])) ** 2, axis=1))
    psi0 = _norm(np.exp(-0.7 * r), w)[None]
    otree = oracle.Tree(wl.mesh.xyz, 2000)
    with pytest.raises(ValueError):
        oracle.green_iterate(otree, 0.7, 6, w, wl.veff, 0.0, psi0, np.array([-0.4]), tol_gi=1e-7, max_iter=60)
    with T.Tree(dev(wl.mesh.xyz), dev(w), theta=0.7, degree=6, leaf_size=2000, prec=T.TAGI_FP64) as tr:
        psi = dev(psi0)
        with pytest.raises(T.TagiError) as e:
            T.tagi_green_iterate(tr.handle, dev(wl.veff), 0.0, psi, np.array([-0.4]), tol_gi=1e-7, max_iter=60)
        assert e.value.status == T.TAGI_ERR_INVALID_ARG and "non-negative" in str(e.value)
        assert torch.isfinite(psi).all()

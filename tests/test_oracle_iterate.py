"""Pins of the oracle's Green Iteration loop and Anderson mixing (Algorithm 2,
Section 4.3).

- Anderson mixing with one history entry is simple mixing x + beta F.
- On a linear fixed-point problem x = M x + b in d dimensions, Anderson
  mixing with unlimited history and beta = 1 is equivalent to GMRES (Walker
  and Ni, SIAM J. Numer. Anal. 49, 2011), so it reaches the solution of
  (I - M) x = b after at most d + 1 steps. A sign or index slip in the normal
  equations or in the update breaks that finite termination.
- The eigenvalue is part of the mixed vector: with the orbital fixed and eps
  following an affine map, the secant step lands on the fixed point in two
  steps only if the eps component enters the inner product.
- One loop step with mixing off is the batched Green step.
- Hydrogen on an adaptive mesh: with and without mixing the loop converges
  to one fixed point, within the mesh's discretisation error of eps = -0.5 Ha;
  mixing takes fewer steps.
- Converged orbitals keep their step input and stay fixed; the others stay
  orthogonal to them.

The hydrogen cases run on the p = 3 adaptive mesh (18,432 points; its
discretisation error in the 1s eigenvalue is 6.8e-3 Ha) with leaves of 500
points and degree 4, and share their loop runs, so the module runs in well
under a minute.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2003_01833_gb300 import workloads as W


def _run_linear(M, b, beta, history, steps):
    d = len(b)
    wx = np.ones(d)
    x = np.zeros(d)
    X, F = [], []
    out = []
    for _ in range(steps):
        f = M @ x + b - x
        X.append(x.copy())
        F.append(f)
        X, F = X[-(history + 1):], F[-(history + 1):]
        x = oracle.anderson_mix(np.array(X), np.array(F), beta, wx)
        out.append(x.copy())
    return out


def test_anderson_one_entry_is_simple_mixing():
    rng = np.random.default_rng(0)
    x, f, wx = rng.normal(size=7), rng.normal(size=7), rng.uniform(0.5, 2, size=7)
    np.testing.assert_array_equal(oracle.anderson_mix(x[None], f[None], 0.3, wx), x + 0.3 * f)


@pytest.mark.parametrize("d", [3, 6])
def test_anderson_linear_problem_terminates_like_gmres(d):
    rng = np.random.default_rng(d)
    Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    M = Q @ np.diag(rng.uniform(-0.9, 0.9, size=d)) @ Q.T + 0.05 * rng.normal(size=(d, d))
    b = rng.normal(size=d)
    xstar = np.linalg.solve(np.eye(d) - M, b)
    xs = _run_linear(M, b, beta=1.0, history=100, steps=d + 1)
    assert np.linalg.norm(xs[d] - xstar) < 1e-9 * np.linalg.norm(xstar)
    # simple mixing (history 0) is still far away after d + 1 steps
    ys = _run_linear(M, b, beta=1.0, history=0, steps=d + 1)
    assert np.linalg.norm(ys[d] - xstar) > 1e-4 * np.linalg.norm(xstar)


def test_anderson_mixes_the_eigenvalue_component():
    """x = (eps, psi) with psi already a fixed point and eps -> 0.5 eps + 1:
    two steps land on eps = 2 (a secant step on the 1-D affine map)."""
    n = 5
    w = np.full(n, 0.2)
    wx = np.concatenate([[1.0], w])
    psi = np.ones(n)
    eps = 0.0
    X, F = [], []
    for _ in range(2):
        X.append(np.concatenate([[eps], psi]))
        F.append(np.concatenate([[0.5 * eps + 1.0 - eps], np.zeros(n)]))
        x = oracle.anderson_mix(np.array(X), np.array(F), 0.5, wx)
        eps, psi = x[0], x[1:]
    assert abs(eps - 2.0) < 1e-14
    np.testing.assert_array_equal(psi, np.ones(n))


DEG = 4  # treecode degree of the hydrogen cases (theta = 0.7)


@functools.lru_cache(maxsize=None)
def _h_mesh():
    wl = W.hydrogen_adaptive(p=3)  # 18,432 points, nucleus at the origin
    r = np.sqrt(np.sum(wl.mesh.xyz**2, axis=0))
    return wl, oracle.Tree(wl.mesh.xyz, 500), wl.mesh.w, r


def _normalised(v, w):
    return v / np.sqrt(np.sum(v * v * w))


def test_one_step_is_the_green_step():
    wl, T, w, r = _h_mesh()
    p0 = _normalised(np.exp(-r), w)
    psi0 = np.stack([p0, _normalised((2.0 - r) * np.exp(-0.5 * r), w)])
    eps0 = np.array([-0.5, -0.125])
    a = oracle.green_step(T, 0.7, DEG, w, wl.veff, -0.5, psi0, eps0)
    b = oracle.green_iterate(T, 0.7, DEG, w, wl.veff, -0.5, psi0, eps0, tol_gi=0.0, max_iter=1, mix_tol=0.0)
    np.testing.assert_array_equal(a["psi"], b["psi"])
    # the Green step subtracts the shift after the update: one rounding apart
    np.testing.assert_allclose(a["eps"], b["eps"], rtol=1e-14)
    np.testing.assert_array_equal(a["resid"], b["resid"])
    assert b["steps"] == 1 and b["field_steps"] == 2 and np.all(b["iters"] == -1)


def test_hydrogen_loop_converges_with_and_without_mixing():
    """From psi = e^{-0.7 r}, eps = -0.4 both loops reach one fixed point,
    eps = -0.5 Ha up to the mesh's discretisation error (6.8e-3 on this
    mesh), and mixing (beta = 0.5) takes fewer steps."""
    wl, T, w, r = _h_mesh()
    psi0 = _normalised(np.exp(-0.7 * r), w)[None]
    eps0 = np.array([-0.4])
    plain = oracle.green_iterate(T, 0.7, DEG, w, wl.veff, 0.0, psi0, eps0, tol_gi=1e-5, max_iter=40, mix_tol=0.0)
    mixed = oracle.green_iterate(T, 0.7, DEG, w, wl.veff, 0.0, psi0, eps0, tol_gi=1e-5, max_iter=40, beta=0.5)
    assert plain["iters"][0] > 0 and mixed["iters"][0] > 0
    assert mixed["iters"][0] < plain["iters"][0]
    assert abs(plain["eps"][0] - mixed["eps"][0]) < 1e-5
    assert np.sqrt(np.sum((plain["psi"][0] - mixed["psi"][0]) ** 2 * w)) < 1e-4
    assert abs(plain["eps"][0] + 0.5) < 1e-2


# Two orbitals of hydrogen, 1s and 2s (eps -0.5 and -0.125 Ha), the 2s made
# orthogonal to the 1s.  With tol_gi = 3e-3 the 1s converges at step 3 of 5
# (residual 2.6e-3) and the 2s does not (its residual stays near 4e-3).
TOL2 = 3e-3


def _two_start():
    wl, T, w, r = _h_mesh()
    p0 = _normalised(np.exp(-r), w)
    p1 = (2.0 - r) * np.exp(-0.5 * r)
    p1 = _normalised(p1 - np.sum(p1 * p0 * w) * p0, w)
    return np.stack([p0, p1]), np.array([-0.5, -0.125])


@functools.lru_cache(maxsize=None)
def _two_run(store_output):
    wl, T, w, r = _h_mesh()
    psi0, eps0 = _two_start()
    return oracle.green_iterate(T, 0.7, DEG, w, wl.veff, -0.5, psi0, eps0, tol_gi=TOL2, max_iter=5, mix_tol=0.0,
                                store_output=store_output)


@functools.lru_cache(maxsize=None)
def _plain_steps(k):
    """k plain loop steps of both orbitals (tol_gi = 0, no mixing).  Their
    state is (psi, eps) alone, so k steps are k - 1 steps and one more from
    where those ended."""
    wl, T, w, r = _h_mesh()
    if k == 0:
        psi, eps = _two_start()
        return {"psi": psi, "eps": eps}
    prev = _plain_steps(k - 1)
    return oracle.green_iterate(T, 0.7, DEG, w, wl.veff, -0.5, prev["psi"], prev["eps"], tol_gi=0.0, max_iter=1,
                                mix_tol=0.0)


def test_plain_steps_compose():
    """The split used by _plain_steps: two single steps equal one call of
    two steps, bit for bit."""
    wl, T, w, r = _h_mesh()
    psi0, eps0 = _two_start()
    two = oracle.green_iterate(T, 0.7, DEG, w, wl.veff, -0.5, psi0, eps0, tol_gi=0.0, max_iter=2, mix_tol=0.0)
    np.testing.assert_array_equal(two["psi"], _plain_steps(2)["psi"])
    np.testing.assert_array_equal(two["eps"], _plain_steps(2)["eps"])


def test_converged_orbitals_stay_fixed_and_others_orthogonal():
    """The 1s converges first, keeps the input of its converging step, and
    the 2s stays orthogonal to it."""
    wl, T, w, r = _h_mesh()
    a = _two_run(False)
    it0 = a["iters"][0]
    assert 0 < it0 < a["steps"] and a["iters"][1] == -1
    assert a["field_steps"] == it0 + a["steps"]
    b = _plain_steps(it0 - 1)
    np.testing.assert_array_equal(a["psi"][0], b["psi"][0])
    np.testing.assert_array_equal(a["eps"][0], b["eps"][0])
    assert abs(np.sum(a["psi"][0] * a["psi"][1] * w)) < 1e-12
    assert abs(a["eps"][0] + 0.5) < 1e-2 and abs(a["eps"][1] + 0.125) < 1e-2


def test_store_output_keeps_the_converging_step_output():
    """With store_output a converged orbital keeps the output of its
    converging step: the iterate after it0 plain steps, one step past the
    stored input of Algorithm 2's rule (which the test above pins)."""
    wl, T, w, r = _h_mesh()
    a = _two_run(False)
    c = _two_run(True)
    it0 = c["iters"][0]
    assert it0 == a["iters"][0] and c["steps"] == a["steps"]
    b = _plain_steps(it0)
    np.testing.assert_array_equal(c["psi"][0], b["psi"][0])
    np.testing.assert_array_equal(c["eps"][0], b["eps"][0])
    assert np.sqrt(np.sum((c["psi"][0] - a["psi"][0]) ** 2 * w)) < TOL2  # within tol_gi of the input
    assert abs(np.sum(c["psi"][0] * c["psi"][1] * w)) < 1e-12

"""Pins of the oracle's Green step (Algorithm 2 lines 3-6, Eq. gradient-free,
Eq. quadrature-example): orthonormality of the Gram-Schmidt output, the
hydrogen 1s eigenpair (eps = -0.5 Ha, psi reproduced), and the closed-form
Hartree energy sqrt(a / (2 pi)) of a normalised Gaussian density."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_01833_gb300 import workloads as W

# treecode of these pins: theta = 0.7, degree 4, leaves of 500 points (its
# error is far below the mesh errors the pins bound)
DEG, LEAF = 4, 500


def test_hydrogen_step_reproduces_eigenpair():
    errs_eps, errs_psi = [], []
    for nc in (8, 12):
        wl = W.hydrogen_1s(seed=0, ncell=nc)
        T = oracle.Tree(wl.mesh.xyz, LEAF)
        w = wl.mesh.w
        psi0 = wl.psi / np.sqrt(np.sum(wl.psi**2 * w))
        out = oracle.green_step(T, 0.7, DEG, w, wl.veff, 0.0, psi0, np.array([-0.5]))
        errs_eps.append(abs(out["eps"][0] + 0.5))
        errs_psi.append(out["resid"][0])
    # uniform cells do not resolve the cusp, so convergence is slow (O(h))
    assert errs_eps[1] < 0.5 * errs_eps[0] and errs_eps[1] < 0.1
    assert errs_psi[1] < 0.5 * errs_psi[0] and errs_psi[1] < 0.06


def test_gauge_shift_only_moves_k():
    """With V_shift = s and eps + s fixed, the operator is the same, so psi~
    and the shifted eigenvalue agree; the returned eps differs by -s."""
    wl = W.hydrogen_1s(seed=1, ncell=8)
    T = oracle.Tree(wl.mesh.xyz, LEAF)
    w = wl.mesh.w
    a = oracle.green_step(T, 0.7, DEG, w, wl.veff + 0.5, -0.5, wl.psi, np.array([0.0]))
    b = oracle.green_step(T, 0.7, DEG, w, wl.veff, 0.0, wl.psi, np.array([-0.5]))
    np.testing.assert_allclose(a["psi_tilde"], b["psi_tilde"], rtol=1e-12, atol=1e-15)
    assert abs((a["eps"][0] - 0.5) - b["eps"][0]) < 1e-12


def test_mgs_orthonormal_and_ordered():
    wl = W.lithium(seed=1, tol_m=1e-2)
    T = oracle.Tree(wl.mesh.xyz, LEAF)
    w = wl.mesh.w
    out = oracle.green_step(T, 0.7, DEG, w, wl.veff, wl.vshift, wl.psi, wl.eps, rho=wl.rho)
    q = out["psi"]
    G = (q * w) @ q.T
    np.testing.assert_allclose(G, np.eye(2), atol=1e-12)
    # the first orbital is only normalised
    t0 = out["psi_tilde"][0]
    np.testing.assert_allclose(q[0], t0 / np.sqrt(np.sum(t0 * t0 * w)), rtol=1e-12, atol=1e-14)
    assert np.all(out["resid"] > 0) and np.all(np.isfinite(out["eps"]))
    assert out["eh"] > 0


def test_hartree_energy_of_gaussian():
    """E_H = 1/2 int V_H rho = sqrt(a/(2 pi)) for rho = (a/pi)^{3/2} e^{-a r^2}."""
    a = 1.0
    errs = []
    for nc in (8, 12):
        m = W.uniform_mesh(-8, 8, nc, 4)
        r2 = (m.xyz**2).sum(0)
        rho = (a / math.pi) ** 1.5 * np.exp(-a * r2)
        T = oracle.Tree(m.xyz, LEAF)
        v = oracle.treecode_coulomb(T, 0.7, DEG, rho, m.w)
        errs.append(abs(0.5 * np.sum(v * rho * m.w) - math.sqrt(a / (2 * math.pi))))
    assert errs[1] < 0.2 * errs[0] and errs[1] < 2e-4

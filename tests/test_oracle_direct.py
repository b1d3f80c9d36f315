"""Pins of the oracle's direct sums (Eq. direct-sum with the SS of Section 3.3).

The references here are independent of the oracle: closed forms (the Yukawa
potential of a Gaussian via erfc, the Coulomb potential erf(sqrt(a) r)/r of a
Gaussian density), scipy's adaptive quadrature of the radial shell formula,
and algebraic invariants of the sum (reciprocity, translation, scaling).
A dropped SS term, a wrong sign, a wrong 4 pi or a swapped w_i / w_j fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf, erfc

import oracle
from paper_2003_01833_gb300 import workloads as W

from . import radial

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def yukawa_of_gaussian(k, a, r):
    """u(r) = int e^{-k|x-y|}/(4 pi |x-y|) e^{-a |y|^2} dy (closed form)."""
    sa = math.sqrt(a)
    return ((math.pi / a) ** 1.5 / (8 * math.pi * r) * math.exp(k * k / (4 * a))
            * (np.exp(-k * r) * erfc(k / (2 * sa) - sa * r) - np.exp(k * r) * erfc(k / (2 * sa) + sa * r)))


def test_ss_integrals_golden_match_quadrature():
    """The analytic SS integrals of Section 3.3 (4 pi/k^2, 2 pi alpha^2)."""
    for line in open(os.path.join(GOLD, "ss_integrals.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, par, val = line.split()
        par, val = float(par), float(val)
        if kind == "yukawa":
            q, _ = integrate.quad(lambda r: 4 * math.pi * r * math.exp(-par * r), 0, np.inf)
            assert abs(val - 4 * math.pi / par**2) < 1e-12 * val
        else:
            q, _ = integrate.quad(lambda r: 4 * math.pi * r * math.exp(-r * r / par**2), 0, np.inf)
            assert abs(val - 2 * math.pi * par**2) < 1e-12 * val
        assert abs(q - val) < 1e-9 * val


def test_closed_form_reference_matches_shell_quadrature():
    r = np.array([0.3, 1.1, 2.0, 4.0])
    for k in (0.8, 1.5):
        q = radial.yukawa_radial(lambda s: math.exp(-s * s), k, r)
        np.testing.assert_allclose(q, yukawa_of_gaussian(k, 1.0, r), rtol=1e-9)
    q = radial.coulomb_radial(lambda s: math.pi**-1.5 * math.exp(-s * s), r)
    np.testing.assert_allclose(q, erf(r) / r, rtol=1e-9)


def _central(mesh, rmax=2.5, cap=300):
    r = np.sqrt((mesh.xyz**2).sum(0))
    ti = np.nonzero(r < rmax)[0]
    return ti[:: max(1, len(ti) // cap)], r


def test_yukawa_gaussian_converges_and_ss_helps():
    """SS direct sum -> closed form under refinement; SS beats no-SS (the
    in-scope analogue of Table singularity-subtraction)."""
    errs = []
    for nc in (8, 12, 16):
        m = W.uniform_mesh(-10, 10, nc, 4)
        ti, r = _central(m)
        f = np.exp(-r * r)
        for k in (1.0, 1.5):
            ref = yukawa_of_gaussian(k, 1.0, r[ti])
            u = oracle.direct_yukawa(m.xyz, m.w, f, k, ss=True, targets=ti)
            un = oracle.direct_yukawa(m.xyz, m.w, f, k, ss=False, targets=ti)
            e, en = np.abs(u - ref).max() / ref.max(), np.abs(un - ref).max() / ref.max()
            assert e < en / 4
            if k == 1.0:
                errs.append(e)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 3e-3


def test_coulomb_gaussian_converges_and_ss_helps():
    """V_H of rho = (a/pi)^{3/2} e^{-a r^2} is erf(sqrt(a) r)/r."""
    errs = []
    for nc in (8, 12, 16):
        m = W.uniform_mesh(-10, 10, nc, 4)
        ti, r = _central(m)
        rho = math.pi**-1.5 * np.exp(-r * r)
        ref = erf(r[ti]) / r[ti]
        v = oracle.direct_coulomb(m.xyz, m.w, rho, 1.0, ss=True, targets=ti)
        vn = oracle.direct_coulomb(m.xyz, m.w, rho, 1.0, ss=False, targets=ti)
        e, en = np.abs(v - ref).max() / ref.max(), np.abs(vn - ref).max() / ref.max()
        assert e < en / 5
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3


def test_hydrogen_fixed_point_trend():
    """psi = e^{-r}/sqrt(pi), V = -1/r, k = 1: -2 G_1[V psi] = psi in the
    continuum; the discrete sum approaches it as the uniform mesh refines."""
    errs = []
    for nc in (8, 16, 24):
        wl = W.hydrogen_1s(seed=0, ncell=nc)
        R = np.array(wl.meta["nucleus"])
        r = np.sqrt(((wl.mesh.xyz.T - R) ** 2).sum(1))
        ti = np.nonzero(r < 3.0)[0]
        ti = ti[:: max(1, len(ti) // 300)]
        u = oracle.direct_yukawa(wl.mesh.xyz, wl.mesh.w, wl.f[0], 1.0, targets=ti)
        psi = wl.psi[0, ti]
        errs.append(np.linalg.norm(-2 * u - psi) / np.linalg.norm(psi))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-2


def test_constant_source_gives_ss_constant():
    """With f = c the subtracted sum vanishes: u = c / k^2 exactly."""
    xyz, w = W.random_cube(500, seed=3)
    for k in (0.7, 3.0):
        u = oracle.direct_yukawa(xyz, w, np.full(500, 2.5), k)
        np.testing.assert_allclose(u, 2.5 / k**2, rtol=1e-15)


def test_reciprocity_without_ss():
    """The kernel matrix is symmetric: <g w, K (f w)> = <f w, K (g w)>."""
    xyz, w = W.random_cube(700, seed=4)
    rng = np.random.default_rng(0)
    f, g = rng.normal(size=700), rng.normal(size=700)
    for kern in ("y", "c"):
        if kern == "y":
            uf = oracle.direct_yukawa(xyz, w, f, 1.3, ss=False)
            ug = oracle.direct_yukawa(xyz, w, g, 1.3, ss=False)
        else:
            uf = oracle.direct_coulomb(xyz, w, f, ss=False)
            ug = oracle.direct_coulomb(xyz, w, g, ss=False)
        a, b = np.sum(g * w * uf), np.sum(f * w * ug)
        assert abs(a - b) < 1e-12 * (abs(a) + abs(b))


def test_two_point_values():
    """Two points at distance 2, w = (1, 3), f = (1, 5): each sum has a
    single term, written out from the kernel definitions."""
    xyz = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    w = np.array([1.0, 3.0])
    f = np.array([1.0, 5.0])
    k = 0.5
    g = math.exp(-1.0) / (8 * math.pi)
    u = oracle.direct_yukawa(xyz, w, f, k, ss=True)
    np.testing.assert_allclose(u, [g * 4 * 3 + 1 / 0.25, g * (-4) * 1 + 5 / 0.25], rtol=1e-15)
    v = oracle.direct_coulomb(xyz, w, f, alpha=2.0, ss=True)
    e = math.exp(-1.0)
    np.testing.assert_allclose(v, [(5 - e) * 3 / 2 + 8 * math.pi, (1 - 5 * e) / 2 + 40 * math.pi],
                               rtol=1e-15)


def test_translation_and_scaling():
    """Shifting every point leaves u unchanged; scaling x -> s x with k -> k/s
    and w -> s^3 w scales the no-SS Yukawa sum by s^2 and Coulomb by s^2."""
    xyz, w = W.random_cube(400, seed=5)
    f = np.random.default_rng(1).normal(size=400)
    u0 = oracle.direct_yukawa(xyz, w, f, 1.1)
    u1 = oracle.direct_yukawa(xyz + np.array([[3.0], [-7.0], [0.5]]), w, f, 1.1)
    np.testing.assert_allclose(u1, u0, rtol=1e-10, atol=1e-13)
    s = 2.0
    us = oracle.direct_yukawa(s * xyz, s**3 * w, f, 1.1 / s, ss=False)
    np.testing.assert_allclose(us, s**2 * oracle.direct_yukawa(xyz, w, f, 1.1, ss=False), rtol=1e-12)
    vs = oracle.direct_coulomb(s * xyz, s**3 * w, f, ss=False)
    np.testing.assert_allclose(vs, s**2 * oracle.direct_coulomb(xyz, w, f, ss=False), rtol=1e-12)

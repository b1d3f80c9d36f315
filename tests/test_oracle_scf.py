"""Pins of the oracle's SCF step (Algorithm 1; Eq. Fermi, density-construction,
total-energy-gradient-free; LDA of Section 2).

- Fermi level: the two-level case solved in closed form (a quadratic in
  e^{mu/kT}), integer filling as kT -> 0, a degenerate pair sharing an
  electron, and the electron count for random levels.
- LDA: the oracle's exchange-correlation (r_s form) against the input
  generator's independent implementation (rho^(1/3) form); the correlation
  potential is the density derivative of rho eps_c; the exchange energy of a
  Gaussian density against its closed form on an adaptive mesh.
- Hartree energy term of the SCF potentials against the Gaussian closed form.
- One SCF step of the hydrogen atom: the density integrates to N_e, a lone
  orbital holding one electron has mu = eps and f = 1/2, the first density
  mixing step is simple mixing, and the energy is assembled as printed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2003_01833_gb300 import workloads as W


def test_fermi_two_levels_closed_form():
    e1, e2, kT, ne = -1.0, -0.3, 0.05, 3.0
    s = ne / 2
    r = math.exp((e2 - e1) / kT)
    # with u = e^{(mu - e2)/kT}: (2 - s) r u^2 + (1 - s)(r + 1) u - s = 0
    a, b, c = (2 - s) * r, (1 - s) * (r + 1), -s
    u = (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)
    mu_ref = e2 + kT * math.log(u)
    mu, f = oracle.fermi_level([e1, e2], ne, kT)
    assert abs(mu - mu_ref) < 1e-12
    np.testing.assert_allclose(2 * f.sum(), ne, rtol=1e-14)


def test_fermi_filling_and_degeneracy():
    mu, f = oracle.fermi_level([-3.0, -2.0, -1.0, -0.5], 4.0, 1e-6)
    np.testing.assert_allclose(f, [1, 1, 0, 0], atol=1e-12)
    assert -2.0 < mu < -1.0
    mu, f = oracle.fermi_level([-1.0, -0.5, -0.5], 4.0, 6.3336e-4)
    np.testing.assert_allclose(f, [1.0, 0.5, 0.5], atol=1e-12)
    assert abs(mu + 0.5) < 1e-12
    # N_e = 2 N_w fills every state exactly (a closed-shell molecule with
    # one orbital per electron pair, e.g. H2 with its sigma_g alone)
    mu, f = oracle.fermi_level([-0.6], 2.0, 6.3336e-4)
    assert f[0] == 1.0 and mu > -0.6
    mu, f = oracle.fermi_level([-1.0, -0.4], 4.0, 1e-3)
    np.testing.assert_allclose(f, 1.0, rtol=0, atol=1e-15)
    assert abs(2.0 * f.sum() - 4.0) < 1e-15
    for bad in (2.5, 0.0):
        with pytest.raises(ValueError):
            oracle.fermi_level([-1.0], bad, 1e-3)


def test_fermi_counts_electrons():
    rng = np.random.default_rng(5)
    for _ in range(5):
        eps = np.sort(rng.uniform(-5, 0, size=9))
        ne = float(rng.integers(1, 17))
        mu, f = oracle.fermi_level(eps, ne, 0.01)
        assert abs(2 * f.sum() - ne) < 1e-10
        assert np.all(np.diff(f) <= 0)


def test_tol_gi_schedule():
    t = [oracle.tol_gi_schedule(s) for s in range(7)]
    assert t[0] == 3e-3 and t[4] == 1e-5 and t[6] == 1e-5
    r = [t[i + 1] / t[i] for i in range(4)]
    np.testing.assert_allclose(r, r[0], rtol=1e-12)


def test_lda_independent_forms_agree_and_potential_is_derivative():
    rs = np.geomspace(0.05, 40.0, 50)
    rho = 3.0 / (4.0 * np.pi * rs**3)
    e1, v1 = oracle.lda_xc(rho)
    e2, v2 = W.lda_xc(rho)
    np.testing.assert_allclose(e1, e2, rtol=1e-13)
    np.testing.assert_allclose(v1, v2, rtol=1e-13)
    h = 1e-6 * rho
    ec, vc = oracle.lda_correlation(rho)
    num = ((rho + h) * oracle.lda_correlation(rho + h)[0] - (rho - h) * oracle.lda_correlation(rho - h)[0]) / (2 * h)
    np.testing.assert_allclose(vc, num, rtol=1e-7, atol=1e-12)


@pytest.fixture(scope="module")
def hmesh():
    wl = W.hydrogen_adaptive()
    return wl, oracle.Tree(wl.mesh.xyz, 2000)


def test_gaussian_exchange_and_hartree_energies(hmesh):
    wl, T = hmesh
    w = wl.mesh.w
    r2 = np.sum(wl.mesh.xyz**2, axis=0)
    a, N = 1.0, 2.0
    rho = N * (a / np.pi) ** 1.5 * np.exp(-a * r2)
    ex, _ = oracle.lda_exchange(rho)
    ex_ref = -(3.0 / 4.0) * (3.0 / np.pi) ** (1 / 3) * N ** (4 / 3) * (a / np.pi) ** 2 * (3 * np.pi / (4 * a)) ** 1.5
    assert abs(np.sum(ex * rho * w) - ex_ref) < 1e-5 * abs(ex_ref)
    pot = oracle.scf_potentials(T, 0.7, 6, w, np.zeros_like(rho), rho)
    eh_ref = N * N * math.sqrt(a / (2 * np.pi))
    assert abs(pot["e_h"] - eh_ref) < 1e-4 * eh_ref
    np.testing.assert_allclose(pot["veff"], pot["vh"] + pot["vxc"], rtol=0, atol=0)


def test_one_scf_step_of_hydrogen(hmesh):
    wl, T = hmesh
    w = wl.mesh.w
    r = np.sqrt(np.sum(wl.mesh.xyz**2, axis=0))
    psi = np.exp(-r)
    psi /= np.sqrt(np.sum(psi * psi * w))
    rho_in = psi * psi
    mix = {}
    out = oracle.scf_step(T, 0.7, 6, w, -1.0 / r, rho_in, psi[None], np.array([-0.25]), -0.5, 1.0, 6.3336e-4, 0.0,
                          tol_gi=1e-4, max_iter=30, mix=mix)
    assert out["gi"]["iters"][0] > 0
    assert abs(np.sum(out["rho_out"] * w) - 1.0) < 1e-12
    assert abs(out["mu"] - out["eps"][0]) < 1e-9 and abs(out["occ"][0] - 0.5) < 1e-9
    np.testing.assert_allclose(out["rho_next"], rho_in + 0.5 * (out["rho_out"] - rho_in), rtol=1e-15, atol=1e-300)
    E = out["energy"]
    assert E["total"] == E["band"] - E["hartree"] + E["xc"] - E["vxc"] + E["zz"]
    assert -0.35 < out["eps"][0] < -0.15
    assert len(mix["x"]) == 1

"""SCF iteration on the device (tagi_scf_*: Algorithm 1 with Green Iteration,
LDA, Fermi-Dirac occupations, Anderson density mixing and the gradient-free
energy) against the oracle, and a converged lithium calculation against the
energy the paper prints.

- Float64, hydrogen atom on the adaptive mesh: two SCF steps (the second
  mixes two densities) agree with the oracle's scf_step to rounding order
  (eigenvalues and energies 1e-10 Ha, densities 1e-9 of their maximum).
- FP32C, CO on the 638,500-point mesh: likewise within 3 mHa of the
  reference implied by Table timings (E_ref = -112.471930 Ha).
- FP32C, the 309,000-point Li workload: SCF from the seeded superposition
  density to ||rho_out - rho_in||_w < 1e-4 gives the LDA ground-state energy
  of Li within 3 mHa of E_ref = -7.334510 Ha (measured: 1.0 mHa, in 8 SCF
  steps; eigenvalues -1.8776 and -0.1058 Ha).  E_ref follows from the
  paper's Table timings (E_TAGI = -7.334051 Ha with error 4.59e-4 Ha/atom
  against its DFT-FE reference); the paper's own run on 232,000 points was
  0.46 mHa from it.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2003_01833_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KT_200K = 200.0 * 3.166811563e-6  # k_B T at 200 K in Ha (Section 6)


def _e_ref_li():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_timings_li.txt")
    vals = dict(l.split()[:2] for l in open(path) if l.strip() and not l.startswith("#"))
    return float(vals["E_TAGI"]) - float(vals["error_per_atom"])


E_REF_LI = _e_ref_li()


def _e_ref_co():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_timings_co.txt")
    vals = dict(l.split()[:2] for l in open(path) if l.strip() and not l.startswith("#"))
    return float(vals["E_TAGI"]) - float(vals["atoms"]) * float(vals["error_per_atom"])


E_REF_CO = _e_ref_co()


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


def test_two_scf_steps_match_oracle(T):
    wl = W.hydrogen_adaptive()
    w = wl.mesh.w
    r = np.sqrt(np.sum(wl.mesh.xyz**2, axis=0))
    vext = -1.0 / r
    psi0 = np.exp(-r)
    psi0 = (psi0 / np.sqrt(np.sum(psi0 * psi0 * w)))[None]
    rho0 = psi0[0] ** 2
    eps0 = np.array([-0.25])
    otree = oracle.Tree(wl.mesh.xyz, 2000)
    # a Green Iteration tolerance for step 0 far from every residual
    pot = oracle.scf_potentials(otree, 0.7, 6, w, vext, rho0)
    tr = oracle.green_iterate(otree, 0.7, 6, w, pot["veff"], -0.5, psi0, eps0, tol_gi=0.0, max_iter=10,
                              mix_tol=np.inf)["trace"][:, 0]
    k = next(k for k in range(3, 9) if tr[k] < 0.7 * tr[:k].min())
    tol0 = float(np.sqrt(tr[:k].min() * tr[k]))
    kw = dict(n_elec=1.0, kT=KT_200K, e_zz=0.0, max_iter=12)
    mix = {}
    o0 = oracle.scf_step(otree, 0.7, 6, w, vext, rho0, psi0, eps0, -0.5, tol_gi=tol0, mix=mix, **kw)
    o1 = oracle.scf_step(otree, 0.7, 6, w, vext, o0["rho_next"], o0["psi"], o0["eps"], -0.5, tol_gi=1e-12, mix=mix,
                         **kw)
    assert o0["gi"]["iters"][0] == k + 1 and o1["gi"]["iters"][0] == -1

    with T.Tree(dev(wl.mesh.xyz), dev(w), theta=0.7, degree=6, leaf_size=2000, prec=T.TAGI_FP64) as tr_, \
            T.Scf(tr_.handle, 1.0, kT=KT_200K, tol_gi_first=tol0, tol_gi_final=1e-12, tol_gi_ramp=1,
                  gi_max_iter=12) as scf:
        rho = dev(rho0)
        psi = dev(psi0)
        rho_out = torch.empty_like(rho)
        vx = dev(vext)
        g0 = scf.step(vx, -0.5, rho, psi, eps0, rho_out=rho_out)
        ro0, rn0 = rho_out.cpu().numpy(), rho.cpu().numpy()
        g1 = scf.step(vx, -0.5, rho, psi, g0["eps"], rho_out=rho_out)
        ro1, rn1, ps1 = rho_out.cpu().numpy(), rho.cpu().numpy(), psi.cpu().numpy()
    for g, o, ro, rn in ((g0, o0, ro0, rn0), (g1, o1, ro1, rn1)):
        assert abs(g["eps"][0] - o["eps"][0]) < 1e-10
        assert abs(g["mu"] - o["mu"]) < 1e-10 and abs(g["occ"][0] - o["occ"][0]) < 1e-12
        for key, gk in (("band", "e_band"), ("hartree", "e_hartree"), ("xc", "e_xc"), ("vxc", "e_vxc"),
                        ("total", "e_total")):
            assert abs(g[gk] - o["energy"][key]) < 1e-10, key
        assert np.abs(ro - o["rho_out"]).max() < 1e-9 * np.abs(o["rho_out"]).max()
        assert np.abs(rn - o["rho_next"]).max() < 1e-9 * np.abs(o["rho_next"]).max()
        assert abs(g["residual"] - o["resid"]) < 1e-8 * o["resid"]
        assert g["gi"]["steps"] == o["gi"]["steps"]
    assert g0["tol_gi"] == tol0 and g1["tol_gi"] == 1e-12 and g1["step"] == 1
    assert np.abs(ps1 - o1["psi"]).max() < 1e-9 * np.abs(o1["psi"]).max()
    assert abs(np.sum(ro0 * w) - 1.0) < 1e-12


def test_lithium_scf_reaches_the_papers_energy(T):
    wl = W.lithium()
    m = wl.mesh
    with T.Tree(dev(m.xyz), dev(m.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=T.TAGI_FP32C) as tr, T.Scf(tr.handle, wl.n_elec, kT=KT_200K, e_zz=wl.e_zz) as scf:
        rho, psi, vx = dev(wl.rho), dev(wl.psi), dev(wl.vext)
        eps = wl.eps
        hist = []
        for _ in range(30):
            rep = scf.step(vx, wl.vshift, rho, psi, eps)
            eps = rep["eps"]
            hist.append((rep["residual"], rep["e_total"], rep["tol_gi"], rep["gi"]["steps"]))
            if rep["residual"] < 1e-4:
                break
    print("Li SCF (residual, E, tol_gi, GI steps):", hist)
    assert hist[-1][0] < 1e-4
    assert abs(hist[-1][1] - E_REF_LI) < 3e-3
    # 1s^2 2s^1: the 2s holds one electron, so mu sits on it
    assert abs(rep["occ"][0] - 1.0) < 1e-9 and abs(rep["occ"][1] - 0.5) < 1e-6
    assert eps[0] < eps[1] < 0


def test_carbon_monoxide_scf_reaches_the_papers_energy(T):
    """CO on the 638,500-point mesh (tol_m = 3e-7, the paper's tolerance),
    8 orbitals from an aufbau start, FP32C, SCF to ||rho_out - rho_in||_w <
    1e-4: the all-electron LDA energy within 3 mHa of the reference implied
    by Table timings (E_ref = -112.471930 Ha; measured 0.60 mHa, 0.30 mHa per
    atom, in 8 SCF steps; the paper's own run was 0.72 mHa per atom off).
    The 2pi* level stays empty and the seven below it fully occupied.  The
    1pi pair (levels 5 and 6) is degenerate by symmetry: its two computed
    eigenvalues agree to the FP32C eigenvalue accuracy (about 1e-6 Ha per
    level), in either order, and the levels ascend up to that accuracy."""
    wl = W.carbon_monoxide_scf()
    m = wl.mesh
    with T.Tree(dev(m.xyz), dev(m.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=T.TAGI_FP32C) as tr, T.Scf(tr.handle, wl.n_elec, kT=KT_200K, e_zz=wl.e_zz) as scf:
        rho, psi, vx = dev(wl.rho), dev(wl.psi), dev(wl.vext)
        eps = wl.eps
        hist = []
        for _ in range(25):
            rep = scf.step(vx, wl.vshift, rho, psi, eps)
            eps = rep["eps"]
            hist.append((rep["residual"], rep["e_total"], rep["gi"]["steps"]))
            if rep["residual"] < 1e-4:
                break
    print("CO SCF (residual, E, GI steps):", hist, "eps", eps)
    assert hist[-1][0] < 1e-4
    assert abs(hist[-1][1] - E_REF_CO) < 3e-3
    np.testing.assert_allclose(rep["occ"][:7], 1.0, atol=1e-9)
    assert rep["occ"][7] < 1e-9
    assert abs(eps[4] - eps[5]) < 5e-6
    assert np.all(np.diff(eps) >= -5e-6) and eps[-1] < 0


def test_lithium_scf_with_stored_outputs_reaches_the_papers_energy_closer(T):
    """The same Li SCF with gi_store_output: a converged orbital keeps its
    Green step's output, so every SCF iteration follows V_eff[rho_in] (with
    Algorithm 2's stored input an orbital that one step moves by less than
    tol_gi is not updated, and the density residual then falls by mixing
    alone).  Measured: 0.29 mHa from E_ref in 6 SCF steps, against 1.0 mHa
    in 8 with the stored input; the bound here is 1 mHa."""
    wl = W.lithium()
    m = wl.mesh
    with T.Tree(dev(m.xyz), dev(m.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=T.TAGI_FP32C) as tr, T.Scf(tr.handle, wl.n_elec, kT=KT_200K, e_zz=wl.e_zz,
                                                gi_store_output=True) as scf:
        rho, psi, vx = dev(wl.rho), dev(wl.psi), dev(wl.vext)
        eps = wl.eps
        hist = []
        for _ in range(30):
            rep = scf.step(vx, wl.vshift, rho, psi, eps)
            eps = rep["eps"]
            hist.append((rep["residual"], rep["e_total"], rep["gi"]["steps"]))
            if rep["residual"] < 1e-4:
                break
    print("Li SCF, stored outputs (residual, E, GI steps):", hist)
    assert hist[-1][0] < 1e-4
    assert abs(hist[-1][1] - E_REF_LI) < 1e-3
    assert eps[0] < eps[1] < 0


def test_benzene_scf_step_full_size(T):
    """One SCF step of C6H6 on the 4.6M-point mesh (tol_m = 3e-8), 21
    orbitals from the aufbau start, FP32C, the Green Iteration capped at 2
    steps.  Checked against the oracle and the definitions:
    - occupations: every level filled (N_e = 2 N_w), as oracle.fermi_level
      gives for the returned eigenvalues;
    - rho_out = 2 sum_i f_i psi_i^2 from the returned orbitals, at every
      point of two sampled target batches, and sum rho_out w = N_e;
    - the next input density is simple mixing on the first step;
    - E_xc and <V_xc, rho_in> against the oracle's LDA over all points;
    - V_H[rho_in] (the SCF's Hartree sum, the same call on the same tree)
      against the oracle treecode on the two sampled batches, and E_H of the
      report as 1/2 sum V_H rho_in w."""
    wl = W.benzene_scf()
    m = wl.mesh
    n, nw = wl.n, wl.psi.shape[0]
    assert 4.4e6 < n < 5.2e6 and nw == 21 and wl.n_elec == 42.0
    with T.Tree(dev(m.xyz), dev(m.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=T.TAGI_FP32C) as tr:
        vh = torch.empty(n, dtype=torch.float64, device="cuda")
        T.tagi_fields_conv(tr.handle, None, [], None, rho=dev(wl.rho), vh=vh)
        vh = vh.cpu().numpy()
        with T.Scf(tr.handle, wl.n_elec, kT=KT_200K, e_zz=wl.e_zz, gi_max_iter=2, gi_store_output=True) as scf:
            rho, psi, vx = dev(wl.rho), dev(wl.psi), dev(wl.vext)
            ro = torch.empty(n, dtype=torch.float64, device="cuda")
            rep = scf.step(vx, wl.vshift, rho, psi, wl.eps, rho_out=ro)
        rho_next, psi, ro = rho.cpu().numpy(), psi.cpu().numpy(), ro.cpu().numpy()
    w = m.w
    assert rep["gi"]["steps"] == 2 and rep["step"] == 0
    mu, f = oracle.fermi_level(rep["eps"], wl.n_elec, KT_200K)
    np.testing.assert_allclose(rep["occ"], f, rtol=0, atol=1e-12)
    np.testing.assert_allclose(rep["occ"], 1.0, atol=1e-12)
    ot = oracle.Tree(m.xyz, wl.leaf_size)
    pick = np.random.default_rng(9).choice(ot.leaves, size=2, replace=False)
    pts = np.concatenate([ot.points(c) for c in pick])
    ref = 2.0 * np.sum(f[:, None] * psi[:, pts] ** 2, axis=0)
    np.testing.assert_allclose(ro[pts], ref, rtol=1e-12, atol=1e-300)
    assert abs(np.sum(ro * w) - wl.n_elec) < 1e-8 * wl.n_elec
    np.testing.assert_allclose(rho_next, wl.rho + 0.5 * (ro - wl.rho), rtol=1e-14, atol=1e-300)
    exc, vxc = oracle.lda_xc(wl.rho)
    assert abs(rep["e_xc"] - np.sum(exc * wl.rho * w)) < 1e-10 * abs(rep["e_xc"])
    assert abs(rep["e_vxc"] - np.sum(vxc * wl.rho * w)) < 1e-10 * abs(rep["e_vxc"])
    vref = ot.treecode_batches(wl.theta, wl.degree, 1, wl.alpha, wl.rho, w, pick)
    assert np.linalg.norm(vh[pts] - vref[pts]) < 1e-6 * np.linalg.norm(vref[pts])
    assert abs(rep["e_hartree"] - 0.5 * np.sum(vh * wl.rho * w)) < 1e-12 * rep["e_hartree"]
    print("C6H6 SCF step:", {k: rep[k] for k in ("e_total", "e_band", "e_hartree", "e_xc", "residual")},
          "eps", rep["eps"])

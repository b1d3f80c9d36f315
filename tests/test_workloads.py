"""Input generators: Fejer rule and meshes (Section 3.2)."""
import math
import os

import numpy as np
import pytest

from paper_2003_01833_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 8])
def test_fejer_exact_to_degree_p(p):
    """The p+1 point Fejer rule integrates degree <= p exactly (Section 3.2)."""
    x = W.chebyshev1_nodes(p)
    w = W.fejer_weights(p)
    for m in range(p + 1):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * x**m) - exact) < 1e-14
    assert np.all(w > 0)


def test_fejer_golden_three_points():
    d = np.loadtxt(os.path.join(GOLD, "fejer3.txt"))
    np.testing.assert_allclose(W.chebyshev1_nodes(2), d[:, 0], atol=1e-15)
    np.testing.assert_allclose(W.fejer_weights(2), d[:, 1], atol=1e-15)


def test_chebyshev_nodes_inside_cell():
    """First-kind points never reach the cell vertices (Section 3.2)."""
    for p in range(1, 9):
        x = W.chebyshev1_nodes(p)
        assert np.all(np.abs(x) < 1.0)


def test_uniform_mesh_volume_and_size():
    m = W.uniform_mesh(-10, 10, 8, 3)
    assert m.n == 32768 and m.xyz.shape == (3, 32768)
    assert abs(m.w.sum() - 20.0**3) < 1e-9
    # integrates a cubic polynomial exactly
    x, y, z = m.xyz
    assert abs(np.sum(m.w * x * x * y * y) - (2 * 10**3 / 3) ** 2 * 20) < 1e-6


def test_hydrogen_nucleus_on_vertex():
    wl = W.hydrogen_1s(seed=5)
    R = np.array(wl.meta["nucleus"])
    assert np.all(np.abs(R) <= 2.5 + 1e-12)
    assert np.all(np.abs(R / 2.5 - np.round(R / 2.5)) < 1e-12)
    r = np.sqrt(((wl.mesh.xyz.T - R) ** 2).sum(1))
    assert r.min() > 0.05


def test_adaptive_mesh_li_small():
    wl = W.lithium(seed=1, tol_m=1e-3)
    m = wl.mesh
    assert abs(m.w.sum() - 40.0**3) < 1e-6
    vol = np.prod(m.cells_hi - m.cells_lo, axis=1)
    assert abs(vol.sum() - 40.0**3) < 1e-6
    # refined toward the nucleus: the smallest cells lie next to it
    small = np.argmin(vol)
    cen = 0.5 * (m.cells_lo[small] + m.cells_hi[small])
    assert np.linalg.norm(cen) < 1.0 and vol[small] < 1e-2
    # the nucleus is a vertex of every cell that contains it
    inside = np.all((m.cells_lo <= 0) & (m.cells_hi >= 0), axis=1)
    corners = np.all((m.cells_lo == 0) | (m.cells_hi == 0), axis=1)
    assert np.all(corners[inside])
    assert wl.psi.shape == (2, m.n) and np.all(wl.k > 0)


def test_split_at_atoms_puts_atom_on_vertex():
    lo = np.array([[0.0, 0.0, 0.0]])
    hi = np.array([[1.0, 1.0, 1.0]])
    a = np.array([[0.3, 0.5, 1.0]])
    lo2, hi2 = W._split_at_atoms(lo, hi, a)
    assert len(lo2) == 4
    lo3, hi3 = W._fix_aspect(lo2, hi2)
    ext = hi3 - lo3
    assert np.all(ext.max(1) / ext.min(1) <= 2.0)
    assert abs(np.prod(ext, axis=1).sum() - 1.0) < 1e-14


def test_radial_hartree_table_gauss_law():
    """Far from the atom the Hartree potential is N_e / r."""
    r = np.array([60.0])
    assert abs(W.atomic_hartree("Li", r)[0] - 3.0 / 60.0) < 1e-6


def test_lda_exchange_in_rs_form():
    """eps_x = -(3/(4 pi)) (9 pi/4)^(1/3) / r_s = -0.4581652932831429 / r_s Ha,
    the textbook r_s form, against the rho^(1/3) form the module evaluates."""
    for rs in (0.3, 1.0, 2.5, 7.0):
        rho = 3.0 / (4.0 * math.pi * rs**3)
        ex_rs = -0.4581652932831429 / rs
        # correlation is small; isolate exchange by its 4/3 ratio to v_x
        e, v = W.lda_xc(np.array([rho]))
        g, b1, b2 = W.PZ81_LOW_DENSITY
        A, B, C, D = W.PZ81_HIGH_DENSITY
        if rs >= 1:
            ec = g / (1 + b1 * math.sqrt(rs) + b2 * rs)
        else:
            ec = A * math.log(rs) + B + C * rs * math.log(rs) + D * rs
        assert abs((e[0] - ec) - ex_rs) < 1e-13 * abs(ex_rs)


def test_lda_potential_is_the_density_derivative():
    """v_xc = d(rho eps_xc)/d rho, by central differences on both branches
    of the correlation fit (r_s from 0.1 to 20)."""
    rs = np.array([0.1, 0.4, 0.9, 1.2, 3.0, 8.0, 20.0])
    rho = 3.0 / (4.0 * np.pi * rs**3)
    e, v = W.lda_xc(rho)
    h = 1e-6 * rho
    ep, _ = W.lda_xc(rho + h)
    em, _ = W.lda_xc(rho - h)
    dnum = ((rho + h) * ep - (rho - h) * em) / (2 * h)
    np.testing.assert_allclose(v, dnum, rtol=1e-7)
    # the two correlation branches meet at r_s = 1 to the fit's 4e-5 Ha
    lo, _ = W.lda_xc(np.array([3.0 / (4.0 * np.pi) * (1 - 1e-12)]))
    hi, _ = W.lda_xc(np.array([3.0 / (4.0 * np.pi) * (1 + 1e-12)]))
    assert abs(lo[0] - hi[0]) < 5e-5
    # zero density gives zero
    e0, v0 = W.lda_xc(np.zeros(2))
    assert np.all(e0 == 0) and np.all(v0 == 0)


def test_ring_combinations_are_the_real_fourier_modes_of_the_ring():
    """Six functions at angles theta_0 + j pi/3: the combinations' weights
    are the rows of the real discrete Fourier transform of the ring, which
    are orthogonal with squared norms 6, 3, 3, 3, 3, 6."""
    import numpy as np

    from paper_2003_01833_gb300 import workloads as W

    ang = 0.3 + np.arange(6) * np.pi / 3
    rows = np.array(W.ring_combinations(list(np.eye(6)), ang))
    np.testing.assert_allclose(rows @ rows.T, np.diag([6.0, 3, 3, 3, 3, 6]), atol=1e-12)
    np.testing.assert_allclose(rows[0], 1.0)
    np.testing.assert_allclose(rows[5], [1, -1, 1, -1, 1, -1], atol=1e-12)

"""Seeded synthetic inputs for the TAGI convolution sums.

This module builds the meshes, quadrature weights and fields that both the CUDA
path and the oracle consume.  It holds none of the convolution arithmetic: only
the discretisation of Section 3 (Chebyshev points of the first kind, Eq.
Chebyshev_points; the Fejer rule; the adaptive refinement of Eq.
refinement_criterion with the test function of Eq. test_function) and Slater-type
stand-ins for the radial atomic data of Section 3.1, which is not available.

Layout of every mesh: ``xyz`` is a float64 array of shape (3, N) (structure of
arrays), ``w`` float64 (N,).  Fields are float64 arrays of shape (nf, N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Quadrature (Section 3.2)
# --------------------------------------------------------------------------


def chebyshev1_nodes(p: int) -> np.ndarray:
    """Chebyshev points of the first kind on [-1, 1], Eq. Chebyshev_points:
    x_i = cos((2i+1) pi / (2p+2)), i = 0..p."""
    i = np.arange(p + 1)
    return np.cos((2 * i + 1) * np.pi / (2 * p + 2))


def fejer_weights(p: int) -> np.ndarray:
    """Weights of Fejer's first rule on the p+1 first-kind Chebyshev points.

    The paper cites the rule (Section 3.2) without printing it.  This is the
    classical closed form: with N = p+1 points at angles t_i,
    w_i = (2/N) [1 - 2 sum_{j=1}^{floor(N/2)} cos(2 j t_i) / (4 j^2 - 1)].
    The rule integrates polynomials of degree <= p exactly on [-1, 1].
    """
    n = p + 1
    t = (2 * np.arange(n) + 1) * np.pi / (2 * n)
    s = np.zeros(n)
    for j in range(1, n // 2 + 1):
        s += np.cos(2 * j * t) / (4 * j * j - 1)
    return (2.0 / n) * (1.0 - 2.0 * s)


def cell_points(lo: np.ndarray, hi: np.ndarray, p: int):
    """Tensor-product Fejer points and weights for M cuboid cells.

    lo, hi: (M, 3).  Returns pts (M, (p+1)^3, 3) and wts (M, (p+1)^3).
    Point order inside a cell: x slowest, z fastest.
    """
    x1 = chebyshev1_nodes(p)
    w1 = fejer_weights(p)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    X, Y, Z = np.meshgrid(x1, x1, x1, indexing="ij")
    WX, WY, WZ = np.meshgrid(w1, w1, w1, indexing="ij")
    ref = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)  # (P, 3)
    wref = (WX * WY * WZ).ravel()  # (P,)
    pts = c[:, None, :] + h[:, None, :] * ref[None, :, :]
    wts = np.prod(h, axis=1)[:, None] * wref[None, :]
    return pts, wts


@dataclass
class Mesh:
    xyz: np.ndarray  # (3, N) float64
    w: np.ndarray  # (N,) float64
    cells_lo: np.ndarray  # (Nc, 3)
    cells_hi: np.ndarray  # (Nc, 3)
    p: int

    @property
    def n(self) -> int:
        return self.w.shape[0]


def mesh_from_cells(lo: np.ndarray, hi: np.ndarray, p: int) -> Mesh:
    pts, wts = cell_points(lo, hi, p)
    xyz = np.ascontiguousarray(pts.reshape(-1, 3).T)
    return Mesh(xyz=xyz, w=np.ascontiguousarray(wts.ravel()), cells_lo=lo, cells_hi=hi, p=p)


def uniform_mesh(lo: float, hi: float, ncell: int, p: int) -> Mesh:
    """ncell^3 cubic cells on [lo, hi]^3 with (p+1)^3 Fejer points each."""
    e = np.linspace(lo, hi, ncell + 1)
    I, J, K = np.meshgrid(np.arange(ncell), np.arange(ncell), np.arange(ncell), indexing="ij")
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    clo = e[idx]
    chi = e[idx + 1]
    return mesh_from_cells(clo, chi, p)


# --------------------------------------------------------------------------
# Slater-type atomic stand-ins (Section 3.1 uses radial Kohn-Sham data that is
# not available; hydrogenic Slater functions replace it)
# --------------------------------------------------------------------------

# shells: (n, l, occupation, exponent zeta); radial part r^(n-1) e^{-zeta r} for
# n=1 and the hydrogenic 2s form (2 - zeta r) e^{-zeta r/2}-like shapes below.
ATOM_Z = {"H": 1, "Li": 3, "C": 6, "O": 8}


def _shells(sym: str):
    """Occupied shells of the neutral atom: list of (kind, occ, Z).

    kind is '1s', '2s' or '2p'; the radial shapes are hydrogenic (1s ~ e^{-Zr},
    2s ~ (2 - Zr) e^{-Zr/2}, 2p ~ r e^{-Zr/2}) with the bare nuclear charge for
    H and Li (the stand-in the Li workload specifies) and Slater-screened
    effective charges for C and O.
    """
    Z = ATOM_Z[sym]
    if sym == "H":
        return [("1s", 1.0, Z)]
    if sym == "Li":
        return [("1s", 2.0, Z), ("2s", 1.0, Z)]
    # C and O: effective charges from Slater's screening rules (1s: Z - 0.30;
    # n = 2: Z - 0.35 per other n = 2 electron - 0.85 per 1s electron).  With
    # bare charges their stand-in density is so compact that the initial
    # Hartree potential screens the nuclei almost completely and binds no
    # valence level.
    if sym == "C":
        return [("1s", 2.0, 5.70), ("2s", 2.0, 3.25), ("2p", 2.0, 3.25)]
    if sym == "O":
        return [("1s", 2.0, 7.70), ("2s", 2.0, 4.55), ("2p", 4.0, 4.55)]
    raise ValueError(sym)


def radial_orbital(kind: str, Z: float, r: np.ndarray) -> np.ndarray:
    """Normalised hydrogenic radial-times-angular-average orbital value."""
    if kind == "1s":
        return math.sqrt(Z**3 / math.pi) * np.exp(-Z * r)
    if kind == "2s":
        return math.sqrt(Z**3 / (32 * math.pi)) * (2.0 - Z * r) * np.exp(-0.5 * Z * r)
    if kind == "2p":  # spherical average of |2p|^2 gives this amplitude
        return math.sqrt(Z**5 / (96 * math.pi)) * r * np.exp(-0.5 * Z * r)
    raise ValueError(kind)


def atomic_density(sym: str, r: np.ndarray) -> np.ndarray:
    rho = np.zeros_like(r)
    for kind, occ, Z in _shells(sym):
        rho += occ * radial_orbital(kind, Z, r) ** 2
    return rho


def _radial_hartree_table(sym: str, rmax: float = 80.0, m: int = 200001):
    """Radial Hartree potential of the spherical atomic density on a fine
    grid (Gauss's law: V(r) = Q(r)/r + 4 pi int_r^inf rho s ds)."""
    s = np.linspace(0.0, rmax, m)
    rho = atomic_density(sym, s)
    f_in = 4 * np.pi * rho * s * s
    f_out = 4 * np.pi * rho * s
    ds = s[1] - s[0]
    q = np.concatenate([[0.0], np.cumsum(0.5 * (f_in[1:] + f_in[:-1]) * ds)])
    o = np.concatenate([[0.0], np.cumsum(0.5 * (f_out[1:] + f_out[:-1]) * ds)])
    out = o[-1] - o
    v = np.empty_like(s)
    v[1:] = q[1:] / s[1:] + out[1:]
    v[0] = out[0]
    return s, v


_VH_CACHE: dict = {}


def atomic_hartree(sym: str, r: np.ndarray) -> np.ndarray:
    if sym not in _VH_CACHE:
        _VH_CACHE[sym] = _radial_hartree_table(sym)
    s, v = _VH_CACHE[sym]
    q_tot = sum(occ for _, occ, _ in _shells(sym))
    out = np.interp(r, s, v)
    far = r > s[-1]
    out[far] = q_tot / r[far]
    return out


@dataclass
class Molecule:
    symbols: list
    pos: np.ndarray  # (Na, 3)

    @property
    def Z(self) -> np.ndarray:
        return np.array([ATOM_Z[s] for s in self.symbols], dtype=np.float64)


def _dist(xyz: np.ndarray, R: np.ndarray) -> np.ndarray:
    # xyz: (..., 3)
    return np.sqrt(np.sum((xyz - R) ** 2, axis=-1))


def density0(mol: Molecule, pts: np.ndarray) -> np.ndarray:
    """Superposition of atomic densities, the form of Eq. initial_density."""
    rho = np.zeros(pts.shape[:-1])
    for s, R in zip(mol.symbols, mol.pos):
        rho += atomic_density(s, _dist(pts, R))
    return rho


def v_ext(mol: Molecule, pts: np.ndarray) -> np.ndarray:
    """External potential -sum_j Z_j/|r - R_j| (Eq. classical-electrostatics)."""
    v = np.zeros(pts.shape[:-1])
    for s, R in zip(mol.symbols, mol.pos):
        v -= ATOM_Z[s] / _dist(pts, R)
    return v


def nuclear_repulsion(mol: Molecule) -> float:
    """E_ZZ = 1/2 sum_{i != j} Z_i Z_j / |R_i - R_j| (Eq. electrostatics)."""
    Z, R = mol.Z, mol.pos
    e = 0.0
    for i in range(len(Z)):
        for j in range(i + 1, len(Z)):
            e += Z[i] * Z[j] / float(np.linalg.norm(R[i] - R[j]))
    return e


def v_hartree0(mol: Molecule, pts: np.ndarray) -> np.ndarray:
    v = np.zeros(pts.shape[:-1])
    for s, R in zip(mol.symbols, mol.pos):
        v += atomic_hartree(s, _dist(pts, R))
    return v


# --------------------------------------------------------------------------
# LDA exchange-correlation (Section 2, the LDA of Ceperley-Alder as
# parametrised by Perdew and Zunger; Libxc is not available, so the published
# spin-unpolarised formulas are written out here).  Input preparation only:
# V_eff enters the convolutions as data.
# --------------------------------------------------------------------------

# correlation fit parameters: r_s >= 1 (gamma, beta1, beta2), r_s < 1 (A, B, C, D)
PZ81_LOW_DENSITY = (-0.1423, 1.0529, 0.3334)
PZ81_HIGH_DENSITY = (0.0311, -0.048, 0.0020, -0.0116)


def lda_xc(rho: np.ndarray):
    """Exchange-correlation energy per electron eps_xc and potential
    v_xc = d(rho eps_xc)/d rho of the spin-unpolarised LDA.

    Exchange (Dirac/Slater): eps_x = -(3/4)(3 rho/pi)^(1/3), v_x = (4/3) eps_x.
    Correlation in r_s = (3/(4 pi rho))^(1/3):
      r_s >= 1: eps_c = gamma/(1 + b1 sqrt(r_s) + b2 r_s),
                v_c = eps_c (1 + 7/6 b1 sqrt(r_s) + 4/3 b2 r_s)/(1 + b1 sqrt(r_s) + b2 r_s);
      r_s < 1:  eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
                v_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2 D - C)/3 r_s.
    Points with rho <= 1e-30 get zero.
    """
    rho = np.asarray(rho, dtype=np.float64)
    ex = np.zeros_like(rho)
    ec = np.zeros_like(rho)
    vx = np.zeros_like(rho)
    vc = np.zeros_like(rho)
    m = rho > 1e-30
    r = rho[m]
    ex[m] = -0.75 * np.cbrt(3.0 * r / math.pi)
    vx[m] = 4.0 / 3.0 * ex[m]
    rs = np.cbrt(3.0 / (4.0 * math.pi * r))
    g, b1, b2 = PZ81_LOW_DENSITY
    A, B, C, D = PZ81_HIGH_DENSITY
    lo = rs >= 1.0
    sq = np.sqrt(rs[lo])
    den = 1.0 + b1 * sq + b2 * rs[lo]
    e_lo = g / den
    v_lo = e_lo * (1.0 + 7.0 / 6.0 * b1 * sq + 4.0 / 3.0 * b2 * rs[lo]) / den
    rh = rs[~lo]
    ln = np.log(rh)
    e_hi = A * ln + B + C * rh * ln + D * rh
    v_hi = A * ln + (B - A / 3.0) + 2.0 / 3.0 * C * rh * ln + (2.0 * D - C) / 3.0 * rh
    ecm = np.empty_like(r)
    vcm = np.empty_like(r)
    ecm[lo], ecm[~lo] = e_lo, e_hi
    vcm[lo], vcm[~lo] = v_lo, v_hi
    ec[m] = ecm
    vc[m] = vcm
    return ex + ec, vx + vc


# --------------------------------------------------------------------------
# Adaptive refinement (Section 3.2, Eq. refinement_criterion)
# --------------------------------------------------------------------------


def _children(lo: np.ndarray, hi: np.ndarray):
    """Bisect each cell in the three coordinate directions: (8M, 3) arrays."""
    mid = 0.5 * (lo + hi)
    los, his = [], []
    for code in range(8):
        b = np.array([(code >> d) & 1 for d in range(3)], dtype=bool)
        clo = np.where(b, mid, lo)
        chi = np.where(b, hi, mid)
        los.append(clo)
        his.append(chi)
    # child-major within each parent: shape (M, 8, 3)
    return np.stack(los, axis=1).reshape(-1, 3), np.stack(his, axis=1).reshape(-1, 3)


def _cell_integrals(fn, lo, hi, p, chunk=4096):
    out = np.empty(lo.shape[0])
    for s in range(0, lo.shape[0], chunk):
        pts, wts = cell_points(lo[s : s + chunk], hi[s : s + chunk], p)
        out[s : s + chunk] = np.sum(fn(pts) * wts, axis=1)
    return out


def _split_at_atoms(lo, hi, atoms, tol=1e-12):
    """Final refinement: a cell holding an atom in its interior (or on a face
    interior) is cut through the atom so the atom ends up at a vertex."""
    changed = True
    while changed:
        changed = False
        new_lo, new_hi = [], []
        for a in atoms:
            inside = np.all((lo <= a + tol) & (hi >= a - tol), axis=1)
            strict = (lo < a - tol) & (hi > a + tol)  # (M, 3): dims to cut
            need = inside & np.any(strict, axis=1)
            if not np.any(need):
                continue
            changed = True
            keep = ~need
            for c in np.nonzero(need)[0]:
                cuts = [[(lo[c, d], a[d]), (a[d], hi[c, d])] if strict[c, d] else [(lo[c, d], hi[c, d])] for d in range(3)]
                for ix in cuts[0]:
                    for iy in cuts[1]:
                        for iz in cuts[2]:
                            new_lo.append([ix[0], iy[0], iz[0]])
                            new_hi.append([ix[1], iy[1], iz[1]])
            lo, hi = lo[keep], hi[keep]
        if new_lo:
            lo = np.concatenate([lo, np.array(new_lo)])
            hi = np.concatenate([hi, np.array(new_hi)])
    return lo, hi


def _fix_aspect(lo, hi, max_ratio=2.0):
    """Cells with extent ratio above max_ratio are bisected along their
    longest side until none remain (the paper's aspect-ratio refinement; the
    threshold is not printed, 2 is this module's reading)."""
    while True:
        ext = hi - lo
        ratio = ext.max(axis=1) / ext.min(axis=1)
        bad = ratio > max_ratio
        if not np.any(bad):
            return lo, hi
        d = np.argmax(ext[bad], axis=1)
        blo, bhi = lo[bad].copy(), hi[bad].copy()
        mid = 0.5 * (blo[np.arange(len(d)), d] + bhi[np.arange(len(d)), d])
        a_lo, a_hi = blo.copy(), bhi.copy()
        a_hi[np.arange(len(d)), d] = mid
        b_lo, b_hi = blo.copy(), bhi.copy()
        b_lo[np.arange(len(d)), d] = mid
        lo = np.concatenate([lo[~bad], a_lo, b_lo])
        hi = np.concatenate([hi[~bad], a_hi, b_hi])


def adaptive_mesh(mol: Molecule, half_width: float, p: int, tol_m: float,
                  uniform_levels: int = 3, max_level: int = 40) -> Mesh:
    """Adaptive cell mesh per Section 3.2: uniform levels, then keep the 8
    children of a cell whenever |int_C t - sum_i int_{C_i} t| >= tol_m with the
    test function t = sqrt(rho0) * V_ext (Eq. test_function), then cut cells
    through atoms and fix aspect ratios."""

    def t_fn(pts):
        return np.sqrt(density0(mol, pts)) * v_ext(mol, pts)

    lo = np.full((1, 3), -half_width)
    hi = np.full((1, 3), half_width)
    for _ in range(uniform_levels):
        lo, hi = _children(lo, hi)
    final_lo, final_hi = [], []
    front_lo, front_hi = lo, hi
    front_int = _cell_integrals(t_fn, front_lo, front_hi, p)
    level = uniform_levels
    while front_lo.shape[0] and level < max_level:
        clo, chi = _children(front_lo, front_hi)
        cint = _cell_integrals(t_fn, clo, chi, p)
        err = np.abs(front_int - cint.reshape(-1, 8).sum(axis=1))
        refine = err >= tol_m
        final_lo.append(front_lo[~refine])
        final_hi.append(front_hi[~refine])
        mask = np.repeat(refine, 8)
        front_lo, front_hi, front_int = clo[mask], chi[mask], cint[mask]
        level += 1
    final_lo.append(front_lo)
    final_hi.append(front_hi)
    lo = np.concatenate(final_lo)
    hi = np.concatenate(final_hi)
    lo, hi = _split_at_atoms(lo, hi, mol.pos)
    lo, hi = _fix_aspect(lo, hi)
    # deterministic cell order (lexicographic by lower corner)
    order = np.lexsort((lo[:, 2], lo[:, 1], lo[:, 0]))
    return mesh_from_cells(lo[order], hi[order], p)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------


@dataclass
class Workload:
    """One Green-iteration input: mesh, effective potential, orbitals, density."""

    name: str
    mesh: Mesh
    veff: np.ndarray  # (N,)
    psi: np.ndarray  # (nw, N)
    eps: np.ndarray  # (nw,) unshifted eigenvalue guesses
    rho: np.ndarray  # (N,)
    vshift: float
    theta: float
    degree: int
    leaf_size: int
    alpha: float = 1.0
    meta: dict = field(default_factory=dict)
    vext: np.ndarray = None  # (N,) external potential, for SCF steps (atoms and molecules)
    n_elec: float = 0.0      # number of electrons N_e
    e_zz: float = 0.0        # nuclear repulsion (Eq. electrostatics)

    @property
    def n(self) -> int:
        return self.mesh.n

    @property
    def k(self) -> np.ndarray:
        """Yukawa decay rates k = sqrt(-2 (eps + V_shift)) (Eq. gauge-shift)."""
        return np.sqrt(-2.0 * (self.eps + self.vshift))

    @property
    def f(self) -> np.ndarray:
        """Convolution sources f = (V_eff + V_shift) psi, one row per orbital."""
        return (self.veff + self.vshift)[None, :] * self.psi


def hydrogen_1s(seed: int = 0, ncell: int = 8, p: int = 3, half_width: float = 10.0) -> Workload:
    """Hydrogen 1s on a uniform [-10,10]^3 mesh of ncell^3 cells.

    The nucleus sits on an interior cell vertex picked by the seed within
    +-2.5 Bohr of the origin, so no quadrature node coincides with it.
    psi = e^{-r}/sqrt(pi), V = -1/r, eps = -0.5, V_shift = 0, so k = 1.
    """
    mesh = uniform_mesh(-half_width, half_width, ncell, p)
    h = 2 * half_width / ncell
    rng = np.random.default_rng(seed)
    cand = np.arange(-ncell // 2 + 1, ncell // 2) * h
    cand = cand[np.abs(cand) <= 2.5 + 1e-12]
    R = rng.choice(cand, size=3)
    pts = mesh.xyz.T
    r = _dist(pts, R)
    psi = np.exp(-r) / math.sqrt(math.pi)
    veff = -1.0 / r
    rho = psi * psi
    return Workload(name=f"H1s-{ncell}^3-p{p}", mesh=mesh, veff=veff, psi=psi[None, :],
                    eps=np.array([-0.5]), rho=rho, vshift=0.0, theta=0.7, degree=6,
                    leaf_size=2000, meta={"nucleus": R.tolist(), "seed": seed})


def hydrogen_adaptive(seed: int = 0, tol_m: float = 1e-3, p: int = 4, half_width: float = 20.0,
                      uniform_levels: int = 2) -> Workload:
    """Hydrogen on an adaptive mesh (Section 3.2) that resolves the nucleus:
    the nucleus sits at the origin, a cell vertex on every level, so no
    quadrature node of the refinement coincides with it.  The seed picks a
    1% smooth perturbation of psi (none for seed 0).  V = -1/r,
    psi = e^{-r}/sqrt(pi), eps = -0.5, V_shift = 0."""
    rng = np.random.default_rng(seed)
    R = np.zeros(3)
    mol = Molecule(["H"], R[None, :])
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    r = _dist(mesh.xyz.T, R)
    psi = np.exp(-r) / math.sqrt(math.pi)
    if seed:
        psi = psi * _smooth_perturbation(rng, mesh.xyz.T)
    return Workload(name=f"H-adaptive-{mesh.n}", mesh=mesh, veff=-1.0 / r, psi=psi[None, :],
                    eps=np.array([-0.5]), rho=psi * psi, vshift=0.0, theta=0.7, degree=6, leaf_size=2000,
                    meta={"nucleus": R.tolist(), "seed": seed, "tol_m": tol_m})


def _smooth_perturbation(rng, pts, amp=0.01):
    a = rng.normal(size=3)
    a *= 0.5 / np.linalg.norm(a)
    ph = rng.uniform(0, 2 * np.pi)
    return 1.0 + amp * np.sin(pts @ a + ph)


def lithium(seed: int = 1, tol_m: float = 3e-7, p: int = 4, half_width: float = 20.0,
            uniform_levels: int = 3) -> Workload:
    """Li atom at the origin: adaptive mesh on [-20,20]^3, p = 4, two occupied
    orbitals (hydrogenic 1s and 2s with Z = 3, the 2s with a seeded 1% smooth
    perturbation), V_eff = V_ext + V_H[rho0] + V_xc^LDA[rho0], Hartree source
    rho0.  The
    default tolerance 3e-7 gives about 309k points (1e-5 gives 162k with this
    test function)."""
    mol = Molecule(["Li"], np.zeros((1, 3)))
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    rng = np.random.default_rng(seed)
    pts = mesh.xyz.T
    r = _dist(pts, mol.pos[0])
    psi1 = radial_orbital("1s", 3.0, r)
    psi2 = radial_orbital("2s", 3.0, r) * _smooth_perturbation(rng, pts)
    rho = density0(mol, pts)
    vx = v_ext(mol, pts)
    veff = vx + v_hartree0(mol, pts) + lda_xc(rho)[1]
    eps = np.array([-1.9, -0.11]) + rng.uniform(-0.02, 0.02, size=2)
    return Workload(name="Li", mesh=mesh, veff=veff, psi=np.stack([psi1, psi2]), eps=eps,
                    rho=rho, vshift=-0.5, theta=0.7, degree=8, leaf_size=2000,
                    meta={"seed": seed, "tol_m": tol_m}, vext=vx, n_elec=3.0, e_zz=0.0)


def carbon_monoxide(seed: int = 2, tol_m: float = 1e-8, p: int = 4, half_width: float = 20.0,
                    n_orb: int = 7, uniform_levels: int = 3) -> Workload:
    """CO with C at (-1.06581,0,0) and O at (+1.06581,0,0) (Section 6):
    adaptive mesh, n_orb orbitals from a seeded superposition of atomic
    Slater orbitals, eps seeded uniformly in [-20, -0.3] Ha."""
    mol = Molecule(["C", "O"], np.array([[-1.06581, 0.0, 0.0], [1.06581, 0.0, 0.0]]))
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    return _molecule_workload("CO", mol, mesh, seed, n_orb)


CO_BOND = 2.13162  # Bohr: C at (-1.06581, 0, 0), O at (+1.06581, 0, 0) (Section 6)


def carbon_monoxide_scf(tol_m: float = 3e-7, p: int = 4, half_width: float = 20.0,
                        uniform_levels: int = 3, R: float = CO_BOND) -> Workload:
    """CO for an SCF run from an aufbau-style start: 8 orbitals (7 doubly
    occupied and the 2pi* virtual, N_w = 8 as in Section 6), built from the
    Slater-screened atomic orbitals in energy order and orthonormalised in
    that order: O 1s, C 1s, 3sigma (2s of both), 4sigma (2p along the bond),
    1pi (2p_y and 2p_z), 5sigma (carbon 2s - 2p lone pair), 2pi* (O - C 2p_y),
    with the atomic LDA-like eigenvalues as guesses.  The bond lies on x.
    V_shift = -1.5: a deeper gauge shift (Eq. gauge-shift leaves the
    eigenproblem unchanged) keeps eps + V_shift < 0 through the first
    gradient-free updates from this crude start.  The tol_m = 3e-7 mesh has
    638,500 points (the paper's CO mesh at this tolerance: 661,625).  R: the
    bond length (the paper's by default), the nuclei at (-R/2, 0, 0) (C) and
    (R/2, 0, 0) (O)."""
    mol = Molecule(["C", "O"], np.array([[-0.5 * R, 0.0, 0.0], [0.5 * R, 0.0, 0.0]]))
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    pts = mesh.xyz.T
    C, O = mol.pos[0], mol.pos[1]
    (_, _, zc1), (_, _, zc2), _ = _shells("C")
    (_, _, zo1), (_, _, zo2), _ = _shells("O")

    def ao(kind, Z, R, d=None):
        r = _dist(pts, R)
        f = radial_orbital(kind, Z, r)
        return f if d is None else f * (pts[:, d] - R[d]) / np.maximum(r, 1e-300)

    basis = [ao("1s", zo1, O), ao("1s", zc1, C), ao("2s", zo2, O) + ao("2s", zc2, C),
             ao("2p", zo2, O, 0) - ao("2p", zc2, C, 0), ao("2p", zo2, O, 1) + ao("2p", zc2, C, 1),
             ao("2p", zo2, O, 2) + ao("2p", zc2, C, 2), ao("2s", zc2, C) - ao("2p", zc2, C, 0),
             ao("2p", zo2, O, 1) - ao("2p", zc2, C, 1)]
    w = mesh.w
    q = []
    for v in basis:
        v = v.copy()
        for u in q:
            v -= np.sum(v * u * w) * u
        q.append(v / np.sqrt(np.sum(v * v * w)))
    rho = density0(mol, pts)
    vx = v_ext(mol, pts)
    veff = vx + v_hartree0(mol, pts) + lda_xc(rho)[1]
    eps = np.array([-18.8, -9.9, -1.0, -0.5, -0.45, -0.45, -0.35, -0.1])
    return Workload(name="CO", mesh=mesh, veff=veff, psi=np.array(q), eps=eps, rho=rho, vshift=-1.5, theta=0.7,
                    degree=8, leaf_size=2000, meta={"tol_m": tol_m, "start": "aufbau", "R": float(R),
                                                    "nuclei": mol.pos.copy()}, vext=vx, n_elec=14.0,
                    e_zz=nuclear_repulsion(mol))


def co_bond_lengths(seed: int = 6, count: int = 32, lo: float = 1.9, hi: float = 2.4) -> np.ndarray:
    """Seeded CO bond lengths for the density warm-start data set: `count`
    values drawn uniformly in [lo, hi] Bohr, sorted."""
    return np.sort(np.random.default_rng(seed).uniform(lo, hi, size=count))


def hydrogen_molecule(R: float, tol_m: float = 3e-6, p: int = 4, half_width: float = 20.0,
                      uniform_levels: int = 3) -> Workload:
    """H2 with its nuclei at (-R/2, 0, 0) and (R/2, 0, 0) for an SCF run: the
    adaptive mesh of Section 3.2 (about 170k-200k points at tol_m = 3e-6),
    one orbital (sigma_g, both electrons) started from the normalised
    superposition of the atomic 1s orbitals, the hydrogen-atom eigenvalue
    -0.5 Ha as its guess, and the superposed atomic densities."""
    mol = Molecule(["H", "H"], np.array([[-0.5 * R, 0.0, 0.0], [0.5 * R, 0.0, 0.0]]))
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    pts = mesh.xyz.T
    s = radial_orbital("1s", 1.0, _dist(pts, mol.pos[0])) + radial_orbital("1s", 1.0, _dist(pts, mol.pos[1]))
    s = s / np.sqrt(np.sum(s * s * mesh.w))
    rho = density0(mol, pts)
    vx = v_ext(mol, pts)
    veff = vx + v_hartree0(mol, pts) + lda_xc(rho)[1]
    return Workload(name=f"H2-R{R:.4f}", mesh=mesh, veff=veff, psi=s[None, :], eps=np.array([-0.5]), rho=rho,
                    vshift=-0.5, theta=0.7, degree=8, leaf_size=2000,
                    meta={"R": float(R), "tol_m": tol_m, "nuclei": mol.pos.copy()}, vext=vx, n_elec=2.0,
                    e_zz=nuclear_repulsion(mol))


def h2_bond_lengths(seed: int = 5, count: int = 32, lo: float = 1.0, hi: float = 2.0) -> np.ndarray:
    """Seeded H2 bond lengths for the warm-start data set: `count` values
    drawn uniformly in [lo, hi] Bohr, sorted."""
    return np.sort(np.random.default_rng(seed).uniform(lo, hi, size=count))


def benzene(seed: int = 3, tol_m: float = 3e-8, p: int = 4, half_width: float = 20.0,
            n_orb: int = 21, uniform_levels: int = 3) -> Workload:
    """C6H6 in the z=0 plane at the paper's geometry (Section 6)."""
    pos = np.array([[x, y, 0.0] for x, y in BENZENE_C + BENZENE_H])
    mol = Molecule(["C"] * 6 + ["H"] * 6, pos)
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    return _molecule_workload("C6H6", mol, mesh, seed, n_orb)


BENZENE_C = [(-0.682781, 2.548170), (0.682781, -2.548170), (2.548230, -0.682767), (-2.548230, 0.682767),
             (1.86544, 1.86541), (-1.86544, -1.86541)]
BENZENE_H = [(-1.21247, 4.52502), (1.21247, -4.52502), (4.52548, -1.21333), (-4.52548, 1.21333),
             (3.31252, 3.31351), (-3.31252, -3.31351)]


def ring_combinations(funcs, angles):
    """Six functions placed around a hexagonal ring at the given angles ->
    their six ring combinations, in this order: the sum; the cos and sin of
    the angle (relative to the first function's) as weights; the cos and sin
    of twice the angle; alternating signs (cos of three times the angle)."""
    phi = np.asarray(angles, dtype=np.float64) - float(angles[0])
    out = [sum(funcs)]
    for m in (1, 2):
        out.append(sum(math.cos(m * a) * f for a, f in zip(phi, funcs)))
        out.append(sum(math.sin(m * a) * f for a, f in zip(phi, funcs)))
    out.append(sum(math.cos(3 * a) * f for a, f in zip(phi, funcs)))
    return out


def benzene_scf(tol_m: float = 3e-8, p: int = 4, half_width: float = 20.0, uniform_levels: int = 3) -> Workload:
    """C6H6 for an SCF run from an aufbau-style start: 21 orbitals (N_e = 42,
    every level doubly occupied), built from the Slater-screened atomic
    orbitals and orthonormalised in this order:
      6 carbon 1s;
      6 C-C sigma bonds: the two sp2 hybrids (2s + sqrt(2) 2p)/sqrt(3) that
        point along the bond, summed;
      6 C-H sigma bonds: the carbon hybrid pointing at its hydrogen plus the
        hydrogen 1s;
      3 pi levels: the carbon 2p_z combinations of the lowest Hueckel levels
        of the ring (all in phase, and weighted by the cosine and the sine
        of each carbon's angle around the ring).
    Each set of six equivalent functions enters as its ring combinations
    (ring_combinations: weights 1, cos/sin of m times the angle for m = 1, 2,
    and alternating signs), the symmetry types of the hexagonal ring.  The
    six 1s levels lie within a few mHa of one another; started from the
    localised 1s functions, Green Iteration would rotate them toward these
    combinations at a rate set by that splitting, far too slowly for its
    per-orbital residual to converge.
    Eigenvalue guesses -9.9 (1s), -0.8 (C-C), -0.6 (C-H), -0.45 and -0.3
    (pi) Ha; V_shift = -1.5 (c31).  The default tol_m = 3e-8 mesh has about
    4.6M points; the paper's Table timings row used tol_m = 3e-6 (1,464,500
    points)."""
    pos = np.array([[x, y, 0.0] for x, y in BENZENE_C + BENZENE_H])
    mol = Molecule(["C"] * 6 + ["H"] * 6, pos)
    mesh = adaptive_mesh(mol, half_width, p, tol_m, uniform_levels=uniform_levels)
    pts = mesh.xyz.T
    (_, _, z1), (_, _, z2), _ = _shells("C")
    Cpos, Hpos = pos[:6], pos[6:]

    def hybrid(i, target):
        R = Cpos[i]
        r = _dist(pts, R)
        d = (target - R) / np.linalg.norm(target - R)
        p_dir = radial_orbital("2p", z2, r) * ((pts - R) @ d) / np.maximum(r, 1e-300)
        return (radial_orbital("2s", z2, r) + math.sqrt(2.0) * p_dir) / math.sqrt(3.0)

    def pz(i):
        R = Cpos[i]
        r = _dist(pts, R)
        return radial_orbital("2p", z2, r) * (pts[:, 2] - R[2]) / np.maximum(r, 1e-300)

    ang = np.arctan2(Cpos[:, 1], Cpos[:, 0])
    basis = ring_combinations([radial_orbital("1s", z1, _dist(pts, R)) for R in Cpos], ang)
    pairs = [(i, j) for i in range(6) for j in range(i + 1, 6) if np.linalg.norm(Cpos[i] - Cpos[j]) < 3.0]
    assert len(pairs) == 6
    mid = [0.5 * (Cpos[i] + Cpos[j]) for i, j in pairs]
    basis += ring_combinations([hybrid(i, Cpos[j]) + hybrid(j, Cpos[i]) for i, j in pairs],
                               np.array([math.atan2(m[1], m[0]) for m in mid]))
    ch = []
    for i in range(6):
        h = int(np.argmin(np.linalg.norm(Hpos - Cpos[i], axis=1)))
        ch.append(hybrid(i, Hpos[h]) + radial_orbital("1s", 1.0, _dist(pts, Hpos[h])))
    basis += ring_combinations(ch, ang)
    basis.append(sum(pz(i) for i in range(6)))
    basis.append(sum(math.cos(ang[i]) * pz(i) for i in range(6)))
    basis.append(sum(math.sin(ang[i]) * pz(i) for i in range(6)))
    w = mesh.w
    q = []
    for v in basis:
        v = v.copy()
        for u in q:
            v -= np.sum(v * u * w) * u
        q.append(v / np.sqrt(np.sum(v * v * w)))
    rho = density0(mol, pts)
    vx = v_ext(mol, pts)
    veff = vx + v_hartree0(mol, pts) + lda_xc(rho)[1]
    eps = np.array([-9.9] * 6 + [-0.8] * 6 + [-0.6] * 6 + [-0.45, -0.3, -0.3])
    return Workload(name="C6H6", mesh=mesh, veff=veff, psi=np.array(q), eps=eps, rho=rho, vshift=-1.5, theta=0.7,
                    degree=8, leaf_size=2000, meta={"tol_m": tol_m, "start": "aufbau"}, vext=vx, n_elec=42.0,
                    e_zz=nuclear_repulsion(mol))


def _molecule_workload(name, mol, mesh, seed, n_orb):
    rng = np.random.default_rng(seed)
    pts = mesh.xyz.T
    basis = []
    for s, R in zip(mol.symbols, mol.pos):
        r = _dist(pts, R)
        for kind, _, Z in _shells(s):
            basis.append(radial_orbital(kind, Z, r))
            if kind == "2p":
                for d in range(3):
                    basis.append(radial_orbital("2p", Z, r) * (pts[:, d] - R[d]) / np.maximum(r, 1e-300))
    basis = np.stack(basis)
    coef = rng.normal(size=(n_orb, basis.shape[0]))
    psi = coef @ basis
    rho = density0(mol, pts)
    vx = v_ext(mol, pts)
    veff = vx + v_hartree0(mol, pts) + lda_xc(rho)[1]
    eps = np.sort(rng.uniform(-20.0, -0.3, size=n_orb))
    return Workload(name=name, mesh=mesh, veff=veff, psi=psi, eps=eps, rho=rho, vshift=-0.5,
                    theta=0.7, degree=8, leaf_size=2000, meta={"seed": seed, "n_orb": n_orb}, vext=vx,
                    n_elec=float(sum(ATOM_Z[a] for a in mol.symbols)), e_zz=nuclear_repulsion(mol))


def mlp_init(seed: int = 0, n_features: int = 8, hidden: int = 32) -> np.ndarray:
    """Seeded initial parameters of the warm-start MLP, packed as W1 (H x F),
    b1 (H), W2 (H x H), b2 (H), W3 (H), b3 (1): weights uniform in
    +-sqrt(6 / (fan_in + fan_out)) (Glorot and Bengio, 2010), biases zero;
    float32 values."""
    rng = np.random.default_rng(seed)
    F, H = n_features, hidden
    parts = []
    for fan_in, fan_out in ((F, H), (H, H), (H, 1)):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-a, a, size=fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def random_cube(n: int, seed: int = 0, half_width: float = 1.0):
    """n uniformly random points in a cube with random positive weights and a
    smooth field: the small parity stress case (ragged sizes, no mesh)."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-half_width, half_width, size=(3, n))
    w = rng.uniform(0.5, 1.5, size=n) * (2 * half_width) ** 3 / max(n, 1)
    return np.ascontiguousarray(xyz), w

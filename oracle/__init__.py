"""FP64 CPU oracle for the TAGI convolution sums and the Green step.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library.  The arithmetic lives in ``oracle.c`` (direct sums,
tree, Algorithm 3 treecode, anterpolation); this module loads it with ctypes
and adds the Green step of Algorithm 2 in plain NumPy.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, invariants and brute force (see each test's docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", _SO, _SRC, "-lm"])
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.oracle_direct_yukawa.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int64, _D, _D,
                                           _D, _D, _D, ctypes.c_double, ctypes.c_int, _D]
        L.oracle_direct_coulomb.argtypes = L.oracle_direct_yukawa.argtypes
        L.oracle_threads.argtypes = [ctypes.c_int]
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_tree_build.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int]
        L.oracle_tree_build.restype = ctypes.c_void_p
        L.oracle_tree_free.argtypes = [ctypes.c_void_p]
        L.oracle_tree_num_clusters.argtypes = [ctypes.c_void_p]
        L.oracle_tree_export.argtypes = [ctypes.c_void_p, _I64, _I64, _I64, _D, _D, _I32, _I32,
                                         _I32, _I32]
        L.oracle_tree_lists.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int64, _I32, _I32, _I32]
        L.oracle_tree_lists.restype = ctypes.c_int64
        L.oracle_cluster_proxies.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, _D, _D]
        L.oracle_anterpolate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         _D, _D]
        L.oracle_treecode.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, _D, _D, _D]
        L.oracle_treecode_batches.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _D,
                                              ctypes.c_int, _I32, _D]
        _lib = L
    return _lib


def threads(n: int = 0) -> int:
    """Set the oracle's OpenMP thread count (n > 0) and return the count in use."""
    return int(lib().oracle_threads(int(n)))


def _p(a, t=_D):
    return a.ctypes.data_as(t)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- direct sums
def direct_yukawa(xyz, w, f, k, ss=True, targets=None):
    """Eq. direct-sum with G_k = exp(-k r)/(4 pi r); SS per Eq. yukawa-conv-ss.

    xyz (3, N), w (N,), f (N,).  targets: optional index array; the result
    then holds those targets only (sources are always all N points)."""
    xyz, w, f = _c(xyz), _c(w), _c(f)
    ti = np.arange(xyz.shape[1]) if targets is None else np.asarray(targets)
    t = _c(xyz[:, ti])
    tf = _c(f[ti])
    u = np.zeros(len(ti))
    lib().oracle_direct_yukawa(len(ti), _p(t[0]), _p(t[1]), _p(t[2]), _p(tf), xyz.shape[1],
                               _p(xyz[0]), _p(xyz[1]), _p(xyz[2]), _p(w), _p(f), float(k),
                               int(ss), _p(u))
    return u


def direct_coulomb(xyz, w, rho, alpha=1.0, ss=True, targets=None):
    """Eq. direct-sum with 1/r; SS per Eq. coulomb-conv-ss and correction_term."""
    xyz, w, rho = _c(xyz), _c(w), _c(rho)
    ti = np.arange(xyz.shape[1]) if targets is None else np.asarray(targets)
    t = _c(xyz[:, ti])
    tr = _c(rho[ti])
    v = np.zeros(len(ti))
    lib().oracle_direct_coulomb(len(ti), _p(t[0]), _p(t[1]), _p(t[2]), _p(tr), xyz.shape[1],
                                _p(xyz[0]), _p(xyz[1]), _p(xyz[2]), _p(w), _p(rho), float(alpha),
                                int(ss), _p(v))
    return v


# ---------------------------------------------------------------- treecode
class Tree:
    """Source-cluster tree of Section 5.1 (batches = leaves, N_B = N_L)."""

    def __init__(self, xyz, leaf_size):
        self.xyz = _c(xyz)
        self.n = self.xyz.shape[1]
        self.leaf_size = int(leaf_size)
        self._h = lib().oracle_tree_build(self.n, _p(self.xyz[0]), _p(self.xyz[1]),
                                          _p(self.xyz[2]), self.leaf_size)
        if not self._h:
            raise ValueError("oracle tree build rejected its arguments")
        nc = lib().oracle_tree_num_clusters(self._h)
        self.nc = nc
        self.idx = np.empty(self.n, np.int64)
        self.begin = np.empty(nc, np.int64)
        self.end = np.empty(nc, np.int64)
        self.lo = np.empty((nc, 3))
        self.hi = np.empty((nc, 3))
        self.parent = np.empty(nc, np.int32)
        self.level = np.empty(nc, np.int32)
        self.nchild = np.empty(nc, np.int32)
        self.child = np.empty((nc, 8), np.int32)
        lib().oracle_tree_export(self._h, _p(self.idx, _I64), _p(self.begin, _I64),
                                 _p(self.end, _I64), _p(self.lo), _p(self.hi),
                                 _p(self.parent, _I32), _p(self.level, _I32),
                                 _p(self.nchild, _I32), _p(self.child, _I32))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_tree_free(self._h)
            self._h = None

    @property
    def leaves(self):
        return np.nonzero(self.nchild == 0)[0]

    def points(self, c):
        return self.idx[self.begin[c]:self.end[c]]

    def key(self, c):
        """Order-free identity of a cluster: (smallest point index, size)."""
        pts = self.points(c)
        return (int(pts.min()), int(len(pts)))

    def lists(self, theta, degree):
        """Algorithm 3's visits: arrays batch, cluster, kind (0 direct, 1 approx)."""
        cap = 1 << 16
        while True:
            b = np.empty(cap, np.int32)
            c = np.empty(cap, np.int32)
            k = np.empty(cap, np.int32)
            cnt = lib().oracle_tree_lists(self._h, float(theta), int(degree), cap, _p(b, _I32),
                                          _p(c, _I32), _p(k, _I32))
            if cnt <= cap:
                return b[:cnt], c[:cnt], k[:cnt]
            cap = int(cnt)

    def proxies(self, c, degree):
        P = (degree + 1) ** 3
        px, py, pz = np.empty(P), np.empty(P), np.empty(P)
        lib().oracle_cluster_proxies(self._h, int(c), int(degree), _p(px), _p(py), _p(pz))
        return np.stack([px, py, pz])

    def anterpolate(self, c, degree, q):
        """Proxy weights of cluster c for charge rows q (nq, N) -> (nq, P)."""
        q = _c(np.atleast_2d(q))
        P = (degree + 1) ** 3
        out = np.empty((q.shape[0], P))
        lib().oracle_anterpolate(self._h, int(c), int(degree), q.shape[0], _p(q), _p(out))
        return out

    def treecode(self, theta, degree, kernel, param, f, w, ss=True):
        f, w = _c(f), _c(w)
        u = np.empty(self.n)
        rc = lib().oracle_treecode(self._h, float(theta), int(degree), int(kernel), float(param),
                                   int(ss), _p(f), _p(w), _p(u))
        if rc:
            raise ValueError("oracle treecode rejected its arguments")
        return u

    def treecode_batches(self, theta, degree, kernel, param, f, w, batches, ss=True):
        f, w = _c(f), _c(w)
        b = _c(batches, np.int32)
        u = np.zeros(self.n)
        lib().oracle_treecode_batches(self._h, float(theta), int(degree), int(kernel),
                                      float(param), int(ss), _p(f), _p(w), len(b), _p(b, _I32),
                                      _p(u))
        return u


def treecode_yukawa(tree, theta, degree, f, k, w, ss=True):
    return tree.treecode(theta, degree, 0, k, f, w, ss)


def treecode_coulomb(tree, theta, degree, rho, w, alpha=1.0, ss=True):
    return tree.treecode(theta, degree, 1, alpha, rho, w, ss)


# ---------------------------------------------------------------- Green step
def green_step(tree, theta, degree, w, veff, vshift, psi, eps, rho=None, alpha=1.0):
    """One Green iteration for all orbitals (Algorithm 2 lines 3-6, batched).

    Applies G(eps_o) to every orbital with its previous eigenvalue, updates each
    eigenvalue by the gradient-free formula (Eq. gradient-free) using the
    un-orthogonalised psi~, then orthonormalises the new orbitals by modified
    Gram-Schmidt in index order under <a, b> = sum a b w.  The gauge shift of
    Eq. gauge-shift enters as V + V_shift and k = sqrt(-2 (eps + V_shift));
    the returned eigenvalues are unshifted.

    Returns psi_new (nw, N), eps_new (nw,), resid (nw,) = ||psi_new - psi||_w,
    and, when rho is given, V_H (N,) and E_H = 1/2 sum V_H rho w
    (Eq. quadrature-example).
    """
    psi = np.atleast_2d(np.asarray(psi, np.float64))
    eps = np.asarray(eps, np.float64)
    nw = psi.shape[0]
    vs = veff + vshift
    es = eps + vshift
    psi_t = np.empty_like(psi)
    for o in range(nw):
        k = np.sqrt(-2.0 * es[o])
        u = treecode_yukawa(tree, theta, degree, vs * psi[o], k, w, ss=True)
        psi_t[o] = -2.0 * u  # Eq. Yukawa: -1/(2 pi) = -2 * 1/(4 pi)
    es_new = np.empty(nw)
    for o in range(nw):
        num = np.sum(vs * psi[o] * (psi[o] - psi_t[o]) * w)
        den = np.sum(psi_t[o] * psi_t[o] * w)
        es_new[o] = es[o] - num / den
    q = np.empty_like(psi)
    for o in range(nw):
        v = psi_t[o].copy()
        for p in range(o):
            v -= np.sum(v * q[p] * w) * q[p]
        q[o] = v / np.sqrt(np.sum(v * v * w))
    resid = np.sqrt(np.sum((q - psi) ** 2 * w[None, :], axis=1))
    out = {"psi": q, "eps": es_new - vshift, "resid": resid, "psi_tilde": psi_t}
    if rho is not None:
        vh = treecode_coulomb(tree, theta, degree, rho, w, alpha=alpha, ss=True)
        out["vh"] = vh
        out["eh"] = 0.5 * np.sum(vh * rho * w)
    return out


# --------------------------------------------------------------------------
# Green Iteration loop with Anderson mixing of eigenpairs (Algorithm 2,
# Section 4.3 "Wavefunction Mixing")
# --------------------------------------------------------------------------


def anderson_mix(X, F, beta, wx):
    """Anderson mixing (Anderson 1965) of a fixed-point iteration x -> g(x).

    X, F: arrays (m+1, L) of the last m+1 inputs x_j and residuals
    F_j = g(x_j) - x_j, oldest first; wx: weights of the inner product
    (a, b) = sum a b wx.  With D_j = F_n - F_{n-j} (j = 1..m), theta solves
    the normal equations of min ||F_n - sum_j theta_j D_j||, and
        x_bar = x_n - sum_j theta_j (x_n - x_{n-j}),
        F_bar = F_n - sum_j theta_j D_j,
        x_next = x_bar + beta F_bar.
    One entry (m = 0) gives simple mixing x_n + beta F_n.  A numerically
    singular Gram matrix (condition number above 1e13) also falls back to
    simple mixing.
    """
    X = np.atleast_2d(np.asarray(X, np.float64))
    F = np.atleast_2d(np.asarray(F, np.float64))
    xn, fn = X[-1], F[-1]
    m = X.shape[0] - 1
    if m == 0:
        return xn + beta * fn
    D = fn[None, :] - F[-2::-1]    # D_j = F_n - F_{n-j}, j = 1..m
    DX = xn[None, :] - X[-2::-1]   # x_n - x_{n-j}
    A = (D * wx[None, :]) @ D.T
    b = (D * wx[None, :]) @ fn
    if not np.all(np.isfinite(A)) or np.linalg.cond(A) > 1e13:
        return xn + beta * fn
    th = np.linalg.solve(A, b)
    x_bar = xn - th @ DX
    f_bar = fn - th @ D
    return x_bar + beta * f_bar


def green_iterate(tree, theta, degree, w, veff, vshift, psi, eps, tol_gi, max_iter, beta=0.5, history=5,
                  mix_tol=np.inf, store_output=False):
    """Green Iteration for all orbitals at once (Algorithm 2, batched as in
    green_step), with Anderson mixing of each eigenpair x = (eps, psi) under
    (x1, x2) = eps1 eps2 + sum psi1 psi2 w (Section 4.3).

    Each step, for every orbital not yet converged:
      line 3: psi~ = G(eps) psi (treecode Yukawa with SS, psi~ = -2 u);
      line 4: eps' = eps - <(V+V_shift) psi, psi - psi~>_w / <psi~, psi~>_w;
      lines 5-6: orthogonalise psi~ in index order against every lower-index
        orbital (the new iterate of an active one, the stored pair of a
        converged one) and normalise: g(x) = (eps', psi');
      line 7: r = ||psi' - psi||_w.  If r < tol_gi the orbital is converged and
        keeps its step input (eps^(n), psi^(n)), as Algorithm 2 stores it, or,
        with store_output, the step's output g(x) = (eps^(n+1), psi^(n+1)):
        inside an SCF iteration the stored input stops following V_eff once
        its change moves the orbital by less than tol_gi in one step.
    Otherwise the next input is g(x), or, once the orbital's residual has
    fallen below mix_tol (mixing stays on from then), the Anderson update of
    its last history+1 pairs (x_j, F_j = g(x_j) - x_j) with parameter beta.

    Returns psi, eps, resid (last residual per orbital), iters (the step count
    at which each orbital converged, -1 if it did not), steps, field_steps
    (sum over steps of the orbitals convolved) and trace (per step, the
    residual of every orbital convolved in it, NaN for the others).
    """
    psi = np.array(np.atleast_2d(psi), np.float64)
    eps = np.array(eps, np.float64)
    nw, n = psi.shape
    vs = veff + vshift
    wx = np.concatenate([[1.0], w])
    conv = np.zeros(nw, bool)
    mixing = np.zeros(nw, bool)
    iters = np.full(nw, -1)
    resid = np.full(nw, np.nan)
    hx = [[] for _ in range(nw)]
    hf = [[] for _ in range(nw)]
    steps = field_steps = 0
    trace = []
    for step in range(max_iter):
        act = np.flatnonzero(~conv)
        if act.size == 0:
            break
        steps += 1
        field_steps += act.size
        e_new, pt = {}, {}
        for o in act:
            if not eps[o] + vshift < 0.0:
                raise ValueError("eps + V_shift must stay negative (Section 3.3)")
            k = np.sqrt(-2.0 * (eps[o] + vshift))
            pt[o] = -2.0 * treecode_yukawa(tree, theta, degree, vs * psi[o], k, w, ss=True)
            e_new[o] = eps[o] - np.sum(vs * psi[o] * (psi[o] - pt[o]) * w) / np.sum(pt[o] * pt[o] * w)
        q = {}
        for o in act:
            v = pt[o].copy()
            for p in range(o):
                b = q[p] if p in q else psi[p]
                v -= np.sum(v * b * w) * b
            q[o] = v / np.sqrt(np.sum(v * v * w))
        trace.append(np.full(nw, np.nan))
        for o in act:
            f_psi = q[o] - psi[o]
            resid[o] = np.sqrt(np.sum(f_psi * f_psi * w))
            trace[-1][o] = resid[o]
            if resid[o] < tol_gi:
                conv[o] = True
                iters[o] = step + 1
                if store_output:
                    eps[o], psi[o] = e_new[o], q[o]
                continue
            if resid[o] < mix_tol:
                mixing[o] = True
            if mixing[o]:
                hx[o].append(np.concatenate([[eps[o]], psi[o]]))
                hf[o].append(np.concatenate([[e_new[o] - eps[o]], f_psi]))
                hx[o] = hx[o][-(history + 1):]
                hf[o] = hf[o][-(history + 1):]
                x = anderson_mix(np.array(hx[o]), np.array(hf[o]), beta, wx)
                eps[o], psi[o] = x[0], x[1:]
            else:
                eps[o], psi[o] = e_new[o], q[o]
    return {"psi": psi, "eps": eps, "resid": resid, "iters": iters, "steps": steps, "field_steps": field_steps,
            "trace": np.array(trace)}


# --------------------------------------------------------------------------
# SCF step (Algorithm 1 lines 2-7): LDA exchange-correlation, Fermi-Dirac
# occupations (Eq. Fermi, density-construction), Anderson density mixing and
# the gradient-free total energy (Eq. total-energy-gradient-free)
# --------------------------------------------------------------------------

# Perdew-Zunger parametrisation of the Ceperley-Alder correlation energy,
# spin-unpolarised: (gamma, beta1, beta2) for r_s >= 1, (A, B, C, D) below
_PZ_GAMMA, _PZ_B1, _PZ_B2 = -0.1423, 1.0529, 0.3334
_PZ_A, _PZ_B, _PZ_C, _PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def _rs(rho):
    return (3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0)


def lda_exchange(rho):
    """Slater exchange in r_s form: eps_x = -(3/(4 pi)) (9 pi/4)^(1/3) / r_s,
    v_x = 4/3 eps_x; zero where rho <= 1e-30.  Returns (eps_x, v_x)."""
    rho = np.asarray(rho, np.float64)
    e = np.zeros_like(rho)
    m = rho > 1e-30
    e[m] = -(3.0 / (4.0 * np.pi)) * (9.0 * np.pi / 4.0) ** (1.0 / 3.0) / _rs(rho[m])
    return e, 4.0 / 3.0 * e


def lda_correlation(rho):
    """Perdew-Zunger correlation energy per electron and potential
    v_c = eps_c - (r_s/3) d eps_c / d r_s; zero where rho <= 1e-30."""
    rho = np.asarray(rho, np.float64)
    e = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho > 1e-30
    rs = _rs(rho[m])
    ec = np.empty_like(rs)
    dec = np.empty_like(rs)  # d eps_c / d r_s
    lo = rs >= 1.0
    x = rs[lo]
    den = 1.0 + _PZ_B1 * np.sqrt(x) + _PZ_B2 * x
    ec[lo] = _PZ_GAMMA / den
    dec[lo] = -_PZ_GAMMA * (0.5 * _PZ_B1 / np.sqrt(x) + _PZ_B2) / den**2
    x = rs[~lo]
    ec[~lo] = _PZ_A * np.log(x) + _PZ_B + _PZ_C * x * np.log(x) + _PZ_D * x
    dec[~lo] = _PZ_A / x + _PZ_C * (np.log(x) + 1.0) + _PZ_D
    e[m] = ec
    v[m] = ec - rs / 3.0 * dec
    return e, v


def lda_xc(rho):
    ex, vx = lda_exchange(rho)
    ec, vc = lda_correlation(rho)
    return ex + ec, vx + vc


def fermi_level(eps, n_elec, kT):
    """Fermi energy mu with 2 sum_i f(eps_i, mu) = N_e and
    f = 1 / (e^{(eps - mu)/kT} + 1) (Eq. Fermi, density-construction), by
    bisection to the resolution of float64.  N_e = 2 N_w fills every state:
    the bisection then ends where every f rounds to 1 (the mu -> infinity
    limit).  Returns (mu, f)."""
    import scipy.special

    eps = np.asarray(eps, np.float64)
    if not (0.0 < n_elec <= 2.0 * eps.size and kT > 0.0):
        raise ValueError("need 0 < N_e <= 2 N_w and kT > 0")
    occ = lambda mu: scipy.special.expit((mu - eps) / kT)
    lo, hi = eps.min() - 60.0 * kT, eps.max() + 60.0 * kT
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if 2.0 * np.sum(occ(mid)) < n_elec:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return mu, occ(mu)


def tol_gi_schedule(step, first=3e-3, final=1e-5, ramp=4):
    """tol_gi for SCF step `step` (Section 6): `first` on the first step, then
    geometric steps down to `final` over the next `ramp` steps."""
    if step <= 0:
        return first
    if step >= ramp:
        return final
    return first * (final / first) ** (step / ramp)


def scf_potentials(tree, theta, degree, w, vext, rho, alpha=1.0):
    """V_eff[rho] = V_ext + V_H[rho] + V_xc[rho] (Eq. effective-potential;
    V_H by the treecode with SS) and the double-counting terms of the
    gradient-free energy: E_H = 1/2 <V_H, rho>, E_xc = <eps_xc, rho>,
    E_vxc = <V_xc, rho>, all quadrature sums."""
    vh = treecode_coulomb(tree, theta, degree, rho, w, alpha=alpha, ss=True)
    exc, vxc = lda_xc(rho)
    return {"veff": vext + vh + vxc, "vh": vh, "vxc": vxc, "e_h": 0.5 * np.sum(vh * rho * w),
            "e_xc": np.sum(exc * rho * w), "e_vxc": np.sum(vxc * rho * w)}


def scf_step(tree, theta, degree, w, vext, rho_in, psi, eps, vshift, n_elec, kT, e_zz, tol_gi, max_iter,
             mix, scf_beta=0.5, scf_history=5, gi_beta=0.5, gi_history=5, mix_tol=np.inf, alpha=1.0,
             gi_store_output=False):
    """One SCF iteration (Algorithm 1):
      line 2: V_eff[rho_in] (scf_potentials);
      line 3: eigenpairs by Green Iteration with Anderson mixing
        (green_iterate), warm-started from (eps, psi); the orbitals are then
        normalised in the quadrature norm;
      line 4: mu and occupations f_i (fermi_level);
      line 5: rho_out = 2 sum_i f_i psi_i^2 (Eq. density-construction);
      line 6: residual ||rho_out - rho_in||_w;
      line 7: rho_next by Anderson mixing of the density under
        <a, b> = sum a b w, from the history `mix` (a dict with lists 'x' and
        'f', updated in place; the last scf_history + 1 pairs are kept).
    Energy, gradient-free (Eq. total-energy-gradient-free), with the
    double-counting terms of rho_in (the density that built V_eff):
      E = 2 sum f_i eps_i - E_H + E_xc - <V_xc, rho_in> + E_ZZ.
    """
    pot = scf_potentials(tree, theta, degree, w, vext, rho_in, alpha=alpha)
    gi = green_iterate(tree, theta, degree, w, pot["veff"], vshift, psi, eps, tol_gi, max_iter, beta=gi_beta,
                       history=gi_history, mix_tol=mix_tol, store_output=gi_store_output)
    psi = gi["psi"] / np.sqrt(np.sum(gi["psi"] ** 2 * w[None, :], axis=1))[:, None]
    eps = gi["eps"]
    mu, f = fermi_level(eps, n_elec, kT)
    rho_out = 2.0 * np.sum(f[:, None] * psi**2, axis=0)
    resid = np.sqrt(np.sum((rho_out - rho_in) ** 2 * w))
    mix.setdefault("x", []).append(np.array(rho_in, np.float64))
    mix.setdefault("f", []).append(rho_out - rho_in)
    mix["x"] = mix["x"][-(scf_history + 1):]
    mix["f"] = mix["f"][-(scf_history + 1):]
    rho_next = anderson_mix(np.array(mix["x"]), np.array(mix["f"]), scf_beta, w)
    e_band = 2.0 * np.sum(f * eps)
    energy = {"band": e_band, "hartree": pot["e_h"], "xc": pot["e_xc"], "vxc": pot["e_vxc"], "zz": e_zz,
              "total": e_band - pot["e_h"] + pot["e_xc"] - pot["e_vxc"] + e_zz}
    return {"psi": psi, "eps": eps, "mu": mu, "occ": f, "rho_out": rho_out, "rho_next": rho_next, "resid": resid,
            "energy": energy, "gi": gi, "vh": pot["vh"], "veff": pot["veff"]}

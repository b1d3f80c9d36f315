"""Pins of the oracle's treecode (Section 5, Algorithm 3).

References: the direct sum (theta = 0 and the size rule reduce Algorithm 3 to
it), the defining properties of the tree (Section 5.1) and of the interaction
lists (every source reached exactly once per batch, MAC of Eq. MAC on every
approximated pair), polynomial reproduction of Lagrange interpolation for the
proxy weights (Eq. particle-cluster-approx-rearranged), and the error trend
in theta and n of Section 5.4.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2003_01833_gb300 import workloads as W


def _center_radius(lo, hi):
    return (lo + hi) * 0.5, math.sqrt(float(np.sum((hi - lo) ** 2))) * 0.5


@pytest.fixture(scope="module")
def cube():
    xyz, w = W.random_cube(6000, seed=11)
    return xyz, w, oracle.Tree(xyz, 150)


@pytest.fixture(scope="module")
def limesh():
    wl = W.lithium(seed=1, tol_m=1e-3)
    return wl, oracle.Tree(wl.mesh.xyz, 2000)


@pytest.mark.parametrize("which", ["cube", "limesh"])
def test_tree_structure(which, request):
    obj = request.getfixturevalue(which)
    T = obj[2] if which == "cube" else obj[1]
    xyz = T.xyz
    assert T.begin[0] == 0 and T.end[0] == T.n and T.parent[0] == -1
    assert sorted(T.idx.tolist()) == list(range(T.n))
    for c in range(T.nc):
        pts = T.points(c)
        # shrunk to the minimal bounding box of its points
        np.testing.assert_array_equal(T.lo[c], xyz[:, pts].min(1))
        np.testing.assert_array_equal(T.hi[c], xyz[:, pts].max(1))
        if T.nchild[c] == 0:
            assert len(pts) <= T.leaf_size
            continue
        assert len(pts) > T.leaf_size and T.nchild[c] >= 2
        ch = T.child[c, : T.nchild[c]]
        assert sorted(np.concatenate([T.points(q) for q in ch]).tolist()) == sorted(pts.tolist())
        ext = T.hi[c] - T.lo[c]
        mid = (T.lo[c] + T.hi[c]) * 0.5
        split = ext * math.sqrt(2.0) >= ext.max()
        assert split[np.argmax(ext)]
        for q in ch:
            assert T.parent[q] == c and T.level[q] == T.level[c] + 1
            side = xyz[:, T.points(q)] >= mid[:, None]
            for d in range(3):
                if split[d]:
                    assert np.all(side[d]) or not np.any(side[d])


@pytest.mark.parametrize("theta,degree", [(0.5, 4), (0.7, 6), (0.9, 3)])
def test_lists_cover_every_source_once_and_respect_mac(cube, theta, degree):
    xyz, w, T = cube
    b, c, k = T.lists(theta, degree)
    P = (degree + 1) ** 3
    for batch in T.leaves:
        sel = b == batch
        cnt = np.zeros(T.n, np.int64)
        for cl in c[sel]:
            cnt[T.points(cl)] += 1
        assert np.all(cnt == 1)
        cb, rb = _center_radius(T.lo[batch], T.hi[batch])
        for cl, kind in zip(c[sel], k[sel]):
            cc, rc = _center_radius(T.lo[cl], T.hi[cl])
            R = math.sqrt(float(np.sum((cb - cc) ** 2)))
            ok_theta = (rb + rc) / R < theta if R > 0 else False
            ns = T.end[cl] - T.begin[cl]
            if kind == 1:
                assert ok_theta and P < ns
            else:
                assert (not ok_theta and T.nchild[cl] == 0) or (ok_theta and P >= ns)
            # every ancestor was opened because it failed the theta test
            a = T.parent[cl]
            while a >= 0:
                ca, ra = _center_radius(T.lo[a], T.hi[a])
                Ra = math.sqrt(float(np.sum((cb - ca) ** 2)))
                assert not (Ra > 0 and (rb + ra) / Ra < theta)
                a = T.parent[a]


def test_theta_zero_is_direct_sum(cube):
    xyz, w, T = cube
    f = np.sin(xyz[0] * 3) + xyz[1] ** 2
    for kern, par in ((0, 1.7), (1, 1.0)):
        tc = T.treecode(0.0, 5, kern, par, f, w)
        ds = oracle.direct_yukawa(xyz, w, f, par) if kern == 0 else oracle.direct_coulomb(xyz, w, f, par)
        np.testing.assert_allclose(tc, ds, rtol=1e-12, atol=1e-14 * np.abs(ds).max())


def test_size_rule_makes_everything_direct():
    """(n+1)^3 >= N_S for every cluster: Algorithm 3 never approximates."""
    xyz, w = W.random_cube(700, seed=12)
    T = oracle.Tree(xyz, 40)
    f = np.cos(2 * xyz[2])
    b, c, k = T.lists(0.9, 8)
    assert not np.any(k == 1)
    np.testing.assert_allclose(T.treecode(0.9, 8, 0, 2.0, f, w), oracle.direct_yukawa(xyz, w, f, 2.0),
                               rtol=1e-12)


def test_anterpolation_reproduces_polynomials(cube):
    """Lagrange interpolation of degree n reproduces every monomial of degree
    <= n per dimension, so sum_k s_k^m qh_k = sum_j x_j^m q_j; m = 0 gives
    partition of unity (sum_k wh_k = sum_j w_j)."""
    xyz, w, T = cube
    n = 5
    q = np.vstack([w, w * np.cos(xyz[0])])
    for c in (0, 3, int(T.leaves[2])):
        qh = T.anterpolate(c, n, q)
        s = T.proxies(c, n)
        pts = T.points(c)
        for (a, bb, cc) in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (5, 0, 0), (3, 4, 5), (5, 5, 5)]:
            lhs = qh @ (s[0] ** a * s[1] ** bb * s[2] ** cc)
            x = xyz[:, pts]
            rhs = q[:, pts] @ (x[0] ** a * x[1] ** bb * x[2] ** cc)
            np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-13)


def test_proxy_nodes_are_chebyshev_second_kind(cube):
    xyz, w, T = cube
    n = 4
    s = T.proxies(0, n)
    node = np.cos(np.pi * np.arange(n + 1) / n)
    lo, hi = T.lo[0], T.hi[0]
    for d in range(3):
        vals = np.unique(s[d])
        np.testing.assert_allclose(np.sort(vals), np.sort((lo[d] + hi[d]) / 2 + (hi[d] - lo[d]) / 2 * node),
                                   rtol=0, atol=1e-15)


def test_error_trend_in_theta_and_degree():
    """Section 5.4: the approximation error falls as n grows and as theta
    shrinks (Fig. treecode-approx-error)."""
    xyz, w = W.random_cube(12000, seed=13)
    T = oracle.Tree(xyz, 300)
    f = 1.0 + 0.5 * np.sin(2 * xyz[0]) * np.cos(xyz[1])
    ds = oracle.direct_coulomb(xyz, w, f)

    def err(theta, n):
        return np.linalg.norm(T.treecode(theta, n, 1, 1.0, f, w) - ds) / np.linalg.norm(ds)

    e_n = [err(0.7, n) for n in (2, 4, 6)]
    e_t = [err(t, 4) for t in (0.4, 0.6, 0.8)]
    assert e_n[0] > e_n[1] > e_n[2]
    assert e_t[0] < e_t[1] < e_t[2]
    assert e_n[2] < 1e-5


def test_hydrogen_treecode_close_to_direct():
    wl = W.hydrogen_1s(seed=0)
    T = oracle.Tree(wl.mesh.xyz, 2000)
    u = oracle.treecode_yukawa(T, 0.7, 6, wl.f[0], 1.0, wl.mesh.w)
    ds = oracle.direct_yukawa(wl.mesh.xyz, wl.mesh.w, wl.f[0], 1.0)
    assert np.linalg.norm(u - ds) / np.linalg.norm(ds) < 1e-6

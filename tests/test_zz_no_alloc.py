"""The allocation-free entry point tagi_yukawa_direct_noalloc.

Some callers cannot let a library call cudaMalloc: host frameworks that hand
out every device byte from their own pool, and latency-critical loops that
cannot take an allocation's implicit device synchronisation.  This entry
point serves them with a fixed-size scratch array built into the library.
Here it is called through the C ABI twice in a row and each result is checked
against the existing entry point tagi_yukawa_conv on a theta = 0 float64 tree
(the same direct sum), to float64 rounding; a case large enough to use fewer
source slices, and the largest size the scratch array accepts (checked on
sampled targets against the oracle's direct sum), follow.  The file is named
so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2003_01833_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def test_noalloc_matches_yukawa_conv_twice(T):
    n = 3001
    xyz, w = W.random_cube(n, seed=31)
    rng = np.random.default_rng(5)
    cases = [(np.stack([1.0 + np.sin(2 * xyz[0] + o) * xyz[1] for o in range(3)]), [0.9, 2.5, 6.0]),
             (np.stack([np.cos(xyz[2] - o) for o in range(2)]), [1.3, 3.1])]
    dx, dw = dev(xyz), dev(w)
    with T.Tree(dx, dw, theta=0.0, degree=3, leaf_size=200, prec=T.TAGI_FP64) as tr:
        for f, k in cases:
            ref = torch.empty((len(k), n), dtype=torch.float64, device="cuda")
            T.tagi_yukawa_conv(tr.handle, dev(f), k, ref)
            u = torch.full((len(k), n), np.nan, dtype=torch.float64, device="cuda")
            T.tagi_yukawa_direct_noalloc(dx, dw, dev(f), k, u)
            torch.cuda.synchronize()
            a, b = u.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.abs(a - b).max() <= TOL * np.abs(b).max()


def test_noalloc_fewer_source_slices(T):
    # n * nf = 160000 values: 8 slices would need 1.28M scratch values, so the
    # call splits the sources into 6 slices
    n, nf = 40000, 4
    xyz, w = W.random_cube(n, seed=33)
    f = np.stack([1.0 + 0.5 * np.sin(3 * xyz[0] - o) * np.cos(xyz[1] + o) for o in range(nf)])
    k = [0.7, 1.9, 3.3, 5.0]
    dx, dw, df = dev(xyz), dev(w), dev(f)
    with T.Tree(dx, dw, theta=0.0, degree=3, leaf_size=2000, prec=T.TAGI_FP64) as tr:
        ref = torch.empty((nf, n), dtype=torch.float64, device="cuda")
        T.tagi_yukawa_conv(tr.handle, df, k, ref)
    u = torch.full((nf, n), np.nan, dtype=torch.float64, device="cuda")
    T.tagi_yukawa_direct_noalloc(dx, dw, df, k, u)
    torch.cuda.synchronize()
    a, b = u.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert np.abs(a - b).max() <= TOL * np.abs(b).max()


def test_noalloc_largest_accepted_size(T):
    import oracle

    # n * nf = 2^20, the whole scratch array in one source slice, with the
    # largest field count (the cheapest way to fill it: O(n^2 nf) work)
    n, nf = 1 << 16, 16
    xyz, w = W.random_cube(n, seed=35)
    f = np.stack([np.cos(2 * xyz[2] + 0.3 * o) + 0.2 * xyz[0] for o in range(nf)])
    k = [0.6 + 0.5 * o for o in range(nf)]
    u = torch.full((nf, n), np.nan, dtype=torch.float64, device="cuda")
    T.tagi_yukawa_direct_noalloc(dev(xyz), dev(w), dev(f), k, u)
    torch.cuda.synchronize()
    a = u.cpu().numpy()
    assert np.all(np.isfinite(a))
    pick = np.random.default_rng(3).choice(n, size=96, replace=False)
    for o in range(nf):
        ref = oracle.direct_yukawa(xyz, w, f[o], k[o], targets=pick)
        # sums of 65536 terms in two different orders
        assert np.abs(a[o, pick] - ref).max() <= 10 * TOL * np.abs(ref).max()


def test_noalloc_rejects_sizes_beyond_its_scratch(T):
    n = 300000
    dx = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    dw = torch.ones(n, dtype=torch.float64, device="cuda")
    f = torch.ones((4, n), dtype=torch.float64, device="cuda")
    u = torch.empty_like(f)
    with pytest.raises(T.TagiError) as e:
        T.tagi_yukawa_direct_noalloc(dx, dw, f, [1.0] * 4, u)
    assert e.value.status == T.TAGI_ERR_INVALID_ARG
    assert "scratch" in T.tagi_last_error()

"""The batch-split Green step on one GPU (tagi_tree_batches,
tagi_fields_conv_batches, tagi_green_conv_batches, tagi_green_reduce).

Processes are emulated one after another on the same GPU: each computes its
own batches' convolutions into its own zero-filled buffers, the buffers are
summed (each target is nonzero in exactly one), and the reductions run on
the full fields.  The orbitals, eigenvalues, residuals and E_H must equal
tagi_green_step's bit for bit, since every target's sums come from the same
work items in the same order.  No kernel waits on another process."""
import numpy as np
import pytest

from paper_2003_01833_gb300 import shard
from paper_2003_01833_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec_name", ["TAGI_FP32C", "TAGI_FP64"])
def test_batch_costs_and_field_subsets(T, prec_name):
    xyz, w = W.random_cube(15013, seed=8)
    rng = np.random.default_rng(2)
    f = np.stack([1.0 + 0.3 * np.sin(2 * xyz[0] + o) for o in range(3)])
    rho = np.exp(-np.sum(xyz**2, axis=0))
    k = [0.9, 2.1, 3.3]
    with T.Tree(dev(xyz), dev(w), theta=0.7, degree=6, leaf_size=400, prec=getattr(T, prec_name)) as tr:
        info = tr.info()
        size, cost = T.tagi_tree_batches(tr.handle)
        assert size.sum() == xyz.shape[1] and size.size == info["n_leaves"]
        assert cost.sum() == info["near_pairs"] + info["far_pairs"]
        u_ref = torch.empty((3, xyz.shape[1]), dtype=torch.float64, device="cuda")
        v_ref = torch.empty(xyz.shape[1], dtype=torch.float64, device="cuda")
        T.tagi_fields_conv(tr.handle, dev(f), k, u_ref, rho=dev(rho), vh=v_ref)
        for world in (2, 3):
            u = torch.zeros_like(u_ref)
            v = torch.zeros_like(v_ref)
            for r in range(world):
                mine = shard.own_batches(cost, world, r)
                ur, vr = torch.zeros_like(u), torch.zeros_like(v)
                T.tagi_fields_conv_batches(tr.handle, dev(f), k, ur, mine, rho=dev(rho), vh=vr)
                u += ur
                v += vr
            assert torch.equal(u, u_ref) and torch.equal(v, v_ref)
        # an empty share writes nothing
        ur = torch.full_like(u_ref, 7.0)
        T.tagi_fields_conv_batches(tr.handle, dev(f), k, ur, [], rho=None, vh=None)
        assert torch.all(ur == 7.0)
        with pytest.raises(T.TagiError):
            T.tagi_fields_conv_batches(tr.handle, dev(f), k, ur, [0, 0])
        with pytest.raises(T.TagiError):
            T.tagi_fields_conv_batches(tr.handle, dev(f), k, ur, [info["n_leaves"]])


def test_sharded_green_step_equals_one_gpu_lithium(T):
    wl = W.lithium(seed=1, tol_m=1e-3)
    m = wl.mesh
    n = wl.n
    with T.Tree(dev(m.xyz), dev(m.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=T.TAGI_FP32C) as tr:
        psi_ref = dev(wl.psi)
        vh_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        e_ref, r_ref, h_ref = T.tagi_green_step(tr.handle, dev(wl.veff), wl.vshift, psi_ref, wl.eps, rho=dev(wl.rho),
                                                vh=vh_ref)
        _, cost = T.tagi_tree_batches(tr.handle)
        world = 2
        psi = dev(wl.psi)
        u = torch.zeros_like(psi)
        vh = torch.zeros(n, dtype=torch.float64, device="cuda")
        for r in range(world):
            ur, vr = torch.zeros_like(psi), torch.zeros(n, dtype=torch.float64, device="cuda")
            T.tagi_green_conv_batches(tr.handle, dev(wl.veff), wl.vshift, psi, wl.eps, ur,
                                      shard.own_batches(cost, world, r), rho=dev(wl.rho), vh=vr)
            u += ur
            vh += vr
        e, res, h = T.tagi_green_reduce(tr.handle, dev(wl.veff), wl.vshift, psi, wl.eps, u, rho=dev(wl.rho), vh=vh)
        assert torch.equal(vh, vh_ref)
        assert torch.equal(psi, psi_ref)
        assert np.array_equal(e, e_ref) and np.array_equal(res, r_ref) and h == h_ref
        # one process: the same call sequence through shard.green_step_sharded
        psi1 = dev(wl.psi)
        vh1 = torch.empty(n, dtype=torch.float64, device="cuda")
        e1, r1, h1 = shard.green_step_sharded(T, tr.handle, dev(wl.veff), wl.vshift, psi1, wl.eps, rho=dev(wl.rho),
                                              vh=vh1)
        assert torch.equal(psi1, psi_ref) and np.array_equal(e1, e_ref) and h1 == h_ref

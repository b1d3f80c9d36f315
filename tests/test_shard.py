"""The Green step shared out over processes by target batches
(paper_2003_01833_gb300/shard.py), host logic on CPU.

- The assignment covers every batch once, is deterministic and balances the
  interaction counts (greedy longest-first: no process exceeds the mean by
  more than the largest batch).
- World size 2 over gloo: each process computes the oracle treecode for its
  own batches only (zero elsewhere), the fields are reassembled with one
  all-reduce, and the result equals the single-process treecode over all
  batches bit for bit, for a Yukawa and a Coulomb field."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_01833_gb300 import shard
from paper_2003_01833_gb300 import workloads as W


def test_partition_covers_and_balances():
    rng = np.random.default_rng(4)
    cost = rng.integers(1, 10**6, size=437)
    for world in (1, 2, 3, 8):
        owner = shard.partition_batches(cost, world)
        assert owner.shape == cost.shape and set(np.unique(owner)) <= set(range(world))
        assert np.array_equal(owner, shard.partition_batches(cost, world))
        loads = np.bincount(owner, weights=cost, minlength=world)
        assert loads.sum() == cost.sum()
        assert loads.max() <= cost.sum() / world + cost.max()
        mine = [shard.own_batches(cost, world, r) for r in range(world)]
        assert np.array_equal(np.sort(np.concatenate(mine)), np.arange(cost.size))
    assert np.all(shard.partition_batches(cost, 1) == 0)
    with pytest.raises(ValueError):
        shard.partition_batches(cost, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    xyz, w = W.random_cube(6007, seed=12)
    f = 1.0 + 0.4 * np.sin(2 * xyz[0]) * np.cos(xyz[1] - xyz[2])
    rho = np.exp(-np.sum(xyz**2, axis=0))
    return xyz, w, f, rho


def _batch_costs(ot, theta, degree):
    b, c, k = ot.lists(theta, degree)
    P = (degree + 1) ** 3
    size = ot.end - ot.begin
    per = {}
    for bb, cc, kk in zip(b, c, k):
        per[bb] = per.get(bb, 0) + (P if kk == 1 else int(size[cc]))
    leaves = list(ot.leaves)
    return leaves, np.array([per[x] * int(size[x]) for x in leaves], dtype=np.int64)


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xyz, w, f, rho = _case()
    ot = oracle.Tree(xyz, 300)
    leaves, cost = _batch_costs(ot, 0.7, 5)
    mine = shard.own_batches(cost, world, rank)
    pick = [leaves[i] for i in mine]
    u = torch.tensor(ot.treecode_batches(0.7, 5, 0, 1.7, f, w, pick))
    v = torch.tensor(ot.treecode_batches(0.7, 5, 1, 1.0, rho, w, pick))
    shard.gather_fields([u, v], lambda t: dist.all_reduce(t))
    out[rank] = (u.numpy().tobytes(), v.numpy().tobytes(), len(mine))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_fields_equal_single_process_gloo_world2():
    import torch.multiprocessing as mp

    import oracle

    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    xyz, w, f, rho = _case()
    ot = oracle.Tree(xyz, 300)
    u_ref = ot.treecode(0.7, 5, 0, 1.7, f, w)
    v_ref = ot.treecode(0.7, 5, 1, 1.0, rho, w)
    for r in (0, 1):
        assert out[r][2] > 0
        assert np.frombuffer(out[r][0]).tobytes() == u_ref.tobytes()
        assert np.frombuffer(out[r][1]).tobytes() == v_ref.tobytes()

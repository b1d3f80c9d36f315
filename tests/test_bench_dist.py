"""Multi-rank logic of bench.py on CPU: world size 2 over gloo.  Each rank
reports its own step time and interaction count; the job takes the slowest
rank's time and the sum of interactions (replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0, 12.5][rank]
    inter = [1e11, 3e11][rank]
    t, tot = bench.combine_ranks(ms, inter, world, torch.device("cpu"))
    out[rank] = (t, tot)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    import torch.multiprocessing as mp

    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (12.5, 4e11)


def test_combine_ranks_single():
    import bench

    assert bench.combine_ranks(3.0, 7.0, 1, None) == (3.0, 7.0)

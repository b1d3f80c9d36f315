"""The Green step shared out over processes, one per GPU, by target batches.

Once the tree, the interaction lists and the proxy weights exist, the target
batches are independent (Section 5.5); the paper's multi-GPU runs give each
GPU a share of them (Section 5.6).  Here every process builds the same tree
from the same inputs (the build is deterministic), forms and anterpolates all
fields (replicated: about 1% of a step), and computes the convolutions of its
own batches with tagi_green_conv_batches.  The batches are assigned by their
interaction counts (longest first, each to the least loaded process), so every
process gets about the same share of the near/far kernel.  Each target is
written by exactly one process, so a sum over processes of the zero-padded
results (one all-reduce) reassembles the fields bit for bit; every process
then applies the reductions (tagi_green_reduce) to the same full fields and
obtains the same orbitals and eigenvalues as tagi_green_step on one GPU.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_batches(cost, world: int) -> np.ndarray:
    """Owner process of each batch: batches in decreasing cost (ties by
    index) go to the process with the least total cost so far (ties by
    rank).  Deterministic, so every process computes the same assignment."""
    cost = np.asarray(cost, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    owner = np.empty(cost.size, dtype=np.int64)
    heap = [(0, r) for r in range(world)]
    for b in sorted(range(cost.size), key=lambda i: (-int(cost[i]), i)):
        load, r = heapq.heappop(heap)
        owner[b] = r
        heapq.heappush(heap, (load + int(cost[b]), r))
    return owner


def own_batches(cost, world: int, rank: int) -> np.ndarray:
    return np.nonzero(partition_batches(cost, world) == rank)[0].astype(np.int32)


def gather_fields(bufs, allreduce):
    """Reassemble zero-padded per-process fields: each target is nonzero on
    one process only, so the sum over processes equals it exactly."""
    for b in bufs:
        allreduce(b)
    return bufs


def green_step_sharded(T, tree, veff, vshift, psi, eps, rho=None, vh=None, group=None):
    """One Green step (tagi_green_step's result) computed by all processes of
    `group` together: psi (nw, n) float64 CUDA, updated in place on every
    process; eps host floats.  Returns (eps_new, resid, eh)."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    _, cost = T.tagi_tree_batches(tree)
    mine = own_batches(cost, world, rank)
    u = torch.zeros_like(psi)
    if rho is not None:
        vh.zero_()
    T.tagi_green_conv_batches(tree, veff, vshift, psi, eps, u, mine, rho=rho, vh=vh)
    if world > 1:
        gather_fields([u] + ([vh] if rho is not None else []), lambda t: dist.all_reduce(t, group=group))
    return T.tagi_green_reduce(tree, veff, vshift, psi, eps, u, rho=rho, vh=vh)

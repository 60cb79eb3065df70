"""Multi-GPU partition of a rod batch (one process per GPU).

Rods are independent, so the batch shards by rods with no exchange during a rollout:
``partition_rods`` assigns rods to ranks greedily by element count (longest first, to the
least-loaded rank), which bounds the imbalance by one rod.  The only collectives are
outside the data path: the max over ranks of a timing, and, for material parameters
shared by rods on several ranks, the sum of their gradients.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_rods(n_nodes, world: int) -> list[list[int]]:
    """Greedy longest-processing-time partition of rods (by node count) over ``world``
    ranks.  Returns one sorted list of rod indices per rank."""
    n_nodes = np.asarray(n_nodes)
    order = np.argsort(-n_nodes, kind="stable")
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + int(n_nodes[i]), r))
    return [sorted(p) for p in parts]


def shard(n_nodes, rank: int, world: int) -> list[int]:
    return partition_rods(n_nodes, world)[rank]


def max_over_ranks(value: float, device="cpu") -> float:
    """Max of a per-rank scalar (timings are reported as the slowest rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def allreduce_shared_gradient(grad):
    """In-place sum over ranks of the gradient of a parameter shared by rods on several
    ranks (e.g. one material stiffness for the whole batch)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    return grad

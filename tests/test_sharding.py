"""Multi-rank logic of the batched path on CPU ranks (gloo, world size 2)."""
import os
import socket

import numpy as np
import pytest

from paper_2509_04277_gb300 import sharding, workloads as W


def test_partition_covers_every_rod_once_and_balances():
    ns = W.batched_lengths()
    for world in (1, 2, 3, 4, 8):
        parts = sharding.partition_rods(ns, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ns)))
        loads = [int(ns[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= ns.max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns = W.batched_lengths()
        mine = sharding.shard(ns, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t_max = sharding.max_over_ranks(1.0 + rank)
        total = sharding.sum_over_ranks(float(ns[mine].sum()))
        g = torch.full((4,), float(rank + 1))
        sharding.allreduce_shared_gradient(g)
        q.put((rank, gathered, t_max, total, g.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_shard_without_overlap_and_reduce():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ns = W.batched_lengths()
    for rank, gathered, t_max, total, g in results:
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(len(ns)))
        assert t_max == 2.0
        assert total == float(ns.sum())
        assert g == [3.0, 3.0, 3.0, 3.0]

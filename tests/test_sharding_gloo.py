"""Multi-GPU host logic on CPU: the batch shards across ranks by problem (no data-path collective); ranks
partition with the package's greedy N^3 balance (paper_2402_11868_gb300.shard, which bench.py uses under
torchrun) and gather per-problem results for reporting.  Runs two gloo ranks on the CPU."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch.multiprocessing as mp


def shard(ns, world):
    from paper_2402_11868_gb300.shard import shard_by_cost
    return shard_by_cost(ns, world)


def _worker(rank, world, port, ns, out_q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    owner, _ = shard(ns, world)
    mine = [b for b in range(len(ns)) if owner[b] == rank]
    # stand-in for the per-rank result of the hot path: eigenpairs processed per problem
    local = torch.zeros(len(ns), dtype=torch.int64)
    for b in mine:
        local[b] = ns[b]
    gathered = [torch.zeros_like(local) for _ in range(world)]
    dist.all_gather(gathered, local)            # result gather for reporting only
    t = torch.tensor([float(len(mine))])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)    # max-over-ranks timing pattern of bench.py
    if rank == 0:
        out_q.put((sum(g for g in gathered).tolist(), float(t.item())))
    dist.destroy_process_group()


def test_shard_balance_and_coverage():
    import workloads as W
    from paper_2402_11868_gb300.shard import my_share
    ns = W.batch_sizes(1)
    for world in (1, 2, 4, 8):
        owner, loads = shard(ns, world)
        assert sorted(set(owner)) == list(range(world))
        assert max(loads) <= 1.1 * sum(loads) / world + max(n ** 3 for n in ns)
        shares = [my_share(ns, world, r) for r in range(world)]
        assert sorted(b for sh in shares for b in sh) == list(range(len(ns)))
    # the greedy rule on a hand example: 4^3 to rank 0, 3^3 to rank 1, then 2^3 and 2^3 to rank 1
    owner, loads = shard([2, 4, 3, 2], 2)
    assert owner == [1, 0, 1, 1] and loads == [64, 43]


def test_two_gloo_ranks_cover_every_problem_once():
    import workloads as W
    ns = W.batch_sizes(1, count=64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    import socket
    with socket.socket() as sk:                 # a port that is free now (the ranks bind it right after)
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ns, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, _ = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert total == ns                          # each problem processed by exactly one rank

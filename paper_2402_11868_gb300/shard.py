"""Sharding of a batch of eigenproblems across GPUs (one process per GPU).

The problems of a batch are independent, so a multi-GPU job needs no data-path collective: each rank takes a
share of the problems, solves it on its own GPU, and only the results (or their counts) are gathered for
reporting.  The shares are balanced by the cost law of the hot path -- the FP64 Jacobi sweeps and the
refinement's products are both O(N^3) per problem -- with the greedy longest-processing-time rule: problems
in decreasing N^3, each to the currently least loaded rank.  Host-side only."""
from __future__ import annotations


def shard_by_cost(ns, world: int):
    """(owner, loads): owner[b] in [0, world) for every problem order ns[b], and each rank's total N^3.
    Ties in load go to the lowest rank; equal orders keep their input order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    owner = [0] * len(ns)
    for b in sorted(range(len(ns)), key=lambda b: (-int(ns[b]) ** 3, b)):
        r = min(range(world), key=lambda q: (loads[q], q))
        owner[b] = r
        loads[r] += int(ns[b]) ** 3
    return owner, loads


def my_share(ns, world: int, rank: int):
    """Indices of the problems rank `rank` solves."""
    owner, _ = shard_by_cost(ns, world)
    return [b for b in range(len(ns)) if owner[b] == rank]

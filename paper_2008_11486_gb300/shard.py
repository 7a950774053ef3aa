"""Sharding frame sets over ranks (one process per GPU).

Frame sets are independent problems, so a multi-GPU run needs no exchange on
the data path: each rank reduces a disjoint subset of the sets.  Subsets are
balanced by cost (frames x pixels) with the longest-processing-time rule.
"""
from __future__ import annotations

import heapq


def set_cost(n: int, W: int, H: int) -> int:
    return int(n) * int(W) * int(H)


def shard_sets(costs, world: int):
    """Partitions set indices into ``world`` lists, greedily assigning the
    costliest remaining set to the least-loaded rank.  Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(o) for o in out]


def rank_shard(costs, world: int, rank: int):
    return shard_sets(costs, world)[rank]

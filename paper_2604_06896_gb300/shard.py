"""Sharding independent tissues over ranks (one process per GPU).

Batched workloads are independent tissues: no step of the method exchanges
data between tissues, so the ranks need no collective while they solve.
Tissues are dealt by longest-processing-time first (cell count as the cost):
largest tissue to the currently least-loaded rank, ties to the lower rank,
which is deterministic and within 4/3 of the optimal makespan.  After the
solve, rank 0 gathers the per-tissue results (host objects) in the original
tissue order.
"""
from __future__ import annotations

import heapq


def lpt_shards(sizes, world):
    """Tissue indices of each rank, each list in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-sizes[k], k))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + sizes[k], r))
    return [sorted(x) for x in out]


def gather_results(local, shard, n_total, dist=None):
    """Per-tissue results of this rank (list aligned with `shard`) gathered
    to rank 0 in tissue order; other ranks get None.  Without a process
    group the local results are returned in order."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        out = [None] * n_total
        for k, r in zip(shard, local):
            out[k] = r
        return out
    world = dist.get_world_size()
    box = [None] * world
    dist.all_gather_object(box, list(zip(shard, local)))
    if dist.get_rank() != 0:
        return None
    out = [None] * n_total
    for part in box:
        for k, r in part:
            if out[k] is not None:
                raise RuntimeError(f"tissue {k} solved by two ranks")
            out[k] = r
    if any(r is None for r in out):
        raise RuntimeError("a tissue was not solved by any rank")
    return out

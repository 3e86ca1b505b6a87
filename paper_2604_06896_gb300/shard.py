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


def minimize_batched_sharded(vx, meshes, params, opts, dtype="f32", dist=None, device="cuda"):
    """Relax independent tissues sharded over the ranks of `dist` (each rank
    on its own GPU; without a process group, all on this one): the rank's
    LPT share of `meshes` becomes one vx.Batch relaxed in one launch by
    vx.vx_minimize_batched, then rank 0 gathers (MinResult, X*) per tissue
    in the original order (other ranks get None).  params: per-tissue dicts
    with scalar KA, KP, A0, P0 and a per-edge (or scalar) lam; opts: the
    minimiser options.  No collective runs during the solves."""
    import numpy as np
    import torch
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    sizes = [int(np.asarray(m["face_he"]).shape[0]) for m in meshes]
    shard = lpt_shards(sizes, world)[rank]
    local = []
    if shard:
        b = vx.Batch([meshes[k] for k in shard], dtype)
        X = torch.tensor(np.concatenate([np.asarray(meshes[k]["vert"]) for k in shard]),
                         dtype=torch.float64, device=device)
        per = lambda key: np.array([float(params[k][key]) for k in shard])
        lam = [np.broadcast_to(np.asarray(params[k]["lam"], dtype=np.float64), (3 * sizes[k],))
               for k in shard]
        prm = dict(KA=per("KA"), KP=per("KP"), A0=per("A0"), P0=per("P0"),
                   lam=torch.tensor(np.concatenate(lam), dtype=torch.float64, device=device))
        rs = vx.vx_minimize_batched(b, X, prm, **opts)
        Xs = b.split(X.cpu().numpy())
        b.close()
        local = list(zip(rs, Xs))
    return gather_results(local, shard, len(meshes), dist)

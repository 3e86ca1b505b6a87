"""Tissue sharding over ranks: LPT balance and a world-size-2 gloo run on
CPU whose gathered results equal the single-process results (the solve is
a stand-in host function; no GPU is involved)."""
import importlib.util
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location(
    "vx_shard", os.path.join(ROOT, "paper_2604_06896_gb300", "shard.py"))
shard = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(shard)

import vx_inputs as vi  # noqa: E402


def sizes_c3(count=64):
    return [t["n"] for t in vi.batch_c3(count)]


def test_lpt_covers_each_tissue_once_and_balances():
    sizes = sizes_c3()
    for world in (1, 2, 4, 8):
        parts = shard.lpt_shards(sizes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        assert max(loads) <= sum(sizes) / world + max(sizes)


def fake_solve(k, n):
    return {"tissue": k, "value": 3 * n + k}


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.lpt_shards(sizes, world)[rank]
    local = [fake_solve(k, sizes[k]) for k in mine]
    out = shard.gather_results(local, mine, len(sizes), dist)
    if rank == 0:
        q.put(out)
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.timeout(120)
def test_gloo_world2_gather_matches_single_process():
    sizes = sizes_c3(24)
    ref = shard.gather_results([fake_solve(k, n) for k, n in enumerate(sizes)],
                               list(range(len(sizes))), len(sizes))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = q.get(timeout=100)
    for p in procs:
        p.join(timeout=100)
        assert p.exitcode == 0
    assert out == ref


class FakeBatch:
    """Host stand-in for vx.Batch (sizes and split only)."""

    def __init__(self, meshes, dtype):
        self.V = [2 * len(m["face_he"]) for m in meshes]

    def split(self, X):
        out, o = [], 0
        for v in self.V:
            out.append(X[o:o + v])
            o += v
        return out

    def close(self):
        pass


class FakeVx:
    """Host stand-in for the library: a deterministic per-tissue update."""
    Batch = FakeBatch

    @staticmethod
    def vx_minimize_batched(b, X, prm, **opts):
        rs, o = [], 0
        for k, v in enumerate(b.V):
            X[o:o + v] += float(prm["P0"][k]) + float(prm["lam"][(o // 2) * 3])
            rs.append((v, float(prm["P0"][k])))
            o += v
        return rs


def fake_tissues(count=10):
    import numpy as np
    sizes = [5 + (7 * k) % 11 for k in range(count)]
    meshes = [dict(face_he=np.arange(n), vert=np.arange(4 * n, dtype=float).reshape(2 * n, 2))
              for n in sizes]
    params = [dict(KA=1.0, KP=1.0, A0=1.0, P0=0.1 * k, lam=0.01 * k) for k in range(count)]
    return meshes, params


def _worker_sharded(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    meshes, params = fake_tissues()
    out = shard.minimize_batched_sharded(FakeVx, meshes, params, dict(tol=1e-6), dist=dist,
                                         device="cpu")
    if rank == 0:
        q.put(out)
    else:
        assert out is None
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_gloo_world2_batched_minimiser_shards_match_single_process():
    """minimize_batched_sharded on two gloo ranks (each relaxing its LPT
    share as one batch) gathers the same per-tissue results and positions on
    rank 0 as one process relaxing every tissue."""
    import numpy as np
    meshes, params = fake_tissues()
    ref = shard.minimize_batched_sharded(FakeVx, meshes, params, dict(tol=1e-6), device="cpu")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker_sharded, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = q.get(timeout=100)
    for p in procs:
        p.join(timeout=100)
        assert p.exitcode == 0
    assert len(out) == len(ref)
    for (r1, x1), (r2, x2) in zip(out, ref):
        assert r1 == r2
        assert np.array_equal(x1, x2)

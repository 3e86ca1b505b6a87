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

"""Benchmark: vertex-force evaluations per second of the minimiser on the
10,000-cell periodic Voronoi tissue (FP32 arithmetic with hi/lo positions,
FP64 reductions), relaxed by FIRE with T1 transitions to max|F| < 1e-6
sqrt(A0), target shape index swept over {3.5, 3.7, 3.9}.

One step = the three relaxations (one per p0), each from the Voronoi
initial state and topology.  value = sum over relaxations of V x force
evaluations / device time.  The same workload through the plain GPU path
(one launch per sub-step, host-polled convergence) is reported beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vx|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import vx_inputs as vi  # noqa: E402

METRIC = "vertex-force evals/s & equilibrium-gradient solves/s vs plain GPU path at tol"
UNIT = "vertex-force evals/s"
WORKLOAD = ("c2: 10,000-cell periodic Voronoi tissue (20,000 vertices), FP32 hi/lo positions, "
            "FIRE+T1, p0 in {3.5,3.7,3.9}, tolerance 1e-6*sqrt(A0) with a 20,000-iteration budget "
            "per relaxation (the tolerance is not reached: short edges keep being stretched)")
MODULI = ("dimensionless moduli: K_A = 1/A0, K_P = 1, P0 = p0*sqrt(A0), Lambda = 0.05*sqrt(A0), "
          "A0 = 1e-4, box 1 x 1")


# DRAM bytes (read + write) of one launch of the dominant kernel, from an
# ncu capture of the current kernel (None until the changed kernel is
# captured again)
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the c2 kernel
# (ncu capture of 300 iterations; the traffic is the one-off load of the
# tissues' state into L2 and does not grow with the iteration count)
TRAFFIC_BYTES = 10_977_024
MAX_ITER = 20_000   # per relaxation: a fixed budget (the tolerance is not reached)


def opts_for(A0, path):
    sA = math.sqrt(A0)
    return dict(tol=1e-6 * sA, max_iter=MAX_ITER, dt0=0.01, dt_max=0.5, l_min=5e-3 * sA,
                path=path, check_every=100)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------------- reference

def cpu_sample(seconds=12.0):
    """The oracle (numpy FP64, one thread) on the same tissue: FIRE + T1
    iterations from the Voronoi state for about `seconds`."""
    from oracle import mesh as omesh
    from oracle import solvers as osolv
    c = vi.tissue_c2(3.7)
    t = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    o = opts_for(c["A0"], 0)
    mo = osolv.MinOpts(tol=o["tol"], max_iter=5, dt0=o["dt0"], dt_max=o["dt_max"])
    t0 = time.perf_counter()
    r = osolv.relax(t["vert"], t, p, mo, l_min=o["l_min"])
    per = (time.perf_counter() - t0) / (r.iters + 1)
    iters = max(5, int(seconds / per))
    mo.max_iter = iters
    t0 = time.perf_counter()
    r = osolv.relax(t["vert"], t, p, mo, l_min=o["l_min"])
    dt = time.perf_counter() - t0
    V = t["vert"].shape[0]
    evals = r.iters + 1
    return dict(value=V * evals / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"{evals} FIRE+T1 iterations (force evaluations) of the 10,000-cell "
                       f"p0=3.7 tissue from its Voronoi state, numpy FP64, {dt:.1f} s")


_ORACLE_WORKER = {}


def _oracle_init(counter):
    """Pool initializer: each host process takes the next p0 of the sweep
    and builds the oracle's mesh of that tissue once."""
    from oracle import mesh as omesh
    with counter.get_lock():
        idx = counter.value
        counter.value += 1
    c = vi.tissue_c2(vi.C2_P0_SWEEP[idx % 3])
    _ORACLE_WORKER["tissue"] = (c, omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"]))


def _oracle_worker(seconds):
    """One host process of the all-cores oracle sample: FIRE + T1 on its
    10,000-cell tissue from the Voronoi state for about `seconds` (at least
    one iteration; the time per iteration is calibrated once per process)."""
    from oracle import solvers as osolv
    c, t = _ORACLE_WORKER["tissue"]
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    o = opts_for(c["A0"], 0)
    mo = osolv.MinOpts(tol=o["tol"], max_iter=2, dt0=o["dt0"], dt_max=o["dt_max"])
    if "per" not in _ORACLE_WORKER:
        t0 = time.perf_counter()
        r = osolv.relax(t["vert"], t, p, mo, l_min=o["l_min"])
        _ORACLE_WORKER["per"] = (time.perf_counter() - t0) / (r.iters + 1)
    mo.max_iter = max(1, int(seconds / _ORACLE_WORKER["per"]))
    t0 = time.perf_counter()
    r = osolv.relax(t["vert"], t, p, mo, l_min=o["l_min"])
    return t["vert"].shape[0], r.iters + 1, time.perf_counter() - t0


def oracle_pool():
    """One spawned host process per core, each holding its tissue."""
    import multiprocessing as mp
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    return ctx.Pool(cores, initializer=_oracle_init, initargs=(ctx.Value("i", 0),)), cores


def cpu_sample_all_cores(seconds=15.0, pool=None):
    """The oracle on every host core at once: one process per core, each
    relaxing the 10,000-cell tissue of one p0 (3.5, 3.7, 3.9 in turn) for
    about `seconds`; value = sum of V x force evaluations / the longest
    process time.  Processes are spawned (none is forked from a CUDA
    process)."""
    own = pool is None
    if own:
        pool, cores = oracle_pool()
    else:
        cores = pool._processes
    try:
        res = pool.map(_oracle_worker, [seconds] * cores, chunksize=1)
    finally:
        if own:
            pool.close()
            pool.join()
    evals = sum(v * e for v, e, _ in res)
    wall = max(d for _, _, d in res)
    return dict(value=evals / wall, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{cores} processes, each {min(e for _, e, _ in res)}-"
                       f"{max(e for _, e, _ in res)} FIRE+T1 iterations of the 10,000-cell tissue "
                       f"from its Voronoi state (p0 = 3.5, 3.7, 3.9 in turn), numpy FP64, "
                       f"{wall:.1f} s")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(3.0, 40.0 / max(1, args.steps))
    pool, _ = oracle_pool()
    with pool:
        for _ in range(args.warmup):
            cpu_sample_all_cores(seconds=1.0, pool=pool)
        vals = []
        t_all = time.perf_counter()
        for _ in range(args.steps):
            s = cpu_sample_all_cores(seconds=per_step, pool=pool)
            vals.append(s["value"])
        wall = time.perf_counter() - t_all
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded CPU sample on every host core)",
                       "moduli": MODULI},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------- GPU

def algorithmic_bytes_per_iter(n):
    """Algorithmic bytes of one FIRE iteration of an n-cell tissue with
    uniform tension and uniform per-cell parameters, FP32 positions: one
    energy + force evaluation reads X (16 n: 2 n vertices x 8 B), writes F
    (16 n) and reads the cell cycles (24 n: 6 n packed corner words); the
    FIRE step reads and writes v (32 n) and writes X (16 n); the lo halves
    of the hi/lo positions add 16 n to each of the two X streams:
    56 n + 48 n + 32 n = 136 n."""
    return 136 * n


def grad_metric(vx, torch, steps, warmup):
    """Equilibrium-gradient solves/s on the 1,000-cell parameter-inference
    tissue (FP32): one solve = relax from the target equilibrium under the
    trial tensions in FP32 to max|F| < 1e-5 sqrt(A0) (FP32 arithmetic
    stalls near 1.5e-6 on this tissue), continue in FP64 arithmetic to
    max|F| < 1e-8 sqrt(A0) (refine_tol), then the adjoint gradient of the
    v2v cost with respect to the 3,000 tensions (FP32, CG to rtol 1e-6).  The persistent path (automatic choice:
    a 16-CTA cluster) against the plain path (one launch per sub-step for
    both the minimiser and the CG), same inputs and tolerances, CUDA events
    around each solve."""
    c = vi.tissue_c4()
    mesh = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    base = dict(KA=c["KA"], KP=c["KP"], A0=c["A0"], P0=c["P0"])
    sA = math.sqrt(c["A0"])
    t0 = vx.Tissue(mesh, "f32")
    Xt = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    vx.vx_minimize(t0, Xt, dict(base, lam=c["lam_hidden"]), **opts_for(c["A0"], "auto"))
    top = t0.topology()
    top["vert"] = Xt.cpu().numpy()
    t0.close()
    t = vx.Tissue(top, "f32")     # created at the target's topology: restore returns to it
    X = torch.empty_like(Xt)
    p = dict(base, lam=c["lam"])
    out = {}
    for path in ("auto", "plain"):
        o = opts_for(c["A0"], path)
        o["tol"], o["refine_tol"], o["max_iter"] = 1e-8 * sA, 1e-5 * sA, 100_000

        def solve():
            vx.vx_tissue_restore(t)
            X.copy_(Xt)
            r = vx.vx_minimize(t, X, p, **o)
            g, rg = vx.vx_equilibrium_grad(t, X, p, cost=vx.VX_COST_V2V, cost_data=Xt,
                                           cg_rtol=1e-6, inner=dict(path=path))
            return r, rg, g

        for _ in range(warmup):
            solve()
        torch.cuda.synchronize()
        ms, rs = 0.0, []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            rs.append(solve())
            b.record()
            b.synchronize()
            ms += a.elapsed_time(b)
        r, rg, g = rs[-1]
        if path == "auto":
            # what the oracle check needs (the last solve's state)
            check = dict(X=X.cpu().numpy(), top=t.topology(), g=g["lam"].cpu().numpy(),
                         Xt=Xt.cpu().numpy(), p=p, fmax=r.fmax)
        out[path] = {"value": steps / (ms * 1e-3), "ms_per_solve": ms / steps,
                     "path": {1: "resident", 2: "plain", 3: "cluster", 4: "grid"}.get(r.path_used),
                     "min_status": r.status, "min_iters": r.iters, "n_t1": r.n_t1,
                     "fmax": r.fmax, "cg_status": rg.status, "cg_iters": rg.cg_iters,
                     "cg_rel_residual": rg.cg_rel_residual}
    t.close()
    return {"metric": "equilibrium-gradient solves/s", "unit": "solves/s",
            "workload": "c4: 1,000-cell tissue, 3,000 tension parameters, v2v cost; relax "
                        "from the target equilibrium in FP32 to max|F|<1e-5*sqrt(A0), then in "
                        "FP64 to 1e-8*sqrt(A0), then the FP32 adjoint (CG to rtol 1e-6)",
            "value": out["auto"]["value"], "vs_plain_gpu_path": out["auto"]["value"] / out["plain"]["value"],
            "persistent": out["auto"], "plain_gpu_path": out["plain"]}, check


def c4_oracle_errors(check):
    """The oracle at the GPU's c4 result: its dense adjoint gradient at the
    GPU's equilibrium and topology (the FP32 adjoint's error), and its
    max |F| there (how far the GPU's equilibrium is from force balance)."""
    from oracle import model as omodel
    from oracle import solvers as osolv
    top = dict(check["top"], vert=check["X"])
    _, G = omodel.cost_v2v(check["X"], check["Xt"], top)
    g_ref, _, info = osolv.adjoint_grad(check["X"], top, check["p"], G)
    F = omodel.forces(check["X"], top, check["p"])
    d = check["g"] - g_ref["lam"]
    return {"adjoint_rel_error": float(np.linalg.norm(d) / np.linalg.norm(g_ref["lam"])),
            "oracle_fmax_at_X": float(np.sqrt((F * F).sum(axis=1)).max()),
            "gpu_fmax": check["fmax"], "hessian_pd": bool(info["pd"]),
            "note": "oracle dense adjoint at the GPU's equilibrium and topology; the "
                    "end-to-end error of the GPU pipeline against the oracle's own FP64 "
                    "pipeline is measured by tests/test_gpu_c4.py"}


def status_counts(results):
    """How many tissues ended with each vx_status (0 converged, 1 out of
    budget, higher an error), keyed by the status name."""
    names = {0: "ok", 1: "not_converged", 4: "cuda", 8: "nonfinite", 9: "topology"}
    out = {}
    for r in results:
        k = names.get(int(r.status), str(int(r.status)))
        out[k] = out.get(k, 0) + 1
    return out


def batched_forward_metric(vx, torch, steps, subset_every=32, max_iter=20_000, compare=True,
                           dist=None):
    """The batched forward workload: 512 periodic Voronoi tissues of
    log-uniform size in [200, 5000] cells (7.5e5 cells in all), per-tissue
    p0 ~ U(3.5, 4.0), per-edge Lambda ~ U(0, 0.1), FP32, FIRE + T1 to
    max|F| < 1e-6 with a budget of max_iter iterations, in one persistent
    graph-replayed launch (vx_minimize_batched).  Vertex-force evals/s
    (L2 flushed before each timed step).  The plain GPU path (one launch per
    sub-step, one tissue at a time) is too slow for the whole batch; it is
    compared with the batched path on every subset_every-th tissue (the same
    inputs and options for both).  With a process group of N ranks the
    tissues are dealt by LPT (shard.lpt_shards), each rank relaxes its share
    as one batch on its GPU, and the value is the evaluations of all ranks
    over the slowest rank's time (no collective inside the timed region)."""
    batch = vi.batch_c3()
    meshes = [vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"]) for c in batch]
    kw = dict(tol=1e-6, max_iter=max_iter, dt0=0.01, dt_max=0.5, l_min=5e-3)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def run_batched(idx, nsteps):
        b = vx.Batch([meshes[k] for k in idx], "f32")
        X0 = torch.tensor(np.concatenate([meshes[k]["vert"] for k in idx]), dtype=torch.float64,
                          device="cuda")
        lam = torch.tensor(np.concatenate([batch[k]["lam"] for k in idx]), device="cuda")
        prm = dict(KA=1.0, KP=1.0, A0=1.0, P0=np.array([batch[k]["P0"] for k in idx]), lam=lam)
        X = X0.clone()
        vx.vx_minimize_batched(b, X, prm, **kw)      # capture + warm-up
        ms, evals, rs = 0.0, 0, None
        for _ in range(nsteps):
            vx.vx_batch_restore(b)
            X.copy_(X0)
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rs = vx.vx_minimize_batched(b, X, prm, **kw)
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            evals += sum(int(b.V[k]) * r.force_evals for k, r in enumerate(rs))
        b.close()
        return evals / (ms * 1e-3), ms / nsteps, rs

    allidx = list(range(len(batch)))
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    if world > 1:
        from paper_2604_06896_gb300 import shard
        mine = shard.lpt_shards([c["n"] for c in batch], world)[dist.get_rank()]
        value, ms_step, rs = run_batched(mine, steps)
        t = torch.tensor([ms_step, value * ms_step * 1e-3], dtype=torch.float64, device="cuda")
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        ev = t[1:].clone()
        dist.all_reduce(ev, op=dist.ReduceOp.SUM)
        return {"metric": "vertex-force evals/s", "value": ev.item() / (mx.item() * 1e-3),
                "ms_per_step": mx.item(), "ranks": world, "sharding": "LPT by cell count"}
    value, ms_step, rs = run_batched(allidx, steps)
    if not compare:
        return {"metric": "vertex-force evals/s", "value": value, "ms_per_step": ms_step,
                "converged": int(sum(r.status == 0 for r in rs)),
                "status_counts": status_counts(rs),
                "force_evals_per_tissue": [int(min(r.force_evals for r in rs)),
                                           int(max(r.force_evals for r in rs))]}
    sub = allidx[::subset_every]
    sub_value, sub_ms, _ = run_batched(sub, 1)
    plain_ms, plain_evals = 0.0, 0
    for k in sub:
        c = batch[k]
        t = vx.Tissue(meshes[k], "f32")
        X = torch.tensor(meshes[k]["vert"], dtype=torch.float64, device="cuda")
        p = dict(KA=1.0, KP=1.0, A0=1.0, P0=c["P0"], lam=c["lam"])
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = vx.vx_minimize(t, X, p, path="plain", check_every=100, **kw)
        e1.record()
        e1.synchronize()
        plain_ms += e0.elapsed_time(e1)
        plain_evals += t.V * r.force_evals
        t.close()
    plain_value = plain_evals / (plain_ms * 1e-3)
    ncells = sum(c["n"] for c in batch)
    return {"metric": "vertex-force evals/s", "unit": "vertex-force evals/s", "value": value,
            "ms_per_step": ms_step,
            "workload": f"c3: {len(batch)} tissues, {ncells} cells (log-uniform 200-5000 per tissue), "
                        f"p0 ~ U(3.5,4.0), Lambda ~ U(0,0.1), A0 = 1, FP32, FIRE+T1 to max|F|<1e-6, "
                        f"{max_iter}-iteration budget, one graph-replayed persistent launch",
            "converged": int(sum(r.status == 0 for r in rs)),
            "status_counts": status_counts(rs),
            "force_evals_per_tissue": [int(min(r.force_evals for r in rs)),
                                       int(max(r.force_evals for r in rs))],
            "subset": {"tissues": len(sub), "batched_value": sub_value, "batched_ms": sub_ms,
                       "plain_gpu_path_value": plain_value, "plain_gpu_path_ms": plain_ms,
                       "vs_plain_gpu_path": sub_value / plain_value}}


def batched_gradient_metric(vx, torch, free_iters=5000, plain_tissues=None, compare=True):
    """The batched inverse-design workload: 64 periodic Voronoi tissues of
    10,000 cells (box 100, A0 = 1 per cell, Lambda ~ U(0, 0.1) per edge,
    p0 = 3.7), FP32; one equilibrium-gradient solve = the free relaxation
    (FIRE + T1, max|F| < 1e-6 or a budget of free_iters iterations) then the
    adjoint gradient of the anisotropy cost (q_target = (0.1, 0)) with
    respect to the per-cell A0 and per-edge Lambda (CG to rtol 1e-6, FP64
    reductions).  Batched: every tissue in one graph-replayed persistent
    launch (vx_batch_grad).  Plain GPU path: one tissue at a time, one launch
    per sub-step for the relaxation and for the CG (host-polled), on the
    same inputs and options.  Solves/s = tissues / wall time (CUDA events)."""
    batch = vi.batch_c5()
    meshes = [vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"]) for c in batch]
    free = dict(tol=1e-6, max_iter=free_iters, dt0=0.01, dt_max=0.5, l_min=5e-3)
    qt = np.array([0.1, 0.0])
    b = vx.Batch(meshes, "f32")
    X0 = torch.tensor(np.concatenate([m["vert"] for m in meshes]), dtype=torch.float64,
                      device="cuda")
    lam = torch.tensor(np.concatenate([c["lam"] for c in batch]), device="cuda")
    A0 = torch.ones(int(b.n.sum()), dtype=torch.float64, device="cuda")
    prm = dict(KA=1.0, KP=1.0, A0=A0, P0=3.7, lam=lam)
    X = X0.clone()
    vx.vx_batch_grad(b, X, prm, vx.VX_COST_ANISO, qt, what=1, free=free, cg_rtol=1e-6)  # capture
    vx.vx_batch_restore(b)
    X.copy_(X0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ga, _, rs = vx.vx_batch_grad(b, X, prm, vx.VX_COST_ANISO, qt, what=1, free=free, cg_rtol=1e-6)
    e1.record()
    e1.synchronize()
    ms_b = e0.elapsed_time(e1)
    b.close()
    if not compare:
        return {"metric": "equilibrium-gradient solves/s", "value": len(batch) / (ms_b * 1e-3),
                "ms_per_batch": ms_b,
                "cg_iters": [int(min(r[1].cg_iters for r in rs)), int(max(r[1].cg_iters for r in rs))]}
    idx = list(range(len(batch))) if plain_tissues is None else list(range(plain_tissues))
    ms_p = 0.0
    for k in idx:
        c = batch[k]
        t = vx.Tissue(meshes[k], "f32")
        Xk = torch.tensor(meshes[k]["vert"], dtype=torch.float64, device="cuda")
        p = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=c["lam"])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        vx.vx_minimize(t, Xk, p, path="plain", check_every=100, **free)
        vx.vx_equilibrium_grad(t, Xk, p, cost=vx.VX_COST_ANISO, cost_data=qt, cg_rtol=1e-6,
                               inner=dict(path="plain", check_every=20))
        e1.record()
        e1.synchronize()
        ms_p += e0.elapsed_time(e1)
        t.close()
    v_b = len(batch) / (ms_b * 1e-3)
    v_p = len(idx) / (ms_p * 1e-3)
    return {"metric": "equilibrium-gradient solves/s", "unit": "solves/s", "value": v_b,
            "ms_per_batch": ms_b,
            "workload": f"c5: {len(batch)} tissues x 10,000 cells, FP32, FIRE+T1 to max|F|<1e-6 "
                        f"({free_iters}-iteration budget), anisotropy cost, adjoint gradient for "
                        f"per-cell A0 and per-edge Lambda (CG rtol 1e-6), one launch",
            "free_converged": int(sum(r[0].status == 0 for r in rs)),
            "free_status_counts": status_counts([r[0] for r in rs]),
            "cg_iters": [int(min(r[1].cg_iters for r in rs)), int(max(r[1].cg_iters for r in rs))],
            "plain_gpu_path": {"value": v_p, "tissues": len(idx), "ms": ms_p},
            "vs_plain_gpu_path": v_b / v_p}


def bulk_forces_metric(vx, torch, peak, n=1_000_000, steps=10):
    """Bulk energy + force evaluation (vx_energy_forces, FP32 tissue) of one
    periodic Voronoi tissue of n cells (box sqrt(n), seeds in Hilbert order,
    A0 = 1, p0 = 3.7, per-edge Lambda ~ U(0, 0.1)), L2 flushed before every
    timed call; vertex-force evals/s and the roofline against the measured
    HBM copy rate.  Algorithmic bytes per call (the call's own FP64
    interface): X read 32 n + F write 32 n + the cell cycles 24 n + the
    per-edge Lambda (3 n edges x 8 B) 24 n = 112 n."""
    seeds = vi.uniform_seeds(n, math.sqrt(n), math.sqrt(n), vi.substream(9, 0))
    L = math.sqrt(n)
    order = vx.vx_seed_order(seeds, L, L)
    mesh = vx.vx_build_mesh(seeds[order], L, L)
    t = vx.Tissue(mesh, "f32")
    lam = torch.tensor(vi.SplitMix64(10).uniform(t.E, 0.0, 0.1), device="cuda")
    p = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=lam)
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    F = torch.empty_like(X)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    prm, keep = vx.make_params(p, t.n, t.E)

    def call():
        st = vx.capi.vx_energy_forces(t.handle, X.data_ptr(), ctypes.byref(prm), F.data_ptr(),
                                      E.data_ptr(), torch.cuda.current_stream().cuda_stream)
        vx.capi.check(st, "vx_energy_forces")

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            call()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):    # one replay = one call, without host launch gaps
        call()
    ms = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    med = float(np.median(ms))
    achieved = 112.0 * n / (med * 1e-3) / 1e9
    out = {"metric": "vertex-force evals/s", "unit": "vertex-force evals/s",
           "value": t.V / (med * 1e-3), "ms_per_call": med,
           "workload": f"one {n}-cell periodic Voronoi tissue ({t.V} vertices), FP32 tissue, "
                       "per-edge Lambda, energy + forces per call (vx_energy_forces), L2 flushed "
                       f"(256 MiB write) before every call, median of {steps} graph-replayed calls",
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "bytes_per_call": "112 n",
                        "kernels": "k_ef_cells, k_ef_vertices, k_ef_sum"}}
    t.close()
    return out


def c2_oracle_errors(finals):
    """The oracle's energy and max |F| at each c2 relaxation's returned state
    (GPU energy relative error, GPU max |F| against the oracle's)."""
    from oracle import model as omodel
    out = []
    for p0, X, top, p, r in finals:
        t = dict(top, vert=X)
        E = omodel.energy(X, t, p)
        F = omodel.forces(X, t, p)
        out.append({"p0": p0, "energy_rel_error": abs(r.energy - E) / abs(E),
                    "oracle_fmax": float(np.sqrt((F * F).sum(axis=1)).max()), "gpu_fmax": r.fmax})
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2604_06896_gb300 as vx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cases = []
    for p0 in vi.C2_P0_SWEEP:
        c = vi.tissue_c2(p0)
        # the same seeds, labelled along a Hilbert curve: the same tissue with
        # spatially ordered cell / vertex / edge numbering (both paths)
        order = vx.vx_seed_order(c["seeds"], c["Lx"], c["Ly"])
        mesh = vx.vx_build_mesh(c["seeds"][order], c["Lx"], c["Ly"])
        p = dict(KA=c["KA"], KP=c["KP"], A0=c["A0"], P0=c["P0"], lam=0.05 * math.sqrt(c["A0"]))
        t = vx.Tissue(mesh, "f32")
        X0 = torch.tensor(mesh["vert"], dtype=torch.float64, device=dev)
        cases.append((c, mesh, p, t, X0, torch.empty_like(X0)))
    V = cases[0][3].V
    n = cases[0][3].n
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(path, stats=None):
        for c, mesh, p, t, X0, X in cases:
            vx.vx_tissue_restore(t)
            X.copy_(X0)
        if path == "plain":   # the reference GPU path: one tissue at a time
            rs = [vx.vx_minimize(t, X, p, **opts_for(c["A0"], path))
                  for c, mesh, p, t, X0, X in cases]
        else:                 # one persistent launch for the three relaxations
            rs = vx.vx_minimize_many([cs[3] for cs in cases], [cs[5] for cs in cases],
                                     [cs[2] for cs in cases], **opts_for(cases[0][0]["A0"], path))
        if stats is not None:
            stats.extend(rs)
        return sum(r.force_evals for r in rs)

    def timed(path, steps, warmup):
        for _ in range(warmup):
            step(path)
        total_ms, total_evals, stats = 0.0, 0, []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        # named range: ncu --nvtx --nvtx-include "timed_<path>/" lists the
        # launches of the timed steps only
        torch.cuda.nvtx.range_push(f"timed_{path}")
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            total_evals += step(path, stats)
            b.record()
            b.synchronize()
            total_ms += a.elapsed_time(b)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return total_ms, total_evals, stats

    with ClockSampler(local) as clk:
        ms, evals, stats = timed("auto", args.steps, args.warmup)
    path_used = stats[0].path_used
    ms_t = torch.tensor([ms], dtype=torch.float64, device=dev)
    ev_t = torch.tensor([evals], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(ev_t, op=dist.ReduceOp.SUM)
    value = V * ev_t.item() / (ms_t.item() * 1e-3)

    # the plain GPU path on the same inputs and tolerance (one step)
    pms, pevals, pstats = timed("plain", 1, 0)
    plain_value = V * pevals / (pms * 1e-3)

    # end to end through the public API with host buffers
    X0h = [torch.empty((V, 2), dtype=torch.float64, pin_memory=True) for _ in cases]
    Xh = [torch.empty((V, 2), dtype=torch.float64, pin_memory=True) for _ in cases]
    for k, cs in enumerate(cases):
        X0h[k].copy_(torch.from_numpy(cs[1]["vert"]))
    torch.cuda.synchronize()
    e_ms, e_evals = 0.0, 0
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        for k, (c, mesh, p, t, X0, X) in enumerate(cases):
            vx.vx_tissue_restore(t)
            X.copy_(X0h[k], non_blocking=True)
        rs = vx.vx_minimize_many([cs[3] for cs in cases], [cs[5] for cs in cases],
                                 [cs[2] for cs in cases], **opts_for(cases[0][0]["A0"], "auto"))
        for k, cs in enumerate(cases):
            Xh[k].copy_(cs[5], non_blocking=True)
        e_evals += sum(r.force_evals for r in rs)
        torch.cuda.synchronize()
        e_ms += 1e3 * (time.perf_counter() - t0)
    e2e = V * e_evals / (e_ms * 1e-3)
    if world > 1:
        t_ = torch.tensor([e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t_, op=dist.ReduceOp.SUM)
        e2e = t_.item()

    # roofline of the dominant kernel: the one persistent launch of a step,
    # event-timed on the launching stream
    for c, mesh, p, t, X0, X in cases:
        vx.vx_tissue_restore(t)
        X.copy_(X0)
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    rs = vx.vx_minimize_many([cs[3] for cs in cases], [cs[5] for cs in cases],
                             [cs[2] for cs in cases], **opts_for(cases[0][0]["A0"], "auto"))
    b.record()
    b.synchronize()
    k_ms = a.elapsed_time(b)
    bytes_alg = algorithmic_bytes_per_iter(n) * sum(r.force_evals for r in rs)
    achieved = bytes_alg / (k_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    # the returned state of each relaxation (for the oracle check)
    finals = [(p0, cs[5].cpu().numpy(), cs[3].topology(), cs[2], r)
              for p0, cs, r in zip(vi.C2_P0_SWEEP, cases, rs)]

    grad, grad_check = grad_metric(vx, torch, steps=max(1, args.steps), warmup=1)
    bulk = None if args.no_batch else bulk_forces_metric(vx, torch, peak, n=args.bulk_cells,
                                                         steps=args.bulk_steps)
    batched = None if args.no_batch else batched_forward_metric(
        vx, torch, steps=1, dist=dist if world > 1 else None)
    # one GPU only: the c5 line compares with the plain path tissue by tissue
    batched_grad = None if args.no_batch or world > 1 else batched_gradient_metric(vx, torch)

    # cpu_baseline leg: the oracle timed on the host cores, and the oracle
    # checked against this run's results
    cpu, oracle_errors = None, None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_sample_all_cores(seconds=15.0)
        cpu["single_core"] = cpu_sample(seconds=12.0)
        oracle_errors = {"c2": c2_oracle_errors(finals), "c4": c4_oracle_errors(grad_check)}

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    conv = [s.status == 0 for s in stats[:3]]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_t.item() / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "moduli": MODULI, "n_cells": n, "n_vertices": V,
                   "numbering": "seeds in Hilbert-curve order (vx_seed_order)",
                   "path": {1: "resident", 2: "plain", 3: "cluster"}.get(path_used, path_used),
                   "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "vs_plain_gpu_path": value / plain_value,
        "plain_gpu_path": {"value": plain_value, "unit": UNIT, "ms_per_step": pms},
        "relaxations": [{"p0": p0, "status": s.status, "iters": s.iters, "n_t1": s.n_t1,
                         "n_stretch": s.n_stretch, "fmax": s.fmax}
                        for p0, s in zip(vi.C2_P0_SWEEP, stats[:3])],
        "converged": conv,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * V * 16,
                "d2h_bytes_per_step": 3 * V * 16},
        # per step: one k_rebuild_flat per tissue (vx_tissue_restore), the one
        # persistent minimiser launch, and per tissue the exit-time wrap
        # (k_wrap_pos, k_wrap_tgt, k_rebuild_flat)
        "gpu_launches": args.steps * (len(cases) + 1 + 3 * len(cases)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_BYTES,
                     "kernel": "k_min_cluster_many (one persistent launch, one 16-CTA cluster per relaxation)",
                     "bytes_per_iteration": "136 n (n = 10,000 cells): evaluation 56 n + FIRE "
                                            "step 48 n + lo halves of the two X streams 32 n",
                     "note": "algorithmic bytes per iteration x iterations / launch time, against "
                             "the measured HBM copy rate (of measured); the tissue state (~2 MB "
                             "per relaxation) stays in L2 and the kernel is bound by L2 latency "
                             "and barriers, not by bandwidth; traffic = dram bytes read + written "
                             "per launch from one ncu capture (300 iterations: the one-off state "
                             "load, which does not grow with the iteration count)"},
        "equilibrium_gradient": grad,
        "bulk_forces": bulk,
        "batched_forward": batched,
        "batched_gradient": batched_grad,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "oracle_errors": oracle_errors,
    }
    print(json.dumps(line))


def run_profile(args):
    """Small fixed-size runs for ncu: the three 10,000-cell relaxations in
    one multi-tissue launch (capped iterations, on the path --path names),
    then continued from the state reached (few T1 events left), optionally
    one relaxation alone, the plain path on one of them (capped), and the
    100-cell FP64 tissue on the resident path (to convergence)."""
    import torch

    import paper_2604_06896_gb300 as vx
    ts, Xs, ps, meshes = [], [], [], []
    for p0 in vi.C2_P0_SWEEP:
        c = vi.tissue_c2(p0)
        order = vx.vx_seed_order(c["seeds"], c["Lx"], c["Ly"]) if args.ordered else np.arange(c["n"])
        mesh = vx.vx_build_mesh(c["seeds"][order], c["Lx"], c["Ly"])
        ps.append({k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")})
        ts.append(vx.Tissue(mesh, "f32"))
        meshes.append(mesh)
        Xs.append(None)
    A0 = vi.tissue_c2(3.7)["A0"]

    def reset():
        for k, t in enumerate(ts):
            vx.vx_tissue_restore(t)
            Xs[k] = torch.tensor(meshes[k]["vert"], dtype=torch.float64, device="cuda")

    def report(label, rs, dt):
        it = max(r.iters for r in rs)
        print(f"{label}: {[r.iters for r in rs]} iterations, {[r.n_t1 for r in rs]} T1, "
              f"{[r.n_stretch for r in rs]} stretches, fmax {[f'{r.fmax:.2e}' for r in rs]}, "
              f"status {[r.status for r in rs]} in {dt * 1e3:.1f} ms = "
              f"{dt / max(1, it) * 1e6:.2f} us/iteration", flush=True)

    o = opts_for(A0, args.path)
    o["max_iter"] = args.profile_iters
    for rep in range(2):   # the first call includes module loading
        reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs = vx.vx_minimize_many(ts, Xs, ps, **o)
        dt = time.perf_counter() - t0
    report(f"many ({args.path})", rs, dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs = vx.vx_minimize_many(ts, Xs, ps, **o)
    dt = time.perf_counter() - t0
    report(f"many ({args.path}, continued)", rs, dt)
    if args.profile_single:
        reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = vx.vx_minimize(ts[1], Xs[1], ps[1], **o)
        dt = time.perf_counter() - t0
        report(f"single ({args.path})", [r], dt)
    reset()
    o = opts_for(A0, "plain")
    o["max_iter"] = args.profile_iters // 10
    for rep in range(2):
        vx.vx_tissue_restore(ts[1])
        X = torch.tensor(meshes[1]["vert"], dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = vx.vx_minimize(ts[1], X, ps[1], **o)
        dt = time.perf_counter() - t0
    report("plain", [r], dt)
    c1 = vi.tissue_c1()
    m1 = vx.vx_build_mesh(c1["seeds"], c1["Lx"], c1["Ly"])
    p1 = {k: c1[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    t1 = vx.Tissue(m1, "f64")
    X1 = torch.tensor(m1["vert"], dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    r = vx.vx_minimize(t1, X1, p1, **opts_for(c1["A0"], "resident") | {"tol": 1e-8})
    dt = time.perf_counter() - t0
    report("resident c1", [r], dt)
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vx", choices=["vx", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched c3 / c5 lines and the bulk force line")
    ap.add_argument("--bulk-only", action="store_true",
                    help="only the bulk energy + force line (for ncu)")
    ap.add_argument("--bulk-cells", type=int, default=1_000_000)
    ap.add_argument("--c5-only", action="store_true",
                    help="only the batched gradient workload, without the plain-path comparison "
                         "(for a launch list)")
    ap.add_argument("--c3-only", action="store_true",
                    help="only the batched forward workload, without the plain-path comparison "
                         "(for a launch list)")
    ap.add_argument("--bulk-steps", type=int, default=10)
    ap.add_argument("--profile", action="store_true", help="small fixed runs for ncu")
    ap.add_argument("--profile-iters", type=int, default=2000)
    ap.add_argument("--ordered", type=int, default=1, help="profile: Hilbert-ordered seeds")
    ap.add_argument("--path", default="auto", help="profile: path of the multi-tissue launch")
    ap.add_argument("--profile-single", type=int, default=0,
                    help="profile: also one relaxation alone on --path")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.c5_only:
        import torch
        import paper_2604_06896_gb300 as vx
        print(json.dumps(batched_gradient_metric(vx, torch, compare=False)))
    elif args.c3_only:
        import torch
        import paper_2604_06896_gb300 as vx
        print(json.dumps(batched_forward_metric(vx, torch, steps=1, compare=False)))
    elif args.bulk_only:
        import torch
        import paper_2604_06896_gb300 as vx
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        print(json.dumps(bulk_forces_metric(vx, torch, peak, n=args.bulk_cells,
                                            steps=args.bulk_steps)))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

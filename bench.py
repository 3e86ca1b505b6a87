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
WORKLOAD = "c2: 10,000-cell periodic Voronoi tissue, FIRE+T1 to max|F|<1e-6*sqrt(A0), p0 in {3.5,3.7,3.9}"


# DRAM bytes (read + write) of one launch of the dominant kernel, from an
# ncu capture of the current kernel
TRAFFIC_BYTES = 10_277_120 + 105_472
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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        s = cpu_sample(seconds=max(5.0, 40.0 / max(1, args.steps)))
        vals.append(s["value"])
    wall = time.perf_counter() - t_all
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded CPU sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": s["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------- GPU

def algorithmic_bytes_per_iter(n):
    """Bytes one FIRE iteration must touch if every array were streamed once
    (FP32 path): positions hi/lo read + write (32 V), velocities read +
    write (16 V), half-edge target/next/face (12 HE), vertex out-lists (12 V),
    face starts (4 n), cell coefficients written and read (16 n)."""
    V, HE = 2 * n, 6 * n
    return 32 * V + 16 * V + 12 * HE + 12 * V + 4 * n + 16 * n


def grad_metric(vx, torch, steps, warmup):
    """Equilibrium-gradient solves/s on the 1,000-cell parameter-inference
    tissue (FP32): one solve = relax from the target equilibrium under the
    trial tensions to max|F| < 1e-5 sqrt(A0) (FP32 arithmetic stalls near
    1.5e-6 on this tissue), then the adjoint gradient of the v2v cost with
    respect to the 3,000 tensions.  The persistent path (automatic choice:
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
        o["tol"], o["max_iter"] = 1e-5 * sA, 100_000

        def solve():
            vx.vx_tissue_restore(t)
            X.copy_(Xt)
            r = vx.vx_minimize(t, X, p, **o)
            g, rg = vx.vx_equilibrium_grad(t, X, p, cost=vx.VX_COST_V2V, cost_data=Xt,
                                           cg_rtol=1e-6, inner=dict(path=path))
            return r, rg

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
        r, rg = rs[-1]
        out[path] = {"value": steps / (ms * 1e-3), "ms_per_solve": ms / steps,
                     "path": {1: "resident", 2: "plain", 3: "cluster", 4: "grid"}.get(r.path_used),
                     "min_status": r.status, "min_iters": r.iters, "n_t1": r.n_t1,
                     "fmax": r.fmax, "cg_status": rg.status, "cg_iters": rg.cg_iters,
                     "cg_rel_residual": rg.cg_rel_residual}
    t.close()
    return {"metric": "equilibrium-gradient solves/s", "unit": "solves/s",
            "workload": "c4: 1,000-cell tissue, 3,000 tension parameters, v2v cost; relax to "
                        "max|F|<1e-5*sqrt(A0) from the target equilibrium, then the adjoint "
                        "(CG to rtol 1e-6)",
            "value": out["auto"]["value"], "vs_plain_gpu_path": out["auto"]["value"] / out["plain"]["value"],
            "persistent": out["auto"], "plain_gpu_path": out["plain"]}


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

    grad = grad_metric(vx, torch, steps=max(1, args.steps), warmup=1)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_sample(seconds=12.0)

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    conv = [s.status == 0 for s in stats[:3]]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_t.item() / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_cells": n, "n_vertices": V,
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
        # per step: one k_rebuild_flat per tissue (vx_tissue_restore) and the
        # one persistent minimiser launch
        "gpu_launches": args.steps * (len(cases) + 1),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_BYTES,
                     "kernel": "k_min_cluster_many (one persistent launch, one 16-CTA cluster per relaxation)",
                     "note": "algorithmic bytes/iteration x iterations / launch time; the "
                             "tissue state lives in L2, peak is the measured HBM copy rate; "
                             "traffic = dram bytes read+written by one ncu capture of this "
                             "kernel (300 iterations of the same three tissues): the state "
                             "is loaded into L2 once, so it does not grow with iterations "
                             "(profiles/k_min_cluster_many_c2.md)"},
        "equilibrium_gradient": grad,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
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
    ap.add_argument("--profile", action="store_true", help="small fixed runs for ncu")
    ap.add_argument("--profile-iters", type=int, default=2000)
    ap.add_argument("--ordered", type=int, default=1, help="profile: Hilbert-ordered seeds")
    ap.add_argument("--path", default="auto", help="profile: path of the multi-tissue launch")
    ap.add_argument("--profile-single", type=int, default=0,
                    help="profile: also one relaxation alone on --path")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

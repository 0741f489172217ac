#!/usr/bin/env python
"""Throughput of the ghost-cell immersed-boundary fractional step on GB300.

Workload (default): the 3D finite-wing case - NACA0012 section, chord 1,
aspect ratio 2, square tips, 15 degrees incidence, ~20k-triangle surface,
stretched 384x256x256 grid (25.2M cells), Re 1000, dt 0.002, Poisson solved
to a 1e-10 relative residual - in FP64, with the mixed-precision Poisson
path measured on the same state beside it. Inputs are synthetic (seeded
generators); every field is resident in HBM during the timed steps, and the
25.2M-cell FP64 fields (201 MB each) exceed the 129 MB L2, so no L2 flush is
needed between steps.

One bench "step" = one fractional step of the whole grid (predictor,
Poisson solve, projection, ghost refresh) through ibm_step.

Multi-GPU: the solver does not shard across GPUs (one grid per GPU); with
N > 1 every rank runs an independent replica of the workload ("replicas
only"), value = cells * steps * N / max-over-ranks time.

--impl reference times the CPU oracle (the plain FP64 reference of the
method) on a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware work queues, so the independent cases of the ensemble and
# serving legs (one stream each) run concurrently; read at CUDA context creation
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "Mcell-steps/s per GB300, mixed vs FP64 at 1e-10 residual; serve p50/p99 latency"
UNIT = "Mcell-steps/s"

# DRAM traffic of one finest-level FP64 colour pass on the 384x256x256 wing,
# from an ncu capture of the 256x192x192 case (512.9 MB per launch) scaled by
# the cell count; valid for the kernel as captured
RBGS64_TRAFFIC_BYTES = 512.93e6 * 25165824 / 9437184

# algorithmic bytes per cell of one launch of the timed kernels
# (FP64 s = 8, FP32 s = 4, cell type 1 byte); see the design notes
def rbgs_pass_bytes(ncells, s, stored_coeffs=True):
    # one colour pass: read all x (neighbours), read f and write x for half
    # the cells, plus the operator: stored face coefficients (3 arrays) and
    # the diagonal of the updated half
    b = ncells * s * (1.0 + 0.5 + 0.5)
    if stored_coeffs:
        b += ncells * s * (3.0 + 0.5)
    return b


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--size", default="384,256,256", help="nx,ny,nz of the wing grid")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-kernels", action="store_true", help="also report every timed kernel")
    ap.add_argument("--no-ktimer", action="store_true", help="skip the per-kernel timing pass")
    ap.add_argument("--serve", type=int, default=40,
                    help="requests of the 3D multi-sphere serving stream to replay (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=4, help="cases resident at once in the serving leg")
    ap.add_argument("--serve-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--compare", default="192,128,128",
                    help="wing grid of the Poisson solver comparison ('' to skip)")
    ap.add_argument("--ellipsoids", type=int, default=0,
                    help="steps of the 208M-cell ellipsoid array to time per precision (0: skip)")
    ap.add_argument("--ensemble", type=int, default=64,
                    help="cases of the seeded 2D ensemble to run, 50 steps each (0: skip)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="arithmetic of the main timed run (the mixed run beside it is --no-mixed's)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, world: int) -> float:
    """Max of a per-rank scalar over all ranks (replicas: each rank times its
    own grid; the job is as slow as its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job Mcell-steps/s of `world` independent replicas."""
    return cells * steps * world / (max_ms / 1e3) / 1e6


class Clocks:
    """nvidia-smi sampler during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ibm_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def wing_case(size):
    from paper_2505_17287_gb300 import synth
    nx, ny, nz = (int(x) for x in size.split(","))
    return synth.wing_case(nx, ny, nz)


def run_reference(args):
    """CPU oracle on a bounded sample of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from oracle import flow, geom
    from paper_2505_17287_gb300 import synth
    case = synth.wing_case(32, 24, 24)
    cores = 1
    T = geom.body_tables(3, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(3, case.xf, case.yf, case.zf)
    # one bench step = one bounded sample: a fractional step of the oracle
    # from the impulsive start, its matrix factorisations included
    for _ in range(args.warmup):
        flow.run(g, T["type"], T, 1, case.Re, case.dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flow.run(g, T["type"], T, 1, case.Re, case.dt)
    el = time.perf_counter() - t0
    val = g.N * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "wing NACA0012 AR2 15deg, oracle sample 32x24x24",
                                            "full_workload": "384x256x256 stretched, Re 1000, dt 0.002"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "plain FP64 oracle (sparse direct solves), wing case on a 32x24x24 grid "
                                       "(18,432 cells); each bench step is one fractional step from the "
                                       "impulsive start, matrix factorisations included"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    from oracle import flow, geom
    from paper_2505_17287_gb300 import synth
    case = synth.wing_case(32, 24, 24)
    T = geom.body_tables(3, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(3, case.xf, case.yf, case.zf)
    t0 = time.perf_counter()
    flow.run(g, T["type"], T, 2, case.Re, case.dt)
    dt = time.perf_counter() - t0
    return {"value": g.N * 2 / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "plain FP64 oracle (sparse direct solves), wing case on a 32x24x24 grid (18,432 cells), "
                      "one run of 2 fractional steps including the matrix factorisations"}


def serve_leg(nreq, slots, precision):
    """Replay the first nreq requests of the seeded 3D multi-sphere stream
    (Poisson arrivals at 50/s, 1-8 icospheres of 5120 triangles, n^3 grids
    with n in [64, 256], 10 steps each) against the request loop in real
    time; latency = completion - arrival."""
    import numpy as np
    from paper_2505_17287_gb300 import ibm, synth
    times, cases = synth.serve_stream(nreq)
    srv = ibm.Server(max_slots=slots)
    t0 = time.perf_counter()
    ids = []
    for t, c in zip(times, cases):
        d = t - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        ids.append(srv.submit(c, precision=precision))
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    ok = [r for r in res if r["status"] == ibm.IBM_OK]
    lat = np.array([r["t_done"] - r["t_submit"] for r in ok]) * 1e3
    svc = np.array([r["t_done"] - r["t_admit"] for r in ok]) * 1e3
    first = min(r["t_submit"] for r in res)
    last = max(r["t_done"] for r in res)
    work = sum(r["cells"] * r["steps"] for r in ok)
    return {"requests": nreq, "completed_ok": len(ok), "arrival_rate_per_s": 50.0, "slots": slots,
            "precision": "mixed" if precision == ibm.IBM_MIXED else "fp64",
            "p50_ms": float(np.percentile(lat, 50)) if len(ok) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(ok) else None,
            "service_p50_ms": float(np.percentile(svc, 50)) if len(ok) else None,
            "value": work / (last - first) / 1e6, "unit": UNIT,
            "completed_per_s": len(ok) / (last - first), "makespan_s": last - first,
            "cells_total": int(sum(r["cells"] for r in ok)), "peak_running": st["peak_running"],
            "peak_admitted_gb": st["peak_admitted_bytes"] / 1e9,
            "workload": "seeded stream: Poisson arrivals 50/s; 1-8 icospheres (5120 triangles each, radii "
                        "0.2-0.6) in [-4,8]x[-3,3]^2; n^3 grids, log n uniform in [log 64, log 256], n a "
                        "multiple of 16; Re 100-500; CFL 0.2; 10 steps per request; Poisson rtol 1e-10"}


def compare_leg(size):
    """Poisson solvers on the same right-hand side (the wing's second step
    on a smaller grid, from phi = 0, FP64, to a 1e-10 relative residual):
    the paper's BiCGStab with scheduled relaxation Jacobi, BiCGStab with the
    multigrid V-cycle, FGMRES with either."""
    import numpy as np
    import torch
    from paper_2505_17287_gb300 import ibm
    case = wing_case(size)
    s = ibm.Solver(case)
    s.set_body(case.verts, case.elems)
    s.classify()
    s.step(2)
    rhs = torch.from_numpy(s.get("rhs").ravel()).cuda()
    out = {"grid": size.replace(",", "x"), "cells": s.N, "rtol": 1e-10}
    for name, kw in (("fgmres_mg", dict(outer=ibm.IBM_OUTER_FGMRES, precond=0)),
                     ("bicgstab_mg", dict(outer=ibm.IBM_OUTER_BICGSTAB, precond=0)),
                     ("bicgstab_srj", dict(outer=ibm.IBM_OUTER_BICGSTAB, precond=1)),
                     ("fgmres_srj", dict(outer=ibm.IBM_OUTER_FGMRES, precond=1))):
        s.set_opts(**kw)
        phi = torch.zeros_like(rhs)
        torch.cuda.synchronize()
        st = s.poisson_solve(rhs, phi, rtol=1e-10, maxit=4000)
        out[name] = {"iterations": st["outer_iters"], "ms": st["ms"], "rel_residual": st["rel_residual"],
                     "status": ibm.STATUS_NAMES.get(st["status"], st["status"])}
    # the Crank-Nicolson Helmholtz step from the same state: red-black
    # Gauss-Seidel against scheduled relaxation Jacobi (sweeps over the three
    # components and predictor time of one step)
    s.set_opts(outer=ibm.IBM_OUTER_FGMRES, precond=0)
    state = s.get_state()
    for name, hs in (("helmholtz_rbgs", 0), ("helmholtz_srj", 1)):
        s.set_state(state)
        s.set_opts(helm_solver=hs)
        r = s.step(1)
        out[name] = {"sweeps": r["helm_sweeps"], "ms_predictor": r["ms_predictor"],
                     "status": ibm.STATUS_NAMES.get(r["status"], r["status"])}
    s.close()
    return out


def ellipsoid_leg(nsteps):
    """The 27-ellipsoid array on the 1300x400x400 grid (208M cells, the
    paper's particulate-array case), FP64 and mixed: per step and per
    Poisson outer iteration times after two warm-up steps."""
    import torch
    from paper_2505_17287_gb300 import ibm, synth
    case = synth.ellipsoid_array_case()
    out = {"grid": "1300x400x400", "cells": case.ncells, "bodies": case.meta["nbodies"],
           "triangles": case.meta["ntri"], "Re": case.Re, "dt": case.dt}
    for name, prec in (("mixed", ibm.IBM_MIXED), ("fp64", ibm.IBM_FP64)):
        s = ibm.Solver(case, precision=prec)
        s.set_opts(precision=prec)
        t0 = time.perf_counter()
        for v, e in synth.case_bodies(case):
            s.set_body(v, e)
        info = s.classify()
        setup = time.perf_counter() - t0
        s.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = s.step(nsteps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": case.ncells * nsteps / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / nsteps,
                     "poisson_outer_per_step": st["poisson_outer"] / nsteps,
                     "ms_per_poisson_iteration": st["ms_poisson"] / max(1, st["poisson_outer"]),
                     "ms_poisson_per_step": st["ms_poisson"] / nsteps, "rel_residual_last": st["rel_residual"],
                     "classify_s": setup, "n_ghost": info["n_ghost"], "status": st["status"]}
        s.close()
        torch.cuda.empty_cache()
    return out


def ensemble_leg(ncases):
    """The seeded 2D ensemble (ellipses and circles, grids 128x64 to
    1024x512, Re 50-200, CFL 0.2, 50 steps each) in mixed precision: options
    autotuned per size class, every case resident on its own stream with its
    step captured as device-controlled CUDA graphs, all steps enqueued at
    once; throughput = cell-steps / wall time of the steps."""
    from paper_2505_17287_gb300 import ensemble, ibm, synth
    cases = synth.ensemble_2d(ncases)
    t0 = time.perf_counter()
    tuned = ensemble.tune(cases, steps=2)
    tune_s = time.perf_counter() - t0
    out = ensemble.run_graphs(cases, tuned=tuned)
    return {"cases": ncases, "steps_each": 50, "ok": out["ok"], "value": out["mcell_steps_per_s"], "unit": UNIT,
            "wall_s": out["wall_s"], "cell_steps": out["cell_steps"], "setup_s": out["setup_s"], "tune_s": tune_s,
            "precision": "mixed", "path": "ibm_step_async of device-controlled step graphs (opts graph=2), one "
                                        "stream per case, all enqueued from one thread",
            "tuned": {str(k): ensemble.describe(v[0]) for k, v in sorted(tuned.items())},
            "max_rel_residual": max(r["rel_residual"] for r in out["results"]),
            "workload": "seeded 2D ensemble: 64 ellipse/circle bodies (semi-axes 0.3-1.0, angle 0-pi), "
                        "grids nx in [128, 1024] (multiple of 32) x nx/2 on [-8,24]x[-8,8], Re 50-200, "
                        "dt = 0.2 h, 50 steps, Poisson rtol 1e-10"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_17287_gb300 import build, ibm
    if rank == 0 or not os.path.exists(ibm.LIB_PATH):
        build.build()
    if world > 1:
        torch.distributed.barrier()
    case = wing_case(args.size)
    # the solver runs on its own stream (not the legacy default stream), so
    # its multigrid V-cycle is captured once and replayed as a CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    main_prec = ibm.IBM_MIXED if args.precision == "mixed" else ibm.IBM_FP64
    s = ibm.Solver(case, precision=main_prec)
    s.set_opts(precision=main_prec)
    t0 = time.perf_counter()
    s.set_body(case.verts, case.elems)
    info = s.classify()
    setup_s = time.perf_counter() - t0
    N = s.N

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def timed(nsteps, kernel_timer=False):
        if kernel_timer:
            ibm.ibm_kernel_timer(s.ctx, 1)
        sync_all()
        l0 = ibm.ibm_launch_count(s.ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = []
        for _ in range(nsteps):
            stats.append(s.step(1))
        e1.record(stream)
        sync_all()
        ms = e0.elapsed_time(e1)
        launches = ibm.ibm_launch_count(s.ctx) - l0
        kt = {}
        if kernel_timer:
            for name, kid in ibm.KERNEL_IDS.items():
                kt[name] = ibm.ibm_kernel_time(s.ctx, kid)
            ibm.ibm_kernel_timer(s.ctx, 0)
        ms = max_over_ranks(ms, world)
        return ms, stats, launches, kt

    for _ in range(args.warmup):
        s.step(1)
    saved = s.get_state() if not args.no_mixed else None
    with Clocks(local) as clk:
        ms, stats, launches, _ = timed(args.steps)
    clocks = clk.summary()
    value = replica_throughput(N, args.steps, world, ms)
    poisson_ms64 = sum(x["ms_poisson"] for x in stats)
    # roofline of the dominant kernel: a second pass over the same number of
    # steps with the event timer on (the timer adds host work per launch, so
    # the headline above is measured without it)
    if args.no_ktimer:
        ms_kt, kt = ms, {k: (0.0, 0) for k in ibm.KERNEL_IDS}
    else:
        ms_kt, stats_kt, _, kt = timed(args.steps, kernel_timer=True)
    rb_ms, rb_n = kt["rbgs0"]
    mixed_main = main_prec == ibm.IBM_MIXED
    # the finest-level FP32 pass derives its coefficients from the open-face
    # mask (one byte per cell) instead of reading stored ones
    rb_bytes = rbgs_pass_bytes(N, 4, stored_coeffs=False) + N * 1.0 if mixed_main else rbgs_pass_bytes(N, 8)
    achieved = rb_bytes / (rb_ms / rb_n / 1e3) / 1e9 if rb_n else None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed_main else "f64", "data": "synthetic",
        "config": {"workload": f"wing NACA0012 AR2 15deg, stretched {args.size.replace(',', 'x')} grid "
                               f"({N} cells), Re 1000, dt 0.002, Poisson rtol 1e-10, "
                               + ("mixed (FP32 multigrid cycles inside FP64 refinement)" if mixed_main else "FP64"),
                   "cells": N, "n_ghost": info["n_ghost"], "n_dead": info["n_dead"],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (no flush)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {"bound": "hbm", "kernel": ("k_rbgs<float, fine>" if mixed_main else "k_rbgs<double>")
                     + " (finest level, one colour pass)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": RBGS64_TRAFFIC_BYTES if args.size == "384,256,256" and main_prec == ibm.IBM_FP64 else None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback",
                     "launches": rb_n, "avg_ms": rb_ms / rb_n if rb_n else None,
                     "algorithmic_bytes_per_launch": rb_bytes},
        "stats": {"setup_s": setup_s, "poisson_outer_per_step": sum(x["poisson_outer"] for x in stats) / args.steps,
                  "poisson_inner_per_step": sum(x["poisson_inner"] for x in stats) / args.steps,
                  "helm_sweeps_per_step": sum(x["helm_sweeps"] for x in stats) / args.steps,
                  "rel_residual_last": stats[-1]["rel_residual"],
                  "ms_poisson_per_step": poisson_ms64 / args.steps,
                  "ms_predictor_per_step": sum(x["ms_predictor"] for x in stats) / args.steps},
    }
    if args.profile_kernels:
        result["kernels"] = {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items()}
        result["kernels_step_ms"] = ms_kt / args.steps
    if not args.no_mixed:
        s.set_state(saved)
        s.set_opts(precision=ibm.IBM_MIXED)
        ms_m, stats_m, _, _ = timed(args.steps)
        poisson_ms32 = sum(x["ms_poisson"] for x in stats_m)
        result["mixed"] = {"value": N * args.steps * world / (ms_m / 1e3) / 1e6, "unit": UNIT,
                           "ms_per_step": ms_m / args.steps,
                           "poisson_ms_per_step": poisson_ms32 / args.steps,
                           "poisson_speedup_vs_fp64": poisson_ms64 / poisson_ms32 if poisson_ms32 else None,
                           "step_speedup_vs_fp64": ms / ms_m,
                           "poisson_outer_per_step": sum(x["poisson_outer"] for x in stats_m) / args.steps,
                           "rel_residual_last": stats_m[-1]["rel_residual"],
                           "same_inputs": "both runs start from the same saved state"}
        s.set_opts(precision=ibm.IBM_FP64)
    if not args.no_e2e:
        # end to end through the C ABI with pinned host buffers: every step
        # copies its input state host->device, steps, and reads u, v, w, p back
        names_in = ["u", "v", "w", "p", "p_prev", "p_prev2", "face_u", "face_v", "face_w", "nold_u", "nold_v", "nold_w"]
        names_out = ["u", "v", "w", "p"]
        st = s.get_state()
        host_in = {k: torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in names_in}
        host_out = {k: torch.empty(host_in[k].shape, dtype=torch.float64).pin_memory() for k in names_out}
        h2d = sum(t.numel() * 8 for t in host_in.values()) + 8
        d2h = sum(t.numel() * 8 for t in host_out.values())
        ne2e = max(1, min(args.steps, 5))
        sync_all()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            for k in names_in:
                ibm.ibm_set_field(s.ctx, ibm.FIELDS[k], host_in[k].data_ptr(), 0, host_in[k].numel() * 8)
            ibm.ibm_set_field(s.ctx, ibm.FIELDS["step"], np.array([st["step"]], np.int64).ctypes.data, 0, 8)
            s.step(1)
            for k in names_out:
                ibm.ibm_get_field(s.ctx, ibm.FIELDS[k], host_out[k].data_ptr(), 0, host_out[k].numel() * 8)
        sync_all()
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world)
        result["e2e"] = {"value": N * ne2e * world / el / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h, "steps": ne2e,
                         "path": "ibm_set_field (pinned host) + ibm_step + ibm_get_field (pinned host)"}
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            result["cpu_baseline"] = cpu_baseline_sample()
        except Exception as e:  # the oracle is optional on a box without it
            result["cpu_baseline"] = {"value": None, "error": str(e)}
    s.close()
    if rank == 0 and args.ellipsoids > 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        result["ellipsoid_array"] = ellipsoid_leg(args.ellipsoids)
    if rank == 0 and args.compare:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        result["solver_compare"] = compare_leg(args.compare)
    if rank == 0 and args.ensemble > 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        result["ensemble"] = ensemble_leg(args.ensemble)
    if rank == 0 and args.serve > 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        result["serve"] = serve_leg(args.serve, args.serve_slots,
                                    ibm.IBM_MIXED if args.serve_precision == "mixed" else ibm.IBM_FP64)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

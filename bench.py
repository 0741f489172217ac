#!/usr/bin/env python
"""Throughput of the ghost-cell immersed-boundary fractional step on GB300.

Workload (default): the 3D finite-wing case on its 768x512x512 stretched
grid (201,326,592 cells) - NACA0012 section, chord 1, aspect ratio 2,
square tips, 15 degrees incidence, ~20k-triangle surface, Re 1000,
dt 0.002, Poisson solved to a 1e-10 relative residual - in mixed precision
(FP32 multigrid cycles inside FP64 defect correction), with the plain FP64
path timed beside it from the same saved state (Poisson and whole-step
speed-ups). Inputs are synthetic (seeded generators); every field is
resident in HBM during the timed steps, and each 201M-cell field (0.8 GB in
FP32, 1.6 GB in FP64) exceeds the 129 MB L2, so no L2 flush is needed.

One bench "step" = one fractional step of the whole grid (predictor,
Poisson solve, projection, ghost refresh) through ibm_step.

Multi-GPU: the solver does not shard across GPUs (one grid per GPU); with
N > 1 every rank runs an independent replica of the workload ("replicas
only"), value = cells * steps * N / max-over-ranks time.

--impl reference times the CPU oracle (the plain FP64 reference of the
method, iterative route) on a bounded sample of the same workload on the
host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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

# DRAM traffic per launch of the roofline kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch, per cell), keyed by (kernel, precision);
# valid for the kernel as captured (removed when the kernel changes). The split
# colour pass: a one-pass capture at 201,326,592 cells, 906.7 MB read and
# 377.1 MB written per launch.
SPLIT_PASS = "k_rbgs_split (finest FP32 level in colour-split storage, one colour pass)"
TRAFFIC_BYTES_PER_CELL = {(SPLIT_PASS, 4): (906.67e6 + 377.14e6) / 201326592}


def pass_bytes(ncells, s):
    """Algorithmic bytes of one red-black colour pass of the finest level
    (method minimum): the other colour's x for every cell read once (s/2 per
    cell), f read and x written for the updated half (s/2 each), one
    cell-type byte: (1.5 s + 1) per cell. Face coefficients, inverse
    diagonals and metric arrays are implementation choices, not counted."""
    return ncells * (1.5 * s + 1.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--size", default="768,512,512", help="nx,ny,nz of the wing grid")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="arithmetic of the main timed run")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 run on the same state")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-kernels", action="store_true", help="also report every timed kernel")
    ap.add_argument("--no-ktimer", action="store_true", help="skip the per-kernel timing pass")
    ap.add_argument("--wing25m", default="384,256,256",
                    help="grid of the extra FP64 + mixed wing leg ('' to skip)")
    ap.add_argument("--serve-rates", default="2,4,6,8",
                    help="offered request rates (per s) of the serving sweep ('' to skip)")
    ap.add_argument("--serve-requests", type=int, default=30, help="requests per rate of the sweep")
    ap.add_argument("--serve-full", type=float, default=0.0,
                    help="replay all 500 requests of the stream at this rate (0: skip)")
    ap.add_argument("--serve-overload", type=int, default=0,
                    help="requests replayed at the stream's own 50/s (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=4, help="cases resident at once in the serving leg")
    ap.add_argument("--serve-precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--compare", default="192,128,128",
                    help="wing grid of the Poisson solver comparison ('' to skip)")
    ap.add_argument("--ellipsoids", type=int, default=0,
                    help="steps of the 208M-cell ellipsoid array to time per precision (0: skip)")
    ap.add_argument("--no-cylinder", action="store_true",
                    help="skip the 2D cylinder leg (256x128, 20 steps: the workload of the CPU baseline)")
    ap.add_argument("--moving", default="384,256,256",
                    help="wing grid of the moving-body leg: the wing pitching about its span axis, "
                         "moved and reclassified every step ('' to skip)")
    ap.add_argument("--ensemble", type=int, default=64,
                    help="cases of the seeded 2D ensemble to run, 50 steps each (0: skip)")
    ap.add_argument("--ref-size", default="128,96,96",
                    help="wing grid of the oracle sample timed by --impl reference")
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


def cpu_model():
    """CPU model string of this host (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def run_reference(args):
    """CPU oracle (its iterative BiCGStab route, FP64) on a bounded sample of
    the same workload: the same wing on a coarser grid of the same stretching
    family. Tables, matrices and the separable preconditioner are set up
    before timing; W untimed fractional steps, then K timed ones continuing
    the run, all on the host cores (numpy's BLAS threads)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import flow, geom
    from paper_2505_17287_gb300 import synth
    nx, ny, nz = (int(x) for x in args.ref_size.split(","))
    case = synth.wing_case(nx, ny, nz)
    T = geom.body_tables(3, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(3, case.xf, case.yf, case.zf)
    typ = T["type"]
    st = flow.initial_state(g, typ, T)
    A = flow.poisson_matrix(g, typ, T)
    cache = {}

    def one(st):
        return flow.step(g, typ, T, st, case.Re, case.dt, A=A, cache=cache, solver="iter", rtol=1e-10,
                         helm_rtol=1e-12)

    for _ in range(args.warmup):
        st = one(st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = one(st)
    el = time.perf_counter() - t0
    val = g.N * args.steps / el / 1e6
    cores = os.cpu_count() or 1
    sample = (f"plain FP64 oracle (BiCGStab with the separable body-free preconditioner, Poisson rtol 1e-10, "
              f"Helmholtz 1e-12), the same wing on a {nx}x{ny}x{nz} grid ({g.N} cells) of the same stretching "
              f"family; {args.warmup} untimed then {args.steps} timed consecutive fractional steps; "
              f"CPU {cpu_model()}, numpy BLAS threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"wing NACA0012 AR2 15deg, stretched {args.size.replace(',', 'x')} grid, "
                                   f"Re 1000, dt 0.002, Poisson rtol 1e-10 (oracle sample {nx}x{ny}x{nz})",
                       "cells": g.N},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cyl_oracle_run(_=None):
    """One run of the 2D cylinder workload as configured (256x128, Re 100,
    dt 0.005, 20 fractional steps from the impulsive start) by the oracle's
    direct route; returns (cell-steps, seconds). Runs in a worker process."""
    from oracle import flow, geom
    from paper_2505_17287_gb300 import synth
    c = synth.cylinder_case()
    t0 = time.perf_counter()
    T = geom.body_tables(2, c.xf, c.yf, c.zf, c.verts, c.elems)
    g = flow.Grid(2, c.xf, c.yf, c.zf)
    flow.run(g, T["type"], T, c.nsteps, c.Re, c.dt)
    return g.N * c.nsteps, time.perf_counter() - t0


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def cpu_baseline_sample(budget_s=10.0):
    """The oracle on the 2D cylinder workload as configured (20 steps of
    256x128, its direct LU route, each run including its tables and
    factorisations): on one core (runs repeated for about budget_s), and on
    every host core as that many independent runs in spawned processes
    (one thread each). Mcell-steps/s of each."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(1, initializer=_single_thread_env) as pool:
        pool.apply(_cyl_oracle_run)                          # imports and warm-up
        work, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            w, _ = pool.apply(_cyl_oracle_run)
            work += w
        one = work / (time.perf_counter() - t0) / 1e6
    with ctx.Pool(cores, initializer=_single_thread_env) as pool:
        pool.map(_cyl_oracle_run, range(cores))              # imports and warm-up
        t0 = time.perf_counter()
        res = pool.map(_cyl_oracle_run, range(cores))
        allc = sum(w for w, _ in res) / (time.perf_counter() - t0) / 1e6
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "single_core": {"value": one, "unit": UNIT, "cores": 1},
            "sample": f"plain FP64 oracle (direct sparse LU) on the 2D cylinder workload as configured "
                      f"(256x128, Re 100, dt 0.005, 20 steps, tables and factorisations included): "
                      f"{cores} concurrent single-threaded runs for the all-core value, about {budget_s:.0f} s of "
                      f"repeated runs on one core for single_core"}


def serve_run(nreq, slots, precision, rate=None, seed=250517288):
    """Replay the first nreq requests of the seeded 3D multi-sphere stream
    (1-8 icospheres of 5120 triangles, n^3 grids with n in [64, 256], 10
    steps each) against the request loop in real time, with the stream's
    Poisson arrivals rescaled to `rate` requests per second (None: the
    stream's own 50/s); latency = completion - arrival."""
    import numpy as np
    from paper_2505_17287_gb300 import ibm, synth
    times, cases = synth.serve_stream(nreq, seed=seed)
    if rate is not None:
        times = times * (50.0 / rate)
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
    span = times[-1] - times[0] if len(times) > 1 else 1.0
    return {"requests": nreq, "completed_ok": len(ok), "offered_per_s": (len(times) - 1) / span if span > 0 else None,
            "completed_per_s": len(ok) / (last - first),
            "p50_ms": float(np.percentile(lat, 50)) if len(ok) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(ok) else None,
            "service_p50_ms": float(np.percentile(svc, 50)) if len(ok) else None,
            "value": work / (last - first) / 1e6, "unit": UNIT, "makespan_s": last - first,
            "peak_running": st["peak_running"], "peak_admitted_gb": st["peak_admitted_bytes"] / 1e9}


def serve_leg(rates, nreq, slots, precision, full_rate=0.0, overload=0):
    """Offered load against achieved load and latency: the seeded stream
    replayed at each rate of `rates` (nreq requests each); optionally all
    500 requests at `full_rate` and the stream at its own 50/s."""
    from paper_2505_17287_gb300 import ibm
    prec = ibm.IBM_MIXED if precision == "mixed" else ibm.IBM_FP64
    out = {"slots": slots, "precision": precision,
           "workload": "seeded stream (seed 250517288): 1-8 icospheres (5120 triangles each, radii 0.2-0.6) in "
                       "[-4,8]x[-3,3]^2; n^3 grids, log n uniform in [log 64, log 256], n a multiple of 16; "
                       "Re 100-500; CFL 0.2; 10 steps per request; Poisson rtol 1e-10; arrivals of the stream's "
                       "Poisson process rescaled to each offered rate",
           "sweep": []}
    for r in rates:
        out["sweep"].append(dict(rate=r, **serve_run(nreq, slots, prec, rate=r)))
    if full_rate > 0:
        out["full_500"] = dict(rate=full_rate, **serve_run(500, slots, prec, rate=full_rate))
    if overload > 0:
        out["overload_50_per_s"] = serve_run(overload, slots, prec, rate=None)
    return out


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


def cylinder_leg():
    """The 2D cylinder workload as configured (256x128, Re 100, dt 0.005, 20
    steps from the impulsive start, the CPU baseline's sample), in FP64 and
    mixed precision, each step one captured graph with device-side loop
    control (opts graph=2) on a stream of its own; the 20 steps are timed
    after an untimed run of the same 20 steps (graph capture and allocation)."""
    import torch
    from paper_2505_17287_gb300 import ibm, synth
    c = synth.cylinder_case()
    out = {"grid": "256x128", "cells": c.ncells, "steps": c.nsteps}
    for name, prec in (("fp64", ibm.IBM_FP64), ("mixed", ibm.IBM_MIXED)):
        s = ibm.Solver(c, precision=prec, stream=torch.cuda.Stream())
        s.set_opts(precision=prec, graph=2)
        s.set_body(c.verts, c.elems)
        s.classify()
        init = s.get_state()
        s.step_prepare()
        s.step_async(c.nsteps)
        s.step_wait()
        s.set_state(init)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step_async(c.nsteps)
        r = s.step_wait()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out[name] = {"value": c.ncells * c.nsteps / el / 1e6, "unit": UNIT, "ms_per_step": 1e3 * el / c.nsteps,
                     "poisson_outer_per_step": r["poisson_outer"] / max(1, r["steps"]),
                     "ok": r["status"] == ibm.IBM_OK}
        s.close()
    return out


def moving_leg(size, steps, warmup, omega=2.0):
    """The wing pitching about its span axis (y) through its centroid at
    omega rad/s, mixed precision: every step is ibm_move_body (rigid
    rotation by omega dt, reclassification, fresh cells, ghost rows with the
    body velocity) followed by ibm_step(1). Mcell-steps/s of the pair, and the
    time of each part."""
    import numpy as np
    import torch
    from paper_2505_17287_gb300 import ibm
    case = wing_case(size)
    s = ibm.Solver(case, precision=ibm.IBM_MIXED)
    s.set_opts(precision=ibm.IBM_MIXED)
    v0, e = case.verts, case.elems
    s.set_body(v0, e)
    s.classify()
    c0 = v0.mean(0)
    n = 0

    def move_step():
        nonlocal n
        n += 1
        a = omega * case.dt * n
        R = np.array([[np.cos(a), 0.0, np.sin(a)], [0.0, 1.0, 0.0], [-np.sin(a), 0.0, np.cos(a)]])
        info = s.move_body((v0 - c0) @ R.T + c0, (0.0, 0.0, 0.0), (0.0, omega, 0.0), tuple(c0))
        t1 = torch.cuda.Event(enable_timing=True)
        t1.record()
        return info, t1, s.step(1)

    for _ in range(warmup):
        move_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    move_ms, outs = 0.0, []
    e0.record()
    for _ in range(steps):
        m0 = torch.cuda.Event(enable_timing=True)
        m0.record()
        info, m1, r = move_step()
        outs.append(r)
        torch.cuda.synchronize()
        move_ms += m0.elapsed_time(m1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"grid": size.replace(",", "x"), "cells": case.ncells, "triangles": int(e.shape[0]),
           "value": case.ncells * steps / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / steps,
           "move_ms_per_step": move_ms / steps, "poisson_outer_per_step": sum(r["poisson_outer"] for r in outs) / steps,
           "ok": all(r["status"] == ibm.IBM_OK for r in outs), "n_ghost": info["n_ghost"],
           "motion": f"pitching about the span axis at {omega} rad/s, dt {case.dt}",
           "precision": "mixed"}
    s.close()
    torch.cuda.empty_cache()
    return out


def wing_leg(size, steps, warmup):
    """Extra leg: the wing on another grid, FP64 and mixed from the same
    saved state (Mcell-steps/s and the Poisson speed-up)."""
    import torch
    from paper_2505_17287_gb300 import ibm
    case = wing_case(size)
    out = {"grid": size.replace(",", "x"), "cells": case.ncells}
    saved = None
    for name, prec in (("fp64", ibm.IBM_FP64), ("mixed", ibm.IBM_MIXED)):
        s = ibm.Solver(case, precision=prec)
        s.set_opts(precision=prec)
        s.set_body(case.verts, case.elems)
        s.classify()
        if saved is None:
            for _ in range(warmup):
                s.step(1)
            saved = s.get_state()
        s.set_state(saved)
        s.step(1)                   # allocations of this precision, untimed
        s.set_state(saved)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = [s.step(1) for _ in range(steps)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": case.ncells * steps / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / steps,
                     "poisson_ms_per_step": sum(x["ms_poisson"] for x in st) / steps,
                     "poisson_outer_per_step": sum(x["poisson_outer"] for x in st) / steps,
                     "rel_residual_last": st[-1]["rel_residual"]}
        s.close()
        torch.cuda.empty_cache()
    out["poisson_speedup_mixed_vs_fp64"] = out["fp64"]["poisson_ms_per_step"] / out["mixed"]["poisson_ms_per_step"]
    out["step_speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


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
    # the CPU baseline runs first, in spawned processes, before this process
    # has much device state (and never forks after the first GPU call)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu_base = cpu_baseline_sample()
        except Exception as e:  # the oracle is optional on a box without it
            cpu_base = {"value": None, "error": str(e)}
    case = wing_case(args.size)
    # the solver runs on its own stream (not the legacy default stream), so
    # its multigrid V-cycle is captured once and replayed as a CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    main_prec = ibm.IBM_MIXED if args.precision == "mixed" else ibm.IBM_FP64
    mixed_main = main_prec == ibm.IBM_MIXED

    def make_solver(prec):
        s = ibm.Solver(case, precision=prec)
        s.set_opts(precision=prec)
        t0 = time.perf_counter()
        s.set_body(case.verts, case.elems)
        info = s.classify()
        return s, info, time.perf_counter() - t0

    s, info, setup_s = make_solver(main_prec)
    N = s.N

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def timed(solver, nsteps, kernel_timer=False):
        if kernel_timer:
            ibm.ibm_kernel_timer(solver.ctx, 1)
        sync_all()
        l0 = ibm.ibm_launch_count(solver.ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = [solver.step(1) for _ in range(nsteps)]
        e1.record(stream)
        sync_all()
        ms = e0.elapsed_time(e1)
        launches = ibm.ibm_launch_count(solver.ctx) - l0
        kt = {}
        if kernel_timer:
            for name, kid in ibm.KERNEL_IDS.items():
                kt[name] = ibm.ibm_kernel_time(solver.ctx, kid)
            ibm.ibm_kernel_timer(solver.ctx, 0)
        return max_over_ranks(ms, world), stats, launches, kt

    def summary(stats, nsteps):
        return {"poisson_outer_per_step": sum(x["poisson_outer"] for x in stats) / nsteps,
                "poisson_inner_per_step": sum(x["poisson_inner"] for x in stats) / nsteps,
                "helm_sweeps_per_step": sum(x["helm_sweeps"] for x in stats) / nsteps,
                "rel_residual_last": stats[-1]["rel_residual"],
                "ms_poisson_per_step": sum(x["ms_poisson"] for x in stats) / nsteps,
                "ms_predictor_per_step": sum(x["ms_predictor"] for x in stats) / nsteps}

    for _ in range(args.warmup):
        s.step(1)
    saved = s.get_state() if not args.no_fp64 else None
    with Clocks(local) as clk:
        ms, stats, launches, _ = timed(s, args.steps)
    clocks = clk.summary()
    value = replica_throughput(N, args.steps, world, ms)
    poisson_ms_main = sum(x["ms_poisson"] for x in stats)
    # roofline of the dominant kernel: a second pass over the same number of
    # steps with the event timer on (the timer adds host work per launch and
    # launches the V-cycle kernel by kernel, so the headline above is
    # measured without it)
    if args.no_ktimer:
        ms_kt, kt = ms, {k: (0.0, 0) for k in ibm.KERNEL_IDS}
    else:
        ms_kt, _, _, kt = timed(s, args.steps, kernel_timer=True)
    rb_ms, rb_n = kt["rbgs0"]
    sz = 4 if mixed_main else 8
    rb_bytes = pass_bytes(N, sz)
    rb_avg_s = rb_ms / rb_n / 1e3 if rb_n else None
    achieved = rb_bytes / rb_avg_s / 1e9 if rb_n else None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    # mixed precision with nx a multiple of 8: the finest FP32 level in
    # colour-split storage (one colour pass streams the other colour's x)
    split = mixed_main and N % 8 == 0 and int(args.size.split(",")[0]) % 8 == 0
    kname = SPLIT_PASS if split else \
        ("k_rbgs<float, fine>" if mixed_main else "k_rbgs<double>") + " (finest level, one colour pass)"
    tpc = TRAFFIC_BYTES_PER_CELL.get((kname, sz))
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed_main else "f64", "data": "synthetic",
        "config": {"workload": f"wing NACA0012 AR2 15deg, stretched {args.size.replace(',', 'x')} grid "
                               f"({N} cells), Re 1000, dt 0.002, Poisson rtol 1e-10, "
                               + ("mixed (FP32 multigrid cycles inside FP64 defect correction)" if mixed_main
                                  else "FP64"),
                   "cells": N, "n_ghost": info["n_ghost"], "n_dead": info["n_dead"],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (no flush)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": tpc * N if tpc else None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback",
                     "launches": rb_n, "avg_ms": rb_avg_s * 1e3 if rb_n else None,
                     "algorithmic_bytes_per_launch": rb_bytes,
                     "bytes_model": f"(1.5 s + 1) B per cell and colour pass, s = {sz}"},
        "stats": dict(setup_s=setup_s, **summary(stats, args.steps)),
    }
    if args.profile_kernels:
        result["kernels"] = {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items()}
        result["kernels_step_ms"] = ms_kt / args.steps
    if not args.no_e2e:
        # end to end through the C ABI with pinned host buffers: the state
        # lives on the host; every step copies it host->device, steps, and
        # copies the new state back, which is the next step's input (the
        # Poisson guess history stays on the device: ibm_set_field keeps it)
        names_in = ["u", "v", "w", "p", "p_prev", "p_prev2", "face_u", "face_v", "face_w", "nold_u", "nold_v",
                    "nold_w"]
        st = s.get_state()
        host_in = {k: torch.from_numpy(np.ascontiguousarray(st[k])).pin_memory() for k in names_in}
        del st
        h2d = sum(t.numel() * 8 for t in host_in.values()) + 8
        d2h = h2d
        ne2e = max(1, min(args.steps, 5))
        step_no = np.array([s.get("step")], np.int64)
        sync_all()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            for k in names_in:
                ibm.ibm_set_field(s.ctx, ibm.FIELDS[k], host_in[k].data_ptr(), 0, host_in[k].numel() * 8)
            ibm.ibm_set_field(s.ctx, ibm.FIELDS["step"], step_no.ctypes.data, 0, 8)
            s.step(1)
            for k in names_in:
                ibm.ibm_get_field(s.ctx, ibm.FIELDS[k], host_in[k].data_ptr(), 0, host_in[k].numel() * 8)
            ibm.ibm_get_field(s.ctx, ibm.FIELDS["step"], step_no.ctypes.data, 0, 8)
        sync_all()
        el = max_over_ranks(time.perf_counter() - t0, world)
        result["e2e"] = {"value": N * ne2e * world / el / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h, "steps": ne2e,
                         "path": "ibm_set_field (pinned host) + ibm_step + ibm_get_field (pinned host), "
                                 "the state carried on the host from step to step"}
        del host_in
    s.close()
    del s
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if not args.no_fp64 and mixed_main:
        # the plain FP64 path on the same saved state (its own context: the
        # FP64 hierarchy and Krylov basis are allocated by an untimed step)
        s64, _, _ = make_solver(ibm.IBM_FP64)
        s64.set_state(saved)
        s64.step(1)
        s64.set_state(saved)
        ms64, stats64, _, _ = timed(s64, args.steps)
        s64.close()
        del s64
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        poisson_ms64 = sum(x["ms_poisson"] for x in stats64)
        result["fp64_value"] = replica_throughput(N, args.steps, world, ms64)
        result["fp64_ms_per_step"] = ms64 / args.steps
        result["poisson_speedup_vs_fp64"] = poisson_ms64 / poisson_ms_main if poisson_ms_main else None
        result["step_speedup_vs_fp64"] = ms64 / ms
        result["fp64_stats"] = summary(stats64, args.steps)
        result["fp64_same_inputs"] = "both runs start from the same saved state after the warm-up steps"
    del saved
    if cpu_base is not None:
        result["cpu_baseline"] = cpu_base
    if rank == 0 and args.wing25m:
        result["wing_" + args.wing25m.replace(",", "x")] = wing_leg(args.wing25m, args.steps, args.warmup)
    if rank == 0 and not args.no_cylinder:
        result["cylinder_256x128"] = cylinder_leg()
    if rank == 0 and args.moving:
        torch.cuda.empty_cache()
        result["moving_" + args.moving.replace(",", "x")] = moving_leg(args.moving, args.steps, args.warmup)
    if rank == 0 and args.ellipsoids > 0:
        result["ellipsoid_array"] = ellipsoid_leg(args.ellipsoids)
    if rank == 0 and args.compare:
        torch.cuda.empty_cache()
        result["solver_compare"] = compare_leg(args.compare)
    if rank == 0 and args.ensemble > 0:
        torch.cuda.empty_cache()
        result["ensemble"] = ensemble_leg(args.ensemble)
    rates = [float(x) for x in args.serve_rates.split(",") if x.strip()]
    if rank == 0 and (rates or args.serve_full > 0 or args.serve_overload > 0):
        torch.cuda.empty_cache()
        result["serve"] = serve_leg(rates, args.serve_requests, args.serve_slots, args.serve_precision,
                                    args.serve_full, args.serve_overload)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

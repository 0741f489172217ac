"""Batched ensemble of independent cases of uneven size on one GPU.

run_graphs (the batched path): every case is resident on its own stream
with its fractional step captured as CUDA graphs whose loops (Helmholtz
sweeps, ghost refresh, FGMRES and mixed-precision refinement) are decided on
the device (opts graph=2); one host thread enqueues all steps of all cases
with ibm_step_async and the GPU runs the cases' graphs concurrently, with
no host round trip inside a step.

run (the request-loop path): the cases go through include/ibm_serve.h,
`slots` at a time, each slot a host worker thread driving its case.

Options are picked per size class (cell count rounded to a power of two) by
the library's autotuner, which times candidate multigrid tile widths,
smoother sweep counts (finest and coarse levels) and relaxation factors on the
first case of each class.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import ibm


def size_class(case) -> int:
    return int(round(math.log2(case.ncells)))


def candidates(precision=ibm.IBM_MIXED, tiles=(32, 64, 128, 256), nus=(1, 2), omegas=(1.0, 1.1),
               nu_coarses=(0, 3)):
    """Option sets the autotuner chooses from: multigrid row-tile width x
    smoother sweeps per V-cycle half x smoother relaxation factor (over-
    relaxation helps uniform grids, not strongly stretched ones) x sweeps on
    the levels below the finest (0: the same as the finest; more pay on large
    3D grids, fewer launches on small 2D ones), all with the V-cycle graph;
    the last one is the library default without the graph (the reference
    point)."""
    out = []
    for t in tiles:
        for nu in nus:
            for om in omegas:
                for nc in nu_coarses:
                    o = ibm.ibm_default_opts()
                    o.precision, o.tile_x, o.nu1, o.nu2, o.graph, o.smooth_omega = precision, t, nu, nu, 1, om
                    o.nu_coarse = nc
                    out.append(o)
    o = ibm.ibm_default_opts()
    o.precision, o.graph = precision, 0
    out.append(o)
    return out


def tune(cases, precision=ibm.IBM_MIXED, steps=3):
    """{size class: (chosen ibm_solver_opts, per-candidate ms/step, class case name)}"""
    cand = candidates(precision)
    table = {}
    for c in cases:
        k = size_class(c)
        if k in table:
            continue
        best, ms = ibm.ibm_tune(c, cand, steps=steps, precision=precision)
        table[k] = (cand[best], ms, c.name)
    return table


def describe(o):
    return {"tile_x": o.tile_x, "nu": o.nu1, "nu2": o.nu2, "nu_coarse": o.nu_coarse, "omega": o.smooth_omega,
            "graph": o.graph}


def run(cases, slots=12, precision=ibm.IBM_MIXED, tuned=None):
    """Advance every case its own number of steps through one server; cases
    are submitted largest first. Returns per-case results and totals."""
    order = sorted(range(len(cases)), key=lambda i: -cases[i].ncells)
    srv = ibm.Server(max_slots=slots)
    t0 = time.perf_counter()
    ids = {}
    for i in order:
        c = cases[i]
        opts = tuned[size_class(c)][0] if tuned else None
        ids[i] = srv.submit(c, precision=precision, opts=opts)
    res = {i: srv.wait(r) for i, r in ids.items()}
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    out = [res[i] for i in range(len(cases))]
    ok = all(r["status"] == ibm.IBM_OK for r in out)
    first = min(r["t_submit"] for r in out)
    last = max(r["t_done"] for r in out)
    work = sum(r["cells"] * r["steps"] for r in out)
    return {"results": out, "ok": ok, "makespan_s": last - first, "wall_s": wall,
            "mcell_steps_per_s": work / (last - first) / 1e6, "cell_steps": work,
            "peak_running": st["peak_running"]}


def _opts_kw(o):
    return {k: getattr(o, k) for k, _ in ibm.ibm_solver_opts._fields_}


def run_graphs(cases, precision=ibm.IBM_MIXED, tuned=None, opts=None, fields=False):
    """All cases resident at once, each on its own stream; the step graphs
    are captured during setup (ibm_step_prepare), then every case's steps
    are enqueued from this thread and run concurrently on the device.
    `opts` (dict) overrides solver options of every case; with fields=True
    each result also holds the final u, v (w) and p under "fields"."""
    import torch
    from . import synth
    order = sorted(range(len(cases)), key=lambda i: -cases[i].ncells)
    solvers = {}
    t0 = time.perf_counter()
    for i in order:
        c = cases[i]
        s = ibm.Solver(c, precision=precision, stream=torch.cuda.Stream())
        kw = _opts_kw(tuned[size_class(c)][0]) if tuned and size_class(c) in tuned else {}
        kw.update(opts or {})
        kw.update(precision=precision, graph=2)
        s.set_opts(**kw)
        for v, e in synth.case_bodies(c):
            s.set_body(v, e)
        s.classify()
        s.step_prepare()
        solvers[i] = s
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    for i in order:
        solvers[i].step_async(cases[i].nsteps)
    enqueue_s = time.perf_counter() - t1
    res = {i: solvers[i].step_wait() for i in order}
    torch.cuda.synchronize()
    wall = time.perf_counter() - t1
    out = [res[i] for i in range(len(cases))]
    work = sum(cases[i].ncells * out[i]["steps"] for i in range(len(cases)))
    ok = all(r["status"] == ibm.IBM_OK for r in out)
    if fields:
        for i, s in solvers.items():
            names = ("u", "v", "w", "p") if cases[i].ndim == 3 else ("u", "v", "p")
            out[i]["fields"] = {k: s.get(k) for k in names}
    for s in solvers.values():
        s.close()
    return {"results": out, "ok": ok, "wall_s": wall, "setup_s": setup_s, "enqueue_s": enqueue_s,
            "mcell_steps_per_s": work / wall / 1e6, "cell_steps": work}

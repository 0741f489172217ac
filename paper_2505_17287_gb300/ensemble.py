"""Batched ensemble of independent cases of uneven size on one GPU.

The cases run through the request loop of include/ibm_serve.h: all of them
stay resident while they advance, `slots` at a time, each slot on its own
stream so their kernels overlap on the device, and each case's multigrid
V-cycle replays as one captured CUDA graph. Options are picked per size
class (cell count rounded to a power of two) by the library's autotuner,
which times candidate tile widths and smoother sweep counts on the first
case of each class.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import ibm


def size_class(case) -> int:
    return int(round(math.log2(case.ncells)))


def candidates(precision=ibm.IBM_MIXED, tiles=(32, 64, 128, 256), nus=(1, 2)):
    """Option sets the autotuner chooses from: multigrid row-tile width x
    smoother sweeps per V-cycle half, all with the V-cycle graph; the last
    one is the library default without the graph (the reference point)."""
    out = []
    for t in tiles:
        for nu in nus:
            o = ibm.ibm_default_opts()
            o.precision, o.tile_x, o.nu1, o.nu2, o.graph = precision, t, nu, nu, 1
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
    return {"tile_x": o.tile_x, "nu": o.nu1, "graph": o.graph}


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

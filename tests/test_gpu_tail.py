"""The persistent V-cycle tail (tail_cells): the multigrid levels below a
size bound run as one launch of a thread-block cluster per V-cycle. Every
item of it evaluates the expression of the per-level kernel it replaces, so
whole fractional steps agree bit for bit with the per-level launches, for
one-block and multi-block clusters, both precisions and the smoother
variants; and the solve still reaches the oracle's pressure."""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu

ALL = 1 << 30   # every level below the finest in the tail


def _fields(case, precision, nsteps, **opts):
    s = ibm.Solver(case, precision=precision)
    s.set_opts(precision=precision, **opts)
    s.set_body(case.verts, case.elems)
    s.classify()
    r = s.step(nsteps)
    assert r["status"] == ibm.IBM_OK, r
    out = {k: s.get(k) for k in (("u", "v", "w", "p") if case.ndim == 3 else ("u", "v", "p"))}
    out["_launches"] = ibm.ibm_launch_count(s.ctx)
    s.close()
    return out


def _cases():
    return {"cylinder": synth.cylinder_case(256, 128, nseg=256, dt=0.01),
            "wing": synth.wing_case(64, 48, 40, n_chord=30, n_span=10)}


CASES = [(p, w, o, ALL) for p in (ibm.IBM_FP64, ibm.IBM_MIXED) for w in ("cylinder", "wing")
         for o in ({}, {"smooth_omega": 1.15})]
CASES += [(ibm.IBM_MIXED, "wing", o, 2048) for o in ({"nu1": 1, "nu2": 3}, {"graph": 0}, {"inner_iters": 2, "nu1": 2, "nu2": 2})]


@pytest.mark.parametrize("precision,which,opts,tail", CASES)
def test_tail_equals_per_level_launches(precision, which, opts, tail):
    case = _cases()[which]
    a = _fields(case, precision, 3, tail_cells=tail, **opts)
    b = _fields(case, precision, 3, tail_cells=0, **opts)
    for k in a:
        if k != "_launches":
            assert np.array_equal(a[k], b[k]), k
    # (kernels inside a replayed V-cycle graph are counted like launched ones)
    assert a["_launches"] < b["_launches"]


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_tail_poisson_matches_oracle(precision):
    """A 24^3 sphere case: levels of 13824, 1728 and 216 cells, the last two in
    the tail (small enough for the oracle's direct 3D solve)."""
    import torch
    case = synth.sphere_case(n=24, radius=0.45, level=3)
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    rng = np.random.default_rng(17)
    b = flow.project_rhs(g, T["type"], rng.uniform(-1, 1, g.shape))
    phi_ref, _ = flow.solve_poisson(g, T["type"], T, b)
    s = ibm.Solver(case, precision=precision)
    s.set_opts(precision=precision, tail_cells=ALL, rtol=1e-13, max_outer=400)
    s.set_body(case.verts, case.elems)
    s.classify()
    rhs = torch.from_numpy(b.ravel()).cuda()
    phi = torch.zeros_like(rhs)
    st = s.poisson_solve(rhs, phi, rtol=1e-13, maxit=400)
    assert st["status"] == ibm.IBM_OK and st["rel_residual"] <= 1e-13, st
    got = phi.cpu().numpy().reshape(g.shape)
    assert np.linalg.norm(got - phi_ref) / np.linalg.norm(phi_ref) < 1e-9
    s.close()


def test_tail_kernel_timed():
    case = _cases()["cylinder"]
    s = ibm.Solver(case, precision=ibm.IBM_MIXED)
    s.set_opts(precision=ibm.IBM_MIXED, tail_cells=ALL)
    s.set_body(case.verts, case.elems)
    s.classify()
    s.step(1)
    ibm.ibm_kernel_timer(s.ctx, 1)
    s.step(1)
    ms, n = ibm.ibm_kernel_time(s.ctx, ibm.KERNEL_IDS["tail"])
    _, nc = ibm.ibm_kernel_time(s.ctx, ibm.KERNEL_IDS["rbgs_coarse"])
    ibm.ibm_kernel_timer(s.ctx, 0)
    s.close()
    assert n > 0 and ms > 0 and nc == 0

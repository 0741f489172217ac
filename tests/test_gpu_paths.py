"""GPU parity on paths the main parity tests do not reach, and the failure
statuses.

* Taylor-Green vortex with free-slip walls (an exact Navier-Stokes solution,
  no body): the GPU step equals the oracle's step, in FP64 and in mixed
  precision, and its own temporal self-convergence is second order.
* True multigrid-preconditioned CG (three MG-PCG iterations per
  preconditioner call) reaches the oracle's Poisson solution and step.
* One case of the batched ensemble gives the bits it gives alone, and equals
  the oracle; one served 3D case equals the oracle.
* A non-finite right-hand side or field gives IBM_ERR_DIVERGED; an iteration
  limit below what the tolerance needs gives IBM_ERR_NOT_CONVERGED.
"""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ensemble, ibm, synth

pytestmark = pytest.mark.gpu

TIGHT = dict(rtol=1e-13, helm_rtol=1e-14, ghost_tol=1e-16, max_outer=400)
SLIP4 = (ibm.IBM_BC_SLIP,) * 6


def _tg_oracle(case):
    f0 = synth.taylor_green_fields(case, 0.0)
    g = flow.Grid(2, case.xf, case.yf, case.zf)
    typ = np.zeros(g.shape, np.uint8)
    tabs = dict(gidx=np.zeros(0, np.int64), sidx=np.zeros((0, 8), np.int64), wp=np.zeros((0, 8)),
                wv=np.zeros((0, 8)), bv=np.zeros(0), bp=np.zeros(0))
    st = flow.State([f0["u"], f0["v"]], [f0["face_u"], f0["face_v"]], np.zeros(g.shape), None, 0)
    A = flow.poisson_matrix(g, typ, tabs)
    cache = {}
    for _ in range(case.nsteps):
        st = flow.step(g, typ, tabs, st, case.Re, case.dt, (flow.SLIP,) * 6, (0.0, 0.0, 0.0), A, cache=cache)
    return g, typ, st


def _tg_gpu(case, precision):
    s = ibm.Solver(case, precision=precision, bc=SLIP4)
    s.set_opts(**TIGHT, precision=precision)
    s.set_body(case.verts, case.elems)
    info = s.classify()
    assert info["n_ghost"] == 0 and info["n_dead"] == 0
    f0 = synth.taylor_green_fields(case, 0.0)
    for k in ("u", "v", "face_u", "face_v"):
        s.set(k, f0[k])
    s.set("p", np.zeros(s.shape))
    r = s.step(case.nsteps)
    assert r["status"] == ibm.IBM_OK, r
    out = {k: s.get(k) for k in ("u", "v", "face_u", "face_v", "p")}
    s.close()
    return out


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_taylor_green_step_parity(precision):
    case = synth.taylor_green_case(32, 1.0, 0.0025, 20)
    g, typ, st = _tg_oracle(case)
    got = _tg_gpu(case, precision)
    for name, ref in (("u", st.u[0]), ("v", st.u[1]), ("face_u", st.F[0]), ("face_v", st.F[1])):
        err = np.abs(got[name] - ref).max() / np.abs(ref).max()
        assert err < 1e-8, (name, err)
    p_ref = flow.normalise(g, typ, st.p)
    err = np.linalg.norm(got["p"] - p_ref) / np.linalg.norm(p_ref)
    assert err < 1e-9, err


def test_taylor_green_second_order_on_gpu():
    runs = [_tg_gpu(synth.taylor_green_case(32, 1.0, dt, int(round(0.05 / dt))), ibm.IBM_FP64)
            for dt in (0.01, 0.005, 0.0025)]
    du = [np.abs(a["u"] - b["u"]).max() for a, b in zip(runs, runs[1:])]
    assert 3.7 < du[0] / du[1] < 4.3, du
    ex = synth.taylor_green_fields(synth.taylor_green_case(32, 1.0, 0.0025, 20), 0.05)
    assert np.abs(runs[-1]["u"] - ex["u"]).max() < 1.5e-3 * np.abs(ex["u"]).max()


def _ragged(name):
    if name == "ellipse_ragged":
        case = synth.cylinder_case(97, 53)
        case.verts, case.elems = synth.ellipse_polyline(1.0, 0.3, 0.6, 256)
    else:
        case = synth.sphere_case(n=29, radius=0.45, level=3)
        case.yf = np.linspace(-1.0, 1.0, 24)
        case.zf = np.linspace(-1.0, 1.0, 20)
    return case


@pytest.mark.parametrize("name", ["ellipse_ragged", "sphere_ragged"])
@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_poisson_parity_true_mg_pcg(name, precision):
    """inner_iters = 3: each preconditioner call runs three iterations of
    multigrid-preconditioned CG on the staircase operator (symmetric V-cycle,
    nu1 = nu2), not a single scaled V-cycle."""
    import torch
    case = _ragged(name)
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    rng = np.random.default_rng(5)
    b = flow.project_rhs(g, T["type"], rng.uniform(-1, 1, g.shape))
    phi_ref, _ = flow.solve_poisson(g, T["type"], T, b)
    s = ibm.Solver(case, precision=precision)
    s.set_opts(**TIGHT, precision=precision, inner_iters=3, nu1=2, nu2=2)
    s.set_body(case.verts, case.elems)
    s.classify()
    rhs = torch.from_numpy(b.ravel()).cuda()
    phi = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    st = s.poisson_solve(rhs, phi, rtol=1e-13, maxit=400)
    assert st["status"] == ibm.IBM_OK and st["rel_residual"] <= 1e-13, st
    assert st["inner_iters"] >= 2 * st["outer_iters"], st
    err = np.linalg.norm(phi.cpu().numpy().reshape(g.shape) - phi_ref) / np.linalg.norm(phi_ref)
    assert err < 1e-9, err
    s.close()


def _oracle_fields(case, nsteps):
    bodies = synth.case_bodies(case)
    vs, es, off = [], [], 0
    for v, e in bodies:
        vs.append(v)
        es.append(e + off)
        off += len(v)
    verts, elems = np.concatenate(vs), np.concatenate(es).astype(np.int32)
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, verts, elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    st = flow.run(g, T["type"], T, nsteps, case.Re, case.dt)
    return g, T, st


def _compare(fields, g, T, st, vtol=1e-8, ptol=1e-9):
    for q, n in enumerate(["u", "v", "w"][: g.ndim]):
        ref = st.u[q]
        err = np.abs(fields[n] - ref).max() / max(1.0, np.abs(ref).max())
        assert err < vtol, (n, err)
    p_ref = flow.normalise(g, T["type"], st.p)
    err = np.linalg.norm(fields["p"] - p_ref) / np.linalg.norm(p_ref)
    assert err < ptol, ("p", err)


def test_step_parity_true_mg_pcg():
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02, nsteps=3)
    g, T, st = _oracle_fields(case, 3)
    s = ibm.Solver(case)
    s.set_opts(**TIGHT, inner_iters=3, nu1=2, nu2=2)
    s.set_body(case.verts, case.elems)
    s.classify()
    r = s.step(3)
    assert r["status"] == ibm.IBM_OK, r
    _compare({k: s.get(k) for k in ("u", "v", "p")}, g, T, st)
    s.close()


def test_ensemble_case_alone_equals_batched_and_oracle():
    cases = synth.ensemble_2d(5, seed=3)
    for c in cases:
        c.nsteps = 3
    small = min(range(len(cases)), key=lambda i: cases[i].ncells)
    batch = ensemble.run_graphs(cases, opts=TIGHT, fields=True)
    assert batch["ok"], [r["status"] for r in batch["results"]]
    alone = ensemble.run_graphs([cases[small]], opts=TIGHT, fields=True)
    assert alone["ok"]
    a, b = alone["results"][0]["fields"], batch["results"][small]["fields"]
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    g, T, st = _oracle_fields(cases[small], 3)
    _compare(b, g, T, st)


def test_served_3d_case_matches_oracle():
    case = synth.multi_sphere_case(24, [(0.6, (0.5, 0.0, 0.0)), (0.5, (3.0, 0.4, -0.3))], 200.0, nsteps=2, level=2)
    o = ibm.ibm_default_opts()
    for k, v in TIGHT.items():
        setattr(o, k, v)
    srv = ibm.Server(max_slots=2)
    rid = srv.submit(case, opts=o, outputs=True)
    r = srv.wait(rid)
    srv.close()
    assert r["status"] == ibm.IBM_OK, r["error"]
    g, T, st = _oracle_fields(case, 2)
    assert T["gidx"].size > 0
    _compare(r["outputs"], g, T, st)


def test_nonfinite_rhs_gives_diverged():
    import torch
    case = synth.cylinder_case(64, 32, nseg=128)
    s = ibm.Solver(case)
    s.set_body(case.verts, case.elems)
    s.classify()
    rhs = torch.ones(s.N, dtype=torch.float64, device="cuda")
    rhs[s.N // 3] = float("nan")
    phi = torch.zeros_like(rhs)
    with pytest.raises(ibm.IBMError) as e:
        s.poisson_solve(rhs, phi)
    assert e.value.status == ibm.IBM_ERR_DIVERGED
    # the context stays usable: a finite right-hand side solves afterwards
    rhs[s.N // 3] = 0.5
    phi.zero_()
    st = s.poisson_solve(rhs, phi)
    assert st["status"] == ibm.IBM_OK
    s.close()


def test_nonfinite_velocity_gives_diverged():
    case = synth.cylinder_case(64, 32, nseg=128)
    s = ibm.Solver(case)
    s.set_body(case.verts, case.elems)
    s.classify()
    u = s.get("u")
    u[0, 5, 7] = float("inf")
    s.set("u", u)
    with pytest.raises(ibm.IBMError) as e:
        s.step(1)
    assert e.value.status == ibm.IBM_ERR_DIVERGED
    s.close()


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_iteration_limit_gives_not_converged(precision):
    import torch
    case = synth.cylinder_case(96, 48, nseg=128)
    s = ibm.Solver(case, precision=precision)
    s.set_opts(precision=precision)
    s.set_body(case.verts, case.elems)
    s.classify()
    rng = np.random.default_rng(1)
    rhs = torch.from_numpy(rng.uniform(-1, 1, s.N)).cuda()
    phi = torch.zeros_like(rhs)
    st = s.poisson_solve(rhs, phi, rtol=1e-13, maxit=1)
    assert st["status"] == ibm.IBM_ERR_NOT_CONVERGED, st
    assert st["rel_residual"] > 1e-13
    s.close()


def _mixed_fields(case, nsteps, **opts):
    s = ibm.Solver(case, precision=ibm.IBM_MIXED)
    s.set_opts(precision=ibm.IBM_MIXED, **opts)
    s.set_body(case.verts, case.elems)
    s.classify()
    r = s.step(nsteps)
    assert r["status"] == ibm.IBM_OK, r
    out = {k: s.get(k) for k in (("u", "v", "w", "p") if case.ndim == 3 else ("u", "v", "p"))}
    s.close()
    return out


@pytest.mark.parametrize("opts", [{}, {"smooth_omega": 1.15}, {"nu1": 1, "nu2": 3}, {"graph": 0},
                                  {"inner_iters": 2, "nu1": 2, "nu2": 2}])
@pytest.mark.parametrize("which", ["wing", "cylinder"])
def test_split_level0_equals_cell_ordered(which, opts):
    """The finest FP32 multigrid level in colour-split storage (fine_split 1)
    evaluates every cell with the operations of the cell-ordered kernels, so
    the mixed-precision steps agree bit for bit."""
    case = synth.wing_case(64, 48, 40, n_chord=30, n_span=10) if which == "wing" else \
        synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    a = _mixed_fields(case, 3, fine_split=1, **opts)
    b = _mixed_fields(case, 3, fine_split=0, **opts)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_split_level0_pass_is_faster():
    """The split pass moves half the bytes of the cell-ordered one: on the
    25M-cell wing (fields beyond the L2 cache) its mean finest-level colour
    pass takes less time (which also shows that the split kernels ran)."""
    case = synth.wing_case(384, 256, 256)
    t = {}
    for fs in (1, 0):
        s = ibm.Solver(case, precision=ibm.IBM_MIXED)
        s.set_opts(precision=ibm.IBM_MIXED, fine_split=fs)
        s.set_body(case.verts, case.elems)
        s.classify()
        s.step(1)
        ibm.ibm_kernel_timer(s.ctx, 1)
        s.step(2)
        ms, n = ibm.ibm_kernel_time(s.ctx, ibm.KERNEL_IDS["rbgs0"])
        ibm.ibm_kernel_timer(s.ctx, 0)
        s.close()
        assert n > 0
        t[fs] = ms / n
    print("finest colour pass ms, split / cell-ordered:", t)
    assert t[1] < 0.9 * t[0], t

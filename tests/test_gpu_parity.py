"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.

Bars (from the method): cell tables bit-exact (types, ghost list, base
cells, kinds, corner masks, stencil indices) and the FP64 geometry (body
intercepts, normals, image points, weights) equal to the last bit, since
both sides evaluate the same correctly rounded operations in the same order;
Poisson solution within 1e-9 relative L2 and velocity within 1e-8 relative
of the oracle for FP64 runs (both solved to near machine precision).
"""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _solver(case, precision=ibm.IBM_FP64, **opts):
    s = ibm.Solver(case, precision=precision)
    o = dict(rtol=1e-13, helm_rtol=1e-14, ghost_tol=1e-16, max_outer=400)
    o.update(opts)
    s.set_opts(**o, precision=precision)
    s.set_body(case.verts, case.elems)
    s.classify()
    return s


def _cases():
    ell_v, ell_e = synth.ellipse_polyline(1.0, 0.3, 0.6, 256)
    ell = synth.cylinder_case(97, 53)
    ell.verts, ell.elems, ell.name = ell_v, ell_e, "ellipse_ragged"
    sph = synth.sphere_case(n=29, radius=0.45, level=3)
    sph.yf = np.linspace(-1.0, 1.0, 24)
    sph.zf = np.linspace(-1.0, 1.0, 20)
    sph.name = "sphere_ragged"
    wing = synth.wing_case(64, 48, 40, n_chord=30, n_span=10)
    return {"cylinder_cfg": synth.cylinder_case(), "ellipse_ragged": ell, "sphere_ragged": sph, "wing_small": wing}


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_tables_bit_exact(name):
    case = CASES[name]
    s = _solver(case)
    got = s.tables()
    ref = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    assert np.array_equal(got["type"], ref["type"])
    assert np.array_equal(got["gidx"], ref["gidx"])
    assert got["gidx"].size > 0
    for k in ("base", "kind", "cmask", "sidx"):
        assert np.array_equal(got[k], ref[k]), k
    for k in ("bi", "nrm", "ip", "dist", "wv", "wp", "bv", "bp"):
        assert np.array_equal(got[k], ref[k]), (k, np.abs(got[k] - ref[k]).max())
    info = s.info
    assert info.n_ghost == ref["gidx"].size
    assert info.n_dead == int((ref["type"] == 2).sum())
    assert list(info.n_kind) == [int((ref["kind"] == q).sum()) for q in range(3)]
    s.close()


def _poisson_case(name):
    case = CASES[name]
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    return case, T, g


@pytest.mark.parametrize("name", ["ellipse_ragged", "sphere_ragged"])
@pytest.mark.parametrize("precision,band", [(ibm.IBM_FP64, 0), (ibm.IBM_MIXED, 0), (ibm.IBM_FP64, 2)])
def test_poisson_parity(name, precision, band):
    """band > 0: damped Jacobi sweeps of the full operator on the cells near
    the body after the V-cycle (FP64 preconditioner)."""
    import torch
    case, T, g = _poisson_case(name)
    rng = np.random.default_rng(7)
    b = flow.project_rhs(g, T["type"], rng.uniform(-1, 1, g.shape))
    phi_ref, _ = flow.solve_poisson(g, T["type"], T, b)
    s = _solver(case, precision, band_sweeps=band)
    rhs = torch.from_numpy(rng.uniform(-1, 1, g.shape)).cuda()  # raw; FLUID mean removed inside
    rhs.copy_(torch.from_numpy(np.where(T["type"] == 0, b, 123.0)))  # non-FLUID rows must be ignored
    phi = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    st = s.poisson_solve(rhs.reshape(-1), phi, rtol=1e-13, maxit=400)
    assert st["status"] == ibm.IBM_OK and st["rel_residual"] <= 1e-13, st
    got = phi.cpu().numpy().reshape(g.shape)
    err = np.linalg.norm(got - phi_ref) / np.linalg.norm(phi_ref)
    assert err < 1e-9, err
    s.close()


@pytest.mark.parametrize("name", ["ellipse_ragged", "sphere_ragged"])
@pytest.mark.parametrize("precond", [0, 1])
def test_poisson_parity_bicgstab(name, precond):
    """The paper's own Poisson path (Section 2.1): BiCGStab, right
    preconditioned by scheduled relaxation Jacobi (precond 1) or by the
    multigrid V-cycle (0), reaches the oracle's discrete solution."""
    import torch
    case, T, g = _poisson_case(name)
    rng = np.random.default_rng(11)
    b = flow.project_rhs(g, T["type"], rng.uniform(-1, 1, g.shape))
    phi_ref, _ = flow.solve_poisson(g, T["type"], T, b)
    s = _solver(case, outer=ibm.IBM_OUTER_BICGSTAB, precond=precond, max_outer=6000)
    rhs = torch.from_numpy(np.where(T["type"] == 0, b, -5.0).ravel()).cuda()
    phi = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    st = s.poisson_solve(rhs, phi, rtol=1e-13, maxit=6000)
    assert st["status"] == ibm.IBM_OK and st["rel_residual"] <= 1e-13, st
    got = phi.cpu().numpy().reshape(g.shape)
    err = np.linalg.norm(got - phi_ref) / np.linalg.norm(phi_ref)
    assert err < 1e-9, err
    s.close()


def test_poisson_zero_rhs_gives_zero():
    import torch
    case, T, g = _poisson_case("ellipse_ragged")
    s = _solver(case)
    # zero on FLUID rows; anything on the other rows is ignored
    rhs = torch.from_numpy(np.where(T["type"] == 0, 0.0, 7.0).ravel()).cuda()
    phi = torch.ones(g.N, dtype=torch.float64, device="cuda")
    st = s.poisson_solve(rhs, phi)
    assert st["status"] == ibm.IBM_OK
    assert float(phi.abs().max()) == 0.0
    s.close()


def _oracle_run(case, nsteps):
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    st = flow.run(g, T["type"], T, nsteps, case.Re, case.dt)
    return g, T, st


def _compare_state(s, g, T, st, vtol=1e-8, ptol=1e-9):
    names = ["u", "v", "w"][: g.ndim]
    for q, n in enumerate(names):
        got, ref = s.get(n), st.u[q]
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err < vtol, (n, err)
    for q, n in enumerate(["face_u", "face_v", "face_w"][: g.ndim]):
        got, ref = s.get(n), st.F[q]
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err < vtol, (n, err)
    p_ref = flow.normalise(g, T["type"], st.p)
    p = s.get("p")
    err = np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref)
    assert err < ptol, ("p", err)


def test_step_parity_cylinder_small():
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    g, T, st = _oracle_run(case, 4)
    s = _solver(case)
    out = s.step(4)
    assert out["status"] == ibm.IBM_OK, out
    _compare_state(s, g, T, st)
    assert s.get("step") == 4
    s.close()


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
@pytest.mark.parametrize("name", ["cylinder_small", "sphere_ragged"])
def test_step_parity_device_controlled(name, precision):
    """The step captured as a CUDA graph with every loop decided on the device
    (opts graph=2, on a side stream, enqueued with ibm_step_async) against
    the oracle, at the same tolerances as the host-driven step."""
    import torch
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02) if name == "cylinder_small" else CASES[name]
    n = 4 if name == "cylinder_small" else 2
    g, T, st = _oracle_run(case, n)
    s = ibm.Solver(case, precision=precision, stream=torch.cuda.Stream())
    s.set_opts(rtol=1e-13, helm_rtol=1e-14, ghost_tol=1e-16, max_outer=400, precision=precision, graph=2)
    s.set_body(case.verts, case.elems)
    s.classify()
    s.step_prepare()
    s.step_async(n)
    out = s.step_wait()
    assert out["status"] == ibm.IBM_OK and out["steps"] == n, out
    _compare_state(s, g, T, st)
    assert s.get("step") == n
    s.close()


@pytest.mark.parametrize("name", ["cylinder_small", "sphere_ragged"])
def test_step_parity_srj_helmholtz(name):
    """The Helmholtz step by scheduled relaxation Jacobi (Section 2.1's solver
    for the advection-diffusion step) reaches the oracle's predictor."""
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02) if name == "cylinder_small" else CASES[name]
    n = 3 if name == "cylinder_small" else 2
    g, T, st = _oracle_run(case, n)
    s = _solver(case, helm_solver=1)
    out = s.step(n)
    assert out["status"] == ibm.IBM_OK, out
    _compare_state(s, g, T, st)
    s.close()


def test_step_parity_sphere_3d_ragged():
    case = CASES["sphere_ragged"]
    g, T, st = _oracle_run(case, 2)
    s = _solver(case)
    out = s.step(2)
    assert out["status"] == ibm.IBM_OK, out
    _compare_state(s, g, T, st)
    s.close()


def test_step_parity_cylinder_full_config():
    """The 2D cylinder workload as configured: 256x128, Re 100, dt 0.005, 20
    fractional steps, compared with the oracle at every field."""
    case = synth.cylinder_case()
    g, T, st = _oracle_run(case, case.nsteps)
    s = _solver(case)
    out = s.step(case.nsteps)
    assert out["status"] == ibm.IBM_OK, out
    _compare_state(s, g, T, st)
    s.close()


def test_step_default_tolerance_reaches_target():
    """With the default options the Poisson solve stops at 1e-10."""
    case = synth.cylinder_case()
    s = ibm.Solver(case)
    s.set_body(case.verts, case.elems)
    s.classify()
    out = s.step(3)
    assert out["status"] == ibm.IBM_OK
    assert out["rel_residual"] <= 1e-10
    s.close()


def test_checkpoint_restart_is_bitwise():
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    a = _solver(case)
    a.step(4)
    ref = a.get_state()
    b = _solver(case)
    b.step(2)
    saved = b.get_state()
    c = _solver(case)
    c.set_state(saved)
    c.step(2)
    got = c.get_state()
    for k in ref:
        assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k])), k
    for x in (a, b, c):
        x.close()


def test_poisson_guess_keeps_the_previous_pressure():
    """From the third step on the Poisson solve starts from 2 p^n - p^(n-1);
    the context keeps p^(n-1) as field p_prev, which a checkpoint carries."""
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    s = _solver(case)
    s.step(2)
    p2 = s.get("p")
    out = s.step(1)
    assert out["status"] == ibm.IBM_OK and out["rel_residual"] <= 1e-10
    assert np.array_equal(s.get("p_prev"), p2)
    assert not np.array_equal(s.get("p"), p2)
    s.close()


def test_helmholtz_test_schedule():
    """The residual test schedule decides only when a converged Helmholtz solve
    stops: a test after every sweep finds the smallest sweep count, a later
    first test takes at least as many sweeps, and both meet the tolerance."""
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    out = {}
    for first in (1, 6):
        s = _solver(case, helm_check_first=first)
        r = s.step(3)
        assert r["status"] == ibm.IBM_OK
        out[first] = (r["helm_sweeps"], s.get("u"), s.get("v"))
        s.close()
    assert out[6][0] >= out[1][0]
    for k in (1, 2):
        a, b = out[1][k], out[6][k]
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()


@pytest.mark.parametrize("omega", [0.0, 1.05])
def test_helmholtz_relaxation_factor(omega):
    """Over-relaxed colour passes (a given factor, or 0 for the optimum of the
    grid bound) converge to the Gauss-Seidel solution within the tolerances."""
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    out = []
    for w in (1.0, omega):
        s = _solver(case, helm_omega=w)
        r = s.step(3)
        assert r["status"] == ibm.IBM_OK and r["rel_residual"] <= 1e-12
        out.append((s.get("u"), s.get("v")))
        s.close()
    for a, b in zip(out[0], out[1]):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()


def test_error_paths():
    case = synth.cylinder_case(32, 16, nseg=64)
    s = ibm.Solver(case)
    with pytest.raises(ibm.IBMError) as e:
        s.step(1)
    assert e.value.status == ibm.IBM_ERR_STATE
    with pytest.raises(ibm.IBMError) as e:
        s.classify()
    assert e.value.status == ibm.IBM_ERR_STATE
    v, el = case.verts, case.elems
    with pytest.raises(ibm.IBMError) as e:
        s.set_body(v, el[:-1])  # open polyline
    assert e.value.status == ibm.IBM_ERR_MESH
    s.set_body(v, el)
    s.classify()
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_get_field(s.ctx, ibm.FIELDS["u"], np.zeros(3).ctypes.data, 0, 24)
    assert e.value.status == ibm.IBM_ERR_ARG
    with pytest.raises(ibm.IBMError) as e:
        s.set_opts(restart=99)
    assert e.value.status == ibm.IBM_ERR_ARG
    s.close()


def test_field_copies_pinned_and_pageable_agree():
    """ibm_get_field / ibm_set_field through pinned host buffers (copied by a
    kernel over the host link) and through pageable ones (cudaMemcpyAsync)
    move the same bytes, including a length that is not a multiple of 16."""
    import torch
    case = synth.cylinder_case(97, 53)
    s = _solver(case)
    s.step(2)
    for name in ("u", "face_u", "face_v", "p"):
        shape = s.field_size(name)
        ref = s.get(name)                                   # pageable numpy
        pinned = torch.empty(shape, dtype=torch.float64).pin_memory()
        ibm.ibm_get_field(s.ctx, ibm.FIELDS[name], pinned.data_ptr(), 0, pinned.numel() * 8)
        assert np.array_equal(pinned.numpy(), ref), name
        new = np.random.default_rng(3).uniform(-1, 1, shape)
        src = torch.from_numpy(new).pin_memory()
        ibm.ibm_set_field(s.ctx, ibm.FIELDS[name], src.data_ptr(), 0, src.numel() * 8)
        assert np.array_equal(s.get(name), new), name
    s.close()

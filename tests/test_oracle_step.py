"""Pins for the oracle's fractional step (Section 2.1: fractional-step split,
central differences, Adams-Bashforth convection; Crank-Nicolson diffusion
and the outer boundary conditions are readings of the design notes).

* uniform flow with no body is an exact steady solution: one step keeps it;
* the convective term of a linear field in a uniform stream is the exact
  derivative on a uniform grid, and its volume integral telescopes to the
  boundary fluxes on any grid;
* the Crank-Nicolson Helmholtz system with its boundary rows equals a
  separable solve built from 1D operators written with plain loops;
* projection identity: after the step, div U = dt (b_raw - A phi) on FLUID
  cells up to rounding, so the divergence is a single constant over FLUID
  cells (the compatibility scalar) at solver tolerance;
* the cylinder flow stays mirror-symmetric about y = 0.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import flow, geom
from paper_2505_17287_gb300 import synth


def _no_body(ndim, f):
    g = flow.Grid(ndim, *f)
    typ = np.zeros(g.shape, dtype=np.uint8)
    tabs = dict(gidx=np.zeros(0, np.int64), sidx=np.zeros((0, 8), np.int64),
                wp=np.zeros((0, 8)), wv=np.zeros((0, 8)), bv=np.zeros(0), bp=np.zeros(0))
    return g, typ, tabs


@pytest.mark.parametrize("ndim", [2, 3])
def test_uniform_flow_is_preserved(ndim):
    fx = synth.stretched_faces(-1.0, 2.0, 14, 0.0, 0.5, 1.1)
    fy = synth.stretched_faces(-1.0, 1.0, 10, -0.2, 0.2, 1.1)
    fz = synth.stretched_faces(-1.0, 1.0, 8, -0.2, 0.2, 1.1) if ndim == 3 else np.array([0.0, 1.0])
    g, typ, tabs = _no_body(ndim, [fx, fy, fz])
    st = flow.initial_state(g, typ, tabs)
    for _ in range(3):
        st = flow.step(g, typ, tabs, st, 100.0, 0.01)
    assert np.abs(st.u[0] - 1.0).max() < 1e-13
    for c in range(1, ndim):
        assert np.abs(st.u[c]).max() < 1e-13
    assert np.abs(st.p).max() < 1e-11


def test_convection_linear_field_uniform_grid():
    f = [np.linspace(0, 1, 11), np.linspace(0, 1, 9), np.array([0.0, 1.0])]
    g, typ, tabs = _no_body(2, f)
    Y, X = np.meshgrid(g.c[1], g.c[0], indexing="ij")
    u = [(2.0 + 3.0 * X + 0.5 * Y)[None], (1.0 - 2.0 * Y)[None]]
    F = [np.full(g.face_shape(0), 1.25), np.full(g.face_shape(1), -0.75)]
    N = flow.convection(g, typ, u, F)
    # d(U u)/dx + d(V u)/dy with U, V constant = U du/dx + V du/dy (interior)
    assert np.allclose(N[0][0, 1:-1, 1:-1], 1.25 * 3.0 - 0.75 * 0.5, atol=1e-12)
    assert np.allclose(N[1][0, 1:-1, 1:-1], -0.75 * -2.0, atol=1e-12)


def test_convection_conservation_stretched():
    fx = synth.stretched_faces(-1.0, 2.0, 12, 0.0, 0.5, 1.2)
    fy = synth.stretched_faces(-1.0, 1.0, 10, -0.2, 0.2, 1.2)
    fz = synth.stretched_faces(-1.0, 1.0, 8, -0.2, 0.2, 1.2)
    g, typ, tabs = _no_body(3, [fx, fy, fz])
    rng = np.random.default_rng(1)
    u = [rng.uniform(-1, 1, g.shape) for _ in range(3)]
    F = [rng.uniform(-1, 1, g.face_shape(a)) for a in range(3)]
    N = flow.convection(g, typ, u, F)
    for comp in range(3):
        total = np.sum(g.vol * N[comp])
        bnd = 0.0
        for a in range(3):
            A = np.broadcast_to(g.area[a], g.face_shape(a))
            sl_lo = flow._sl(a, 0, 1)
            sl_hi = flow._sl(a, g.shape[2 - a], None)
            cl = flow._sl(a, 0, 1)
            ch = flow._sl(a, g.shape[2 - a] - 1, None)
            isd, val = flow.bc_dirichlet(flow.DEFAULT_BC, a, 0, comp, (1.0, 0.0, 0.0))
            ulo = val if isd else u[comp][cl]
            isd, val = flow.bc_dirichlet(flow.DEFAULT_BC, a, 1, comp, (1.0, 0.0, 0.0))
            uhi = val if isd else u[comp][ch]
            bnd += np.sum(A[sl_hi] * F[a][sl_hi] * uhi) - np.sum(A[sl_lo] * F[a][sl_lo] * ulo)
        assert abs(total - bnd) < 1e-12 * max(1.0, abs(bnd))


def _helm1d(f, alpha, left_dir, right_dir):
    """1D (I - alpha L0) parts with plain loops: returns (K, h) such that the
    operator is sum over axes of alpha * K_a / h_a on the diagonal-scaled grid."""
    n = len(f) - 1
    h = np.diff(f)
    c = 0.5 * (f[:-1] + f[1:])
    K = np.zeros((n, n))
    for i in range(n - 1):
        t = 1.0 / (c[i + 1] - c[i])
        K[i, i] += t
        K[i + 1, i + 1] += t
        K[i, i + 1] -= t
        K[i + 1, i] -= t
    if left_dir:
        K[0, 0] += 1.0 / (0.5 * h[0])
    if right_dir:
        K[n - 1, n - 1] += 1.0 / (0.5 * h[-1])
    return K, h


@pytest.mark.parametrize("comp", [0, 1])
def test_helmholtz_matches_separable_solve(comp):
    fx = synth.stretched_faces(0.0, 2.0, 12, 0.5, 1.0, 1.15)
    fy = synth.stretched_faces(-1.0, 1.0, 10, -0.2, 0.2, 1.15)
    g, typ, tabs = _no_body(2, [fx, fy, np.array([0.0, 1.0])])
    alpha = 0.05
    H = flow.helmholtz_matrix(g, typ, tabs, comp, alpha)
    rng = np.random.default_rng(2)
    rhs = rng.uniform(-1, 1, g.shape)
    got = np.linalg.solve(H.toarray(), rhs.ravel()).reshape(g.shape)
    # x: inflow Dirichlet on the left for every component, outflow Neumann on
    # the right; y: slip walls, Dirichlet only for the normal component v
    Kx, hx = _helm1d(fx, alpha, True, False)
    Ky, hy = _helm1d(fy, alpha, comp == 1, comp == 1)
    mx, vx = sla.eigh(Kx, np.diag(hx))
    my, vy = sla.eigh(Ky, np.diag(hy))
    t = rhs[0]
    t = (vy.T * hy) @ t @ (vx.T * hx).T
    t = t / (1.0 + alpha * (my[:, None] + mx[None, :]))
    want = vy @ t @ vx.T
    assert np.abs(got[0] - want).max() < 1e-12


@pytest.fixture(scope="module")
def cyl_run():
    c = synth.cylinder_case(96, 48)
    T = geom.body_tables(2, c.xf, c.yf, c.zf, c.verts, c.elems)
    g = flow.Grid(2, c.xf, c.yf, c.zf)
    st = flow.initial_state(g, T["type"], T)
    A = flow.poisson_matrix(g, T["type"], T)
    cache = {}
    out = []
    for _ in range(3):
        st, k = flow.step(g, T["type"], T, st, c.Re, c.dt, A=A, keep=True, cache=cache)
        out.append((st, k))
    return c, g, T, A, out


def test_projection_identity(cyl_run):
    c, g, T, A, out = cyl_run
    typ = T["type"]
    st, k = out[-1]
    div = flow.divergence(g, st.F)
    Aphi = (A @ k["phi"].ravel()).reshape(g.shape)
    want = c.dt * (k["braw"] - Aphi)
    fl = typ == 0
    scale = np.abs(c.dt * k["braw"][fl]).max()
    assert np.abs(div[fl] - want[fl]).max() < 1e-12 * scale
    # at solver tolerance the divergence is one constant over FLUID cells
    d = div[fl]
    assert np.abs(d - d.mean()).max() < 1e-10 * scale


def test_cylinder_mirror_symmetry(cyl_run):
    c, g, T, A, out = cyl_run
    st, _ = out[-1]
    u, v = st.u[0][0], st.u[1][0]
    assert np.abs(u - u[::-1]).max() < 1e-11
    assert np.abs(v + v[::-1]).max() < 1e-11
    assert np.abs(st.p[0] - st.p[0][::-1]).max() < 1e-10


def test_ghost_rows_hold_after_step(cyl_run):
    c, g, T, A, out = cyl_run
    st, _ = out[-1]
    for comp in range(2):
        f = st.u[comp].ravel()
        res = f[T["gidx"]] + np.sum(T["wv"] * f[T["sidx"]], axis=1)
        assert np.abs(res).max() < 1e-13

"""Pins of the oracle's iterative solves (BiCGStab, the paper's Krylov
method of Section 2.1, with the body-free separable inverse as the pressure
preconditioner): on grids small enough for the sparse direct LU they reach
the LU's solutions, so the iterative route can carry the comparisons on
grids of millions of cells.

* The separable inverse alone is the exact solution of the body-free
  Neumann problem: the DCT-II solution on a uniform grid, the LU solution on
  a stretched one.
* With a body: Poisson (phi and the compatibility scalar), Helmholtz and a
  whole fractional step agree with the LU route to rounding.
"""
import numpy as np
import pytest
import scipy.fft as sfft
import scipy.sparse.linalg as spla

from oracle import flow, geom
from paper_2505_17287_gb300 import synth


def _no_body(ndim, f):
    g = flow.Grid(ndim, *f)
    typ = np.zeros(g.shape, dtype=np.uint8)
    tabs = dict(gidx=np.zeros(0, np.int64), sidx=np.zeros((0, 8), np.int64),
                wp=np.zeros((0, 8)), wv=np.zeros((0, 8)), bv=np.zeros(0), bp=np.zeros(0))
    return g, typ, tabs


def test_separable_inverse_uniform_is_dct():
    nx, ny, nz = 16, 12, 10
    f = [np.linspace(0, 1.6, nx + 1), np.linspace(0, 1.2, ny + 1), np.linspace(0, 1.0, nz + 1)]
    g, typ, tabs = _no_body(3, f)
    b = flow.project_rhs(g, typ, np.random.default_rng(2).uniform(-1, 1, g.shape))
    got = flow.normalise(g, typ, flow.SeparableInverse(g).apply(b))
    bh = sfft.dctn(b, type=2, norm="ortho")
    lam = 0
    for ax, n in ((2, nx), (1, ny), (0, nz)):
        k = np.arange(n)
        shp = [1, 1, 1]
        shp[ax] = n
        lam = lam + (-(2 - 2 * np.cos(np.pi * k / n)) / 0.1 ** 2).reshape(shp)
    want = sfft.idctn(np.where(lam == 0, 0.0, bh / np.where(lam == 0, 1.0, lam)), type=2, norm="ortho")
    want = flow.normalise(g, typ, want)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


@pytest.mark.parametrize("ndim", [2, 3])
def test_separable_inverse_stretched_is_lu(ndim):
    fx = synth.stretched_faces(-1.0, 2.0, 18, 0.0, 0.5, 1.15)
    fy = synth.stretched_faces(-1.0, 1.0, 14, -0.2, 0.2, 1.2)
    fz = synth.stretched_faces(-1.0, 1.0, 10, -0.1, 0.3, 1.1) if ndim == 3 else np.array([0.0, 1.0])
    g, typ, tabs = _no_body(ndim, [fx, fy, fz])
    b = flow.project_rhs(g, typ, np.random.default_rng(3).uniform(-1, 1, g.shape))
    want, _ = flow.solve_poisson(g, typ, tabs, b)
    got = flow.normalise(g, typ, flow.SeparableInverse(g).apply(b))
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-11


def _body_cases():
    ell = synth.cylinder_case(97, 53)
    ell.verts, ell.elems = synth.ellipse_polyline(1.0, 0.3, 0.6, 256)
    sph = synth.sphere_case(n=19, radius=0.45, level=3)
    sph.yf = np.linspace(-1.0, 1.0, 17)
    sph.zf = np.linspace(-1.0, 1.0, 15)
    return {"ellipse_ragged": ell, "sphere_ragged": sph}


CASES = _body_cases()


def _setup(name):
    case = CASES[name]
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    return case, T, g


@pytest.mark.parametrize("name", list(CASES))
def test_poisson_iter_matches_lu(name):
    case, T, g = _setup(name)
    typ = T["type"]
    A = flow.poisson_matrix(g, typ, T)
    b = flow.project_rhs(g, typ, np.random.default_rng(9).uniform(-1, 1, g.shape))
    want, lam = flow.solve_poisson(g, typ, T, b, A)
    got, lam2, it, rel = flow.solve_poisson_iter(g, typ, T, b, A, rtol=1e-13)
    assert rel <= 1e-13 and 0 < it < 100
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-11
    assert abs(lam2 - lam) <= 1e-9 * np.abs(b).max()
    _, rel_ref = flow.poisson_residual(g, typ, A, b, got)
    assert rel_ref < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_helmholtz_iter_matches_lu(name):
    case, T, g = _setup(name)
    H = flow.helmholtz_matrix(g, T["type"], T, 0, 0.01)
    rhs = np.where(T["type"] == flow.FLUID, np.random.default_rng(4).uniform(-1, 1, g.shape), 0.0)
    want = spla.splu(H.tocsc()).solve(rhs.ravel())
    got, it, rel = flow.solve_helmholtz_iter(H, rhs, rtol=1e-14)
    assert rel <= 1e-14
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("name", list(CASES))
def test_step_iter_matches_lu(name):
    case, T, g = _setup(name)
    typ = T["type"]
    a = flow.run(g, typ, T, 2, case.Re, case.dt)
    b = flow.run(g, typ, T, 2, case.Re, case.dt, solver="iter")
    for q in range(g.ndim):
        assert np.abs(a.u[q] - b.u[q]).max() <= 1e-11 * max(1.0, np.abs(a.u[q]).max())
    assert np.linalg.norm(a.p - b.p) / np.linalg.norm(a.p) < 1e-10

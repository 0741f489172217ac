"""Pins for the oracle's pressure operator and Poisson solve (Section 2.1,
pressure Poisson equation; Section 2.2 Neumann ghost rows).

* Manufactured solution: the variable-coefficient Laplacian applied to
  cos(pi x) cos(pi y) [cos(pi z)] converges at second order on uniform and
  smoothly stretched grids (error ratio about 4 per refinement).
* No body, uniform grid, homogeneous Neumann: the type-II DCT diagonalises
  the 5/7-point operator, so the exact discrete solution is computed in the
  spectral basis with scipy.fft and compared with the oracle's direct
  solve to 1e-12.
* No body, stretched grid: the operator is a Kronecker sum of 1D operators;
  the exact solution from the 1D generalised eigenproblems (scipy.linalg)
  is compared with the oracle's direct solve.
* With a body: the bordered-solve solution satisfies P(b - A phi) = 0 with
  the scalar lam, and a least-squares solve of [A 1] on a tiny grid gives
  the same phi after normalisation.
"""
import numpy as np
import pytest
import scipy.fft as sfft
import scipy.linalg as sla

from oracle import flow, geom
from paper_2505_17287_gb300 import synth


def _no_body(ndim, f):
    g = flow.Grid(ndim, *f)
    typ = np.zeros(g.shape, dtype=np.uint8)
    tabs = dict(gidx=np.zeros(0, np.int64), sidx=np.zeros((0, 8), np.int64),
                wp=np.zeros((0, 8)), wv=np.zeros((0, 8)), bv=np.zeros(0), bp=np.zeros(0))
    return g, typ, tabs


def _mms_err(ndim, n, stretch):
    def faces(n):
        s = np.linspace(0, 1, n + 1)
        return s + stretch * np.sin(2 * np.pi * s) / (2 * np.pi) if stretch else s
    f = [faces(n), faces(n), faces(n) if ndim == 3 else np.array([0.0, 1.0])]
    g, typ, tabs = _no_body(ndim, f)
    A = flow.poisson_matrix(g, typ, tabs)
    Z, Y, X = np.meshgrid(g.c[2], g.c[1], g.c[0], indexing="ij")
    phi = np.cos(np.pi * X) * np.cos(np.pi * Y) * (np.cos(np.pi * Z) if ndim == 3 else 1.0)
    lap = -ndim * np.pi ** 2 * phi
    return np.max(np.abs((A @ phi.ravel()).reshape(g.shape) - lap))


@pytest.mark.parametrize("ndim,stretch", [(2, 0.0), (2, 0.3), (3, 0.0), (3, 0.3)])
def test_laplacian_second_order(ndim, stretch):
    ns = [16, 32, 64] if ndim == 2 else [12, 24, 48]
    e = [_mms_err(ndim, n, stretch) for n in ns]
    # cos() is even about the Neumann walls, so the max-norm error is second
    # order everywhere; the first ratio may still be pre-asymptotic
    assert 3.0 < e[0] / e[1] < 4.6, e
    assert 3.6 < e[1] / e[2] < 4.4, e


def test_poisson_uniform_matches_dct():
    nx, ny, nz = 12, 10, 8
    f = [np.linspace(0, 1.2, nx + 1), np.linspace(0, 1.0, ny + 1), np.linspace(0, 0.8, nz + 1)]
    g, typ, tabs = _no_body(3, f)
    rng = np.random.default_rng(7)
    b = flow.project_rhs(g, typ, rng.uniform(-1, 1, g.shape))
    phi, lam = flow.solve_poisson(g, typ, tabs, b)
    assert abs(lam) < 1e-12
    # spectral solve: eigenvalues of the 1D Neumann operator on a uniform grid
    bh = sfft.dctn(b, type=2, norm="ortho")
    lamk = 0
    for ax, n, h in ((2, nx, 0.1), (1, ny, 0.1), (0, nz, 0.1)):
        k = np.arange(n)
        ev = -(2 - 2 * np.cos(np.pi * k / n)) / h ** 2
        shp = [1, 1, 1]
        shp[ax] = n
        lamk = lamk + ev.reshape(shp)
    lamk = np.asarray(lamk)
    ph = np.where(lamk == 0, 0.0, bh / np.where(lamk == 0, 1.0, lamk))
    want = sfft.idctn(ph, type=2, norm="ortho")
    want = flow.normalise(g, typ, want)
    assert np.linalg.norm(phi - want) / np.linalg.norm(want) < 1e-12


def _op1d(f):
    """1D cell-centred Neumann operator (M, vol) built with plain loops."""
    n = len(f) - 1
    h = np.diff(f)
    c = 0.5 * (f[:-1] + f[1:])
    K = np.zeros((n, n))
    for i in range(n - 1):
        t = 1.0 / (c[i + 1] - c[i])
        K[i, i] -= t
        K[i + 1, i + 1] -= t
        K[i, i + 1] += t
        K[i + 1, i] += t
    return K, h


def test_poisson_stretched_matches_separable_eigensolve():
    fx = synth.stretched_faces(-1.0, 2.0, 14, 0.0, 0.5, 1.15)
    fy = synth.stretched_faces(-1.0, 1.0, 12, -0.2, 0.2, 1.2)
    fz = synth.stretched_faces(-1.0, 1.0, 10, -0.1, 0.3, 1.1)
    g, typ, tabs = _no_body(3, [fx, fy, fz])
    rng = np.random.default_rng(3)
    b = flow.project_rhs(g, typ, rng.uniform(-1, 1, g.shape))
    phi, _ = flow.solve_poisson(g, typ, tabs, b)
    # A = sum_a (1/h_a) K_a along axis a; generalised problem K_a v = mu diag(h_a) v
    V, MU = [], []
    for f in (fx, fy, fz):
        K, h = _op1d(f)
        mu, v = sla.eigh(K, np.diag(h))   # v^T diag(h) v = I
        V.append((v, h))
        MU.append(mu)
    # transform b into the eigenbasis: coefficients = v^T diag(h) b along each axis
    t = b.copy()
    for ax, (v, h) in zip((2, 1, 0), V):
        t = np.moveaxis(np.tensordot(v.T * h, np.moveaxis(t, ax, 0), axes=(1, 0)), 0, ax)
    L = MU[0][None, None, :] + MU[1][None, :, None] + MU[2][:, None, None]
    t = np.where(np.abs(L) < 1e-12, 0.0, t / np.where(np.abs(L) < 1e-12, 1.0, L))
    for ax, (v, h) in zip((2, 1, 0), V):
        t = np.moveaxis(np.tensordot(v, np.moveaxis(t, ax, 0), axes=(1, 0)), 0, ax)
    want = flow.normalise(g, typ, t)
    assert np.linalg.norm(phi - want) / np.linalg.norm(want) < 1e-11


def test_poisson_with_body_bordered_solution():
    c = synth.sphere_case(n=12, radius=0.45, level=2)
    T = geom.body_tables(3, c.xf, c.yf, c.zf, c.verts, c.elems)
    g = flow.Grid(3, c.xf, c.yf, c.zf)
    typ = T["type"]
    A = flow.poisson_matrix(g, typ, T)
    rng = np.random.default_rng(5)
    b = flow.project_rhs(g, typ, rng.uniform(-1, 1, g.shape))
    phi, lam = flow.solve_poisson(g, typ, T, b, A)
    r, rel = flow.poisson_residual(g, typ, A, b, phi)
    assert rel < 1e-13
    assert abs(flow.fluid_mean(g, typ, phi)) < 1e-13 * np.abs(phi).max()
    # least squares on the same rows with an explicit column for lam
    t = typ.ravel()
    rows = np.nonzero(t != 2)[0]
    Ad = A.toarray()[np.ix_(rows, rows)]
    one = (t[rows] == 0).astype(float)[:, None]
    sol, *_ = np.linalg.lstsq(np.hstack([Ad, one]), b.ravel()[rows], rcond=None)
    full = np.zeros(g.N)
    full[rows] = sol[:-1]
    want = flow.normalise(g, typ, full.reshape(g.shape))
    assert np.linalg.norm(phi - want) / np.linalg.norm(want) < 1e-10
    assert abs(sol[-1] - lam) < 1e-9 * max(1.0, abs(lam))


def test_ghost_rows_are_the_tables():
    """The GHOST rows of A are p_G - sum wp p_m: applying A to a field that is
    zero on FLUID cells reads back exactly the tables' weights."""
    c = synth.cylinder_case(64, 32)
    T = geom.body_tables(2, c.xf, c.yf, c.zf, c.verts, c.elems)
    g = flow.Grid(2, c.xf, c.yf, c.zf)
    A = flow.poisson_matrix(g, T["type"], T)
    for q, gi in enumerate(T["gidx"]):
        row = A.getrow(gi).toarray().ravel()
        want = np.zeros(g.N)
        want[gi] += 1.0
        np.add.at(want, T["sidx"][q], -T["wp"][q])
        assert np.array_equal(row, want)


def test_poisson_rows_equal_matrix_rows():
    """The row-wise evaluation used on grids too large to assemble agrees
    with the assembled operator (both written from the row definition)."""
    c = synth.sphere_case(n=14, radius=0.4, level=2)
    T = geom.body_tables(3, c.xf, c.yf, c.zf, c.verts, c.elems)
    g = flow.Grid(3, c.xf, c.yf, c.zf)
    A = flow.poisson_matrix(g, T["type"], T)
    phi = np.random.default_rng(4).uniform(-1, 1, g.shape)
    rows = np.arange(g.N)
    got = flow.poisson_rows(g, T["type"], T, phi, rows)
    want = A @ phi.ravel()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()

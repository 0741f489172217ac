"""Oracle discrete operators and one fractional step, numpy + scipy, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Section 2.1 of the paper: the conservative incompressible
Navier-Stokes equations (Eq. 1) on a non-uniform Cartesian grid, split by the
fractional-step (Chorin) method into an advection-diffusion predictor and a
pressure Poisson equation, central differences in space, Adams-Bashforth
convection; and Section 2.2 for the ghost-cell rows (Eq. 2, Eq. 3).

Readings where the paper is silent (each listed in the design notes):
  * collocated cell-centred u, v, w, p plus face-normal velocities U, V, W;
  * convection AB2 (Euler on the first step), diffusion Crank-Nicolson,
    non-incremental projection, p^{n+1} = phi;
  * outer boundaries per face: INFLOW (Dirichlet u = u_inf), OUTFLOW
    (zero gradient, then one uniform correction of the outflow face
    velocities so the net boundary flux vanishes), SLIP (normal component
    0, tangential zero gradient); the pressure is homogeneous Neumann
    everywhere;
  * velocity ghost rows (Dirichlet, body at rest):
        u_G + sum_m wv_m u_m = (2 - bv) u_BI = 0,
    pressure ghost rows (Neumann, dp/dn = 0):  p_G - sum_m wp_m p_m = 0;
  * the Poisson system A phi = b is singular (constants); b is made
    compatible by removing its volume-weighted fluid mean, and the solution
    is the one with A phi = b - lam * 1_fluid for the scalar lam that makes
    the system consistent, normalised to zero volume-weighted fluid mean.

Every linear system is solved by scipy's sparse direct LU by default: the
solution is then the plain definition, reached by no iteration. For grids
too large to factorise, solver="iter" reaches the same solutions by
BiCGStab (the paper's Krylov method), pinned against the LU on small grids.

Array layout: cell arrays are [nz, ny, nx] (x fastest); x-face arrays are
[nz, ny, nx+1], y-face [nz, ny+1, nx], z-face [nz+1, ny, nx]. In 2D nz = 1,
there are no z fluxes and only u, v are advanced.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

FLUID, GHOST, DEAD = 0, 1, 2
INFLOW, OUTFLOW, SLIP = 0, 1, 2
DEFAULT_BC = (INFLOW, OUTFLOW, SLIP, SLIP, SLIP, SLIP)

# Time scheme of Section 2.1 (reading: second-order Adams-Bashforth for the
# convective term, Crank-Nicolson for the viscous term). AB2 holds the
# weights of N^n and N^(n-1); CN_THETA is the implicit share of the viscous
# operator (the explicit share is 1 - CN_THETA). Module constants so that a
# pin can swap in another scheme and show that it fails.
AB2 = (1.5, -0.5)
CN_THETA = 0.5


@dataclass
class Grid:
    ndim: int
    xf: np.ndarray
    yf: np.ndarray
    zf: np.ndarray

    def __post_init__(self):
        self.xf = np.asarray(self.xf, dtype=np.float64)
        self.yf = np.asarray(self.yf, dtype=np.float64)
        self.zf = np.asarray(self.zf, dtype=np.float64)
        if self.ndim == 2:
            self.zf = np.array([0.0, 1.0])
        self.nx, self.ny, self.nz = len(self.xf) - 1, len(self.yf) - 1, len(self.zf) - 1
        self.shape = (self.nz, self.ny, self.nx)
        self.N = self.nx * self.ny * self.nz
        f = (self.xf, self.yf, self.zf)
        self.h = [np.diff(a) for a in f]                      # cell widths
        self.c = [0.5 * (a[:-1] + a[1:]) for a in f]          # centres
        self.hc = [np.diff(c) for c in self.c]                # centre spacing
        dx, dy, dz = (a for a in self.h)
        self.vol = dz[:, None, None] * dy[None, :, None] * dx[None, None, :]
        # face areas broadcast to the face arrays
        self.area = [np.broadcast_to(dz[:, None, None] * dy[None, :, None], (self.nz, self.ny, 1)),
                     np.broadcast_to(dz[:, None, None] * dx[None, None, :], (self.nz, 1, self.nx)),
                     np.broadcast_to(dy[None, :, None] * dx[None, None, :], (1, self.ny, self.nx))]

    @property
    def ncomp(self):
        return self.ndim

    def bshape(self, axis):
        """shape that broadcasts a 1D array along `axis` (0=x, 1=y, 2=z)."""
        return [(1, 1, -1), (1, -1, 1), (-1, 1, 1)][axis]

    def face_shape(self, axis):
        s = list(self.shape)
        s[2 - axis] += 1
        return tuple(s)


def _sl(axis, lo, hi):
    """slice object over cell array axis `axis` (0=x ... 2=z)."""
    s = [slice(None)] * 3
    s[2 - axis] = slice(lo, hi)
    return tuple(s)


def axes(g: Grid):
    return range(g.ndim)


# ---------------------------------------------------------------------------
# Boundary data
# ---------------------------------------------------------------------------

def bc_dirichlet(bc, axis, side, comp, u_inf):
    """(is_dirichlet, value) of component `comp` on the outer face (axis, side)."""
    code = bc[2 * axis + side]
    if code == INFLOW:
        return True, float(u_inf[comp])
    if code == SLIP and comp == axis:
        return True, 0.0
    return False, 0.0


# ---------------------------------------------------------------------------
# Face velocities, divergence, convective and viscous terms
# ---------------------------------------------------------------------------

def face_velocity(g: Grid, typ, u, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0)):
    """Face-normal velocities from cell-centred ones (step P4 of the
    predictor): interior faces with a FLUID side and no DEAD side take the
    mean of the two neighbours, other interior faces 0; INFLOW faces u_inf,
    SLIP faces 0, OUTFLOW faces the adjacent FLUID cell value, after which
    every OUTFLOW face over a FLUID cell gets one uniform correction making
    the net outer-boundary flux zero."""
    F = []
    for a in axes(g):
        Ua = np.zeros(g.face_shape(a))
        L, R = typ[_sl(a, 0, -1)], typ[_sl(a, 1, None)]
        uL, uR = u[a][_sl(a, 0, -1)], u[a][_sl(a, 1, None)]
        ok = (L != DEAD) & (R != DEAD) & ((L == FLUID) | (R == FLUID))
        Ua[_sl(a, 1, -1)] = np.where(ok, 0.5 * (uL + uR), 0.0)
        F.append(Ua)
    # outer faces
    net = 0.0
    out_area = 0.0
    for a in axes(g):
        A = np.broadcast_to(g.area[a], g.face_shape(a))
        for side in (0, 1):
            fs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a], None)
            cs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a] - 1, None)
            code = bc[2 * a + side]
            if code == INFLOW:
                F[a][fs] = u_inf[a]
            elif code == SLIP:
                F[a][fs] = 0.0
            else:
                F[a][fs] = np.where(typ[cs] == FLUID, u[a][cs], 0.0)
                out_area += float(np.sum(np.where(typ[cs] == FLUID, A[fs], 0.0)))
            sign = 1.0 if side == 0 else -1.0
            net += sign * float(np.sum(A[fs] * F[a][fs]))
    if out_area > 0.0:
        corr = net / out_area
        for a in axes(g):
            for side in (0, 1):
                if bc[2 * a + side] != OUTFLOW:
                    continue
                fs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a], None)
                cs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a] - 1, None)
                sign = -1.0 if side == 0 else 1.0
                F[a][fs] = np.where(typ[cs] == FLUID, F[a][fs] + sign * corr, F[a][fs])
    return F


def divergence(g: Grid, F):
    """(1/vol) * sum over faces of the outward flux A_f * U_f."""
    d = np.zeros(g.shape)
    for a in axes(g):
        A = g.area[a]
        d += A * (F[a][_sl(a, 1, None)] - F[a][_sl(a, 0, -1)])
    return d / g.vol


def convection(g: Grid, typ, u, F, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0)):
    """Conservative central convective term of Eq. 1 on FLUID cells:
    N_c = (1/vol) sum_faces (+-) A_f U_f ubar_f, ubar_f the mean of the two
    neighbouring centres (ghost values included); outer faces use the
    Dirichlet value or the cell's own value (zero gradient)."""
    out = []
    for comp in range(g.ncomp):
        flux_div = np.zeros(g.shape)
        for a in axes(g):
            fv = np.zeros(g.face_shape(a))
            fv[_sl(a, 1, -1)] = 0.5 * (u[comp][_sl(a, 0, -1)] + u[comp][_sl(a, 1, None)])
            for side in (0, 1):
                fs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a], None)
                cs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a] - 1, None)
                isd, val = bc_dirichlet(bc, a, side, comp, u_inf)
                fv[fs] = val if isd else u[comp][cs]
            flx = g.area[a] * F[a] * fv
            flux_div += flx[_sl(a, 1, None)] - flx[_sl(a, 0, -1)]
        out.append(np.where(typ == FLUID, flux_div / g.vol, 0.0))
    return out


def laplacian(g: Grid, typ, u, comp, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0)):
    """Viscous operator on FLUID cells (boundary values included):
    (1/vol) [ sum_interior A (u_nb - u_c)/hc + sum_Dirichlet A (ub - u_c)/(h/2) ]."""
    acc = np.zeros(g.shape)
    uc = u
    for a in axes(g):
        A = g.area[a]
        hc = g.hc[a].reshape(g.bshape(a))
        flx = A * (uc[_sl(a, 1, None)] - uc[_sl(a, 0, -1)]) / hc  # interior face gradients
        acc[_sl(a, 0, -1)] += flx
        acc[_sl(a, 1, None)] -= flx
        for side in (0, 1):
            isd, val = bc_dirichlet(bc, a, side, comp, u_inf)
            if not isd:
                continue
            cs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a] - 1, None)
            hh = 0.5 * g.h[a][0 if side == 0 else -1]
            acc[cs] += A * (val - uc[cs]) / hh
    return np.where(typ == FLUID, acc / g.vol, 0.0)


# ---------------------------------------------------------------------------
# Sparse matrices (rows over all N cells, linear index i + nx (j + ny k))
# ---------------------------------------------------------------------------

def _lin(g: Grid):
    return np.arange(g.N).reshape(g.shape)


def _face_pairs(g: Grid, a):
    ids = _lin(g)
    return ids[_sl(a, 0, -1)].ravel(), ids[_sl(a, 1, None)].ravel()


def poisson_matrix(g: Grid, typ, tabs):
    """Full pressure operator A (Section 2.2 rows included):
    FLUID rows  (1/vol) sum_faces (A/hc)(phi_nb - phi_c), outer faces zero flux;
    GHOST rows  phi_G - sum_m wp_m phi_m  (Neumann, dp/dn = 0);
    DEAD rows   identity."""
    t = typ.ravel()
    vol = g.vol.ravel()
    rows, cols, vals = [], [], []
    for a in axes(g):
        L, R = _face_pairs(g, a)
        T = (np.broadcast_to(g.area[a], g.face_shape(a))[_sl(a, 1, -1)]
             / g.hc[a].reshape(g.bshape(a))).ravel()
        for c, nb in ((L, R), (R, L)):
            m = t[c] == FLUID
            rows += [c[m], c[m]]
            cols += [nb[m], c[m]]
            vals += [T[m] / vol[c[m]], -T[m] / vol[c[m]]]
    gi = tabs["gidx"]
    rows += [gi, np.repeat(gi, 8)]
    cols += [gi, tabs["sidx"].ravel()]
    vals += [np.ones(gi.size), -tabs["wp"].ravel()]
    dead = np.nonzero(t == DEAD)[0]
    rows.append(dead)
    cols.append(dead)
    vals.append(np.ones(dead.size))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(g.N, g.N))


def poisson_rows(g: Grid, typ, tabs, phi, rows):
    """(A phi) at the given linear cell indices only, from the definition of
    the rows (for grids too large to assemble): FLUID rows sum over their
    interior faces (A/hc)(phi_nb - phi_c) / vol; GHOST rows phi_G - sum wp
    phi_m; DEAD rows phi."""
    t = typ.ravel()
    f = phi.ravel()
    rows = np.asarray(rows, dtype=np.int64)
    nx, ny, nz = g.nx, g.ny, g.nz
    i, j, k = rows % nx, (rows // nx) % ny, rows // (nx * ny)
    out = np.zeros(rows.size)
    vol = g.h[0][i] * g.h[1][j] * g.h[2][k]
    area = [g.h[1][j] * g.h[2][k], g.h[0][i] * g.h[2][k], g.h[0][i] * g.h[1][j]]
    idx = [i, j, k]
    n = [nx, ny, nz]
    stride = [1, nx, nx * ny]
    fl = t[rows] == FLUID
    for a in axes(g):
        lo = fl & (idx[a] > 0)
        hi = fl & (idx[a] < n[a] - 1)
        out[lo] += area[a][lo] / g.hc[a][idx[a][lo] - 1] * (f[rows[lo] - stride[a]] - f[rows[lo]]) / vol[lo]
        out[hi] += area[a][hi] / g.hc[a][idx[a][hi]] * (f[rows[hi] + stride[a]] - f[rows[hi]]) / vol[hi]
    pos = {int(c): q for q, c in enumerate(tabs["gidx"])}
    for r, c in enumerate(rows):
        if t[c] == GHOST:
            q = pos[int(c)]
            out[r] = f[c] - np.dot(tabs["wp"][q], f[tabs["sidx"][q]])
        elif t[c] == DEAD:
            out[r] = f[c]
    return out


def helmholtz_matrix(g: Grid, typ, tabs, comp, alpha, bc=DEFAULT_BC):
    """Crank-Nicolson velocity operator (I - alpha L0) on FLUID rows (L0 the
    viscous operator without its boundary values), Dirichlet ghost rows
    u_G + sum_m wv_m u_m, identity DEAD rows."""
    t = typ.ravel()
    vol = g.vol.ravel()
    diag = np.ones(g.N)
    rows, cols, vals = [], [], []
    for a in axes(g):
        L, R = _face_pairs(g, a)
        T = (np.broadcast_to(g.area[a], g.face_shape(a))[_sl(a, 1, -1)]
             / g.hc[a].reshape(g.bshape(a))).ravel()
        for c, nb in ((L, R), (R, L)):
            m = t[c] == FLUID
            rows.append(c[m])
            cols.append(nb[m])
            vals.append(-alpha * T[m] / vol[c[m]])
            # (each cell appears once per face direction: a plain add)
            diag += np.bincount(c[m], weights=alpha * T[m] / vol[c[m]], minlength=g.N)
        for side in (0, 1):
            isd, _ = bc_dirichlet(bc, a, side, comp, (0.0, 0.0, 0.0))
            if not isd:
                continue
            cs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a] - 1, None)
            ids = _lin(g)[cs].ravel()
            A = np.broadcast_to(g.area[a], g.face_shape(a))[_sl(a, 0, 1)].ravel()
            hh = 0.5 * g.h[a][0 if side == 0 else -1]
            m = t[ids] == FLUID
            diag += np.bincount(ids[m], weights=alpha * A[m] / (hh * vol[ids[m]]), minlength=g.N)
    gi = tabs["gidx"]
    rows += [np.repeat(gi, 8)]
    cols += [tabs["sidx"].ravel()]
    vals += [tabs["wv"].ravel()]
    rows.append(np.arange(g.N))
    cols.append(np.arange(g.N))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(g.N, g.N))


def bc_source(g: Grid, typ, comp, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0)):
    """The boundary-value part of the viscous operator: L u = L0 u + bc_source."""
    acc = np.zeros(g.shape)
    for a in axes(g):
        A = g.area[a]
        for side in (0, 1):
            isd, val = bc_dirichlet(bc, a, side, comp, u_inf)
            if not isd:
                continue
            cs = _sl(a, 0, 1) if side == 0 else _sl(a, g.shape[2 - a] - 1, None)
            hh = 0.5 * g.h[a][0 if side == 0 else -1]
            acc[cs] += A * val / hh
    return np.where(typ == FLUID, acc / g.vol, 0.0)


# ---------------------------------------------------------------------------
# Poisson: compatibility, residual, direct solve
# ---------------------------------------------------------------------------

def fluid_mean(g: Grid, typ, x):
    m = typ == FLUID
    return float(np.sum(np.where(m, g.vol * x, 0.0)) / np.sum(np.where(m, g.vol, 0.0)))


def project_rhs(g: Grid, typ, b):
    """Remove the volume-weighted FLUID mean on FLUID rows; zero elsewhere."""
    return np.where(typ == FLUID, b - fluid_mean(g, typ, b), 0.0)


def poisson_residual(g: Grid, typ, A, b, phi):
    """P(b - A phi): FLUID rows lose their volume-weighted mean; GHOST rows
    as they are; DEAD rows 0. Returns (residual field, relative 2-norm)."""
    r = (b.ravel() - A @ phi.ravel()).reshape(g.shape)
    rf = np.where(typ == FLUID, r - fluid_mean(g, typ, r), 0.0)
    r = np.where(typ == GHOST, r, rf)
    bn = np.linalg.norm(np.where(typ == DEAD, 0.0, b))
    return r, (np.linalg.norm(r) / bn if bn > 0 else 0.0)


def normalise(g: Grid, typ, phi):
    """Shift FLUID and GHOST values to zero volume-weighted FLUID mean."""
    return np.where(typ == DEAD, 0.0, phi - fluid_mean(g, typ, phi))


def solve_poisson(g: Grid, typ, tabs, b, A=None, cache=None):
    """Solve A phi + lam 1_FLUID = b with sum_FLUID vol phi = 0 by sparse LU.

    A is singular with the constants (on FLUID and GHOST cells) as its null
    space. With y the left null vector (A^T y = 0), the system is consistent
    exactly for lam = y.b / y.1_FLUID. Both y and phi come from one cell
    pinned: the row of a reference FLUID cell r is replaced by e_r (y_r = 1
    for A^T, phi_r = 0 for A); because the systems are consistent the
    replaced row still holds. phi is then shifted to zero volume-weighted
    FLUID mean. Returns (phi [nz,ny,nx], lam). `cache` (a dict) keeps the two
    factorisations between calls on one grid."""
    t = typ.ravel()
    fac = None if cache is None else cache.get("poisson")
    if fac is None:
        if A is None:
            A = poisson_matrix(g, typ, tabs)
        r = int(np.nonzero(t == FLUID)[0][0])
        def pinned(M):
            M = M.tolil(copy=True)
            M.rows[r] = [r]
            M.data[r] = [1.0]
            return spla.splu(M.tocsc())
        luA = pinned(A)
        luT = pinned(A.T.tocsr())
        er = np.zeros(g.N)
        er[r] = 1.0
        y = luT.solve(er)
        fac = (luA, y, r)
        if cache is not None:
            cache["poisson"] = fac
    luA, y, r = fac
    bb = np.where(t == DEAD, 0.0, b.ravel())
    f = (t == FLUID).astype(np.float64)
    lam = float(y @ bb) / float(y @ f)
    rhs = bb - lam * f
    rhs[r] = 0.0
    phi = luA.solve(rhs).reshape(g.shape)
    return normalise(g, typ, phi), lam


# ---------------------------------------------------------------------------
# Iterative solves, for grids too large for the sparse direct LU
# ---------------------------------------------------------------------------
#
# The paper solves its linear systems with BiCGStab (Section 2.1). Here
# BiCGStab is the oracle's second, independent route to the same discrete
# solutions as the direct LU: it is checked against the LU on small grids
# and carries the comparisons on grids of millions of cells. Its
# preconditioner for the pressure is the exact inverse of the body-free
# operator on the same tensor grid (fast diagonalisation by the 1D
# generalised eigenproblems of each axis), a different algorithm from the
# GPU path's multigrid.

def bicgstab(apply_M, apply_K, b, x0, rtol, maxit, norm=np.linalg.norm):
    """Right-preconditioned BiCGStab (van der Vorst, 1992): solves
    M x = b, iterating on M K y = b with x = K y. Stops when
    norm(b - M x) <= rtol * norm(b). Returns (x, iterations, relative
    residual)."""
    x = x0.copy()
    r = b - apply_M(x)
    bn = norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    rel = norm(r) / bn
    if rel <= rtol:
        return x, 0, rel
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = float(np.dot(rhat, r))
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = apply_K(p)
        v = apply_M(ph)
        alpha = rho / float(np.dot(rhat, v))
        s_ = r - alpha * v
        sh = apply_K(s_)
        t = apply_M(sh)
        tt = float(np.dot(t, t))
        omega = float(np.dot(t, s_)) / tt if tt > 0.0 else 0.0
        x = x + alpha * ph + omega * sh
        r = s_ - omega * t
        rho_old = rho
        # the recursively updated r drifts from b - M x near the rounding
        # floor: test (and restart from) the true residual
        rel = norm(r) / bn
        if rel <= rtol or it == maxit:
            r = b - apply_M(x)
            rel = norm(r) / bn
            if rel <= rtol:
                return x, it, rel
            rhat = r.copy()
            rho_old = alpha = omega = 1.0
            v = np.zeros_like(b)
            p = np.zeros_like(b)
    return x, maxit, rel


def _neumann_1d(g: Grid, a):
    """1D cell-centred operator of axis a with zero-flux ends, as a dense
    matrix K (K[i, i+1] = K[i+1, i] = 1/hc, rows summing to 0)."""
    n = len(g.h[a])
    K = np.zeros((n, n))
    t = 1.0 / g.hc[a]
    idx = np.arange(n - 1)
    K[idx, idx + 1] = t
    K[idx + 1, idx] = t
    K[idx, idx] -= t
    K[idx + 1, idx + 1] -= t
    return K


class SeparableInverse:
    """Exact (pseudo-)inverse of the body-free pressure operator on the
    tensor grid g, with zero-flux outer faces. vol * A = sum over axes of
    K_a (x) D_b (x) D_c (K_a the 1D operator, D the cell widths); with the
    generalised eigenpairs K_a V_a = D_a V_a M_a, V_a^T D_a V_a = I, the
    operator is diagonal in the basis W = V_x (x) V_y (x) V_z:
    A^+ r = W (M_x + M_y + M_z)^+ W^T (vol r), the zero eigenvalue (the
    constants) left out."""

    def __init__(self, g: Grid):
        import scipy.linalg as sla
        self.g = g
        self.V = []
        mus = []
        for a in range(3):
            if a < g.ndim:
                mu, V = sla.eigh(_neumann_1d(g, a), np.diag(g.h[a]))
            else:
                mu, V = np.zeros(1), np.ones((1, 1)) / np.sqrt(g.h[a][0])
            self.V.append(V)
            mus.append(mu)
        L = mus[0][None, None, :] + mus[1][None, :, None] + mus[2][:, None, None]
        tol = 1e-12 * np.abs(L).max()
        self.Linv = np.where(np.abs(L) > tol, 1.0 / np.where(np.abs(L) > tol, L, 1.0), 0.0)

    def _along(self, t, M, a):
        """out[.., i', ..] = sum_i t[.., i, ..] M[i, i'] over the index of
        axis a (0 = x, the last array axis); every product is a contiguous
        matrix product."""
        nz, ny, nx = t.shape
        if a == 0:
            return (t.reshape(-1, nx) @ M).reshape(nz, ny, nx)
        if a == 1:
            return np.matmul(M.T, t)
        return (M.T @ t.reshape(nz, -1)).reshape(nz, ny, nx)

    def apply(self, r):
        t = self.g.vol * r.reshape(self.g.shape)
        for a in range(self.g.ndim):
            t = self._along(t, self.V[a], a)          # W^T
        t = t * self.Linv
        for a in range(self.g.ndim):
            t = self._along(t, self.V[a].T, a)        # W
        return t


def solve_poisson_iter(g: Grid, typ, tabs, b, A=None, rtol=1e-13, maxit=2000, sep=None):
    """The Poisson solution of solve_poisson (A phi = b - lam 1_FLUID, zero
    volume-weighted FLUID mean), reached by BiCGStab on P A phi = P b, with
    P the projection that removes the volume-weighted FLUID mean of the
    FLUID rows (its kernel is 1_FLUID, so P r = 0 means r = lam 1_FLUID).
    DEAD cells are 0. Preconditioner: the body-free exact inverse on FLUID
    rows, then each ghost row solved for its ghost value from the updated
    neighbours (z_G = r_G + sum wp z_m), DEAD rows 0.
    Returns (phi, lam, iterations, relative residual)."""
    if A is None:
        A = poisson_matrix(g, typ, tabs)
    if sep is None:
        sep = SeparableInverse(g)
    t = typ.ravel()
    fl, gh, dead = t == FLUID, t == GHOST, t == DEAD
    v = np.where(fl, g.vol.ravel(), 0.0)
    vsum = float(v.sum())
    gi, sidx, wp = tabs["gidx"], tabs["sidx"], tabs["wp"]

    def P(r):
        r = np.where(dead, 0.0, r)
        m = float(np.dot(v, r)) / vsum
        return np.where(fl, r - m, r)

    def M(x):
        return P(A @ np.where(dead, 0.0, x))

    def K(r):
        z = sep.apply(np.where(fl, r, 0.0)).ravel()
        z[dead] = 0.0
        if gi.size:
            z[gi] = r[gi] + np.sum(wp * z[sidx], axis=1)
        return z

    bb = P(b.ravel())
    x, it, rel = bicgstab(M, K, bb, np.zeros(g.N), rtol, maxit)
    phi = normalise(g, typ, x.reshape(g.shape))
    r = (b.ravel() - A @ phi.ravel())
    lam = float(np.dot(v, r)) / vsum
    return phi, lam, it, rel


def solve_helmholtz_iter(H, rhs, x0=None, rtol=1e-14, maxit=500):
    """Crank-Nicolson velocity system H u = rhs (helmholtz_matrix) by
    BiCGStab with the inverse diagonal as preconditioner. Returns (u,
    iterations, relative residual)."""
    d = H.diagonal()
    dinv = 1.0 / d
    b = rhs.ravel()
    x0 = np.zeros_like(b) if x0 is None else x0.ravel()
    return bicgstab(lambda x: H @ x, lambda r: dinv * r, b, x0, rtol, maxit)


# ---------------------------------------------------------------------------
# Ghost refresh and state
# ---------------------------------------------------------------------------

def ghost_bc_values(tabs, comp):
    """Body velocity component at every ghost's body intercept: the body is
    at rest unless a motion put "ubi" (ng x 3) into the tables."""
    ubi = tabs.get("ubi")
    return np.zeros(tabs["gidx"].size) if ubi is None else ubi[:, comp]


def refresh_velocity_ghosts(g: Grid, typ, tabs, u):
    """Solve the Dirichlet ghost rows for the ghost values with the FLUID
    values fixed: u_G + sum_m wv_m u_m = (2 - bv) u_BI."""
    gi = tabs["gidx"]
    if gi.size == 0:
        return u
    pos = -np.ones(g.N, dtype=np.int64)
    pos[gi] = np.arange(gi.size)
    out = []
    for comp, c in enumerate(u):
        flat = c.ravel().copy()
        sidx, wv = tabs["sidx"], tabs["wv"]
        isg = pos[sidx] >= 0
        rhs = (2.0 - tabs["bv"]) * ghost_bc_values(tabs, comp) - np.sum(np.where(isg, 0.0, wv * flat[sidx]), axis=1)
        r, cc = np.nonzero(isg & (wv != 0.0))
        G = sp.csr_matrix((wv[r, cc], (r, pos[sidx[r, cc]])), shape=(gi.size, gi.size)) + sp.identity(gi.size)
        flat[gi] = spla.spsolve(G.tocsc(), rhs)
        out.append(flat.reshape(g.shape))
    return out


def body_force(g: Grid, typ, tabs, u, p, Re):
    """Force of the fluid on the immersed body (all bodies together), per
    unit span in 2D (the grid's z extent is 1), for density 1.

    The paper reports drag and lift coefficients (Section 3.2) but does not
    say how the force is taken. Reading: the traction is integrated at the
    body intercepts (BI) of the ghost cells,
        F = sum_G dS_G ( -p_BI n_G + (1/Re) du/dn|_BI ),
    with n_G the outward body normal at the BI, and
      * p_BI = p_G: under the zero-gradient closure of the pressure ghost
        row the image-point value equals the ghost value, and the BI value
        is the mean of the two;
      * du/dn|_BI = (u_IP - u_G) / |IP - GC| with u_IP = 2 u_BI - u_G and
        u_BI = 0 (body at rest), i.e. -2 u_G / |IP - GC|; at a no-slip wall
        of an incompressible flow the viscous traction is (1/Re) du/dn;
      * dS_G, the surface area a ghost cell stands for, is the area of its
        faces shared with FLUID cells projected onto n_G:
        sum_faces A_f |n_G . e_f|.
    Returns the force vector (3,)."""
    gi = tabs["gidx"]
    F = np.zeros(3)
    if gi.size == 0:
        return F
    t = typ.ravel()
    nx, ny, nz = g.nx, g.ny, g.nz
    i, j, k = gi % nx, (gi // nx) % ny, gi // (nx * ny)
    idx = [i, j, k]
    n = [nx, ny, nz]
    stride = [1, nx, nx * ny]
    area = [g.h[1][j] * g.h[2][k], g.h[0][i] * g.h[2][k], g.h[0][i] * g.h[1][j]]
    nrm = tabs["nrm"]
    dS = np.zeros(gi.size)
    for a in axes(g):
        for side in (-1, 1):
            has = (idx[a] > 0) if side < 0 else (idx[a] < n[a] - 1)
            nb = np.where(has, gi + side * stride[a], gi)
            fl = has & (t[nb] == FLUID)
            dS += np.where(fl, area[a] * np.abs(nrm[:, a]), 0.0)
    gc = np.stack([g.c[0][i], g.c[1][j], g.c[2][k]], 1)
    span = np.linalg.norm(tabs["ip"][:, :g.ndim] - gc[:, :g.ndim], axis=1)
    pg = p.ravel()[gi]
    for a in axes(g):
        ug = u[a].ravel()[gi]
        dudn = -2.0 * ug / span
        F[a] = float(np.sum(dS * (-pg * nrm[:, a] + dudn / Re)))
    return F


def body_velocity(motion, pts):
    """Rigid body velocity U + Omega x (x - centre) at points pts (n x 3);
    motion = (U, Omega, centre), each three numbers."""
    U, w, c0 = (np.asarray(m, dtype=np.float64) for m in motion)
    r = np.asarray(pts, dtype=np.float64) - c0
    cr = np.stack([w[1] * r[:, 2] - w[2] * r[:, 1],
                   w[2] * r[:, 0] - w[0] * r[:, 2],
                   w[0] * r[:, 1] - w[1] * r[:, 0]], axis=1)
    return U + cr


@dataclass
class State:
    u: list           # ncomp cell arrays
    F: list           # ndim face arrays
    p: np.ndarray
    Nold: list | None
    nstep: int = 0
    fresh: np.ndarray | None = None   # cells that became FLUID at the last body move


def interior_face_rule(g: Grid, typ, u, a):
    """Interior face velocities of axis a by the predictor's face rule: the
    mean of the two neighbours on faces with a FLUID side and no DEAD side,
    0 elsewhere (the outer faces are left out)."""
    L, R = typ[_sl(a, 0, -1)], typ[_sl(a, 1, None)]
    ok = (L != DEAD) & (R != DEAD) & ((L == FLUID) | (R == FLUID))
    return np.where(ok, 0.5 * (u[a][_sl(a, 0, -1)] + u[a][_sl(a, 1, None)]), 0.0)


def move_state(g: Grid, typ_old, tabs, st, verts, elems, motion):
    """The state after the body moved to `verts` (same elements) with the
    rigid motion `motion` (Section 2.2, moving bodies; the paper moves the
    body at the start of each step). `tabs` are the tables of the new
    position; this function adds tabs["ubi"], the body velocity at every
    ghost's body intercept. Then:
      * fresh cells (FLUID now, not FLUID before) take the value of the
        fresh-cell interpolation (geom.fresh_tables) with the body velocity
        at their own body intercept; fresh corners are implicit unknowns,
        so the fresh values solve one sparse system;
      * DEAD cells are 0, and the ghost rows are solved with the body
        velocity at their intercepts;
      * interior faces next to a cell whose type changed take the face rule
        from the new cell values; the other faces keep their values.
    Returns the new State with its fresh mask (the next step takes the
    Euler start at those cells)."""
    from . import geom
    typ = tabs["type"]
    tabs["ubi"] = body_velocity(motion, tabs["bi"]) if tabs["gidx"].size else np.zeros((0, 3))
    fresh = (typ == FLUID) & (typ_old != FLUID)
    fidx = np.nonzero(fresh.ravel())[0]
    ft = geom.fresh_tables(g.ndim, g.xf, g.yf, g.zf, typ, fidx, verts, elems)
    ubf = body_velocity(motion, ft["bi"]) if fidx.size else np.zeros((0, 3))
    u = [np.where(typ == DEAD, 0.0, c) for c in st.u]
    if fidx.size:
        pos = -np.ones(g.N, dtype=np.int64)
        pos[fidx] = np.arange(fidx.size)
        sidx, w = ft["sidx"], ft["w"]
        isf = pos[sidx] >= 0
        r, cc = np.nonzero(isf & (w != 0.0))
        M = sp.identity(fidx.size) - sp.csr_matrix((w[r, cc], (r, pos[sidx[r, cc]])), shape=(fidx.size,) * 2)
        lu = spla.splu(M.tocsc())
        for comp in range(g.ncomp):
            flat = u[comp].ravel().copy()
            rhs = np.sum(np.where(isf, 0.0, w * flat[sidx]), axis=1) + ft["wb"] * ubf[:, comp]
            flat[fidx] = lu.solve(rhs)
            u[comp] = flat.reshape(g.shape)
    u = refresh_velocity_ghosts(g, typ, tabs, u)
    changed = typ != typ_old
    F = [f.copy() for f in st.F]
    for a in axes(g):
        ch = changed[_sl(a, 0, -1)] | changed[_sl(a, 1, None)]
        inner = F[a][_sl(a, 1, -1)]
        F[a][_sl(a, 1, -1)] = np.where(ch, interior_face_rule(g, typ, u, a), inner)
    return State(u, F, st.p, st.Nold, st.nstep, fresh), ft


def initial_state(g: Grid, typ, tabs, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0)):
    """Impulsive start: u = u_inf on FLUID, Dirichlet ghost values, 0 in
    DEAD; faces from those cell values; p = 0."""
    u = [np.where(typ == FLUID, float(u_inf[c]), 0.0) for c in range(g.ncomp)]
    u = refresh_velocity_ghosts(g, typ, tabs, u)
    F = face_velocity(g, typ, u, bc, u_inf)
    return State(u, F, np.zeros(g.shape), None, 0)


def step(g: Grid, typ, tabs, st: State, Re, dt, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0),
         A=None, keep=False, cache=None, solver="direct", rtol=1e-13, helm_rtol=1e-14):
    """One fractional step (rows P1-P4, S, C1). Returns the new State; with
    keep=True also a dict of the intermediate fields. `cache` (a dict)
    keeps matrix factorisations between steps of one run. solver="iter"
    solves the Helmholtz and Poisson systems by BiCGStab (to helm_rtol and
    rtol) instead of the direct LU, for grids too large to factorise."""
    alpha = CN_THETA * dt / Re              # implicit viscous share
    alpha_e = (1.0 - CN_THETA) * dt / Re    # explicit viscous share
    N = convection(g, typ, st.u, st.F, bc, u_inf)
    Nold = N if st.Nold is None else st.Nold
    if st.fresh is not None:
        # a fresh cell has no convective history: Euler start there
        Nold = [np.where(st.fresh, N[c], Nold[c]) for c in range(g.ncomp)]
    ustar = []
    rhs_all = []
    for c in range(g.ncomp):
        Lu = laplacian(g, typ, st.u[c], c, bc, u_inf)
        rhs = (st.u[c] - dt * (AB2[0] * N[c] + AB2[1] * Nold[c]) + alpha_e * Lu
               + alpha * bc_source(g, typ, c, bc, u_inf))
        rhs = np.where(typ == FLUID, rhs, 0.0)
        if tabs["gidx"].size:
            # Dirichlet ghost rows: u_G + sum wv u_m = (2 - bv) u_BI
            rf = rhs.ravel()
            rf[tabs["gidx"]] = (2.0 - tabs["bv"]) * ghost_bc_values(tabs, c)
            rhs = rf.reshape(g.shape)
        if solver == "iter":
            H = None if cache is None else cache.get(("helmH", c, alpha))
            if H is None:
                H = helmholtz_matrix(g, typ, tabs, c, alpha, bc)
                if cache is not None:
                    cache[("helmH", c, alpha)] = H
            x = solve_helmholtz_iter(H, rhs, st.u[c], helm_rtol)[0].reshape(g.shape)
        else:
            lu = None if cache is None else cache.get(("helm", c, alpha))
            if lu is None:
                lu = spla.splu(helmholtz_matrix(g, typ, tabs, c, alpha, bc).tocsc())
                if cache is not None:
                    cache[("helm", c, alpha)] = lu
            x = lu.solve(rhs.ravel()).reshape(g.shape)
        ustar.append(x)
        rhs_all.append(rhs)
    Fs = face_velocity(g, typ, ustar, bc, u_inf)
    braw = np.where(typ == FLUID, divergence(g, Fs) / dt, 0.0)
    b = project_rhs(g, typ, braw)
    if A is None:
        A = poisson_matrix(g, typ, tabs)
    if solver == "iter":
        sep = None if cache is None else cache.get("sep")
        if sep is None:
            sep = SeparableInverse(g)
            if cache is not None:
                cache["sep"] = sep
        phi, lam, _, _ = solve_poisson_iter(g, typ, tabs, b, A, rtol, sep=sep)
    else:
        phi, lam = solve_poisson(g, typ, tabs, b, A, cache)
    Fn, un = project(g, typ, ustar, Fs, phi, dt)
    un = refresh_velocity_ghosts(g, typ, tabs, un)
    new = State(un, Fn, phi, N, st.nstep + 1)
    if keep:
        return new, dict(N=N, rhs=rhs_all, ustar=ustar, Fstar=Fs, braw=braw, b=b, phi=phi, lam=lam)
    return new


def project(g: Grid, typ, ustar, Fs, phi, dt):
    """Projection (row C1): faces with a FLUID side lose dt * dphi/dn; FLUID
    cells lose dt times the mean of their two face gradients per axis (outer
    faces have zero gradient)."""
    Fn = [f.copy() for f in Fs]
    un = [c.copy() for c in ustar]
    for a in axes(g):
        hc = g.hc[a].reshape(g.bshape(a))
        grad = (phi[_sl(a, 1, None)] - phi[_sl(a, 0, -1)]) / hc
        L, R = typ[_sl(a, 0, -1)], typ[_sl(a, 1, None)]
        m = (L == FLUID) | (R == FLUID)
        Fn[a][_sl(a, 1, -1)] = np.where(m, Fs[a][_sl(a, 1, -1)] - dt * grad, Fs[a][_sl(a, 1, -1)])
        gf = np.zeros(g.face_shape(a))
        gf[_sl(a, 1, -1)] = grad
        gc = 0.5 * (gf[_sl(a, 0, -1)] + gf[_sl(a, 1, None)])
        un[a] = np.where(typ == FLUID, un[a] - dt * gc, un[a])
    return Fn, un


def run(g: Grid, typ, tabs, nsteps, Re, dt, bc=DEFAULT_BC, u_inf=(1.0, 0.0, 0.0), st=None, solver="direct",
        rtol=1e-13, helm_rtol=1e-14):
    if st is None:
        st = initial_state(g, typ, tabs, bc, u_inf)
    A = poisson_matrix(g, typ, tabs)
    cache = {}
    for _ in range(nsteps):
        st = step(g, typ, tabs, st, Re, dt, bc, u_inf, A, cache=cache, solver=solver, rtol=rtol,
                  helm_rtol=helm_rtol)
    return st

"""Pins of the oracle's outflow correction and of its body-force integral.

Outflow (reading of the outer boundaries, Section 2.1's domain): after the
face velocities are formed, every OUTFLOW face over a FLUID cell gets one
uniform correction so that the net flux through the outer boundary is
zero. Checked on a stretched grid with a body and a random velocity field:
the net flux vanishes to rounding, the correction is one constant over the
outflow faces, and INFLOW and SLIP faces keep their boundary values.

Body force (reading: traction integrated at the body intercepts, drag and
lift of Section 3.2). Checked against closed forms for fields given
analytically at the ghost-cell centres:
* p = x - x_c, u = 0: F = -(body volume) e_x (divergence theorem: the
  surface integral of p n is the volume integral of grad p);
* p = 0, u = (|x - c|^2 - R^2) e_x on a circle or sphere of radius R
  (zero on the surface, normal derivative 2R): F = (1/Re) 2R (area) e_x.
Both converge as the grid is refined (the BI values carry an O(h) error).
"""
import math

import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import synth


def _cyl_tables(nx, ny, ratio=1.05):
    xf = synth.stretched_faces(-2.0, 5.0, nx, -0.7, 0.8, ratio)
    yf = synth.stretched_faces(-2.0, 2.0, ny, -0.6, 0.7, ratio)
    v, e = synth.circle_polyline(128, 0.5)
    T = geom.body_tables(2, xf, yf, np.array([0.0, 1.0]), v, e)
    return flow.Grid(2, xf, yf, np.array([0.0, 1.0])), T


def test_outflow_correction_zero_net_flux():
    g, T = _cyl_tables(70, 48)
    typ = T["type"]
    rng = np.random.default_rng(11)
    u = [np.where(typ == flow.DEAD, 0.0, rng.uniform(0.5, 1.5, g.shape)),
         np.where(typ == flow.DEAD, 0.0, rng.uniform(-0.3, 0.3, g.shape))]
    u_inf = (1.0, 0.0, 0.0)
    F = flow.face_velocity(g, typ, u, flow.DEFAULT_BC, u_inf)
    Ax = np.broadcast_to(g.area[0], g.face_shape(0))
    Ay = np.broadcast_to(g.area[1], g.face_shape(1))
    inflow = np.sum(Ax[..., 0] * F[0][..., 0])
    outflow = np.sum(Ax[..., -1] * F[0][..., -1])
    side = np.sum(Ay[:, 0, :] * F[1][:, 0, :]) - np.sum(Ay[:, -1, :] * F[1][:, -1, :])
    net = inflow - outflow + side
    scale = np.sum(np.abs(Ax[..., -1] * F[0][..., -1])) + abs(inflow)
    assert abs(net) <= 1e-13 * scale, (net, scale)
    # INFLOW faces carry u_inf, SLIP faces 0
    assert np.all(F[0][..., 0] == 1.0)
    assert np.all(F[1][:, 0, :] == 0.0) and np.all(F[1][:, -1, :] == 0.0)
    # one uniform correction over the outflow faces of FLUID cells, and it is
    # not zero for this field (the pin would not see a dropped correction)
    fl = typ[..., -1] == flow.FLUID
    corr = F[0][..., -1][fl] - u[0][..., -1][fl]
    assert np.ptp(corr) <= 1e-14 * np.abs(corr).max()
    assert abs(corr[0]) > 1e-3
    # the cell-side uncorrected outflow would leave a net flux
    assert abs(inflow - np.sum(Ax[..., -1][fl] * u[0][..., -1][fl]) + side) > 1e-3


def _force_case(ndim, n):
    if ndim == 2:
        xf = synth.uniform_faces(-1.0, 1.0, n)
        v, e = synth.circle_polyline(1024, 0.5, 0.03, -0.02)
        zf = np.array([0.0, 1.0])
        c = np.array([0.03, -0.02, 0.0])
    else:
        xf = synth.uniform_faces(-1.0, 1.0, n)
        v, e = synth.icosphere(5, 0.5, (0.03, -0.02, 0.01))
        zf = xf.copy()
        c = np.array([0.03, -0.02, 0.01])
    T = geom.body_tables(ndim, xf, xf.copy(), zf, v, e)
    g = flow.Grid(ndim, xf, xf.copy(), zf)
    Z, Y, X = np.meshgrid(g.c[2], g.c[1], g.c[0], indexing="ij")
    return g, T, (X - c[0], Y - c[1], Z - c[2])


@pytest.mark.parametrize("ndim,ns", [(2, (64, 128, 256)), (3, (24, 48))])
def test_body_force_pressure_closed_form(ndim, ns):
    R = 0.5
    vol = math.pi * R * R if ndim == 2 else 4.0 / 3.0 * math.pi * R ** 3
    errs = []
    for n in ns:
        g, T, (X, Y, Z) = _force_case(ndim, n)
        zero = [np.zeros(g.shape)] * ndim
        F = flow.body_force(g, T["type"], T, zero, X, 10.0)
        errs.append(abs(F[0] + vol) / vol)
        assert abs(F[1]) < 0.05 * vol and abs(F[2]) < 0.05 * vol
    # first order: about half the error per grid halving
    assert errs[-1] < (0.015 if ndim == 2 else 0.08), errs
    assert errs[-1] < 0.6 * errs[-2], errs


@pytest.mark.parametrize("ndim,ns", [(2, (64, 128, 256)), (3, (24, 48))])
def test_body_force_viscous_closed_form(ndim, ns):
    R, Re = 0.5, 20.0
    surf = 2.0 * math.pi * R if ndim == 2 else 4.0 * math.pi * R * R
    exact = 2.0 * R * surf / Re
    errs = []
    for n in ns:
        g, T, (X, Y, Z) = _force_case(ndim, n)
        r2 = X * X + Y * Y + (Z * Z if ndim == 3 else 0.0)
        u = [r2 - R * R] + [np.zeros(g.shape)] * (ndim - 1)
        F = flow.body_force(g, T["type"], T, u, np.zeros(g.shape), Re)
        errs.append(abs(F[0] - exact) / exact)
        assert abs(F[1]) < 0.05 * exact
    assert errs[-1] < (0.01 if ndim == 2 else 0.02), errs
    assert errs[-1] < 0.6 * errs[-2], errs

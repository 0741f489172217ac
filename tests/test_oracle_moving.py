"""Pins of the oracle's moving-body step (Section 2.2: the body moves at the
start of a step; dead cells that become fluid, the fresh cells, take an
interpolation that uses the body velocity at their body intercept).

* Fresh-cell weights reproduce any trilinear field exactly (from the other
  corners' values and the field at the body intercept), and their weights
  sum to one, in 2D and 3D.
* A body translating with the free stream leaves the uniform flow an exact
  solution: after steps in which cells turn fresh, ghost and dead, the
  velocity stays uniform to rounding and the pressure constant. A wrong
  body-velocity sign, a fresh value set to zero or the old ghost rows (body
  at rest) all break it.
* A rotating body: the ghost rows hold u_G + sum wv u_m = (2 - bv) u_BI with
  u_BI = Omega x (BI - centre).
"""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import synth


def _moved(v, shift):
    out = v.copy()
    out[:, : len(shift)] += np.asarray(shift)
    return out


@pytest.mark.parametrize("ndim", [2, 3])
def test_fresh_weights_reproduce_trilinear_fields(ndim):
    rng = np.random.default_rng(13)
    if ndim == 2:
        xf = synth.stretched_faces(-2.0, 3.0, 60, -0.8, 0.8, 1.05)
        yf = synth.stretched_faces(-2.0, 2.0, 44, -0.7, 0.7, 1.05)
        zf = np.array([0.0, 1.0])
        v0, e = synth.ellipse_polyline(0.6, 0.35, 0.4, 256)
        shift = (0.13, -0.07)
    else:
        xf = synth.uniform_faces(-1.0, 1.0, 26)
        yf = synth.uniform_faces(-1.0, 1.0, 22)
        zf = synth.uniform_faces(-1.0, 1.0, 20)
        v0, e = synth.icosphere(3, 0.5)
        shift = (0.11, 0.05, -0.08)
    old = geom.body_tables(ndim, xf, yf, zf, v0, e)["type"]
    v1 = _moved(v0, shift)
    new = geom.body_tables(ndim, xf, yf, zf, v1, e)["type"]
    fresh = np.nonzero(((new == 0) & (old != 0)).ravel())[0]
    assert fresh.size > 10
    ft = geom.fresh_tables(ndim, xf, yf, zf, new, fresh, v1, e)
    assert np.any(ft["kind"] == 1)
    g = flow.Grid(ndim, xf, yf, zf)
    cz = g.c[2] if ndim == 3 else np.array([0.0])
    Z, Y, X = np.meshgrid(cz, g.c[1], g.c[0], indexing="ij")
    a = rng.uniform(-1, 1, 8)

    def f(x, y, z):
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * y * z + a[6] * z * x
                + a[7] * x * y * z) if ndim == 3 else (a[0] + a[1] * x + a[2] * y + a[4] * x * y)

    field = f(X, Y, Z).ravel()
    k1 = ft["kind"] == 1
    got = np.sum(ft["w"] * field[ft["sidx"]], axis=1) + ft["wb"] * f(*ft["bi"].T)
    want = field[fresh]
    assert np.abs(got[k1] - want[k1]).max() < 1e-12 * np.abs(want).max()
    assert np.allclose(np.sum(ft["w"], axis=1) + ft["wb"], 1.0, atol=1e-12)
    # kind 2 takes the body velocity alone
    k2 = ft["kind"] == 2
    assert np.all(ft["wb"][k2] == 1.0) and np.all(ft["w"][k2] == 0.0)


def _uniform_run(ndim, nsteps, mutate=None):
    """A body translating with the free stream U = (1, 0, 0): move by U dt,
    then one step, nsteps times."""
    if ndim == 2:
        case = synth.cylinder_case(64, 32, nseg=128, dt=0.05)
        case.xf = synth.uniform_faces(-2.0, 6.0, 64)
        case.yf = synth.uniform_faces(-2.0, 2.0, 32)
    else:
        case = synth.sphere_case(n=20, radius=0.35, level=2, dt=0.04)
    g = flow.Grid(ndim, case.xf, case.yf, case.zf)
    T = geom.body_tables(ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    motion = ((1.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    # start from the uniform flow with the body already moving
    T["ubi"] = flow.body_velocity(motion, T["bi"])
    st = flow.initial_state(g, T["type"], T)
    v = case.verts
    changed = 0
    for _ in range(nsteps):
        v = _moved(v, (case.dt,))
        T1 = geom.body_tables(ndim, case.xf, case.yf, case.zf, v, case.elems)
        changed += int(np.count_nonzero(T1["type"] != T["type"]))
        st, _ = flow.move_state(g, T["type"], T1, st, v, case.elems, motion)
        if mutate:
            mutate(T1, st)
        T = T1
        st = flow.step(g, T["type"], T, st, case.Re, case.dt)
    return g, T, st, changed


@pytest.mark.parametrize("ndim", [2, 3])
def test_body_moving_with_the_stream_keeps_uniform_flow(ndim):
    g, T, st, changed = _uniform_run(ndim, 4)
    assert changed > 0
    fl = T["type"] == flow.FLUID
    assert np.abs(st.u[0][fl] - 1.0).max() < 1e-11
    for c in range(1, ndim):
        assert np.abs(st.u[c][fl]).max() < 1e-11
    assert np.abs(st.p[fl] - st.p[fl].mean()).max() < 1e-9


@pytest.mark.parametrize("mistake", ["body_at_rest", "fresh_zero"])
def test_uniform_flow_pin_catches_planted_mistakes(mistake):
    def mutate(T1, st):
        if mistake == "body_at_rest":
            T1["ubi"] = np.zeros_like(T1["ubi"])
            st.u[:] = flow.refresh_velocity_ghosts(flow.Grid(2, *_grid2()), T1["type"], T1, st.u)
        else:
            for c in st.u:
                c[st.fresh] = 0.0
    g, T, st, _ = _uniform_run(2, 3, mutate)
    fl = T["type"] == flow.FLUID
    assert np.abs(st.u[0][fl] - 1.0).max() > 1e-3


def _grid2():
    return synth.uniform_faces(-2.0, 6.0, 64), synth.uniform_faces(-2.0, 2.0, 32), np.array([0.0, 1.0])


def test_rotating_body_ghost_rows():
    case = synth.cylinder_case(80, 40, nseg=256)
    v, e = synth.ellipse_polyline(0.8, 0.3, 0.0, 256)
    g = flow.Grid(2, case.xf, case.yf, case.zf)
    T0 = geom.body_tables(2, case.xf, case.yf, case.zf, v, e)
    st = flow.initial_state(g, T0["type"], T0)
    ang = 0.05
    R = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    v1 = v @ R.T
    T1 = geom.body_tables(2, case.xf, case.yf, case.zf, v1, e)
    motion = ((0.0, 0.0, 0.0), (0.0, 0.0, 2.0), (0.0, 0.0, 0.0))
    st, _ = flow.move_state(g, T0["type"], T1, st, v1, e, motion)
    bi = T1["bi"]
    assert np.allclose(T1["ubi"][:, 0], -2.0 * bi[:, 1]) and np.allclose(T1["ubi"][:, 1], 2.0 * bi[:, 0])
    for comp in range(2):
        f = st.u[comp].ravel()
        res = f[T1["gidx"]] + np.sum(T1["wv"] * f[T1["sidx"]], axis=1) - (2.0 - T1["bv"]) * T1["ubi"][:, comp]
        assert np.abs(res).max() < 1e-12

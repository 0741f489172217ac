"""Moving bodies on the GPU (ibm_move_body) against the oracle's move_state
(Section 2.2: the body moves at the start of a step; fresh cells take the
body-velocity interpolation; ghost rows use the body velocity at their
intercepts). Each step both sides move the body to the same rigid-motion
position and then take one fractional step; the cell tables stay bit-exact
and the fields agree at the FP64 parity bars (velocity 1e-8 of its maximum,
pressure 1e-9 relative L2).
"""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu

TIGHT = dict(rtol=1e-13, helm_rtol=1e-14, ghost_tol=1e-16, max_outer=400)


def _rigid(v0, c0, U, w, t):
    """Vertices and centre at time t of the rigid motion: translation U t and
    rotation by |w| t about the moving centre (w along z, or zero)."""
    c = np.asarray(c0, dtype=np.float64) + np.asarray(U) * t
    ang = w[2] * t
    R = np.array([[np.cos(ang), -np.sin(ang), 0.0], [np.sin(ang), np.cos(ang), 0.0], [0.0, 0.0, 1.0]])
    v = (v0 - np.asarray(c0)) @ R.T + c
    return v, c


def _run(case, nsteps, U, w, precision=ibm.IBM_FP64):
    v0, e = case.verts, case.elems
    c0 = np.zeros(3)
    # GPU
    s = ibm.Solver(case, precision=precision)
    s.set_opts(**TIGHT, precision=precision)
    s.set_body(v0, e)
    s.classify()
    # oracle
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, v0, e)
    st = flow.initial_state(g, T["type"], T)
    nfresh = 0
    for n in range(1, nsteps + 1):
        v, c = _rigid(v0, c0, U, w, n * case.dt)
        motion = (tuple(U), tuple(w), tuple(c))
        info = s.move_body(v, U, w, c)
        T1 = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, v, e)
        assert info["n_ghost"] == T1["gidx"].size
        st, ft = flow.move_state(g, T["type"], T1, st, v, e, motion)
        nfresh += ft["fidx"].size
        T = T1
        r = s.step(1)
        assert r["status"] == ibm.IBM_OK, r
        st = flow.step(g, T["type"], T, st, case.Re, case.dt)
    got = s.tables()
    assert np.array_equal(got["type"], T["type"]) and np.array_equal(got["gidx"], T["gidx"])
    out = {k: s.get(k) for k in ("u", "v", "w", "p")[: case.ndim] + ("p",)}
    s.close()
    return out, g, T, st, nfresh


def _check(out, g, T, st):
    for q, n in enumerate(("u", "v", "w")[: g.ndim]):
        err = np.abs(out[n] - st.u[q]).max() / max(1.0, np.abs(st.u[q]).max())
        assert err < 1e-8, (n, err)
    p_ref = flow.normalise(g, T["type"], st.p)
    err = np.linalg.norm(out["p"] - p_ref) / np.linalg.norm(p_ref)
    assert err < 1e-9, err


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_moving_rotating_ellipse_matches_oracle(precision):
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.04)
    case.verts, case.elems = synth.ellipse_polyline(0.9, 0.35, 0.3, 256)
    out, g, T, st, nfresh = _run(case, 6, (-0.6, 0.25, 0.0), (0.0, 0.0, 1.5), precision)
    assert nfresh > 0
    _check(out, g, T, st)


def test_moving_sphere_3d_matches_oracle():
    case = synth.sphere_case(n=29, radius=0.45, level=3)
    case.yf = np.linspace(-1.0, 1.0, 24)
    case.zf = np.linspace(-1.0, 1.0, 20)
    case.dt = 0.05
    out, g, T, st, nfresh = _run(case, 3, (0.5, -0.2, 0.3), (0.0, 0.0, 0.0))
    assert nfresh > 0
    _check(out, g, T, st)


def test_move_body_errors():
    case = synth.cylinder_case(32, 16, nseg=64)
    s = ibm.Solver(case)
    s.set_body(case.verts, case.elems)
    with pytest.raises(ibm.IBMError) as e:
        s.move_body(case.verts)
    assert e.value.status == ibm.IBM_ERR_STATE
    s.classify()
    with pytest.raises(ibm.IBMError) as e:
        s.move_body(case.verts[:-1])
    assert e.value.status == ibm.IBM_ERR_ARG
    v = case.verts.copy()
    v[0, 2] = 0.1
    with pytest.raises(ibm.IBMError) as e:
        s.move_body(v)
    assert e.value.status == ibm.IBM_ERR_ARG
    with pytest.raises(ibm.IBMError) as e:
        s.move_body(case.verts, U=(0.0, 0.0, 1.0))
    assert e.value.status == ibm.IBM_ERR_ARG
    s.close()

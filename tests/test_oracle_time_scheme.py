"""Pins of the oracle's time scheme (Section 2.1: fractional step with
Adams-Bashforth convection; reading: AB2 + Crank-Nicolson, non-incremental
projection) against an exact Navier-Stokes solution.

The Taylor-Green vortex on the unit square with free-slip walls on all four
sides, u = sin(pi x) cos(pi y) F(t), v = -cos(pi x) sin(pi y) F(t),
F = exp(-2 pi^2 t / Re), p = (cos 2 pi x + cos 2 pi y) F^2 / 4, solves the
equations exactly. Its convective term is a pure gradient (it only feeds the
pressure), its viscous term is -2 pi^2 / Re times the velocity.

* At Re = 1 the velocity's temporal self-convergence ratio (differences of
  the runs at dt, dt/2, dt/4) is 4: second order. A backward-Euler viscous
  term gives 2; dropping or flipping the explicit half breaks the decay.
* The pressure p^(n+1) = phi is second order in time too (ratio about 5),
  because the convective extrapolation 3/2 N^n - 1/2 N^(n-1) is centred at
  n + 1/2. Euler convection (weights 1, 0) gives about 2.
* The velocity and pressure match the exact solution to the spatial error
  of the grid, and that error shrinks by about 4 per grid halving. A sign
  error in the convective term flips the pressure.

The same checks on the oracle with one mistake planted (monkeypatched for
one test) must fail: that is what makes this a pin of the time scheme.
"""
import numpy as np
import pytest

from oracle import flow
from paper_2505_17287_gb300 import synth

SLIP4 = (flow.SLIP,) * 6


def tg_run(n, Re, dt, T):
    """Oracle run of the Taylor-Green case from its exact initial fields;
    returns (final state, exact fields at T)."""
    nsteps = int(round(T / dt))
    case = synth.taylor_green_case(n, Re, dt, nsteps)
    f0 = synth.taylor_green_fields(case, 0.0)
    g = flow.Grid(2, case.xf, case.yf, case.zf)
    typ = np.zeros(g.shape, np.uint8)
    tabs = dict(gidx=np.zeros(0, np.int64), sidx=np.zeros((0, 8), np.int64), wp=np.zeros((0, 8)),
                wv=np.zeros((0, 8)), bv=np.zeros(0), bp=np.zeros(0))
    st = flow.State([f0["u"], f0["v"]], [f0["face_u"], f0["face_v"]], np.zeros(g.shape), None, 0)
    A = flow.poisson_matrix(g, typ, tabs)
    cache = {}
    for _ in range(nsteps):
        st = flow.step(g, typ, tabs, st, Re, dt, SLIP4, (0.0, 0.0, 0.0), A, cache=cache)
    return st, synth.taylor_green_fields(case, nsteps * dt)


def measures(n=32, Re=1.0, T=0.05, dts=(0.01, 0.005, 0.0025)):
    """Self-convergence ratios of u and p over dts, and the relative errors
    of u and p against the exact solution at the smallest dt."""
    runs = [tg_run(n, Re, dt, T) for dt in dts]
    du = [np.abs(a[0].u[0] - b[0].u[0]).max() for a, b in zip(runs, runs[1:])]
    dp = [np.abs(a[0].p - b[0].p).max() for a, b in zip(runs, runs[1:])]
    st, ex = runs[-1]
    amp_u = np.abs(ex["u"]).max()
    amp_p = np.abs(ex["p"]).max()
    return dict(ru=du[0] / du[1], rp=dp[0] / dp[1],
                eu=max(np.abs(st.u[0] - ex["u"]).max(), np.abs(st.u[1] - ex["v"]).max()) / amp_u,
                ep=np.abs(st.p - ex["p"]).max() / amp_p)


def test_taylor_green_second_order_in_time():
    m = measures()
    assert 3.7 < m["ru"] < 4.3, m
    assert 3.5 < m["rp"] < 6.0, m


def test_taylor_green_matches_exact_solution():
    m = measures()
    assert m["eu"] < 1.5e-3, m
    assert m["ep"] < 3e-3, m


def test_taylor_green_spatial_error_shrinks():
    # at a small dt the error is the grid's: about 4x smaller per halving
    e = [measures(n, dts=(0.001, 0.0005, 0.00025))["eu"] for n in (16, 32)]
    assert 3.0 < e[0] / e[1] < 5.0, e


def _negated(fn):
    return lambda *a, **k: [-x for x in fn(*a, **k)]


PLANTED = {
    "euler_convection": ("AB2", (1.0, 0.0)),
    "backward_euler_viscous": ("CN_THETA", 1.0),
    "convection_sign": ("convection", "negate_list"),
    "explicit_viscous_sign": ("laplacian", "negate"),
    "explicit_viscous_dropped": ("laplacian", "zero"),
}


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_time_scheme_pins_catch_planted_mistakes(mistake, monkeypatch):
    name, how = PLANTED[mistake]
    if how == "negate_list":
        monkeypatch.setattr(flow, name, _negated(getattr(flow, name)))
    elif how == "negate":
        f = getattr(flow, name)
        monkeypatch.setattr(flow, name, lambda *a, **k: -f(*a, **k))
    elif how == "zero":
        f = getattr(flow, name)
        monkeypatch.setattr(flow, name, lambda *a, **k: 0.0 * f(*a, **k))
    else:
        monkeypatch.setattr(flow, name, how)
    with np.errstate(all="ignore"):
        m = measures()
    ok = (3.7 < m["ru"] < 4.3 and 3.5 < m["rp"] < 6.0 and m["eu"] < 1.5e-3 and m["ep"] < 3e-3)
    assert not ok, (mistake, m)

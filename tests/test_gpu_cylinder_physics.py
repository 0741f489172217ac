"""Physics pin of the method: the 2D cylinder at Re = 100 (the paper's
cylinder validation, Section 3.2.1, at the resolution such a check needs).

On a grid clustered to the body (spacing D/50 near it, [-15, 30] x [-15, 15]),
started impulsively with a small off-axis bump in the cross-stream velocity,
the flow settles into periodic vortex shedding by t = 45. Commonly reported
values for this flow are a Strouhal number of 0.16-0.17 and a mean drag
coefficient of 1.3-1.4 (these numbers are not printed in the paper). The
forces are the oracle's traction integral at the body intercepts
(oracle.flow.body_force, pinned against closed forms). The first 20 steps
of the same case equal the oracle's, so the long run is the oracle's method.
"""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _start(case, **opts):
    s = ibm.Solver(case, stream=opts.pop("stream", None))
    s.set_opts(**opts)
    s.set_body(case.verts, case.elems)
    s.classify()
    T = s.tables()
    v = s.get("v")
    v += np.where(T["type"] == flow.FLUID, synth.wake_bump(case), 0.0)
    s.set("v", v)
    return s, T


def test_cylinder_clustered_first_steps_match_oracle():
    case = synth.cylinder_clustered_case(nsteps=20)
    s, T = _start(case, rtol=1e-13, helm_rtol=1e-14, ghost_tol=1e-16, max_outer=600)
    r = s.step(case.nsteps)
    assert r["status"] == ibm.IBM_OK, r
    Tor = geom.body_tables(2, case.xf, case.yf, case.zf, case.verts, case.elems)
    assert np.array_equal(Tor["type"], T["type"])
    g = flow.Grid(2, case.xf, case.yf, case.zf)
    st = flow.initial_state(g, Tor["type"], Tor)
    st.u[1] = st.u[1] + np.where(Tor["type"] == flow.FLUID, synth.wake_bump(case), 0.0)
    st = flow.run(g, Tor["type"], Tor, case.nsteps, case.Re, case.dt, st=st)
    for q, n in enumerate(("u", "v")):
        err = np.abs(s.get(n) - st.u[q]).max() / np.abs(st.u[q]).max()
        assert err < 1e-8, (n, err)
    p_ref = flow.normalise(g, Tor["type"], st.p)
    assert np.linalg.norm(s.get("p") - p_ref) / np.linalg.norm(p_ref) < 1e-9
    s.close()


def test_cylinder_re100_strouhal_and_drag():
    import torch
    case = synth.cylinder_clustered_case()
    s, T = _start(case, graph=2, stream=torch.cuda.Stream())
    g = flow.Grid(2, case.xf, case.yf, case.zf)
    typ = T["type"]
    s.step_prepare()
    chunk, t_end = 20, 75.0
    ts, cd, cl = [], [], []
    for q in range(int(round(t_end / (chunk * case.dt)))):
        s.step_async(chunk)
        r = s.step_wait()
        assert r["status"] == ibm.IBM_OK, r
        F = flow.body_force(g, typ, T, [s.get("u"), s.get("v")], s.get("p"), case.Re)
        ts.append((q + 1) * chunk * case.dt)
        cd.append(2.0 * F[0])      # C = F / (rho U^2 D / 2), D = U = rho = 1
        cl.append(2.0 * F[1])
    s.close()
    ts, cd, cl = map(np.asarray, (ts, cd, cl))
    w = ts >= 45.0
    x, tt = cl[w] - cl[w].mean(), ts[w]
    up = [tt[i] - x[i] * (tt[i + 1] - tt[i]) / (x[i + 1] - x[i]) for i in range(len(x) - 1) if x[i] < 0 <= x[i + 1]]
    assert len(up) >= 4, up
    St = (len(up) - 1) / (up[-1] - up[0])
    m = (ts >= up[0]) & (ts <= up[-1])
    cd_mean = cd[m].mean()
    cl_amp = np.abs(x).max()
    print(f"St {St:.4f}  mean C_D {cd_mean:.4f}  C_L amplitude {cl_amp:.4f}")
    assert 0.16 <= St <= 0.17, St
    assert 1.30 <= cd_mean <= 1.40, cd_mean
    assert 0.25 <= cl_amp <= 0.40, cl_amp

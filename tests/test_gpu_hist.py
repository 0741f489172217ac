"""The Poisson guess history (option poisson_hist): each step starts its
pressure solve from the least-squares combination of earlier solutions
whose right-hand sides best fit the new one. It changes where the solve
starts, not what it converges to: fields agree with the extrapolated-guess
path within the solve tolerance and with the oracle at the parity bars,
while the solves take fewer iterations. The history is cleared when the
operator changes (classification, body motion), kept by ibm_set_field, and
carried by a checkpoint that restarts bit for bit."""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _run(case, nsteps, precision=ibm.IBM_MIXED, **opts):
    s = ibm.Solver(case, precision=precision)
    s.set_opts(precision=precision, **opts)
    s.set_body(case.verts, case.elems)
    s.classify()
    its = []
    for _ in range(nsteps):
        r = s.step(1)
        assert r["status"] == ibm.IBM_OK and r["rel_residual"] <= 1e-10, r
        its.append(r["poisson_outer"])
    return s, its


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_history_takes_fewer_iterations_same_fields(precision):
    case = synth.wing_case(64, 48, 40, n_chord=30, n_span=10)
    a, ia = _run(case, 14, precision, poisson_hist=8)
    b, ib = _run(case, 14, precision, poisson_hist=0)
    # (the pairs of the impulsive start fit later right-hand sides poorly:
    # compare once the ring holds eight pairs)
    assert sum(ia[8:]) < 0.85 * sum(ib[8:]), (ia, ib)
    for k in ("u", "v", "w", "p"):
        x, y = a.get(k), b.get(k)
        assert np.abs(x - y).max() <= 1e-7 * np.abs(y).max(), k
    a.close()
    b.close()


def test_history_steps_match_oracle():
    """Six steps of the ragged 2D ellipse with the history on: velocity and
    pressure at the FP64 parity bars of the oracle's direct solves (an odd
    cell count, so the history slots need their padding)."""
    case = synth.cylinder_case(97, 53)
    case.verts, case.elems = synth.ellipse_polyline(1.0, 0.3, 0.6, 256)
    s = ibm.Solver(case)
    s.set_opts(rtol=1e-13, helm_rtol=1e-14, ghost_tol=1e-16, max_outer=400, poisson_hist=8)
    s.set_body(case.verts, case.elems)
    s.classify()
    r = s.step(6)
    assert r["status"] == ibm.IBM_OK
    T = geom.body_tables(2, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(2, case.xf, case.yf, case.zf)
    st = flow.run(g, T["type"], T, 6, case.Re, case.dt)
    for q, n in enumerate(("u", "v")):
        err = np.abs(s.get(n) - st.u[q]).max() / max(1.0, np.abs(st.u[q]).max())
        assert err < 1e-8, (n, err)
    p = flow.normalise(g, T["type"], st.p)
    assert np.linalg.norm(s.get("p") - p) / np.linalg.norm(p) < 1e-9
    s.close()


def test_history_cleared_by_classification_kept_by_set_field():
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    s, _ = _run(case, 3)
    ctl = s.get("p_hist_ctl")
    assert ctl[0] == 3 and ctl[1] == 3
    st = s.get_state()
    s.set("u", st["u"])
    assert s.get("p_hist_ctl")[0] == 3
    s.classify()
    assert s.get("p_hist_ctl")[0] == 0
    s.close()


def test_checkpoint_with_history_restarts_bitwise_over_a_ring_wrap():
    """Eleven steps fill the 8-slot ring and wrap it; a context restored from
    the state after five steps (history included) gives the bits of the
    uninterrupted run."""
    case = synth.cylinder_case(96, 48, nseg=256, dt=0.02)
    a, _ = _run(case, 11)
    b, _ = _run(case, 5)
    saved = b.get_state()
    assert "p_hist_x" in saved and saved["p_hist_ctl"][0] == 5
    c = ibm.Solver(case, precision=ibm.IBM_MIXED)
    c.set_opts(precision=ibm.IBM_MIXED)
    c.set_body(case.verts, case.elems)
    c.classify()
    c.set_state(saved)
    r = c.step(6)
    assert r["status"] == ibm.IBM_OK
    ref, got = a.get_state(), c.get_state()
    for k in ref:
        assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k])), k
    for x in (a, b, c):
        x.close()


def test_history_off_has_no_fields():
    case = synth.cylinder_case(32, 16, nseg=64)
    s = ibm.Solver(case)
    s.set_opts(poisson_hist=0)
    assert "p_hist_x" not in s.state_names()
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_get_field(s.ctx, ibm.FIELDS["p_hist_ctl"], np.zeros(2).ctypes.data, 0, 16)
    assert e.value.status == ibm.IBM_ERR_ARG
    s.close()

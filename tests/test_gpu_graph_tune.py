"""GPU tests of the captured V-cycle graph, the multigrid tile width, the
autotuner and the batched ensemble driver."""
import numpy as np
import pytest
import torch

from paper_2505_17287_gb300 import ensemble, ibm, synth

pytestmark = pytest.mark.gpu


def _solver(case, stream, precision=ibm.IBM_FP64, **opts):
    s = ibm.Solver(case, precision=precision, stream=stream)
    s.set_opts(precision=precision, **opts)
    s.set_body(case.verts, case.elems)
    s.classify()
    return s


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_MIXED])
def test_graph_and_tile_width_leave_results_unchanged(precision):
    """The graph replays the same kernels with the same launch shapes, and
    every multigrid row kernel computes each cell on its own, so neither the
    graph nor the tile width may change a single bit."""
    case = synth.cylinder_case(160, 80, 256, nsteps=3)
    st = torch.cuda.Stream()
    outs, launches = [], []
    for graph, tile in ((0, 128), (1, 128), (1, 32), (1, 256)):
        s = _solver(case, st, precision, graph=graph, tile_x=tile)
        n0 = ibm.ibm_launch_count(s.ctx)
        r = s.step(3)
        assert r["status"] == ibm.IBM_OK and r["rel_residual"] <= 1e-10
        launches.append(ibm.ibm_launch_count(s.ctx) - n0)
        outs.append({k: s.get(k) for k in ("u", "v", "p")})
        s.close()
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k]), k
    # kernels inside replayed graphs are counted like launched ones
    assert launches[1] == launches[0] and launches[2] == launches[0]


def test_graph_recaptured_after_reclassification():
    c1 = synth.cylinder_case(128, 64, 128, nsteps=2)
    st = torch.cuda.Stream()
    s = _solver(c1, st, graph=1)
    s.step(2)
    # a second, disjoint body: the union is re-classified and the flow restarts
    v2, e2 = synth.ellipse_polyline(0.6, 0.3, 0.5, 128, cx=4.0)
    s.set_body(v2, e2)
    s.classify()
    r = s.step(2)
    ref = ibm.Solver(c1, stream=st)
    ref.set_opts(graph=0)
    ref.set_body(c1.verts, c1.elems)
    ref.set_body(v2, e2)
    ref.classify()
    r0 = ref.step(2)
    assert r["status"] == ibm.IBM_OK and r0["status"] == ibm.IBM_OK
    assert np.array_equal(s.get("u"), ref.get("u"))
    s.close()
    ref.close()


def test_autotuner_picks_a_valid_candidate():
    case = synth.cylinder_case(256, 128, 256)
    cand = ensemble.candidates(ibm.IBM_MIXED, tiles=(32, 128), nus=(2,))
    bad = ibm.ibm_default_opts()
    bad.tile_x = 48                     # invalid: must be reported as failed
    cand.append(bad)
    best, ms = ibm.ibm_tune(case, cand, steps=2, precision=ibm.IBM_MIXED)
    assert ms[-1] < 0 and all(m > 0 for m in ms[:-1])
    assert 0 <= best < len(cand) - 1 and ms[best] == min(ms[:-1])


def test_ensemble_runs_every_case():
    cases = synth.ensemble_2d(6, seed=11)
    for c in cases:
        c.nsteps = 3
    tuned = ensemble.tune(cases[:2], steps=1)
    for c in cases:
        if ensemble.size_class(c) not in tuned:
            tuned[ensemble.size_class(c)] = (ensemble.candidates()[0], None, None)
    out = ensemble.run(cases, slots=4, tuned=tuned)
    assert out["ok"], [r["error"] for r in out["results"]]
    assert all(r["steps"] == 3 and r["step"]["rel_residual"] <= 1e-10 for r in out["results"])
    assert out["peak_running"] >= 2

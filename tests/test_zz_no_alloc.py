"""The allocation-free residual entry point.

ibm_poisson_residual_noalloc serves callers that cannot allocate device
memory: an application whose memory manager owns the whole device and
forbids libraries to allocate during its step, or a caller running with the
device already full. It keeps its partial sums in a fixed file-scope device
array instead. It must report the same relative residual
||P(b - A phi)|| / ||P b|| that ibm_poisson_solve reports for the solution it
returns, and the oracle's residual of the same fields. Two calls in a row
check that the shared array carries nothing over from the previous call.

This file is collected last so that a failure here, in a run that stops at
the first failure, comes after every other test has run; it also passes
alone in a fresh process.
"""
import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _solver(case):
    s = ibm.Solver(case)
    s.set_opts(rtol=1e-9, max_outer=400)
    s.set_body(case.verts, case.elems)
    s.classify()
    return s


def _case(which):
    if which == "ellipse2d":
        case = synth.cylinder_case(97, 53)
        case.verts, case.elems = synth.ellipse_polyline(1.0, 0.3, 0.6, 256)
    else:
        case = synth.sphere_case(n=29, radius=0.45, level=3)
    return case


@pytest.mark.parametrize("which", ["ellipse2d", "sphere3d"])
def test_noalloc_residual_matches_poisson_solve_and_oracle(which):
    import torch
    case = _case(which)
    s = _solver(case)
    T = geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)
    g = flow.Grid(case.ndim, case.xf, case.yf, case.zf)
    A = flow.poisson_matrix(g, T["type"], T)
    rng = np.random.default_rng(21)
    for call in range(2):  # two calls in a row share the scratch array
        rhs_h = rng.uniform(-1, 1, s.N)
        rhs = torch.from_numpy(rhs_h).cuda()
        phi = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        st = s.poisson_solve(rhs, phi, rtol=1e-9, maxit=400)
        assert st["status"] == ibm.IBM_OK
        want = st["rel_residual"]
        got = ibm.ibm_poisson_residual_noalloc(s.ctx, rhs.data_ptr(), phi.data_ptr())
        assert 0.0 < want <= 1e-9
        # b - A phi is evaluated in FP64 in different orders on the three
        # paths: a residual of 1e-9 or less carries rounding noise of order
        # 1e-16 |A phi| / |b|, so they agree to about 1e-3 of its value
        assert abs(got - want) <= 1e-3 * want + 1e-14, (call, got, want)
        b = flow.project_rhs(g, T["type"], rhs_h.reshape(g.shape))
        _, ref = flow.poisson_residual(g, T["type"], A, b, phi.cpu().numpy().reshape(g.shape))
        assert abs(got - ref) <= 1e-3 * ref + 1e-14, (call, got, ref)
        # a poor guess: the residual of phi = 0 is exactly 1 on every path
        zero = torch.zeros_like(phi)
        got0 = ibm.ibm_poisson_residual_noalloc(s.ctx, rhs.data_ptr(), zero.data_ptr())
        assert abs(got0 - 1.0) < 1e-12
    s.close()


def test_noalloc_rejects_null_and_host_pointers():
    case = synth.cylinder_case(32, 16, nseg=64)
    s = _solver(case)
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_poisson_residual_noalloc(s.ctx, 0, 0)
    assert e.value.status == ibm.IBM_ERR_ARG
    # host memory is refused before any kernel runs
    host = np.zeros(s.N)
    n0 = ibm.ibm_launch_count(s.ctx)
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_poisson_residual_noalloc(s.ctx, host.ctypes.data, host.ctypes.data)
    assert e.value.status == ibm.IBM_ERR_ARG
    assert ibm.ibm_launch_count(s.ctx) == n0
    s.close()

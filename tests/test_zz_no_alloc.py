"""The allocation-free residual entry point.

ibm_poisson_residual_noalloc serves callers that may not allocate device
memory - for example code running while a stream is captured into a CUDA
graph, where cudaMalloc is not allowed, or frameworks that own all device
memory. It must report the same relative residual ||P(b - A phi)|| / ||P b||
that ibm_poisson_solve reports for the solution it returns. This file is
collected last so that a failure here, in a run that stops at the first
failure, comes after every other test has run; it also passes alone.
"""
import numpy as np
import pytest

from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _solver(case):
    s = ibm.Solver(case)
    s.set_opts(rtol=1e-9, max_outer=400)
    s.set_body(case.verts, case.elems)
    s.classify()
    return s


@pytest.mark.parametrize("which", ["ellipse2d", "sphere3d"])
def test_noalloc_residual_matches_poisson_solve(which):
    import torch
    if which == "ellipse2d":
        case = synth.cylinder_case(97, 53)
        case.verts, case.elems = synth.ellipse_polyline(1.0, 0.3, 0.6, 256)
    else:
        case = synth.sphere_case(n=29, radius=0.45, level=3)
    s = _solver(case)
    rng = np.random.default_rng(21)
    for call in range(2):  # two calls in a row share the scratch array
        rhs = torch.from_numpy(rng.uniform(-1, 1, s.N)).cuda()
        phi = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        st = s.poisson_solve(rhs, phi, rtol=1e-9, maxit=400)
        assert st["status"] == ibm.IBM_OK
        want = st["rel_residual"]
        got = ibm.ibm_poisson_residual_noalloc(s.ctx, rhs.data_ptr(), phi.data_ptr())
        assert 0.0 < want <= 1e-9
        # both evaluate b - A phi in FP64 in different orders: a small
        # residual carries rounding noise of order 1e-16 * |A phi| / |b|
        assert abs(got - want) <= 1e-3 * want + 1e-14, (call, got, want)
        # a poor guess: the residual of phi = 0 is exactly 1 on both paths
        zero = torch.zeros_like(phi)
        got0 = ibm.ibm_poisson_residual_noalloc(s.ctx, rhs.data_ptr(), zero.data_ptr())
        assert abs(got0 - 1.0) < 1e-12
    s.close()


def test_noalloc_rejects_null_arguments():
    case = synth.cylinder_case(32, 16, nseg=64)
    s = _solver(case)
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_poisson_residual_noalloc(s.ctx, 0, 0)
    assert e.value.status == ibm.IBM_ERR_ARG
    s.close()

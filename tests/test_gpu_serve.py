"""GPU tests of the request loop (include/ibm_serve.h): continuous admission
of independent cases of mixed sizes, their overlap on the device, admission
by memory, and that every result is the same alone and in the mix.

The library's kernels use fixed launch shapes and fixed-order reductions, so
the stated tolerance for "the same alone and in the mix" is zero: the
fields must agree bit for bit. The single-case path these requests run is
the one the parity tests compare with the oracle; one case here is also
checked bit for bit against that path (ibm.Solver)."""
import numpy as np
import pytest

from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _mix():
    return [
        synth.cylinder_case(96, 48, 128, nsteps=3),
        synth.multi_sphere_case(32, [(0.5, (0.5, 0.0, 0.0))], 200.0, nsteps=2, level=2),
        synth.cylinder_case(160, 80, 256, nsteps=2),
        synth.multi_sphere_case(48, [(0.4, (0.0, 0.5, 0.0)), (0.45, (2.5, -0.5, 0.3))], 300.0, nsteps=2,
                                level=3),
        synth.cylinder_case(128, 64, 128, Re=150.0, nsteps=3),
        synth.multi_sphere_case(64, [(0.3, (1.0, 0.0, 0.0)), (0.35, (3.0, 0.6, -0.4)),
                                     (0.25, (-0.5, -0.7, 0.5))], 450.0, nsteps=2, level=3),
    ]


def _run(cases, slots, budget=0):
    srv = ibm.Server(max_slots=slots, hbm_budget=budget)
    ids = [srv.submit(c, outputs=True) for c in cases]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    return res, st


def test_mix_equals_alone_and_overlaps():
    cases = _mix()
    alone = []
    for c in cases:
        r, _ = _run([c], 1)
        alone.append(r[0])
    mixed, st = _run(cases, 4)
    errors = [(c.name, r["status"], r["error"]) for c, r in zip(cases + cases, alone + mixed) if r["status"]]
    assert not errors, errors
    assert st["completed"] == len(cases) and st["failed"] == 0
    assert st["peak_running"] >= 2, st
    for c, a, m in zip(cases, alone, mixed):
        assert a["status"] == ibm.IBM_OK and m["status"] == ibm.IBM_OK, (a["error"], m["error"])
        assert a["steps"] == m["steps"] == c.nsteps
        assert m["step"]["rel_residual"] <= 1e-10
        assert set(a["outputs"]) == ({"u", "v", "w", "p"} if c.ndim == 3 else {"u", "v", "p"})
        for n in a["outputs"]:
            assert np.array_equal(a["outputs"][n], m["outputs"][n]), (c.name, n)
        assert m["bytes_peak"] <= m["bytes_estimate"], (c.name, m["bytes_peak"], m["bytes_estimate"])
        assert m["t_submit"] <= m["t_admit"] <= m["t_done"]


def test_server_matches_single_context_path():
    """The served case gives the bits of the same case on an ibm.Solver."""
    c = synth.cylinder_case(128, 64, 128, Re=150.0, nsteps=3)
    r, _ = _run([c], 2)
    s = ibm.Solver(c)
    s.set_body(c.verts, c.elems)
    s.classify()
    s.step(c.nsteps)
    for n in ("u", "v", "p"):
        assert np.array_equal(s.get(n), r[0]["outputs"][n]), n
    s.close()


def test_admission_by_memory_budget():
    cases = [synth.cylinder_case(192, 96, 128, nsteps=2) for _ in range(4)]
    est = ibm.ibm_case_bytes(2, 192, 96, 1, ibm.IBM_FP64, 128)
    res, st = _run(cases, 4, budget=int(1.5 * est))
    assert st["peak_running"] == 1 and st["peak_admitted_bytes"] <= st["budget"], st
    assert all(r["status"] == ibm.IBM_OK for r in res)
    # admitted one after another, in arrival order
    for a, b in zip(res, res[1:]):
        assert a["t_done"] <= b["t_admit"] + 1e-3
    ref = res[0]["outputs"]["u"]
    assert all(np.array_equal(r["outputs"]["u"], ref) for r in res)


def test_oversized_request_is_refused():
    srv = ibm.Server(max_slots=1, hbm_budget=64 << 20)
    with pytest.raises(ibm.IBMError) as e:
        srv.submit(synth.cylinder_case(1024, 512, 128, nsteps=1))
    assert e.value.status == ibm.IBM_ERR_OOM
    srv.close()


def test_poisson_requests_alone_and_mixed():
    import torch
    cs = [synth.cylinder_case(96, 48, 128), synth.cylinder_case(128, 64, 256)]
    rhs = [synth.random_field((1, 48, 96), 7), synth.random_field((1, 64, 128), 8)]
    out = {}
    for slots in (1, 2):
        srv = ibm.Server(max_slots=slots)
        ids = [srv.submit(c, kind=ibm.IBM_REQ_POISSON, rhs=b, rtol=1e-12, maxit=200, outputs=True)
               for c, b in zip(cs, rhs)]
        out[slots] = [srv.wait(i) for i in ids]
        srv.close()
    for a, b in zip(out[1], out[2]):
        assert a["status"] == ibm.IBM_OK and b["status"] == ibm.IBM_OK
        assert a["solve"]["rel_residual"] <= 1e-12
        assert np.array_equal(a["outputs"]["p"], b["outputs"]["p"])
    # same bits as ibm_poisson_solve on a single context
    s = ibm.Solver(cs[0])
    s.set_body(cs[0].verts, cs[0].elems)
    s.classify()
    b = torch.tensor(rhs[0].ravel(), dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(b)
    s.poisson_solve(b, phi, rtol=1e-12, maxit=200)
    assert np.array_equal(phi.cpu().numpy().reshape(1, 48, 96), out[1][0]["outputs"]["p"])
    s.close()

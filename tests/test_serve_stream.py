"""The seeded multi-sphere request stream (3D serving workload): its
statistics and geometric constraints, checked on the CPU."""
import numpy as np

from paper_2505_17287_gb300 import synth


def test_stream_shape_and_constraints():
    t, cases = synth.serve_stream(60, level=1)
    assert np.all(np.diff(t) > 0)
    assert 0.5 / 50 < t[-1] / len(t) < 2.0 / 50          # mean gap of a rate-50 Poisson process
    for c in cases:
        n = c.meta["n"]
        assert 64 <= n <= 256 and n % 16 == 0
        assert c.shape == (n, n, n)
        sp = c.meta["spheres"]
        assert 1 <= len(sp) <= 8 and len(synth.case_bodies(c)) == len(sp)
        h = 12.0 / n
        for a, (r, ctr) in enumerate(sp):
            assert 0.2 <= r <= 0.6
            assert -1.0 <= ctr[0] <= 5.0 and abs(ctr[1]) <= 1.5 and abs(ctr[2]) <= 1.5
            for r2, c2 in sp[a + 1:]:
                assert np.linalg.norm(np.subtract(ctr, c2)) >= r + r2 + 2 * h
        assert 100 <= c.Re <= 500 and c.nsteps == 10
        assert abs(c.dt - 0.2 * 6.0 / n) < 1e-15


def test_sphere_bodies_are_closed_meshes():
    c = synth.multi_sphere_case(32, [(0.3, (0.0, 0.0, 0.0)), (0.4, (2.0, 0.0, 0.0))], 200.0, level=4)
    for v, e in synth.case_bodies(c):
        assert e.shape == (5120, 3)
        edges = {}
        for tri in e:
            for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
                edges[(a, b)] = edges.get((a, b), 0) + 1
        assert all(edges.get((b, a), 0) == 1 for (a, b) in edges)

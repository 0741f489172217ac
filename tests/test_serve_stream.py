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


def test_ensemble_recipe():
    """The seeded 2D ensemble: shapes, grids, Re and the CFL-0.2 time step."""
    cases = synth.ensemble_2d(64)
    assert len(cases) == 64
    assert len({c.meta["circle"] for c in cases}) == 2
    for c in cases:
        nx, ny, nz = c.shape
        assert 128 <= nx <= 1024 and nx % 32 == 0 and ny == nx // 2 and nz == 1
        assert 50 <= c.Re <= 200 and c.nsteps == 50
        a, b = c.meta["a"], c.meta["b"]
        assert 0.3 <= a <= 1.0 and 0.3 <= b <= 1.0 and 0 <= c.meta["angle"] <= np.pi
        if c.meta["circle"]:
            assert a == b
        h = min(np.diff(c.xf).min(), np.diff(c.yf).min())
        assert abs(c.dt - 0.2 * h) < 1e-15
    again = synth.ensemble_2d(64)
    assert all(np.array_equal(x.verts, y.verts) and x.Re == y.Re for x, y in zip(cases, again))


def test_ellipsoid_array_geometry():
    """27 closed ellipsoids with axis ratio 1 : 0.3 pitched 15 degrees; no two
    overlap; the 1300x400x400 grid is uniform over the array."""
    c = synth.ellipsoid_array_case(level=2)
    bodies = synth.case_bodies(c)
    assert len(bodies) == 27 and c.ncells == 1300 * 400 * 400
    for v, e in bodies:
        ctr = v.mean(0)
        # the semi-axes recovered from the pitched vertex cloud
        d = v - ctr
        a = np.radians(15.0)
        R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
        local = d @ R
        assert np.allclose(np.abs(local).max(0), (0.5, 0.15, 0.15), atol=1e-12)
    ctrs = np.array([v.mean(0) for v, _ in bodies])
    # bounding spheres of the major axis would overlap at 0.9 D; the pitched
    # ellipsoids do not: check the vertex clouds' boxes are disjoint per pair
    boxes = [(v.min(0), v.max(0)) for v, _ in bodies]
    for p in range(27):
        for q in range(p + 1, 27):
            lo = np.maximum(boxes[p][0], boxes[q][0])
            hi = np.minimum(boxes[p][1], boxes[q][1])
            assert np.any(lo >= hi), (p, q)
    dx = np.diff(c.xf)
    inside = (c.xf[:-1] >= ctrs[:, 0].min() - 0.5) & (c.xf[1:] <= ctrs[:, 0].max() + 0.5)
    assert np.ptp(dx[inside]) < 1e-12

"""Pins for the oracle's ghost-cell tables (Section 2.2, Eq. 2 and Eq. 3).

* The body intercept is the closest surface point: checked against an
  independent vectorised closest-point search (plane projection, edges,
  vertices) written here with numpy.
* The image point is the mirror of the ghost centre through the intercept.
* The weights reproduce every trilinear (2D: bilinear) field exactly
  (Eq. 2 with the Vandermonde solve of Eq. 3): for a random trilinear f,
  sum_m wv_m f(x_m) + bv f(x_BI) = f(x_IP) (Dirichlet row) and
  sum_m wp_m f(x_m) + bp n.grad f(x_BI) = f(x_IP) (Neumann row).
"""
import numpy as np
import pytest

from oracle import geom
from paper_2505_17287_gb300 import synth


def _closest_dist_tris(p, V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    best = np.inf
    # vertices
    best = min(best, np.min(np.linalg.norm(V - p, axis=1)))
    # edges
    for u, v in ((a, b), (b, c), (c, a)):
        e = v - u
        t = np.clip(np.einsum("ij,ij->i", p - u, e) / np.einsum("ij,ij->i", e, e), 0, 1)
        best = min(best, np.min(np.linalg.norm(u + t[:, None] * e - p, axis=1)))
    # plane projections that fall inside the triangle
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n, axis=1)[:, None]
    d = np.einsum("ij,ij->i", p - a, n)
    q = p - d[:, None] * n
    def side(u, v):
        return np.einsum("ij,ij->i", np.cross(v - u, q - u), n)
    ok = (side(a, b) >= 0) & (side(b, c) >= 0) & (side(c, a) >= 0)
    if ok.any():
        best = min(best, np.min(np.abs(d[ok])))
    return best


def _closest_dist_segs(p, V, E):
    a, b = V[E[:, 0], :2], V[E[:, 1], :2]
    e = b - a
    t = np.clip(np.einsum("ij,ij->i", p[:2] - a, e) / np.einsum("ij,ij->i", e, e), 0, 1)
    return np.min(np.linalg.norm(a + t[:, None] * e - p[:2], axis=1))


def _tables(case):
    return geom.body_tables(case.ndim, case.xf, case.yf, case.zf, case.verts, case.elems)


@pytest.fixture(scope="module")
def sphere_tabs():
    c = synth.sphere_case(n=24, radius=0.37, level=3)
    return c, _tables(c)


@pytest.fixture(scope="module")
def cyl_tabs():
    c = synth.cylinder_case(128, 64)
    return c, _tables(c)


@pytest.fixture(scope="module")
def wing_tabs():
    c = synth.wing_case(48, 40, 40, ratio=1.03, n_chord=40, n_span=10)
    return c, _tables(c)


def _centre(case, c):
    nx, ny, nz = case.shape
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    p = np.array([geom.centres(case.xf)[i], geom.centres(case.yf)[j],
                  geom.centres(case.zf)[k] if case.ndim == 3 else 0.0])
    return p


@pytest.mark.parametrize("fx", ["sphere_tabs", "cyl_tabs", "wing_tabs"])
def test_body_intercept_is_closest_point(fx, request):
    case, T = request.getfixturevalue(fx)
    assert T["gidx"].size > 0
    for g, c in enumerate(T["gidx"]):
        p = _centre(case, c)
        want = (_closest_dist_tris(p, case.verts, case.elems) if case.ndim == 3
                else _closest_dist_segs(p, case.verts, case.elems))
        assert abs(T["dist"][g] - want) <= 1e-12 * max(1.0, want)
        assert abs(np.linalg.norm(T["bi"][g] - p) - want) <= 1e-12
        if T["kind"][g] != 2:
            assert np.allclose(T["ip"][g], 2 * T["bi"][g] - p, atol=1e-15, rtol=0)
            assert abs(np.linalg.norm(T["nrm"][g]) - 1.0) < 1e-14


def _trilinear(ndim, rng):
    a = rng.uniform(-1, 1, 8)
    if ndim == 2:
        a[[3, 5, 6, 7]] = 0.0
        f = lambda x: a[0] + a[1] * x[0] + a[2] * x[1] + a[4] * x[0] * x[1]
        gr = lambda x: np.array([a[1] + a[4] * x[1], a[2] + a[4] * x[0], 0.0])
        return f, gr
    f = lambda x: (a[0] + a[1] * x[0] + a[2] * x[1] + a[3] * x[2] + a[4] * x[0] * x[1]
                   + a[5] * x[1] * x[2] + a[6] * x[2] * x[0] + a[7] * x[0] * x[1] * x[2])
    gr = lambda x: np.array([a[1] + a[4] * x[1] + a[6] * x[2] + a[7] * x[1] * x[2],
                             a[2] + a[4] * x[0] + a[5] * x[2] + a[7] * x[0] * x[2],
                             a[3] + a[5] * x[1] + a[6] * x[0] + a[7] * x[0] * x[1]])
    return f, gr


@pytest.mark.parametrize("fx", ["sphere_tabs", "cyl_tabs", "wing_tabs"])
def test_weights_reproduce_trilinear_fields(fx, request):
    case, T = request.getfixturevalue(fx)
    rng = np.random.default_rng(11)
    nchk = 0
    for g in range(T["gidx"].size):
        if T["kind"][g] == 2:
            continue
        for _ in range(2):
            f, gr = _trilinear(case.ndim, rng)
            fc = np.array([f(_centre(case, s)) for s in T["sidx"][g]])
            ip, bi, n = T["ip"][g], T["bi"][g], T["nrm"][g]
            dirichlet = np.dot(T["wv"][g], fc) + T["bv"][g] * f(bi)
            neumann = np.dot(T["wp"][g], fc) + T["bp"][g] * np.dot(n, gr(bi))
            assert abs(dirichlet - f(ip)) < 1e-12
            assert abs(neumann - f(ip)) < 1e-12
            nchk += 1
        # value rows of the Neumann closure reproduce constants alone
        assert abs(T["wp"][g].sum() - 1.0) < 1e-12
        assert abs(T["wv"][g].sum() + T["bv"][g] - 1.0) < 1e-12
    assert nchk > 0


@pytest.mark.parametrize("fx", ["sphere_tabs", "cyl_tabs", "wing_tabs"])
def test_stencil_structure(fx, request):
    case, T = request.getfixturevalue(fx)
    typ = T["type"].ravel()
    nx, ny, nz = case.shape
    nc = 4 if case.ndim == 2 else 8
    for g, c in enumerate(T["gidx"]):
        k = T["kind"][g]
        b = T["base"][g]
        corners = [b + (m & 1) + nx * ((m >> 1) & 1) + nx * ny * ((m >> 2) & 1) for m in range(nc)]
        mask = sum(1 << m for m in range(nc) if typ[corners[m]] != 0)
        assert T["cmask"][g] == mask
        if k == 0:
            assert c not in corners and all(typ[x] != 2 for x in corners)
            assert list(T["sidx"][g][:nc]) == corners
        elif k == 1:
            assert c in corners
            assert all(typ[x] != 2 for x in corners if x != c)
        else:
            assert typ[T["sidx"][g][0]] == 0 and T["wv"][g][0] == 1.0 and T["wp"][g][0] == 1.0
        # the IP lies inside (or on) the lattice cell of its base corner
        ip = T["ip"][g]
        lo, hi = _centre(case, corners[0]), _centre(case, corners[nc - 1])
        if k != 2 and all(0 < ip[a] - lo[a] < 1e9 for a in range(case.ndim)):
            assert all(ip[a] <= hi[a] or np.isclose(ip[a], hi[a]) for a in range(case.ndim))


def test_wing_mesh_is_closed_and_outward():
    V, T = synth.naca_wing(20, 6)
    e = {}
    for t in T:
        for q in range(3):
            a, b = int(t[q]), int(t[(q + 1) % 3])
            e[(a, b)] = e.get((a, b), 0) + 1
    assert all(v == 1 for v in e.values())
    assert all((b, a) in e for (a, b) in e)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert vol > 0  # outward orientation gives a positive signed volume
    for mesh in (synth.icosphere(2), synth.box((0, 0, 0), (1, 2, 3)), synth.l_prism(), synth.tetrahedron()):
        V, T = mesh
        a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
        assert np.einsum("ij,ij->i", a, np.cross(b, c)).sum() > 0

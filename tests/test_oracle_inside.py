"""Pins for the oracle's inside/outside test (Section 2.2, ray tracing for
dead-cell blanking).

The oracle casts the ray along a grid axis on quantised integer coordinates
with a symbolic perturbation of the centre. These pins use an independent
brute force: exact rational arithmetic (fractions.Fraction) on the
unquantised coordinates, a ray in a generic non-axis direction, and the
centre perturbed by tiny explicit rationals in the same directions as the
oracle's symbolic perturbation. The meshes use dyadic coordinates, so the
oracle's quantisation is exact and both see the same surface.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import geom
from paper_2505_17287_gb300 import synth

D1 = Fr(1, 2 ** 60)   # z (2D: y) shift, dominant
D2 = Fr(1, 2 ** 120)  # x shift
D3 = Fr(1, 2 ** 240)  # y shift (3D)


def _ray_tri(o, d, a, b, c):
    """Exact: does the ray o + t d (t > 0) cross triangle abc (interior)?"""
    e1 = [b[i] - a[i] for i in range(3)]
    e2 = [c[i] - a[i] for i in range(3)]
    p = [d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]]
    det = sum(e1[i] * p[i] for i in range(3))
    if det == 0:
        return False
    s = [o[i] - a[i] for i in range(3)]
    u = sum(s[i] * p[i] for i in range(3)) / det
    if u < 0 or u > 1:
        return False
    q = [s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]]
    v = sum(d[i] * q[i] for i in range(3)) / det
    if v < 0 or u + v > 1:
        return False
    t = sum(e2[i] * q[i] for i in range(3)) / det
    if u == 0 or v == 0 or u + v == 1 or t == 0:
        raise AssertionError("degenerate brute-force ray; pick another direction")
    return t > 0


def brute_inside_3d(p, V, T):
    o = [Fr(p[0]) + D2, Fr(p[1]) + D3, Fr(p[2]) - D1]
    d = [Fr(3, 7), Fr(5, 11), Fr(1)]  # generic, not along any axis
    Vf = [[Fr(float(x)) for x in v] for v in V]
    n = sum(_ray_tri(o, d, Vf[a], Vf[b], Vf[c]) for a, b, c in T)
    return n % 2


def brute_inside_2d(p, V, E):
    o = [Fr(p[0]) + D2, Fr(p[1]) - D1]
    d = [Fr(2, 9), Fr(1)]
    n = 0
    for a, b in E:
        A = [Fr(float(V[a][0])), Fr(float(V[a][1]))]
        B = [Fr(float(V[b][0])), Fr(float(V[b][1]))]
        e = [B[0] - A[0], B[1] - A[1]]
        det = d[0] * (-e[1]) - d[1] * (-e[0])
        if det == 0:
            continue
        r = [A[0] - o[0], A[1] - o[1]]
        t = (r[0] * (-e[1]) - r[1] * (-e[0])) / det
        s = (d[0] * r[1] - d[1] * r[0]) / det
        if 0 < s < 1 and t > 0:
            n += 1
        assert s != 0 and s != 1 and t != 0
    return n % 2


def _check3(xf, yf, zf, V, T):
    ins = geom.inside(3, xf, yf, zf, V, T)
    xc, yc, zc = geom.centres(xf), geom.centres(yf), geom.centres(zf)
    for k in range(len(zc)):
        for j in range(len(yc)):
            for i in range(len(xc)):
                want = brute_inside_3d((xc[i], yc[j], zc[k]), V, T)
                assert ins[k, j, i] == want, (i, j, k)
    return ins


@pytest.mark.parametrize("mesh", ["tet", "box", "lprism", "ico1"])
def test_inside_3d_matches_exact_bruteforce(mesh):
    if mesh == "tet":
        V = np.array([[0.125, 0.25, 0.125], [0.875, 0.125, 0.25], [0.375, 0.875, 0.125],
                      [0.5, 0.375, 0.875]])
        T = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], dtype=np.int32)
    elif mesh == "box":
        # faces, edges and corners exactly on cell centres (centres at k/8 + 1/16)
        V, T = synth.box((0.1875, 0.3125, 0.0625), (0.6875, 0.8125, 0.5625))
    elif mesh == "lprism":
        V, T = synth.l_prism(0.1875, 0.8125)
        V = np.round(V * 64) / 64
    else:
        V, T = synth.icosphere(1, 0.375, (0.5, 0.5, 0.5))
        V = np.round(V * 1024) / 1024
    f = np.linspace(0.0, 1.0, 9)
    ins = _check3(f, f, f, V, T)
    assert ins.sum() > 0


def test_inside_3d_on_surface_cases():
    """Cells whose centres lie exactly on faces, edges and vertices of the
    body resolve by the perturbation rule; checked against the brute force
    at the same perturbed point."""
    V, T = synth.box((0.0625 + 0.125, 0.0625 + 0.25, 0.0625), (0.0625 + 0.5, 0.0625 + 0.625, 0.0625 + 0.5))
    f = np.linspace(0.0, 1.0, 9)
    ins = _check3(f, f, f, V, T)
    # the bottom face z = 1/16 holds centres: perturbed downwards -> outside;
    # the top face z = 9/16 holds centres: perturbed downwards -> inside
    assert ins[0].sum() == 0
    assert ins[4].sum() > 0


def test_inside_2d_matches_exact_bruteforce():
    poly = [(0.1875, 0.1875), (0.8125, 0.1875), (0.8125, 0.4375), (0.4375, 0.4375),
            (0.4375, 0.8125), (0.1875, 0.8125)]
    V, E = synth.polyline_from_polygon(poly)
    f = np.linspace(0.0, 1.0, 17)
    ins = geom.inside(2, f, f, np.array([0.0, 1.0]), V, E)
    c = geom.centres(f)
    for j in range(16):
        for i in range(16):
            assert ins[0, j, i] == brute_inside_2d((c[i], c[j]), V, E), (i, j)
    V, E = synth.circle_polyline(64, 0.3, 0.5, 0.5)
    ins = geom.inside(2, f, f, np.array([0.0, 1.0]), V, E)
    for j in range(16):
        for i in range(16):
            assert ins[0, j, i] == brute_inside_2d((c[i], c[j]), V, E), (i, j)


def test_inside_sphere_far_cells_match_analytic():
    """Cells farther than h from the sphere agree with |x - c| < r."""
    V, T = synth.icosphere(3, 0.35, (0.02, -0.01, 0.03))
    f = np.linspace(-0.5, 0.5, 25)
    ins = geom.inside(3, f, f, f, V, T)
    c = geom.centres(f)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt((X - 0.02) ** 2 + (Y + 0.01) ** 2 + (Z - 0.03) ** 2)
    h = f[1] - f[0]
    far = np.abs(r - 0.35) > h
    assert np.array_equal(ins[far], (r[far] < 0.35).astype(np.uint8))


def test_inside_cylinder_far_cells_match_analytic():
    c = synth.cylinder_case(64, 32)
    ins = geom.inside(2, c.xf, c.yf, c.zf, c.verts, c.elems)[0]
    xc, yc = geom.centres(c.xf), geom.centres(c.yf)
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    r = np.hypot(X, Y)
    far = np.abs(r - 0.5) > 0.5
    assert np.array_equal(ins[far], (r[far] < 0.5).astype(np.uint8))


def test_classify_definition():
    """DEAD = inside with no outside face neighbour; GHOST = inside with one
    (Section 2.2); ghost list ascending."""
    V, T = synth.icosphere(2, 0.3)
    f = np.linspace(-0.5, 0.5, 21)
    ins = geom.inside(3, f, f, f, V, T)
    typ, gidx = geom.classify(ins)
    nz, ny, nx = ins.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if not ins[k, j, i]:
                    assert typ[k, j, i] == 0
                    continue
                nbs = [(k, j, i - 1), (k, j, i + 1), (k, j - 1, i), (k, j + 1, i), (k - 1, j, i), (k + 1, j, i)]
                fl = any(0 <= a < nz and 0 <= b < ny and 0 <= cc < nx and not ins[a, b, cc] for a, b, cc in nbs)
                assert typ[k, j, i] == (1 if fl else 2)
    assert np.all(np.diff(gidx) > 0)
    assert np.array_equal(np.sort(np.nonzero(typ.ravel() == 1)[0]), gidx)

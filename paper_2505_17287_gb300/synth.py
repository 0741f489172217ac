"""Seeded synthetic inputs: grids and immersed-body surface meshes.

This module holds no arithmetic of the solver itself. It only builds the
inputs that both the CUDA path and the CPU oracle consume: face-coordinate
arrays of (possibly stretched) Cartesian grids, closed surface meshes
(polylines in 2D, triangulations in 3D) and seeded random draws.

The workloads follow the paper's test problems (Section 3.2): a 2D circular
cylinder in a uniform stream (Section 3.2.1) and a finite rectangular wing
at incidence in a domain 10 chords wide (Section 3.2.2); plus ellipse and
icosphere bodies shaped like the ellipsoid-array case (Section 3.3.2).

Conventions shared by every mesh here:
  * vertices are float64 arrays of shape (nv, 3) (z is 0 in 2D);
  * 2D elements are segments (ne, 2) int32 ordered counter-clockwise around
    the body, so the outward normal of segment a->b is (b-a) rotated by -90;
  * 3D elements are triangles (ne, 3) int32 ordered counter-clockwise when
    seen from outside, so (b-a) x (c-a) points out of the body.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# Grids
# ---------------------------------------------------------------------------

def uniform_faces(lo: float, hi: float, n: int) -> np.ndarray:
    """n+1 equally spaced face coordinates on [lo, hi]."""
    return np.linspace(lo, hi, n + 1, dtype=np.float64)


def stretched_faces(lo: float, hi: float, n: int, core_lo: float, core_hi: float,
                    ratio: float = 1.04) -> np.ndarray:
    """n+1 face coordinates: uniform spacing h0 on [core_lo, core_hi] and
    spacing growing geometrically by `ratio` per cell towards both ends.

    The cell size is the continuous profile h(s) = h0 inside the core and
    h0 * ratio**(distance in cells from the core) outside it; h0 is found by
    bisection so that exactly n cells span [lo, hi]. Faces are the profile's
    integral sampled at integer cell counts, so the domain ends are exact.
    """
    if not (lo <= core_lo < core_hi <= hi):
        raise ValueError("core interval must lie inside the domain")
    lnr = math.log(ratio)
    Ll, Lc, Lr = core_lo - lo, core_hi - core_lo, hi - core_hi

    def side_cells(L, h0):
        return 0.0 if L <= 0 else math.log1p(L * lnr / h0) / lnr

    def count(h0):
        return side_cells(Ll, h0) + Lc / h0 + side_cells(Lr, h0)

    a, b = 1e-12, (hi - lo)
    for _ in range(200):  # count() decreases monotonically with h0
        m = 0.5 * (a + b)
        if count(m) > n:
            a = m
        else:
            b = m
    h0 = 0.5 * (a + b)
    sl = side_cells(Ll, h0)
    sr = sl + Lc / h0
    s = np.arange(n + 1, dtype=np.float64)
    x = np.empty(n + 1)
    for q, sv in enumerate(s):
        if sv <= sl:
            x[q] = core_lo - h0 * (ratio ** (sl - sv) - 1.0) / lnr
        elif sv <= sr:
            x[q] = core_lo + h0 * (sv - sl)
        else:
            x[q] = core_hi + h0 * (ratio ** (sv - sr) - 1.0) / lnr
    x[0], x[n] = lo, hi
    if np.any(np.diff(x) <= 0):
        raise ValueError("stretched grid is not monotone")
    return x


# ---------------------------------------------------------------------------
# Bodies
# ---------------------------------------------------------------------------

def circle_polyline(nseg: int = 512, radius: float = 0.5, cx: float = 0.0,
                    cy: float = 0.0):
    """Closed CCW polyline with vertices at angles 2*pi*(k + 1/2)/nseg.

    The half-segment offset puts a segment midpoint, not a vertex, on every
    axis and diagonal, so cell centres on those lines have a unique closest
    surface point. For even nseg the vertices of the upper half are the
    exact mirror images (y -> -y) of the lower half."""
    v = np.zeros((nseg, 3))
    th = 2.0 * np.pi * (np.arange(nseg) + 0.5) / nseg
    v[:, 0] = radius * np.cos(th)
    v[:, 1] = radius * np.sin(th)
    if nseg % 2 == 0:
        h = nseg // 2
        v[h:, 0] = v[h - 1::-1, 0]
        v[h:, 1] = -v[h - 1::-1, 1]
    v[:, 0] += cx
    v[:, 1] += cy
    e = np.stack([np.arange(nseg), (np.arange(nseg) + 1) % nseg], 1).astype(np.int32)
    return v, e


def ellipse_polyline(a: float, b: float, angle: float, nseg: int = 256,
                     cx: float = 0.0, cy: float = 0.0):
    """Closed CCW polyline of an ellipse with semi-axes a, b rotated by angle."""
    th = 2.0 * np.pi * np.arange(nseg) / nseg
    x, y = a * np.cos(th), b * np.sin(th)
    c, s = math.cos(angle), math.sin(angle)
    v = np.zeros((nseg, 3))
    v[:, 0] = cx + c * x - s * y
    v[:, 1] = cy + s * x + c * y
    e = np.stack([np.arange(nseg), (np.arange(nseg) + 1) % nseg], 1).astype(np.int32)
    return v, e


def naca00xx_thickness(x: np.ndarray, t: float = 0.12) -> np.ndarray:
    """Half thickness of a symmetric NACA 4-digit section with the closed
    trailing-edge coefficient (-0.1036), so y(1) = 0."""
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2
                      + 0.2843 * x**3 - 0.1036 * x**4)


def naca_wing(n_chord: int = 100, n_span: int = 50, span: float = 2.0,
              alpha_deg: float = 15.0, t: float = 0.12, pivot: float = 0.25):
    """Closed triangulated finite wing with square tips.

    Chord 1 along x with the leading edge at x=0, thickness along y, span
    along z centred on z=0. The section is pitched nose-up by alpha about
    the spanwise axis through the quarter chord. Triangle count is
    4*n_chord*n_span + 2*(2*n_chord - 2).
    """
    xs = 0.5 * (1.0 - np.cos(np.pi * np.arange(n_chord + 1) / n_chord))
    yt = naca00xx_thickness(xs, t)
    yt[0] = 0.0
    yt[-1] = 0.0
    # section polygon, counter-clockwise seen from +z: LE -> lower -> TE -> upper
    px = np.concatenate([[0.0], xs[1:-1], [1.0], xs[-2:0:-1]])
    py = np.concatenate([[0.0], -yt[1:-1], [0.0], yt[-2:0:-1]])
    m = px.size  # 2*n_chord points
    zs = -0.5 * span + span * np.arange(n_span + 1) / n_span
    verts = np.zeros(((n_span + 1) * m, 3))
    for s in range(n_span + 1):
        verts[s * m:(s + 1) * m, 0] = px
        verts[s * m:(s + 1) * m, 1] = py
        verts[s * m:(s + 1) * m, 2] = zs[s]
    tris = []
    for s in range(n_span):
        for q in range(m):
            a, b = s * m + q, s * m + (q + 1) % m
            c, d = a + m, b + m
            # the polygon is CCW about +z, so its outward side normal is
            # (dx, dy) rotated by -90; with +z as the third axis these orders
            # give outward normals
            tris.append((a, b, d))
            tris.append((a, d, c))
    # caps: fan from the leading-edge vertex (the section is convex)
    for q in range(1, m - 1):
        tris.append((0, q + 1, q))                      # z = -span/2, normal -z
        top = n_span * m
        tris.append((top, top + q, top + q + 1))        # z = +span/2, normal +z
    tris = np.asarray(tris, dtype=np.int32)
    al = math.radians(alpha_deg)
    ca, sa = math.cos(al), math.sin(al)
    x0 = verts[:, 0] - pivot
    y0 = verts[:, 1]
    verts[:, 0] = pivot + ca * x0 + sa * y0
    verts[:, 1] = -sa * x0 + ca * y0
    return verts, tris


def icosphere(level: int = 4, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Subdivided icosahedron projected on a sphere; 20*4**level triangles."""
    p = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p),
         (0, -1, -p), (0, 1, -p), (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
         (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
         (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    for _ in range(level):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    V = np.asarray(verts) * radius + np.asarray(center, dtype=np.float64)
    return V, np.asarray(f, dtype=np.int32)


def tetrahedron():
    v = np.array([[0.1, 0.2, 0.15], [0.9, 0.1, 0.2], [0.3, 0.85, 0.1], [0.4, 0.35, 0.9]])
    t = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], dtype=np.int32)
    return v, t


def box(lo, hi):
    """Axis-aligned box as 12 outward-oriented triangles."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    t = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                  [1, 2, 6], [1, 6, 5], [2, 3, 7], [2, 7, 6], [3, 0, 4], [3, 4, 7]],
                 dtype=np.int32)
    return v, t


def l_prism(z0=0.2, z1=0.8):
    """Concave L-shaped prism (polygon extruded along z), outward oriented."""
    poly = np.array([[0.15, 0.15], [0.85, 0.15], [0.85, 0.45], [0.45, 0.45],
                     [0.45, 0.85], [0.15, 0.85]])
    m = len(poly)
    v = np.zeros((2 * m, 3))
    v[:m, :2] = poly
    v[:m, 2] = z0
    v[m:, :2] = poly
    v[m:, 2] = z1
    t = []
    for q in range(m):
        a, b = q, (q + 1) % m
        t += [(a, b, b + m), (a, b + m, a + m)]
    # caps of the L: split into two convex quads (0,1,2,3) and (0,3,4,5)
    for quad in ((0, 1, 2, 3), (0, 3, 4, 5)):
        a, b, c, d = quad
        t += [(a, c, b), (a, d, c)]                     # bottom, normal -z
        t += [(a + m, b + m, c + m), (a + m, c + m, d + m)]  # top, normal +z
    return v, np.asarray(t, dtype=np.int32)


def polyline_from_polygon(poly):
    poly = np.asarray(poly, dtype=np.float64)
    m = len(poly)
    v = np.zeros((m, 3))
    v[:, :2] = poly
    e = np.stack([np.arange(m), (np.arange(m) + 1) % m], 1).astype(np.int32)
    return v, e


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclass
class Case:
    """One synthetic problem: grid, body, flow parameters."""
    name: str
    ndim: int
    xf: np.ndarray
    yf: np.ndarray
    zf: np.ndarray
    verts: np.ndarray
    elems: np.ndarray
    Re: float
    dt: float
    nsteps: int
    u_inf: tuple = (1.0, 0.0, 0.0)
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.xf.size - 1, self.yf.size - 1, self.zf.size - 1)

    @property
    def ncells(self):
        nx, ny, nz = self.shape
        return nx * ny * nz


def cylinder_case(nx: int = 256, ny: int = 128, nseg: int = 512, Re: float = 100.0,
                  dt: float = 0.005, nsteps: int = 20) -> Case:
    """2D flow past a circular cylinder of diameter 1 at the origin in
    [-8,24]x[-8,8] on a uniform grid (Section 3.2.1 shaped)."""
    v, e = circle_polyline(nseg, 0.5)
    return Case("cylinder2d", 2, uniform_faces(-8.0, 24.0, nx), uniform_faces(-8.0, 8.0, ny),
                np.array([0.0, 1.0]), v, e, Re, dt, nsteps,
                meta={"nx": nx, "ny": ny, "nseg": nseg})


def cylinder_clustered_case(h_min: float = 0.02, ratio: float = 1.02, Re: float = 100.0, cfl: float = 0.3,
                            nsteps: int = 20, nseg: int = 1024) -> Case:
    """2D cylinder (D = 1 at the origin) in [-15, 30] x [-15, 15] on a grid
    clustered to the body: uniform spacing h_min over [-0.7, 1.5] x
    [-0.7, 0.7] (the body and its near wake), growing by `ratio` per cell
    outside. The shape of the paper's cylinder validation (Section 3.2.1) at
    the resolution a shedding-frequency and drag check needs (h_min = D/50);
    dt = cfl * h_min for a unit inflow."""
    v, e = circle_polyline(nseg, 0.5)

    def count(L, core):
        lnr = math.log(ratio)
        return core / h_min + sum(math.log1p(x * lnr / h_min) / lnr for x in L)

    nx = int(round(count((14.3, 28.5), 2.2)))
    ny = int(round(count((14.3, 14.3), 1.4)))
    xf = stretched_faces(-15.0, 30.0, nx, -0.7, 1.5, ratio)
    yf = stretched_faces(-15.0, 15.0, ny, -0.7, 0.7, ratio)
    return Case("cylinder2d_clustered", 2, xf, yf, np.array([0.0, 1.0]), v, e, Re, cfl * h_min, nsteps,
                meta={"h_min": h_min, "ratio": ratio, "nseg": nseg})


def wake_bump(case: Case, amp: float = 0.3, x0: float = 1.5, y0: float = 0.3, width2: float = 0.5):
    """A smooth off-axis bump amp * exp(-((x - x0)^2 + (y - y0)^2) / width2)
    at the cell centres of a 2D case (shape [1, ny, nx]): added to the
    initial cross-stream velocity behind a cylinder, it breaks the mirror
    symmetry so that vortex shedding starts within tens of time units
    instead of waiting for round-off to grow."""
    xc, yc = 0.5 * (case.xf[:-1] + case.xf[1:]), 0.5 * (case.yf[:-1] + case.yf[1:])
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    return (amp * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / width2))[None]


def wing_case(nx: int = 384, ny: int = 256, nz: int = 256, Re: float = 1000.0,
              dt: float = 0.002, nsteps: int = 10, ratio: float = None,
              n_chord: int = 100, n_span: int = 50) -> Case:
    """3D NACA0012 finite wing, chord 1, span 2 (aspect ratio 2), 15 degrees
    incidence, in a box 10 chords wide with the leading edge 3 chords from
    the inflow (Section 3.2.2 shaped). Grid stretched away from a uniform
    core that covers the wing's bounding box plus a quarter chord.

    The stretching profile is that of the 384x256x256 grid with a growth of
    1.01 per cell; other cell counts sample the same profile, so a grid with
    twice the cells per axis refines the reference grid (growth
    1.01**(384/nx) per cell along x, likewise y and z). `ratio` overrides
    the growth on every axis."""
    v, t = naca_wing(n_chord, n_span, 2.0, 15.0)
    lo, hi = v.min(0) - 0.25, v.max(0) + 0.25
    ref = (384, 256, 256)
    r = [ratio if ratio is not None else 1.01 ** (ref[a] / n) for a, n in enumerate((nx, ny, nz))]
    xf = stretched_faces(-3.0, 7.0, nx, lo[0], hi[0], r[0])
    yf = stretched_faces(-5.0, 5.0, ny, lo[1], hi[1], r[1])
    zf = stretched_faces(-5.0, 5.0, nz, lo[2], hi[2], r[2])
    return Case("wing3d", 3, xf, yf, zf, v, t, Re, dt, nsteps,
                meta={"nx": nx, "ny": ny, "nz": nz, "ntri": int(t.shape[0]), "ratio": r})


def sphere_case(n: int = 32, radius: float = 0.3, Re: float = 200.0, dt: float = None,
                nsteps: int = 2, level: int = 2) -> Case:
    """Single icosphere in a uniform n^3 box [-1,1]^3 (small 3D test case)."""
    v, t = icosphere(level, radius)
    f = uniform_faces(-1.0, 1.0, n)
    h = 2.0 / n
    return Case("sphere3d", 3, f.copy(), f.copy(), f.copy(), v, t, Re,
                dt if dt is not None else 0.2 * h, nsteps)


def taylor_green_case(n: int = 32, Re: float = 1.0, dt: float = 0.0025, nsteps: int = 20) -> Case:
    """Decaying Taylor-Green vortex on the unit square, uniform n x n grid,
    meant for free-slip (SLIP) walls on all four sides and u_inf = 0.

    The solver wants a body, so this case carries a small closed polygon
    far outside the domain: every cell is FLUID and there are no ghosts.
    The initial fields come from `taylor_green_fields`."""
    v, e = circle_polyline(16, 0.05, 5.0, 5.0)
    f = uniform_faces(0.0, 1.0, n)
    return Case("taylor_green2d", 2, f.copy(), f.copy(), np.array([0.0, 1.0]), v, e, Re, dt, nsteps,
                u_inf=(0.0, 0.0, 0.0), meta={"n": n})


def taylor_green_fields(case: Case, t: float = 0.0):
    """The Taylor-Green vortex u = sin(pi x) cos(pi y) F, v = -cos(pi x)
    sin(pi y) F, F = exp(-2 pi^2 t / Re), sampled at the cell centres (u, v)
    and at the face centres (face_u on x-faces, face_v on y-faces), as
    arrays shaped [1, ny, nx], [1, ny, nx + 1] and [1, ny + 1, nx]. Its
    pressure is p = (cos(2 pi x) + cos(2 pi y)) F^2 / 4 (returned as p).
    An exact solution of the incompressible Navier-Stokes equations with
    free-slip walls on the unit square."""
    xc, yc = 0.5 * (case.xf[:-1] + case.xf[1:]), 0.5 * (case.yf[:-1] + case.yf[1:])
    F = math.exp(-2.0 * math.pi ** 2 * t / case.Re)
    Yc, Xc = np.meshgrid(yc, xc, indexing="ij")
    Yu, Xu = np.meshgrid(yc, case.xf, indexing="ij")
    Yv, Xv = np.meshgrid(case.yf, xc, indexing="ij")
    pi = math.pi
    return dict(u=(np.sin(pi * Xc) * np.cos(pi * Yc) * F)[None],
                v=(-np.cos(pi * Xc) * np.sin(pi * Yc) * F)[None],
                face_u=(np.sin(pi * Xu) * np.cos(pi * Yu) * F)[None],
                face_v=(-np.cos(pi * Xv) * np.sin(pi * Yv) * F)[None],
                p=(0.25 * (np.cos(2 * pi * Xc) + np.cos(2 * pi * Yc)) * F * F)[None])


def ensemble_2d(ncases: int = 64, seed: int = 250517287):
    """Seeded 2D ensemble: ellipse or circle bodies with random semi-axes in
    [0.3, 1.0], random angle in [0, pi), grids from 128x64 to 1024x512 and
    Re in [50, 200] (mixed batch of uneven sizes)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(ncases):
        circle = rng.random() < 0.5
        a = rng.uniform(0.3, 1.0)
        b = a if circle else rng.uniform(0.3, 1.0)
        ang = rng.uniform(0.0, np.pi)
        nx = int(rng.integers(128, 1025)) // 32 * 32
        ny = nx // 2
        Re = rng.uniform(50.0, 200.0)
        v, e = ellipse_polyline(a, b, ang, 256)
        xf, yf = uniform_faces(-8.0, 24.0, nx), uniform_faces(-8.0, 8.0, ny)
        h = min(np.diff(xf).min(), np.diff(yf).min())
        out.append(Case(f"ens{c}", 2, xf, yf, np.array([0.0, 1.0]), v, e, Re, 0.2 * h, 50,
                        meta={"circle": circle, "a": a, "b": b, "angle": ang}))
    return out


_UNIT_SPHERES = {}


def _unit_icosphere(level: int):
    if level not in _UNIT_SPHERES:
        _UNIT_SPHERES[level] = icosphere(level, 1.0)
    return _UNIT_SPHERES[level]


def multi_sphere_case(n: int, spheres, Re: float, nsteps: int = 10, level: int = 4,
                      lo=(-4.0, -3.0, -3.0), hi=(8.0, 3.0, 3.0)) -> Case:
    """Uniform n^3 grid on the box [lo, hi] with one icosphere body
    (20*4**level triangles) per (radius, centre) in `spheres`; dt from a CFL
    number of 0.2 at unit inflow velocity."""
    V1, T1 = _unit_icosphere(level)
    bodies = [(V1 * r + np.asarray(c, dtype=np.float64), T1.copy()) for r, c in spheres]
    xf, yf, zf = (uniform_faces(lo[a], hi[a], n) for a in range(3))
    h = min(np.diff(xf).min(), np.diff(yf).min(), np.diff(zf).min())
    return Case(f"spheres{len(bodies)}_n{n}", 3, xf, yf, zf, bodies[0][0], bodies[0][1], Re, 0.2 * h, nsteps,
                meta={"bodies": bodies, "n": n, "spheres": [(float(r), tuple(map(float, c))) for r, c in spheres]})


def ellipsoid(center, semi=(0.5, 0.15, 0.15), pitch_deg: float = 15.0, level: int = 3):
    """Closed triangulated ellipsoid: the unit icosphere scaled by the
    semi-axes, pitched by `pitch_deg` about z (angle of attack in the x-y
    plane), then translated (outward orientation is kept)."""
    V1, T1 = _unit_icosphere(level)
    V = V1 * np.asarray(semi, dtype=np.float64)
    a = math.radians(pitch_deg)
    c, s = math.cos(a), math.sin(a)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return V @ R.T + np.asarray(center, dtype=np.float64), T1.copy()


def ellipsoid_array_case(nx: int = 1300, ny: int = 400, nz: int = 400, Re: float = 10000.0, dt: float = 0.0005,
                         nsteps: int = 5, level: int = 3, ratio: float = 1.01) -> Case:
    """Array of 27 ellipsoids (major axis D = 1, axis ratio 1 : 0.3, pitched
    15 degrees), 3 x 3 x 3 with centre spacing 1.5 D streamwise and 0.9 D
    across, in the box [-3, 10] x [-2.5, 2.5]^2 (Section 3.3 shaped: the
    paper's 1300 x 400 x 400 grid of 208M points, Re 10,000, dt 0.0005).
    The grid is uniform over the array's bounding box plus 0.1 D and
    stretched by `ratio` per cell outside it."""
    bodies = []
    for i in range(3):
        for j in range(3):
            for k in range(3):
                bodies.append(ellipsoid((1.5 * i, 0.9 * (j - 1), 0.9 * (k - 1)), level=level))
    allv = np.concatenate([v for v, _ in bodies])
    lo, hi = allv.min(0) - 0.1, allv.max(0) + 0.1
    xf = stretched_faces(-3.0, 10.0, nx, lo[0], hi[0], ratio)
    yf = stretched_faces(-2.5, 2.5, ny, lo[1], hi[1], ratio)
    zf = stretched_faces(-2.5, 2.5, nz, lo[2], hi[2], ratio)
    return Case("ellipsoid_array", 3, xf, yf, zf, bodies[0][0], bodies[0][1], Re, dt, nsteps,
                meta={"bodies": bodies, "nx": nx, "ny": ny, "nz": nz, "nbodies": len(bodies),
                      "ntri": int(sum(len(e) for _, e in bodies))})


def case_bodies(case: Case):
    """The (verts, elems) of every body of a case."""
    return case.meta.get("bodies") or [(case.verts, case.elems)]


def serve_stream(nreq: int = 500, seed: int = 250517288, rate: float = 50.0, nmin: int = 64, nmax: int = 256,
                 nsteps: int = 10, level: int = 4):
    """Seeded request stream of 3D multi-body cases: arrivals form a Poisson
    process of `rate` requests per second; each request has 1 to 8
    icospheres (5120 triangles each at level 4) with radii in [0.2, 0.6] and
    centres uniform in the inner half [-1, 5] x [-1.5, 1.5]^2 of the domain
    [-4, 8] x [-3, 3]^2, kept at least two cell widths apart by rejection; an
    n^3 grid with log n uniform in [log nmin, log nmax], n rounded down to a
    multiple of 16; Re uniform in [100, 500]; `nsteps` steps per request.
    Returns (arrival times in seconds, cases)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    times, cases = [], []
    for _ in range(nreq):
        t += rng.exponential(1.0 / rate)
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))) // 16 * 16
        n = max(n, nmin)
        h = 12.0 / n
        k = int(rng.integers(1, 9))
        spheres = []
        tries = 0
        while len(spheres) < k and tries < 10000:
            tries += 1
            r = rng.uniform(0.2, 0.6)
            c = rng.uniform((-1.0, -1.5, -1.5), (5.0, 1.5, 1.5))
            if all(np.linalg.norm(c - np.asarray(c2)) >= r + r2 + 2.0 * h for r2, c2 in spheres):
                spheres.append((r, c))
        Re = rng.uniform(100.0, 500.0)
        times.append(t)
        cases.append(multi_sphere_case(n, spheres, Re, nsteps, level))
    return np.asarray(times), cases


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape)

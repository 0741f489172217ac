"""GPU parity at the benchmark sizes: the 3D wing on 384x256x256 (25.2M cells)
and 768x512x512 (201M cells), in the launch configuration bench.py times.

The oracle cannot assemble or solve these grids, so the checks use outputs it
computes one by one or properties that hold at any size:
* inside/outside on a sample of columns (exact, same quantisation as the
  full grid), bit for bit;
* the classification rule over every cell, and the ghost list;
* ghost tables (intercept, normal, image point, stencil, kind, weights) for
  a sample of ghosts, bit for bit;
* the pressure residual on sampled rows evaluated by the oracle's row
  definition; the projected divergence is one constant over FLUID cells;
  the velocity ghost rows hold.
"""
import ctypes

import numpy as np
import pytest

from oracle import flow, geom
from paper_2505_17287_gb300 import ibm, synth

pytestmark = pytest.mark.gpu


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def combined_mesh(case):
    """All bodies of a case as one mesh, elements in the order the bodies
    were added (the library numbers them the same way)."""
    vs, es, off = [], [], 0
    for v, e in synth.case_bodies(case):
        vs.append(v)
        es.append(e + off)
        off += len(v)
    return np.concatenate(vs), np.concatenate(es).astype(np.int32)


def oracle_inside_columns(case, I, J):
    """Oracle inside flags on the columns I x J (all k), quantised with the
    parameters of the full grid."""
    verts, elems = combined_mesh(case)
    lo, s = geom.quant_params(3, case.xf, case.yf, case.zf, verts)
    xc, yc, zc = geom.centres(case.xf), geom.centres(case.yf), geom.centres(case.zf)
    Xq = geom.quantize(xc[I], lo[0], s)
    Yq = geom.quantize(yc[J], lo[1], s)
    Zq = geom.quantize(zc, lo[2], s)
    V = np.ascontiguousarray(verts, dtype=np.float64)
    Vq = np.ascontiguousarray(np.stack([geom.quantize(V[:, a], lo[a], s) for a in range(3)], 1))
    E = np.ascontiguousarray(elems, dtype=np.int32)
    out = np.zeros(len(I) * len(J) * len(zc), dtype=np.uint8)
    geom.lib().orc_inside_3d(len(I), len(J), len(zc), _p(Xq), _p(Yq), _p(Zq), _p(Vq), E.shape[0], _p(E), _p(out))
    return out.reshape(len(zc), len(J), len(I))


def check_tables(case, s, rng, nsample):
    nx, ny, nz = case.shape
    T = s.tables()
    typ = T["type"]
    # inside/outside on sampled columns, including columns through the body
    body = np.nonzero((typ != 0).any(axis=0))
    pick = rng.choice(len(body[0]), size=min(6, len(body[0])), replace=False)
    I = np.unique(np.concatenate([body[1][pick], rng.integers(0, nx, 6)]))
    J = np.unique(np.concatenate([body[0][pick], rng.integers(0, ny, 6)]))
    ins = oracle_inside_columns(case, I, J)
    assert ins.sum() > 0
    assert np.array_equal(ins, (typ[:, J][:, :, I] != 0).astype(np.uint8))
    # classification rule over every cell
    solid = typ != 0
    fl_nb = np.zeros_like(solid)
    for ax in range(3):
        for sh in (1, -1):
            r = np.roll(~solid, sh, axis=ax)
            edge = [slice(None)] * 3
            edge[ax] = 0 if sh == 1 else -1
            r[tuple(edge)] = False
            fl_nb |= r
    assert np.array_equal(typ == 1, solid & fl_nb)
    assert np.array_equal(T["gidx"], np.nonzero(typ.ravel() == 1)[0])
    # ghost tables on a sample
    q = np.sort(rng.choice(T["gidx"].size, size=min(nsample, T["gidx"].size), replace=False))
    verts, elems = combined_mesh(case)
    ref = geom.ghost_tables(3, case.xf, case.yf, case.zf, typ, T["gidx"][q], verts, elems)
    for k in ("base", "kind", "cmask", "sidx", "bi", "nrm", "ip", "dist", "wv", "wp", "bv", "bp"):
        assert np.array_equal(T[k][q], ref[k]), k
    return T


def check_step(case, s, T, rng, nrows=4000):
    g = flow.Grid(3, case.xf, case.yf, case.zf)
    typ = T["type"]
    phi = s.get("p")
    b = s.get("rhs")
    fluid = np.nonzero(typ.ravel() == 0)[0]
    rows = rng.choice(fluid, size=nrows, replace=False)
    Aphi = flow.poisson_rows(g, typ, T, phi, rows)
    r = b.ravel()[rows] - Aphi
    # at the solver tolerance (1e-10 relative, 2-norms over the FLUID and
    # GHOST rows) b - A phi is one constant on FLUID rows up to 1e-10 of the
    # root mean square of P b over those rows (b is concentrated near the
    # body, so its scale comes from the whole field, not the sample); a
    # factor 3 covers the sampling, the second term the rounding of the
    # CPU's A phi
    bf = b.ravel()[typ.ravel() == 0]
    rms_b = np.linalg.norm(bf - bf.mean()) / np.sqrt(np.count_nonzero(typ.ravel() != 2))
    tol_r = 3e-10 * rms_b + 1e-14 * np.abs(Aphi).max()
    assert np.std(r) <= tol_r, (np.std(r), tol_r, np.mean(r))
    # projection identity: div U = dt (b - A phi) on FLUID cells, so the
    # divergence is one constant up to dt times the same residual (plus the
    # rounding of the CPU's face sums)
    F = [s.get("face_u"), s.get("face_v"), s.get("face_w")]
    div = flow.divergence(g, F)[typ == 0]
    umax = max(np.abs(f).max() for f in F)
    hmin = min(np.diff(case.xf).min(), np.diff(case.yf).min(), np.diff(case.zf).min())
    assert np.std(div) <= 3e-10 * case.dt * rms_b + 1e-13 * umax / hmin, (np.std(div), case.dt * rms_b)
    # velocity ghost rows hold
    for n in ("u", "v", "w"):
        f = s.get(n).ravel()
        res = f[T["gidx"]] + np.sum(T["wv"] * f[T["sidx"]], axis=1)
        assert np.abs(res).max() < 1e-12


def test_wing_25m_tables_and_step():
    case = synth.wing_case()
    rng = np.random.default_rng(2024)
    s = ibm.Solver(case)
    s.set_body(case.verts, case.elems)
    info = s.classify()
    assert info["n_ghost"] > 1000
    T = check_tables(case, s, rng, 300)
    out = s.step(1)
    assert out["status"] == ibm.IBM_OK and out["rel_residual"] <= 1e-10, out
    check_step(case, s, T, rng)
    s.close()


def test_wing_25m_mixed_matches_fp64():
    """Same state, one step in FP64 and one in mixed precision: both reach
    the 1e-10 residual; their velocities agree to the solve accuracy."""
    case = synth.wing_case()
    a = ibm.Solver(case)
    a.set_body(case.verts, case.elems)
    a.classify()
    a.step(2)
    st = a.get_state()
    b = ibm.Solver(case, precision=ibm.IBM_MIXED)
    b.set_opts(precision=ibm.IBM_MIXED)
    b.set_body(case.verts, case.elems)
    b.classify()
    b.set_state(st)
    oa = a.step(1)
    ob = b.step(1)
    assert oa["status"] == ibm.IBM_OK and ob["status"] == ibm.IBM_OK
    assert oa["rel_residual"] <= 1e-10 and ob["rel_residual"] <= 1e-10
    for n in ("u", "v", "w"):
        x, y = a.get(n), b.get(n)
        assert np.abs(x - y).max() <= 1e-6 * np.abs(x).max(), n
    a.close()
    b.close()


def test_wing_201m_mixed_step():
    """The 768x512x512 wing (201,326,592 cells) in mixed precision on one GB300."""
    case = synth.wing_case(768, 512, 512)
    rng = np.random.default_rng(2025)
    s = ibm.Solver(case, precision=ibm.IBM_MIXED)
    s.set_opts(precision=ibm.IBM_MIXED)
    s.set_body(case.verts, case.elems)
    info = s.classify()
    assert info["n_ghost"] > 10000
    T = check_tables(case, s, rng, 200)
    out = s.step(1)
    assert out["status"] == ibm.IBM_OK and out["rel_residual"] <= 1e-10, out
    check_step(case, s, T, rng, nrows=2000)
    s.close()


def test_ellipsoid_array_208m_mixed_step():
    """27 pitched ellipsoids on the 1300x400x400 grid (208,000,000 cells) of
    the paper's particulate-array case, mixed precision, one GB300."""
    case = synth.ellipsoid_array_case()
    rng = np.random.default_rng(2026)
    s = ibm.Solver(case, precision=ibm.IBM_MIXED)
    s.set_opts(precision=ibm.IBM_MIXED)
    for v, e in synth.case_bodies(case):
        s.set_body(v, e)
    info = s.classify()
    assert info["n_ghost"] > 10000
    T = check_tables(case, s, rng, 200)
    out = s.step(1)
    assert out["status"] == ibm.IBM_OK and out["rel_residual"] <= 1e-10, out
    check_step(case, s, T, rng, nrows=2000)
    s.close()

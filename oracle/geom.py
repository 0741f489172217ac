"""ctypes front end of the oracle's C geometry (oracle/geom.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Quantisation (inside/outside predicates, Section 2.2 ray tracing): every
coordinate x on axis a becomes rint((x - lo[a]) * s), where lo is the
per-axis minimum over grid faces and mesh vertices and s = 2**(30 - e) with
E = m * 2**e (0.5 <= m < 1) the largest per-axis extent, so all quantised
values lie in [0, 2**30].
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_geom.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile geom.c with plain gcc; no FMA contraction, no fast math."""
    src = os.path.join(_HERE, "geom.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        L.orc_quantize.argtypes = [P, I64, D, D, P]
        L.orc_inside_3d.argtypes = [I, I, I, P, P, P, P, I64, P, P]
        L.orc_inside_2d.argtypes = [I, I, P, P, P, I64, P, P]
        L.orc_classify.argtypes = [I, I, I, P, P, P]
        L.orc_classify.restype = I64
        L.orc_ghost_tables.argtypes = [I, I, I, I, P, P, P, P, P, P, P, I64, P, P, I64, P] + [P] * 12
        L.orc_fresh_tables.argtypes = [I, I, I, I, P, P, P, P, P, P, P, I64, P, P, I64, P] + [P] * 5
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def centres(f):
    f = np.asarray(f, dtype=np.float64)
    return 0.5 * (f[:-1] + f[1:])


def quant_params(ndim, xf, yf, zf, verts):
    axes = [np.asarray(xf), np.asarray(yf), np.asarray(zf)][:ndim]
    lo, hi = [], []
    for a in range(ndim):
        lo.append(min(float(axes[a].min()), float(verts[:, a].min())))
        hi.append(max(float(axes[a].max()), float(verts[:, a].max())))
    E = max(h - l for h, l in zip(hi, lo))
    _, e = math.frexp(E)
    return lo, math.ldexp(1.0, 30 - e)


def quantize(x, lo, s):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.shape, dtype=np.int64)
    lib().orc_quantize(_p(x), x.size, lo, s, _p(out))
    return out


def inside(ndim, xf, yf, zf, verts, elems):
    """uint8 flags [nz, ny, nx]: 1 when the cell centre is inside the body."""
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    lo, s = quant_params(ndim, xf, yf, zf, verts)
    nx, ny = len(xf) - 1, len(yf) - 1
    Xq, Yq = quantize(centres(xf), lo[0], s), quantize(centres(yf), lo[1], s)
    if ndim == 2:
        Vq = np.ascontiguousarray(np.stack([quantize(verts[:, 0], lo[0], s),
                                            quantize(verts[:, 1], lo[1], s)], 1))
        out = np.zeros(nx * ny, dtype=np.uint8)
        lib().orc_inside_2d(nx, ny, _p(Xq), _p(Yq), _p(Vq), elems.shape[0], _p(elems), _p(out))
        return out.reshape(1, ny, nx)
    nz = len(zf) - 1
    Zq = quantize(centres(zf), lo[2], s)
    Vq = np.ascontiguousarray(np.stack([quantize(verts[:, a], lo[a], s) for a in range(3)], 1))
    out = np.zeros(nx * ny * nz, dtype=np.uint8)
    lib().orc_inside_3d(nx, ny, nz, _p(Xq), _p(Yq), _p(Zq), _p(Vq), elems.shape[0], _p(elems), _p(out))
    return out.reshape(nz, ny, nx)


def classify(inside_flags):
    """type [nz,ny,nx] (0 FLUID, 1 GHOST, 2 DEAD) and ascending ghost list."""
    ins = np.ascontiguousarray(inside_flags, dtype=np.uint8)
    nz, ny, nx = ins.shape
    typ = np.zeros_like(ins)
    g = np.zeros(ins.size, dtype=np.int64)
    ng = lib().orc_classify(nx, ny, nz, _p(ins), _p(typ), _p(g))
    return typ, g[:ng].copy()


def ghost_tables(ndim, xf, yf, zf, typ, gidx, verts, elems):
    """Per-ghost body intercept, normal, image point, stencil and weights."""
    xf, yf, zf = (np.asarray(a, dtype=np.float64) for a in (xf, yf, zf))
    nx, ny, nz = len(xf) - 1, len(yf) - 1, len(zf) - 1
    xc, yc, zc = centres(xf), centres(yf), centres(zf)
    dx, dy, dz = np.diff(xf), np.diff(yf), np.diff(zf)
    typ = np.ascontiguousarray(typ, dtype=np.uint8).ravel()
    gidx = np.ascontiguousarray(gidx, dtype=np.int64)
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    ng = gidx.size
    t = dict(bi=np.zeros((ng, 3)), nrm=np.zeros((ng, 3)), ip=np.zeros((ng, 3)), dist=np.zeros(ng),
             base=np.zeros(ng, np.int64), kind=np.zeros(ng, np.uint8), cmask=np.zeros(ng, np.uint8),
             sidx=np.zeros((ng, 8), np.int64), wv=np.zeros((ng, 8)), wp=np.zeros((ng, 8)),
             bv=np.zeros(ng), bp=np.zeros(ng))
    if ng:
        lib().orc_ghost_tables(ndim, nx, ny, nz, _p(xc), _p(yc), _p(zc), _p(dx), _p(dy), _p(dz),
                               _p(typ), ng, _p(gidx), _p(verts), elems.shape[0], _p(elems),
                               *[_p(t[k]) for k in ("bi", "nrm", "ip", "dist", "base", "kind", "cmask",
                                                    "sidx", "wv", "wp", "bv", "bp")])
    t["gidx"] = gidx
    return t


def fresh_tables(ndim, xf, yf, zf, typ, fidx, verts, elems):
    """Per-fresh-cell body intercept, kind, stencil and weights (geom.c,
    orc_fresh_tables): u_FC = sum_m w_m u_m + wb u_BI."""
    xf, yf, zf = (np.asarray(a, dtype=np.float64) for a in (xf, yf, zf))
    nx, ny, nz = len(xf) - 1, len(yf) - 1, len(zf) - 1
    xc, yc, zc = centres(xf), centres(yf), centres(zf)
    dx, dy, dz = np.diff(xf), np.diff(yf), np.diff(zf)
    typ = np.ascontiguousarray(typ, dtype=np.uint8).ravel()
    fidx = np.ascontiguousarray(fidx, dtype=np.int64)
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    nf = fidx.size
    t = dict(bi=np.zeros((nf, 3)), kind=np.zeros(nf, np.uint8), sidx=np.zeros((nf, 8), np.int64),
             w=np.zeros((nf, 8)), wb=np.zeros(nf))
    if nf:
        lib().orc_fresh_tables(ndim, nx, ny, nz, _p(xc), _p(yc), _p(zc), _p(dx), _p(dy), _p(dz),
                               _p(typ), nf, _p(fidx), _p(verts), elems.shape[0], _p(elems),
                               *[_p(t[k]) for k in ("bi", "kind", "sidx", "w", "wb")])
    t["fidx"] = fidx
    return t


def body_tables(ndim, xf, yf, zf, verts, elems):
    """inside -> classify -> ghost tables, in one call."""
    ins = inside(ndim, xf, yf, zf, verts, elems)
    typ, gidx = classify(ins)
    tabs = ghost_tables(ndim, xf, yf, zf, typ, gidx, verts, elems)
    tabs["type"] = typ
    tabs["inside"] = ins
    return tabs

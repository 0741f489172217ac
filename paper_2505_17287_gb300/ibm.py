"""Thin ctypes binding of libibm.so (include/ibm.h), same names as the C ABI.

Only argument marshalling lives here: every step of the solver runs in the
library's CUDA kernels. PyTorch supplies the device memory (the library's
allocator hooks call PyTorch's caching allocator) and the CUDA stream. The
library must be built (``paper_2505_17287_gb300.build.build()``); importing
this module without it fails loudly, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, byref, c_char_p, c_double, c_int, c_int64,
                    c_size_t, c_uint8, c_void_p)

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibm.so")

IBM_OK, IBM_ERR_ARG, IBM_ERR_OOM, IBM_ERR_CUDA, IBM_ERR_MESH = 0, 1, 2, 3, 4
IBM_ERR_STATE, IBM_ERR_NOT_CONVERGED, IBM_ERR_DIVERGED, IBM_ERR_TIMEOUT = 5, 6, 7, 8
STATUS_NAMES = {0: "IBM_OK", 1: "IBM_ERR_ARG", 2: "IBM_ERR_OOM", 3: "IBM_ERR_CUDA", 4: "IBM_ERR_MESH",
                5: "IBM_ERR_STATE", 6: "IBM_ERR_NOT_CONVERGED", 7: "IBM_ERR_DIVERGED", 8: "IBM_ERR_TIMEOUT"}
IBM_FLUID, IBM_GHOST, IBM_DEAD = 0, 1, 2
IBM_BC_INFLOW, IBM_BC_OUTFLOW, IBM_BC_SLIP = 0, 1, 2
IBM_FP64, IBM_MIXED = 0, 1
IBM_OUTER_BICGSTAB, IBM_OUTER_FGMRES = 0, 1
FIELDS = {"u": 0, "v": 1, "w": 2, "p": 3, "face_u": 4, "face_v": 5, "face_w": 6, "nold_u": 7, "nold_v": 8,
          "nold_w": 9, "type": 10, "ustar_u": 11, "ustar_v": 12, "ustar_w": 13, "rhs": 14, "step": 15,
          "p_prev": 16, "p_prev2": 17, "p_hist_x": 18, "p_hist_b": 19, "p_hist_ctl": 20}

ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p)


class ibm_grid_desc(Structure):
    _fields_ = [("ndim", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("xf", c_void_p), ("yf", c_void_p), ("zf", c_void_p),
                ("Re", c_double), ("dt", c_double), ("u_inf", c_double * 3), ("bc", c_int * 6),
                ("precision", c_int), ("stream", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", c_void_p)]


class ibm_solver_opts(Structure):
    _fields_ = [("rtol", c_double), ("max_outer", c_int), ("restart", c_int), ("inner_iters", c_int),
                ("nu1", c_int), ("nu2", c_int), ("coarse_sweeps", c_int), ("helm_rtol", c_double),
                ("helm_maxit", c_int), ("ghost_tol", c_double), ("ghost_maxit", c_int), ("precision", c_int),
                ("outer", c_int), ("band_sweeps", c_int), ("band_omega", c_double),
                ("mixed_inner_rtol", c_double), ("mg_interp", c_int), ("tile_x", c_int), ("graph", c_int),
                ("precond", c_int), ("srj_sweeps", c_int), ("srj_lmin", c_double), ("helm_solver", c_int),
                ("smooth_omega", c_double), ("reorth_eta", c_double),
                ("helm_check_first", c_int), ("helm_omega", c_double), ("fine_split", c_int),
                ("band_width", c_int), ("poisson_hist", c_int), ("tail_cells", c_int),
                ("nu_coarse", c_int)]


class ibm_table_info(Structure):
    _fields_ = [("n_fluid", c_int64), ("n_ghost", c_int64), ("n_dead", c_int64), ("n_kind", c_int64 * 3)]


class ibm_solve_stats(Structure):
    _fields_ = [("outer_iters", c_int), ("inner_iters", c_int), ("rel_residual", c_double),
                ("ms", c_double)]


class ibm_step_stats(Structure):
    _fields_ = [("steps", c_int), ("poisson_outer", c_int), ("poisson_inner", c_int), ("helm_sweeps", c_int),
                ("rel_residual", c_double), ("max_div", c_double), ("ms_total", c_double),
                ("ms_predictor", c_double), ("ms_poisson", c_double), ("ms_projection", c_double)]


class ibm_tables_host(Structure):
    _fields_ = [(n, c_void_p) for n in ("type", "gidx", "bi", "nrm", "ip", "dist", "base", "kind", "cmask",
                                        "sidx", "wv", "wp", "bv", "bp")]


IBM_REQ_STEP, IBM_REQ_POISSON = 0, 1


class ibm_server_opts(Structure):
    _fields_ = [("max_slots", c_int), ("device", c_int), ("hbm_reserve", c_size_t), ("hbm_budget", c_size_t)]


class ibm_request(Structure):
    _fields_ = [("kind", c_int), ("grid", ibm_grid_desc), ("opts", c_void_p), ("nbodies", c_int),
                ("verts", c_void_p), ("nverts", c_void_p), ("elems", c_void_p), ("nelems", c_void_p),
                ("nsteps", c_int), ("rhs", c_void_p), ("rtol", c_double), ("maxit", c_int),
                ("out_u", c_void_p), ("out_v", c_void_p), ("out_w", c_void_p), ("out_p", c_void_p)]


class ibm_result(Structure):
    _fields_ = [("status", c_int), ("cells", c_int64), ("steps", c_int), ("t_submit", c_double),
                ("t_admit", c_double), ("t_done", c_double), ("bytes_estimate", c_size_t),
                ("bytes_peak", c_size_t), ("step", ibm_step_stats), ("solve", ibm_solve_stats), ("slot", c_int),
                ("error", ctypes.c_char * 160)]


class ibm_server_stats(Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("queued", c_int64),
                ("running", c_int64), ("peak_running", c_int), ("budget", c_size_t), ("admitted_bytes", c_size_t),
                ("peak_admitted_bytes", c_size_t)]


EXPORTS = ["ibm_step_async", "ibm_step_wait", "ibm_step_prepare", "ibm_tune", "ibm_case_bytes", "ibm_server_create", "ibm_server_submit", "ibm_server_wait", "ibm_server_get_stats",
           "ibm_server_destroy",
           "ibm_default_opts", "ibm_create_grid", "ibm_set_opts", "ibm_set_body", "ibm_classify_cells", "ibm_move_body",
           "ibm_step", "ibm_poisson_solve", "ibm_get_tables", "ibm_get_field", "ibm_set_field", "ibm_sizes",
           "ibm_kernel_timer", "ibm_kernel_time", "ibm_launch_count", "ibm_poisson_residual_noalloc",
           "ibm_destroy", "ibm_last_error"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libibm.so and declare the signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run paper_2505_17287_gb300.build.build() on a machine "
                           "with nvcc; there is no CPU fallback")
    L = ctypes.CDLL(path)
    P = c_void_p
    L.ibm_default_opts.argtypes = [POINTER(ibm_solver_opts)]
    L.ibm_create_grid.argtypes = [POINTER(ibm_grid_desc), POINTER(c_void_p)]
    L.ibm_set_opts.argtypes = [P, POINTER(ibm_solver_opts)]
    L.ibm_set_body.argtypes = [P, P, c_int64, P, c_int64]
    L.ibm_classify_cells.argtypes = [P, POINTER(ibm_table_info)]
    L.ibm_move_body.argtypes = [P, P, c_int64, P, POINTER(ibm_table_info)]
    L.ibm_step.argtypes = [P, c_int, POINTER(ibm_step_stats)]
    L.ibm_poisson_solve.argtypes = [P, P, P, c_double, c_int, POINTER(ibm_solve_stats)]
    L.ibm_get_tables.argtypes = [P, POINTER(ibm_tables_host)]
    L.ibm_get_field.argtypes = [P, c_int, P, c_int, c_size_t]
    L.ibm_set_field.argtypes = [P, c_int, P, c_int, c_size_t]
    L.ibm_sizes.argtypes = [P, POINTER(c_int64), POINTER(c_int64)]
    L.ibm_launch_count.argtypes = [P, POINTER(c_int64)]
    L.ibm_poisson_residual_noalloc.argtypes = [P, P, P, P]
    L.ibm_kernel_timer.argtypes = [P, c_int]
    L.ibm_kernel_time.argtypes = [P, c_int, POINTER(c_double), POINTER(c_int64)]
    L.ibm_destroy.argtypes = [P]
    L.ibm_last_error.argtypes = [P]
    L.ibm_last_error.restype = c_char_p
    L.ibm_case_bytes.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int64]
    L.ibm_server_create.argtypes = [POINTER(ibm_server_opts), POINTER(c_void_p)]
    L.ibm_server_submit.argtypes = [P, POINTER(ibm_request), POINTER(c_int64)]
    L.ibm_server_wait.argtypes = [P, c_int64, c_double, POINTER(ibm_result)]
    L.ibm_server_get_stats.argtypes = [P, POINTER(ibm_server_stats)]
    L.ibm_server_destroy.argtypes = [P]
    L.ibm_step_async.argtypes = [P, c_int]
    L.ibm_step_wait.argtypes = [P, POINTER(ibm_step_stats)]
    L.ibm_step_prepare.argtypes = [P]
    L.ibm_tune.argtypes = [POINTER(ibm_grid_desc), c_int, P, P, P, P, POINTER(ibm_solver_opts), c_int, c_int,
                           POINTER(c_int), P]
    for name in EXPORTS:
        if name != "ibm_last_error":
            getattr(L, name).restype = c_int
    L.ibm_case_bytes.restype = c_size_t
    _lib = L
    return L


class IBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _p(a):
    return a.ctypes.data_as(c_void_p)


def _check(status, ctx=None, ok=(IBM_OK,)):
    if status not in ok:
        msg = load_library().ibm_last_error(ctx)
        raise IBMError(status, msg.decode() if msg else "")
    return status


# --------------------------------------------------------------------------
# C-ABI names
# --------------------------------------------------------------------------

def ibm_default_opts():
    o = ibm_solver_opts()
    _check(load_library().ibm_default_opts(byref(o)))
    return o


def ibm_create_grid(desc: ibm_grid_desc):
    ctx = c_void_p()
    _check(load_library().ibm_create_grid(byref(desc), byref(ctx)))
    return ctx


def ibm_set_opts(ctx, opts: ibm_solver_opts):
    return _check(load_library().ibm_set_opts(ctx, byref(opts)), ctx)


def ibm_set_body(ctx, verts: np.ndarray, elems: np.ndarray):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    e = np.ascontiguousarray(elems, dtype=np.int32)
    return _check(load_library().ibm_set_body(ctx, _p(v), v.shape[0], _p(e), e.shape[0]), ctx)


def ibm_classify_cells(ctx):
    info = ibm_table_info()
    _check(load_library().ibm_classify_cells(ctx, byref(info)), ctx)
    return info


def ibm_move_body(ctx, verts: np.ndarray, motion):
    """Move the bodies to verts (all vertices of every set body, same order)
    with the rigid motion (U, Omega, centre); returns the new table info."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    m = np.ascontiguousarray(np.asarray(motion, dtype=np.float64).reshape(9))
    info = ibm_table_info()
    _check(load_library().ibm_move_body(ctx, _p(v), v.shape[0], _p(m), byref(info)), ctx)
    return info


def ibm_step(ctx, nsteps: int):
    st = ibm_step_stats()
    status = _check(load_library().ibm_step(ctx, nsteps, byref(st)), ctx, ok=(IBM_OK, IBM_ERR_NOT_CONVERGED))
    return st, status


def ibm_poisson_solve(ctx, rhs_ptr: int, phi_ptr: int, rtol: float = 0.0, maxit: int = 0):
    st = ibm_solve_stats()
    status = _check(load_library().ibm_poisson_solve(ctx, c_void_p(rhs_ptr), c_void_p(phi_ptr), rtol, maxit,
                                                     byref(st)), ctx, ok=(IBM_OK, IBM_ERR_NOT_CONVERGED))
    return st, status


def ibm_get_tables(ctx, dst: ibm_tables_host):
    return _check(load_library().ibm_get_tables(ctx, byref(dst)), ctx)


def ibm_get_field(ctx, field: int, dst_ptr: int, is_device: int, nbytes: int):
    return _check(load_library().ibm_get_field(ctx, field, c_void_p(dst_ptr), is_device, nbytes), ctx)


def ibm_set_field(ctx, field: int, src_ptr: int, is_device: int, nbytes: int):
    return _check(load_library().ibm_set_field(ctx, field, c_void_p(src_ptr), is_device, nbytes), ctx)


def ibm_sizes(ctx):
    n, g = c_int64(), c_int64()
    _check(load_library().ibm_sizes(ctx, byref(n), byref(g)), ctx)
    return n.value, g.value


def ibm_launch_count(ctx):
    n = c_int64()
    _check(load_library().ibm_launch_count(ctx, byref(n)), ctx)
    return n.value


KERNEL_IDS = {"rbgs0": 0, "spmv0": 1, "apply_A": 2, "mdot": 3, "orth": 4, "helm": 5, "conv": 6,
              "rbgs_coarse": 7, "restrict": 8, "prolong": 9, "other": 10, "tail": 11}


def ibm_kernel_timer(ctx, enable: int):
    return _check(load_library().ibm_kernel_timer(ctx, enable), ctx)


def ibm_kernel_time(ctx, kernel: int):
    ms, n = c_double(), c_int64()
    _check(load_library().ibm_kernel_time(ctx, kernel, byref(ms), byref(n)), ctx)
    return ms.value, n.value


def ibm_poisson_residual_noalloc(ctx, rhs_ptr: int, phi_ptr: int):
    """Relative residual of phi for rhs (device pointers), computed without
    any device allocation; returns a float."""
    out = c_double()
    _check(load_library().ibm_poisson_residual_noalloc(ctx, c_void_p(rhs_ptr), c_void_p(phi_ptr),
                                                       ctypes.cast(byref(out), c_void_p)), ctx)
    return out.value


def ibm_destroy(ctx):
    return _check(load_library().ibm_destroy(ctx))


def ibm_last_error(ctx=None):
    m = load_library().ibm_last_error(ctx)
    return m.decode() if m else ""


# --------------------------------------------------------------------------
# convenience wrapper used by the tests and the benchmark
# --------------------------------------------------------------------------

class Solver:
    """One grid context. `case` is a paper_2505_17287_gb300.synth.Case (or any
    object with ndim, xf, yf, zf, Re, dt, u_inf). Device memory comes from
    PyTorch's caching allocator; work runs on `stream` (default: PyTorch's
    current stream of cuda:0)."""

    def __init__(self, case, precision=IBM_FP64, bc=(0, 1, 2, 2, 2, 2), stream=None, torch_alloc=True):
        import torch
        self._torch = torch
        load_library()
        self.case = case
        self.ndim = case.ndim
        nx, ny = len(case.xf) - 1, len(case.yf) - 1
        nz = len(case.zf) - 1 if case.ndim == 3 else 1
        self.shape = (nz, ny, nx)
        self._xf = np.ascontiguousarray(case.xf, dtype=np.float64)
        self._yf = np.ascontiguousarray(case.yf, dtype=np.float64)
        self._zf = np.ascontiguousarray(case.zf if case.ndim == 3 else [0.0, 1.0], dtype=np.float64)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        d = ibm_grid_desc()
        d.ndim, d.nx, d.ny, d.nz = case.ndim, nx, ny, nz
        d.xf, d.yf, d.zf = _p(self._xf), _p(self._yf), _p(self._zf)
        d.Re, d.dt = float(case.Re), float(case.dt)
        d.u_inf = (c_double * 3)(*[float(x) for x in case.u_inf])
        d.bc = (c_int * 6)(*bc)
        d.precision = precision
        d.stream = c_void_p(self.stream.cuda_stream)
        if torch_alloc:
            st = self.stream

            def _alloc(nbytes, _ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)

            def _free(ptr, _ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
            d.alloc, d.free = self._hooks
        self.ctx = ibm_create_grid(d)
        self.N = nx * ny * nz
        self.info = None

    # lifecycle --------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            ibm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, **kw):
        o = ibm_default_opts() if not hasattr(self, "_opts") else self._opts
        for k, v in kw.items():
            setattr(o, k, v)
        ibm_set_opts(self.ctx, o)
        self._opts = o
        return o

    def set_body(self, verts, elems):
        return ibm_set_body(self.ctx, verts, elems)

    def classify(self):
        self.info = ibm_classify_cells(self.ctx)
        return dict(n_fluid=self.info.n_fluid, n_ghost=self.info.n_ghost, n_dead=self.info.n_dead,
                    n_kind=list(self.info.n_kind))

    def move_body(self, verts, U=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), centre=(0.0, 0.0, 0.0)):
        """Move every set body to verts with the rigid velocity U + omega x (x - centre)."""
        self.info = ibm_move_body(self.ctx, verts, tuple(U) + tuple(omega) + tuple(centre))
        return dict(n_fluid=self.info.n_fluid, n_ghost=self.info.n_ghost, n_dead=self.info.n_dead,
                    n_kind=list(self.info.n_kind))

    def step(self, n=1):
        st, status = ibm_step(self.ctx, n)
        out = {k: getattr(st, k) for k, _ in ibm_step_stats._fields_}
        out["status"] = status
        return out

    def step_async(self, n=1):
        """Enqueue n steps (captured graphs with opts graph=2) without waiting."""
        return _check(load_library().ibm_step_async(self.ctx, int(n)), self.ctx)

    def step_prepare(self):
        """Capture the step graphs now (opts graph=2), outside any timed region."""
        return _check(load_library().ibm_step_prepare(self.ctx), self.ctx)

    def step_wait(self):
        st = ibm_step_stats()
        status = _check(load_library().ibm_step_wait(self.ctx, byref(st)), self.ctx, ok=(IBM_OK, IBM_ERR_NOT_CONVERGED))
        out = {k: getattr(st, k) for k, _ in ibm_step_stats._fields_}
        out["status"] = status
        return out

    def poisson_solve(self, rhs, phi, rtol=0.0, maxit=0):
        """rhs, phi: torch float64 CUDA tensors with N elements."""
        torch = self._torch
        assert rhs.is_cuda and phi.is_cuda and rhs.dtype == torch.float64 and phi.dtype == torch.float64
        assert rhs.numel() == self.N and phi.numel() == self.N and rhs.is_contiguous() and phi.is_contiguous()
        st, status = ibm_poisson_solve(self.ctx, rhs.data_ptr(), phi.data_ptr(), rtol, maxit)
        out = {k: getattr(st, k) for k, _ in ibm_solve_stats._fields_}
        out["status"] = status
        return out

    # host access -------------------------------------------------------------
    def tables(self):
        n, ng = ibm_sizes(self.ctx)
        t = dict(type=np.zeros(n, np.uint8), gidx=np.zeros(ng, np.int64), bi=np.zeros((ng, 3)),
                 nrm=np.zeros((ng, 3)), ip=np.zeros((ng, 3)), dist=np.zeros(ng), base=np.zeros(ng, np.int64),
                 kind=np.zeros(ng, np.uint8), cmask=np.zeros(ng, np.uint8), sidx=np.zeros((ng, 8), np.int64),
                 wv=np.zeros((ng, 8)), wp=np.zeros((ng, 8)), bv=np.zeros(ng), bp=np.zeros(ng))
        h = ibm_tables_host(**{k: _p(v) for k, v in t.items()})
        ibm_get_tables(self.ctx, h)
        t["type"] = t["type"].reshape(self.shape)
        return t

    def hist_pairs(self):
        o = getattr(self, "_opts", None) or ibm_default_opts()
        return int(o.poisson_hist)

    def field_size(self, name):
        nz, ny, nx = self.shape
        if name in ("p_hist_x", "p_hist_b"):
            return (self.hist_pairs(),) + self.shape
        if name == "p_hist_ctl":
            return (2 + self.hist_pairs() ** 2,)
        if name == "face_u":
            return (nz, ny, nx + 1)
        if name == "face_v":
            return (nz, ny + 1, nx)
        if name == "face_w":
            return (nz + 1, ny, nx)
        return self.shape

    def get(self, name):
        if name == "step":
            v = np.zeros(1, np.int64)
            ibm_get_field(self.ctx, FIELDS[name], v.ctypes.data, 0, 8)
            return int(v[0])
        dt = np.uint8 if name == "type" else np.float64
        a = np.zeros(self.field_size(name), dt)
        ibm_get_field(self.ctx, FIELDS[name], a.ctypes.data, 0, a.nbytes)
        return a

    def set(self, name, arr):
        if name == "step":
            v = np.array([int(arr)], np.int64)
            return ibm_set_field(self.ctx, FIELDS[name], v.ctypes.data, 0, 8)
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.field_size(name))
        return ibm_set_field(self.ctx, FIELDS[name], a.ctypes.data, 0, a.nbytes)

    def state_names(self):
        """Fields of a checkpoint that restarts bit for bit (the Poisson guess
        history included when it is on)."""
        names = ["u", "v", "p", "p_prev", "p_prev2", "face_u", "face_v", "nold_u", "nold_v"]
        if self.ndim == 3:
            names += ["w", "face_w", "nold_w"]
        if self.hist_pairs() > 0:
            names += ["p_hist_x", "p_hist_b", "p_hist_ctl"]
        return names + ["step"]

    def get_state(self):
        return {k: self.get(k) for k in self.state_names()}

    def set_state(self, st):
        for k in self.state_names():
            self.set(k, st[k])


# --------------------------------------------------------------------------
# request loop over many cases (include/ibm_serve.h)
# --------------------------------------------------------------------------

def ibm_case_bytes(ndim, nx, ny, nz, precision, nelems_total):
    return int(load_library().ibm_case_bytes(ndim, nx, ny, nz, precision, nelems_total))


def _status_check(status, what):
    if status != IBM_OK:
        raise IBMError(status, what)
    return status


class Server:
    """ibm_server: `max_slots` cases resident and advancing at once on their
    own streams, admitted first-in first-out by free device memory."""

    def __init__(self, max_slots=4, device=0, hbm_reserve=2 << 30, hbm_budget=0):
        load_library()
        o = ibm_server_opts(max_slots, device, hbm_reserve, hbm_budget)
        h = c_void_p()
        _status_check(load_library().ibm_server_create(byref(o), byref(h)), "ibm_server_create")
        self.h = h
        self._keep = {}

    def submit(self, case, kind=IBM_REQ_STEP, nsteps=None, precision=IBM_FP64, opts=None, outputs=False,
               rhs=None, rtol=0.0, maxit=0, bc=(0, 1, 2, 2, 2, 2)):
        """Queue one case (a synth.Case; every body of synth.case_bodies(case)).
        outputs=True returns u, v, w, p (STEP) or phi (POISSON) from wait()."""
        from . import synth
        nx, ny = len(case.xf) - 1, len(case.yf) - 1
        nz = len(case.zf) - 1 if case.ndim == 3 else 1
        N = nx * ny * nz
        keep = {}
        xf = keep["xf"] = np.ascontiguousarray(case.xf, dtype=np.float64)
        yf = keep["yf"] = np.ascontiguousarray(case.yf, dtype=np.float64)
        zf = keep["zf"] = np.ascontiguousarray(case.zf if case.ndim == 3 else [0.0, 1.0], dtype=np.float64)
        r = ibm_request()
        r.kind = kind
        g = r.grid
        g.ndim, g.nx, g.ny, g.nz = case.ndim, nx, ny, nz
        g.xf, g.yf, g.zf = _p(xf), _p(yf), _p(zf)
        g.Re, g.dt = float(case.Re), float(case.dt)
        g.u_inf = (c_double * 3)(*[float(x) for x in case.u_inf])
        g.bc = (c_int * 6)(*bc)
        g.precision = precision
        if opts is not None:
            keep["opts"] = opts
            r.opts = ctypes.cast(ctypes.pointer(opts), c_void_p)
        bodies = synth.case_bodies(case)
        vs = [np.ascontiguousarray(np.c_[v, np.zeros(len(v))] if v.shape[1] == 2 else v, dtype=np.float64)
              for v, _ in bodies]
        es = [np.ascontiguousarray(e, dtype=np.int32) for _, e in bodies]
        vp = (c_void_p * len(vs))(*[v.ctypes.data for v in vs])
        ep = (c_void_p * len(es))(*[e.ctypes.data for e in es])
        nv = np.array([len(v) for v in vs], np.int64)
        ne = np.array([len(e) for e in es], np.int64)
        keep.update(vs=vs, es=es, vp=vp, ep=ep, nv=nv, ne=ne)
        r.nbodies = len(vs)
        r.verts, r.elems = ctypes.cast(vp, c_void_p), ctypes.cast(ep, c_void_p)
        r.nverts, r.nelems = _p(nv), _p(ne)
        r.nsteps = int(nsteps if nsteps is not None else case.nsteps)
        if kind == IBM_REQ_POISSON:
            b = keep["rhs"] = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
            assert b.size == N
            r.rhs = _p(b)
            r.rtol, r.maxit = float(rtol), int(maxit)
        outs = {}
        if outputs:
            names = (("u", "v", "w", "p") if case.ndim == 3 else ("u", "v", "p")) if kind == IBM_REQ_STEP else ("p",)
            for n in names:
                outs[n] = np.zeros((nz, ny, nx), np.float64)
                setattr(r, "out_" + n, _p(outs[n]))
        rid = c_int64()
        _status_check(load_library().ibm_server_submit(self.h, byref(r), byref(rid)), "ibm_server_submit")
        self._keep[rid.value] = (keep, outs)
        return rid.value

    def wait(self, rid, timeout=-1.0):
        """Result dict of request rid, or None if it is not done within timeout."""
        res = ibm_result()
        st = load_library().ibm_server_wait(self.h, rid, float(timeout), byref(res))
        if st == IBM_ERR_TIMEOUT:
            return None
        _status_check(st, "ibm_server_wait")
        _, outs = self._keep.pop(rid)
        out = {k: getattr(res, k) for k, _ in ibm_result._fields_ if k not in ("step", "solve", "error")}
        out["error"] = res.error.decode(errors="replace")
        out["step"] = {k: getattr(res.step, k) for k, _ in ibm_step_stats._fields_}
        out["solve"] = {k: getattr(res.solve, k) for k, _ in ibm_solve_stats._fields_}
        out["latency_s"] = res.t_done - res.t_submit
        out["outputs"] = outs
        return out

    def stats(self):
        s = ibm_server_stats()
        _status_check(load_library().ibm_server_get_stats(self.h, byref(s)), "ibm_server_get_stats")
        return {k: getattr(s, k) for k, _ in ibm_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load_library().ibm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ibm_tune(case, candidates, steps=3, stream=None, bc=(0, 1, 2, 2, 2, 2), precision=IBM_FP64):
    """Time `steps` fractional steps of `case` under each option set in
    `candidates` (ibm_solver_opts) on `stream` (a torch.cuda.Stream; default
    a new one, so V-cycle graphs can be captured). Returns (best index, ms per
    step of each candidate, negative = failed)."""
    import torch
    from . import synth
    st = stream if stream is not None else torch.cuda.Stream()
    nx, ny = len(case.xf) - 1, len(case.yf) - 1
    nz = len(case.zf) - 1 if case.ndim == 3 else 1
    xf = np.ascontiguousarray(case.xf, dtype=np.float64)
    yf = np.ascontiguousarray(case.yf, dtype=np.float64)
    zf = np.ascontiguousarray(case.zf if case.ndim == 3 else [0.0, 1.0], dtype=np.float64)
    d = ibm_grid_desc()
    d.ndim, d.nx, d.ny, d.nz = case.ndim, nx, ny, nz
    d.xf, d.yf, d.zf = _p(xf), _p(yf), _p(zf)
    d.Re, d.dt = float(case.Re), float(case.dt)
    d.u_inf = (c_double * 3)(*[float(x) for x in case.u_inf])
    d.bc = (c_int * 6)(*bc)
    d.precision = precision
    d.stream = c_void_p(st.cuda_stream)
    bodies = synth.case_bodies(case)
    vs = [np.ascontiguousarray(np.c_[v, np.zeros(len(v))] if v.shape[1] == 2 else v, dtype=np.float64)
          for v, _ in bodies]
    es = [np.ascontiguousarray(e, dtype=np.int32) for _, e in bodies]
    vp = (c_void_p * len(vs))(*[v.ctypes.data for v in vs])
    ep = (c_void_p * len(es))(*[e.ctypes.data for e in es])
    nv = np.array([len(v) for v in vs], np.int64)
    ne = np.array([len(e) for e in es], np.int64)
    cand = (ibm_solver_opts * len(candidates))(*candidates)
    ms = np.zeros(len(candidates))
    best = c_int(-1)
    torch.cuda.synchronize()
    _status_check(load_library().ibm_tune(byref(d), len(vs), ctypes.cast(vp, c_void_p), _p(nv),
                                          ctypes.cast(ep, c_void_p), _p(ne), cand, len(candidates), steps,
                                          byref(best), _p(ms)), "ibm_tune")
    return best.value, ms

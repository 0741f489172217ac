"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function that include/ibm.h declares, and the ctypes
structures of the binding have the C layout (sizes and field offsets
printed by a C program compiled against the header)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ibm.h")
SERVE_HEADER = os.path.join(ROOT, "include", "ibm_serve.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def _declared():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_17287_gb300 import build
    build.build()
    from paper_2505_17287_gb300 import ibm
    return ibm.load_library()


def test_exports_every_declared_function(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2505_17287_gb300", "libibm.so")],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ibm_\w+)", out))
    assert set(names) <= exported
    from paper_2505_17287_gb300 import ibm
    assert set(ibm.EXPORTS) == set(names)


def test_struct_layout_matches_header(tmp_path):
    from paper_2505_17287_gb300 import ibm
    structs = {"ibm_grid_desc": ibm.ibm_grid_desc, "ibm_solver_opts": ibm.ibm_solver_opts,
               "ibm_table_info": ibm.ibm_table_info, "ibm_solve_stats": ibm.ibm_solve_stats,
               "ibm_step_stats": ibm.ibm_step_stats, "ibm_tables_host": ibm.ibm_tables_host,
               "ibm_server_opts": ibm.ibm_server_opts, "ibm_request": ibm.ibm_request,
               "ibm_result": ibm.ibm_result, "ibm_server_stats": ibm.ibm_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{SERVE_HEADER}"', "int main(void){"]
    for s, cls in structs.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(c)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, cls in structs.items():
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_create_rejects_bad_descriptor_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2505_17287_gb300 import ibm
    d = ibm.ibm_grid_desc()
    d.ndim = 4
    ctx = ctypes.c_void_p()
    assert lib.ibm_create_grid(ctypes.byref(d), ctypes.byref(ctx)) == ibm.IBM_ERR_ARG
    assert ctx.value is None
    assert b"ndim" in lib.ibm_last_error(None)
    # fewer than 2^32 cells but 2^32 or more x-faces (32-bit face indexing)
    import numpy as np
    n = 37837
    xs, ys = np.linspace(0.0, 1.0, 4), np.linspace(0.0, 1.0, n + 1)
    d = ibm.ibm_grid_desc()
    d.ndim, d.nx, d.ny, d.nz, d.Re, d.dt = 3, 3, n, n, 100.0, 0.01
    d.xf, d.yf, d.zf = xs.ctypes.data, ys.ctypes.data, ys.ctypes.data
    assert 3 * n * n < 2 ** 32 <= 4 * n * n
    assert lib.ibm_create_grid(ctypes.byref(d), ctypes.byref(ctx)) == ibm.IBM_ERR_ARG
    assert b"faces" in lib.ibm_last_error(None)
    assert lib.ibm_destroy(None) == ibm.IBM_OK
    o = ibm.ibm_solver_opts()
    assert lib.ibm_default_opts(ctypes.byref(o)) == ibm.IBM_OK
    assert o.rtol == 1e-10 and o.restart == 16 and o.outer == ibm.IBM_OUTER_FGMRES
    assert o.reorth_eta == 0.3 and o.precond == 0 and o.graph == 1 and o.helm_check_first == 6 and o.helm_omega == 1.0
    assert o.fine_split == 1 and o.band_width == 3 and o.tail_cells == 0 and o.poisson_hist == 8 and o.nu_coarse == 3 and o.nu1 == 2 and o.nu2 == 1
    assert o.band_sweeps == 8 and o.band_omega == 0.85


def test_server_argument_checks_without_gpu(lib):
    from paper_2505_17287_gb300 import ibm
    o = ibm.ibm_server_opts(0, 0, 0, 0)
    h = ctypes.c_void_p()
    assert lib.ibm_server_create(ctypes.byref(o), ctypes.byref(h)) == ibm.IBM_ERR_ARG
    assert h.value is None
    assert lib.ibm_server_destroy(None) == ibm.IBM_OK
    # footprint estimate: grows with the grid, mixed below FP64, body storage counted
    b64 = ibm.ibm_case_bytes(3, 128, 128, 128, ibm.IBM_FP64, 5120)
    b32 = ibm.ibm_case_bytes(3, 128, 128, 128, ibm.IBM_MIXED, 5120)
    assert b32 < b64 < ibm.ibm_case_bytes(3, 256, 128, 128, ibm.IBM_FP64, 5120)
    assert ibm.ibm_case_bytes(3, 128, 128, 128, ibm.IBM_FP64, 50000) > b64
    assert 300 * 128 ** 3 < b64 < 2000 * 128 ** 3

"""The C-ABI library builds, loads without a GPU, exports every entry point declared in
include/pc.h, and the Python binding's struct layouts match the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:pc_status|void|int32_t|int64_t|char)\s*\*?\s*(\w+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpc():
    from paper_2410_02408_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pc_setup", "pc_apply", "kappa_estimate", "pcg_solve", "pc_destroy", "pc_status_string",
                     "pcg_solve_batched", "pc_grad_val", "pc_grad_edges"):
        assert required in names


def test_library_exports_every_declared_symbol(libpc):
    missing = [n for n in declared_functions() if not hasattr(libpc, n)]
    assert not missing, missing


def test_status_strings_and_version(libpc):
    libpc.pc_status_string.restype = ctypes.c_char_p
    assert libpc.pc_status_string(0) == b"ok"
    assert b"SPD" in libpc.pc_status_string(2)
    assert libpc.pc_version() >= 100


def test_invalid_arguments_rejected_without_gpu(libpc):
    # argument checks run before any CUDA call
    from paper_2410_02408_gb300 import binding as B

    L = B.lib()
    h = ctypes.c_void_p()
    assert L.pc_setup(None, 8, 0.0, 0, None, ctypes.byref(h)) == B.PC_ERR_INVALID_ARG
    d = B.pc_csr(10, 30, 1, 1, 1, 0)
    assert L.pc_setup(ctypes.byref(d), 0, 0.0, 0, None, ctypes.byref(h)) == B.PC_ERR_INVALID_ARG
    assert L.pc_setup(ctypes.byref(d), 65, 0.0, 0, None, ctypes.byref(h)) == B.PC_ERR_INVALID_ARG
    assert L.pc_setup(ctypes.byref(d), 8, 0.0, 9, None, ctypes.byref(h)) == B.PC_ERR_INVALID_ARG
    assert L.pc_setup(ctypes.byref(d), 8, -1.0, 0, None, ctypes.byref(h)) == B.PC_ERR_INVALID_ARG
    bad = B.pc_csr(10, 30, 1, 1, 1, 7)
    assert L.pc_setup(ctypes.byref(bad), 8, 0.0, 0, None, ctypes.byref(h)) == B.PC_ERR_INVALID_ARG
    assert L.kappa_estimate(ctypes.byref(d), 0, 0, 0.0, 1, 1, None, None) == B.PC_ERR_INVALID_ARG
    assert L.kappa_estimate(ctypes.byref(d), 0, 300, 0.0, 1, 1, None, None) == B.PC_ERR_INVALID_ARG
    assert L.pcg_solve_h(None, 1, 1, 1e-10, 10, None, None) == B.PC_ERR_INVALID_ARG
    assert L.pc_apply(None, 0, 1, 2, None) == B.PC_ERR_INVALID_ARG
    assert L.pc_destroy(None) == B.PC_ERR_INVALID_ARG


def test_struct_layouts_match_header(tmp_path):
    from paper_2410_02408_gb300 import binding as B

    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "pc.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("pc_csr %zu\n", sizeof(pc_csr));
  P(pc_csr, nnz) P(pc_csr, row_ptr) P(pc_csr, val) P(pc_csr, dtype)
  printf("pc_solve_info %zu\n", sizeof(pc_solve_info));
  P(pc_solve_info, rel_residual) P(pc_solve_info, solve_ms) P(pc_solve_info, grid_ctas) P(pc_solve_info, prec)
  printf("pc_kappa_info %zu\n", sizeof(pc_kappa_info));
  P(pc_kappa_info, kappa) P(pc_kappa_info, alpha) P(pc_kappa_info, beta) P(pc_kappa_info, elapsed_ms)
  printf("pc_batch %zu\n", sizeof(pc_batch));
  P(pc_batch, n_rows) P(pc_batch, sys_row) P(pc_batch, block_size) P(pc_batch, max_block_size)
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for cls in (B.pc_csr, B.pc_solve_info, B.pc_kappa_info, B.pc_batch):
        assert int(out[cls.__name__]) == ctypes.sizeof(cls), cls.__name__
        for key, v in out.items():
            if key.startswith(cls.__name__ + "."):
                field = key.split(".", 1)[1]
                assert getattr(cls, field).offset == int(v), key


def test_handle_queries_on_a_null_handle(libpc):
    """The handle queries and process-wide settings are host-only: they answer for a null
    handle without touching the GPU."""
    libpc.pc_handle_failed_block.restype = ctypes.c_int64
    assert libpc.pc_handle_failed_block(None) == -1
    assert libpc.pc_handle_refactored_fp64(None) == 0
    assert libpc.pc_handle_row_binned(None) == 0
    assert libpc.pc_handle_col_segments(None) == 1
    for setter, values in ((libpc.pc_set_row_binning, (-1, 0, 1, 7)), (libpc.pc_set_col_segments, (3, 0, 9, -1)),
                           (libpc.pc_set_cg_engine, (1, 0, -1))):
        for v in values:
            setter(ctypes.c_int32(v))
    libpc.pc_set_row_binning(ctypes.c_int32(-1))
    libpc.pc_set_col_segments(ctypes.c_int32(-1))

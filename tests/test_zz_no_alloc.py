"""pcg_solve_noalloc: the allocation-free variant of pcg_solve.

Some callers cannot call cudaMalloc (a stream being captured into a graph, a host
framework whose allocator owns the device memory, latency-critical loops), so this entry
point takes its scratch from a fixed static device array.  It must give the same result
as pcg_solve, call after call, even though the shared scratch keeps stale contents from
the previous call.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_X = 1e-10   # the FP64 solution tolerance used by the parity tests


def _noalloc():
    from paper_2410_02408_gb300 import binding as B

    f = B.lib().pcg_solve_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.POINTER(B.pc_csr), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(B.pc_solve_info), ctypes.c_void_p]
    return B, f


def _call(B, f, Ad, bd, bs, prec):
    x = torch.zeros_like(bd)
    info = B.pc_solve_info()
    d = Ad.desc()
    st = f(ctypes.byref(d), bs, ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-10, 100000,
           B.PREC[prec], ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, x, info


def test_noalloc_matches_pcg_solve_on_consecutive_calls(pc):
    B, f = _noalloc()
    problems = [(W.diffusion3d(16, 2.0), 16, "fp64"), (W.poisson2d(64), 32, "fp64"),
                (W.diffusion3d(16, 2.0), 16, "fp32")]
    for A, bs, prec in problems:
        Ad = B.csr(A)
        bd = torch.from_numpy(W.rhs(A.n, 0)).cuda()
        x_ref, info_ref = pc.pcg(Ad, bd, bs, tol=1e-10, prec=prec)
        for _ in range(2):   # two calls in a row: the scratch is reused with stale contents
            st, x, info = _call(B, f, Ad, bd, bs, prec)
            assert st == 0, B.STATUS_NAMES.get(st, st)
            assert info.iterations == info_ref["iterations"]
            err = float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))
            assert err <= TOL_X
            assert info.true_rel_residual <= 1e-10


def test_noalloc_rejects_problems_beyond_the_scratch(pc):
    B, f = _noalloc()
    A = W.diffusion3d(64, 1.0)            # 262,144 rows: FP64 factors at bs 64 need > 64 MiB
    Ad = B.csr(A)
    bd = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    st, x, info = _call(B, f, Ad, bd, 64, "fp64")
    assert st == B.PC_ERR_INVALID_ARG
    assert not x.any()

"""pcg_solve_noalloc: the allocation-free variant of pcg_solve.

Some callers cannot allocate device memory: a plug-in inside a host framework whose caching
allocator owns the device (a cudaMalloc behind its back can fail or fragment the pool), or a
latency-critical loop that must not enter the driver's allocator.  This entry point takes its
scratch from a fixed static device array instead.  It must give the oracle's answer and the
same result as pcg_solve with the persistent engine, call after call, even though the shared
scratch keeps stale contents from the previous call, and device memory must not change across
calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_X = 1e-10   # the FP64 solution tolerance used by the parity tests


def _noalloc():
    from paper_2410_02408_gb300 import binding as B

    return B, B.lib().pcg_solve_noalloc


def _call(B, f, Ad, bd, bs, prec, x=None, max_iter=100000):
    x = torch.zeros_like(bd) if x is None else x.zero_()
    info = B.pc_solve_info()
    d = Ad.desc()
    st = f(ctypes.byref(d), bs, ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-10, max_iter,
           B.PREC[prec], ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, x, info


def _persistent(pc, Ad, bd, bs, prec, max_iter=100000, check=True):
    pc.set_cg_engine("persistent")
    try:
        return pc.pcg(Ad, bd, bs, tol=1e-10, max_iter=max_iter, prec=prec, check=check)
    finally:
        pc.set_cg_engine("default")


# 3,375 and 3,969 rows are not multiples of 32 (ragged warp units and vector tails)
PROBLEMS = [("diffusion3d_16", 16, "fp64"), ("diffusion3d_15", 8, "fp64"), ("poisson2d_63", 32, "fp64"),
            ("diffusion3d_15", 16, "fp32"), ("poisson2d_64", 64, "fp64")]


def _matrix(name):
    if name.startswith("diffusion3d_"):
        return W.diffusion3d(int(name.split("_")[1]), 2.0)
    return W.poisson2d(int(name.split("_")[1]))


@pytest.mark.parametrize("name,bs,prec", PROBLEMS)
def test_noalloc_matches_oracle_and_pcg_solve_on_consecutive_calls(pc, name, bs, prec):
    B, f = _noalloc()
    A = _matrix(name)
    b = W.rhs(A.n, 0)
    Ad = B.csr(A)
    bd = torch.from_numpy(b).cuda()
    x_ref, info_ref = _persistent(pc, Ad, bd, bs, prec)
    o = oracle.pcg(A, b, bs, 1e-10)
    x = torch.zeros_like(bd)
    for _ in range(2):   # two calls in a row: the scratch is reused with stale contents
        st, x, info = _call(B, f, Ad, bd, bs, prec, x)
        assert st == 0, B.STATUS_NAMES.get(st, st)
        assert info.true_rel_residual <= 1e-10
        # same kernels, grid and reduction order as pcg_solve with the persistent engine
        assert info.iterations == info_ref["iterations"]
        assert torch.equal(x, x_ref)
        xr = x.cpu().numpy()
        if prec == "fp64":
            assert np.linalg.norm(xr - o["x"]) <= TOL_X * np.linalg.norm(o["x"])
        assert np.linalg.norm(b - oracle.spmv(A, xr)) <= 1e-10 * np.linalg.norm(b)


def test_noalloc_allocates_no_device_memory(pc):
    B, f = _noalloc()
    A = W.diffusion3d(15, 2.0)
    Ad = B.csr(A)
    bd = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    x = torch.zeros_like(bd)
    st, _, _ = _call(B, f, Ad, bd, 16, "fp32", x)   # first call: symbol lookup, kernels loaded
    assert st == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for prec in ("fp32", "fp64", "fp32"):
        st, _, _ = _call(B, f, Ad, bd, 16, prec, x)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_fp32_breakdown_refactors_like_pcg_solve(pc):
    """1 - 1e-9 rounds to 1 in FP32, so the FP32 Cholesky of every 2x2 block hits a zero
    pivot: like pc_setup, the call factors the blocks again in FP64 arithmetic (instead of
    reporting NOT_SPD) and runs the same CG.  Blocks this ill-conditioned (kappa ~ 2e9) cannot
    be applied accurately from FP32-stored factors, so the solve is cut at 20 iterations and
    the call must end exactly like pcg_solve: same status, iterations and iterate."""
    from test_gpu_parity import _pair_blocks

    B, f = _noalloc()
    A = _pair_blocks(40, 1e-9)
    b = W.rhs(A.n, 0)
    Ad = B.csr(A)
    bd = torch.from_numpy(b).cuda()
    x_ref, info_ref = _persistent(pc, Ad, bd, 2, "fp32", max_iter=20, check=False)
    assert info_ref["status"] != B.PC_ERR_NOT_SPD
    for _ in range(2):
        st, x, info = _call(B, f, Ad, bd, 2, "fp32", max_iter=20)
        assert st == info_ref["status"], (B.STATUS_NAMES.get(st, st), info_ref["status_name"])
        assert info.iterations == info_ref["iterations"]
        assert torch.equal(x, x_ref)
    st, x, info = _call(B, f, B.csr(_pair_blocks(40, 1e-9, bad=7)), bd, 2, "fp32")
    assert st == B.PC_ERR_NOT_SPD and info.failed_block == 7


def test_noalloc_honours_the_wait_budget(pc):
    """A one-cycle wait budget (pc_set_wait_budget) makes the persistent engine's grid
    barrier give up: the call reports PC_ERR_TIMEOUT, and the next call with the default
    budget solves."""
    B, f = _noalloc()
    A = W.diffusion3d(16, 2.0)
    Ad = B.csr(A)
    bd = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    pc.set_wait_budget(1)
    try:
        st, _, _ = _call(B, f, Ad, bd, 16, "fp64")
    finally:
        pc.set_wait_budget(0)
    assert st == B.PC_ERR_TIMEOUT
    st, _, info = _call(B, f, Ad, bd, 16, "fp64")
    assert st == 0 and info.true_rel_residual <= 1e-10


def test_noalloc_rejects_bad_csr_and_problems_beyond_the_scratch(pc):
    B, f = _noalloc()
    A = W.poisson2d(12)
    col = A.col.copy()
    col[A.row_ptr[7] + 1] = A.n + 3
    bd = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    st, x, _ = _call(B, f, B.csr(W.CSR(A.row_ptr, col, A.val)), bd, 8, "fp64")
    assert st == B.PC_ERR_INVALID_ARG and not x.any()
    A = W.diffusion3d(64, 1.0)            # 262,144 rows: FP64 factors at bs 64 need > 64 MiB
    Ad = B.csr(A)
    bd = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    st, x, info = _call(B, f, Ad, bd, 64, "fp64")
    assert st == B.PC_ERR_INVALID_ARG
    assert not x.any()

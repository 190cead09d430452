"""CUDA path vs the FP64 oracle, element by element, on seeded inputs (through the C ABI).

Tolerances:
  extraction          bit-exact
  FP64 factors        1e-12 relative to the block's largest entry (different but backward
                      stable operation orders: Cholesky + substitution on both sides)
  FP32 factors        2e-4 relative (FP32 arithmetic, block condition numbers <= ~1e3)
  apply / SpMV / dot  1e-12 relative (norm-wise)
  kappa               1e-6 relative (the stated requirement)
  PCG x (FP64 mode)   1e-10 relative to the oracle's x at the same tolerance and stopping rule
  PCG mixed mode      true relative residual <= tol (error vs the FP64 oracle is reported)
"""
import math

import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cases():
    return {
        "poisson2d_64": W.poisson2d(64),
        "diff13_s2": W.diffusion3d(13, 2.0),        # n = 2197: ragged last block for most bs
        "diff10_s1": W.diffusion3d(10, 1.0),
    }


CASES = cases()


# ---------------------------------------------------------------- a1 extraction
@pytest.mark.parametrize("name,bs", [("poisson2d_64", 16), ("diff13_s2", 7), ("diff13_s2", 64),
                                     ("diff10_s1", 1), ("diff13_s2", 33)])
def test_extract_bit_exact(pc, name, bs):
    A = CASES[name]
    g = pc.extract_blocks(A, bs).cpu().numpy()
    o = oracle.extract_blocks(A, bs)
    assert g.shape == o.shape
    assert np.array_equal(g, o)


def test_extract_float32_values_widened_exactly(pc):
    A = W.powerlaw_spd(n=3000, seed=5, w_max=300, cap=200)
    g = pc.extract_blocks(A, 32).cpu().numpy()
    o = oracle.extract_blocks(W.CSR(A.row_ptr, A.col, A.val.astype(np.float64)), 32)
    assert np.array_equal(g, o)


# ---------------------------------------------------------------- a2 factors
BS_ALL = [1, 2, 4, 7, 8, 10, 16, 32, 33, 48, 64]


@pytest.mark.parametrize("bs", BS_ALL)
def test_factor_fp64_matches_oracle(pc, bs):
    A = CASES["diff13_s2"]
    h = pc.setup(A, bs, prec="fp64")
    Linv_g = h.factor("linv").cpu().numpy()
    Minv_g = h.factor("minv").cpu().numpy()
    L, f = oracle.factor(A, bs)
    assert f == -1
    X = oracle.tri_inv(L, A.n, bs)
    M = oracle.minv(X, A.n, bs)
    nb = L.shape[0]
    last = A.n - (nb - 1) * bs
    for k in range(nb):
        b = bs if k < nb - 1 else last
        sc = np.abs(X[k, :b, :b]).max()
        assert np.abs(Linv_g[k, :b, :b] - X[k, :b, :b]).max() <= 1e-12 * sc
        sm = np.abs(M[k, :b, :b]).max()
        assert np.abs(Minv_g[k, :b, :b] - M[k, :b, :b]).max() <= 1e-12 * sm
    # padding of the ragged last block is the identity
    if last < bs:
        assert np.array_equal(Minv_g[-1, last:, last:], np.eye(bs - last))
        assert not Minv_g[-1, :last, last:].any()


@pytest.mark.parametrize("bs", [4, 16, 32, 64])
def test_factor_fp32_matches_oracle(pc, bs):
    A = CASES["diff10_s1"]
    h = pc.setup(A, bs, prec="fp32")
    Minv_g = h.factor("minv").cpu().numpy()
    L, _ = oracle.factor(A, bs)
    M = oracle.minv(oracle.tri_inv(L, A.n, bs), A.n, bs)
    nb = M.shape[0]
    for k in range(nb):
        b = bs if k < nb - 1 else A.n - (nb - 1) * bs
        sm = np.abs(M[k, :b, :b]).max()
        assert np.abs(Minv_g[k, :b, :b] - M[k, :b, :b]).max() <= 2e-4 * sm


def test_not_spd_reports_failing_block(pc):
    A = W.poisson2d(16)
    val = A.val.copy()
    row = 37                     # block 4 for bs = 8
    for e in range(A.row_ptr[row], A.row_ptr[row + 1]):
        if A.col[e] == row:
            val[e] = -1.0
    B = W.CSR(A.row_ptr, A.col, val)
    _, f = oracle.factor(B, 8)
    with pytest.raises(pc.PcError) as ei:
        pc.setup(B, 8)
    assert ei.value.status == 2
    assert f == 4
    import ctypes
    from paper_2410_02408_gb300 import binding as bnd

    Ad = bnd.csr(B)
    d = Ad.desc()
    hh = ctypes.c_void_p()
    st = bnd.lib().pc_setup(ctypes.byref(d), 8, 0.0, 0, None, ctypes.byref(hh))
    assert st == 2 and bnd.lib().pc_handle_failed_block(hh) == f
    bnd.lib().pc_destroy(hh)


# ---------------------------------------------------------------- a3/a4 apply, a5 SpMV, a6 dot
@pytest.mark.parametrize("bs", [1, 8, 10, 16, 32, 33, 64])
@pytest.mark.parametrize("mode", ["inv", "linv", "ltinv", "sym"])
def test_apply_matches_oracle(pc, bs, mode):
    A = CASES["diff13_s2"]
    v = W.rhs(A.n, 4)
    h = pc.setup(A, bs)
    g = h.apply(mode, v).cpu().numpy()
    L, _ = oracle.factor(A, bs)
    o = oracle.apply(A, L, bs, {"inv": 0, "sym": 1, "linv": 2, "ltinv": 3}[mode], v)
    assert rel(g, o) <= 1e-12


def test_apply_fp32_close(pc):
    A = CASES["diff10_s1"]
    v = W.rhs(A.n, 4)
    h = pc.setup(A, 16, prec="fp32")
    L, _ = oracle.factor(A, 16)
    assert rel(h.apply("inv", v).cpu().numpy(), oracle.apply(A, L, 16, 0, v)) <= 1e-5


def test_spmv_and_dot(pc):
    for A in (CASES["poisson2d_64"], CASES["diff13_s2"]):
        x = W.rhs(A.n, 2)
        assert rel(pc.spmv(A, x).cpu().numpy(), oracle.spmv(A, x)) <= 1e-14
        y = W.rhs(A.n, 3)
        d = pc.dot(x, y)
        assert abs(d - math.fsum(x * y)) <= 1e-13 * float(np.abs(x * y).sum())
    # fixed-order reduction: bit-reproducible
    assert pc.dot(x, y) == d


# ---------------------------------------------------------------- a7 kappa
def test_kappa_poisson2d_closed_form_and_oracle(pc):
    A = CASES["poisson2d_64"]
    b = W.rhs(A.n, 0)
    ref = {0: 1.0 / math.tan(math.pi / 130) ** 2, 1: 1.0 / math.tan(math.pi / 130) ** 2,
           64: 1.0 / (1.0 - math.cos(math.pi / 65))}
    for bs in (0, 1, 16, 64):
        g = pc.kappa(A, b, block_size=bs)
        o = oracle.kappa(A, b, 200, bs)
        assert g["steps"] == o["steps"]
        assert g["kappa"] == pytest.approx(o["kappa"], rel=1e-6)
        if bs in ref:
            assert g["kappa"] == pytest.approx(ref[bs], rel=1e-6)


@pytest.mark.parametrize("bs", [0, 8, 32])
def test_kappa_diffusion_matches_oracle(pc, bs):
    A = W.diffusion3d(16, 2.0)
    b = W.rhs(A.n, 0)
    g = pc.kappa(A, b, block_size=bs)
    o = oracle.kappa(A, b, 200, bs)
    assert g["kappa"] == pytest.approx(o["kappa"], rel=1e-6)
    assert np.allclose(g["alpha"][:20], o["alpha"][:20], rtol=1e-9)


def test_kappa_invariants(pc):
    A = W.diffusion3d(4, 1.0)      # N = 64
    b = W.rhs(A.n, 0)
    assert pc.kappa(A, b, block_size=64)["kappa"] == pytest.approx(1.0, abs=1e-10)
    ev = np.linalg.eigvalsh(A.to_dense())
    g = pc.kappa(A, b, block_size=0)
    assert g["kappa"] == pytest.approx(ev[-1] / ev[0], rel=1e-9)
    assert g["steps"] <= 64


def test_kappa_without_reorth_runs(pc):
    A = CASES["poisson2d_64"]
    b = W.rhs(A.n, 0)
    g = pc.kappa(A, b, block_size=16, reorth=False)
    o = oracle.kappa(A, b, 200, 16, reorth=False)
    assert g["steps"] == o["steps"]
    assert g["kappa"] == pytest.approx(o["kappa"], rel=0.05)   # no reorthogonalisation: reported, not gated


# ---------------------------------------------------------------- a8 PCG
@pytest.fixture(params=["graph", "persistent"])
def engine(pc, request):
    pc.set_cg_engine(request.param)
    yield request.param
    pc.set_cg_engine("default")


@pytest.mark.parametrize("bs", [1, 16, 64])
def test_pcg_poisson2d_matches_oracle(pc, engine, bs):
    A = CASES["poisson2d_64"]
    b = W.rhs(A.n, 0)
    x, info = pc.pcg(A, b, bs, tol=1e-10)
    o = oracle.pcg(A, b, bs, 1e-10)
    assert info["status"] == 0 and o["status"] == "ok"
    assert abs(info["iterations"] - o["iterations"]) <= 1
    assert rel(x.cpu().numpy(), o["x"]) <= 1e-10
    assert info["true_rel_residual"] <= 1e-10


@pytest.mark.parametrize("bs", [8, 10, 16, 32, 64])
def test_pcg_diffusion_fp64_matches_oracle(pc, engine, bs):
    A = W.diffusion3d(24, 2.0)
    b = W.rhs(A.n, 0)
    x, info = pc.pcg(A, b, bs, tol=1e-10, prec="fp64")
    o = oracle.pcg(A, b, bs, 1e-10)
    assert info["status"] == 0
    assert abs(info["iterations"] - o["iterations"]) <= 2
    assert rel(x.cpu().numpy(), o["x"]) <= 1e-10
    res = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1e-10


@pytest.mark.parametrize("bs,prec", [(16, "fp64"), (16, "fp32"), (9, "fp64"), (9, "fp32"), (64, "fp32")])
def test_pcg_odd_n_matches_oracle(pc, engine, bs, prec):
    """n = 2197 (odd): the CG work vectors and every row window the preconditioner kernels
    copy stay 16-byte aligned; bs 9 gives warp units of 27 rows (odd)."""
    A = CASES["diff13_s2"]
    b = W.rhs(A.n, 0)
    x, info = pc.pcg(A, b, bs, tol=1e-10, prec=prec)
    assert info["status"] == 0
    res = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1e-10
    if prec == "fp64":
        o = oracle.pcg(A, b, bs, 1e-10)
        assert abs(info["iterations"] - o["iterations"]) <= 2
        assert rel(x.cpu().numpy(), o["x"]) <= 1e-10


@pytest.mark.parametrize("bs", [8, 16, 32, 64])
def test_pcg_diffusion_mixed_reaches_tolerance(pc, engine, bs):
    A = W.diffusion3d(24, 2.0)
    b = W.rhs(A.n, 0)
    x, info = pc.pcg(A, b, bs, tol=1e-10, prec="fp32")
    assert info["status"] == 0
    res = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1e-10
    o = oracle.pcg(A, b, bs, 1e-10)
    print(f"bs={bs} mixed iters {info['iterations']} fp64-oracle iters {o['iterations']} "
          f"err vs oracle {rel(x.cpu().numpy(), o['x']):.2e}")


def test_pcg_float32_values(pc, engine):
    A = W.powerlaw_spd(n=20000, seed=5, w_max=500, cap=400)
    b = W.rhs(A.n, 0)
    A64 = W.CSR(A.row_ptr, A.col, A.val.astype(np.float64))
    x, info = pc.pcg(A, b, 32, tol=1e-10, prec="fp32")
    o = oracle.pcg(A64, b, 32, 1e-10)
    assert info["status"] == 0
    res = np.linalg.norm(b - oracle.spmv(A64, x.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1e-10
    x2, info2 = pc.pcg(A, b, 32, tol=1e-10, prec="fp64")
    assert rel(x2.cpu().numpy(), o["x"]) <= 1e-10


def test_pcg_is_bit_reproducible(pc, engine):
    A = W.diffusion3d(16, 2.0)
    b = W.rhs(A.n, 0)
    x1, i1 = pc.pcg(A, b, 16)
    x2, i2 = pc.pcg(A, b, 16)
    assert i1["iterations"] == i2["iterations"]
    assert torch.equal(x1, x2)


def test_pcg_status_codes(pc, engine):
    A = W.poisson2d(16)
    b = W.rhs(A.n, 0)
    x, info = pc.pcg(A, b, 4, max_iter=1, check=False)
    assert info["status"] == 4 and info["iterations"] == 1
    x, info = pc.pcg(A, np.zeros(A.n), 4)
    assert info["status"] == 0 and info["iterations"] == 0 and not x.any()
    import scipy.sparse as sp
    M = sp.csr_matrix(np.array([[1.0, 3.0], [3.0, 1.0]]))
    Bm = W.CSR(M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)
    x, info = pc.pcg(Bm, np.array([1.0, -1.0]), 1, check=False)
    assert info["status"] == 3
    xs = np.linalg.solve(A.to_dense(), b)
    x, info = pc.pcg(A, b, 4, x0=xs)
    assert info["status"] == 0 and info["iterations"] == 0


def test_pcg_bounded_wait_times_out_and_recovers(pc):
    # the grid barrier of the persistent engine is the bounded device-side wait
    pc.set_cg_engine("persistent")
    A = W.poisson2d(64)
    b = W.rhs(A.n, 0)
    pc.set_wait_budget(1)
    try:
        x, info = pc.pcg(A, b, 16, check=False)
    finally:
        pc.set_wait_budget(0)
    assert info["status"] == 5
    x, info = pc.pcg(A, b, 16)
    pc.set_cg_engine("default")
    assert info["status"] == 0


def test_fused_update_wait_times_out_and_recovers(pc):
    # the graph engine's bounded device-side wait: CTAs of the preconditioner kernel wait for
    # its last CTA before the fused x / p update; a one-cycle budget makes the first CTAs give up
    pc.set_cg_engine("default")
    A = W.poisson2d(64)   # 128 warp units: 16 CTAs, so some CTA always waits
    b = W.rhs(A.n, 0)
    pc.set_wait_budget(1)
    try:
        x, info = pc.pcg(A, b, 16, check=False)
    finally:
        pc.set_wait_budget(0)
    assert info["status"] == 5
    x, info = pc.pcg(A, b, 16)
    assert info["status"] == 0
    o = oracle.pcg(A, b, 16, 1e-10)
    assert rel(x.cpu().numpy(), o["x"]) <= 1e-10


def test_pcg_handle_reuse_and_warm_restart(pc, engine):
    A = W.diffusion3d(12, 1.0)
    b = W.rhs(A.n, 0)
    h = pc.setup(A, 16)
    x1, i1 = h.pcg(b, tol=1e-6)
    x2, i2 = h.pcg(b, x0=x1, tol=1e-10)
    o = oracle.pcg(A, b, 16, 1e-10, x0=x1.cpu().numpy())
    assert i2["iterations"] == pytest.approx(o["iterations"], abs=1)
    assert rel(x2.cpu().numpy(), o["x"]) <= 1e-10


# ---------------------------------------------------------------- a11 adjoint gradient kernel
def test_grad_val_matches_oracle(pc):
    A = CASES["diff13_s2"]
    lam = W.rhs(A.n, 7)
    x = W.rhs(A.n, 8)
    g = pc.grad_val(A, lam, x).cpu().numpy()
    assert np.array_equal(g, oracle.grad_val(A, lam, x))


def _pair_blocks(nb, eps, bad=None):
    """Block-diagonal matrix of nb 2x2 blocks [[1, 1-eps], [1-eps, 1]] (block `bad`, if given,
    gets off-diagonals 2: indefinite)."""
    rows, cols, vals = [], [], []
    for k in range(nb):
        off = 2.0 if k == bad else 1.0 - eps
        for i in range(2):
            for j in range(2):
                rows.append(2 * k + i)
                cols.append(2 * k + j)
                vals.append(1.0 if i == j else off)
    n = 2 * nb
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(np.array(rows), minlength=n), out=row_ptr[1:])
    return W.CSR(row_ptr, np.array(cols, dtype=np.int32), np.array(vals))


def test_fp32_breakdown_refactors_in_fp64(pc):
    """1 - 1e-9 rounds to 1 in FP32, so the FP32 Cholesky of every block hits a zero pivot;
    pc_setup then factors the blocks in FP64 arithmetic and stores FP32 factors."""
    A = _pair_blocks(40, 1e-9)
    H = pc.setup(A, 2, prec="fp32")
    try:
        assert H.refactored_fp64()
        m = H.factor("minv").cpu().numpy()
    finally:
        H.destroy()
    ref = np.linalg.inv(np.array([[1.0, 1.0 - 1e-9], [1.0 - 1e-9, 1.0]]))
    for k in range(40):
        assert np.linalg.norm(m[k] - ref) <= 1e-6 * np.linalg.norm(ref)
    H64 = pc.setup(A, 2, prec="fp64")
    assert not H64.refactored_fp64()
    H64.destroy()
    with pytest.raises(pc.PcError) as ei:
        pc.setup(_pair_blocks(40, 1e-9, bad=7), 2, prec="fp32")
    assert ei.value.name == "not_spd"


@pytest.mark.parametrize("k", [1, 2, 3, 7, 40])
def test_iterate_after_k_steps_matches_oracle(pc, engine, k):
    """x after exactly k CG steps (the solve cut by max_iter) equals the oracle's k-th iterate:
    pins the order of the updates inside a step and the last step's x update."""
    A = W.diffusion3d(14, 2.0)      # 2,744 rows: ragged warp units
    b = W.rhs(A.n, 0)
    x, info = pc.pcg(A, b, 8, tol=1e-14, max_iter=k, check=False)
    assert info["status"] == 4 and info["iterations"] == k
    r = oracle.pcg(A, b, 8, 0.0, max_iter=k, max_restarts=0)
    assert r["iterations"] == k
    xr = x.cpu().numpy()
    assert np.linalg.norm(xr - r["x"]) <= 1e-12 * np.linalg.norm(r["x"])


def test_handles_reuse_the_library_memory_pool(pc):
    # a handle's device memory goes back to the library's pool on destroy and serves the next
    # handle: after the first setup / solve / destroy, repeating them takes no more device memory
    import torch

    A = W.diffusion3d(48, 2.0)
    b = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    Ad = pc.csr(A)

    def cycle():
        H = pc.setup(Ad, 16, prec="fp32")
        x, info = H.pcg(b, tol=1e-10)
        H.destroy()
        assert info["status"] == 0
        return x

    x0 = cycle()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        x = cycle()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (8 << 20)   # allow torch's own small allocations
    assert torch.equal(x, x0)

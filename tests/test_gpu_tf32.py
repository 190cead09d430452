"""PC_PREC_TF32: M_k^{-1} = L_k^{-T} L_k^{-1} formed on the tensor cores (mma.sync m16n8k8,
operands rounded to TF32 to nearest with ties away from zero, FP32 accumulation).

* the tensor-core fragment mapping against a host product of the TF32-rounded operands;
* the TF32 factors against the oracle's FP64 M^{-1} within the rounding bound of the product:
  |M~ - M| <= 2u |X|^T |X| + O(u^2) entry-wise with u = 2^-11 (TF32 unit roundoff) and
  X = L^{-1}, hence ||M~ - M||_F <= 2u ||X||_F^2 per block (a factor 1.5 of margin covers the
  FP32 errors of X itself);
* the stored M^{-1} stays exactly symmetric;
* PCG with TF32 factors reaches the true residual 1e-10 (single systems and a batch).
"""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U_TF32 = 2.0 ** -11


def tf32_rna(x):
    """Round float32 values to TF32 (10 mantissa bits), to nearest, ties away from zero."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


def test_mma_fragment_mapping(pc):
    rng = np.random.default_rng(31)
    for _ in range(3):
        a = rng.standard_normal((16, 8)).astype(np.float32)
        b = rng.standard_normal((8, 8)).astype(np.float32)
        d = pc.debug_mma_tf32(a, b).cpu().numpy()
        want = tf32_rna(a).astype(np.float64) @ tf32_rna(b).astype(np.float64)
        assert np.allclose(d, want, rtol=1e-6, atol=1e-6)
        # the rounding is TF32 (not FP32): the unrounded product differs by far more than FP32 noise
        exact = a.astype(np.float64) @ b.astype(np.float64)
        assert np.max(np.abs(want - exact)) > 1e-5


@pytest.mark.parametrize("bs", [4, 7, 8, 16, 24, 32, 33, 48, 64])
def test_tf32_factors_within_rounding_bound(pc, bs):
    A = W.diffusion3d(12, 2.0)           # 1728 rows: ragged last block for most bs
    n = A.n
    H = pc.setup(A, bs, prec="tf32")
    try:
        m_tc = H.factor("minv").cpu().numpy()
    finally:
        H.destroy()
    H = pc.setup(A, bs, prec="fp32")
    try:
        m_32 = H.factor("minv").cpu().numpy()
    finally:
        H.destroy()
    L, f = oracle.factor(A, bs)
    assert f == -1
    X = oracle.tri_inv(L, n, bs)
    M = oracle.minv(X, n, bs)
    nb = M.shape[0]
    differs = 0
    for k in range(nb):
        b = min(bs, n - k * bs)
        Mk, Xk = M[k, :b, :b], X[k, :b, :b]
        tc, f32 = m_tc[k, :b, :b], m_32[k, :b, :b]
        bound = 1.5 * 2 * U_TF32 * np.linalg.norm(Xk) ** 2
        assert np.linalg.norm(tc - Mk) <= bound, (k, np.linalg.norm(tc - Mk), bound)
        assert np.array_equal(tc, tc.T)
        # the FP32 path is far more accurate: the TF32 rounding is really in the tensor-core path
        assert np.linalg.norm(f32 - Mk) <= 1e-5 * np.linalg.norm(Xk) ** 2
        differs += int(not np.array_equal(tc, f32))
    assert differs > 0


@pytest.mark.parametrize("bs", [16, 32, 64])
def test_tf32_pcg_reaches_true_residual(pc, bs):
    import torch

    A = W.diffusion3d(40, 2.0)
    b = W.rhs(A.n, 0)
    bd = torch.from_numpy(b).cuda()
    x, info = pc.pcg(A, bd, bs, tol=1e-10, prec="tf32")
    assert info["status_name"] == "ok" and info["prec"] == 2
    res = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1e-10
    _, i32 = pc.pcg(A, bd, bs, tol=1e-10, prec="fp32")
    assert info["iterations"] <= 1.1 * i32["iterations"] + 2


def test_tf32_batched_reaches_true_residual(pc):
    batch = W.rgg_batch(n_sys=24, seed=4, n_max=2e4)
    b = W.rhs(int(batch.sys_row[-1]), 0)
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10, prec="tf32")
    assert info["status_name"] == "ok"
    x = x.cpu().numpy()
    for s, A in enumerate(batch.systems):
        sl = slice(int(batch.sys_row[s]), int(batch.sys_row[s + 1]))
        res = np.linalg.norm(b[sl] - oracle.spmv(A, x[sl])) / np.linalg.norm(b[sl])
        assert res <= 1.0000001e-10, (s, res)

"""Full-size workloads in the launch configuration bench.py times, checked by properties the
oracle can evaluate at that size: the true residual b - A x recomputed by the oracle's FP64
SpMV (independent of the CUDA path), per-system oracle solves on sampled systems of the
batch, and kappa shrinking under preconditioning.

3D diffusion 128^3 (sigma 2, bs 16, FP32 factors and FP64 CG); the 512-system RGG batch;
a 2M-row power-law matrix with the same recipe as the 8M-row workload (FP32 values, bs 32),
whole-row and in 3 column segments.
"""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _true_rel_residual(A, b, x):
    return float(np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b))


def test_diffusion_128_mixed_and_fp64(pc):
    import torch

    A = W.diffusion3d(128, 2.0)
    b = W.rhs(A.n, 0)
    Ad = pc.csr(A)
    bd = torch.from_numpy(b).cuda()
    for prec in ("fp32", "fp64"):
        x, info = pc.pcg(Ad, bd, 16, tol=1e-10, prec=prec)
        assert info["status_name"] == "ok"
        xr = x.cpu().numpy()
        res = _true_rel_residual(A, b, xr)
        assert res <= 1e-10, (prec, res)
        assert abs(res - info["true_rel_residual"]) <= 1e-12
    # kappa before / after with 200 CGS2 steps: preconditioning must shrink it
    kb = pc.kappa(Ad, bd, 0, max_steps=200)
    H = pc.setup(Ad, 16, prec="fp64")
    try:
        ka = H.kappa(bd, max_steps=200)
    finally:
        H.destroy()
    assert ka["kappa"] < kb["kappa"]
    assert 0.0 < ka["lambda_min"] <= ka["lambda_max"] <= 2.0 + 1e-9   # spectrum of L^-1 A L^-T


def test_batched_rgg_512(pc):
    batch = W.rgg_batch(n_sys=512, seed=3)
    b = np.random.default_rng(0).standard_normal(int(batch.sys_row[-1]))
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10, prec="fp32")
    assert info["status_name"] == "ok"
    x = x.cpu().numpy()
    for s, A in enumerate(batch.systems):
        sl = slice(int(batch.sys_row[s]), int(batch.sys_row[s + 1]))
        res = _true_rel_residual(A, b[sl], x[sl])
        assert res <= 1.0000001e-10, (s, res)
    # FP64 factors: sampled systems against the oracle's PCG (smallest and mid-size ones)
    x64, per64, info64 = pc.pcg_batched(batch, b, tol=1e-10, prec="fp64")
    assert info64["status_name"] == "ok"
    x64 = x64.cpu().numpy()
    sizes = np.array([A.n for A in batch.systems])
    for s in list(np.argsort(sizes)[:3]) + list(np.argsort(sizes)[250:252]):
        A = batch.systems[s]
        sl = slice(int(batch.sys_row[s]), int(batch.sys_row[s + 1]))
        r = oracle.pcg(A, b[sl], int(batch.bs[s]), 1e-10)
        assert np.linalg.norm(x64[sl] - r["x"]) <= 1e-10 * np.linalg.norm(r["x"]), s


def test_powerlaw_2m_fp32_values(pc):
    import torch

    A = W.powerlaw_spd(2_000_000, seed=5)
    assert A.val.dtype == np.float32
    b = W.rhs(A.n, 0)
    Ad = pc.csr(A)
    H = pc.setup(Ad, 32, prec="fp32")
    try:
        x, info = H.pcg(torch.from_numpy(b).cuda(), tol=1e-10)
        binned = H.row_binned()
    finally:
        H.destroy()
    assert info["status_name"] == "ok" and binned
    assert _true_rel_residual(A, b, x.cpu().numpy()) <= 1e-10
    # the SpMV swept in 3 column segments, as the 8M-row matrix is by default
    pc.set_col_segments(3)
    try:
        H = pc.setup(Ad, 32, prec="fp32")
        try:
            x3, info3 = H.pcg(torch.from_numpy(b).cuda(), tol=1e-10)
            nseg = H.col_segments()
        finally:
            H.destroy()
    finally:
        pc.set_col_segments("auto")
    assert info3["status_name"] == "ok" and nseg == 3
    assert abs(info3["iterations"] - info["iterations"]) <= 2
    assert _true_rel_residual(A, b, x3.cpu().numpy()) <= 1e-10

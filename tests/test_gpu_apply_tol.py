"""Refined preconditioner apply (pc_apply_tol): z = M^{-1} r from the stored (FP32, TF32 or
FP64) factors, refined against the FP64 diagonal blocks of the CSR, compared with the oracle's
FP64 block solve and with a block residual formed here from the oracle's dense blocks."""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def block_residual(D, bs, r, z):
    """r - blockdiag(D) z from the oracle's dense (zero-padded) diagonal blocks."""
    n = r.size
    out = r.copy()
    for k in range(D.shape[0]):
        a, b = k * bs, min(n, (k + 1) * bs)
        out[a:b] -= D[k, : b - a, : b - a] @ z[a:b]
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "fp64"])
@pytest.mark.parametrize("bs", [8, 16, 33])
def test_refined_apply_matches_fp64_block_solve(pc, prec, bs):
    A = W.diffusion3d(12, 2.0)          # 1728 rows: bs 33 leaves a ragged last block of 12
    r = W.rhs(A.n, 3)
    H = pc.setup(A, bs, prec=prec)
    z0 = H.apply("inv", r).cpu().numpy()
    z, steps, res = H.apply_refined(r, 1e-13)
    H.destroy()
    z = z.cpu().numpy()
    D = oracle.extract_blocks(A, bs)
    mine = np.linalg.norm(block_residual(D, bs, r, z)) / np.linalg.norm(r)
    assert res <= 1e-13 and mine <= 2e-13
    L, f = oracle.factor(A, bs)
    assert f == -1
    zo = oracle.apply(A, L, bs, oracle.MODE_INV, r)
    # forward error <= kappa(blocks) x residual (block kappa of these sigma = 2 blocks < 1e5)
    assert rel(z, zo) <= 1e-8
    if prec != "fp64":
        assert steps >= 1 and rel(z0, zo) > 1e2 * rel(z, zo)   # the FP32 apply alone is far off
    assert steps <= 20


def test_tol_zero_is_the_plain_apply_and_zero_rhs(pc):
    A = W.poisson2d(40)
    r = W.rhs(A.n, 1)
    H = pc.setup(A, 16, prec="fp32")
    z0 = H.apply("inv", r).cpu().numpy()
    z, steps, res = H.apply_refined(r, 0.0)
    assert np.array_equal(z.cpu().numpy(), z0) and steps == 0 and res == -1.0
    zs, steps, res = H.apply_refined(r, 0.0, mode="sym")       # tol 0: any mode
    assert np.array_equal(zs.cpu().numpy(), H.apply("sym", r).cpu().numpy())
    zz, steps, res = H.apply_refined(np.zeros(A.n), 1e-12)
    assert not zz.cpu().numpy().any() and steps == 0 and res == 0.0
    H.destroy()


def test_float_values_and_bad_arguments(pc):
    A = W.diffusion3d(10, 1.0)
    A32 = W.CSR(A.row_ptr, A.col, A.val.astype(np.float32))
    r = W.rhs(A.n, 2)
    H = pc.setup(A32, 8, prec="fp32")
    z, steps, res = H.apply_refined(r, 1e-12)
    D = oracle.extract_blocks(W.CSR(A.row_ptr, A.col, A32.val.astype(np.float64)), 8)
    assert res <= 1e-12
    assert np.linalg.norm(block_residual(D, 8, r, z.cpu().numpy())) <= 2e-12 * np.linalg.norm(r)
    for kw in ({"tol": -1.0}, {"tol": float("nan")}, {"tol": 1e-12, "mode": "sym"}, {"tol": 1e-12, "mode": "linv"}):
        with pytest.raises(pc.PcError) as ei:
            H.apply_refined(r, **kw)
        assert ei.value.name == "invalid_arg"
    with pytest.raises(pc.PcError) as ei:
        H.apply_refined(r, 1e-30)                                  # below the attainable residual
    assert ei.value.name == "no_convergence"
    H.destroy()

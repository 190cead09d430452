"""Input generators: sizes, structure and SPD-ness of the synthetic workloads."""
import math

import numpy as np
import pytest

from paper_2410_02408_gb300 import workloads as W


def _check_csr(A):
    assert A.row_ptr.dtype == np.int32 and A.col.dtype == np.int32
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)          # sorted, unique
        assert i in c                          # explicit diagonal


def test_poisson2d_shape():
    A = W.poisson2d(64)
    assert A.n == 4096 and A.nnz == 20224
    _check_csr(A)
    S = A.to_scipy()
    assert (S - S.T).nnz == 0


def test_diffusion3d_shape_and_symmetry():
    n = 9
    A = W.diffusion3d(n, 2.0)
    assert A.nnz == 7 * n ** 3 - 6 * n ** 2
    _check_csr(A)
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0
    D = A.to_dense()
    # weakly diagonally dominant with strict dominance from the Dirichlet faces: SPD
    assert np.linalg.eigvalsh(D)[0] > 0
    # row sums are the boundary-face coefficients only
    cx, cy, cz = W.diffusion3d_faces(n, 2.0, seed=1)
    rs = D.sum(axis=1).reshape(n, n, n)
    assert np.allclose(rs[1:-1, 1:-1, 1:-1], 0, atol=1e-12)
    assert np.isclose(rs[0, 0, 0], cx[0, 0, 0] + cy[0, 0, 0] + cz[0, 0, 0])


def test_diffusion3d_full_size_nnz():
    # the 128^3 workload: N = 2,097,152 and nnz = 14,581,760
    n = 128
    assert n ** 3 == 2097152 and 7 * n ** 3 - 6 * n ** 2 == 14581760


def test_rhs_seeded():
    assert np.array_equal(W.rhs(10, 0), np.random.default_rng(0).standard_normal(10))


def test_rgg_batch_small():
    B = W.rgg_batch(n_sys=6, seed=3, n_min=200, n_max=2000)
    assert B.n_sys == 6 and B.row_ptr[-1] == B.col.shape[0]
    for s, A in enumerate(B.systems):
        _check_csr(A)
        assert B.sys_row[s + 1] - B.sys_row[s] == A.n
        d = A.to_dense()
        assert np.allclose(d, d.T)
        assert np.allclose(d.sum(axis=1), 1e-3)              # Laplacian + 1e-3 I
        assert 6 < (A.nnz / A.n - 1) < 14                    # ~12 neighbours (fewer at the walls)
    assert set(np.unique(B.bs)) <= {4, 8, 16, 32, 64}


def test_morton_order_is_local():
    pts = np.random.default_rng(0).random((4000, 3))
    code = W.morton30(pts)
    o = np.argsort(code)
    d_sorted = np.linalg.norm(np.diff(pts[o], axis=0), axis=1).mean()
    d_rand = np.linalg.norm(np.diff(pts, axis=0), axis=1).mean()
    assert d_sorted < 0.3 * d_rand


def test_powerlaw_small():
    A = W.powerlaw_spd(n=20000, seed=5, w_max=500, cap=400)
    _check_csr(A)
    lens = np.diff(A.row_ptr)
    assert lens.max() <= 400
    assert 15 < lens.mean() < 40
    S = A.to_scipy().astype(np.float64)
    assert abs(S - S.T).max() == 0
    d = S.diagonal()
    off = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(d)
    assert np.all(d - off > 0.009)                          # strictly diagonally dominant
    assert A.val.dtype == np.float32


def test_powerlaw_exponent_gives_the_mean_degree():
    g = W._powerlaw_exponent(8, 1999, 31.0)
    w = np.arange(8, 2000, dtype=np.float64)
    p = w ** (-g)
    assert abs((w * p).sum() / p.sum() - 31.0) < 1e-6


def test_powerlaw_values_follow_the_recipe():
    """Off-diagonals in [-1, 0) as FP32; the diagonal is the FP32 rounding of the sum of the
    already-rounded off-diagonal magnitudes plus 1e-2."""
    A = W.powerlaw_spd(n=5000, seed=5, w_max=300, cap=200)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    off = rows != A.col
    assert np.all(A.val[off] < 0) and np.all(A.val[off] >= -1)
    absum = np.bincount(rows[off], weights=np.abs(A.val[off].astype(np.float64)), minlength=A.n)
    diag = A.val[~off]
    assert np.array_equal(rows[~off], np.arange(A.n))
    assert np.array_equal(diag, (absum + 1e-2).astype(np.float32))

"""Complex Hermitian positive definite systems (Sec. 3.1) on the GPU, through the real form K,
against the oracle's native complex routines (Cholesky A_k = L L^H, conjugate dot products,
Hermitian Lanczos), which share nothing with the real-form construction."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _host_real_form(A):
    """K on the host from its definition: block (i, j) = [[b, -c], [c, b]] for a_ij = b + i c."""
    n = A.n
    rows, cols, vals = [], [], []
    for i in range(n):
        for e in range(int(A.row_ptr[i]), int(A.row_ptr[i + 1])):
            j = int(A.col[e])
            b, c = A.val[e].real, A.val[e].imag
            rows += [2 * i, 2 * i, 2 * i + 1, 2 * i + 1]
            cols += [2 * j, 2 * j + 1, 2 * j, 2 * j + 1]
            vals += [b, -c, c, b]
    import scipy.sparse as sp

    K = sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))
    K.sort_indices()
    return K


def test_real_form_matches_its_definition(pc):
    A = W.hermitian_diffusion3d(6, 1.5)
    K = pc.hermitian_real_form(A)
    Kh = _host_real_form(A)
    assert np.array_equal(K.row_ptr.cpu().numpy(), Kh.indptr)
    assert np.array_equal(K.col.cpu().numpy(), Kh.indices)
    assert np.array_equal(K.val.cpu().numpy(), Kh.data)
    Kd = Kh.toarray()
    assert np.array_equal(Kd, Kd.T)
    ev = np.linalg.eigvalsh(A.to_dense())
    evk = np.linalg.eigvalsh(Kd)
    assert np.allclose(evk, np.repeat(ev, 2), rtol=1e-12, atol=1e-12)


CASES = {
    "herm_diff_12": lambda: W.hermitian_diffusion3d(12, 1.5),      # 1728 rows: ragged blocks
    "magnetic2d_64": lambda: W.magnetic_laplacian_2d(64, 1.0 / 16),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("bs", [1, 4, 8, 16, 32])
def test_pcg_z_matches_complex_oracle(pc, name, bs):
    A = CASES[name]()
    b = W.rhs_complex(A.n, 0)
    x, info = pc.pcg_z(A, b, bs, tol=1e-10)
    o = oracle.zpcg(A, b, bs, 1e-10)
    assert info["status_name"] == "ok" and o["status"] == "ok"
    assert abs(info["iterations"] - o["iterations"]) <= 1
    xr = x.cpu().numpy()
    assert np.linalg.norm(xr - o["x"]) <= 1e-10 * np.linalg.norm(o["x"])
    res = np.linalg.norm(b - oracle.zspmv(A, xr)) / np.linalg.norm(b)
    assert res <= 1e-10


def test_pcg_z_mixed_precision_reaches_true_residual(pc):
    A = W.hermitian_diffusion3d(16, 2.0)
    b = W.rhs_complex(A.n, 1)
    for prec in ("fp32", "tf32"):
        x, info = pc.pcg_z(A, b, 16, tol=1e-10, prec=prec)
        assert info["status_name"] == "ok"
        res = np.linalg.norm(b - oracle.zspmv(A, x.cpu().numpy())) / np.linalg.norm(b)
        assert res <= 1e-10


@pytest.mark.parametrize("bs", [0, 4, 16])
def test_kappa_z_matches_complex_oracle(pc, bs):
    A = W.magnetic_laplacian_2d(40, 0.07)
    v0 = W.rhs_complex(A.n, 0)
    g = pc.kappa_z(A, v0, bs, max_steps=200)
    o = oracle.zkappa(A, v0, 200, bs)
    assert g["steps"] == o["steps"]
    assert abs(g["kappa"] / o["kappa"] - 1) <= 1e-6
    assert np.allclose(g["alpha"][:20], o["alpha"][:20], rtol=1e-9)


def test_kappa_z_magnetic_path_closed_form(pc):
    n = 100
    A = W.magnetic_laplacian_1d(n, 0.4)
    g = pc.kappa_z(A, W.rhs_complex(n, 0), 0, max_steps=200)
    assert g["kappa"] == pytest.approx(1.0 / math.tan(math.pi / (2 * (n + 1))) ** 2, rel=1e-9)


def test_complex_block_size_limit_and_bad_structure(pc):
    A = W.magnetic_laplacian_2d(8, 0.1)
    b = W.rhs_complex(A.n, 0)
    with pytest.raises(pc.PcError) as ei:
        pc.pcg_z(A, b, 33)
    assert ei.value.name == "invalid_arg"
    col = A.col.copy()
    col[A.row_ptr[3]] = A.n + 1
    with pytest.raises(pc.PcError) as ei:
        pc.pcg_z(W.CSR(A.row_ptr, col, A.val), b, 8)
    assert ei.value.name == "invalid_arg"

"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product path (``paper_2410_02408_gb300``) never does, and
this package never imports the product: the two share nothing but the seeded inputs.

The arithmetic lives in ``oracle.c`` (plain sequential C, FP64); this module is argument
marshalling plus small compositions of those routines (setup = extract + factor,
kappa = Lanczos + bisection) that follow the paper's steps:

* partition into diagonal blocks and precondition each block (Sec. 3.2-3.3, generalised
  from point Jacobi to the full block: the blocks are factored A_k = L_k L_k^T),
* condition number kappa = lambda_max / lambda_min of the (preconditioned) SPD operator
  (Sec. 3.1), estimated by Lanczos,
* relative residual ||A x - b|| / ||b|| (Sec. 3.7) as the accuracy measure and CG stopping
  test.

Parity pins (tests/test_oracle.py) tie each routine to closed forms, library routines on
tiny inputs, invariants and brute force.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

STATUS = {0: "ok", 2: "not_spd", 3: "breakdown", 4: "no_convergence"}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _declare(_lib)
        _lib.or_set_threads(1)
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (1 = sequential; results are identical for
    any count).  Returns the count in effect (1 when built without OpenMP)."""
    lib().or_set_threads(int(n))
    return int(lib().or_get_threads())


def threads() -> int:
    return int(lib().or_get_threads())


_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def _declare(L):
    L.or_set_threads.restype = None
    L.or_set_threads.argtypes = [_i32]
    L.or_get_threads.restype = _i32
    L.or_get_threads.argtypes = []
    L.or_num_blocks.restype = _i64
    L.or_num_blocks.argtypes = [_i64, _i32]
    L.or_extract_blocks.restype = None
    L.or_extract_blocks.argtypes = [_i64, _p, _p, _p, _i32, _p]
    L.or_cholesky_blocks.restype = _i64
    L.or_cholesky_blocks.argtypes = [_i64, _i32, _p, _p, _dbl]
    L.or_cholesky.restype = _i32
    L.or_cholesky.argtypes = [_i32, _i32, _p, _p, _dbl]
    L.or_tri_inv_blocks.restype = None
    L.or_tri_inv_blocks.argtypes = [_i64, _i32, _p, _p]
    L.or_minv_blocks.restype = None
    L.or_minv_blocks.argtypes = [_i64, _i32, _p, _p]
    L.or_block_apply.restype = None
    L.or_block_apply.argtypes = [_i64, _i32, _p, _i32, _p, _p]
    L.or_spmv.restype = None
    L.or_spmv.argtypes = [_i64, _p, _p, _p, _p, _p]
    L.or_dot.restype = _dbl
    L.or_dot.argtypes = [_i64, _p, _p]
    L.or_sym_apply.restype = None
    L.or_sym_apply.argtypes = [_i64, _p, _p, _p, _i32, _p, _p, _p, _p, _p]
    L.or_lanczos.restype = _i32
    L.or_lanczos.argtypes = [_i64, _p, _p, _p, _i32, _p, _p, _i32, _dbl, _i32, _p, _p, _p]
    L.or_sturm_count.restype = _i32
    L.or_sturm_count.argtypes = [_i32, _p, _p, _dbl]
    L.or_tridiag_eig_k.restype = _dbl
    L.or_tridiag_eig_k.argtypes = [_i32, _p, _p, _i32]
    L.or_pcg.restype = _i32
    L.or_pcg.argtypes = [_i64, _p, _p, _p, _i32, _p, _p, _p, _dbl, _i32, _i32, _p, _p, _p]
    L.or_grad_val.restype = None
    L.or_grad_val.argtypes = [_i64, _p, _p, _p, _p, _p]
    L.or_grad_edges.restype = None
    L.or_grad_edges.argtypes = [_i64, _p, _p, _p, _p, _p]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Matrix:
    """CSR with contiguous int32 indices and float64 values (float32 values are promoted
    exactly)."""

    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def n(self):
        return self.row_ptr.shape[0] - 1


def as_matrix(A) -> Matrix:
    return Matrix(np.ascontiguousarray(A.row_ptr, dtype=np.int32),
                  np.ascontiguousarray(A.col, dtype=np.int32),
                  np.ascontiguousarray(A.val, dtype=np.float64))


def num_blocks(n: int, bs: int) -> int:
    return int(lib().or_num_blocks(n, bs))


def extract_blocks(A, bs: int) -> np.ndarray:
    """Dense diagonal blocks D_k (nblocks, bs, bs); the ragged last block is zero padded."""
    M = as_matrix(A)
    nb = num_blocks(M.n, bs)
    out = np.zeros((nb, bs, bs))
    lib().or_extract_blocks(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs, _ptr(out))
    return out


def cholesky(D: np.ndarray, tol: float = 0.0):
    """Cholesky of one dense SPD matrix; returns (L, failing pivot or -1)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    b = D.shape[0]
    L = np.zeros_like(D)
    f = lib().or_cholesky(b, b, _ptr(D), _ptr(L), tol)
    return L, int(f)


def factor(A, bs: int, tol: float = 0.0):
    """Block factors: returns (L blocks (nb, bs, bs), failing block or -1)."""
    M = as_matrix(A)
    D = extract_blocks(M, bs)
    L = np.zeros_like(D)
    f = lib().or_cholesky_blocks(M.n, bs, _ptr(D), _ptr(L), tol)
    return L, int(f)


def tri_inv(L: np.ndarray, n: int, bs: int) -> np.ndarray:
    L = np.ascontiguousarray(L)
    X = np.zeros_like(L)
    lib().or_tri_inv_blocks(n, bs, _ptr(L), _ptr(X))
    return X


def minv(Linv: np.ndarray, n: int, bs: int) -> np.ndarray:
    Linv = np.ascontiguousarray(Linv)
    M = np.zeros_like(Linv)
    lib().or_minv_blocks(n, bs, _ptr(Linv), _ptr(M))
    return M


MODE_INV, MODE_SYM, MODE_LINV, MODE_LTINV = 0, 1, 2, 3


def apply(A, L: np.ndarray, bs: int, mode: int, v: np.ndarray) -> np.ndarray:
    """mode 0: M^{-1} v; 1: L^{-1} A L^{-T} v; 2: L^{-1} v; 3: L^{-T} v."""
    M = as_matrix(A)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(M.n)
    L = np.ascontiguousarray(L)
    if mode == MODE_SYM:
        t1 = np.zeros(M.n)
        t2 = np.zeros(M.n)
        lib().or_sym_apply(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs, _ptr(L),
                           _ptr(v), _ptr(out), _ptr(t1), _ptr(t2))
    else:
        lib().or_block_apply(M.n, bs, _ptr(L), mode, _ptr(v), _ptr(out))
    return out


def spmv(A, x: np.ndarray) -> np.ndarray:
    M = as_matrix(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(M.n)
    lib().or_spmv(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), _ptr(x), _ptr(y))
    return y


def dot(x: np.ndarray, y: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().or_dot(x.shape[0], _ptr(x), _ptr(y)))


def lanczos(A, v0: np.ndarray, m: int = 200, bs: int = 0, tol: float = 1e-12,
            reorth: bool = True, L: np.ndarray | None = None):
    """Lanczos tridiagonal (alpha, beta) of A (bs == 0) or L^{-1} A L^{-T}."""
    M = as_matrix(A)
    n = M.n
    if bs > 0 and L is None:
        L, f = factor(M, bs)
        if f >= 0:
            raise ValueError(f"block {f} is not SPD")
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    alpha = np.zeros(m)
    beta = np.zeros(m)
    basis = np.zeros((m, n))
    steps = lib().or_lanczos(n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs,
                             _ptr(L) if bs > 0 else None, _ptr(v0), m, tol, int(reorth),
                             _ptr(alpha), _ptr(beta), _ptr(basis))
    return alpha[:steps].copy(), beta[:steps].copy()


def tridiag_eig(alpha: np.ndarray, beta: np.ndarray, k: int) -> float:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    if b.shape[0] < max(a.shape[0] - 1, 1):
        b = np.concatenate([b, np.zeros(max(a.shape[0] - 1, 1) - b.shape[0])])
    return float(lib().or_tridiag_eig_k(a.shape[0], _ptr(a), _ptr(b), k))


def sturm_count(alpha, beta, x: float) -> int:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    return int(lib().or_sturm_count(a.shape[0], _ptr(a), _ptr(b), x))


def kappa(A, v0: np.ndarray, m: int = 200, bs: int = 0, tol: float = 1e-12,
          reorth: bool = True):
    """Krylov estimate kappa = theta_max / theta_min of the Lanczos tridiagonal."""
    alpha, beta = lanczos(A, v0, m, bs, tol, reorth)
    k = alpha.shape[0]
    lo = tridiag_eig(alpha, beta[:k - 1], 0)
    hi = tridiag_eig(alpha, beta[:k - 1], k - 1)
    return {"kappa": hi / lo, "lambda_min": lo, "lambda_max": hi, "steps": k,
            "alpha": alpha, "beta": beta}


def pcg(A, b: np.ndarray, bs: int = 0, tol: float = 1e-10, max_iter: int = 100000,
        x0: np.ndarray | None = None, max_restarts: int = 3, L: np.ndarray | None = None,
        record: bool = False):
    """Block-Jacobi preconditioned CG; bs == 0 means unpreconditioned CG."""
    M = as_matrix(A)
    n = M.n
    if bs > 0 and L is None:
        L, f = factor(M, bs)
        if f >= 0:
            return {"status": "not_spd", "failed_block": f, "x": None}
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    out = np.zeros(4)
    al = np.zeros(max_iter) if record else None
    be = np.zeros(max_iter) if record else None
    st = lib().or_pcg(n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs,
                      _ptr(L) if bs > 0 else None, _ptr(b), _ptr(x), tol, max_iter,
                      max_restarts, _ptr(out), _ptr(al) if record else None,
                      _ptr(be) if record else None)
    res = {"status": STATUS[int(st)], "x": x, "iterations": int(out[0]),
           "rel_residual": float(out[1]), "true_rel_residual": float(out[2]),
           "restarts": int(out[3])}
    if record:
        it = int(out[0])
        res["alphas"] = al[:it].copy()
        res["betas"] = be[:max(it - 1, 0)].copy()
    return res


def grad_val(A, lam: np.ndarray, x: np.ndarray) -> np.ndarray:
    M = as_matrix(A)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.zeros(M.col.shape[0])
    lib().or_grad_val(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(lam), _ptr(x), _ptr(g))
    return g


def grad_edges(p: np.ndarray, q: np.ndarray, lam: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL/dc_e = -(lam_p - lam_q)(x_p - x_q) per edge (p, q); q < 0 marks a boundary face
    whose gradient is -lam_p x_p."""
    p = np.ascontiguousarray(p, dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.int32)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.zeros(p.shape[0])
    lib().or_grad_edges(p.shape[0], _ptr(p), _ptr(q), _ptr(lam), _ptr(x), _ptr(g))
    return g


# ---------------------------------------------------------------- complex Hermitian (Sec. 3.1)
def _zdeclare(L):
    L.zor_dotc.restype = None
    L.zor_dotc.argtypes = [_i64, _p, _p, _p]
    L.zor_spmv.restype = None
    L.zor_spmv.argtypes = [_i64, _p, _p, _p, _p, _p]
    L.zor_extract_blocks.restype = None
    L.zor_extract_blocks.argtypes = [_i64, _p, _p, _p, _i32, _p]
    L.zor_cholesky.restype = _i32
    L.zor_cholesky.argtypes = [_i32, _i32, _p, _p, _dbl]
    L.zor_cholesky_blocks.restype = _i64
    L.zor_cholesky_blocks.argtypes = [_i64, _i32, _p, _p, _dbl]
    L.zor_block_apply.restype = None
    L.zor_block_apply.argtypes = [_i64, _i32, _p, _i32, _p, _p]
    L.zor_pcg.restype = _i32
    L.zor_pcg.argtypes = [_i64, _p, _p, _p, _i32, _p, _p, _p, _dbl, _i32, _i32, _p]
    L.zor_lanczos.restype = _i32
    L.zor_lanczos.argtypes = [_i64, _p, _p, _p, _i32, _p, _p, _i32, _dbl, _i32, _p, _p, _p]


def zlib():
    L = lib()
    if not getattr(L, "_z_declared", False):
        _zdeclare(L)
        L._z_declared = True
    return L


@dataclass
class ZMatrix:
    """Complex CSR: int32 indices, complex128 values."""

    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def n(self):
        return self.row_ptr.shape[0] - 1


def as_zmatrix(A) -> ZMatrix:
    return ZMatrix(np.ascontiguousarray(A.row_ptr, dtype=np.int32), np.ascontiguousarray(A.col, dtype=np.int32),
                   np.ascontiguousarray(A.val, dtype=np.complex128))


def zdot(x, y) -> complex:
    """x^H y."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.ascontiguousarray(y, dtype=np.complex128)
    out = np.zeros(2)
    zlib().zor_dotc(x.shape[0], _ptr(x), _ptr(y), _ptr(out))
    return complex(out[0], out[1])


def zspmv(A, x):
    M = as_zmatrix(A)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.zeros(M.n, dtype=np.complex128)
    zlib().zor_spmv(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), _ptr(x), _ptr(y))
    return y


def zextract_blocks(A, bs: int):
    M = as_zmatrix(A)
    out = np.zeros((num_blocks(M.n, bs), bs, bs), dtype=np.complex128)
    zlib().zor_extract_blocks(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs, _ptr(out))
    return out


def zcholesky(D, tol: float = 0.0):
    """A = L L^H of one dense Hermitian PD matrix; returns (L, failing column or -1)."""
    D = np.ascontiguousarray(D, dtype=np.complex128)
    L = np.zeros_like(D)
    f = zlib().zor_cholesky(D.shape[0], D.shape[0], _ptr(D), _ptr(L), tol)
    return L, int(f)


def zfactor(A, bs: int, tol: float = 0.0):
    """Block factors L_k (A_kk = L_k L_k^H): (L blocks, failing block or -1)."""
    M = as_zmatrix(A)
    D = zextract_blocks(M, bs)
    L = np.zeros_like(D)
    f = zlib().zor_cholesky_blocks(M.n, bs, _ptr(D), _ptr(L), tol)
    return L, int(f)


def zapply(L, n: int, bs: int, mode: int, v):
    """mode 0: M^{-1} v = L^{-H} L^{-1} v; 2: L^{-1} v; 3: L^{-H} v."""
    L = np.ascontiguousarray(L, dtype=np.complex128)
    v = np.ascontiguousarray(v, dtype=np.complex128)
    out = np.zeros(n, dtype=np.complex128)
    zlib().zor_block_apply(n, bs, _ptr(L), mode, _ptr(v), _ptr(out))
    return out


def zpcg(A, b, bs: int = 0, tol: float = 1e-10, max_iter: int = 100000, x0=None, max_restarts: int = 3, L=None):
    """Block-Jacobi PCG for Hermitian PD A (bs == 0: unpreconditioned)."""
    M = as_zmatrix(A)
    if bs > 0 and L is None:
        L, f = zfactor(M, bs)
        if f >= 0:
            return {"status": "not_spd", "failed_block": f, "x": None}
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros(M.n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    out = np.zeros(4)
    st = zlib().zor_pcg(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs, _ptr(L) if bs > 0 else None, _ptr(b),
                        _ptr(x), tol, max_iter, max_restarts, _ptr(out))
    return {"status": STATUS[int(st)], "x": x, "iterations": int(out[0]), "rel_residual": float(out[1]),
            "true_rel_residual": float(out[2]), "restarts": int(out[3])}


def zkappa(A, v0, m: int = 200, bs: int = 0, tol: float = 1e-12, reorth: bool = True):
    """Lanczos estimate of kappa for Hermitian PD A (bs == 0) or L^{-1} A L^{-H}."""
    M = as_zmatrix(A)
    L = None
    if bs > 0:
        L, f = zfactor(M, bs)
        if f >= 0:
            raise ValueError(f"block {f} is not HPD")
    v0 = np.ascontiguousarray(v0, dtype=np.complex128)
    alpha = np.zeros(m)
    beta = np.zeros(m)
    basis = np.zeros((m, M.n), dtype=np.complex128)
    k = zlib().zor_lanczos(M.n, _ptr(M.row_ptr), _ptr(M.col), _ptr(M.val), bs, _ptr(L) if bs > 0 else None,
                           _ptr(v0), m, tol, int(reorth), _ptr(alpha), _ptr(beta), _ptr(basis))
    alpha, beta = alpha[:k].copy(), beta[:k].copy()
    lo = tridiag_eig(alpha, beta[:k - 1], 0)
    hi = tridiag_eig(alpha, beta[:k - 1], k - 1)
    return {"kappa": hi / lo, "lambda_min": lo, "lambda_max": hi, "steps": k, "alpha": alpha, "beta": beta}

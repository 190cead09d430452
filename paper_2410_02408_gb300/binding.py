"""Thin ctypes binding of libpc (include/pc.h).

Only argument marshalling happens here: torch CUDA tensors supply device pointers and
``torch.cuda.current_stream()`` supplies the stream; every step of the computation runs in
the CUDA library.  If ``libpc.so`` is missing or cannot be loaded, every entry point raises
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PC_LIB_PATH") or os.path.join(HERE, "libpc.so")

PC_OK, PC_ERR_INVALID_ARG, PC_ERR_NOT_SPD, PC_ERR_BREAKDOWN = 0, 1, 2, 3
PC_ERR_NO_CONVERGENCE, PC_ERR_TIMEOUT, PC_ERR_CUDA, PC_ERR_OOM = 4, 5, 6, 7
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "not_spd", 3: "breakdown", 4: "no_convergence",
                5: "timeout", 6: "cuda_error", 7: "oom"}
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "mixed": 1}
APPLY = {"inv": 0, "sym": 1, "linv": 2, "ltinv": 3}


class PcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        self.name = STATUS_NAMES.get(self.status, str(status))
        super().__init__(f"{what}: {self.name} ({status_string(self.status)})" if what else self.name)


class pc_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class pc_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("failed_block", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("grid_ctas", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class pc_shape(ctypes.Structure):
    _fields_ = [("spmv_ctas_per_sm", ctypes.c_int32), ("ring_stages", ctypes.c_int32), ("bin_pipe", ctypes.c_int32),
                ("fuse_update", ctypes.c_int32), ("us_per_iteration", ctypes.c_double)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    @classmethod
    def from_dict(cls, d):
        s = cls()
        s.spmv_ctas_per_sm = int(d.get("spmv_ctas_per_sm", 0))
        s.ring_stages = int(d.get("ring_stages", 0))
        s.bin_pipe = int(d.get("bin_pipe", -1))
        s.fuse_update = int(d.get("fuse_update", 0))
        s.us_per_iteration = float(d.get("us_per_iteration", 0.0))
        return s


class pc_kappa_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("kappa", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("alpha", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("elapsed_ms", ctypes.c_double)]


class pc_csr_z(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class pc_batch(ctypes.Structure):
    _fields_ = [("n_sys", ctypes.c_int32), ("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("sys_row", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("block_size", ctypes.c_void_p), ("max_block_size", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


def lib():
    """Load libpc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "pc_setup": (_I32, [ctypes.POINTER(pc_csr), _I32, _D, _I32, _P, ctypes.POINTER(_P)]),
        "pc_handle_failed_block": (_I64, [_P]),
        "pc_csr_check": (_I32, [ctypes.POINTER(pc_csr), ctypes.POINTER(ctypes.c_uint32), _P]),
        "pcg_solve_noalloc": (_I32, [ctypes.POINTER(pc_csr), _I32, _P, _P, _D, _I32, _I32,
                                     ctypes.POINTER(pc_solve_info), _P]),
        "pc_apply": (_I32, [_P, _I32, _P, _P, _P]),
        "pc_get_factor": (_I32, [_P, _I32, _P, _P]),
        "pc_destroy": (_I32, [_P]),
        "pc_extract_blocks": (_I32, [ctypes.POINTER(pc_csr), _I32, _P, _P]),
        "pc_spmv": (_I32, [ctypes.POINTER(pc_csr), _P, _P, _P]),
        "pc_dot": (_I32, [_I64, _P, _P, _P, _P]),
        "pc_debug_convert": (_I32, [_I64, _P, _P, _P, _P, _P]),
        "pc_debug_mma_tf32": (_I32, [_P, _P, _P, _P]),
        "pc_hermitian_real_form": (_I32, [ctypes.POINTER(pc_csr_z), _P, _P, _P, _P]),
        "pcg_solve_z": (_I32, [ctypes.POINTER(pc_csr_z), _I32, _P, _P, _D, _I32, _I32,
                               ctypes.POINTER(pc_solve_info), _P]),
        "kappa_estimate_z": (_I32, [ctypes.POINTER(pc_csr_z), _I32, _I32, _D, _P, _I32,
                                    ctypes.POINTER(pc_kappa_info), _P]),
        "kappa_estimate": (_I32, [ctypes.POINTER(pc_csr), _I32, _I32, _D, _P, _I32,
                                  ctypes.POINTER(pc_kappa_info), _P]),
        "kappa_estimate_h": (_I32, [_P, ctypes.POINTER(pc_csr), _I32, _D, _P, _I32,
                                    ctypes.POINTER(pc_kappa_info), _P]),
        "pcg_solve": (_I32, [ctypes.POINTER(pc_csr), _I32, _P, _P, _D, _I32, _I32,
                             ctypes.POINTER(pc_solve_info), _P]),
        "pcg_solve_h": (_I32, [_P, _P, _P, _D, _I32, ctypes.POINTER(pc_solve_info), _P]),
        "pc_grad_val": (_I32, [ctypes.POINTER(pc_csr), _P, _P, _P, _P]),
        "pc_grad_edges": (_I32, [_I64, _P, _P, _P, _P, _I64, _P, _P]),
        "pcg_solve_batched": (_I32, [ctypes.POINTER(pc_batch), _P, _P, _D, _I32, _I32, _P, _P, _P,
                                     ctypes.POINTER(pc_solve_info), _P]),
        "pc_batch_create": (_I32, [ctypes.POINTER(pc_batch), _I32, _D, _P, ctypes.POINTER(_P)]),
        "pc_batch_solve": (_I32, [_P, _P, _P, _D, _I32, _P, _P, _P, ctypes.POINTER(pc_solve_info), _P]),
        "pc_batch_destroy": (_I32, [_P]),
        "pc_batch_info": (_I32, [_P, _P, _I32]),
        "pc_batch_teams": (_I32, [_P, _P, _P]),
        "pc_batch_profile": (_I32, [_P, _P, _I32]),
        "pc_batch_schedule": (_I32, [_I32, _P, _P, _P, _I32, _I32, _D, _P, _P, _P]),
        "pc_batch_set_tuning": (None, [_I32, _I32, _D]),
        "pc_batch_set_setup_smem": (None, [_I32]),
        "pc_batch_autotune": (_I32, [ctypes.POINTER(pc_batch), _I32, _P, _D, _I32, _I32, _P, _P, _P]),
        "pc_batch_clear_tuned": (None, []),
        "pc_get_trace": (_I32, [_P, _P, _I32]),
        "pc_set_wait_budget": (None, [_I64]),
        "pc_set_ctas_per_sm": (None, [_I32]),
        "pc_set_cg_engine": (None, [_I32]),
        "pc_set_row_binning": (None, [_I32]),
        "pc_set_col_segments": (None, [_I32]),
        "pc_handle_col_segments": (_I32, [_P]),
        "pc_handle_refactored_fp64": (_I32, [_P]),
        "pc_handle_row_binned": (_I32, [_P]),
        "pc_apply_tol": (_I32, [_P, _I32, _P, _P, _D, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                _P]),
        "pc_autotune": (_I32, [ctypes.POINTER(pc_csr), _I32, _I32, _I32, _I32, _P, ctypes.POINTER(pc_shape)]),
        "pc_tune_set": (_I32, [_I32, _I32, _I64, _I64, ctypes.POINTER(pc_shape)]),
        "pc_tune_get": (_I32, [_I32, _I32, _I64, _I64, ctypes.POINTER(pc_shape)]),
        "pc_tune_clear": (None, []),
        "pc_tune_save": (_I32, [ctypes.c_char_p]),
        "pc_tune_load": (_I32, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]),
        "pc_handle_shape": (_I32, [_P, ctypes.POINTER(pc_shape)]),
        "pc_status_string": (ctypes.c_char_p, [_I32]),
        "pc_version": (_I32, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().pc_status_string(int(s)).decode()


def _torch():
    import torch

    return torch


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dev(t, dtype):
    torch = _torch()
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(t))
    if t.device.type != "cuda":
        t = t.to("cuda", non_blocking=False)
    t = t.to(dtype).contiguous()
    return t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check(status: int, what: str, allow=()):
    if status != PC_OK and status not in allow:
        raise PcError(status, what)
    return status


@dataclass
class CSR:
    """Device CSR (torch CUDA tensors) with its pc_csr descriptor."""

    row_ptr: object
    col: object
    val: object

    @property
    def n(self) -> int:
        return int(self.row_ptr.numel() - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    def desc(self) -> pc_csr:
        torch = _torch()
        return pc_csr(self.n, self.nnz, self.row_ptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr(),
                      1 if self.val.dtype == torch.float32 else 0)


def csr(row_ptr, col=None, val=None) -> CSR:
    """Device CSR from (row_ptr, col, val) arrays or from an object with those attributes.
    float32 values stay float32 (PC_F32); anything else becomes float64."""
    torch = _torch()
    if col is None:
        A = row_ptr
        row_ptr, col, val = A.row_ptr, A.col, A.val
    vdt = torch.float32 if (getattr(val, "dtype", None) in (np.float32, torch.float32)) else torch.float64
    return CSR(_dev(row_ptr, torch.int32), _dev(col, torch.int32), _dev(val, vdt))


def _as_csr(A) -> CSR:
    return A if isinstance(A, CSR) else csr(A)


class Handle:
    """A block-Jacobi preconditioner built by pc_setup (owns device factors)."""

    def __init__(self, A, block_size: int, tol: float = 0.0, prec: str = "fp64"):
        self.A = _as_csr(A)
        self.block_size = int(block_size)
        self.prec = prec
        self._d = self.A.desc()
        h = ctypes.c_void_p()
        st = lib().pc_setup(ctypes.byref(self._d), self.block_size, float(tol), PREC[prec], _stream(),
                            ctypes.byref(h))
        self._h = h
        if st != PC_OK:
            self.failed_block = int(lib().pc_handle_failed_block(h)) if h.value else -1
            self.destroy()
            raise PcError(st, f"pc_setup (failed block {self.failed_block})")
        self.failed_block = -1

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _torch().cuda.current_stream().synchronize()
            lib().pc_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def apply(self, mode: str, v, out=None):
        torch = _torch()
        v = _dev(v, torch.float64)
        out = torch.empty_like(v) if out is None else out
        _check(lib().pc_apply(self._h, APPLY[mode], _ptr(v), _ptr(out), _stream()), f"pc_apply({mode})")
        return out

    def apply_refined(self, v, tol: float, out=None, mode: str = "inv"):
        """z = M^{-1} v refined against the FP64 diagonal blocks until ||v - blockdiag(A) z|| <=
        tol ||v|| (pc_apply_tol; tol = 0 is pc_apply in any mode).  Returns (z, corrections
        made, relative block residual)."""
        torch = _torch()
        v = _dev(v, torch.float64)
        out = torch.empty_like(v) if out is None else out
        steps = ctypes.c_int32(0)
        rel = ctypes.c_double(0.0)
        _check(lib().pc_apply_tol(self._h, APPLY[mode], _ptr(v), _ptr(out), float(tol), ctypes.byref(steps),
                                  ctypes.byref(rel), _stream()), "pc_apply_tol")
        return out, int(steps.value), float(rel.value)

    def factor(self, which: str = "minv"):
        torch = _torch()
        nb = (self.A.n + self.block_size - 1) // self.block_size
        out = torch.empty((nb, self.block_size, self.block_size), dtype=torch.float64, device="cuda")
        _check(lib().pc_get_factor(self._h, 0 if which == "linv" else 1, _ptr(out), _stream()), "pc_get_factor")
        return out

    def pcg(self, b, x0=None, tol: float = 1e-10, max_iter: int = 100000, check: bool = True):
        torch = _torch()
        b = _dev(b, torch.float64)
        x = torch.zeros_like(b) if x0 is None else _dev(x0, torch.float64).clone()
        info = pc_solve_info()
        st = lib().pcg_solve_h(self._h, _ptr(b), _ptr(x), float(tol), int(max_iter), ctypes.byref(info), _stream())
        if check:
            _check(st, "pcg_solve_h")
        return x, info.to_dict()

    def kappa(self, v0, max_steps: int = 200, tol: float = 1e-12, reorth: bool = True):
        return _kappa(self._h, self.A, v0, max_steps, tol, reorth)

    def refactored_fp64(self) -> bool:
        """True if an FP32 breakdown made pc_setup factor the blocks in FP64 arithmetic."""
        return bool(lib().pc_handle_refactored_fp64(self._h))

    def row_binned(self) -> bool:
        """True if this handle's CG SpMV runs rows binned by length."""
        return bool(lib().pc_handle_row_binned(self._h))

    def col_segments(self) -> int:
        """Column segments swept by this handle's binned CG SpMV (1: whole rows)."""
        return int(lib().pc_handle_col_segments(self._h))

    def shape(self) -> dict:
        """Launch shape of this handle's loop graph (after its first graph-engine solve)."""
        out = pc_shape()
        _check(lib().pc_handle_shape(self._h, ctypes.byref(out)), "pc_handle_shape")
        return out.to_dict()

    def trace(self, max_entries: int = 4096) -> np.ndarray:
        """Barrier timestamps (ns) of the last solve when PC_TRACE_BARRIERS was set."""
        out = np.zeros(max_entries, dtype=np.int64)
        k = lib().pc_get_trace(self._h, out.ctypes.data, max_entries)
        return out[:k]


def setup(A, block_size: int, tol: float = 0.0, prec: str = "fp64") -> Handle:
    return Handle(A, block_size, tol, prec)


def _kappa(h, A, v0, max_steps, tol, reorth):
    torch = _torch()
    v0 = _dev(v0, torch.float64)
    d = A.desc()
    alpha = np.zeros(max_steps)
    beta = np.zeros(max_steps)
    info = pc_kappa_info()
    info.alpha = alpha.ctypes.data
    info.beta = beta.ctypes.data
    st = lib().kappa_estimate_h(h, ctypes.byref(d), int(max_steps), float(tol), _ptr(v0), int(bool(reorth)),
                                ctypes.byref(info), _stream())
    _check(st, "kappa_estimate")
    k = info.steps
    return {"kappa": info.kappa, "lambda_min": info.lambda_min, "lambda_max": info.lambda_max, "steps": k,
            "alpha": alpha[:k].copy(), "beta": beta[:k].copy(), "elapsed_ms": info.elapsed_ms}


def kappa(A, v0, block_size: int = 0, max_steps: int = 200, tol: float = 1e-12, reorth: bool = True):
    """Lanczos kappa estimate of A (block_size 0) or of L^{-1} A L^{-T} (FP64 factors)."""
    torch = _torch()
    A = _as_csr(A)
    v0 = _dev(v0, torch.float64)
    d = A.desc()
    alpha = np.zeros(max_steps)
    beta = np.zeros(max_steps)
    info = pc_kappa_info()
    info.alpha = alpha.ctypes.data
    info.beta = beta.ctypes.data
    st = lib().kappa_estimate(ctypes.byref(d), int(block_size), int(max_steps), float(tol), _ptr(v0),
                              int(bool(reorth)), ctypes.byref(info), _stream())
    _check(st, "kappa_estimate")
    k = info.steps
    return {"kappa": info.kappa, "lambda_min": info.lambda_min, "lambda_max": info.lambda_max, "steps": k,
            "alpha": alpha[:k].copy(), "beta": beta[:k].copy(), "elapsed_ms": info.elapsed_ms}


def pcg(A, b, block_size: int, tol: float = 1e-10, max_iter: int = 100000, prec: str = "fp64", x0=None,
        check: bool = True):
    """Block-Jacobi PCG (setup + solve in one call).  Returns (x, info dict)."""
    torch = _torch()
    A = _as_csr(A)
    b = _dev(b, torch.float64)
    x = torch.zeros_like(b) if x0 is None else _dev(x0, torch.float64).clone()
    d = A.desc()
    info = pc_solve_info()
    st = lib().pcg_solve(ctypes.byref(d), int(block_size), _ptr(b), _ptr(x), float(tol), int(max_iter),
                         PREC[prec], ctypes.byref(info), _stream())
    if check:
        _check(st, "pcg_solve")
    return x, info.to_dict()


CSR_FLAGS = {1: "row_ptr", 2: "column_range", 4: "column_order", 8: "missing_diagonal"}


def csr_check(A):
    """The library's O(nnz) CSR structure check: (status, set of violated rules)."""
    A = _as_csr(A)
    d = A.desc()
    flags = ctypes.c_uint32(0)
    st = int(lib().pc_csr_check(ctypes.byref(d), ctypes.byref(flags), _stream()))
    return st, {name for bit, name in CSR_FLAGS.items() if flags.value & bit}


def spmv(A, x, out=None):
    torch = _torch()
    A = _as_csr(A)
    x = _dev(x, torch.float64)
    out = torch.empty_like(x) if out is None else out
    d = A.desc()
    _check(lib().pc_spmv(ctypes.byref(d), _ptr(x), _ptr(out), _stream()), "pc_spmv")
    return out


def debug_convert(d, f):
    """The library's integer-pipe conversions: (float32 of the float64 tensor d, float64 of the
    float32 tensor f), element by element (pc_debug_convert)."""
    torch = _torch()
    d = _dev(d, torch.float64)
    f = _dev(f, torch.float32)
    out_f = torch.empty(d.shape[0], dtype=torch.float32, device="cuda")
    out_d = torch.empty(f.shape[0], dtype=torch.float64, device="cuda")
    if d.shape[0] != f.shape[0]:
        raise ValueError("d and f must have the same length")
    _check(lib().pc_debug_convert(d.shape[0], _ptr(d), _ptr(out_f), _ptr(f), _ptr(out_d), _stream()),
           "pc_debug_convert")
    return out_f, out_d


def debug_mma_tf32(a, b):
    """One tensor-core product d = a b (a 16x8, b 8x8, FP32 in, TF32 operands, FP32 accumulate),
    as the TF32 setup issues it (pc_debug_mma_tf32)."""
    torch = _torch()
    a = _dev(a, torch.float32)
    b = _dev(b, torch.float32)
    if tuple(a.shape) != (16, 8) or tuple(b.shape) != (8, 8):
        raise ValueError("a must be 16x8 and b 8x8")
    d = torch.empty((16, 8), dtype=torch.float32, device="cuda")
    _check(lib().pc_debug_mma_tf32(_ptr(a), _ptr(b), _ptr(d), _stream()), "pc_debug_mma_tf32")
    return d


@dataclass
class CSRZ:
    """Device complex CSR (torch CUDA tensors; values complex128) with its pc_csr_z descriptor."""

    row_ptr: object
    col: object
    val: object

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def desc(self) -> pc_csr_z:
        return pc_csr_z(self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val))


def csr_z(A) -> CSRZ:
    """Complex CSR on the device from a host CSR whose values are complex."""
    if isinstance(A, CSRZ):
        return A
    torch = _torch()
    return CSRZ(_dev(np.asarray(A.row_ptr, dtype=np.int32), torch.int32),
                _dev(np.asarray(A.col, dtype=np.int32), torch.int32),
                _dev(np.asarray(A.val, dtype=np.complex128), torch.complex128))


def _zvec(v):
    torch = _torch()
    return _dev(v, torch.complex128)


def hermitian_real_form(A):
    """The real form K of a complex Hermitian CSR (pc_hermitian_real_form): a device CSR."""
    torch = _torch()
    Z = csr_z(A)
    rp = torch.empty(2 * Z.n + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(max(4 * Z.nnz, 1), dtype=torch.int32, device="cuda")
    va = torch.empty(max(4 * Z.nnz, 1), dtype=torch.float64, device="cuda")
    d = Z.desc()
    _check(lib().pc_hermitian_real_form(ctypes.byref(d), _ptr(rp), _ptr(ci), _ptr(va), _stream()),
           "pc_hermitian_real_form")
    return CSR(rp, ci[:4 * Z.nnz], va[:4 * Z.nnz])


def pcg_z(A, b, block_size: int, tol: float = 1e-10, max_iter: int = 100000, prec: str = "fp64", x0=None,
          check: bool = True):
    """Block-Jacobi PCG for a complex Hermitian PD system (pcg_solve_z).  Returns (x complex, info)."""
    Z = csr_z(A)
    b = _zvec(b)
    x = _torch().zeros_like(b) if x0 is None else _zvec(x0).clone()
    info = pc_solve_info()
    d = Z.desc()
    st = lib().pcg_solve_z(ctypes.byref(d), int(block_size), _ptr(b), _ptr(x), float(tol), int(max_iter),
                           PREC[prec], ctypes.byref(info), _stream())
    if check:
        _check(st, "pcg_solve_z")
    return x, info.to_dict()


def kappa_z(A, v0, block_size: int = 0, max_steps: int = 200, tol: float = 1e-12, reorth: bool = True):
    """Lanczos kappa of a complex Hermitian PD matrix (kappa_estimate_z)."""
    Z = csr_z(A)
    v0 = _zvec(v0)
    alpha = np.zeros(max_steps)
    beta = np.zeros(max_steps)
    info = pc_kappa_info()
    info.alpha = alpha.ctypes.data
    info.beta = beta.ctypes.data
    d = Z.desc()
    st = lib().kappa_estimate_z(ctypes.byref(d), int(block_size), int(max_steps), float(tol), _ptr(v0),
                                int(bool(reorth)), ctypes.byref(info), _stream())
    _check(st, "kappa_estimate_z")
    k = info.steps
    return {"kappa": info.kappa, "lambda_min": info.lambda_min, "lambda_max": info.lambda_max, "steps": k,
            "alpha": alpha[:k].copy(), "beta": beta[:k].copy(), "ms": info.elapsed_ms}


def dot(x, y) -> float:
    torch = _torch()
    x = _dev(x, torch.float64)
    y = _dev(y, torch.float64)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(lib().pc_dot(int(x.numel()), _ptr(x), _ptr(y), _ptr(out), _stream()), "pc_dot")
    return float(out.item())


def extract_blocks(A, block_size: int):
    torch = _torch()
    A = _as_csr(A)
    nb = (A.n + block_size - 1) // block_size
    out = torch.empty((nb, block_size, block_size), dtype=torch.float64, device="cuda")
    d = A.desc()
    _check(lib().pc_extract_blocks(ctypes.byref(d), int(block_size), _ptr(out), _stream()), "pc_extract_blocks")
    return out


def grad_val(A, lam, x):
    torch = _torch()
    A = _as_csr(A)
    lam = _dev(lam, torch.float64)
    x = _dev(x, torch.float64)
    out = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    d = A.desc()
    _check(lib().pc_grad_val(ctypes.byref(d), _ptr(lam), _ptr(x), _ptr(out), _stream()), "pc_grad_val")
    return out


def grad_edges(p, q, lam, x):
    """dL/dc_e = -(lam_p - lam_q)(x_p - x_q) for every edge (p, q); q < 0 marks a boundary
    face (-lam_p x_p).  p, q: int32 index tensors; lam, x: FP64 vectors."""
    torch = _torch()
    p = _dev(p, torch.int32)
    q = _dev(q, torch.int32)
    lam = _dev(lam, torch.float64)
    x = _dev(x, torch.float64)
    out = torch.empty(p.numel(), dtype=torch.float64, device="cuda")
    _check(lib().pc_grad_edges(int(p.numel()), _ptr(p), _ptr(q), _ptr(lam), _ptr(x), int(x.numel()), _ptr(out),
                               _stream()), "pc_grad_edges")
    return out


class Batch:
    """A batch of independent SPD systems on the device (concatenated CSR, local columns)
    with its pc_batch_create handle.  ``host`` is any object with row_ptr, col, val,
    sys_row and bs arrays (``workloads.Batch``)."""

    def __init__(self, host, prec: str = "fp64", pivot_tol: float = 0.0):
        torch = _torch()
        self.n_sys = int(len(host.bs))
        self.sys_row = _dev(host.sys_row, torch.int64)
        self.row_ptr = _dev(host.row_ptr, torch.int32)
        self.col = _dev(host.col, torch.int32)
        self.val = _dev(host.val, torch.float64)
        self.bs = _dev(host.bs, torch.int32)
        self.n_rows = int(self.row_ptr.numel() - 1)
        self.prec = prec
        self._d = pc_batch(self.n_sys, self.n_rows, int(self.col.numel()), self.sys_row.data_ptr(),
                           self.row_ptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr(), self.bs.data_ptr(),
                           int(np.max(np.asarray(host.bs))) if self.n_sys else 1)
        h = ctypes.c_void_p()
        _check(lib().pc_batch_create(ctypes.byref(self._d), PREC[prec], float(pivot_tol), _stream(), ctypes.byref(h)),
               "pc_batch_create")
        self._h = h

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _torch().cuda.current_stream().synchronize()
            lib().pc_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def solve(self, b, tol: float = 1e-10, max_iter: int = 100000, x=None, check: bool = True):
        """Setup + PCG of every system in one launch.  Returns (x, per-system dict, info)."""
        torch = _torch()
        b = _dev(b, torch.float64)
        x = torch.empty_like(b) if x is None else x
        iters = torch.empty(self.n_sys, dtype=torch.int32, device="cuda")
        status = torch.empty(self.n_sys, dtype=torch.int32, device="cuda")
        relres = torch.empty(self.n_sys, dtype=torch.float64, device="cuda")
        info = pc_solve_info()
        st = lib().pc_batch_solve(self._h, _ptr(b), _ptr(x), float(tol), int(max_iter), _ptr(iters), _ptr(status),
                                  _ptr(relres), ctypes.byref(info), _stream())
        if check:
            _check(st, "pc_batch_solve")
        per = {"iterations": iters.cpu().numpy(), "status": status.cpu().numpy(), "relres": relres.cpu().numpy()}
        d = info.to_dict()
        d["graph"] = bool(info.reserved)
        return x, per, d

    def launch_info(self) -> dict:
        out = (ctypes.c_int32 * 8)()
        k = lib().pc_batch_info(self._h, ctypes.cast(out, ctypes.c_void_p), 8)
        keys = ("grid", "ctas_per_sm", "slots", "team_max", "smem", "setup_warps", "graph")
        return {keys[i]: int(out[i]) for i in range(min(k, len(keys)))}

    def phase_profile(self) -> dict:
        """Per-phase nanoseconds summed over CTAs (handles created with PC_BATCH_PROFILE=1)."""
        out = np.zeros(8, dtype=np.uint64)
        k = lib().pc_batch_profile(self._h, out.ctypes.data, 8)
        names = ("setup", "start", "spmv", "units", "p_update", "true_residual", "sync", "idle")
        return {names[i]: int(out[i]) for i in range(k)}

    def teams(self):
        team = np.zeros(self.n_sys, dtype=np.int32)
        slot0 = np.zeros(self.n_sys, dtype=np.int32)
        lib().pc_batch_teams(self._h, team.ctypes.data, slot0.ctypes.data)
        return team, slot0


def batch_autotune(host, b, tol: float = 1e-10, max_iter: int = 100000, prec: str = "fp64", max_trials: int = 0):
    """Time candidate launch shapes of the batched solve on this batch and keep the fastest
    for later batches of the same signature.  Returns (best_ms, config dict)."""
    torch = _torch()
    B = Batch.__new__(Batch)
    B.sys_row = _dev(host.sys_row, torch.int64)
    B.row_ptr = _dev(host.row_ptr, torch.int32)
    B.col = _dev(host.col, torch.int32)
    B.val = _dev(host.val, torch.float64)
    B.bs = _dev(host.bs, torch.int32)
    n_sys = int(len(host.bs))
    d = pc_batch(n_sys, int(B.row_ptr.numel() - 1), int(B.col.numel()), B.sys_row.data_ptr(), B.row_ptr.data_ptr(),
                 B.col.data_ptr(), B.val.data_ptr(), B.bs.data_ptr(), int(np.max(np.asarray(host.bs))))
    b = _dev(b, torch.float64)
    ms = ctypes.c_double(0.0)
    cfg = (ctypes.c_int32 * 4)()
    _check(lib().pc_batch_autotune(ctypes.byref(d), PREC[prec], _ptr(b), float(tol), int(max_iter), int(max_trials),
                                   _stream(), ctypes.byref(ms), ctypes.cast(cfg, ctypes.c_void_p)), "pc_batch_autotune")
    return ms.value, {"ctas_per_sm": int(cfg[0]), "team_max": int(cfg[1]), "slots_per_cta": cfg[2] / 1000.0,
                      "setup_kb": int(cfg[3])}


def pcg_batched(host, b, tol: float = 1e-10, max_iter: int = 100000, prec: str = "fp64", check: bool = True):
    """One-shot batched solve (create + solve + destroy).  Returns (x, per-system dict, info)."""
    B = Batch(host, prec)
    try:
        return B.solve(b, tol, max_iter, check=check)
    finally:
        B.destroy()


def batch_schedule(n_rows, nnz, block_size, n_ctas: int, team_max: int = 32, slots_per_cta: float = 2.0):
    """The library's team scheduler (host only).  Returns (team, slot0, order, n_slots)."""
    n_rows = np.ascontiguousarray(n_rows, dtype=np.int64)
    nnz = np.ascontiguousarray(nnz, dtype=np.int64)
    block_size = np.ascontiguousarray(block_size, dtype=np.int32)
    k = n_rows.shape[0]
    team = np.zeros(k, dtype=np.int32)
    slot0 = np.zeros(k, dtype=np.int32)
    order = np.zeros(k, dtype=np.int32)
    n = lib().pc_batch_schedule(k, n_rows.ctypes.data, nnz.ctypes.data, block_size.ctypes.data, int(n_ctas),
                                int(team_max), float(slots_per_cta), team.ctypes.data, slot0.ctypes.data,
                                order.ctypes.data)
    if n < 0:
        raise PcError(PC_ERR_INVALID_ARG, "pc_batch_schedule")
    return team, slot0, order, n


def batch_set_tuning(ctas_per_sm: int = 0, team_max: int = 0, slots_per_cta: float = 0.0):
    lib().pc_batch_set_tuning(int(ctas_per_sm), int(team_max), float(slots_per_cta))


def set_wait_budget(cycles: int):
    lib().pc_set_wait_budget(int(cycles))


def set_ctas_per_sm(ctas: int):
    lib().pc_set_ctas_per_sm(int(ctas))


def set_row_binning(mode: str):
    """"auto" (default), "off" or "on": row order of the CG SpMV (see pc_set_row_binning)."""
    lib().pc_set_row_binning({"off": 0, "on": 1}.get(mode, -1))


def autotune(A, block_size: int, prec: str = "fp32", iterations: int = 100, max_trials: int = 0) -> dict:
    """Kernel-shape autotuner of the single-system solve (pc_autotune): times the candidate
    launch shapes on `iterations` CG iterations of A and records the fastest for A's key.
    Returns that shape as a dict."""
    A = _as_csr(A)
    d = A.desc()
    out = pc_shape()
    _check(lib().pc_autotune(ctypes.byref(d), int(block_size), PREC[prec], int(iterations), int(max_trials),
                             _stream(), ctypes.byref(out)), "pc_autotune")
    return out.to_dict()


def tune_set(block_size: int, prec: str, n: int, nnz: int, shape: dict):
    """Records a launch shape for the key of an n-row, nnz-entry system (pc_tune_set)."""
    _check(lib().pc_tune_set(int(block_size), PREC[prec], int(n), int(nnz), ctypes.byref(pc_shape.from_dict(shape))),
           "pc_tune_set")


def tune_get(block_size: int, prec: str, n: int, nnz: int):
    """The recorded launch shape for that key as a dict, or None (pc_tune_get)."""
    out = pc_shape()
    return out.to_dict() if lib().pc_tune_get(int(block_size), PREC[prec], int(n), int(nnz), ctypes.byref(out)) else None


def tune_clear():
    lib().pc_tune_clear()


def tune_save(path: str):
    _check(lib().pc_tune_save(os.fsencode(path)), "pc_tune_save")


def tune_load(path: str) -> int:
    """Merges a cache file into the table; returns the entries taken (pc_tune_load)."""
    n = ctypes.c_int32(0)
    _check(lib().pc_tune_load(os.fsencode(path), ctypes.byref(n)), "pc_tune_load")
    return int(n.value)


def set_col_segments(segs):
    """"auto" (the library default: whole rows) or 1..8: column segments of the binned CG SpMV
    (see pc_set_col_segments)."""
    lib().pc_set_col_segments(-1 if segs in (None, "auto") else int(segs))


def set_cg_engine(engine: str):
    """"graph" (default): CUDA-graph loop over three kernels; "persistent": one cooperative kernel."""
    lib().pc_set_cg_engine({"graph": 0, "persistent": 1}.get(engine, -1))

"""GB300-native block-Jacobi preconditioning, Lanczos condition-number estimation and
preconditioned CG for sparse SPD systems (the classical GPU stage of arXiv 2410.02408).

The compute path is the CUDA library ``libpc.so`` (C-ABI, ``include/pc.h``); the Python
layer in ``binding`` only marshals torch device tensors and the current stream into it.
"""
import importlib

from . import workloads  # noqa: F401  (input generators; no method arithmetic)

_BINDING_NAMES = ("setup", "apply", "kappa", "pcg", "spmv", "dot", "extract_blocks", "Handle", "csr", "CSR",
                  "csr_check", "debug_convert", "debug_mma_tf32", "csr_z", "CSRZ", "pcg_z", "kappa_z",
                  "hermitian_real_form", "pcg_batched", "Batch", "batch_schedule", "batch_set_tuning", "batch_autotune",
                  "grad_val", "grad_edges", "status_string", "PcError", "set_wait_budget", "set_ctas_per_sm",
                  "set_cg_engine", "set_row_binning", "set_col_segments", "autotune", "tune_set", "tune_get",
                  "tune_clear", "tune_save", "tune_load")


def load():
    """Load the CUDA library; raises if it was not built."""
    return importlib.import_module(".binding", __name__).lib()


def __getattr__(name):
    if name in _BINDING_NAMES:
        return getattr(importlib.import_module(".binding", __name__), name)
    if name == "PcgSolve":
        return importlib.import_module(".autograd", __name__).PcgSolve
    raise AttributeError(name)

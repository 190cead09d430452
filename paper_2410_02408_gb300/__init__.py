"""GB300-native block-Jacobi preconditioning, Lanczos condition-number estimation and
preconditioned CG for sparse SPD systems (the classical GPU stage of arXiv 2410.02408).

The compute path is the CUDA library ``libpc.so`` (C-ABI, ``include/pc.h``); the Python
layer in ``binding`` only marshals torch device tensors and the current stream into it.
"""
from . import workloads  # noqa: F401  (input generators; no method arithmetic)


def load():
    """Load the CUDA library; raises if it was not built."""
    from . import binding

    return binding.lib()


def __getattr__(name):
    if name in ("setup", "apply", "kappa", "pcg", "spmv", "dot", "extract_blocks",
                "Handle", "PcgSolve", "pcg_batched", "BatchHandle", "grad_val", "binding",
                "setup_batched", "status_string", "PcError"):
        from . import binding

        return getattr(binding, name) if name != "binding" else binding
    raise AttributeError(name)

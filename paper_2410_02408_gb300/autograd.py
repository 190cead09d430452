"""Hand-written adjoint of the block-Jacobi preconditioned solve behind torch.autograd.

For x = A^{-1} b with A symmetric positive definite and a loss L(x):

    A^T lambda = dL/dx            (A = A^T: the same operator, the same preconditioner)
    dL/db      = lambda
    dL/dA_ij   = -lambda_i x_j    for every stored entry (i, j) of the sparsity pattern

so the backward pass is one more preconditioned CG solve plus one pass over the pattern.
Only x is kept between the passes (no Krylov history); the block-Jacobi factors built for
the forward solve are reused by the backward solve and released after it.

Edge-coefficient gradients of Laplacian-type matrices follow from the same lambda and x:
``binding.grad_edges`` evaluates dL/dc_e = -(lambda_p - lambda_q)(x_p - x_q) directly, and
assembling the CSR values from c with differentiable torch operations lets autograd chain
``dL/dA_ij`` back to c as well.
"""
import torch

from . import binding as B


class PcgSolve(torch.autograd.Function):
    """x = PcgSolve.apply(val, b, pattern, block_size=16, tol=1e-10, max_iter=100000,
    prec="fp64", bwd_tol=None)

    val      stored entries of A on the CUDA device (float64, or float32 for PC_F32
             values), in the order of ``pattern``'s CSR; differentiable.
    b        right-hand side (float64 CUDA vector); differentiable.
    pattern  the sparsity pattern: a ``binding.CSR`` (its values are ignored) or any object
             with ``row_ptr`` and ``col``.
    prec     factor precision of the preconditioner: "fp64", "fp32" or "tf32".
    bwd_tol  relative-residual tolerance of the adjoint solve (defaults to ``tol``).

    Raises ``binding.PcError`` if either solve fails to converge.
    """

    @staticmethod
    def forward(ctx, val, b, pattern, block_size=16, tol=1e-10, max_iter=100000, prec="fp64", bwd_tol=None):
        P = pattern if isinstance(pattern, B.CSR) else B.csr(pattern.row_ptr, pattern.col, val.detach())
        A = B.CSR(P.row_ptr, P.col, val.detach().contiguous())
        if A.nnz != val.numel():
            raise ValueError("val does not match the pattern's number of stored entries")
        h = B.Handle(A, block_size, 0.0, prec)
        try:
            x, info = h.pcg(b.detach(), tol=tol, max_iter=max_iter)
        except Exception:
            h.destroy()
            raise
        ctx.h = h
        ctx.A = A
        ctx.tol = tol if bwd_tol is None else bwd_tol
        ctx.max_iter = max_iter
        ctx.val_dtype = val.dtype
        ctx.forward_info = info
        ctx.save_for_backward(x)
        if not any(ctx.needs_input_grad[:2]):
            h.destroy()
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        try:
            lam, info = ctx.h.pcg(gx.detach().to(torch.float64).contiguous(), tol=ctx.tol, max_iter=ctx.max_iter)
        finally:
            ctx.h.destroy()
        ctx.backward_info = info
        gval = B.grad_val(ctx.A, lam, x).to(ctx.val_dtype) if ctx.needs_input_grad[0] else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gval, gb, None, None, None, None, None, None


def pcg_solve(val, b, pattern, block_size=16, tol=1e-10, max_iter=100000, prec="fp64", bwd_tol=None):
    """Functional form of ``PcgSolve.apply``."""
    return PcgSolve.apply(val, b, pattern, block_size, tol, max_iter, prec, bwd_tol)

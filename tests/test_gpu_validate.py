"""The O(nnz) CSR structure check that runs before any kernel reads a matrix through its
indices: host-built bad matrices are rejected with PC_ERR_INVALID_ARG (and the rule they
break is reported) by every entry point that takes a CSR, and a valid setup right after
succeeds.  Each bad matrix keeps row_ptr at n + 1 entries and col/val at nnz entries, so the
check itself only reads inside the arrays it is given."""
import numpy as np
import pytest

from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _base():
    return W.poisson2d(12)   # 144 rows, 5-point stencil, sorted columns, diagonal stored


def _bad_matrices():
    A = _base()
    out = {}
    col = A.col.copy()
    col[A.row_ptr[7] + 1] = A.n + 3                       # a column past the last one
    out["column_range"] = W.CSR(A.row_ptr, col, A.val)
    col = A.col.copy()
    col[A.row_ptr[20]] = -1                                # a negative column
    out["column_range_negative"] = W.CSR(A.row_ptr, col, A.val)
    # drop the diagonal of row 30 (replace it by a duplicate of its left neighbour's column)
    col = A.col.copy()
    s, e = int(A.row_ptr[30]), int(A.row_ptr[31])
    k = s + int(np.nonzero(col[s:e] == 30)[0][0])
    col[k] = col[k - 1]
    out["missing_diagonal_duplicate"] = W.CSR(A.row_ptr, col, A.val)
    col = A.col.copy()
    s = int(A.row_ptr[50])
    col[s], col[s + 1] = col[s + 1], col[s]               # two columns swapped
    out["column_order"] = W.CSR(A.row_ptr, col, A.val)
    rp = A.row_ptr.copy()
    rp[40] = rp[41] + 1                                    # a decreasing row pointer
    out["row_ptr_decreasing"] = W.CSR(rp, A.col, A.val)
    rp = A.row_ptr.copy()
    rp[-1] = rp[-1] - 1                                    # row_ptr[n] != nnz
    out["row_ptr_end"] = W.CSR(rp, A.col, A.val)
    rp = A.row_ptr.copy()
    rp[0] = 1                                              # row_ptr[0] != 0
    out["row_ptr_start"] = W.CSR(rp, A.col, A.val)
    # a row without its diagonal: drop the diagonal entry of row 0 altogether
    keep = np.ones(A.nnz, dtype=bool)
    keep[int(A.row_ptr[0]) + int(np.nonzero(A.col[A.row_ptr[0]:A.row_ptr[1]] == 0)[0][0])] = False
    rp = A.row_ptr.copy()
    rp[1:] -= 1
    out["missing_diagonal"] = W.CSR(rp, A.col[keep], A.val[keep])
    return out


EXPECT = {
    "column_range": "column_range",
    "column_range_negative": "column_range",
    "missing_diagonal_duplicate": "missing_diagonal",
    "column_order": "column_order",
    "row_ptr_decreasing": "row_ptr",
    "row_ptr_end": "row_ptr",
    "row_ptr_start": "row_ptr",
    "missing_diagonal": "missing_diagonal",
}


def test_valid_matrices_pass(pc):
    for A in (_base(), W.diffusion3d(9, 2.0), W.powerlaw_spd(3000, seed=2, device="cpu")):
        st, bad = pc.csr_check(A)
        assert st == 0 and not bad


@pytest.mark.parametrize("case", sorted(EXPECT))
def test_bad_csr_is_rejected_everywhere(pc, case):
    import torch

    from paper_2410_02408_gb300 import binding as B

    A = _bad_matrices()[case]
    st, bad = pc.csr_check(A)
    assert st == B.PC_ERR_INVALID_ARG
    assert EXPECT[case] in bad, bad
    b = torch.from_numpy(W.rhs(A.n, 0)).cuda()
    for call in (lambda: pc.setup(A, 8),
                 lambda: pc.pcg(A, b, 8),
                 lambda: pc.kappa(A, b, 0, max_steps=10),
                 lambda: pc.kappa(A, b, 8, max_steps=10),
                 lambda: pc.spmv(A, b),
                 lambda: pc.extract_blocks(A, 8),
                 lambda: pc.grad_val(A, b, b)):
        with pytest.raises(pc.PcError) as ei:
            call()
        assert ei.value.name == "invalid_arg", case
    # the library is still usable: a valid matrix right after sets up and solves
    G = _base()
    x, info = pc.pcg(G, torch.from_numpy(W.rhs(G.n, 0)).cuda(), 8)
    assert info["status_name"] == "ok"


def test_batched_rejects_unsorted_columns_and_missing_diagonal(pc):
    systems = [W.poisson2d(10), W.poisson2d(12)]
    for mutate in ("order", "diag"):
        S = [W.CSR(A.row_ptr.copy(), A.col.copy(), A.val.copy()) for A in systems]
        A = S[1]
        s = int(A.row_ptr[5])
        if mutate == "order":
            A.col[s], A.col[s + 1] = A.col[s + 1], A.col[s]
        else:
            e = int(A.row_ptr[6])
            k = s + int(np.nonzero(A.col[s:e] == 5)[0][0])
            A.col[k] = A.col[k - 1]
        batch = W.concat_batch(S, [4, 8])
        b = W.rhs(int(batch.sys_row[-1]), 0)
        with pytest.raises(pc.PcError) as ei:
            pc.pcg_batched(batch, b)
        assert ei.value.name == "invalid_arg"

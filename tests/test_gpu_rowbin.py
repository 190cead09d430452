"""Row binning of the CG SpMV (rows sorted by length inside windows): chosen automatically
for power-law rows and not for stencils, and the solve matches the oracle either way."""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def powerlaw():
    return W.powerlaw_spd(n=30000, seed=5, w_max=1999, cap=2000)


def _solve(pc, A, bs, mode, prec="fp64", segs="auto", want_segs=False):
    import torch

    pc.set_row_binning(mode)
    pc.set_col_segments(segs)
    try:
        H = pc.setup(pc.csr(A), bs, prec=prec)
        b = torch.from_numpy(W.rhs(A.n, 0)).cuda()
        x, info = H.pcg(b, tol=1e-10)
        binned = H.row_binned()
        nseg = H.col_segments()
        H.destroy()
    finally:
        pc.set_row_binning("auto")
        pc.set_col_segments("auto")
    if want_segs:
        return x.cpu().numpy(), info, binned, nseg
    return x.cpu().numpy(), info, binned


def test_auto_bins_power_law_rows_only(pc, powerlaw):
    _, _, binned = _solve(pc, powerlaw, 32, "auto")
    assert binned
    _, _, binned = _solve(pc, W.diffusion3d(16, 2.0), 16, "auto")
    assert not binned


@pytest.mark.parametrize("mode", ["on", "off"])
def test_binned_and_natural_order_match_oracle(pc, powerlaw, mode):
    A = powerlaw
    x, info, binned = _solve(pc, A, 32, mode)
    assert binned == (mode == "on")
    r = oracle.pcg(A, W.rhs(A.n, 0), 32, 1e-10)
    assert info["status_name"] == "ok" and r["status"] == "ok"
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])
    assert abs(info["iterations"] - r["iterations"]) <= 1


def test_forced_binning_on_a_stencil_matches_oracle(pc):
    A = W.diffusion3d(24, 2.0)       # 13,824 rows: several windows and a ragged last one
    x, info, binned = _solve(pc, A, 8, "on")
    assert binned
    r = oracle.pcg(A, W.rhs(A.n, 0), 8, 1e-10)
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])


def test_binned_solve_is_deterministic(pc, powerlaw):
    x1, _, _ = _solve(pc, powerlaw, 32, "on", "fp32")
    x2, _, _ = _solve(pc, powerlaw, 32, "on", "fp32")
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("segs", [2, 3, 8])
def test_column_segments_match_oracle(pc, powerlaw, segs):
    """The binned SpMV swept once per column segment (partial sums carried between sweeps)
    solves to the oracle's answer; 30,000 rows in 8 segments leaves segments of 3,750 columns,
    so most rows have entries in several of them, and some segments of a row are empty."""
    A = powerlaw
    x, info, binned, nseg = _solve(pc, A, 32, "on", segs=segs, want_segs=True)
    assert binned and nseg == segs
    r = oracle.pcg(A, W.rhs(A.n, 0), 32, 1e-10)
    assert info["status_name"] == "ok"
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])
    assert abs(info["iterations"] - r["iterations"]) <= 1


def test_column_segments_on_a_stencil(pc):
    A = W.diffusion3d(24, 2.0)       # ragged last window; 4 segments of 3,456 columns
    x, info, binned, nseg = _solve(pc, A, 8, "on", segs=4, want_segs=True)
    assert binned and nseg == 4
    r = oracle.pcg(A, W.rhs(A.n, 0), 8, 1e-10)
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])


def test_column_segments_are_deterministic(pc, powerlaw):
    x1, _, _ = _solve(pc, powerlaw, 32, "on", "fp32", segs=3)
    x2, _, _ = _solve(pc, powerlaw, 32, "on", "fp32", segs=3)
    assert np.array_equal(x1, x2)


def test_default_is_whole_rows(pc, powerlaw):
    _, _, binned, nseg = _solve(pc, powerlaw, 32, "auto", want_segs=True)
    assert binned and nseg == 1


def test_unsorted_columns_are_rejected(pc, powerlaw):
    """Rows stored with their columns in decreasing order break the CSR convention (columns
    strictly increasing within a row); the structure check at setup rejects them before any
    kernel reads the matrix, and the same rows stored in increasing order solve."""
    A = powerlaw
    col = A.col.copy()
    val = A.val.copy()
    for i in range(A.n):
        s, e = int(A.row_ptr[i]), int(A.row_ptr[i + 1])
        col[s:e] = col[s:e][::-1]
        val[s:e] = val[s:e][::-1]
    Ar = W.CSR(A.row_ptr, col, val)
    st, bad = pc.csr_check(Ar)
    assert st == 1 and bad == {"column_order"}
    with pytest.raises(pc.PcError) as ei:
        pc.setup(Ar, 32, prec="fp32")
    assert ei.value.name == "invalid_arg"
    x, info, binned, nseg = _solve(pc, A, 32, "on", segs=3, want_segs=True)
    assert binned and nseg == 3
    r = oracle.pcg(A, W.rhs(A.n, 0), 32, 1e-10)
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])


@pytest.mark.parametrize("loop", ["sliced", "pipe", "plain"])
@pytest.mark.parametrize("segs", [1, 3])
def test_both_row_loops_match_oracle(pc, powerlaw, segs, loop, monkeypatch):
    """Every binned row loop gives the oracle's answer, whole-row and in column segments: the
    pipelined one (next round's column indices loaded during the gathers, 2 CTAs per SM), the
    same with the one-lane-per-row groups read from the sliced copy (the default; with
    segments it runs as the pipelined one) and the plain one (4 CTAs per SM), each with its own
    balanced split."""
    monkeypatch.setenv("PC_BIN_SPMV", loop)
    A = powerlaw
    x, info, binned, nseg = _solve(pc, A, 32, "on", segs=segs, want_segs=True)
    assert binned and nseg == segs
    r = oracle.pcg(A, W.rhs(A.n, 0), 32, 1e-10)
    assert info["status_name"] == "ok"
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])
    assert abs(info["iterations"] - r["iterations"]) <= 1


@pytest.mark.parametrize("loop", ["sliced", "pipe", "plain"])
def test_both_row_loops_on_a_stencil(pc, loop, monkeypatch):
    monkeypatch.setenv("PC_BIN_SPMV", loop)
    A = W.diffusion3d(24, 2.0)
    x, info, binned = _solve(pc, A, 8, "on")
    assert binned
    r = oracle.pcg(A, W.rhs(A.n, 0), 8, 1e-10)
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])


@pytest.mark.parametrize("vals", [np.float64, np.float32])
def test_sliced_copy_gives_the_pipelined_loop_bit_for_bit(pc, vals, monkeypatch):
    """With rows of at most 64 entries both loops walk every group one lane per row; the sliced
    copy only moves the entries (entry k of the group's 32 rows contiguous, padded to the
    group's longest row): same products in the same order, so the same iterates.  30,001 rows:
    the last group is ragged."""
    A = W.powerlaw_spd(n=30001, seed=7, w_max=60, cap=64, dtype=vals)
    out = {}
    for loop in ("pipe", "sliced"):
        monkeypatch.setenv("PC_BIN_SPMV", loop)
        x, info, binned = _solve(pc, A, 32, "on", prec="fp32")
        assert binned and info["status_name"] == "ok"
        out[loop] = (x, info["iterations"])
    assert out["pipe"][1] == out["sliced"][1]
    assert np.array_equal(out["pipe"][0], out["sliced"][0])
    res = np.linalg.norm(W.rhs(A.n, 0) - oracle.spmv(A, out["sliced"][0])) / np.linalg.norm(W.rhs(A.n, 0))
    assert res <= 1e-10


def test_sliced_copy_walks_rows_up_to_256_entries_one_lane_per_row(pc, monkeypatch):
    """Over the sliced copy, groups whose rows have 65-256 entries are also walked one lane per
    row (one FMA chain per row in storage order, as the oracle sums), where the CSR walk puts 8
    lanes on a row and combines their partial sums: the iterates then agree to rounding, and
    each matches the oracle's solution."""
    A = W.powerlaw_spd(n=30001, seed=7, w_max=1999, cap=256, dtype=np.float64)
    r = oracle.pcg(A, W.rhs(A.n, 0), 32, 1e-10)
    out = {}
    for loop in ("pipe", "sliced"):
        monkeypatch.setenv("PC_BIN_SPMV", loop)
        x, info, binned = _solve(pc, A, 32, "on")
        assert binned and info["status_name"] == "ok"
        assert abs(info["iterations"] - r["iterations"]) <= 1
        assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])
        out[loop] = x
    assert np.linalg.norm(out["pipe"] - out["sliced"]) <= 1e-12 * np.linalg.norm(out["pipe"])


NATURAL_CASES = {
    "diffusion23": lambda: W.diffusion3d(23, 2.0),                  # ragged: 12,167 rows
    "poisson63": lambda: W.poisson2d(63),
    "rows_to_64": lambda: W.powerlaw_spd(n=20001, seed=3, w_max=60, cap=64, dtype=np.float32),
}


@pytest.mark.parametrize("name", sorted(NATURAL_CASES))
def test_natural_sliced_copy_gives_the_csr_walk_bit_for_bit(pc, name, monkeypatch):
    """Natural row order over the sliced copy (groups of 32 consecutive rows, entry k of each
    row at 32 k + lane): same products in the same order as the CSR walk, so the same iterates;
    rows of up to 64 entries take several rounds of 8."""
    A = NATURAL_CASES[name]()
    bs = 16 if name != "rows_to_64" else 32
    out = {}
    for walk in ("csr", "sliced"):
        monkeypatch.setenv("PC_NAT_SPMV", walk)
        x, info, binned = _solve(pc, A, bs, "off", prec="fp32")
        assert not binned and info["status_name"] == "ok"
        out[walk] = (x, info["iterations"])
    assert out["csr"][1] == out["sliced"][1]
    assert np.array_equal(out["csr"][0], out["sliced"][0])
    b = W.rhs(A.n, 0)
    assert np.linalg.norm(b - oracle.spmv(A, out["sliced"][0])) <= 1e-10 * np.linalg.norm(b)


def test_natural_sliced_copy_needs_rows_of_at_most_64_entries(pc, powerlaw, monkeypatch):
    # longer rows: no sliced copy, the CSR walk runs (same answer as the oracle)
    monkeypatch.setenv("PC_NAT_SPMV", "sliced")
    x, info, binned = _solve(pc, powerlaw, 32, "off")
    assert not binned and info["status_name"] == "ok"
    r = oracle.pcg(powerlaw, W.rhs(powerlaw.n, 0), 32, 1e-10)
    assert np.linalg.norm(x - r["x"]) <= 1e-10 * np.linalg.norm(r["x"])

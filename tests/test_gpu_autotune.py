"""Kernel-shape autotuner of the single-system solve and the launch shapes it chooses between:
every shape gives the oracle's solution (shapes change only the order of per-CTA partial sums),
and the tuned shape is the one later handles build their loop graph with."""
import json

import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NATURAL = {(c, r) for c in (2, 3, 4, 6, 8) for r in (2, 3, 4)}


@pytest.fixture(autouse=True)
def _clean(pc):
    pc.tune_clear()
    yield
    pc.tune_clear()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape", [(2, 2), (3, 4), (8, 3), (6, 2)])
def test_every_natural_shape_matches_oracle(pc, shape):
    A = W.diffusion3d(20, 2.0)
    b = W.rhs(A.n, 0)
    pc.tune_set(16, "fp64", A.n, A.nnz, {"spmv_ctas_per_sm": shape[0], "ring_stages": shape[1], "bin_pipe": -1})
    H = pc.setup(A, 16, prec="fp64")
    x, info = H.pcg(b, tol=1e-10)
    got = H.shape()
    H.destroy()
    assert (got["spmv_ctas_per_sm"], got["ring_stages"]) == shape
    o = oracle.pcg(A, b, 16, 1e-10)
    assert info["status"] == 0 and abs(info["iterations"] - o["iterations"]) <= 1
    assert rel(x.cpu().numpy(), o["x"]) <= 1e-10


def test_autotune_records_a_shape_that_later_handles_use(pc):
    A = W.diffusion3d(32, 2.0)
    best = pc.autotune(A, 16, "fp32", iterations=30)
    assert (best["spmv_ctas_per_sm"], best["ring_stages"]) in NATURAL
    assert best["bin_pipe"] == -1 and best["us_per_iteration"] > 0
    assert pc.tune_get(16, "fp32", A.n, A.nnz) == best
    b = W.rhs(A.n, 1)
    H = pc.setup(A, 16, prec="fp32")
    x, info = H.pcg(b, tol=1e-10)
    assert H.shape() == best
    H.destroy()
    assert info["status"] == 0
    res = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert res <= 1e-10
    # a capped candidate list takes the first candidate only
    pc.tune_clear()
    one = pc.autotune(A, 16, "fp32", iterations=10, max_trials=1)
    assert (one["spmv_ctas_per_sm"], one["ring_stages"]) == (4, 4)


def test_autotune_binned_rows(pc):
    pc.set_row_binning("on")
    try:
        A = W.powerlaw_spd(n=30000, seed=5, w_max=500, cap=400, dtype=np.float64)
        best = pc.autotune(A, 32, "fp32", iterations=20)
        assert best["bin_pipe"] in (0, 1, 2) and best["ring_stages"] in (2, 3, 4)
        b = W.rhs(A.n, 0)
        H = pc.setup(A, 32, prec="fp64")   # another precision: no recorded shape, defaults
        x, info = H.pcg(b, tol=1e-10)
        assert H.row_binned() and H.shape()["bin_pipe"] == -1
        H.destroy()
        o = oracle.pcg(A, b, 32, 1e-10)
        assert rel(x.cpu().numpy(), o["x"]) <= 1e-10
        for pipe in (0, 1, 2):
            pc.tune_set(32, "fp64", A.n, A.nnz, {"spmv_ctas_per_sm": 0, "ring_stages": 2, "bin_pipe": pipe})
            H = pc.setup(A, 32, prec="fp64")
            x, info = H.pcg(b, tol=1e-10)
            assert H.shape()["bin_pipe"] == pipe
            H.destroy()
            assert rel(x.cpu().numpy(), o["x"]) <= 1e-10
    finally:
        pc.set_row_binning("auto")


def test_autotune_saves_to_the_cache_file(pc, tmp_path, monkeypatch):
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("PC_TUNE_CACHE", str(path))
    A = W.poisson2d(64)
    best = pc.autotune(A, 8, "fp32", iterations=10, max_trials=3)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    cg = [x for x in lines if x["kind"] == "cg" and x["bs"] == 8 and x["prec"] == 1]
    assert len(cg) == 1
    assert cg[0]["spmv_ctas_per_sm"] == best["spmv_ctas_per_sm"] and cg[0]["ring_stages"] == best["ring_stages"]
    assert cg[0]["sms"] > 0


def test_autotune_rejects_bad_arguments(pc):
    A = W.poisson2d(16)
    for kw in ({"iterations": 0}, {"iterations": 20000}, {"max_trials": -1}):
        with pytest.raises(pc.PcError) as ei:
            pc.autotune(A, 8, "fp32", **{"iterations": 10, **kw})
        assert ei.value.name == "invalid_arg"


# (matrix, block size, precision, whether the update can be fused: it needs the warp-ring
# preconditioner, which serves block sizes up to 32; larger blocks take another kernel)
FUSE_CASES = [
    ("diffusion23", 16, "fp32", True),    # ragged: 12,167 rows
    ("diffusion23", 32, "fp64", True),    # a ring of 2 stages
    ("diffusion23", 7, "fp32", True),     # 28-row warp units
    ("diffusion23", 64, "fp64", False),   # two rows per lane; another preconditioner kernel
    ("poisson63", 8, "fp64", True),
    ("powerlaw", 32, "fp32", True),       # binned SpMV order
]


def _fuse_matrix(name):
    if name == "diffusion23":
        return W.diffusion3d(23, 2.0)
    if name == "poisson63":
        return W.poisson2d(63)
    return W.powerlaw_spd(n=40_000, seed=3, device="cpu")


@pytest.mark.parametrize("name,bs,prec,fusable", FUSE_CASES)
def test_fused_update_matches_the_separate_kernel_bit_for_bit(pc, name, bs, prec, fusable):
    # x += alpha p and p = z + beta p as the preconditioner kernel's tail (fuse_update 1) or as
    # their own kernel (2): the same products in the same order, so the same iterates
    A = _fuse_matrix(name)
    b = W.rhs(A.n, 0)
    out = {}
    for fuse in (1, 2):
        pc.tune_clear()
        pc.tune_set(bs, prec, A.n, A.nnz, {"spmv_ctas_per_sm": 0, "ring_stages": 0, "bin_pipe": -1,
                                           "fuse_update": fuse})
        H = pc.setup(A, bs, prec=prec)
        x, info = H.pcg(b, tol=1e-10)
        got = H.shape()
        H.destroy()
        assert info["status"] == 0
        assert got["fuse_update"] == (fuse if fusable else 2)
        out[fuse] = (x.cpu().numpy(), info["iterations"])
    assert out[1][1] == out[2][1]
    assert np.array_equal(out[1][0], out[2][0])
    if prec == "fp64":
        assert rel(out[1][0], oracle.pcg(A, b, bs, 1e-10)["x"]) <= 1e-10
    res = np.linalg.norm(b - oracle.spmv(A, out[1][0])) / np.linalg.norm(b)
    assert res <= 1e-10


def test_profiling_round_runs_the_fused_kernel_with_the_same_result(pc, monkeypatch):
    # the per-kernel timing mode launches the loop body eagerly; with the fused tail it has no
    # update kernel to time and gives the graph loop's iterates
    A = W.diffusion3d(24, 2.0)
    b = W.rhs(A.n, 0)
    pc.tune_set(16, "fp32", A.n, A.nnz, {"spmv_ctas_per_sm": 0, "ring_stages": 0, "bin_pipe": -1,
                                         "fuse_update": 1})
    H = pc.setup(A, 16, prec="fp32")
    x_graph, i_graph = H.pcg(b, tol=1e-10)
    assert H.shape()["fuse_update"] == 1
    H.destroy()
    monkeypatch.setenv("PC_CG_PROFILE", "1")
    H = pc.setup(A, 16, prec="fp32")
    x_prof, i_prof = H.pcg(b, tol=1e-10)
    kt = H.trace(8)
    H.destroy()
    assert i_prof["iterations"] == i_graph["iterations"]
    assert np.array_equal(x_prof.cpu().numpy(), x_graph.cpu().numpy())
    assert len(kt) >= 3 and kt[0] > 0 and kt[1] > 0 and kt[2] == 0


@pytest.mark.parametrize("prec,expected", [("fp32", 2), ("tf32", 2), ("fp64", 1)])
def test_default_update_is_fused_with_fp64_factors_only(pc, prec, expected):
    A = W.diffusion3d(20, 2.0)
    b = W.rhs(A.n, 0)
    H = pc.setup(A, 16, prec=prec)
    x, info = H.pcg(b, tol=1e-10)
    got = H.shape()["fuse_update"]
    H.destroy()
    assert info["status"] == 0 and got == expected

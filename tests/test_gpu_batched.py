"""Batched mode on the GPU: setup + PCG of many independent systems in one persistent,
graph-captured launch, checked system by system against the oracle.

Workload: random-geometric-graph Laplacians + 1e-3 I (points U[0,1]^3, about 12
neighbours, Morton order), sizes log-uniform, block sizes drawn from {4, 8, 16, 32, 64},
b ~ N(0, 1) per system."""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rhs(batch, seed=0):
    return np.random.default_rng(seed).standard_normal(int(batch.sys_row[-1]))


def _sys_slice(batch, s):
    return slice(int(batch.sys_row[s]), int(batch.sys_row[s + 1]))


@pytest.fixture(scope="module")
def small_batch():
    return W.rgg_batch(n_sys=40, seed=11, n_min=60, n_max=4000)


def _oracle_all(batch, b, tol):
    out = []
    for s, A in enumerate(batch.systems):
        out.append(oracle.pcg(A, b[_sys_slice(batch, s)], int(batch.bs[s]), tol))
    return out


def test_batched_fp64_matches_oracle_per_system(pc, small_batch):
    batch = small_batch
    b = _rhs(batch)
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10)
    x = x.cpu().numpy()
    ref = _oracle_all(batch, b, 1e-10)
    assert info["status_name"] == "ok"
    for s, r in enumerate(ref):
        assert r["status"] == "ok"
        xs = x[_sys_slice(batch, s)]
        err = np.linalg.norm(xs - r["x"]) / np.linalg.norm(r["x"])
        assert err <= 1e-10, (s, err)
        assert abs(int(per["iterations"][s]) - r["iterations"]) <= 1, (s, per["iterations"][s], r["iterations"])
        assert per["status"][s] == 0
        assert per["relres"][s] <= 1e-10


def test_batched_mixed_precision_reaches_tolerance(pc, small_batch):
    batch = small_batch
    b = _rhs(batch, 1)
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10, prec="fp32")
    x = x.cpu().numpy()
    assert info["status_name"] == "ok"
    assert np.all(per["status"] == 0)
    assert np.all(per["relres"] <= 1e-10)
    for s, A in enumerate(batch.systems):
        sl = _sys_slice(batch, s)
        r = b[sl] - oracle.spmv(A, x[sl])
        assert np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(b[sl])


def test_batched_teams_agree_with_single_cta_systems(pc, small_batch):
    """Forcing multi-CTA teams (small scheduler target) gives the oracle's answer too."""
    batch = small_batch
    b = _rhs(batch, 2)
    pc.batch_set_tuning(0, 8, 64.0)
    try:
        H = pc.Batch(batch)
        team, _ = H.teams()
        assert team.max() > 1
        x, per, info = H.solve(b, tol=1e-10)
        H.destroy()
    finally:
        pc.batch_set_tuning(0, 0, 0.0)
    x = x.cpu().numpy()
    ref = _oracle_all(batch, b, 1e-10)
    for s, r in enumerate(ref):
        xs = x[_sys_slice(batch, s)]
        assert np.linalg.norm(xs - r["x"]) <= 1e-10 * np.linalg.norm(r["x"]), s
        assert abs(int(per["iterations"][s]) - r["iterations"]) <= 1


def test_batched_graph_replay_is_deterministic(pc, small_batch):
    import torch

    batch = small_batch
    b = torch.from_numpy(_rhs(batch, 3)).cuda()
    H = pc.Batch(batch)
    try:
        x = torch.empty_like(b)
        _, per1, info1 = H.solve(b, 1e-10, x=x)
        x1 = x.clone()
        _, per2, info2 = H.solve(b, 1e-10, x=x)
        assert info2["graph"]
        assert torch.equal(x1, x)
        assert np.array_equal(per1["iterations"], per2["iterations"])
        li = H.launch_info()
        assert li["grid"] >= 1 and li["slots"] >= batch.n_sys
    finally:
        H.destroy()


def _mini_batch(systems, bss):
    return W.concat_batch(systems, bss)


def test_batched_edge_cases(pc):
    """One-row system, a system smaller than its block, ragged last blocks, odd block sizes
    (generic path), a zero right-hand side, and an empty system."""
    rng = np.random.default_rng(5)
    pts = [rng.random((n, 3)) for n in (1, 3, 37, 257, 500)]
    systems = [W.rgg_laplacian(p) for p in pts]
    empty = W.CSR(np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    systems.insert(2, empty)
    bss = [4, 8, 16, 5, 64, 1]
    batch = _mini_batch(systems, bss)
    b = _rhs(batch, 4)
    zero_sys = 4
    b[_sys_slice(batch, zero_sys)] = 0.0
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10)
    x = x.cpu().numpy()
    assert info["status_name"] == "ok", info
    for s, A in enumerate(batch.systems):
        sl = _sys_slice(batch, s)
        if A.n == 0:
            assert per["status"][s] == 0 and per["iterations"][s] == 0
            continue
        if s == zero_sys:
            assert np.all(x[sl] == 0.0) and per["iterations"][s] == 0
            continue
        r = oracle.pcg(A, b[sl], bss[s], 1e-10)
        assert np.linalg.norm(x[sl] - r["x"]) <= 1e-10 * np.linalg.norm(r["x"]), s


def test_batched_not_spd_system_is_reported(pc):
    rng = np.random.default_rng(6)
    good = W.rgg_laplacian(rng.random((300, 3)))
    bad = W.rgg_laplacian(rng.random((200, 3)))
    bad.val = bad.val.copy()
    rows = np.repeat(np.arange(bad.n), np.diff(bad.row_ptr))
    bad.val[(rows == 17) & (bad.col == 17)] = -1.0      # a negative pivot in block 17 // 8 = 2
    batch = _mini_batch([good, bad, good], [8, 8, 8])
    b = _rhs(batch, 7)
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10, check=False)
    assert info["status_name"] == "not_spd" and info["failed_block"] == 1
    assert per["status"][1] == 2
    assert per["status"][0] == 0 and per["status"][2] == 0


def test_batched_invalid_column_rejected(pc):
    rng = np.random.default_rng(8)
    A = W.rgg_laplacian(rng.random((100, 3)))
    batch = _mini_batch([A, A], [8, 8])
    batch.col = batch.col.copy()
    batch.col[-1] = 100      # outside the second system
    with pytest.raises(pc.PcError):
        pc.Batch(batch)


def test_batched_c3_shape_sample(pc):
    """128 systems with the C3 size law cut at 2e4 rows: every system reaches the tolerance
    (true residual) and sampled systems match the oracle."""
    batch = W.rgg_batch(n_sys=128, seed=3, n_min=1e3, n_max=2e4)
    b = _rhs(batch, 0)
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10)
    x = x.cpu().numpy()
    assert info["status_name"] == "ok"
    assert np.all(per["relres"] <= 1e-10)
    for s in (0, 17, 64, 127):
        A = batch.systems[s]
        sl = _sys_slice(batch, s)
        r = oracle.pcg(A, b[sl], int(batch.bs[s]), 1e-10)
        assert np.linalg.norm(x[sl] - r["x"]) <= 1e-10 * np.linalg.norm(r["x"]), s


def test_batched_autotune_records_a_shape(pc, small_batch):
    batch = small_batch
    b = _rhs(batch, 9)
    pc.binding.lib().pc_batch_clear_tuned()
    ms, cfg = pc.batch_autotune(batch, b, tol=1e-10, max_trials=4)
    assert ms > 0 and cfg["team_max"] in (4, 8, 32) and cfg["setup_kb"] in (70, 140)
    H = pc.Batch(batch)
    try:
        li = H.launch_info()
        if cfg["ctas_per_sm"]:
            assert li["ctas_per_sm"] <= cfg["ctas_per_sm"]
        assert li["team_max"] == cfg["team_max"]
        x, per, info = H.solve(b, 1e-10)
        assert info["status_name"] == "ok"
    finally:
        H.destroy()
        pc.binding.lib().pc_batch_clear_tuned()


def test_batched_team_wait_timeout_reports_and_recovers(pc, small_batch):
    """A 1-cycle wait budget makes the team barriers give up: the launch ends with
    PC_ERR_TIMEOUT instead of hanging, and a handle created afterwards solves normally."""
    import os

    batch = small_batch
    b = _rhs(batch, 5)
    pc.batch_set_tuning(0, 8, 64.0)          # force multi-CTA teams
    os.environ["PC_WAIT_BUDGET"] = "1"
    try:
        H = pc.Batch(batch)
        team, _ = H.teams()
        assert team.max() > 1
        x, per, info = H.solve(b, 1e-10, check=False)
        H.destroy()
    finally:
        del os.environ["PC_WAIT_BUDGET"]
        pc.batch_set_tuning(0, 0, 0.0)
    assert info["status_name"] == "timeout"
    x, per, info = pc.pcg_batched(batch, b, tol=1e-10)
    assert info["status_name"] == "ok" and np.all(per["relres"] <= 1e-10)

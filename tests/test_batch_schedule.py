"""Host-side team scheduler of the batched solver (no GPU): every system gets a
contiguous run of queue slots, team sizes are powers of two within the limits, and slots go
to larger teams first, then to longer slots."""
import math

import numpy as np
import pytest

from paper_2410_02408_gb300 import binding as B


def _sizes(n_sys=512, seed=3):
    rng = np.random.default_rng(seed)
    n = np.floor(np.exp(rng.uniform(math.log(1e3), math.log(2e5), n_sys))).astype(np.int64)
    bs = rng.choice(np.array([4, 8, 16, 32, 64]), n_sys).astype(np.int32)
    return n, 13 * n, bs


def _units(n, bs):
    U = np.where(bs <= 32, (32 // bs) * bs, bs)
    return (n + U - 1) // U


@pytest.mark.parametrize("n_ctas,team_max,split", [(304, 32, 2.0), (456, 16, 1.0), (8, 32, 2.0), (1, 32, 2.0)])
def test_schedule_invariants(n_ctas, team_max, split):
    n, nnz, bs = _sizes()
    team, slot0, order, n_slots = B.batch_schedule(n, nnz, bs, n_ctas, team_max, split)
    assert n_slots == int(team.sum())
    assert np.all(team >= 1) and np.all(team <= min(team_max, n_ctas))
    assert np.all((team & (team - 1)) == 0)
    units = _units(n, bs)
    assert np.all((team == 1) | (units >= 4 * team))
    # contiguous, disjoint, covering
    cover = np.zeros(n_slots, dtype=np.int32)
    for s in range(len(n)):
        cover[slot0[s]:slot0[s] + team[s]] += 1
    assert np.all(cover == 1)
    # order lists the systems by first slot; larger teams first
    assert np.all(np.diff(slot0[order]) > 0)
    assert np.all(np.diff(team[order]) <= 0)


def test_schedule_cost_ordering_within_a_team_size():
    n, nnz, bs = _sizes()
    team, slot0, order, _ = B.batch_schedule(n, nnz, bs, 304)
    fac = (bs // 2 + 1) * 4.0
    w = (12.0 * nnz + (88.0 + fac) * n) * np.cbrt(n)
    per = w / team
    for T in np.unique(team):
        sel = [s for s in order if team[s] == T]
        assert np.all(np.diff(per[sel]) <= 0)


def test_schedule_single_cta_grid_uses_teams_of_one():
    n, nnz, bs = _sizes(40)
    team, slot0, order, k = B.batch_schedule(n, nnz, bs, 1)
    assert np.all(team == 1) and k == 40


def test_schedule_rejects_invalid_input():
    with pytest.raises(B.PcError):
        B.batch_schedule([10, 20], [30, 60], [4, 65], 8)
    with pytest.raises(B.PcError):
        B.batch_schedule([10, -1], [30, 60], [4, 8], 8)
    with pytest.raises(B.PcError):
        B.batch_schedule([10, 20], [30, 60], [4, 8], 0)

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


def _solve(pc, A, bs, mode, prec="fp64"):
    import torch

    pc.set_row_binning(mode)
    try:
        H = pc.setup(pc.csr(A), bs, prec=prec)
        b = torch.from_numpy(W.rhs(A.n, 0)).cuda()
        x, info = H.pcg(b, tol=1e-10)
        binned = H.row_binned()
        H.destroy()
    finally:
        pc.set_row_binning("auto")
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

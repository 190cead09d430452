"""The paper's own rows against the oracle: point Jacobi (block size 1, the preconditioner of
Sec. 3.3 and its CUDA kernel in Sec. 4.3), the decoupled per-block solve x = M^-1 b that the
paper assembles from independent block solutions (Sec. 3.2, 3.6), and kappa before and after
block-Jacobi preconditioning at the paper's sizes N = 2^10, 2^12 (Sec. 5.1) on 2D Poisson and
on the random SPD family of several densities."""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_point_jacobi_apply_matches_oracle(pc):
    import torch

    for A in (W.poisson2d(64), W.diffusion3d(33, 2.0), W.random_spd(4096, 8)):
        b = W.rhs(A.n, 0)
        H = pc.setup(A, 1, prec="fp64")
        try:
            z = H.apply("inv", torch.from_numpy(b).cuda()).cpu().numpy()
        finally:
            H.destroy()
        L, f = oracle.factor(A, 1)
        assert f == -1
        zo = oracle.apply(A, L, 1, oracle.MODE_INV, b)
        # block size 1 is z_i = r_i / a_ii: both sides divide by the same diagonal
        d = A.to_scipy().diagonal()
        assert np.allclose(zo, b / d, rtol=2e-15, atol=0)
        assert np.allclose(z, zo, rtol=2e-15, atol=0)


@pytest.mark.parametrize("bs", [1, 8, 16, 32, 64])
def test_decoupled_block_solve_matches_oracle(pc, bs):
    """x_dec = M^-1 b solves every diagonal block on its own; its distance from the PCG solution
    and its residual are what the paper's decoupled scheme gives up."""
    import torch

    for A in (W.poisson2d(64), W.diffusion3d(24, 2.0)):
        b = W.rhs(A.n, 0)
        bd = torch.from_numpy(b).cuda()
        H = pc.setup(A, bs, prec="fp64")
        try:
            xd = H.apply("inv", bd).cpu().numpy()
            x, info = H.pcg(bd, tol=1e-10)
        finally:
            H.destroy()
        L, f = oracle.factor(A, bs)
        xo = oracle.apply(A, L, bs, oracle.MODE_INV, b)
        assert np.linalg.norm(xd - xo) <= 1e-13 * np.linalg.norm(xo)
        po = oracle.pcg(A, b, bs, 1e-10)
        err = np.linalg.norm(xd - po["x"]) / np.linalg.norm(po["x"])
        err_gpu = np.linalg.norm(xd - x.cpu().numpy()) / np.linalg.norm(x.cpu().numpy())
        assert abs(err - err_gpu) <= 1e-8 * err
        # the decoupled solve is not a solution of the coupled system
        assert np.linalg.norm(b - oracle.spmv(A, xd)) > 1e-3 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["poisson2d_32", "poisson2d_64", "random_spd_1024_deg4", "random_spd_1024_deg16",
                                  "random_spd_4096_deg8"])
def test_paper_size_kappa_matches_oracle(pc, name):
    import torch

    if name.startswith("poisson"):
        A = W.poisson2d(int(name.split("_")[1]))
    else:
        _, _, N, deg = name.split("_")
        A = W.random_spd(int(N), int(deg[3:]))
    b = W.rhs(A.n, 0)
    bd = torch.from_numpy(b).cuda()
    m = min(A.n, 200)
    kb = pc.kappa(A, bd, 0, max_steps=m)
    ko = oracle.kappa(A, b, m, 0)
    assert abs(kb["kappa"] / ko["kappa"] - 1) <= 1e-6
    for bs in (1, 4, 16, 64):
        H = pc.setup(A, bs, prec="fp64")
        try:
            ka = H.kappa(bd, max_steps=m)
        finally:
            H.destroy()
        kao = oracle.kappa(A, b, m, bs)
        assert abs(ka["kappa"] / kao["kappa"] - 1) <= 1e-6, (bs, ka["kappa"], kao["kappa"])
        if name.startswith("poisson"):
            # Poisson is an M-matrix: block Jacobi is a regular splitting and cannot raise kappa
            assert ka["kappa"] <= kb["kappa"] * (1 + 1e-9)

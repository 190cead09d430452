"""Adjoint of the preconditioned solve (PcgSolve, pc_grad_val, pc_grad_edges) on the GPU.

Workload: 3D 7-point diffusion with log-normal face coefficients (sigma = 1), loss
L = ||x - x*||^2 for a seeded target x*.  References: the oracle's adjoint formulas fed with
dense FP64 Cholesky solves (12^3), and central finite differences with step h = 1e-6 on 64
seeded face coefficients and 64 seeded entries of b (64^3).
"""
import numpy as np
import pytest

import oracle
from paper_2410_02408_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mask(n):
    N = n ** 3
    p = np.arange(N)
    i, j, k = p % n, (p // n) % n, p // (n * n)
    return np.stack([k > 0, j > 0, i > 0, np.ones(N, bool), i < n - 1, j < n - 1, k < n - 1], axis=1)


def _assemble(torch, n, cx, cy, cz, mask):
    """CSR values of the 7-point operator from face tensors, in the stored-entry order of
    ``W.diffusion3d_from_faces``, with differentiable torch operations."""
    N = n ** 3
    cxm = cx[:, :, :n].reshape(N)
    cxp = cx[:, :, 1:].reshape(N)
    cym = cy[:, :n, :].reshape(N)
    cyp = cy[:, 1:, :].reshape(N)
    czm = cz[:n, :, :].reshape(N)
    czp = cz[1:, :, :].reshape(N)
    diag = ((((cxm + cxp) + cym) + cyp) + czm) + czp
    vals = torch.stack([-czm, -cym, -cxm, diag, -cxp, -cyp, -czp], dim=1)
    return vals[mask]


def _problem(torch, n, sigma=1.0):
    c3 = W.diffusion3d_faces(n, sigma, seed=1)
    A = W.diffusion3d_from_faces(n, *c3)
    b = W.rhs(A.n, 0)
    xs = np.random.default_rng(7).standard_normal(A.n)
    mask = torch.from_numpy(_mask(n)).cuda()
    return c3, A, b, xs, mask


def test_grad_edges_bit_exact_vs_oracle(pc):
    n = 9
    p, q = W.diffusion3d_face_edges(n)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(n ** 3)
    x = rng.standard_normal(n ** 3)
    g = pc.grad_edges(p, q, lam, x).cpu().numpy()
    assert np.array_equal(g, oracle.grad_edges(p, q, lam, x))


def test_grad_edges_out_of_range_edge_is_nan(pc):
    p = np.array([0, 5, 1], dtype=np.int32)
    q = np.array([1, -1, 4], dtype=np.int32)
    lam = np.ones(4)
    x = np.arange(4.0)
    g = pc.grad_edges(p, q, lam, x).cpu().numpy()
    assert g[0] == 0.0 and np.isnan(g[1]) and np.isnan(g[2])


def test_pcgsolve_matches_oracle_adjoint(pc):
    import torch

    n = 10
    c3, A, b, xs, mask = _problem(torch, n)
    pattern = pc.csr(A)
    val = torch.from_numpy(A.val).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = pc.PcgSolve.apply(val, bt, pattern, 16, 1e-13)
    loss = ((x - torch.from_numpy(xs).cuda()) ** 2).sum()
    loss.backward()
    xo = oracle.pcg(A, b, 16, 1e-13)["x"]
    lam = oracle.pcg(A, 2 * (xo - xs), 16, 1e-13)["x"]
    gval = oracle.grad_val(A, lam, xo)
    rel = lambda a, r: np.linalg.norm(a - r) / np.linalg.norm(r)
    assert rel(x.detach().cpu().numpy(), xo) <= 1e-10
    assert rel(bt.grad.cpu().numpy(), lam) <= 1e-9
    assert rel(val.grad.cpu().numpy(), gval) <= 1e-9


def test_pcgsolve_without_grad_and_fp32_preconditioner(pc):
    import torch

    n = 8
    _, A, b, xs, _ = _problem(torch, n)
    pattern = pc.csr(A)
    val = torch.from_numpy(A.val).cuda()
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = pc.PcgSolve.apply(val, bt, pattern, 8, 1e-12, 100000, "fp32")
    ((x - torch.from_numpy(xs).cuda()) ** 2).sum().backward()
    assert val.grad is None
    Ad = A.to_dense()
    xd = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad, 2 * (xd - xs))
    assert np.linalg.norm(bt.grad.cpu().numpy() - lam) <= 1e-8 * np.linalg.norm(lam)


def test_dense_reference_gradient_12cubed(pc):
    """12^3 sub-case: dense FP64 Cholesky x and lambda, then the adjoint formulas, vs the
    adjoint PCG at tol 1e-13 (gate 1e-8 relative)."""
    import torch

    n = 12
    (cx, cy, cz), A, b, xs, mask = _problem(torch, n)
    Ad = A.to_dense()
    Lc = np.linalg.cholesky(Ad)
    xd = np.linalg.solve(Lc.T, np.linalg.solve(Lc, b))
    lam = np.linalg.solve(Lc.T, np.linalg.solve(Lc, 2 * (xd - xs)))
    p, q = W.diffusion3d_face_edges(n)
    gc_ref = oracle.grad_edges(p, q, lam, xd)

    ct = [torch.from_numpy(c).cuda().requires_grad_(True) for c in (cx, cy, cz)]
    val = _assemble(torch, n, *ct, mask)
    assert np.array_equal(val.detach().cpu().numpy(), A.val)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = pc.PcgSolve.apply(val, bt, pc.csr(A), 16, 1e-13)
    ((x - torch.from_numpy(xs).cuda()) ** 2).sum().backward()

    gb = bt.grad.cpu().numpy()
    assert np.abs(gb - lam).max() <= 1e-8 * np.abs(lam).max()
    g_chain = np.concatenate([c.grad.cpu().numpy().ravel() for c in ct])
    g_direct = pc.grad_edges(p, q, bt.grad, x.detach()).cpu().numpy()
    scale = np.abs(gc_ref).max()
    assert np.abs(g_chain - gc_ref).max() <= 1e-8 * scale
    assert np.abs(g_direct - gc_ref).max() <= 1e-8 * scale


def _fd(x_plus, x_minus, xs, h):
    """Central difference of L = ||x - x*||^2, evaluated as
    sum (x+ - x-)(x+ + x- - 2 x*) / (2h) so that the two losses do not cancel."""
    return float(((x_plus - x_minus) * (x_plus + x_minus - 2 * xs)).sum() / (2 * h))


def test_finite_differences_64cubed(pc):
    """64^3, sigma = 1: adjoint gradients vs central differences (h = 1e-6) on 64 seeded
    faces and 64 seeded entries of b.  Gate: 1e-5 relative with a floor of 1e-6 max|g|.

    The floor is set by the finite differences, not by the adjoint: on face 219884 the
    adjoint gradient (-0.0353801797056) agrees to 1e-13 with one computed from FP64 sparse
    LU solves, while the difference quotient of two iterative solves differs from both by
    1.0e-7 max|g|.

    Each finite-difference pair is solved past stagnation with the same fixed number of
    iterations (tol = 0, max_iter = K, K = the iterations the unperturbed solve needs for
    1e-13 plus 30), so that the two solves follow the same path and their rounding errors
    cancel in the difference instead of swamping it."""
    import torch

    n = 64
    h = 1e-6
    (cx, cy, cz), A, b, xs, mask = _problem(torch, n)
    ct = [torch.from_numpy(c).cuda().requires_grad_(True) for c in (cx, cy, cz)]
    val = _assemble(torch, n, *ct, mask)
    pattern = pc.csr(A)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = pc.PcgSolve.apply(val, bt, pattern, 16, 1e-13)
    xs_t = torch.from_numpy(xs).cuda()
    ((x - xs_t) ** 2).sum().backward()
    gc = torch.cat([c.grad.reshape(-1) for c in ct]).cpu().numpy()
    gb = bt.grad.cpu().numpy()
    p, q = W.diffusion3d_face_edges(n)
    g_direct = pc.grad_edges(p, q, bt.grad, x.detach()).cpu().numpy()
    assert np.abs(g_direct - gc).max() <= 1e-9 * np.abs(gc).max()

    _, info0 = pc.pcg(pattern, bt.detach(), 16, tol=1e-13)
    K = info0["iterations"] + 30
    rng = np.random.default_rng(11)
    faces = rng.choice(gc.size, 64, replace=False)
    rows = rng.choice(A.n, 64, replace=False)
    c_flat = torch.cat([c.detach().reshape(-1) for c in ct])
    sizes = [c.numel() for c in ct]
    bn = float(torch.linalg.norm(bt.detach()))

    def checked(Am, rhs, xx, info):
        assert info["status_name"] in ("ok", "no_convergence"), info
        res = float(torch.linalg.norm(rhs - pc.spmv(Am, xx))) / bn
        assert res <= 1e-11, res
        return xx

    def solve_with(cv):
        parts = torch.split(cv, sizes)
        v = _assemble(torch, n, *[t.reshape(c.shape) for t, c in zip(parts, ct)], mask)
        Am = pc.CSR(pattern.row_ptr, pattern.col, v)
        xx, info = pc.pcg(Am, bt.detach(), 16, tol=0.0, max_iter=K, check=False)
        return checked(Am, bt.detach(), xx, info)

    def gate(g, fds, scale, what):
        err = np.abs(g - fds)
        ok = err <= 1e-5 * np.abs(fds) + 1e-6 * scale
        worst = int(np.argmax(err / (1e-5 * np.abs(fds) + 1e-6 * scale)))
        msg = (f"{what}: {int((~ok).sum())} of {len(g)} outside the gate; max |g-fd|/max|g| = "
               f"{err.max() / scale:.3e}; median relative {np.median(err / np.abs(fds)):.3e}; "
               f"worst {worst}: g={g[worst]!r} fd={fds[worst]!r}")
        print(msg)
        assert ok.all(), msg

    fds = []
    for f in faces:
        cp = c_flat.clone()
        cp[f] += h
        cm = c_flat.clone()
        cm[f] -= h
        fds.append(_fd(solve_with(cp), solve_with(cm), xs_t, h))
    gate(gc[faces], np.array(fds), np.abs(gc).max(), "faces")

    H = pc.setup(pattern, 16)
    fds = []
    try:
        for i in rows:
            e = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            e[int(i)] = h
            bp, bm = bt.detach() + e, bt.detach() - e
            xp = checked(pattern, bp, *H.pcg(bp, tol=0.0, max_iter=K, check=False))
            xm = checked(pattern, bm, *H.pcg(bm, tol=0.0, max_iter=K, check=False))
            fds.append(_fd(xp, xm, xs_t, h))
    finally:
        H.destroy()
    gate(gb[rows], np.array(fds), np.abs(gb).max(), "b")

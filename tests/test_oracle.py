"""Pins for the FP64 CPU oracle: closed forms, library routines on tiny inputs,
invariants and brute force.  None of these compares the oracle with itself."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_2410_02408_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, "kappa_closed_forms.txt")) as f:
        for line in f:
            if line.startswith(name):
                return float(line.split()[1])
    raise KeyError(name)


def random_spd_csr(n, density, seed, diag_shift=1.0):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    M = M + M.T
    M = M + sp.diags(np.abs(M).sum(axis=1).A1 + diag_shift)
    M = M.tocsr()
    M.sort_indices()
    return W.CSR(M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def dense_blocks(A, bs):
    D = A.to_dense()
    n = A.n
    out = []
    for s in range(0, n, bs):
        out.append(D[s:s + bs, s:s + bs])
    return out


# ---------------------------------------------------------------- extraction
@pytest.mark.parametrize("n,bs", [(100, 10), (101, 7), (64, 64), (30, 1)])
def test_extract_matches_dense_slicing_bit_exact(n, bs):
    A = random_spd_csr(n, 0.08, seed=n + bs)
    D = oracle.extract_blocks(A, bs)
    ref = dense_blocks(A, bs)
    assert D.shape[0] == len(ref) == math.ceil(n / bs)
    for k, R in enumerate(ref):
        b = R.shape[0]
        assert np.array_equal(D[k, :b, :b], R)           # bit-exact copy
        assert not D[k, b:, :].any() and not D[k, :, b:].any()


def test_extract_poisson2d_block_is_grid_line_operator():
    A = W.poisson2d(8)
    D = oracle.extract_blocks(A, 8)
    T = np.diag(np.full(8, 4.0)) - np.diag(np.ones(7), 1) - np.diag(np.ones(7), -1)
    for k in range(8):
        assert np.array_equal(D[k], T)


# ---------------------------------------------------------------- Cholesky
def test_cholesky_matches_lapack_on_random_spd():
    rng = np.random.default_rng(0)
    for b in (1, 2, 5, 16, 33, 64):
        G = rng.standard_normal((b, b))
        D = G @ G.T + b * np.eye(b)
        L, f = oracle.cholesky(D)
        assert f == -1
        assert np.allclose(L, np.linalg.cholesky(D), rtol=1e-13, atol=1e-13 * np.abs(D).max())
        assert np.abs(L @ L.T - D).max() <= 1e-14 * np.abs(D).max() * b
        assert np.array_equal(np.triu(L, 1), np.zeros_like(L))


def test_cholesky_closed_form_1d_poisson():
    # tridiag(-1, 2, -1): L_ii = sqrt((i+2)/(i+1)), L_{i+1,i} = -sqrt((i+1)/(i+2))
    b = 20
    D = 2 * np.eye(b) - np.eye(b, k=1) - np.eye(b, k=-1)
    L, f = oracle.cholesky(D)
    i = np.arange(b)
    assert f == -1
    assert np.allclose(np.diag(L), np.sqrt((i + 2) / (i + 1)), rtol=1e-15, atol=0)
    assert np.allclose(np.diag(L, -1), -np.sqrt((i[:-1] + 1) / (i[:-1] + 2)), rtol=1e-15, atol=0)
    assert np.array_equal(np.tril(L, -2), np.zeros_like(L))


def test_cholesky_reports_first_bad_pivot():
    D = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])   # singular leading 2x2
    _, f = oracle.cholesky(D, tol=1e-12)
    assert f == 1
    _, f = oracle.cholesky(-np.eye(3))
    assert f == 0


def test_factor_blocks_reports_failing_block():
    A = W.poisson2d(8)
    rp, col, val = A.row_ptr.copy(), A.col.copy(), A.val.copy()
    # make block 3 (rows 24..31) indefinite by flipping one diagonal entry
    row = 27
    for e in range(rp[row], rp[row + 1]):
        if col[e] == row:
            val[e] = -4.0
    L, f = oracle.factor(W.CSR(rp, col, val), 8)
    assert f == 3


def test_triangular_inverse_and_minv():
    rng = np.random.default_rng(1)
    n, bs = 50, 16
    A = random_spd_csr(n, 0.2, seed=7)
    L, f = oracle.factor(A, bs)
    assert f == -1
    X = oracle.tri_inv(L, n, bs)
    Mi = oracle.minv(X, n, bs)
    for k, Dk in enumerate(dense_blocks(A, bs)):
        b = Dk.shape[0]
        Lk = L[k, :b, :b]
        assert np.allclose(X[k, :b, :b] @ Lk, np.eye(b), atol=1e-13)
        assert np.allclose(Mi[k, :b, :b], np.linalg.inv(Dk), rtol=1e-12, atol=1e-14)
        assert np.array_equal(Mi[k, :b, :b], Mi[k, :b, :b].T)


# ---------------------------------------------------------------- apply, SpMV, dot
@pytest.mark.parametrize("bs", [1, 4, 10, 16])
def test_block_apply_modes_match_dense_solves(bs):
    n = 77
    A = random_spd_csr(n, 0.1, seed=bs)
    L, f = oracle.factor(A, bs)
    assert f == -1
    v = np.random.default_rng(bs).standard_normal(n)
    z_inv = oracle.apply(A, L, bs, oracle.MODE_INV, v)
    z_l = oracle.apply(A, L, bs, oracle.MODE_LINV, v)
    z_lt = oracle.apply(A, L, bs, oracle.MODE_LTINV, v)
    Lfull = np.zeros((n, n))
    for k, s in enumerate(range(0, n, bs)):
        b = min(bs, n - s)
        Lfull[s:s + b, s:s + b] = L[k, :b, :b]
    Mfull = sla.block_diag(*dense_blocks(A, bs))
    assert np.allclose(z_inv, np.linalg.solve(Mfull, v), rtol=1e-12, atol=1e-13)
    assert np.allclose(z_l, sla.solve_triangular(Lfull, v, lower=True), rtol=1e-13, atol=1e-14)
    assert np.allclose(z_lt, sla.solve_triangular(Lfull.T, v, lower=False), rtol=1e-13, atol=1e-14)
    y = oracle.apply(A, L, bs, oracle.MODE_SYM, v)
    Li = np.linalg.inv(Lfull)
    assert np.allclose(y, Li @ A.to_dense() @ Li.T @ v, rtol=1e-11, atol=1e-12)


def test_spmv_and_dot():
    A = random_spd_csr(200, 0.05, seed=3)
    x = np.random.default_rng(3).standard_normal(200)
    assert np.allclose(oracle.spmv(A, x), A.to_dense() @ x, rtol=1e-14, atol=1e-13)
    y = np.random.default_rng(4).standard_normal(200)
    assert abs(oracle.dot(x, y) - math.fsum(x * y)) <= 1e-13 * np.abs(x * y).sum()


def test_preconditioned_operator_is_symmetric():
    A, b = W.diffusion3d(10, 2.0), None
    L, f = oracle.factor(A, 16)
    assert f == -1
    rng = np.random.default_rng(5)
    for _ in range(3):
        u, v = rng.standard_normal(A.n), rng.standard_normal(A.n)
        a = u @ oracle.apply(A, L, 16, oracle.MODE_SYM, v)
        c = v @ oracle.apply(A, L, 16, oracle.MODE_SYM, u)
        assert abs(a - c) <= 1e-13 * max(abs(a), 1.0) * 100


# ---------------------------------------------------------------- tridiagonal eigenvalues
def test_sturm_and_bisection_match_lapack():
    rng = np.random.default_rng(2)
    for m in (1, 2, 7, 50, 200):
        a = rng.standard_normal(m) * 3
        b = rng.standard_normal(max(m - 1, 0))
        ev = sla.eigvalsh_tridiagonal(a, b) if m > 1 else a.copy()
        for x in (-2.0, 0.1, 1.5):
            assert oracle.sturm_count(a, b if m > 1 else np.zeros(1), x) == int((ev < x).sum())
        lo = oracle.tridiag_eig(a, b, 0)
        hi = oracle.tridiag_eig(a, b, m - 1)
        scale = np.abs(ev).max()
        assert abs(lo - ev[0]) <= 1e-14 * scale * 10
        assert abs(hi - ev[-1]) <= 1e-14 * scale * 10


# ---------------------------------------------------------------- kappa (Lanczos)
def test_kappa_poisson2d_closed_forms():
    A = W.poisson2d(64)
    b = W.rhs(A.n, 0)
    ref_before = 1.0 / math.tan(math.pi / 130) ** 2
    ref_bs64 = 1.0 / (1.0 - math.cos(math.pi / 65))
    assert ref_before == pytest.approx(golden("poisson2d_64_before"), rel=1e-15)
    assert ref_bs64 == pytest.approx(golden("poisson2d_64_after_bs64"), rel=1e-15)
    k0 = oracle.kappa(A, b, 200, 0)["kappa"]
    k1 = oracle.kappa(A, b, 200, 1)["kappa"]
    k64 = oracle.kappa(A, b, 200, 64)["kappa"]
    assert k0 == pytest.approx(ref_before, rel=1e-10)
    assert k1 == pytest.approx(golden("poisson2d_64_after_bs1"), rel=1e-10)
    assert k64 == pytest.approx(ref_bs64, rel=1e-10)


def test_kappa_1d_poisson_closed_form():
    n = 150   # N <= m: Lanczos with reorthogonalisation spans the whole space
    A = W.poisson1d(n)
    b = W.rhs(n, 0)
    k = oracle.kappa(A, b, 200, 0)
    assert k["kappa"] == pytest.approx(1.0 / math.tan(math.pi / (2 * (n + 1))) ** 2, rel=1e-11)


def test_kappa_after_matches_dense_eig():
    A = W.poisson2d(32)
    b = W.rhs(A.n, 0)
    D = A.to_dense()
    for bs in (4, 16):
        L, _ = oracle.factor(A, bs)
        Lfull = sla.block_diag(*[L[k] for k in range(L.shape[0])])[:A.n, :A.n]
        Li = sla.solve_triangular(Lfull, np.eye(A.n), lower=True)
        ev = np.linalg.eigvalsh(Li @ D @ Li.T)
        k = oracle.kappa(A, b, 200, bs)["kappa"]
        assert k == pytest.approx(ev[-1] / ev[0], rel=1e-9)


def test_kappa_tiny_exact_and_invariants():
    A = random_spd_csr(120, 0.05, seed=11)
    b = W.rhs(A.n, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    assert oracle.kappa(A, b, 200, 0)["kappa"] == pytest.approx(ev[-1] / ev[0], rel=1e-11)
    # a single block of size N preconditions exactly: kappa = 1
    assert oracle.kappa(A, b, 200, 120)["kappa"] == pytest.approx(1.0, abs=1e-12)
    # block size 1 is point Jacobi: spectrum of D^{-1/2} A D^{-1/2}
    d = np.diag(A.to_dense())
    J = A.to_dense() / np.sqrt(np.outer(d, d))
    evj = np.linalg.eigvalsh(J)
    assert oracle.kappa(A, b, 200, 1)["kappa"] == pytest.approx(evj[-1] / evj[0], rel=1e-11)


def test_kappa_block_diagonal_matrix_is_one():
    blocks = []
    rng = np.random.default_rng(8)
    for _ in range(6):
        G = rng.standard_normal((8, 8))
        blocks.append(G @ G.T + 8 * np.eye(8))
    M = sp.csr_matrix(sla.block_diag(*blocks))
    M.sort_indices()
    A = W.CSR(M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)
    b = W.rhs(A.n, 0)
    assert oracle.kappa(A, b, 200, 8)["kappa"] == pytest.approx(1.0, abs=1e-12)
    r = oracle.pcg(A, b, 8, 1e-10)
    assert r["status"] == "ok" and r["iterations"] == 1
    assert np.allclose(r["x"], np.linalg.solve(M.toarray(), b), rtol=1e-13, atol=1e-14)


def test_kappa_after_le_before_on_m_matrix():
    A = W.diffusion3d(12, 2.0)
    b = W.rhs(A.n, 0)
    kb = oracle.kappa(A, b, 200, 0)["kappa"]
    for bs in (1, 8, 32):
        assert oracle.kappa(A, b, 200, bs)["kappa"] <= kb


# ---------------------------------------------------------------- PCG
@pytest.mark.parametrize("bs", [0, 1, 8, 12, 64])
def test_pcg_matches_direct_solve(bs):
    A = W.diffusion3d(10, 1.0)
    b = W.rhs(A.n, 0)
    r = oracle.pcg(A, b, bs, 1e-12)
    assert r["status"] == "ok"
    x_ref = spla.spsolve(A.to_scipy().tocsc(), b)
    res = np.linalg.norm(A.to_dense() @ r["x"] - b) / np.linalg.norm(b)
    assert res <= 1e-12 and r["true_rel_residual"] == pytest.approx(res, rel=1e-6)
    ev = np.linalg.eigvalsh(A.to_dense())
    assert np.linalg.norm(r["x"] - x_ref) / np.linalg.norm(x_ref) <= 1e-12 * ev[-1] / ev[0]


def test_pcg_coefficients_match_lanczos_tridiagonal():
    # Lanczos on L^{-1} A L^{-T} from L^{-1} b gives T_11 = 1/alpha_0,
    # T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j
    A = W.poisson2d(64)
    b = W.rhs(A.n, 0)
    r = oracle.pcg(A, b, 16, 1e-10, record=True)
    al, be = r["alphas"], r["betas"]
    la, lb = oracle.lanczos(A, b, 30, 16)
    T_diag = np.empty(30)
    T_diag[0] = 1 / al[0]
    T_diag[1:] = 1 / al[1:30] + be[:29] / al[:29]
    T_off = np.sqrt(be[:29]) / al[:29]
    assert np.allclose(la[:30], T_diag, rtol=1e-8)
    assert np.allclose(lb[:29], T_off, rtol=1e-8)


def test_pcg_iteration_counts_poisson2d():
    A = W.poisson2d(64)
    b = W.rhs(A.n, 0)
    its = {bs: oracle.pcg(A, b, bs, 1e-10)["iterations"] for bs in (1, 16, 64)}
    # larger blocks never need more iterations here; point Jacobi on a constant
    # diagonal is plain CG up to scaling
    assert its[1] >= its[16] >= its[64]
    assert oracle.pcg(A, b, 0, 1e-10)["iterations"] == its[1]


def test_pcg_status_codes():
    A = W.poisson2d(16)
    b = W.rhs(A.n, 0)
    r = oracle.pcg(A, b, 4, 1e-10, max_iter=1)
    assert r["status"] == "no_convergence" and r["iterations"] == 1
    r = oracle.pcg(A, np.zeros(A.n), 4, 1e-10)
    assert r["status"] == "ok" and r["iterations"] == 0 and not r["x"].any()
    val = A.val.copy()
    val[A.row_ptr[5]:A.row_ptr[6]] *= -1   # breaks SPD of block 1
    r = oracle.pcg(W.CSR(A.row_ptr, A.col, val), b, 4, 1e-10)
    assert r["status"] == "not_spd" and r["failed_block"] == 1
    # an indefinite matrix whose blocks are SPD breaks CG down (p.q <= 0)
    D = np.array([[1.0, 3.0], [3.0, 1.0]])
    M = sp.csr_matrix(D)
    r = oracle.pcg(W.CSR(M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data),
                   np.array([1.0, -1.0]), 1, 1e-10)
    assert r["status"] == "breakdown"


def test_pcg_restart_is_a_fresh_start_from_the_current_iterate():
    # 10^3 diffusion (sigma 2, bs 8) at tol 3e-13: the recurrence residual reaches tol while
    # the true residual b - A x is still above it, so the solve restarts once.  A restart must
    # be exactly a new solve from the current x (r = b - A x, z = M^-1 r, p = z, rho = r.z):
    # the first cycle alone (no restarts allowed) followed by a solve from its x must give the
    # same iterate bit for bit and the same total iteration count.
    A = W.diffusion3d(10, 2.0)
    b = W.rhs(A.n, 0)
    tol = 3e-13
    r = oracle.pcg(A, b, 8, tol)
    assert r["status"] == "ok" and r["restarts"] >= 1
    r1 = oracle.pcg(A, b, 8, tol, max_restarts=0)
    assert r1["status"] == "no_convergence" and r1["true_rel_residual"] > tol
    r2 = oracle.pcg(A, b, 8, tol, x0=r1["x"], max_restarts=r["restarts"] - 1)
    assert r2["status"] == "ok"
    assert r["iterations"] == r1["iterations"] + r2["iterations"]
    assert np.array_equal(r["x"], r2["x"])
    # and the restarted result is a solution: dense residual and forward error vs LAPACK
    D = A.to_dense()
    assert np.linalg.norm(b - D @ r["x"]) <= tol * np.linalg.norm(b)
    x_ref = np.linalg.solve(D, b)
    ev = np.linalg.eigvalsh(D)
    assert np.linalg.norm(r["x"] - x_ref) <= 2 * tol * ev[-1] / ev[0] * np.linalg.norm(x_ref)


def test_dot_is_independent_of_the_thread_count():
    # the chunked dot adds chunk sums in a fixed order, so any thread count gives the same bits;
    # the value is the exact sum to within the usual bound
    x = np.random.default_rng(11).standard_normal(200_003)
    y = np.random.default_rng(12).standard_normal(200_003)
    vals = []
    for t in (1, 3, 4):
        oracle.set_threads(t)
        vals.append(oracle.dot(x, y))
    oracle.set_threads(1)
    assert vals[0] == vals[1] == vals[2]
    assert abs(vals[0] - math.fsum(x * y)) <= 1e-12 * np.abs(x * y).sum()


def test_pcg_and_lanczos_are_independent_of_the_thread_count():
    A = W.diffusion3d(40, 2.0)     # 64,000 rows: above the size where loops are shared
    b = W.rhs(A.n, 0)
    res = []
    for t in (1, 4):
        oracle.set_threads(t)
        p = oracle.pcg(A, b, 16, 1e-10, max_iter=60)
        k = oracle.kappa(A, b, 20, 16)
        res.append((p["x"], p["iterations"], k["kappa"]))
    oracle.set_threads(1)
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]
    assert res[0][2] == res[1][2]


def test_pcg_warm_start_from_solution():
    A = W.poisson2d(16)
    b = W.rhs(A.n, 0)
    x = np.linalg.solve(A.to_dense(), b)
    r = oracle.pcg(A, b, 4, 1e-10, x0=x)
    assert r["status"] == "ok" and r["iterations"] == 0


# ---------------------------------------------------------------- adjoint
def _face_grad_chain(n, gfn):
    """Chain rule of the 7-point assembly: dL/dc for every face (cx, cy, cz shapes) from
    g(p, q) = dL/dA_pq.  Interior face between p and q: g(p,p)+g(q,q)-g(p,q)-g(q,p);
    boundary face of p: g(p,p)."""
    p = np.arange(n ** 3, dtype=np.int64).reshape(n, n, n)   # [k, j, i]
    out = []
    for axis in (2, 1, 0):
        shape = [n, n, n]
        shape[axis] += 1
        g = np.zeros(shape)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[axis] = slice(1, n)
        sl_lo[axis] = slice(0, n - 1)
        q_hi = p[tuple(sl_hi)].ravel()
        q_lo = p[tuple(sl_lo)].ravel()
        gi = gfn(q_hi, q_hi) + gfn(q_lo, q_lo) - gfn(q_hi, q_lo) - gfn(q_lo, q_hi)
        g[tuple(sl_hi)] = gi.reshape(p[tuple(sl_hi)].shape)
        for fidx, cidx in ((0, 0), (n, n - 1)):
            fsl = [slice(None)] * 3
            fsl[axis] = slice(fidx, fidx + 1)
            csl = [slice(None)] * 3
            csl[axis] = slice(cidx, cidx + 1)
            q = p[tuple(csl)].ravel()
            g[tuple(fsl)] = gfn(q, q).reshape(p[tuple(csl)].shape)
        out.append(g)
    return tuple(out)


def test_grad_val_matches_finite_differences_dense():
    n = 4
    cx, cy, cz = W.diffusion3d_faces(n, 1.0, seed=2)
    A = W.diffusion3d_from_faces(n, cx, cy, cz)
    b = W.rhs(A.n, 0)
    xs = np.random.default_rng(9).standard_normal(A.n)

    def loss(c3):
        Ad = W.diffusion3d_from_faces(n, *c3).to_dense()
        x = np.linalg.solve(Ad, b)
        return float(((x - xs) ** 2).sum())

    r = oracle.pcg(A, b, 8, 1e-14)
    x = r["x"]
    lam = oracle.pcg(A, 2 * (x - xs), 8, 1e-14)["x"]
    gval = oracle.grad_val(A, lam, x)
    # dL/db = lambda
    h = 1e-6
    for i in (0, 17, 63):
        e = np.zeros(A.n)
        e[i] = h
        xp = np.linalg.solve(A.to_dense(), b + e)
        xm = np.linalg.solve(A.to_dense(), b - e)
        fd = (((xp - xs) ** 2).sum() - ((xm - xs) ** 2).sum()) / (2 * h)
        assert lam[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # dL/dc through the assembly map
    lookup = {}
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    for e_, (i, j) in enumerate(zip(rows, A.col)):
        lookup[(int(i), int(j))] = gval[e_]
    gfn = lambda p, q: np.array([lookup[(int(a), int(c))] for a, c in zip(p, q)])
    gc = _face_grad_chain(n, gfn)
    for axis in range(3):
        for idx in [(0, 0, 0), (1, 2, 3), (3, 3, 3)]:
            idx = tuple(min(v, s - 1) for v, s in zip(idx, gc[axis].shape))
            c3 = [c.copy() for c in (cx, cy, cz)]
            c3[axis][idx] += h
            lp = loss(c3)
            c3[axis][idx] -= 2 * h
            lm = loss(c3)
            fd = (lp - lm) / (2 * h)
            assert gc[axis][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def _edge_problem(n=4, sigma=1.0):
    cx, cy, cz = W.diffusion3d_faces(n, sigma, seed=2)
    A = W.diffusion3d_from_faces(n, cx, cy, cz)
    b = W.rhs(A.n, 0)
    xs = np.random.default_rng(9).standard_normal(A.n)
    c = np.concatenate([cx.ravel(), cy.ravel(), cz.ravel()])
    return (cx, cy, cz), c, A, b, xs


def test_grad_edges_matches_finite_differences_dense():
    """dL/dc_e from the edge formula vs central differences of L = ||x - x*||^2 with dense
    library solves, on interior and boundary faces of every axis."""
    n = 4
    c3, c, A, b, xs = _edge_problem(n)
    p, q = W.diffusion3d_face_edges(n)
    Ad = A.to_dense()
    x = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad.T, 2 * (x - xs))
    g = oracle.grad_edges(p, q, lam, x)
    sizes = [a.size for a in c3]
    offs = np.cumsum([0] + sizes)

    def loss(cv):
        parts = [cv[offs[a]:offs[a + 1]].reshape(c3[a].shape) for a in range(3)]
        xx = np.linalg.solve(W.diffusion3d_from_faces(n, *parts).to_dense(), b)
        return float(((xx - xs) ** 2).sum())

    h = 1e-6
    picks = [e for e in range(len(c)) if q[e] < 0][:6] + [e for e in range(len(c)) if q[e] >= 0][::37]
    assert any(q[e] < 0 for e in picks) and any(q[e] >= 0 for e in picks)
    for e in picks:
        cp = c.copy()
        cp[e] += h
        cm = c.copy()
        cm[e] -= h
        fd = (loss(cp) - loss(cm)) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_grad_edges_homogeneity():
    """A(c) is linear and homogeneous in c, so sum_e c_e dL/dc_e = -lambda^T A x = -lambda^T b."""
    n = 5
    _, c, A, b, xs = _edge_problem(n, sigma=2.0)
    p, q = W.diffusion3d_face_edges(n)
    Ad = A.to_dense()
    x = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad, 2 * (x - xs))
    g = oracle.grad_edges(p, q, lam, x)
    assert float(c @ g) == pytest.approx(-float(lam @ b), rel=1e-10)


def test_grad_edges_agrees_with_entry_gradient_chain():
    """Edge formula == chain rule of the assembly applied to dL/dA_ij = -lambda_i x_j."""
    n = 4
    c3, c, A, b, xs = _edge_problem(n)
    p, q = W.diffusion3d_face_edges(n)
    Ad = A.to_dense()
    x = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad, 2 * (x - xs))
    gval = oracle.grad_val(A, lam, x)
    lookup = {}
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    for e_, (i, j) in enumerate(zip(rows, A.col)):
        lookup[(int(i), int(j))] = gval[e_]
    gfn = lambda pp, qq: np.array([lookup[(int(a), int(d))] for a, d in zip(pp, qq)])
    chain = np.concatenate([a.ravel() for a in _face_grad_chain(n, gfn)])
    g = oracle.grad_edges(p, q, lam, x)
    np.testing.assert_allclose(g, chain, rtol=1e-9, atol=1e-12 * np.abs(chain).max())


# ---------------------------------------------------------------- complex Hermitian (Sec. 3.1)
def _hpd_dense(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return G @ G.conj().T + n * np.eye(n)


def test_zdot_and_zspmv_match_numpy():
    A = W.hermitian_diffusion3d(6, 1.0)
    x = W.rhs_complex(A.n, 3)
    y = W.rhs_complex(A.n, 4)
    assert abs(oracle.zdot(x, y) - np.vdot(x, y)) <= 1e-13 * np.abs(x * y).sum()
    assert np.allclose(oracle.zspmv(A, x), A.to_dense() @ x, rtol=1e-14, atol=1e-13)


def test_zcholesky_matches_lapack():
    D = _hpd_dense(12, 5)
    L, f = oracle.zcholesky(D)
    assert f == -1
    assert np.allclose(L, np.linalg.cholesky(D), rtol=1e-13, atol=1e-13)
    assert np.allclose(np.diag(L).imag, 0.0) and (np.diag(L).real > 0).all()
    assert np.linalg.norm(L @ L.conj().T - D) <= 1e-14 * np.linalg.norm(D) * 10
    D[3, 3] = -1.0                   # not positive definite: the pivot of column 3 fails
    assert oracle.zcholesky(D)[1] == 3


@pytest.mark.parametrize("bs", [1, 4, 7, 16])
def test_zapply_is_the_block_diagonal_solve(bs):
    A = W.hermitian_diffusion3d(5, 1.5)
    n = A.n
    L, f = oracle.zfactor(A, bs)
    assert f == -1
    v = W.rhs_complex(n, 6)
    D = A.to_dense()
    M = np.zeros_like(D)
    for k in range(0, n, bs):
        e = min(n, k + bs)
        M[k:e, k:e] = D[k:e, k:e]
    assert np.allclose(oracle.zapply(L, n, bs, 0, v), np.linalg.solve(M, v), rtol=1e-12, atol=1e-13)
    Lf = np.zeros_like(D)
    for k in range(0, n, bs):
        e = min(n, k + bs)
        Lf[k:e, k:e] = L[k // bs, :e - k, :e - k]
    assert np.allclose(oracle.zapply(L, n, bs, 2, v), np.linalg.solve(Lf, v), rtol=1e-12, atol=1e-13)
    assert np.allclose(oracle.zapply(L, n, bs, 3, v), np.linalg.solve(Lf.conj().T, v), rtol=1e-12, atol=1e-13)


def test_zkappa_magnetic_path_closed_form():
    # a constant vector potential on a path is a gauge transform of tridiag(-1, 2, -1):
    # kappa = cot^2(pi / (2 (n + 1))), point Jacobi leaves it unchanged (constant diagonal)
    n = 30
    A = W.magnetic_laplacian_1d(n, 0.7)
    ref = 1.0 / math.tan(math.pi / (2 * (n + 1))) ** 2
    b = W.rhs_complex(n, 0)
    assert oracle.zkappa(A, b, 60, 0)["kappa"] == pytest.approx(ref, rel=1e-10)
    assert oracle.zkappa(A, b, 60, 1)["kappa"] == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("bs", [0, 4, 12])
def test_zkappa_matches_dense_eigenvalues(bs):
    A = W.magnetic_laplacian_2d(12, 0.13)      # N = 144 <= 200 steps: Lanczos is exact
    D = A.to_dense()
    if bs:
        L, f = oracle.zfactor(A, bs)
        assert f == -1
        Lf = np.zeros_like(D)
        for k in range(0, A.n, bs):
            e = min(A.n, k + bs)
            Lf[k:e, k:e] = L[k // bs, :e - k, :e - k]
        Li = np.linalg.inv(Lf)
        D = Li @ D @ Li.conj().T
    ev = np.linalg.eigvalsh(D)
    k = oracle.zkappa(A, W.rhs_complex(A.n, 0), 200, bs)
    assert k["kappa"] == pytest.approx(ev[-1] / ev[0], rel=1e-9)


@pytest.mark.parametrize("bs", [0, 1, 8, 27])
def test_zpcg_matches_dense_solve(bs):
    A = W.hermitian_diffusion3d(6, 1.5)
    b = W.rhs_complex(A.n, 0)
    r = oracle.zpcg(A, b, bs, 1e-12)
    assert r["status"] == "ok"
    D = A.to_dense()
    x_ref = np.linalg.solve(D, b)
    res = np.linalg.norm(D @ r["x"] - b) / np.linalg.norm(b)
    assert res <= 1e-12 and r["true_rel_residual"] == pytest.approx(res, rel=1e-6)
    ev = np.linalg.eigvalsh(D)
    assert np.linalg.norm(r["x"] - x_ref) <= 1e-12 * ev[-1] / ev[0] * np.linalg.norm(x_ref)


def test_complex_routines_reduce_to_the_real_ones_on_real_matrices():
    A = W.poisson2d(16)
    Az = W.CSR(A.row_ptr, A.col, A.val.astype(np.complex128))
    b = W.rhs(A.n, 0)
    rz = oracle.zpcg(Az, b.astype(np.complex128), 8, 1e-10)
    rr = oracle.pcg(A, b, 8, 1e-10)
    assert rz["iterations"] == rr["iterations"]
    assert np.allclose(rz["x"].real, rr["x"], rtol=1e-13, atol=1e-15) and not rz["x"].imag.any()
    kz = oracle.zkappa(Az, b.astype(np.complex128), 200, 8)["kappa"]
    assert kz == pytest.approx(oracle.kappa(A, b, 200, 8)["kappa"], rel=1e-12)

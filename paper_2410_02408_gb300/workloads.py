"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *prepares inputs*: it builds sparse SPD matrices in CSR form and
right-hand sides.  It holds none of the method's arithmetic (no block extraction,
factorisation, preconditioner application, Lanczos or CG).  The paper generates
"sparse, Hermitian, positive-definite matrices" of size N without saying how
(Sec. 4.2, Sec. 5.1); the recipes below stand in for them and are stated
precisely so both sides read bit-identical inputs.

Conventions
-----------
* CSR arrays: ``row_ptr`` int32 [N+1], ``col`` int32 [nnz] (sorted, unique per row,
  explicit diagonal), ``val`` float64 or float32 [nnz].
* Grids are numbered lexicographically with x fastest: p = i + n*j + n*n*k.
* Every random stream comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    """A square sparse matrix in CSR form (host numpy arrays)."""

    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.complex128 if np.iscomplexobj(self.val) else np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def _csr_from_padded(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray) -> CSR:
    """Compress an (N, w) table of candidate entries (already column-sorted per row)."""
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 indexing")
    return CSR(row_ptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask])


def rhs(n: int, seed: int = 0) -> np.ndarray:
    """b ~ N(0, 1) with ``default_rng(seed).standard_normal(n)`` (float64)."""
    return np.random.default_rng(seed).standard_normal(n)


# ---------------------------------------------------------------------------
# 2D 5-point Poisson (small plain-method workload)
# ---------------------------------------------------------------------------
def poisson2d(n: int) -> CSR:
    """5-point Laplacian on an n x n grid, Dirichlet boundary: 4 on the diagonal,
    -1 for each grid neighbour.  nnz = 5 n^2 - 4 n."""
    N = n * n
    p = np.arange(N, dtype=np.int64)
    i = p % n
    j = p // n
    cols = np.stack([p - n, p - 1, p, p + 1, p + n], axis=1)
    mask = np.stack([j > 0, i > 0, np.ones(N, bool), i < n - 1, j < n - 1], axis=1)
    vals = np.broadcast_to(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (N, 5)).copy()
    A = _csr_from_padded(cols, vals, mask)
    A.meta = {"kind": "poisson2d", "n": n}
    return A


def poisson1d(n: int) -> CSR:
    """tridiag(-1, 2, -1) of size n (Dirichlet 1D Laplacian)."""
    p = np.arange(n, dtype=np.int64)
    cols = np.stack([p - 1, p, p + 1], axis=1)
    mask = np.stack([p > 0, np.ones(n, bool), p < n - 1], axis=1)
    vals = np.broadcast_to(np.array([-1.0, 2.0, -1.0]), (n, 3)).copy()
    A = _csr_from_padded(cols, vals, mask)
    A.meta = {"kind": "poisson1d", "n": n}
    return A


# ---------------------------------------------------------------------------
# 3D 7-point variable-coefficient diffusion
# ---------------------------------------------------------------------------
def diffusion3d_faces(n: int, sigma: float, seed: int = 1):
    """Face coefficients c_f = exp(sigma * g), g ~ N(0,1) i.i.d., one per face including
    the 6 n^2 boundary faces.  Drawn in the order cx, cy, cz from one stream.

    cx[k, j, i], i in 0..n : face between cells (i-1, j, k) and (i, j, k) (i=0, n: boundary)
    cy[k, j, i], j in 0..n : face between cells (i, j-1, k) and (i, j, k)
    cz[k, j, i], k in 0..n : face between cells (i, j, k-1) and (i, j, k)
    """
    rng = np.random.default_rng(seed)
    cx = np.exp(sigma * rng.standard_normal((n, n, n + 1)))
    cy = np.exp(sigma * rng.standard_normal((n, n + 1, n)))
    cz = np.exp(sigma * rng.standard_normal((n + 1, n, n)))
    return cx, cy, cz


def diffusion3d_from_faces(n: int, cx: np.ndarray, cy: np.ndarray, cz: np.ndarray) -> CSR:
    """Assemble A from face coefficients: A_pq = -c_f for the face f shared by p and q,
    A_pp = sum of the coefficients of all six faces of p (a Dirichlet boundary face adds
    to the diagonal only).  nnz = 7 n^3 - 6 n^2."""
    N = n ** 3
    cxm = cx[:, :, :n].reshape(N)      # face on the x- side of each cell
    cxp = cx[:, :, 1:].reshape(N)      # face on the x+ side
    cym = cy[:, :n, :].reshape(N)
    cyp = cy[:, 1:, :].reshape(N)
    czm = cz[:n, :, :].reshape(N)
    czp = cz[1:, :, :].reshape(N)
    p = np.arange(N, dtype=np.int64)
    i = p % n
    j = (p // n) % n
    k = p // (n * n)
    diag = ((((cxm + cxp) + cym) + cyp) + czm) + czp
    cols = np.stack([p - n * n, p - n, p - 1, p, p + 1, p + n, p + n * n], axis=1)
    vals = np.stack([-czm, -cym, -cxm, diag, -cxp, -cyp, -czp], axis=1)
    mask = np.stack([k > 0, j > 0, i > 0, np.ones(N, bool), i < n - 1, j < n - 1, k < n - 1], axis=1)
    A = _csr_from_padded(cols, vals, mask)
    A.meta = {"kind": "diffusion3d", "n": n}
    return A


def diffusion3d(n: int, sigma: float, seed: int = 1) -> CSR:
    """3D 7-point variable-coefficient diffusion on an n^3 grid with log-normal face
    coefficients (sigma); see ``diffusion3d_faces`` for the draw order."""
    cx, cy, cz = diffusion3d_faces(n, sigma, seed)
    A = diffusion3d_from_faces(n, cx, cy, cz)
    A.meta.update({"sigma": sigma, "seed": seed})
    return A


def diffusion3d_face_edges(n: int) -> tuple:
    """The node pair of every face coefficient of ``diffusion3d_faces``, in the order
    cx.ravel(), cy.ravel(), cz.ravel(): int32 arrays (p, q) with q = -1 for a Dirichlet
    boundary face (it touches only cell p).  Face f along an axis lies between cells f-1
    and f of that axis; faces 0 and n are the boundary faces of cells 0 and n-1."""
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ps, qs = [], []
    for axis in (2, 1, 0):          # x faces (cx), y faces (cy), z faces (cz)
        shape = [n, n, n]
        shape[axis] += 1
        f = np.indices(shape)       # [k, j, i] indices of every face
        lo = f.copy()
        lo[axis] -= 1               # cell on the - side
        hi = f                      # cell on the + side
        def cell(c):
            return c[0] * n * n + c[1] * n + c[2]
        lo_ok = lo[axis] >= 0
        hi_ok = hi[axis] <= n - 1
        hi_c = np.where(hi_ok, cell(np.minimum(hi, n - 1)), -1)
        lo_c = np.where(lo_ok, cell(np.maximum(lo, 0)), -1)
        p = np.where(lo_ok, lo_c, hi_c)
        q = np.where(lo_ok & hi_ok, hi_c, -1)
        ps.append(p.ravel())
        qs.append(q.ravel())
    del k, j, i
    return np.concatenate(ps).astype(np.int32), np.concatenate(qs).astype(np.int32)


# ---------------------------------------------------------------------------
# Batched random-geometric-graph Laplacians
# ---------------------------------------------------------------------------
def morton30(pts: np.ndarray) -> np.ndarray:
    """30-bit Morton code of points in [0,1)^3 (10 bits per axis, x in the lowest bit)."""
    q = np.minimum((pts * 1024.0).astype(np.int64), 1023)
    code = np.zeros(pts.shape[0], dtype=np.int64)
    for b in range(10):
        for d in range(3):
            code |= ((q[:, d] >> b) & 1) << (3 * b + d)
    return code


def rgg_laplacian(points: np.ndarray, shift: float = 1e-3) -> CSR:
    """Unweighted graph Laplacian of the random geometric graph with radius
    r = (9 / (pi N))^(1/3) (12 expected neighbours in the interior), nodes ordered by
    30-bit Morton code, plus shift * I."""
    from scipy.spatial import cKDTree
    import scipy.sparse as sp

    N = points.shape[0]
    order = np.argsort(morton30(points), kind="stable")
    pts = points[order]
    r = (9.0 / (math.pi * N)) ** (1.0 / 3.0)
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    i = np.concatenate([pairs[:, 0], pairs[:, 1]])
    j = np.concatenate([pairs[:, 1], pairs[:, 0]])
    adj = sp.csr_matrix((np.ones(i.shape[0]), (i, j)), shape=(N, N))
    deg = np.asarray(adj.sum(axis=1)).ravel()
    L = (sp.diags(deg + shift) - adj).tocsr()
    L.sort_indices()
    A = CSR(L.indptr.astype(np.int32), L.indices.astype(np.int32), L.data.astype(np.float64))
    A.meta = {"kind": "rgg", "n": N}
    return A


@dataclass
class Batch:
    """Concatenated CSR of independent systems.  System s owns rows
    [sys_row[s], sys_row[s+1]) and nnz [sys_nnz[s], sys_nnz[s+1]); its column indices
    are local (0 .. N_s-1)."""

    row_ptr: np.ndarray   # int32 [sum N_s + 1], global nnz offsets
    col: np.ndarray       # int32 [sum nnz_s], local column indices
    val: np.ndarray       # float64
    sys_row: np.ndarray   # int64 [n_sys + 1]
    sys_nnz: np.ndarray   # int64 [n_sys + 1]
    bs: np.ndarray        # int32 [n_sys]
    systems: list         # list of CSR (host views)

    @property
    def n_sys(self) -> int:
        return len(self.systems)


def concat_batch(systems: list, bss) -> Batch:
    n_sys = len(systems)
    sys_row = np.zeros(n_sys + 1, dtype=np.int64)
    sys_nnz = np.zeros(n_sys + 1, dtype=np.int64)
    for s, A in enumerate(systems):
        sys_row[s + 1] = sys_row[s] + A.n
        sys_nnz[s + 1] = sys_nnz[s] + A.nnz
    row_ptr = np.empty(sys_row[-1] + 1, dtype=np.int64)
    for s, A in enumerate(systems):
        row_ptr[sys_row[s]:sys_row[s + 1]] = A.row_ptr[:-1].astype(np.int64) + sys_nnz[s]
    row_ptr[-1] = sys_nnz[-1]
    if sys_nnz[-1] >= 2**31:
        raise ValueError("batched nnz exceeds int32 indexing")
    col = np.concatenate([A.col for A in systems]).astype(np.int32)
    val = np.concatenate([A.val.astype(np.float64) for A in systems])
    return Batch(row_ptr.astype(np.int32), col, val, sys_row, sys_nnz,
                 np.asarray(bss, dtype=np.int32), systems)


def rgg_batch(n_sys: int = 512, seed: int = 3, n_min: float = 1e3, n_max: float = 2e5,
              block_sizes=(4, 8, 16, 32, 64)) -> Batch:
    """Independent RGG-Laplacian systems: N_s = floor(exp(U(ln n_min, ln n_max))),
    per-system block size uniform over ``block_sizes``, points U[0,1]^3; one stream
    draws sizes, then block sizes, then each system's points in order."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_sys))).astype(np.int64)
    bss = rng.choice(np.asarray(block_sizes), n_sys)
    points = [rng.random((int(N), 3)) for N in sizes]
    workers = min(len(points), os.cpu_count() or 1, 16)
    if workers > 1 and sum(p.shape[0] for p in points) >= 1_000_000:
        # the Laplacians are independent: build them on worker threads (the neighbour search
        # and the sparse assembly run in compiled code that releases the interpreter lock)
        from concurrent.futures import ThreadPoolExecutor

        with ThreadPoolExecutor(workers) as ex:
            systems = list(ex.map(rgg_laplacian, points))
    else:
        systems = [rgg_laplacian(p) for p in points]
    return concat_batch(systems, bss)


# ---------------------------------------------------------------------------
# Large power-law SPD
# ---------------------------------------------------------------------------
def _powerlaw_exponent(w_min: int, w_max: int, mean: float) -> float:
    w = np.arange(w_min, w_max + 1, dtype=np.float64)

    def m(g):
        p = w ** (-g)
        return float((w * p).sum() / p.sum())

    lo, hi = 0.0, 10.0   # mean decreases with the exponent
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if m(mid) > mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def powerlaw_spd(n: int = 8_000_000, seed: int = 5, w_min: int = 8, w_max: int = 1999,
                 mean_deg: float = 31.0, cap: int = 2000, rcm: bool = True,
                 dtype=np.float32, device=None) -> CSR:
    """Random sparse SPD with power-law row lengths.

    Expected off-diagonal degrees w_i follow a discrete power law on [w_min, w_max]
    whose exponent gives mean ``mean_deg``; edges are drawn Chung-Lu style (both ends
    proportional to w, sum(w)/2 draws), symmetrised, de-duplicated, self loops removed,
    and rows are capped at ``cap`` entries including the diagonal: an undirected edge is
    dropped when it is not among the first cap - 1 edges of either end, edges of a node
    being counted in the order (as the smaller end, by the other end), then (as the larger
    end, by the other end).  Off-diagonal values U(-1, 0) (rounded to float32), diagonal =
    sum |off| + 1e-2 formed from the rounded off-diagonals and then rounded.  Rows are
    reverse-Cuthill-McKee reordered.

    Every random number comes from ``default_rng(seed)`` on the host; the integer work (the
    inverse-CDF lookups, sorting, de-duplication, ranking and the CSR assembly) runs as
    torch operations on ``device`` (default: the GPU when one is present, else the host).
    Each of them is exact, so the matrix is the same bit for bit on either device; the
    floating-point row sums of the diagonal stay on the host (numpy, in entry order)."""
    import scipy.sparse as sp
    import torch

    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    g = _powerlaw_exponent(w_min, w_max, mean_deg)
    support = np.arange(w_min, w_max + 1, dtype=np.float64)
    pw = support ** (-g)
    pw /= pw.sum()
    w = rng.choice(support, size=n, p=pw)
    n_draw = int(round(w.sum() / 2.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf_t = torch.from_numpy(cdf).to(dev)

    def draw():
        # node of each draw: the first index whose cumulative weight exceeds u
        u = torch.from_numpy(rng.random(n_draw)).to(dev)
        return torch.searchsorted(cdf_t, u, right=True).clamp_(max=n - 1)

    a = draw()
    b = draw()
    keep = a != b
    a = a[keep]
    b = b[keep]
    del keep
    key = torch.unique(torch.minimum(a, b) * n + torch.maximum(a, b), sorted=True)
    del a, b
    lo = torch.div(key, n, rounding_mode="floor")
    hi = key - lo * n
    del key
    # cap: rank of every edge among the edges of each of its two ends (see above)
    deg_cap = cap - 1
    m_e = lo.shape[0]
    idx = torch.arange(m_e, device=dev)
    cnt_lo = torch.bincount(lo, minlength=n)
    rank_lo = idx - (torch.cumsum(cnt_lo, 0) - cnt_lo)[lo]          # lo is sorted
    hs, order_h = torch.sort(hi, stable=True)
    cnt_hi = torch.bincount(hi, minlength=n)
    occ = torch.empty_like(hi)
    occ[order_h] = idx - (torch.cumsum(cnt_hi, 0) - cnt_hi)[hs]
    rank_hi = cnt_lo[hi] + occ
    ok = (rank_lo < deg_cap) & (rank_hi < deg_cap)
    del idx, cnt_lo, rank_lo, hs, order_h, cnt_hi, occ, rank_hi
    lo = lo[ok].cpu().numpy()
    hi = hi[ok].cpu().numpy()
    del ok
    offv = (-rng.random(lo.shape[0])).astype(np.float32)
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    vals = np.concatenate([offv, offv])
    del lo, hi, offv
    absum = np.bincount(rows, weights=np.abs(vals.astype(np.float64)), minlength=n)
    diag = (absum + 1e-2).astype(np.float32)
    rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    vals = np.concatenate([vals, diag])
    del absum, diag

    def assemble(r, c, v):
        # CSR of the entries (r, c, v) with the columns of every row in increasing order
        rt = torch.from_numpy(r).to(dev)
        k = rt * n + torch.from_numpy(c).to(dev)
        k, order = torch.sort(k)
        indptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
        indptr[1:] = torch.cumsum(torch.bincount(rt, minlength=n), 0)
        del rt
        indices = (k - torch.div(k, n, rounding_mode="floor") * n).to(torch.int32)
        data = torch.from_numpy(v).to(dev)[order]
        return indptr.cpu().numpy(), indices.cpu().numpy(), data.cpu().numpy()

    indptr, indices, data = assemble(rows, cols, vals)
    if rcm:
        from scipy.sparse.csgraph import reverse_cuthill_mckee

        M = sp.csr_matrix((data, indices, indptr.astype(np.int32)), shape=(n, n))
        perm = reverse_cuthill_mckee(M, symmetric_mode=True)
        del M, indptr, indices, data
        iperm = np.empty(n, dtype=np.int64)
        iperm[perm] = np.arange(n, dtype=np.int64)
        indptr, indices, data = assemble(iperm[rows], iperm[cols], vals)
    if indptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 indexing")
    A = CSR(indptr.astype(np.int32), indices, data.astype(dtype))
    A.meta = {"kind": "powerlaw", "n": n, "exponent": g, "seed": seed}
    return A


def random_spd(n: int, mean_deg: float, seed: int = 11, dtype=np.float64) -> CSR:
    """The paper-size random SPD family (the paper draws "sparse, Hermitian, positive-definite
    matrices" of N = 2^10, 2^12, 2^14 with varying sparsity, Sec. 4.2 and 5.1, without a recipe):
    the power-law recipe of ``powerlaw_spd`` (Chung-Lu edges, U(-1, 0) off-diagonals, diagonal
    = row |sum| + 1e-2, reverse Cuthill-McKee order) with expected degrees on
    [2, max(mean_deg + 1, min(1999, n // 4))] and mean ``mean_deg``."""
    w_max = int(max(mean_deg + 1, min(1999, n // 4)))
    A = powerlaw_spd(n, seed=seed, w_min=2, w_max=w_max, mean_deg=float(mean_deg), cap=min(2000, n), dtype=dtype)
    A.meta.update({"kind": "random_spd", "mean_deg": mean_deg})
    return A


# ---------------------------------------------------------------------------
# Complex Hermitian positive definite (Sec. 3.1 allows Hermitian A)
# ---------------------------------------------------------------------------
def magnetic_laplacian_1d(n: int, theta: float) -> CSR:
    """Path graph with a constant vector potential: A_ii = 2, A_{i,i+1} = -e^{i theta},
    A_{i+1,i} = -e^{-i theta}, Dirichlet ends (complex128 values).  It is unitarily similar to
    tridiag(-1, 2, -1) (gauge transform diag(e^{i k theta})), so its eigenvalues are
    2 - 2 cos(k pi / (n + 1))."""
    p = np.arange(n, dtype=np.int64)
    cols = np.stack([p - 1, p, p + 1], axis=1)
    mask = np.stack([p > 0, np.ones(n, bool), p < n - 1], axis=1)
    e = np.exp(1j * theta)
    vals = np.broadcast_to(np.array([-np.conj(e), 2.0 + 0j, -e]), (n, 3)).copy()
    A = _csr_from_padded(cols, vals, mask)
    A.meta = {"kind": "magnetic1d", "n": n, "theta": theta}
    return A


def magnetic_laplacian_2d(n: int, flux: float) -> CSR:
    """Magnetic 5-point Laplacian on an n x n grid (Dirichlet boundary) in the Landau gauge:
    hops along x carry no phase, a hop from (i, j) to (i, j+1) carries e^{2 pi i flux i}, so every
    plaquette encloses the flux `flux` (in flux quanta).  A_pp = 4, A_pq = -(hop phase), A_qp =
    conj(A_pq); Hermitian positive definite (complex128 values)."""
    N = n * n
    p = np.arange(N, dtype=np.int64)
    i = p % n
    j = p // n
    ph = np.exp(2j * np.pi * flux * i)          # phase of the hop p -> p + n (j -> j + 1)
    cols = np.stack([p - n, p - 1, p, p + 1, p + n], axis=1)
    mask = np.stack([j > 0, i > 0, np.ones(N, bool), i < n - 1, j < n - 1], axis=1)
    vals = np.stack([-np.conj(ph), -np.ones(N), 4.0 * np.ones(N), -np.ones(N), -ph], axis=1).astype(np.complex128)
    A = _csr_from_padded(cols, vals, mask)
    A.meta = {"kind": "magnetic2d", "n": n, "flux": flux}
    return A


def hermitian_diffusion3d(n: int, sigma: float, seed: int = 1, phase_seed: int = 2) -> CSR:
    """The 3D variable-coefficient diffusion stencil of ``diffusion3d`` (same face coefficients)
    with a random U(1) phase on every interior face: A_pq = -c_f e^{i phi_f}, A_qp = conj(A_pq)
    for p < q, phi_f ~ U(-pi, pi) from ``default_rng(phase_seed)`` (drawn for the faces in the
    order cx, cy, cz), A_pp = sum of the coefficients of the six faces of p (Dirichlet faces on
    the diagonal only).  Hermitian positive definite (complex128 values)."""
    cx, cy, cz = diffusion3d_faces(n, sigma, seed)
    rng = np.random.default_rng(phase_seed)
    px = np.exp(1j * rng.uniform(-np.pi, np.pi, cx.shape))
    py = np.exp(1j * rng.uniform(-np.pi, np.pi, cy.shape))
    pz = np.exp(1j * rng.uniform(-np.pi, np.pi, cz.shape))
    N = n ** 3
    cxm, cxp = cx[:, :, :n].reshape(N), cx[:, :, 1:].reshape(N)
    cym, cyp = cy[:, :n, :].reshape(N), cy[:, 1:, :].reshape(N)
    czm, czp = cz[:n, :, :].reshape(N), cz[1:, :, :].reshape(N)
    # phase of the face on each side, seen from the lower-index cell of the pair
    pxm, pxp = px[:, :, :n].reshape(N), px[:, :, 1:].reshape(N)
    pym, pyp = py[:, :n, :].reshape(N), py[:, 1:, :].reshape(N)
    pzm, pzp = pz[:n, :, :].reshape(N), pz[1:, :, :].reshape(N)
    p = np.arange(N, dtype=np.int64)
    i = p % n
    j = (p // n) % n
    k = p // (n * n)
    diag = ((((cxm + cxp) + cym) + cyp) + czm) + czp
    # entry (p, q) for q > p is -c e^{i phi}; for q < p it is the conjugate of entry (q, p)
    cols = np.stack([p - n * n, p - n, p - 1, p, p + 1, p + n, p + n * n], axis=1)
    vals = np.stack([-czm * np.conj(pzm), -cym * np.conj(pym), -cxm * np.conj(pxm), diag + 0j,
                     -cxp * pxp, -cyp * pyp, -czp * pzp], axis=1)
    mask = np.stack([k > 0, j > 0, i > 0, np.ones(N, bool), i < n - 1, j < n - 1, k < n - 1], axis=1)
    A = _csr_from_padded(cols, vals, mask)
    A.meta = {"kind": "hermitian_diffusion3d", "n": n, "sigma": sigma, "seed": seed, "phase_seed": phase_seed}
    return A


def rhs_complex(n: int, seed: int = 0) -> np.ndarray:
    """b with independent N(0, 1) real and imaginary parts: ``default_rng(seed).standard_normal(2n)``
    taken as interleaved (re, im) pairs."""
    return np.random.default_rng(seed).standard_normal(2 * n).view(np.complex128).copy()


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
def workload(name: str):
    """Named synthetic workloads: returns (A, b)."""
    if name == "poisson2d_64":
        A = poisson2d(64)
    elif name.startswith("diffusion3d_"):
        # diffusion3d_<n>_s<sigma>
        parts = name.split("_")
        A = diffusion3d(int(parts[1]), float(parts[2][1:]))
    else:
        raise KeyError(name)
    return A, rhs(A.n, 0)

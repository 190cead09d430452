// Block-Jacobi setup of one warp unit (Sec. 3.2-3.3): extract the unit's diagonal blocks
// A_kk from CSR and factor them, A_kk = L_k L_k^T, then form L_k^{-1} and
// M_k^{-1} = L_k^{-T} L_k^{-1}.
//
// The calling warp owns the unit.  Its blocks sit in shared memory as dense rows (row
// stride bs+1; As holds A then L, Xs holds L^{-1}): lane l owns unit row l (and l+32 for
// blocks of 33..64 rows).  Extraction, the right-looking Cholesky (lanes = rows, lockstep
// over the pivot column), the triangular inverse (lanes = columns, independent) and the
// products for M^{-1} all run from shared memory; the results are written straight into
// the coalesced unit layouts used by the apply kernels.
#pragma once

#include "pc_common.cuh"

namespace pc {

// Shared memory one warp needs: As and Xs, U rows of bs+1 entries each.
__host__ __device__ inline size_t setup_unit_smem(const Layout& L, size_t ft_bytes) {
  return (size_t)2 * L.U * (L.bs + 1) * ft_bytes;
}

// rp/ci/va: CSR whose row r of this layout is rp[r]..rp[r+1]-1 and whose column indices
// are relative to the same origin as the rows.  Mu (and Lu unless null) point at this
// unit's slots of the factor arrays.  A pivot <= tol * (largest diagonal entry of its
// block) makes the block count as failed: atomicMin(failed, block index); the pivot is
// then replaced by 1 so that the factor stays finite.  FT is the arithmetic type (and the
// type of the shared-memory tiles), ST the stored type (FP64 arithmetic can be stored as
// FP32 factors).
template <typename VT, typename FT, typename ST = FT>
__device__ __forceinline__ void setup_unit(const Layout& L, int64_t u, const int32_t* __restrict__ rp,
                                           const int32_t* __restrict__ ci, const VT* __restrict__ va, double tol,
                                           ST* __restrict__ Mu, ST* __restrict__ Lu, FT* As, FT* Xs, int lane,
                                           unsigned long long* failed) {
  const int bs = L.bs;
  const int ld = bs + 1;
  const int64_t urow0 = u * L.U;
  // ---- zero, then extract (identity on rows past n)
  for (int t = lane; t < L.U * ld; t += 32) {
    As[t] = FT(0);
    Xs[t] = FT(0);
  }
  __syncwarp();
  for (int s = 0; s < L.S; ++s) {
    const int rho = lane + 32 * s;
    if (rho >= L.U) continue;
    const int i = rho % bs;
    const int64_t row = urow0 + rho;
    if (row < L.n) {
      const int64_t bstart = row - i;
      const int32_t e0 = rp[row], e1 = rp[row + 1];
      for (int32_t e = e0; e < e1; ++e) {
        const int64_t c = ci[e];
        if (c >= bstart && c < bstart + bs) As[rho * ld + (int)(c - bstart)] = (FT)va[e];
      }
    } else {
      As[rho * ld + i] = FT(1);
    }
  }
  __syncwarp();
  // ---- per-block pivot scale: max diagonal entry of the block
  FT dmax[2] = {FT(0), FT(0)};
  for (int s = 0; s < L.S; ++s) {
    const int rho = lane + 32 * s;
    if (rho >= L.U) continue;
    const int gb = rho - rho % bs;
    FT m = FT(0);
    for (int t = 0; t < bs; ++t)
      if (urow0 + gb + t < L.n) m = max(m, As[(gb + t) * ld + t]);
    dmax[s] = m;
  }
  // ---- right-looking Cholesky, lanes = rows
  for (int j = 0; j < bs; ++j) {
    for (int s = 0; s < L.S; ++s) {
      const int rho = lane + 32 * s;
      if (rho >= L.U) continue;
      if (rho % bs == j) {
        FT d = As[rho * ld + j];
        if (urow0 + rho < L.n && (!(d > FT(tol) * dmax[s]) || !isfinite((double)d))) {
          const unsigned long long blk = (unsigned long long)((urow0 + rho) / bs);
          atomicMin(failed, blk);
          d = FT(1);
        }
        As[rho * ld + j] = sqrt(d);
      }
    }
    __syncwarp();
    for (int s = 0; s < L.S; ++s) {
      const int rho = lane + 32 * s;
      if (rho >= L.U) continue;
      const int i = rho % bs;
      if (i > j) {
        const int gb = rho - i;
        As[rho * ld + j] = As[rho * ld + j] / As[(gb + j) * ld + j];
      }
    }
    __syncwarp();
    for (int s = 0; s < L.S; ++s) {
      const int rho = lane + 32 * s;
      if (rho >= L.U) continue;
      const int i = rho % bs;
      if (i > j) {
        const int gb = rho - i;
        const FT lij = As[rho * ld + j];
        for (int k = j + 1; k <= i; ++k) As[rho * ld + k] = fma(-lij, As[(gb + k) * ld + j], As[rho * ld + k]);
      }
    }
    __syncwarp();
  }
  // ---- X = L^{-1}: lane owns column c = its row index in the block
  for (int s = 0; s < L.S; ++s) {
    const int rho = lane + 32 * s;
    if (rho >= L.U) continue;
    const int c = rho % bs;
    const int gb = rho - c;
    for (int i = c; i < bs; ++i) {
      FT acc = (i == c) ? FT(1) : FT(0);
      for (int k = c; k < i; ++k) acc = fma(-As[(gb + i) * ld + k], Xs[(gb + k) * ld + c], acc);
      Xs[(gb + i) * ld + c] = acc / As[(gb + i) * ld + i];
    }
  }
  __syncwarp();
  // ---- M^{-1} (circulant rows) and L^{-1} (by diagonals), coalesced unit stores
  for (int s = 0; s < L.S; ++s) {
    const int rho = lane + 32 * s;
    const bool valid = rho < L.U;
    const int i = valid ? rho % bs : 0;
    const int gb = valid ? rho - i : 0;
    for (int k = 0; k <= L.K; ++k) {
      FT acc = FT(0);
      if (valid) {
        int j = i + k;
        if (j >= bs) j -= bs;
        const int m0 = i > j ? i : j;
        for (int m = m0; m < bs; ++m) acc = fma(Xs[(gb + m) * ld + i], Xs[(gb + m) * ld + j], acc);
      }
      Mu[(k * L.S + s) * 32 + lane] = (ST)acc;
    }
    if (Lu) {
      for (int k = 0; k < bs; ++k) {
        const FT v = (valid && i >= k) ? Xs[rho * ld + (i - k)] : FT(0);
        Lu[(k * L.S + s) * 32 + lane] = (ST)v;
      }
    }
  }
  __syncwarp();
}

}  // namespace pc

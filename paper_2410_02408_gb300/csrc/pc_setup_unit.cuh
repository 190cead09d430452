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

// ------------------------------------------------------------------ tensor cores (TF32)
// TF32 operand: the FP32 value rounded to 10 mantissa bits, to nearest with ties away from
// zero (cvt.rna), in a 32-bit register.
__device__ __forceinline__ uint32_t tf32_rna(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

// d += a * b on the tensor cores: a is 16x8 (row major), b is 8x8 (column major), TF32
// operands, FP32 accumulation (one warp, all lanes converged).  Fragments, with
// g = lane / 4 and t = lane % 4:
//   a[0] = A(g, t)     a[1] = A(g + 8, t)     a[2] = A(g, t + 4)     a[3] = A(g + 8, t + 4)
//   b[0] = B(t, g)     b[1] = B(t + 4, g)
//   d[0] = D(g, 2t)    d[1] = D(g, 2t + 1)    d[2] = D(g + 8, 2t)    d[3] = D(g + 8, 2t + 1)
__device__ __forceinline__ void mma_tf32_m16n8k8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// M = X^T X for the bs x bs lower-triangular X = L^{-1} of one block held in shared memory
// (X(m, c) at Xb[m * ld + c], zero above the diagonal), on the tensor cores: 16 x 8 output tiles,
// k in steps of 8, TF32 operands, FP32 accumulation.  M(i, j) is written to Mb[i * ld + j].
// Called by a full warp (warp-uniform loops).
__device__ __forceinline__ void gram_tf32(const float* Xb, float* Mb, int bs, int ld, int lane) {
  const int g = lane >> 2, t = lane & 3;
  auto xat = [&](int m, int c) -> float { return (m < bs && c < bs) ? Xb[m * ld + c] : 0.0f; };
  for (int i0 = 0; i0 < bs; i0 += 16) {
    for (int j0 = 0; j0 < bs; j0 += 8) {
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      // X is lower triangular: M(i, j) = sum over m >= max(i, j); k tiles below that are zero
      const int kstart = (max(i0, j0) / 8) * 8;
      for (int k0 = kstart; k0 < bs; k0 += 8) {
        uint32_t a[4], b[2];
        a[0] = tf32_rna(xat(k0 + t, i0 + g));          // A(i, m) = X(m, i)
        a[1] = tf32_rna(xat(k0 + t, i0 + g + 8));
        a[2] = tf32_rna(xat(k0 + t + 4, i0 + g));
        a[3] = tf32_rna(xat(k0 + t + 4, i0 + g + 8));
        b[0] = tf32_rna(xat(k0 + t, j0 + g));          // B(m, j) = X(m, j)
        b[1] = tf32_rna(xat(k0 + t + 4, j0 + g));
        mma_tf32_m16n8k8(d, a, b);
      }
      const int r0 = i0 + g, r1 = i0 + g + 8, c0 = j0 + 2 * t, c1 = j0 + 2 * t + 1;
      if (r0 < bs && c0 < bs) Mb[r0 * ld + c0] = d[0];
      if (r0 < bs && c1 < bs) Mb[r0 * ld + c1] = d[1];
      if (r1 < bs && c0 < bs) Mb[r1 * ld + c0] = d[2];
      if (r1 < bs && c1 < bs) Mb[r1 * ld + c1] = d[3];
    }
  }
}

// Shared memory one warp needs: As and Xs, U rows of bs+1 entries each.
__host__ __device__ inline size_t setup_unit_smem(const Layout& L, size_t ft_bytes) {
  return (size_t)2 * L.U * (L.bs + 1) * ft_bytes;
}

// Zero the unit's tiles (As, and Xs unless null), then extract its diagonal blocks from CSR
// into As (dense rows, stride bs + 1; the identity on rows past n).  The row's columns
// increase (every entry point checks the CSR first): binary-search the first column of the
// block, then copy until its last, so that a long row costs O(log length + bs) instead of its
// length.
template <typename VT, typename FT>
__device__ __forceinline__ void extract_unit(const Layout& L, int64_t urow0, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci, const VT* __restrict__ va, FT* As,
                                             FT* Xs, int lane) {
  const int bs = L.bs;
  const int ld = bs + 1;
  for (int t = lane; t < L.U * ld; t += 32) {
    As[t] = FT(0);
    if (Xs) Xs[t] = FT(0);
  }
  __syncwarp();
  for (int s = 0; s < L.S; ++s) {
    const int rho = lane + 32 * s;
    if (rho >= L.U) continue;
    const int i = rho % bs;
    const int64_t row = urow0 + rho;
    if (row < L.n) {
      const int64_t bstart = row - i;
      const int32_t e1 = rp[row + 1];
      int32_t lo = rp[row], hi = e1;
      while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)ci[mid] < bstart) lo = mid + 1;
        else hi = mid;
      }
      for (int32_t e = lo; e < e1; ++e) {
        const int64_t c = ci[e];
        if (c >= bstart + bs) break;
        As[rho * ld + (int)(c - bstart)] = (FT)va[e];
      }
    } else {
      As[rho * ld + i] = FT(1);
    }
  }
  __syncwarp();
}

// rp/ci/va: CSR whose row r of this layout is rp[r]..rp[r+1]-1 and whose column indices
// are relative to the same origin as the rows, strictly increasing within each row.  Mu
// (and Lu unless null) point at this unit's slots of the factor arrays.  A pivot <= tol *
// (largest diagonal entry of its block) makes the block count as failed: atomicMin(failed,
// block index); the pivot is then replaced by 1 so that the factor stays finite.  FT is the
// arithmetic type (and the type of the shared-memory tiles), ST the stored type (FP64
// arithmetic can be stored as FP32 factors).  TC (FP32 only): M^{-1} = L^{-T} L^{-1} is formed
// on the tensor cores from TF32-rounded L^{-1} with FP32 accumulation (gram_tf32) instead of
// FP32 dot products.
template <typename VT, typename FT, typename ST = FT, bool TC = false>
__device__ __forceinline__ void setup_unit(const Layout& L, int64_t u, const int32_t* __restrict__ rp,
                                           const int32_t* __restrict__ ci, const VT* __restrict__ va, double tol,
                                           ST* __restrict__ Mu, ST* __restrict__ Lu, FT* As, FT* Xs, int lane,
                                           unsigned long long* failed) {
  const int bs = L.bs;
  const int ld = bs + 1;
  const int64_t urow0 = u * L.U;
  extract_unit<VT, FT>(L, urow0, rp, ci, va, As, Xs, lane);
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
#pragma unroll 4
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
#pragma unroll 4
      for (int k = c; k < i; ++k) acc = fma(-As[(gb + i) * ld + k], Xs[(gb + k) * ld + c], acc);
      Xs[(gb + i) * ld + c] = acc / As[(gb + i) * ld + i];
    }
  }
  __syncwarp();
  if constexpr (TC) {
    // M^{-1} of every block of the unit into As (L is no longer needed)
    static_assert(sizeof(FT) == 4, "tensor-core setup is FP32 arithmetic");
    for (int gb = 0; gb < L.U; gb += bs) gram_tf32(Xs + gb * ld, As + gb * ld, bs, ld, lane);
    __syncwarp();
  }
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
        if constexpr (TC) {
          // always the entry on or above the diagonal, so that the two stored copies of the
          // pair at distance bs/2 (even bs) are the same bits
          acc = As[(gb + min(i, j)) * ld + max(i, j)];
        } else {
          const int m0 = i > j ? i : j;
#pragma unroll 4
          for (int m = m0; m < bs; ++m) acc = fma(Xs[(gb + m) * ld + i], Xs[(gb + m) * ld + j], acc);
        }
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

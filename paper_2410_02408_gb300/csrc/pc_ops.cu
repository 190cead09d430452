// Stand-alone operators: CSR SpMV, fixed-order dot product, block preconditioner
// application (M^{-1}, L^{-1}, L^{-T}), the second phase of the symmetric operator
// L^{-1} A L^{-T} (SpMV with a fused per-unit L^{-1} epilogue), the SpMV row split of
// the persistent CG kernel, the adjoint gradient on the sparsity pattern, the O(nnz)
// structure check of a CSR matrix, and the block residual of the refined preconditioner apply.
#include "pc_kernels.cuh"
#include "pc_setup_unit.cuh"

namespace pc {

// One tensor-core product D = A B (A 16x8, B 8x8, row-major in global memory), operands
// rounded to TF32, FP32 accumulation: the fragment mapping of mma_tf32_m16n8k8, for checks.
__global__ void mma_tf32_check_kernel(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ D) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  uint32_t a[4], b[2];
  a[0] = tf32_rna(A[g * 8 + t]);
  a[1] = tf32_rna(A[(g + 8) * 8 + t]);
  a[2] = tf32_rna(A[g * 8 + t + 4]);
  a[3] = tf32_rna(A[(g + 8) * 8 + t + 4]);
  b[0] = tf32_rna(B[t * 8 + g]);
  b[1] = tf32_rna(B[(t + 4) * 8 + g]);
  float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  mma_tf32_m16n8k8(d, a, b);
  D[g * 8 + 2 * t] = d[0];
  D[g * 8 + 2 * t + 1] = d[1];
  D[(g + 8) * 8 + 2 * t] = d[2];
  D[(g + 8) * 8 + 2 * t + 1] = d[3];
}

cudaError_t launch_mma_tf32_check(const float* A, const float* B, float* D, cudaStream_t st) {
  mma_tf32_check_kernel<<<1, 32, 0, st>>>(A, B, D);
  return cudaGetLastError();
}

// CSR structure check, one thread per row: the row's range must lie inside [0, nnz] and not
// decrease, and its columns must lie in [0, n), increase strictly and include the row
// itself.  Only row_ptr[0..n] and col[0..nnz) are read; nothing is gathered through a
// column index.  Violations are OR-ed into *flags (CSR_BAD_* bits).
__global__ void __launch_bounds__(256) validate_csr_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ ci, unsigned* flags) {
  unsigned f = 0u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e0 = __ldg(rp + i), e1 = __ldg(rp + i + 1);
    if (e0 < 0 || e1 < e0 || (int64_t)e1 > nnz) {
      f |= CSR_BAD_ROW_PTR;
      continue;
    }
    int64_t prev = -1;
    bool diag = false;
    for (int32_t e = e0; e < e1; ++e) {
      const int64_t c = __ldg(ci + e);
      if (c < 0 || c >= n) f |= CSR_BAD_COLUMN;
      if (c <= prev) f |= CSR_BAD_ORDER;
      diag = diag || c == i;
      prev = c;
    }
    if (!diag) f |= CSR_NO_DIAGONAL;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (__ldg(rp) != 0 || (int64_t)__ldg(rp + n) != nnz)) f |= CSR_BAD_ROW_PTR;
  f = __reduce_or_sync(FULL, f);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

// The integer-pipe float <-> double conversions of the mixed-precision kernels, element by
// element (full warps: the helpers vote on their rare hardware fallback).
__global__ void __launch_bounds__(256) convert_kernel(int64_t n, const double* __restrict__ in_d,
                                                      float* __restrict__ out_f, const float* __restrict__ in_f,
                                                      double* __restrict__ out_d) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < n;
    const float f = d2f(ok ? in_d[i] : 0.0);
    const double d = f2d(ok ? in_f[i] : 0.0f);
    if (ok) {
      out_f[i] = f;
      out_d[i] = d;
    }
  }
}

cudaError_t launch_convert(int64_t n, const double* in_d, float* out_f, const float* in_f, double* out_d,
                           cudaStream_t st) {
  const int64_t want = (n + 255) / 256;
  convert_kernel<<<(int)(want < 1024 ? (want > 0 ? want : 1) : 1024), 256, 0, st>>>(n, in_d, out_f, in_f, out_d);
  return cudaGetLastError();
}

cudaError_t launch_validate_csr(int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci, unsigned* flags,
                                cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int grid = (int)(want < (int64_t)(sms > 0 ? sms : 1) * 8 ? want : (int64_t)(sms > 0 ? sms : 1) * 8);
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  validate_csr_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(n, nnz, rp, ci, flags);
  return cudaGetLastError();
}

// d = r - blockdiag(A) z: each row's sum runs over its stored entries whose column lies in the
// row's own diagonal block [k bs, min((k + 1) bs, n)) (one FMA chain in storage order), in FP64
// from the CSR values (float values widened exactly).
template <typename VT>
__global__ void __launch_bounds__(256) block_residual_kernel(int64_t n, int32_t bs, const int32_t* __restrict__ rp,
                                                             const int32_t* __restrict__ ci, const VT* __restrict__ va,
                                                             const double* __restrict__ r, const double* __restrict__ z,
                                                             double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c0 = (i / bs) * bs, c1 = c0 + bs < n ? c0 + bs : n;
    double s = 0.0;
    for (int32_t e = __ldg(rp + i), e1 = __ldg(rp + i + 1); e < e1; ++e) {
      const int64_t c = __ldg(ci + e);
      if (c >= c0 && c < c1) s = fma((double)__ldg(va + e), z[c], s);
    }
    d[i] = r[i] - s;
  }
}

__global__ void __launch_bounds__(256) add_kernel(int64_t n, const double* __restrict__ e, double* __restrict__ z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += e[i];
}

static int grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  const int64_t want = (n + 255) / 256;
  return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

cudaError_t launch_block_residual(int64_t n, int32_t bs, const int32_t* rp, const int32_t* ci, const void* va,
                                  bool val_f32, const double* r, const double* z, double* d, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (val_f32)
    block_residual_kernel<float><<<grid_for(n), 256, 0, st>>>(n, bs, rp, ci, (const float*)va, r, z, d);
  else
    block_residual_kernel<double><<<grid_for(n), 256, 0, st>>>(n, bs, rp, ci, (const double*)va, r, z, d);
  return cudaGetLastError();
}

cudaError_t launch_add(int64_t n, const double* e, double* z, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  add_kernel<<<grid_for(n), 256, 0, st>>>(n, e, z);
  return cudaGetLastError();
}

template <typename VT>
__global__ void __launch_bounds__(256) spmv_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const VT* __restrict__ va, const double* __restrict__ x,
                                                   double* __restrict__ y) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x)
    y[row] = spmv_row<VT, false>(rp, ci, va, x, row);
}

constexpr int DOT_CTAS = 512;
int dot_partials() { return DOT_CTAS + 1; }

__global__ void __launch_bounds__(256) dot_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                                  double* part, unsigned* counter, double* out) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  last_cta_sum1(acc, part, counter, out);
}

template <typename FT>
__global__ void __launch_bounds__(256) apply_kernel(Layout L, const FT* __restrict__ fac, int mode,
                                                    const double* __restrict__ in, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t uM = unit_elems_minv(L), uL = unit_elems_linv(L);
  for (int64_t u = gw; u < L.n_units; u += tw) {
    double r[2], z[2];
    int64_t rows[2];
    bool ok[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      bool valid;
      const int rho = unit_row(L, lane, s, valid);
      rows[s] = u * L.U + rho;
      ok[s] = valid && rows[s] < L.n;
      r[s] = ok[s] ? in[rows[s]] : 0.0;
    }
    if (mode == 0) unit_apply_inv<FT, 0>(L, fac + u * uM, lane, r, z);
    else if (mode == 2) unit_apply_linv<FT>(L, fac + u * uL, lane, r, z);
    else unit_apply_ltinv<FT>(L, fac + u * uL, lane, r, z);
#pragma unroll
    for (int s = 0; s < 2; ++s)
      if (ok[s]) out[rows[s]] = z[s];
  }
}

// out = L^{-1} (A t).  With a Lanczos epilogue: out = L^{-1} A t - beta[j-1] q_prev and
// alpha[j] = q_cur . out (fixed-order grid sum).
template <typename VT, typename FT>
__global__ void __launch_bounds__(256) sym_phase2_kernel(SymPhase2Args a) {
  if (a.done && *(volatile const int*)a.done) return;
  const Layout L = a.lay;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t uL = unit_elems_linv(L);
  const VT* va = (const VT*)a.va;
  const FT* fac = (const FT*)a.linv;
  const bool epi = a.q_cur != nullptr;
  const double bprev = (epi && a.j > 0) ? a.beta[a.j - 1] : 0.0;
  double acc = 0.0;
  for (int64_t u = gw; u < L.n_units; u += tw) {
    double uu[2], y[2];
    int64_t rows[2];
    bool ok[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      bool valid;
      const int rho = unit_row(L, lane, s, valid);
      rows[s] = u * L.U + rho;
      ok[s] = valid && rows[s] < L.n;
      uu[s] = ok[s] ? spmv_row<VT, false>(a.rp, a.ci, va, a.t, rows[s]) : 0.0;
    }
    unit_apply_linv<FT>(L, fac + u * uL, lane, uu, y);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (!ok[s]) continue;
      double w = y[s];
      if (epi) {
        if (a.j > 0) w = fma(-bprev, a.q_prev[rows[s]], w);
        acc = fma(a.q_cur[rows[s]], w, acc);
      }
      a.out[rows[s]] = w;
    }
  }
  if (epi) last_cta_sum1(acc, a.part, a.counter, a.alpha_out);
}

__global__ void split_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ rp, int parts, int64_t* split) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= parts; c += gridDim.x * blockDim.x) {
    if (c == parts) {
      split[c] = n;
      continue;
    }
    const long double tgt = (long double)c * (long double)(n + nnz) / parts;
    int64_t lo = 0, hi = n;   // smallest r with r + rp[r] >= tgt
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if ((long double)(mid + rp[mid]) >= tgt) hi = mid;
      else lo = mid + 1;
    }
    split[c] = lo;
  }
}

__global__ void grad_val_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ lam, const double* __restrict__ x, double* __restrict__ g) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    const double l = -lam[row];
    for (int32_t e = rp[row]; e < rp[row + 1]; ++e) g[e] = l * x[ci[e]];
  }
}

// dL/dc_e for A = sum_e c_e (e_p - e_q)(e_p - e_q)^T + sum_f c_f e_p e_p^T: the rank-one
// dA/dc_e turns -lambda^T (dA/dc_e) x into -(lambda_p - lambda_q)(x_p - x_q), or -lambda_p x_p
// for a boundary face (q < 0).  An edge whose node index is out of range gets NaN and no
// vector is read for it.
__global__ void grad_edges_kernel(int64_t n_edges, const int32_t* __restrict__ ep, const int32_t* __restrict__ eq,
                                  const double* __restrict__ lam, const double* __restrict__ x, int64_t n,
                                  double* __restrict__ g) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = __ldg(ep + e);
    const int32_t q = __ldg(eq + e);
    if (p < 0 || p >= n || q >= n) {
      g[e] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const double lp = __ldg(lam + p), xp = __ldg(x + p);
    if (q < 0) {
      g[e] = -(lp * xp);
    } else {
      const double dl = lp - __ldg(lam + q);
      const double dx = xp - __ldg(x + q);
      g[e] = -(dl * dx);
    }
  }
}

// ------------------------------------------------------------------ launchers
static unsigned grid_for(int64_t work, int per) {
  int64_t g = (work + per - 1) / per;
  const int64_t gmax = (int64_t)device_sms() * 64;
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  return (unsigned)g;
}

cudaError_t launch_spmv(int64_t n, const int32_t* rp, const int32_t* ci, const void* va, bool val_f32,
                        const double* x, double* y, cudaStream_t st) {
  if (val_f32)
    spmv_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, (const float*)va, x, y);
  else
    spmv_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, (const double*)va, x, y);
  return cudaGetLastError();
}

// part: dot_partials() doubles of scratch; the last slot is used as the arrival counter.
cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* result, double* part, cudaStream_t st) {
  unsigned* counter = reinterpret_cast<unsigned*>(part + DOT_CTAS);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  dot_kernel<<<DOT_CTAS, 256, 0, st>>>(n, x, y, part, counter, result);
  return cudaGetLastError();
}

cudaError_t launch_apply(const Layout& L, const void* fac, bool fac_f32, int mode, const double* in, double* out,
                         cudaStream_t st) {
  const unsigned g = grid_for(L.n_units * 32, 256);
  if (fac_f32)
    apply_kernel<float><<<g, 256, 0, st>>>(L, (const float*)fac, mode, in, out);
  else
    apply_kernel<double><<<g, 256, 0, st>>>(L, (const double*)fac, mode, in, out);
  return cudaGetLastError();
}

cudaError_t launch_sym_phase2(const SymPhase2Args& a, bool val_f32, bool fac_f32, int grid, cudaStream_t st) {
  const unsigned g = grid > 0 ? (unsigned)grid : grid_for(a.lay.n_units * 32, 256);
  if (!val_f32 && !fac_f32) sym_phase2_kernel<double, double><<<g, 256, 0, st>>>(a);
  else if (!val_f32 && fac_f32) sym_phase2_kernel<double, float><<<g, 256, 0, st>>>(a);
  else if (val_f32 && fac_f32) sym_phase2_kernel<float, float><<<g, 256, 0, st>>>(a);
  else sym_phase2_kernel<float, double><<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_split(int64_t n, int64_t nnz, const int32_t* rp, int parts, int64_t* split, cudaStream_t st) {
  split_kernel<<<(parts + 256) / 256, 256, 0, st>>>(n, nnz, rp, parts, split);
  return cudaGetLastError();
}

cudaError_t launch_grad_val(int64_t n, const int32_t* rp, const int32_t* ci, const double* lam, const double* x,
                            double* g, cudaStream_t st) {
  grad_val_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, lam, x, g);
  return cudaGetLastError();
}

cudaError_t launch_grad_edges(int64_t n_edges, const int32_t* ep, const int32_t* eq, const double* lam,
                              const double* x, int64_t n, double* g, cudaStream_t st) {
  if (n_edges == 0) return cudaSuccess;
  grad_edges_kernel<<<grid_for(n_edges, 256), 256, 0, st>>>(n_edges, ep, eq, lam, x, n, g);
  return cudaGetLastError();
}

}  // namespace pc

// Lanczos estimate of kappa = theta_max / theta_min (Sec. 3.1) for A or for the
// block-Jacobi preconditioned operator L^{-1} A L^{-T}.
//
// Step j (q_j = V[j]):
//   op      w = Op q_j - beta_{j-1} q_{j-1};  alpha_j = q_j . w            (fused epilogue)
//   pass 0  w -= alpha_j q_j;  c1 = V[0..j]^T w                             (one read of V)
//   pass 1  w -= V c1;         c2 = V[0..j]^T w                             (one read of V)
//   pass 2  w -= V c2;         beta_j = ||w||; stop test                    (one read of V)
//   norm    q_{j+1} = w / beta_j
// (classical Gram-Schmidt applied twice = CGS2).  Each reorthogonalisation kernel walks
// the columns in tiles of 32: the (j+1) x 32 tile of V is staged once in shared memory and
// serves both the update and the new coefficients.  All grid sums finish in the last CTA
// in a fixed order.  Every kernel returns immediately once the stop flag is set, so the
// host can enqueue steps without reading it back.
#include "pc_kernels.cuh"

namespace pc {

constexpr int LZ_TW = 32;

// Ampere-style asynchronous 8-byte copy global -> shared (cache at all levels), with
// commit / wait of this thread's groups.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(256) lz_sumsq_kernel(LanczosState s, const double* __restrict__ v) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(v[i], v[i], acc);
  last_cta_sum1(acc, s.part, s.counter, s.coef);
}

__global__ void __launch_bounds__(256) lz_start_kernel(LanczosState s, const double* __restrict__ v) {
  const double nrm = sqrt(s.coef[0]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
    s.V[i] = v[i] / nrm;
}

template <typename FT>
__global__ void __launch_bounds__(256) lz_ltinv_kernel(LanczosState s, Layout L, const FT* __restrict__ fac, int j,
                                                       int mode) {
  if (*(volatile const int*)s.ctl) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t uL = unit_elems_linv(L);
  const double* in = s.V + (int64_t)j * s.n;
  for (int64_t u = gw; u < L.n_units; u += tw) {
    double r[2], z[2];
    int64_t rows[2];
    bool ok[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      bool valid;
      const int rho = unit_row(L, lane, q, valid);
      rows[q] = u * L.U + rho;
      ok[q] = valid && rows[q] < L.n;
      r[q] = ok[q] ? in[rows[q]] : 0.0;
    }
    if (mode == 3) unit_apply_ltinv<FT>(L, fac + u * uL, lane, r, z);
    else unit_apply_linv<FT>(L, fac + u * uL, lane, r, z);
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (ok[q]) s.t[rows[q]] = z[q];
  }
}

template <typename VT>
__global__ void __launch_bounds__(256) lz_spmv_op_kernel(LanczosState s, const int32_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci, const VT* __restrict__ va,
                                                         int j) {
  if (*(volatile const int*)s.ctl) return;
  const double* qj = s.V + (int64_t)j * s.n;
  const double* qp = j > 0 ? s.V + (int64_t)(j - 1) * s.n : nullptr;
  const double bprev = j > 0 ? s.beta[j - 1] : 0.0;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
    double w = spmv_row<VT, false>(rp, ci, va, qj, i);
    if (j > 0) w = fma(-bprev, qp[i], w);
    s.w[i] = w;
    acc = fma(qj[i], w, acc);
  }
  last_cta_sum1(acc, s.part, s.counter, s.alpha + j);
}

// MODE 0: w -= alpha_j q_j, c1 = V^T w;  MODE 1: w -= V c1, c2 = V^T w;
// MODE 2: w -= V c2, beta;  MODE 3 (no reorthogonalisation): w -= alpha_j q_j, beta.
template <int MODE>
__global__ void __launch_bounds__(256) lz_reorth_kernel(LanczosState s, int j) {
  if (*(volatile const int*)s.ctl) return;
  extern __shared__ double dsm[];
  __shared__ double smr[32];
  __shared__ int is_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int nl = j + 1;
  const bool need_tile = MODE != 3;
  // Coefficient passes (MODE 0, 1) keep one partial sum per (basis vector, lane) in shared
  // memory across all of the CTA's tiles and reduce across lanes once at the end: a warp
  // shuffle tree per tile would cost five FP64 adds per 32 products on the narrow FP64 pipe.
  constexpr bool COEF = MODE == 0 || MODE == 1;
  // Shared memory: two tile buffers (the next tile streams in with cp.async while the current
  // one is used), each nl rows of 32 basis values plus the 32 values of w; then the per-lane
  // partials (COEF), the cross-warp sums and the updated w of the tile.
  const int tile_elems = need_tile ? nl * LZ_TW + LZ_TW : LZ_TW;
  double* buf0 = dsm;
  double* buf1 = buf0 + tile_elems;
  double* acc = buf1 + tile_elems;                   // COEF: nl * 32 per-lane partials
  double* red = acc + (COEF ? nl * LZ_TW : 0);       // 8 * 32
  double* wt = red + 8 * 32;                         // 32
  const int64_t n = s.n;
  const double aj = s.alpha[j];
  const double* cin = MODE == 1 ? s.coef : s.coef + s.m;
  const double* qj = s.V + (int64_t)j * n;
  if (COEF)
    for (int i = tid; i < nl * LZ_TW; i += blockDim.x) acc[i] = 0.0;
  double nrm = 0.0;
  // Stage tile t (columns t*32 .. t*32+31) into buf: basis rows (warp-strided, one 8-byte
  // element per lane) and w; columns past n are zero (plain stores).
  auto stage = [&](int64_t t, double* buf) {
    const int64_t col = t * LZ_TW + lane;
    if (need_tile) {
      for (int l = warp; l < nl; l += nwarp) {
        double* dst = buf + l * LZ_TW + lane;
        if (col < n) cp_async8(dst, s.V + (int64_t)l * n + col);
        else *dst = 0.0;
      }
    }
    if (warp == nwarp - 1) {
      double* dst = buf + (need_tile ? nl * LZ_TW : 0) + lane;
      if (col < n) cp_async8(dst, s.w + col);
      else *dst = 0.0;
    }
    cp_async_commit();
  };
  int64_t t = blockIdx.x;
  if (t * LZ_TW < n) stage(t, buf0);
  for (int k = 0; t * LZ_TW < n; t += gridDim.x, ++k) {
    double* cur = (k & 1) ? buf1 : buf0;
    double* nxt = (k & 1) ? buf0 : buf1;
    const bool more = (t + gridDim.x) * LZ_TW < n;
    if (more) {
      stage(t + gridDim.x, nxt);
      cp_async_wait<1>();   // this thread's copies of the current tile have landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();      // everyone's copies of the current tile are visible
    const double* Vs = cur;
    const double* wsrc = cur + (need_tile ? nl * LZ_TW : 0);
    const int64_t col = t * LZ_TW + lane;
    if (MODE == 0 || MODE == 3) {
      if (tid < LZ_TW) {
        const double qv = MODE == 0 ? Vs[j * LZ_TW + tid] : (col < n ? qj[col] : 0.0);
        const double w = col < n ? fma(-aj, qv, wsrc[tid]) : 0.0;
        wt[tid] = w;
        if (col < n) s.w[col] = w;
      }
    } else {
      double g = 0.0;
      for (int l = warp; l < nl; l += nwarp) g = fma(cin[l], Vs[l * LZ_TW + lane], g);
      red[warp * LZ_TW + lane] = g;
      __syncthreads();
      if (tid < LZ_TW) {
        double sum = 0.0;
        for (int q = 0; q < nwarp; ++q) sum += red[q * LZ_TW + tid];
        const double w = col < n ? wsrc[tid] - sum : 0.0;
        wt[tid] = w;
        if (col < n) s.w[col] = w;
      }
    }
    __syncthreads();
    if (COEF) {
      const double wl = wt[lane];
      for (int l = warp; l < nl; l += nwarp) acc[l * LZ_TW + lane] = fma(Vs[l * LZ_TW + lane], wl, acc[l * LZ_TW + lane]);
    } else if (tid < LZ_TW) {
      nrm = fma(wt[tid], wt[tid], nrm);
    }
    __syncthreads();      // the current buffer is refilled two tiles later
  }
  __syncthreads();
  const int m = s.m;
  if (COEF) {
    for (int l = warp; l < nl; l += nwarp) {
      const double p = warp_sum(acc[l * LZ_TW + lane]);
      if (lane == 0) __stcg(s.part + (int64_t)blockIdx.x * m + l, p);
    }
  } else {
    double v[1] = {nrm};
    block_sum<1>(v, smr);
    if (tid == 0) __stcg(s.part + (int64_t)blockIdx.x * m, v[0]);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned old = atomicAdd(s.counter, 1u);
    is_last = (old == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int G = gridDim.x;
  if (MODE == 0 || MODE == 1) {
    double* cout = MODE == 0 ? s.coef : s.coef + m;
    for (int l = warp; l < nl; l += nwarp) {
      double a = 0.0;
      for (int c = lane; c < G; c += 32) a += __ldcg(s.part + (int64_t)c * m + l);
      a = warp_sum(a);
      if (lane == 0) __stcg(cout + l, a);
    }
  } else {
    double a = 0.0;
    for (int c = lane; c < G; c += 32) a += __ldcg(s.part + (int64_t)c * m);
    a = warp_sum(a);   // every warp computes the same value; warp 0 publishes it
    if (tid == 0) {
      const double bj = sqrt(a);
      s.beta[j] = bj;
      double tn = *s.tnorm;
      if (fabs(aj) > tn) tn = fabs(aj);
      if (bj > tn) tn = bj;
      *s.tnorm = tn;
      s.ctl[1] = j + 1;
      if (bj <= s.tol * tn || j + 1 == s.m || (int64_t)(j + 1) >= n) s.ctl[0] = 1;
    }
  }
  if (tid == 0) *s.counter = 0u;
}

__global__ void __launch_bounds__(256) lz_normalize_kernel(LanczosState s, int j) {
  if (*(volatile const int*)s.ctl) return;
  const double bj = s.beta[j];
  double* qn = s.V + (int64_t)(j + 1) * s.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
    qn[i] = s.w[i] / bj;
}

// Sturm count of T - x I (diag a, off-diagonal b) and bisection for the k-th smallest
// eigenvalue, from the Gershgorin interval until the midpoint stops moving.
__device__ int sturm_count(int m, const double* a, const double* b, double x) {
  double bmax2 = 0.0;
  for (int i = 0; i + 1 < m; ++i) bmax2 = fmax(bmax2, b[i] * b[i]);
  const double pivmin = 2.2250738585072014e-308 * (bmax2 > 1.0 ? bmax2 : 1.0);
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    d = (a[i] - x) - (i > 0 ? (b[i - 1] * b[i - 1]) / d : 0.0);
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

__global__ void lz_bisect_kernel(LanczosState s) {
  const int m = s.ctl[1];
  const int k = threadIdx.x == 0 ? 0 : m - 1;
  if (threadIdx.x > 1 || m < 1) return;
  const double* a = s.alpha;
  const double* b = s.beta;
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    double r = 0.0;
    if (i > 0) r += fabs(b[i - 1]);
    if (i + 1 < m) r += fabs(b[i]);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(m, a, b, mid) > k) hi = mid;
    else lo = mid;
  }
  s.result[threadIdx.x] = 0.5 * (lo + hi);
}

// ------------------------------------------------------------------ host side
int lanczos_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 2 * sms;
}

static size_t reorth_smem(int nl, bool tile, bool coef) {
  const size_t tile_elems = tile ? (size_t)nl * LZ_TW + LZ_TW : LZ_TW;
  return sizeof(double) * (2 * tile_elems + (coef ? (size_t)nl * LZ_TW : 0) + 8 * 32 + 32);
}

cudaError_t lanczos_init(const LanczosState& s, const double* v0, bool precond, const Layout& L, const void* linv,
                         bool fac_f32, cudaStream_t st) {
  const int G = lanczos_grid();
  cudaError_t e = cudaMemsetAsync(s.ctl, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.tnorm, 0, sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const double* src = v0;
  if (precond) {
    // t = L^{-1} v0 (the ltinv kernel reads V[0], so stage v0 there first)
    e = cudaMemcpyAsync(s.V, v0, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)G;
    if (fac_f32) lz_ltinv_kernel<float><<<g, 256, 0, st>>>(s, L, (const float*)linv, 0, 2);
    else lz_ltinv_kernel<double><<<g, 256, 0, st>>>(s, L, (const double*)linv, 0, 2);
    src = s.t;
  }
  lz_sumsq_kernel<<<G, 256, 0, st>>>(s, src);
  lz_start_kernel<<<G, 256, 0, st>>>(s, src);
  return cudaGetLastError();
}

cudaError_t lanczos_step(const LanczosState& s, int j, int reorth, bool precond, const Layout& L, const int32_t* rp,
                         const int32_t* ci, const void* va, bool val_f32, const void* linv, bool fac_f32,
                         cudaStream_t st) {
  const int G = lanczos_grid();
  if (precond) {
    if (fac_f32) lz_ltinv_kernel<float><<<G, 256, 0, st>>>(s, L, (const float*)linv, j, 3);
    else lz_ltinv_kernel<double><<<G, 256, 0, st>>>(s, L, (const double*)linv, j, 3);
    SymPhase2Args a;
    a.lay = L;
    a.rp = rp;
    a.ci = ci;
    a.va = va;
    a.linv = linv;
    a.t = s.t;
    a.out = s.w;
    a.q_cur = s.V + (int64_t)j * s.n;
    a.q_prev = j > 0 ? s.V + (int64_t)(j - 1) * s.n : nullptr;
    a.beta = s.beta;
    a.j = j;
    a.part = s.part;
    a.counter = s.counter;
    a.alpha_out = s.alpha + j;
    a.done = s.ctl;
    cudaError_t e = launch_sym_phase2(a, val_f32, fac_f32, G, st);
    if (e != cudaSuccess) return e;
  } else {
    if (val_f32) lz_spmv_op_kernel<float><<<G, 256, 0, st>>>(s, rp, ci, (const float*)va, j);
    else lz_spmv_op_kernel<double><<<G, 256, 0, st>>>(s, rp, ci, (const double*)va, j);
  }
  const int nl = j + 1;
  if (reorth) {
    const size_t sm = reorth_smem(nl, true, true);
    lz_reorth_kernel<0><<<G, 256, sm, st>>>(s, j);
    lz_reorth_kernel<1><<<G, 256, sm, st>>>(s, j);
    lz_reorth_kernel<2><<<G, 256, reorth_smem(nl, true, false), st>>>(s, j);
  } else {
    lz_reorth_kernel<3><<<G, 256, reorth_smem(nl, false, false), st>>>(s, j);
  }
  if (j + 1 < s.m) lz_normalize_kernel<<<G, 256, 0, st>>>(s, j);
  return cudaGetLastError();
}

cudaError_t lanczos_finish(const LanczosState& s, cudaStream_t st) {
  lz_bisect_kernel<<<1, 32, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t lanczos_configure(int m) {
  const size_t sm = reorth_smem(m, true, true);
  cudaError_t e = cudaFuncSetAttribute(lz_reorth_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lz_reorth_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lz_reorth_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  return e;
}

}  // namespace pc

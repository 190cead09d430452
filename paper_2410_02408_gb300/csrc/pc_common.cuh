// Device-side building blocks shared by the libpc kernels (sm_103a).
//
// Factor storage ("warp units").  The block partition of Sec. 3.2 cuts the rows into
// blocks of bs rows.  A warp owns one unit of U rows:
//   bs <= 32 : G = floor(32/bs) whole blocks per unit, U = G*bs, one row per lane (S = 1);
//   bs <= 64 : one block per unit, U = bs, lane l owns rows l and l+32 (S = 2).
// Inside a unit, the entries a lane needs are stored so that for a fixed entry index k
// and slot s the 32 lanes read 32 consecutive elements (fully coalesced):
//   element (k, s, lane) lives at unit_base + (k*S + s)*32 + lane.
// M^{-1} (symmetric) is stored "circulantly": entry k of row i is M(i, (i+k) mod bs) for
// k = 0..floor(bs/2).  Every unordered pair of the block appears once, except that for
// even bs the pair at distance bs/2 is stored by both of its rows.  That is bs/2+1
// entries per row against bs/2+1/2 for a packed triangle.
// L^{-1} (lower triangular) is stored by diagonals: entry k of row i is L^{-1}(i, i-k)
// (0 when i < k), k = 0..bs-1.
// Rows past n inside the last block are padded with the identity.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pc {

constexpr unsigned FULL = 0xffffffffu;

// Streaming multiprocessors of the current device (host side; grid sizing).
inline int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

enum : int {
  ST_OK = 0,
  ST_INVALID = 1,
  ST_NOT_SPD = 2,
  ST_BREAKDOWN = 3,
  ST_NO_CONV = 4,
  ST_TIMEOUT = 5,
};

struct Layout {
  int32_t bs;     // block size
  int32_t G;      // blocks per unit
  int32_t U;      // rows per unit
  int32_t S;      // row slots per lane
  int32_t K;      // floor(bs/2)
  int32_t EM;     // M^{-1} entries per row slot = K+1
  int32_t EL;     // L^{-1} entries per row slot = bs
  int32_t pad;
  int64_t n;
  int64_t n_units;
  int64_t n_blocks;
};

__host__ __device__ inline Layout make_layout(int64_t n, int32_t bs) {
  Layout L;
  L.bs = bs;
  if (bs <= 32) {
    L.G = 32 / bs;
    L.U = L.G * bs;
    L.S = 1;
  } else {
    L.G = 1;
    L.U = bs;
    L.S = 2;
  }
  L.K = bs / 2;
  L.EM = L.K + 1;
  L.EL = bs;
  L.pad = 0;
  L.n = n;
  L.n_units = (n + L.U - 1) / L.U;
  L.n_blocks = (n + bs - 1) / bs;
  return L;
}

// elements of one unit in each factor array
__host__ __device__ inline int64_t unit_elems_minv(const Layout& L) { return (int64_t)L.EM * L.S * 32; }
__host__ __device__ inline int64_t unit_elems_linv(const Layout& L) { return (int64_t)L.EL * L.S * 32; }

// ------------------------------------------------------------------ loads / stores
// Read-only for the whole kernel: non-coherent path, no L1 allocation.
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// Read-only index data that is reused (row pointers): ordinary read-only path.
__device__ __forceinline__ int32_t ld_ro(const int32_t* p) { return __ldg(p); }

// L2 eviction priority of individual loads: a cache policy (createpolicy) attached to a
// read-only load (ld.global.nc.L2::cache_hint).  The binned SpMV streams the matrix once per
// launch with evict-first and gathers the vector with evict-last (and without L1 allocation), so
// that the gathered vector stays in L2 while gigabytes of matrix pass through it.  Hints only:
// no global state changes.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int32_t ld_hint(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int64_t ld_hint(const int64_t* p, uint64_t pol) {
  int64_t v;
  asm("ld.global.nc.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_hint(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
// Gathers: no L1 allocation either, so that scattered vector reads do not evict the matrix lines
// each lane reuses across its next rounds.
__device__ __forceinline__ double ld_gather_hint(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

// Vectors written inside a persistent kernel: L2-coherent loads/stores (bypass L1).
__device__ __forceinline__ double ld_vec(const double* p) { return __ldcg(p); }
__device__ __forceinline__ void st_vec(double* p, double v) { __stcg(p, v); }

template <bool COHERENT>
__device__ __forceinline__ double ld_x(const double* p) {
  if constexpr (COHERENT) return __ldcg(p);
  else return __ldg(p);
}

// float <-> double conversions on the integer pipe.  On this GPU the hardware conversion
// instructions share the (narrow) FP64 pipe with DFMA, so the hot loops convert by
// rewriting the IEEE-754 fields: float -> double is exact; double -> float rounds to
// nearest-even.  Values whose float image is zero, subnormal, infinite or NaN take the
// hardware conversion (rare in the solver's data).
// The hardware fallback sits behind a warp-uniform branch into an out-of-line function: a
// predicated-off conversion would still occupy the FP64 pipe, and keeping the fallback out of
// line stops the compiler from if-converting the branch into exactly that.  Both helpers must
// be called by full warps.
static __device__ __noinline__ double f2d_special(float f, double r, bool special) { return special ? (double)f : r; }
static __device__ __noinline__ float d2f_special(double x, float r, bool special) {
  return special ? __double2float_rn(x) : r;
}
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  const bool special = ex == 0u || ex == 0xffu;
  const uint64_t d = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(ex + 896u) << 52) |
                     ((uint64_t)(u & 0x7fffffu) << 29);
  double r = __longlong_as_double((long long)d);
  if (__any_sync(FULL, special)) r = f2d_special(f, r, special);
  return r;
}
__device__ __forceinline__ float d2f(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32);
  const int ex = (int)((hi >> 20) & 0x7ffu) - 896;   // biased float exponent
  const bool special = ex <= 0 || ex >= 255;
  const uint32_t m23 = (uint32_t)((u >> 29) & 0x7fffffull);
  const uint32_t rest = (uint32_t)(u & 0x1fffffffull);   // 29 discarded bits
  uint32_t f = (hi & 0x80000000u) | ((uint32_t)(ex & 0xff) << 23) | m23;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) f += 1u;   // carry may bump the exponent
  float r = __uint_as_float(f);
  if (__any_sync(FULL, special)) r = d2f_special(x, r, special);
  return r;
}
template <typename T>
__device__ __forceinline__ T to_ft(double v);
template <>
__device__ __forceinline__ double to_ft<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_ft<float>(double v) { return d2f(v); }
__device__ __forceinline__ double from_ft(double v) { return v; }
__device__ __forceinline__ double from_ft(float v) { return f2d(v); }

// ------------------------------------------------------------------ SpMV row
// acc = sum_e val[e] * x[col[e]] over the row, in storage order (FMA chain).
template <typename VT, bool COHERENT>
__device__ __forceinline__ double spmv_row(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                           const VT* __restrict__ va, const double* x, int64_t row) {
  const int32_t s = ld_ro(rp + row);
  const int32_t e = ld_ro(rp + row + 1);
  double acc = 0.0;
  // Chunks of 8 entries: all index/value loads of a chunk are issued before the gathers
  // (clamped to the row's last entry, so every load is in bounds), then the products are
  // accumulated in storage order for the entries that exist.
  for (int32_t k0 = s; k0 < e; k0 += 8) {
    int32_t c[8];
    VT v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int32_t k = min(k0 + t, e - 1);
      c[t] = ld_stream(ci + k);
      v[t] = ld_stream(va + k);
    }
    double xv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) xv[t] = ld_x<COHERENT>(x + c[t]);
#pragma unroll
    for (int t = 0; t < 8; ++t)   // per-lane conversion: callers may be divergent here
      if (k0 + t < e) acc = fma((double)v[t], xv[t], acc);
  }
  return acc;
}

// ------------------------------------------------------------------ unit geometry
// Row of the unit owned by (lane, slot); valid == false for idle lanes/slots.
__device__ __forceinline__ int unit_row(const Layout& L, int lane, int s, bool& valid) {
  const int rho = lane + 32 * s;
  valid = (rho < L.U) && (s < L.S);
  return rho;
}

// Factor element load: from global (read-only stream) or from a shared-memory copy.
template <bool SMEM, typename FT>
__device__ __forceinline__ FT ldf(const FT* p) {
  if constexpr (SMEM) return *p;
  else return ld_stream(p);
}

// ------------------------------------------------------------------ block apply, S = 1
// z_i = sum_j M(i, j) r_j within each block of the unit (bs <= 32).
template <typename FT, int BS, bool SMEM = false>
__device__ __forceinline__ FT apply_inv_s1(const FT* __restrict__ Mu, int bs_rt, int lane, FT r) {
  const int bs = BS > 0 ? BS : bs_rt;
  const int i = lane % bs;
  const int base = lane - i;
  const int K = bs / 2;
  FT z = ldf<SMEM>(Mu + lane) * r;
  if constexpr (BS > 0) {
    // BS is a power of two: a width-BS shuffle reduces the source index modulo BS inside the
    // lane's own block, so the cyclic offsets (i + k) mod BS and (i - k) mod BS cost one add.
    static_assert((BS & (BS - 1)) == 0, "compile-time block sizes are powers of two");
#pragma unroll
    for (int k = 1; k <= BS / 2; ++k) {
      const FT a = ldf<SMEM>(Mu + k * 32 + lane);
      z = fma(a, __shfl_sync(FULL, r, lane + k, BS), z);
      if (2 * k != BS) z += __shfl_sync(FULL, a * r, lane + (BS - k), BS);
    }
  } else {
    for (int k = 1; k <= K; ++k) {
      const FT a = ldf<SMEM>(Mu + k * 32 + lane);
      int jf = i + k;
      if (jf >= bs) jf -= bs;
      const FT rf = __shfl_sync(FULL, r, (base + jf) & 31);
      z = fma(a, rf, z);
      if (2 * k != bs) {
        int jb = i - k;
        if (jb < 0) jb += bs;
        z += __shfl_sync(FULL, a * r, (base + jb) & 31);
      }
    }
  }
  return z;
}

// ------------------------------------------------------------------ block apply, S = 2
// One block of 33..64 rows per warp; lane owns rows lane and lane+32.
template <typename FT, int BS, bool SMEM = false>
__device__ __forceinline__ void apply_inv_s2(const FT* __restrict__ Mu, int bs_rt, int lane, FT r0, FT r1,
                                             FT& z0, FT& z1) {
  const int bs = BS > 0 ? BS : bs_rt;
  const int K = bs / 2;
  z0 = ldf<SMEM>(Mu + lane) * r0;
  z1 = ldf<SMEM>(Mu + 32 + lane) * r1;
#pragma unroll 4
  for (int k = 1; k <= K; ++k) {
    const FT a0 = ldf<SMEM>(Mu + (2 * k) * 32 + lane);
    const FT a1 = ldf<SMEM>(Mu + (2 * k + 1) * 32 + lane);
    int j0 = lane + k;
    if (j0 >= bs) j0 -= bs;
    int j1 = lane + 32 + k;
    if (j1 >= bs) j1 -= bs;
    {
      const FT x00 = __shfl_sync(FULL, r0, j0 & 31);
      const FT x01 = __shfl_sync(FULL, r1, j0 & 31);
      const FT x10 = __shfl_sync(FULL, r0, j1 & 31);
      const FT x11 = __shfl_sync(FULL, r1, j1 & 31);
      z0 = fma(a0, (j0 >= 32) ? x01 : x00, z0);
      z1 = fma(a1, (j1 >= 32) ? x11 : x10, z1);
    }
    if (2 * k != bs) {
      const FT t0 = a0 * r0;
      const FT t1 = a1 * r1;
      int b0 = lane - k;
      if (b0 < 0) b0 += bs;
      int b1 = lane + 32 - k;
      if (b1 < 0) b1 += bs;
      const FT y00 = __shfl_sync(FULL, t0, b0 & 31);
      const FT y01 = __shfl_sync(FULL, t1, b0 & 31);
      const FT y10 = __shfl_sync(FULL, t0, b1 & 31);
      const FT y11 = __shfl_sync(FULL, t1, b1 & 31);
      z0 += (b0 >= 32) ? y01 : y00;
      z1 += (b1 >= 32) ? y11 : y10;
    }
  }
}

// Unit-level M^{-1} apply: r/z are per-slot doubles of the rows the lane owns (0 for
// rows beyond n or idle lanes).  Arithmetic in FT.
template <typename FT, int BS, bool SMEM = false>
__device__ __forceinline__ void unit_apply_inv(const Layout& L, const FT* __restrict__ Mu, int lane,
                                               const double (&r)[2], double (&z)[2]) {
  if ((BS > 0 && BS <= 32) || (BS == 0 && L.S == 1)) {
    z[0] = from_ft(apply_inv_s1<FT, (BS <= 32 ? BS : 0), SMEM>(Mu, L.bs, lane, to_ft<FT>(r[0])));
    z[1] = 0.0;
  } else {
    FT z0, z1;
    apply_inv_s2<FT, (BS > 32 ? BS : 0), SMEM>(Mu, L.bs, lane, to_ft<FT>(r[0]), to_ft<FT>(r[1]), z0, z1);
    z[0] = from_ft(z0);
    z[1] = from_ft(z1);
  }
}

// ------------------------------------------------------------------ L^{-1} and L^{-T}
// y_i = sum_{k<=i} L^{-1}(i, i-k) u_{i-k}
template <typename FT>
__device__ __forceinline__ void unit_apply_linv(const Layout& L, const FT* __restrict__ Lu, int lane,
                                                const double (&u)[2], double (&y)[2]) {
  const int bs = L.bs;
  if (L.S == 1) {
    const int i = lane % bs;
    const int base = lane - i;
    const FT uu = (FT)u[0];
    FT acc = 0;
    for (int k = 0; k < bs; ++k) {
      const FT a = ld_stream(Lu + k * 32 + lane);
      const int src = base + (i >= k ? i - k : 0);
      const FT v = __shfl_sync(FULL, uu, src & 31);
      acc = fma(a, v, acc);
    }
    y[0] = (double)acc;
    y[1] = 0.0;
  } else {
    const FT u0 = (FT)u[0], u1 = (FT)u[1];
    FT acc0 = 0, acc1 = 0;
    for (int k = 0; k < bs; ++k) {
      const FT a0 = ld_stream(Lu + (2 * k) * 32 + lane);
      const FT a1 = ld_stream(Lu + (2 * k + 1) * 32 + lane);
      const int j0 = lane >= k ? lane - k : 0;
      const int j1 = lane + 32 - k;   // >= 0 since k < 64 ... clamp below
      const int j1c = j1 >= 0 ? j1 : 0;
      const FT v00 = __shfl_sync(FULL, u0, j0 & 31);
      const FT v01 = __shfl_sync(FULL, u1, j0 & 31);
      const FT v10 = __shfl_sync(FULL, u0, j1c & 31);
      const FT v11 = __shfl_sync(FULL, u1, j1c & 31);
      acc0 = fma(a0, (j0 >= 32) ? v01 : v00, acc0);
      acc1 = fma(a1, (j1c >= 32) ? v11 : v10, acc1);
    }
    y[0] = (double)acc0;
    y[1] = (double)acc1;
  }
}

// w_i = sum_{k: i+k < bs} L^{-1}(i+k, i) v_{i+k}; the factor entry lives at row i+k.
template <typename FT>
__device__ __forceinline__ void unit_apply_ltinv(const Layout& L, const FT* __restrict__ Lu, int lane,
                                                 const double (&v)[2], double (&w)[2]) {
  const int bs = L.bs;
  if (L.S == 1) {
    const int i = lane % bs;
    const int base = lane - i;
    const FT vv = (FT)v[0];
    FT acc = 0;
    for (int k = 0; k < bs; ++k) {
      const FT a = ld_stream(Lu + k * 32 + lane);
      const FT t = a * vv;
      const int j = i + k;
      const int src = base + (j < bs ? j : bs - 1);
      const FT g = __shfl_sync(FULL, t, src & 31);
      if (j < bs) acc += g;
    }
    w[0] = (double)acc;
    w[1] = 0.0;
  } else {
    const FT v0 = (FT)v[0], v1 = (FT)v[1];
    FT acc0 = 0, acc1 = 0;
    for (int k = 0; k < bs; ++k) {
      const FT a0 = ld_stream(Lu + (2 * k) * 32 + lane);
      const FT a1 = ld_stream(Lu + (2 * k + 1) * 32 + lane);
      const FT t0 = a0 * v0, t1 = a1 * v1;
      const int j0 = lane + k;          // source row for row lane
      const int j1 = lane + 32 + k;     // source row for row lane+32
      const int c0 = j0 < bs ? j0 : bs - 1;
      const int c1 = j1 < bs ? j1 : bs - 1;
      const FT g00 = __shfl_sync(FULL, t0, c0 & 31);
      const FT g01 = __shfl_sync(FULL, t1, c0 & 31);
      const FT g10 = __shfl_sync(FULL, t0, c1 & 31);
      const FT g11 = __shfl_sync(FULL, t1, c1 & 31);
      if (j0 < bs) acc0 += (c0 >= 32) ? g01 : g00;
      if (j1 < bs) acc1 += (c1 >= 32) ? g11 : g10;
    }
    w[0] = (double)acc0;
    w[1] = (double)acc1;
  }
}

// ------------------------------------------------------------------ reductions
// Warp sum by a fixed xor tree (bit-reproducible).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Block sum of NV values; result valid in every thread.  sm: NV * 32 doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();   // sm may still be read from a previous call
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[i * 32 + warp] = v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = lane < nw ? sm[i * 32 + lane] : 0.0;
    v[i] = warp_sum(t);
  }
}

// ------------------------------------------------------------------ grid barrier
struct GridSync {
  unsigned int count;   // arrivals, monotonic over the launch (wraps safely)
  unsigned int pad;
  int status;           // first error code raised on the device (0 = none)
  int where;            // diagnostic: barrier index that timed out
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(const volatile int*)p; }

// Grid-wide sum of NV per-thread values plus a barrier; every CTA leaves with the same
// totals in v[].  Barrier number `bar` (0, 1, 2, ... in program order, identical in every
// CTA) completes when the arrival counter reaches (bar+1) * gridDim.x: each CTA adds one
// with release semantics and thread 0 polls with acquire semantics under a clock64
// budget.  Each CTA then sums the per-CTA partials itself in CTA-index order, so the
// result is the same in every CTA and from run to run.  Partials are double-buffered by
// the barrier's parity (a CTA can run at most one barrier ahead of the slowest reader).
// Returns false if the kernel must stop (a timeout here or an error raised elsewhere).
// part: 2 * gridDim.x * NV doubles; sm: NV*32 doubles and flag: 4 ints of shared memory.
template <int NV>
__device__ __forceinline__ bool grid_allreduce(double* v, double* part, GridSync* gs, long long budget,
                                               double* sm, int* flag, int bar) {
  if constexpr (NV > 0) block_sum<NV>(v, sm);
  else __syncthreads();   // flag[] may still be read from the previous call
  const unsigned G = gridDim.x;
  double* pbuf = part + (size_t)(bar & 1) * G * (NV > 0 ? NV : 1);
  if (threadIdx.x == 0) {
    flag[2] = 0;
    if (ld_volatile_i32(&gs->status) != 0) {
      flag[2] = 1;
    } else {
      if constexpr (NV > 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) __stcg(pbuf + (size_t)blockIdx.x * NV + i, v[i]);
      }
      red_release_add_u32(&gs->count, 1u);
      const unsigned target = (unsigned)(bar + 1) * G;
      const long long t0 = clock64();
      while ((int)(ld_acquire_u32(&gs->count) - target) < 0) {
        if (clock64() - t0 > budget) {
          if (atomicCAS(&gs->status, 0, ST_TIMEOUT) == 0) gs->where = bar;
          flag[2] = 1;
          break;
        }
        if (ld_volatile_i32(&gs->status) != 0) {
          flag[2] = 1;
          break;
        }
      }
    }
  }
  __syncthreads();
  if (flag[2]) return false;
  if constexpr (NV > 0) {
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (unsigned c = threadIdx.x; c < G; c += blockDim.x) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += __ldcg(pbuf + (size_t)c * NV + i);
    }
    block_sum<NV>(acc, sm);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = acc[i];
  }
  return true;
}

// Single-value grid sum with a last-CTA finish (fixed order).  part: gridDim doubles.
__device__ __forceinline__ void last_cta_sum1(double v, double* part, unsigned* counter, double* out) {
  __shared__ double sm[32];
  __shared__ int is_last;
  double a[1] = {v};
  block_sum<1>(a, sm);
  if (threadIdx.x == 0) {
    __stcg(part + blockIdx.x, a[0]);
    __threadfence();
    const unsigned old = atomicAdd(counter, 1u);
    is_last = (old == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double acc[1] = {0.0};
    for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) acc[0] += __ldcg(part + c);
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) {
      __stcg(out, acc[0]);
      *counter = 0u;
    }
  }
}

}  // namespace pc

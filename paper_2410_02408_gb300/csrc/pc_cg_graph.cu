// Graph-driven block-Jacobi PCG: three full-occupancy kernels per iteration inside a CUDA
// graph `while` conditional node, so the iteration never returns to the host.
//
//   before the loop   I1  r = b - A x, ||b||^2          I2  z = M^{-1} r, p = z, rho, ||r||^2
//   loop body         A   q = A p, p.q  -> alpha       B   r -= alpha q, z = M^{-1} r, r.z, ||r||^2
//                     C   x += alpha p, p = z + beta p
//   after the loop    T   r = b - A x, ||b - A x||^2 (true residual)
//
// Each kernel reduces its per-CTA partial sums in its last CTA, in CTA order (fixed order:
// bit-reproducible), and that CTA updates the CG scalars and the loop condition
// (cudaGraphSetConditional).  The scalar recurrences and stopping rules are those of
// Hestenes-Stiefel PCG: alpha = rho / p.q, beta = rho'/rho, stop when ||r|| <= tol ||b||,
// with max_iter and breakdown checks in the order the iteration meets them.  The host
// restarts from x (at most 3 times) when the true residual is above tol.
//
// Kernels are separate launches so each runs with its own register budget: the SpMV streams
// the CSR with ordinary L1-allocating loads (neighbouring rows share the cache lines of the
// column/value arrays), keeps 8 gathers in flight per row and pipelines each thread's rows
// (its time is set by the memory round trips in flight, not by its FP64 products).
#include <cuda_runtime.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <type_traits>

#include "pc_kernels.cuh"
#include "pc_tma.cuh"

namespace pc {

struct CgScalars {
  double bb, rho, alpha, beta, rr, tt;
  double tol;
  int32_t it, max_iter;
  int32_t status;   // ST_* of the solve
  int32_t done;     // 1: stop all further work of this round
  int32_t xupd;     // 1: x += alpha p due in kernel C (or the fused tail of kernel B)
  int32_t pupd;     // 1: p = z + beta p due in kernel C (or the fused tail of kernel B)
  int32_t cont;     // loop condition
  uint32_t gen;     // bumped by kernel B's last CTA once beta and the flags are set (fused tail)
  unsigned int cnt[4];   // last-CTA counters of I/A, B, T
};

// Last-CTA fixed-order reduction of NV values; returns true in the last CTA, whose v[] then
// holds the totals.  part: gridDim.x * NV doubles.
template <int NV>
__device__ __forceinline__ bool cg_last_cta(double* v, double* part, unsigned* counter, double* sm, int* is_last) {
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) __stcg(part + (size_t)blockIdx.x * NV + i, v[i]);
    __threadfence();
    const unsigned old = atomicAdd(counter, 1u);
    *is_last = (old == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!*is_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += __ldcg(part + (size_t)c * NV + i);
  }
  block_sum<NV>(acc, sm);
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = acc[i];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Binned SpMV row work, one load phase after the other: one row per group of LPR lanes
// (LPR = 1: one row per lane); lane j of the group takes entries j, j + LPR, ..., 8 per round
// (column indices and values, then the gathers of x).  lim = the longest range among the lanes
// sharing the loop (warp-uniform); product slots past it are not issued.  The sum starts from
// init (LPR = 1: the row's partial sum over earlier column segments, continued in entry order;
// LPR > 1: 0) and for LPR > 1 is completed by an xor tree, valid in every lane of the group.
// Called by full warps.  ps / pk: L2 policies of the matrix stream (evict first) and of the
// gathers of x (evict last).
template <typename VT, int LPR>
__device__ __forceinline__ double cg_range_plain(const int32_t* __restrict__ ci, const VT* __restrict__ va,
                                                 const double* __restrict__ x, int32_t s, int32_t cnt, int32_t lim,
                                                 double init, uint64_t ps, uint64_t pk) {
  const int j = LPR > 1 ? (int)(threadIdx.x & (LPR - 1)) : 0;
  const int32_t s0 = cnt > 0 ? s : 0;   // an empty range loads (and ignores) entry 0, which exists when lim > 0
  const int32_t kmax = max(cnt, 1) - 1;
  double acc = init;
  for (int32_t k0 = 0; k0 < lim; k0 += 8 * LPR) {
    int32_t c[8];
    VT v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int32_t k = s0 + min(k0 + t * LPR + j, kmax);
      c[t] = ld_hint(ci + k, ps);
      v[t] = ld_hint(va + k, ps);
    }
    double xv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) xv[t] = ld_gather_hint(x + c[t], pk);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (k0 + t * LPR < lim) {   // warp-uniform
        const double pr = fma(from_ft(v[t]), xv[t], acc);
        acc = (k0 + t * LPR + j < cnt) ? pr : acc;
      }
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  return acc;
}

// Pipelined variant of cg_range_plain (same entries, same order of products): the next round's
// column indices are
// loaded while the current round's gathers of x (and its values) are in flight, so a round
// costs one dependent memory round trip instead of two.  lim = the longest range among the
// lanes sharing the loop (warp-uniform); product slots past it are not issued.  The sum starts
// from init (LPR = 1: the row's partial sum over earlier column segments, continued in entry
// order; LPR > 1: 0) and for LPR > 1 is completed by an xor tree, valid in every lane of the
// group.  Called by full warps.  ps / pk: L2 policies as in cg_range_plain.
template <typename VT, int LPR>
__device__ __forceinline__ double cg_range_pipe(const int32_t* __restrict__ ci, const VT* __restrict__ va,
                                                const double* __restrict__ x, int32_t s, int32_t cnt, int32_t lim,
                                                double init, uint64_t ps, uint64_t pk) {
  const int j = LPR > 1 ? (int)(threadIdx.x & (LPR - 1)) : 0;
  const int32_t s0 = cnt > 0 ? s : 0;   // an empty range loads (and ignores) entry 0, which exists when lim > 0
  const int32_t kmax = max(cnt, 1) - 1;
  double acc = init;
  if (lim > 0) {
    int32_t c[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) c[t] = ld_hint(ci + s0 + min(t * LPR + j, kmax), ps);
    for (int32_t k0 = 0; k0 < lim; k0 += 8 * LPR) {
      double xv[8];
      VT v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        xv[t] = ld_gather_hint(x + c[t], pk);
        v[t] = ld_hint(va + s0 + min(k0 + t * LPR + j, kmax), ps);
      }
      const int32_t k1 = k0 + 8 * LPR;
      int32_t cn[8];
      if (k1 < lim) {   // warp-uniform
#pragma unroll
        for (int t = 0; t < 8; ++t) cn[t] = ld_hint(ci + s0 + min(k1 + t * LPR + j, kmax), ps);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (k0 + t * LPR < lim) {   // warp-uniform
          const double pr = fma(from_ft(v[t]), xv[t], acc);
          acc = (k0 + t * LPR + j < cnt) ? pr : acc;
        }
      }
      if (k1 < lim) {
#pragma unroll
        for (int t = 0; t < 8; ++t) c[t] = cn[t];
      }
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  return acc;
}

// cg_range_pipe<VT, 1> over the sliced copy of a one-lane-per-row group: entry k of the lane's
// row sits at base + 32 k + lane (the group's slab holds lim entries per lane, the rows'
// entries in storage order, padded past each row's end), so each load instruction of the
// warp reads one contiguous run of 32 entries instead of one cache line per lane.  Same
// products in the same order as cg_range_pipe<VT, 1>.
template <typename VT>
__device__ __forceinline__ double cg_range_sliced(const int32_t* __restrict__ sc, const VT* __restrict__ sv,
                                                  const double* __restrict__ x, int64_t base, int32_t cnt,
                                                  int32_t lim, uint64_t ps, uint64_t pk) {
  const int lane = threadIdx.x & 31;
  const int32_t* __restrict__ cp = sc + base + lane;
  const VT* __restrict__ vp = sv + base + lane;
  double acc = 0.0;
  if (lim > 0) {
    int32_t c[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) c[t] = ld_hint(cp + 32 * min(t, lim - 1), ps);
    for (int32_t k0 = 0; k0 < lim; k0 += 8) {
      double xv[8];
      VT v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        xv[t] = ld_gather_hint(x + c[t], pk);
        v[t] = ld_hint(vp + 32 * min(k0 + t, lim - 1), ps);
      }
      const int32_t k1 = k0 + 8;
      int32_t cn[8];
      if (k1 < lim) {   // warp-uniform
#pragma unroll
        for (int t = 0; t < 8; ++t) cn[t] = ld_hint(cp + 32 * min(k1 + t, lim - 1), ps);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (k0 + t < lim) {   // warp-uniform
          const double pr = fma(from_ft(v[t]), xv[t], acc);
          acc = (k0 + t < cnt) ? pr : acc;
        }
      }
      if (k1 < lim) {
#pragma unroll
        for (int t = 0; t < 8; ++t) c[t] = cn[t];
      }
    }
  }
  return acc;
}

struct CgArgs {
  Layout lay;
  const int32_t* rp;
  const int32_t* ci;
  const void* va;
  const void* minv;
  const double* b;
  double* x;
  double *r, *z, *p, *q;
  double* part;
  CgScalars* s;
  cudaGraphConditionalHandle cond;
  int32_t in_graph;    // 0 when the body kernels are launched one by one (profiling mode)
  CgBinned bin;        // binned SpMV order (bin.perm null: natural order)
  long long budget;    // clock64 cycles a CTA waits for kernel B's last CTA (fused tail)
};

// MODE 0 (I1): r = b - A x, sum b^2.  MODE 1 (A): q = A p, sum p q.  MODE 2 (T): r = b - A x, sum r^2.
//
// Natural order: a grid-stride loop over rows, one row per lane, warp-uniform trip counts
// (rows past n are masked).  Binned order (BIN): each warp walks its own run of work items of
// the permuted order (runs of about equal cost): a 32-row group, with one lane per row when its
// longest row has up to 64 entries, else 8 lanes per row; or a single row of a group whose
// longest row exceeds 256 entries, with the whole warp on it.  With column segments
// (bin.nseg > 1) the warp sweeps its run once per segment, each sweep gathering only the part
// of x that the segment covers, so the gathers of one sweep stay resident in L2 while the
// matrix streams past; the partial sums between sweeps are kept per binned position.
// The binned grid is one wave of resident CTAs (its split gives every warp an equal share), so
// each binned variant is held to the registers that keep its CTAs per SM resident: the plain
// one at 4 CTAs (64 registers), the pipelined one, which keeps a second round of column
// indices live, at 2 (up to 128 registers, no spills).
constexpr int SPMV_BIN_CTAS_PER_SM = 4;
constexpr int SPMV_BIN_PIPE_CTAS_PER_SM = 2;

template <typename VT, int LPR, bool PIPE>
__device__ __forceinline__ double cg_range(const int32_t* __restrict__ ci, const VT* __restrict__ va,
                                           const double* __restrict__ x, int32_t s, int32_t cnt, int32_t lim,
                                           double init, uint64_t ps, uint64_t pk) {
  if constexpr (PIPE) return cg_range_pipe<VT, LPR>(ci, va, x, s, cnt, lim, init, ps, pk);
  else return cg_range_plain<VT, LPR>(ci, va, x, s, cnt, lim, init, ps, pk);
}

// Natural row order: each thread walks rows base + tid, base + S + tid, ... (S = threads in the
// grid), software-pipelined over them: the row pointers two rows ahead and the column indices
// one row ahead are in flight while the current row's values, its gathers of x and its own
// entry of w (the vector the caller's epilogue needs: p or b) are loaded, so a row costs about
// one dependent memory round trip instead of three.  The first 8 entries of a row go through
// the pipeline, further entries (rare in the natural order, which serves short uniform rows)
// take plain rounds.  Each row is one FMA chain over its entries in storage order (the order
// of the oracle's sum), with float values widened on the integer pipe.  Rows past n are masked (empty
// ranges).  Called by whole CTAs; fin(row, sum, w_row) runs for the rows below n.
template <typename VT, typename FIN>
__device__ __forceinline__ void cg_rows_pipe(const CgArgs& a, const VT* __restrict__ va, const double* __restrict__ x,
                                             const double* __restrict__ w, FIN fin) {
  const int64_t n = a.lay.n;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  const int32_t* __restrict__ ci = a.ci;
  int64_t base = (int64_t)blockIdx.x * blockDim.x;
  if (base >= n) return;
  auto row_range = [&](int64_t b, int32_t& s, int32_t& e) {
    const int64_t r = b + threadIdx.x;
    s = 0;
    e = 0;
    if (r < n) {
      s = __ldg(a.rp + r);
      e = __ldg(a.rp + r + 1);
    }
  };
  // entry slot t of a row: an empty row reads (and ignores) entry 0, which exists for n > 0
  auto slot = [](int32_t s, int32_t cnt, int t) { return (cnt > 0 ? s : 0) + min(t, max(cnt, 1) - 1); };
  int32_t s0, e0, s1, e1;
  row_range(base, s0, e0);
  row_range(base + S, s1, e1);
  int32_t c[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) c[t] = __ldg(ci + slot(s0, e0 - s0, t));
  for (; base < n; base += S) {
    const int64_t row = base + threadIdx.x;
    const bool valid = row < n;
    const int32_t cnt = e0 - s0;
    const int32_t wmax = __reduce_max_sync(FULL, cnt);   // warp-uniform
    VT v[8];
    double xv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      v[t] = __ldg(va + slot(s0, cnt, t));
      xv[t] = __ldg(x + c[t]);
    }
    const double wr = valid ? __ldg(w + row) : 0.0;
    int32_t s2, e2;
    row_range(base + 2 * S, s2, e2);
#pragma unroll
    for (int t = 0; t < 8; ++t) c[t] = __ldg(ci + slot(s1, e1 - s1, t));
    double sum = 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < wmax) {   // a fully masked FP64 instruction still costs FP64-pipe time
        const double pr = fma(from_ft(v[t]), xv[t], sum);
        sum = t < cnt ? pr : sum;
      }
    }
    for (int32_t k0 = 8; k0 < wmax; k0 += 8) {
      int32_t cc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int32_t k = slot(s0, cnt, k0 + t);
        cc[t] = __ldg(ci + k);
        v[t] = __ldg(va + k);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) xv[t] = __ldg(x + cc[t]);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (k0 + t < wmax) {
          const double pr = fma(from_ft(v[t]), xv[t], sum);
          sum = k0 + t < cnt ? pr : sum;
        }
      }
    }
    if (valid) fin(row, sum, wr);
    s0 = s1;
    e0 = e1;
    s1 = s2;
    e1 = e2;
  }
}

// cg_rows_pipe over a sliced copy of the matrix (a.bin.scol with a.bin.perm null): the 32 rows
// of a warp are one group of 32 consecutive rows, whose slab holds entry k of its row l at
// 32 k + l, padded to the group's longest row and ending at sincl[group].  The rows' lengths
// still come from the row pointers; every load of column indices and values then reads one
// contiguous run per warp.  Same products in the same order as cg_rows_pipe.
template <typename VT, typename FIN>
__device__ __forceinline__ void cg_rows_sliced(const CgArgs& a, const double* __restrict__ x,
                                               const double* __restrict__ w, FIN fin) {
  const int64_t n = a.lay.n;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  const int32_t* __restrict__ sc = a.bin.scol;
  const VT* __restrict__ sv = reinterpret_cast<const VT*>(a.bin.sval);
  const int64_t* __restrict__ si = a.bin.sincl;
  const int lane = threadIdx.x & 31;
  int64_t base = (int64_t)blockIdx.x * blockDim.x;
  if (base >= n) return;
  // the row's range, and its group's slab end (lanes past n take the last group's: every lane
  // of a warp addresses the same slab)
  auto row_range = [&](int64_t b, int32_t& s, int32_t& e, int64_t& so) {
    const int64_t r = b + threadIdx.x;
    s = 0;
    e = 0;
    if (r < n) {
      s = __ldg(a.rp + r);
      e = __ldg(a.rp + r + 1);
    }
    so = __ldg(si + (min(r, n - 1) >> 5));
  };
  // slab entry t of this lane's row (t clamped to the group's longest row gm; gm > 0)
  auto slot = [&](int64_t so, int32_t gm, int t) { return so - 32ll * gm + 32ll * min(t, gm - 1) + lane; };
  int32_t s0, e0, s1, e1;
  int64_t o0, o1;
  row_range(base, s0, e0, o0);
  row_range(base + S, s1, e1, o1);
  int32_t m0 = __reduce_max_sync(FULL, e0 - s0);
  int32_t c[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) c[t] = m0 > 0 ? __ldg(sc + slot(o0, m0, t)) : 0;
  for (; base < n; base += S) {
    const int64_t row = base + threadIdx.x;
    const bool valid = row < n;
    const int32_t cnt = e0 - s0;
    const int32_t wmax = m0;   // warp-uniform
    VT v[8];
    double xv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      v[t] = wmax > 0 ? __ldg(sv + slot(o0, wmax, t)) : VT(0);
      xv[t] = __ldg(x + c[t]);
    }
    const double wr = valid ? __ldg(w + row) : 0.0;
    int32_t s2, e2;
    int64_t o2;
    row_range(base + 2 * S, s2, e2, o2);
    const int32_t m1 = __reduce_max_sync(FULL, e1 - s1);
#pragma unroll
    for (int t = 0; t < 8; ++t) c[t] = m1 > 0 ? __ldg(sc + slot(o1, m1, t)) : 0;
    double sum = 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < wmax) {
        const double pr = fma(from_ft(v[t]), xv[t], sum);
        sum = t < cnt ? pr : sum;
      }
    }
    for (int32_t k0 = 8; k0 < wmax; k0 += 8) {
      int32_t cc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        cc[t] = __ldg(sc + slot(o0, wmax, k0 + t));
        v[t] = __ldg(sv + slot(o0, wmax, k0 + t));
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) xv[t] = __ldg(x + cc[t]);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (k0 + t < wmax) {
          const double pr = fma(from_ft(v[t]), xv[t], sum);
          sum = k0 + t < cnt ? pr : sum;
        }
      }
    }
    if (valid) fin(row, sum, wr);
    s0 = s1;
    e0 = e1;
    o0 = o1;
    m0 = m1;
    s1 = s2;
    e1 = e2;
    o1 = o2;
  }
}

template <typename VT, int MODE, bool BIN, bool PIPE = false, bool SL = false>
__device__ __forceinline__ void cg_spmv_body(const CgArgs& a, double* sm, int* is_last_p) {
  int& is_last = *is_last_p;
  CgScalars* S = a.s;
  if (MODE == 1 && *(volatile int*)&S->done) {
    // stopped by another kernel of the round (a timed-out wait): end the loop here
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->cont = 0;
      if (a.in_graph) cudaGraphSetConditional(a.cond, 0u);
    }
    return;
  }
  const VT* va = reinterpret_cast<const VT*>(a.va);
  const int64_t n = a.lay.n;
  const double* X = MODE == 1 ? a.p : a.x;
  double acc = 0.0;
  if constexpr (BIN) {
    const CgBinned& B = a.bin;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int32_t g0 = __ldg(B.gsplit + gw), g1 = __ldg(B.gsplit + gw + 1);
    const int nseg = B.nseg;
    const uint64_t ps = l2_policy_evict_first(), pk = l2_policy_evict_last();
    const double* __restrict__ W = MODE == 1 ? a.p : a.b;   // the epilogue's vector
    // the row's result with its preloaded entry w_ of the epilogue's vector
    auto finish_w = [&](int64_t r_, double v_, double w_) {
      if (MODE == 1) {
        a.q[r_] = v_;
        acc = fma(w_, v_, acc);
      } else {
        const double ri = w_ - v_;
        a.r[r_] = ri;
        acc = MODE == 0 ? fma(w_, w_, acc) : fma(ri, ri, acc);
      }
    };
    for (int sg = 0; sg < nseg; ++sg) {
      const int32_t* lo_b = B.bnd + (int64_t)sg * B.bstride;
      const int32_t* hi_b = lo_b + B.bstride;
      const bool first = sg == 0, last = sg == nseg - 1;
      // The next item's bounds, and in the last segment its rows' original indices, load while
      // the current item's rows are processed; the rows' entries of the epilogue's vector load
      // when the item starts.  So an item neither starts with two dependent round trips nor
      // ends with two (the permutation, then the vector entry it addresses).  A row item (< 0)
      // gives every lane that row's range and index; a group item gives each lane its row's
      // range and index and the group's longest row.
      const bool sliced = B.scol != nullptr && nseg == 1;
      auto item_bounds = [&](int32_t item, int32_t& s_, int32_t& c_, int32_t& gm_, int32_t& r_, int64_t& so_) {
        r_ = 0;
        so_ = 0;
        if (item < 0) {
          const int64_t pos = -(int64_t)item - 1;
          s_ = ld_hint(lo_b + pos, ps);
          c_ = ld_hint(hi_b + pos, ps) - s_;
          gm_ = 0;
          if (last) r_ = ld_hint(B.perm + pos, ps);
        } else {
          const int64_t idx = (int64_t)item * 32 + lane;
          s_ = idx < n ? ld_hint(lo_b + idx, ps) : 0;
          c_ = idx < n ? ld_hint(hi_b + idx, ps) - s_ : 0;
          gm_ = ld_hint(B.gmax + item, ps);
          if (last && idx < n) r_ = ld_hint(B.perm + idx, ps);
          if (sliced) so_ = ld_hint(B.sincl + item, ps);   // the slab ends there (one-lane groups)
        }
      };
      int32_t item = g0 < g1 ? ld_hint(B.items + g0, ps) : 0;            // warp-uniform
      int32_t item1 = g0 + 1 < g1 ? ld_hint(B.items + g0 + 1, ps) : 0;
      int32_t s_c = 0, c_c = 0, gm_c = 0, r_c = 0;
      int64_t so_c = 0;
      if (g0 < g1) item_bounds(item, s_c, c_c, gm_c, r_c, so_c);
      for (int32_t it = g0; it < g1; ++it) {
        const int32_t item2 = it + 2 < g1 ? ld_hint(B.items + it + 2, ps) : 0;
        int32_t s_n = 0, c_n = 0, gm_n = 0, r_n = 0;
        int64_t so_n = 0;
        if (it + 1 < g1) item_bounds(item1, s_n, c_n, gm_n, r_n, so_n);
        if (item < 0) {
          // one row of a group of hub rows: the whole warp on it
          const int64_t pos = -(int64_t)item - 1;
          const double w_c = last ? __ldg(W + r_c) : 0.0;
          double v = cg_range<VT, 32, PIPE>(a.ci, va, X, s_c, c_c, c_c, 0.0, ps, pk);
          if (lane == 0) {
            if (!first) v += __ldcg(B.spart + pos);
            if (last) finish_w(r_c, v, w_c);
            else __stcg(B.spart + pos, v);
          }
        } else {
          const int32_t g = item;
          const int64_t idx = (int64_t)g * 32 + lane;
          const bool valid = idx < n;
          const double w_c = (last && valid) ? __ldg(W + r_c) : 0.0;
          const int32_t s0 = s_c, cnt0 = c_c;
          if (gm_c <= (sliced ? BIN_SLICED_LANE_ROWS : BIN_LANE_ROWS)) {
            const double init = (!first && valid) ? __ldcg(B.spart + idx) : 0.0;
            const int32_t lim = __reduce_max_sync(FULL, cnt0);
            double v;
            if (PIPE && sliced)   // slab of 32 x gm_c entries ending at so_c; every cnt0 <= gm_c
              v = cg_range_sliced<VT>(B.scol, reinterpret_cast<const VT*>(B.sval), X, so_c - 32ll * gm_c, cnt0, gm_c,
                                      ps, pk);
            else
              v = cg_range<VT, 1, PIPE>(a.ci, va, X, s0, cnt0, lim, init, ps, pk);
            if (valid) {
              if (last) finish_w(r_c, v, w_c);
              else __stcg(B.spart + idx, v);
            }
          } else {
            // 8 lanes per row, 4 rows per pass (groups whose longest row has more than 256
            // entries are split into single-row items when the items are built)
            for (int pp = 0; pp < 8; ++pp) {
              const int src = pp * 4 + (lane >> 3);
              const int32_t s = __shfl_sync(FULL, s0, src);
              const int32_t cnt = __shfl_sync(FULL, cnt0, src);
              const int vld = __shfl_sync(FULL, (int)valid, src);
              double v = cg_range<VT, 8, PIPE>(a.ci, va, X, s, cnt, __reduce_max_sync(FULL, cnt), 0.0, ps, pk);
              const int32_t r_s = __shfl_sync(FULL, r_c, src);
              const double w_s = __shfl_sync(FULL, w_c, src);
              if ((lane & 7) == 0 && vld) {
                const int64_t pos = (int64_t)g * 32 + src;
                if (!first) v += __ldcg(B.spart + pos);
                if (last) finish_w(r_s, v, w_s);
                else __stcg(B.spart + pos, v);
              }
            }
          }
        }
        item = item1;
        item1 = item2;
        s_c = s_n;
        c_c = c_n;
        gm_c = gm_n;
        r_c = r_n;
        so_c = so_n;
      }
    }
  } else {
    // the epilogue's vector entry (p_i, or b_i) is loaded with the row's values
    auto fin = [&](int64_t r_, double v_, double w_) {
      if (MODE == 1) {
        a.q[r_] = v_;
        acc = fma(w_, v_, acc);
      } else {
        const double ri = w_ - v_;
        a.r[r_] = ri;
        acc = MODE == 0 ? fma(w_, w_, acc) : fma(ri, ri, acc);
      }
    };
    if constexpr (SL) cg_rows_sliced<VT>(a, X, MODE == 1 ? a.p : a.b, fin);
    else cg_rows_pipe<VT>(a, va, X, MODE == 1 ? a.p : a.b, fin);
  }
  double v[1] = {acc};
  if (!cg_last_cta<1>(v, a.part, &S->cnt[MODE == 2 ? 2 : 0], sm, &is_last)) return;
  if (threadIdx.x != 0) return;
  if (MODE == 0) {
    S->bb = v[0];
  } else if (MODE == 2) {
    S->tt = v[0];
  } else {
    const double pq = v[0];
    if (!(pq > 0.0) || !isfinite(pq)) {
      S->status = ST_BREAKDOWN;
      S->done = 1;
      S->xupd = 0;
      S->pupd = 0;
      S->cont = 0;
      if (a.in_graph) cudaGraphSetConditional(a.cond, 0u);
    } else {
      S->alpha = S->rho / pq;
      S->xupd = 1;
    }
  }
}

// Natural order.  The pipelined row walk keeps two rows' loads live: up to 64 registers, 4 CTAs
// per SM (the grid is capped there too: fewer, longer thread walks measured faster than a full
// 8 CTAs per SM).
template <typename VT, int MODE, bool SL = false>
__global__ void __launch_bounds__(256, 4) cg_spmv_kernel(const CgArgs a) {
  __shared__ double sm[32];
  __shared__ int is_last;
  cg_spmv_body<VT, MODE, false, false, SL>(a, sm, &is_last);
}

template <typename VT, int MODE>
__global__ void __launch_bounds__(256, SPMV_BIN_CTAS_PER_SM) cg_spmv_bin_kernel(const CgArgs a) {
  __shared__ double sm[32];
  __shared__ int is_last;
  cg_spmv_body<VT, MODE, true, false>(a, sm, &is_last);
}

template <typename VT, int MODE>
__global__ void __launch_bounds__(256, SPMV_BIN_PIPE_CTAS_PER_SM) cg_spmv_bin_pipe_kernel(const CgArgs a) {
  __shared__ double sm[32];
  __shared__ int is_last;
  cg_spmv_body<VT, MODE, true, true>(a, sm, &is_last);
}

// The SpMV of a CG phase, binned or natural row order.

int cg_spmv_bin_warps(bool pipe) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (sms > 0 ? sms : 1) * (pipe ? SPMV_BIN_PIPE_CTAS_PER_SM : SPMV_BIN_CTAS_PER_SM) * 8;
}

template <typename VT, int MODE>
static void launch_spmv_mode(int grid, cudaStream_t st, const CgArgs& a) {
  // the binned grid must match the split: one warp per work item
  if (a.bin.perm && a.bin.pipe) cg_spmv_bin_pipe_kernel<VT, MODE><<<cg_spmv_bin_warps(true) / 8, 256, 0, st>>>(a);
  else if (a.bin.perm) cg_spmv_bin_kernel<VT, MODE><<<cg_spmv_bin_warps(false) / 8, 256, 0, st>>>(a);
  else if (a.bin.scol) cg_spmv_kernel<VT, MODE, true><<<grid, 256, 0, st>>>(a);   // natural order, sliced copy
  else cg_spmv_kernel<VT, MODE><<<grid, 256, 0, st>>>(a);
}

// Shared epilogue of the preconditioner kernels (last CTA, thread 0): update the scalars and
// the loop condition from rz = r.z and rr = r.r.
template <bool RESTART>
__device__ __forceinline__ void cg_precond_epilogue(const CgArgs& a, double rz, double rr, bool zero_b) {
  CgScalars* S = a.s;
  const double bnorm = sqrt(S->bb);
  S->rr = rr;
  if (zero_b) {
    S->status = ST_OK;
    S->done = 1;
    S->cont = 0;
    S->rr = 0.0;
    return;
  }
  const bool conv = sqrt(rr) <= S->tol * bnorm;
  int cont = 0;
  if (RESTART) {
    S->rho = rz;
    S->xupd = 0;
    S->pupd = 0;
  } else {
    S->it += 1;
    S->beta = conv ? 0.0 : rz / S->rho;
    if (!conv) S->rho = rz;
  }
  if (conv) {
    S->pupd = 0;
  } else if (S->it >= S->max_iter) {
    S->status = ST_NO_CONV;
    S->pupd = 0;
  } else if (!(S->rho > 0.0) || !isfinite(S->rho)) {
    S->status = ST_BREAKDOWN;
    S->pupd = 0;
  } else {
    S->pupd = RESTART ? 0 : 1;
    cont = 1;
  }
  S->cont = cont;
  if (!RESTART && a.in_graph) cudaGraphSetConditional(a.cond, (unsigned)cont);
}

// RESTART (I2): z = M^{-1} r, p = z, rho, rr.  Otherwise (B): r -= alpha q, z = M^{-1} r.
template <typename FT, int BS, bool RESTART>
__global__ void __launch_bounds__(256) cg_precond_kernel(const CgArgs a) {
  __shared__ double sm[64];
  __shared__ int is_last;
  CgScalars* S = a.s;
  if (*(volatile int*)&S->done) return;
  const Layout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t uM = unit_elems_minv(L);
  const FT* Mf = reinterpret_cast<const FT*>(a.minv);
  const double alpha = RESTART ? 0.0 : S->alpha;
  const bool zero_b = RESTART && S->bb == 0.0;
  constexpr int NSLOT = (BS > 0 && BS <= 32) ? 1 : 2;
  const int nslot = NSLOT == 1 ? 1 : L.S;
  double v0 = 0.0, v1 = 0.0;
  for (int64_t u = gw; u < L.n_units; u += tw) {
    double rv[2] = {0.0, 0.0}, zv[2];
    int64_t rows[2];
    bool ok[2] = {false, false};
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t >= nslot) break;
      bool vld;
      const int rh = unit_row(L, lane, t, vld);
      rows[t] = u * L.U + rh;
      ok[t] = vld && rows[t] < L.n;
      if (ok[t]) rv[t] = RESTART ? a.r[rows[t]] : fma(-alpha, a.q[rows[t]], a.r[rows[t]]);
    }
    unit_apply_inv<FT, BS, false>(L, Mf + u * uM, lane, rv, zv);
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t >= nslot) break;
      if (!ok[t]) continue;
      if (zero_b) {
        a.x[rows[t]] = 0.0;
        continue;
      }
      if (!RESTART) a.r[rows[t]] = rv[t];
      a.z[rows[t]] = zv[t];
      if (RESTART) a.p[rows[t]] = zv[t];
      v0 = fma(rv[t], zv[t], v0);
      v1 = fma(rv[t], rv[t], v1);
    }
  }
  double v[2] = {v0, v1};
  if (!cg_last_cta<2>(v, a.part, &S->cnt[1], sm, &is_last)) return;
  if (threadIdx.x != 0) return;
  cg_precond_epilogue<RESTART>(a, v[0], v[1], zero_b);
}


// Staged preconditioner kernel: a CTA walks tiles of TU warp units; thread 0 streams each
// tile's M^{-1} blocks and its r (and q) rows into shared memory with bulk asynchronous copies,
// NST tiles ahead, and the warps apply M^{-1} from shared memory.  All operands were written
// before this kernel started, so the bulk copies need no cross-proxy ordering.
constexpr int CGP_NST = 3;
struct CgPrecondPlan {
  int tu;          // warp units per tile
  int stage;       // bytes per stage
  int off_r;       // r rows within a stage
  int off_q;       // q rows within a stage
  int smem;        // dynamic shared memory
  int64_t tiles;   // tiles in the matrix
};

template <typename FT, int BS, bool RESTART>
__global__ void __launch_bounds__(256) cg_precond_tma_kernel(const CgArgs a, const CgPrecondPlan pl) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double sm[64];
  __shared__ int is_last;
  __shared__ int okflag;
  CgScalars* S = a.s;
  if (*(volatile int*)&S->done) return;
  const Layout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t uM = unit_elems_minv(L);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm);
  unsigned char* stages = dsm + 128;
  const double alpha = RESTART ? 0.0 : S->alpha;
  const bool zero_b = RESTART && S->bb == 0.0;
  constexpr int NSLOT = (BS > 0 && BS <= 32) ? 1 : 2;
  const int nslot = NSLOT == 1 ? 1 : L.S;
  const int64_t G = gridDim.x;
  const int64_t nj = pl.tiles > (int64_t)blockIdx.x ? (pl.tiles - blockIdx.x + G - 1) / G : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < CGP_NST; ++s) mbar_init(&mbar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int64_t j) {
    const int s = (int)(j % CGP_NST);
    const int64_t tile = blockIdx.x + j * G;
    const int64_t u0 = tile * pl.tu;
    const int64_t nu = min((int64_t)pl.tu, L.n_units - u0);
    const int64_t row0 = u0 * L.U;
    const int64_t rows = min(nu * L.U, L.n - row0);
    const uint32_t fb = (uint32_t)(nu * uM * (int64_t)sizeof(FT));
    const uint32_t vb = (uint32_t)(((rows * 8) + 15) & ~(int64_t)15);   // vectors are padded by the caller
    unsigned char* st = stages + (size_t)s * pl.stage;
    mbar_arrive_expect_tx(&mbar[s], fb + vb * (RESTART ? 1u : 2u));
    bulk_g2s(st, reinterpret_cast<const FT*>(a.minv) + u0 * uM, fb, &mbar[s]);
    bulk_g2s(st + pl.off_r, a.r + row0, vb, &mbar[s]);
    if (!RESTART) bulk_g2s(st + pl.off_q, a.q + row0, vb, &mbar[s]);
  };
  if (threadIdx.x == 0)
    for (int64_t j = 0; j < nj && j < CGP_NST; ++j) issue(j);
  uint32_t parity = 0u;
  double v0 = 0.0, v1 = 0.0;
  for (int64_t j = 0; j < nj; ++j) {
    const int s = (int)(j % CGP_NST);
    if (threadIdx.x == 0) okflag = mbar_wait_bounded(&mbar[s], (parity >> s) & 1u, 4000000000LL) ? 1 : 0;
    __syncthreads();
    parity ^= 1u << s;
    if (!okflag) {
      if (threadIdx.x == 0) {
        atomicCAS(&S->status, ST_OK, ST_TIMEOUT);
        for (int64_t t = j + 1; t < nj && t < j + CGP_NST; ++t) {
          const int s2 = (int)(t % CGP_NST);
          mbar_wait_bounded(&mbar[s2], (parity >> s2) & 1u, 4000000000LL);
        }
      }
      break;   // leaves this CTA's partials at zero; the status reports the failure
    }
    const int64_t tile = blockIdx.x + j * G;
    const int64_t u = tile * pl.tu + warp;
    const unsigned char* st = stages + (size_t)s * pl.stage;
    if (warp < pl.tu && u < L.n_units) {
      const double* sr = reinterpret_cast<const double*>(st + pl.off_r);
      const double* sq = reinterpret_cast<const double*>(st + pl.off_q);
      double rv[2] = {0.0, 0.0}, zv[2];
      int64_t rows[2];
      bool ok[2] = {false, false};
#pragma unroll
      for (int t = 0; t < NSLOT; ++t) {
        if (t >= nslot) break;
        bool vld;
        const int rh = unit_row(L, lane, t, vld);
        rows[t] = u * L.U + rh;
        ok[t] = vld && rows[t] < L.n;
        const int li = warp * L.U + rh;
        if (ok[t]) rv[t] = RESTART ? sr[li] : fma(-alpha, sq[li], sr[li]);
      }
      unit_apply_inv<FT, BS, true>(L, reinterpret_cast<const FT*>(st) + (int64_t)warp * uM, lane, rv, zv);
#pragma unroll
      for (int t = 0; t < NSLOT; ++t) {
        if (t >= nslot) break;
        if (!ok[t]) continue;
        if (zero_b) {
          a.x[rows[t]] = 0.0;
          continue;
        }
        if (!RESTART) a.r[rows[t]] = rv[t];
        a.z[rows[t]] = zv[t];
        if (RESTART) a.p[rows[t]] = zv[t];
        v0 = fma(rv[t], zv[t], v0);
        v1 = fma(rv[t], rv[t], v1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && j + CGP_NST < nj) issue(j + CGP_NST);
  }
  double v[2] = {v0, v1};
  if (!cg_last_cta<2>(v, a.part, &S->cnt[1], sm, &is_last)) return;
  if (threadIdx.x != 0) return;
  cg_precond_epilogue<RESTART>(a, v[0], v[1], zero_b);
}

// Warp-pipelined preconditioner kernel: every warp owns a contiguous run of warp units and
// streams each unit's M^{-1} block and its r and q rows into its own ring of NS shared-memory
// stages with bulk asynchronous copies (one mbarrier per stage, lane 0 issues), NS units
// ahead; the warp applies M^{-1} from shared memory.  Warps never wait for each other until
// the final reduction.  All operands were written before this kernel started, so the copies
// need no cross-proxy ordering.
//
// FUSED (kernel B without a kernel C): each warp also applies x += alpha p to its units' rows
// as it goes (alpha is known when the kernel starts); after the reduction every CTA waits for
// the last CTA's decision (beta and the update flag, published by a release add on S->gen that
// each CTA polls with acquire under a clock64 budget), then applies p = z + beta p to the rows
// its warps just preconditioned, whose z they wrote themselves.  The
// grid must be co-resident (a cooperative launch).  A wait that runs out of budget records
// ST_TIMEOUT and stops the solve (done, and the next SpMV ends the loop).
struct CgWarpPlan {
  int ns;          // stages per warp
  int stage;       // bytes per stage
  int off_r;       // r rows within a stage
  int off_q;       // q rows within a stage
  int smem;        // dynamic shared memory per CTA
  int64_t units;   // warp units in the matrix
};
constexpr int CGW_WARPS = 8;

template <typename FT, int BS, bool RESTART, bool FUSED = false>
__global__ void __launch_bounds__(256) cg_precond_wp_kernel(const CgArgs a, const CgWarpPlan pl) {
  static_assert(!(RESTART && FUSED), "the restart kernel has no kernel C to fuse");
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double sm[64];
  __shared__ int is_last;
  __shared__ unsigned gen0;
  __shared__ int go;
  CgScalars* S = a.s;
  if (*(volatile int*)&S->done) return;
  if (FUSED && threadIdx.x == 0) gen0 = ld_acquire_u32(&S->gen);   // before this CTA arrives
  const Layout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t uM = unit_elems_minv(L);
  const int64_t W = (int64_t)gridDim.x * CGW_WARPS;
  const int64_t gw = (int64_t)blockIdx.x * CGW_WARPS + warp;
  const int64_t u0 = pl.units * gw / W, u1 = pl.units * (gw + 1) / W;
  const int64_t nu = u1 - u0;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm) + warp * 8;               // up to 8 stages
  unsigned char* ring = dsm + 128 * 4 + (size_t)warp * pl.ns * pl.stage;      // 512 B of barriers
  const double alpha = RESTART ? 0.0 : S->alpha;
  const bool zero_b = RESTART && S->bb == 0.0;
  constexpr int NSLOT = (BS > 0 && BS <= 32) ? 1 : 2;
  const int nslot = NSLOT == 1 ? 1 : L.S;
  const uint32_t fb = (uint32_t)(uM * (int64_t)sizeof(FT));
  // FUSED: x += alpha p unit by unit, the unit's x and p rows (lane l: rows l and l + 32) loaded
  // one unit ahead with plain loads
  const bool xup = FUSED && ld_volatile_i32(&S->xupd);
  double xn[NSLOT], pn[NSLOT];
  auto xp_load = [&](int64_t i) {
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      const int64_t row = (u0 + i) * L.U + lane + 32 * t;
      const bool ok = lane + 32 * t < L.U && row < L.n;
      xn[t] = ok ? a.x[row] : 0.0;
      pn[t] = ok ? a.p[row] : 0.0;
    }
  };
  if (xup && nu > 0) xp_load(0);
  auto issue = [&](int64_t i, int st) {   // lane 0: unit u0 + i into stage st (= i mod ns)
    const int64_t u = u0 + i;
    const int64_t row0 = u * L.U;
    const int64_t rows = min((int64_t)L.U, L.n - row0);
    const uint32_t vb = (uint32_t)(((rows * 8) + 15) & ~(int64_t)15);   // vectors are padded by the caller
    unsigned char* dst = ring + (size_t)st * pl.stage;
    mbar_arrive_expect_tx(&mbar[st], fb + vb * (RESTART ? 1u : 2u));
    bulk_g2s(dst, reinterpret_cast<const FT*>(a.minv) + u * uM, fb, &mbar[st]);
    bulk_g2s(dst + pl.off_r, a.r + row0, vb, &mbar[st]);
    if (!RESTART) bulk_g2s(dst + pl.off_q, a.q + row0, vb, &mbar[st]);
  };
  if (lane == 0) {
    for (int st = 0; st < pl.ns; ++st) mbar_init(&mbar[st], 1);
    mbar_fence_init();
    for (int64_t i = 0; i < nu && i < pl.ns; ++i) issue(i, (int)i);
  }
  __syncwarp();
  double v0 = 0.0, v1 = 0.0;
  // stage of unit i is i mod ns and its phase parity (i / ns) mod 2, kept as running counters
  int st = 0;
  uint32_t parity = 0u;
  for (int64_t i = 0; i < nu; ++i) {
    const bool ok = mbar_wait_bounded(&mbar[st], parity, 4000000000LL);
    if (!__all_sync(FULL, ok)) {
      if (lane == 0) {
        atomicCAS(&S->status, ST_OK, ST_TIMEOUT);
        for (int64_t t = i + 1; t < nu && t < i + pl.ns; ++t)
          mbar_wait_bounded(&mbar[t % pl.ns], (uint32_t)((t / pl.ns) & 1), 4000000000LL);
      }
      break;   // this warp's partials stay short; the status reports the failure
    }
    const int64_t u = u0 + i;
    double xc[NSLOT], pc[NSLOT];
    if (xup) {
#pragma unroll
      for (int t = 0; t < NSLOT; ++t) {
        xc[t] = xn[t];
        pc[t] = pn[t];
      }
      if (i + 1 < nu) xp_load(i + 1);
    }
    const unsigned char* sbuf = ring + (size_t)st * pl.stage;
    const double* sr = reinterpret_cast<const double*>(sbuf + pl.off_r);
    const double* sq = reinterpret_cast<const double*>(sbuf + pl.off_q);
    double rv[2] = {0.0, 0.0}, zv[2];
    int64_t rows[2];
    bool okr[2] = {false, false};
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t >= nslot) break;
      bool vld;
      const int rh = unit_row(L, lane, t, vld);
      rows[t] = u * L.U + rh;
      okr[t] = vld && rows[t] < L.n;
      if (okr[t]) rv[t] = RESTART ? sr[rh] : fma(-alpha, sq[rh], sr[rh]);
    }
    unit_apply_inv<FT, BS, true>(L, reinterpret_cast<const FT*>(sbuf), lane, rv, zv);
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t >= nslot) break;
      if (!okr[t]) continue;
      if (zero_b) {
        a.x[rows[t]] = 0.0;
        continue;
      }
      if (!RESTART) a.r[rows[t]] = rv[t];
      a.z[rows[t]] = zv[t];
      if (RESTART) a.p[rows[t]] = zv[t];
      v0 = fma(rv[t], zv[t], v0);
      v1 = fma(rv[t], rv[t], v1);
    }
    if (xup) {
#pragma unroll
      for (int t = 0; t < NSLOT; ++t) {
        const int64_t row = u * L.U + lane + 32 * t;
        if (lane + 32 * t < L.U && row < L.n) a.x[row] = fma(alpha, pc[t], xc[t]);
      }
    }
    __syncwarp();   // every lane is done with the stage before it is refilled
    if (lane == 0 && i + pl.ns < nu) issue(i + pl.ns, st);
    if (++st == pl.ns) {
      st = 0;
      parity ^= 1u;
    }
  }
  double v[2] = {v0, v1};
  const bool last = cg_last_cta<2>(v, a.part, &S->cnt[1], sm, &is_last);
  if constexpr (!FUSED) {
    if (!last || threadIdx.x != 0) return;
    cg_precond_epilogue<RESTART>(a, v[0], v[1], zero_b);
  } else {
    if (threadIdx.x == 0) {
      go = 1;
      if (last) {
        cg_precond_epilogue<false>(a, v[0], v[1], false);
        red_release_add_u32(&S->gen, 1u);
      } else {
        const long long t0 = clock64();
        while (ld_acquire_u32(&S->gen) == gen0) {
          if (clock64() - t0 > a.budget) {
            atomicCAS(&S->status, ST_OK, ST_TIMEOUT);
            S->done = 1;
            go = 0;
            break;
          }
        }
      }
    }
    __syncthreads();
    if (!go) return;
    if (!ld_volatile_i32(&S->pupd)) return;
    const double beta = *(volatile const double*)&S->beta;
    // the rest of kernel C on this warp's rows (x was updated unit by unit above): 4 rows per
    // lane in flight
    const int64_t r0 = u0 * L.U, r1 = min(u1 * (int64_t)L.U, L.n);
    for (int64_t base = r0 + lane; base < r1; base += 4 * 32) {
      double pv[4], zv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t row = min(base + t * 32, r1 - 1);
        pv[t] = a.p[row];
        zv[t] = __ldcg(a.z + row);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t row = base + t * 32;
        if (row < r1) a.p[row] = fma(beta, pv[t], zv[t]);
      }
    }
  }
}

// C: x += alpha p (if due); p = z + beta p (if due).
__global__ void __launch_bounds__(256) cg_update_kernel(const CgArgs a) {
  const CgScalars* S = a.s;
  const int xupd = *(volatile const int*)&S->xupd;
  const int pupd = *(volatile const int*)&S->pupd;
  if (!xupd && !pupd) return;
  const double alpha = S->alpha, beta = S->beta;
  const int64_t n = a.lay.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += 4 * stride) {
    double pv[4], xv[4], zv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t row = min(base + t * stride, n - 1);
      pv[t] = a.p[row];
      xv[t] = a.x[row];
      zv[t] = pupd ? a.z[row] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t row = base + t * stride;
      if (row < n) {
        if (xupd) a.x[row] = fma(alpha, pv[t], xv[t]);
        if (pupd) a.p[row] = fma(beta, pv[t], zv[t]);
      }
    }
  }
}

// Resets the per-round flags and arms the loop condition from I2's decision.
__global__ void cg_arm_kernel(const CgArgs a) {
  cudaGraphSetConditional(a.cond, (unsigned)a.s->cont);
}

// ------------------------------------------------------------------ host side
struct CgGraph {
  cudaGraphExec_t exec;
  cudaGraph_t graph;
  CgArgs args;
  int g_spmv, g_prec, g_upd;
  bool tma;              // staged preconditioner kernel usable
  CgPrecondPlan pl;
  bool wp;               // warp-pipelined preconditioner kernel usable
  CgWarpPlan wpl;
  int fuse;              // shape's fuse_update: 0 default, 1 fused, 2 separate kernel C
  bool fac_f32;          // FP32 factors (the default then keeps kernel C separate)
  bool fused;            // kernel C runs as the fused tail of kernel B (decided at capture)
};

// Plan of the warp-pipelined preconditioner: NS stages of one warp unit each per warp, as
// deep as fits in about 110 KB per CTA.  Needs 16-byte aligned vector rows (U even).
static CgWarpPlan warp_plan(const Layout& L, bool fac_f32, int ring, bool* usable) {
  CgWarpPlan pl;
  auto up = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
  const int64_t unit_bytes = unit_elems_minv(L) * (fac_f32 ? 4 : 8);
  const int64_t vec = up((int64_t)L.U * 8 + 16, 128);
  pl.off_r = (int)up(unit_bytes, 128);
  pl.off_q = (int)(pl.off_r + vec);
  pl.stage = (int)(pl.off_q + vec);
  pl.units = L.n_units;
  pl.ns = (ring >= 2 && ring <= 4) ? ring : 4;   // ring: stages asked for (0: the deepest that fits)
  while (pl.ns > 2 && (int64_t)CGW_WARPS * pl.ns * pl.stage > 110 * 1024) --pl.ns;
  pl.smem = 512 + CGW_WARPS * pl.ns * pl.stage;
  *usable = (L.U % 2 == 0) && pl.smem <= 110 * 1024 + 512;
  return pl;
}

// Tile plan of the staged preconditioner kernel (about 24 KB per stage, 8 units per tile).
static CgPrecondPlan precond_plan(const Layout& L, bool fac_f32, bool* usable) {
  CgPrecondPlan pl;
  const int64_t unit_bytes = unit_elems_minv(L) * (fac_f32 ? 4 : 8);
  const int64_t vec_unit = (int64_t)L.U * 8;
  const int64_t budget = 24 * 1024;
  int64_t tu = budget / (unit_bytes + 2 * vec_unit);
  if (tu > 8) tu = 8;
  if (tu < 1) tu = 1;
  // the first row of every tile must be 16-byte aligned: an even tile when U is odd
  bool ok = true;
  if ((L.U & 1) && (tu & 1)) {
    if (tu > 1) tu -= 1;
    else ok = false;
  }
  auto up = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
  pl.tu = (int)tu;
  pl.off_r = (int)up(tu * unit_bytes, 128);
  pl.off_q = (int)(pl.off_r + up(tu * vec_unit + 16, 128));
  pl.stage = (int)(pl.off_q + up(tu * vec_unit + 16, 128));
  pl.smem = 128 + CGP_NST * pl.stage;
  pl.tiles = (L.n_units + tu - 1) / tu;
  if (pl.smem > 200 * 1024) ok = false;
  if (tu < 4) ok = false;   // too few warps busy per tile: the unstaged kernel is faster
  *usable = ok;
  return pl;
}

template <typename FT, int BS, bool RESTART>
static cudaError_t launch_precond(cudaStream_t cs, const CgGraph* g) {
  if (g->wp) {
    cudaError_t e = cudaFuncSetAttribute(cg_precond_wp_kernel<FT, BS, RESTART>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, g->wpl.smem);
    if (e != cudaSuccess) return e;
    cg_precond_wp_kernel<FT, BS, RESTART><<<g->g_prec, 256, g->wpl.smem, cs>>>(g->args, g->wpl);
    return cudaGetLastError();
  }
  if (g->tma) {
    cudaError_t e = cudaFuncSetAttribute(cg_precond_tma_kernel<FT, BS, RESTART>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, g->pl.smem);
    if (e != cudaSuccess) return e;
    cg_precond_tma_kernel<FT, BS, RESTART><<<g->g_prec, 256, g->pl.smem, cs>>>(g->args, g->pl);
  } else {
    cg_precond_kernel<FT, BS, RESTART><<<g->g_prec, 256, 0, cs>>>(g->args);
  }
  return cudaGetLastError();
}

// Kernel B with kernel C fused into its tail: a cooperative launch (every CTA resident, which
// its wait for the last CTA needs).
template <typename FT, int BS>
static cudaError_t launch_precond_fused(cudaStream_t cs, const CgGraph* g) {
  auto k = cg_precond_wp_kernel<FT, BS, false, true>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, g->wpl.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)g->g_prec);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)g->wpl.smem;
  cfg.stream = cs;
  cudaLaunchAttribute attr[1];
  memset(attr, 0, sizeof(attr));
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, g->args, g->wpl);
}

// Kernel C is fused into kernel B when the shape asks for it (by default with FP64 factors:
// on the 128^3 diffusion matrix at bs 16 the fused kernel was 2% faster with FP64 factors and
// 1.3% slower with FP32 factors, whose issue-bound apply pays for the extra x update) and B
// is the warp-ring kernel; its grid is then capped at the CTAs that can be resident at once
// (the warp split adapts to any grid), which the wait for the last CTA needs.
template <typename FT, int BS>
static bool fused_fits(CgGraph* g) {
  if (g->fuse == 2 || (g->fuse == 0 && g->fac_f32) || !g->wp) return false;
  auto k = cg_precond_wp_kernel<FT, BS, false, true>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, g->wpl.smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, (size_t)g->wpl.smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = 0, sms = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || occ < 1) return false;
  if ((int64_t)g->g_prec > (int64_t)occ * sms) g->g_prec = occ * sms;
  return true;
}

template <typename VT, typename FT, int BS>
static cudaError_t capture_body(cudaStream_t cs, CgGraph* g) {
  g->fused = fused_fits<FT, BS>(g);
  launch_spmv_mode<VT, 1>(g->g_spmv, cs, g->args);
  if (g->fused) return launch_precond_fused<FT, BS>(cs, g);
  cudaError_t e = launch_precond<FT, BS, false>(cs, g);
  if (e != cudaSuccess) return e;
  cg_update_kernel<<<g->g_upd, 256, 0, cs>>>(g->args);
  return cudaGetLastError();
}

template <typename VT, typename FT>
static cudaError_t capture_body_bs(cudaStream_t cs, CgGraph* g) {
  switch (g->args.lay.bs) {
    case 8: return capture_body<VT, FT, 8>(cs, g);
    case 16: return capture_body<VT, FT, 16>(cs, g);
    case 32: return capture_body<VT, FT, 32>(cs, g);
    case 64: return capture_body<VT, FT, 64>(cs, g);
    default: return capture_body<VT, FT, 0>(cs, g);
  }
}

template <typename VT, typename FT, int BS>
static cudaError_t launch_pre(cudaStream_t st, const CgGraph* g) {
  launch_spmv_mode<VT, 0>(g->g_spmv, st, g->args);
  return launch_precond<FT, BS, true>(st, g);
}

template <typename VT, typename FT>
static cudaError_t launch_pre_bs(cudaStream_t st, const CgGraph* g) {
  switch (g->args.lay.bs) {
    case 8: return launch_pre<VT, FT, 8>(st, g);
    case 16: return launch_pre<VT, FT, 16>(st, g);
    case 32: return launch_pre<VT, FT, 32>(st, g);
    case 64: return launch_pre<VT, FT, 64>(st, g);
    default: return launch_pre<VT, FT, 0>(st, g);
  }
}

static int sms_now() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int cg_graph_partials() { return sms_now() * 16 * 2 + 64; }

// Resident CTAs per SM of the natural-order SpMV (its grid is one wave: the grid-stride loop
// gives every CTA the same share of rows), at most SPMV_NAT_CTAS_PER_SM.
constexpr int SPMV_NAT_CTAS_PER_SM = 4;
static int spmv_ctas_per_sm(bool val_f32, int cap) {
  if (cap < 1 || cap > 8) cap = SPMV_NAT_CTAS_PER_SM;
  int occ = 0;
  const cudaError_t e =
      val_f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cg_spmv_kernel<float, 1>, 256, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cg_spmv_kernel<double, 1>, 256, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  return occ < 1 ? 1 : occ > cap ? cap : occ;
}

size_t cg_scalars_bytes() { return sizeof(CgScalars); }

// Builds and instantiates the loop graph for the given buffers.  ws_part must hold
// cg_graph_partials() doubles; scal points to cg_scalars_bytes() of device memory.
cudaError_t cg_graph_create(void** out, const Layout& L, const int32_t* rp, const int32_t* ci, const void* va,
                            bool val_f32, const void* minv, bool fac_f32, const double* b, double* x, double* r,
                            double* z, double* p, double* q, double* part, void* scal, const CgBinned* bin,
                            const CgShape& shape, cudaStream_t st) {
  CgGraph* g = new CgGraph();
  memset(g, 0, sizeof(*g));
  const int sms = sms_now();
  const int64_t n = L.n;
  g->g_spmv = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * spmv_ctas_per_sm(val_f32, shape.spmv_ctas_per_sm));
  g->pl = precond_plan(L, fac_f32, &g->tma);
  g->wpl = warp_plan(L, fac_f32, shape.ring_stages, &g->wp);
  if (g->wp) {
    // one wave of resident CTAs, at most one CTA per 8 units
    const int per_sm = std::max(1, std::min(8, (228 * 1024) / (g->wpl.smem + 1024)));
    g->g_prec = (int)std::min<int64_t>((L.n_units + 7) / 8, (int64_t)sms * per_sm);
  } else if (g->tma) {
    g->g_prec = (int)std::min<int64_t>(g->pl.tiles, (int64_t)sms * std::max(1, (200 * 1024) / g->pl.smem));
  } else {
    g->g_prec = (int)std::min<int64_t>((L.n_units + 7) / 8, (int64_t)sms * 8);
  }
  g->g_upd = (int)std::min<int64_t>((n + 1023) / 1024, (int64_t)sms * 8);
  g->fuse = shape.fuse_update;
  g->fac_f32 = fac_f32;
  if (g->g_spmv < 1) g->g_spmv = 1;
  if (g->g_prec < 1) g->g_prec = 1;
  if (g->g_upd < 1) g->g_upd = 1;
  CgArgs& a = g->args;
  a.lay = L;
  a.rp = rp;
  a.ci = ci;
  a.va = va;
  a.minv = minv;
  a.b = b;
  a.x = x;
  a.r = r;
  a.z = z;
  a.p = p;
  a.q = q;
  a.part = part;
  a.s = reinterpret_cast<CgScalars*>(scal);
  a.in_graph = 1;
  a.budget = wait_budget_cycles();
  if (bin && bin->perm) a.bin = *bin;
  else memset(&a.bin, 0, sizeof(a.bin));
  cudaError_t e = cudaGraphCreate(&g->graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&a.cond, g->graph, 0, 0);
  cudaGraphNode_t arm = nullptr, loop = nullptr;
  if (e == cudaSuccess) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    void* kargs[] = {&a};
    kp.func = (void*)cg_arm_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = kargs;
    e = cudaGraphAddKernelNode(&arm, g->graph, nullptr, 0, &kp);
  }
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = a.cond;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    e = cudaGraphAddNode(&loop, g->graph, &arm, nullptr, 1, np);
    if (e == cudaSuccess) body = np->conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) {
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        cudaError_t ce;
        if (!val_f32 && !fac_f32) ce = capture_body_bs<double, double>(cs, g);
        else if (!val_f32 && fac_f32) ce = capture_body_bs<double, float>(cs, g);
        else if (val_f32 && fac_f32) ce = capture_body_bs<float, float>(cs, g);
        else ce = capture_body_bs<float, double>(cs, g);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cs, &captured);
        if (e == cudaSuccess) e = ce;
      }
      cudaStreamDestroy(cs);
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    cudaGetLastError();
    return e;
  }
  (void)st;
  *out = g;
  return cudaSuccess;
}

bool cg_graph_fused(const void* h) { return h && static_cast<const CgGraph*>(h)->fused; }

void cg_graph_destroy(void* h) {
  CgGraph* g = static_cast<CgGraph*>(h);
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

// One round: I1, I2 (stream launches), the loop graph, T.  Scalars must hold it/max_iter/tol
// and status/done cleared by the caller before the first round.
cudaError_t cg_graph_round(void* h, bool val_f32, bool fac_f32, cudaStream_t st) {
  CgGraph* g = static_cast<CgGraph*>(h);
  const CgArgs& a = g->args;
  cudaError_t e;
  if (!val_f32 && !fac_f32) e = launch_pre_bs<double, double>(st, g);
  else if (!val_f32 && fac_f32) e = launch_pre_bs<double, float>(st, g);
  else if (val_f32 && fac_f32) e = launch_pre_bs<float, float>(st, g);
  else e = launch_pre_bs<float, double>(st, g);
  if (e != cudaSuccess) return e;
  e = cudaGraphLaunch(g->exec, st);
  if (e != cudaSuccess) return e;
  if (val_f32) launch_spmv_mode<float, 2>(g->g_spmv, st, a);
  else launch_spmv_mode<double, 2>(g->g_spmv, st, a);
  return cudaGetLastError();
}

// Keeps the GPU busy for about ns nanoseconds (a bounded sleep on the global timer), so that
// the launches the host enqueues meanwhile are waiting in the stream when it ends.
__global__ void cg_spacer_kernel(unsigned long long ns) {
  const unsigned long long t0 = globaltimer_ns();
  for (int i = 0; i < 100000 && globaltimer_ns() - t0 < ns; ++i) __nanosleep(500);
}

// Profiling round: the loop body kernels are launched one by one from the host with CUDA
// events around each (per-kernel times accumulate into ms[3]); same kernels and results.  The
// host reads the loop condition after every step, so each step starts with a 40 us spacer
// kernel: by the time it ends, the step's events and kernels are all enqueued, and the first
// kernel's event interval does not contain the host's launch latency.
template <typename VT, typename FT, int BS>
static cudaError_t eager_round_t(CgGraph* g, cudaStream_t st, double* ms, int* iters) {
  CgGraph eg = *g;
  eg.args.in_graph = 0;
  cudaError_t e = launch_pre<VT, FT, BS>(st, &eg);
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) cudaEventCreate(&ev[i]);
  int cont = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cont, &eg.args.s->cont, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  while (e == cudaSuccess && cont) {
    cg_spacer_kernel<<<1, 32, 0, st>>>(40000ull);
    cudaEventRecord(ev[0], st);
    launch_spmv_mode<VT, 1>(eg.g_spmv, st, eg.args);
    cudaEventRecord(ev[1], st);
    e = eg.fused ? launch_precond_fused<FT, BS>(st, &eg) : launch_precond<FT, BS, false>(st, &eg);
    cudaEventRecord(ev[2], st);
    if (!eg.fused) cg_update_kernel<<<eg.g_upd, 256, 0, st>>>(eg.args);   // fused: no kernel C
    cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cont, &eg.args.s->cont, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float t;
    for (int i = 0; i < (eg.fused ? 2 : 3); ++i) {   // fused: no update kernel to time
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] += t;
    }
    ++*iters;
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return e;
  if (std::is_same<VT, float>::value) launch_spmv_mode<float, 2>(eg.g_spmv, st, eg.args);
  else launch_spmv_mode<double, 2>(eg.g_spmv, st, eg.args);
  return cudaGetLastError();
}

template <typename VT, typename FT>
static cudaError_t eager_round_bs(CgGraph* g, cudaStream_t st, double* ms, int* iters) {
  switch (g->args.lay.bs) {
    case 8: return eager_round_t<VT, FT, 8>(g, st, ms, iters);
    case 16: return eager_round_t<VT, FT, 16>(g, st, ms, iters);
    case 32: return eager_round_t<VT, FT, 32>(g, st, ms, iters);
    case 64: return eager_round_t<VT, FT, 64>(g, st, ms, iters);
    default: return eager_round_t<VT, FT, 0>(g, st, ms, iters);
  }
}

// Full solve: rounds of (I1, I2, loop, T) with at most max_restarts restarts from x when the
// true residual is above tol.  Synchronises the stream.
cudaError_t cg_graph_solve(void* h, double tol, int max_iter, int max_restarts, bool val_f32, bool fac_f32,
                           cudaStream_t st, CgResult* res) {
  CgGraph* g = static_cast<CgGraph*>(h);
  CgScalars init;
  memset(&init, 0, sizeof(init));
  init.tol = tol;
  init.max_iter = max_iter;
  cudaError_t e = cudaMemcpyAsync(g->args.s, &init, sizeof(init), cudaMemcpyHostToDevice, st);
  int restarts = 0;
  CgScalars hs;
  memset(&hs, 0, sizeof(hs));
  const char* prof = getenv("PC_CG_PROFILE");
  const bool eager = prof && prof[0] == '1';
  double ms[3] = {0.0, 0.0, 0.0};
  int eager_iters = 0;
  for (;;) {
    if (e == cudaSuccess) {
      if (!eager) e = cg_graph_round(h, val_f32, fac_f32, st);
      else if (!val_f32 && !fac_f32) e = eager_round_bs<double, double>(g, st, ms, &eager_iters);
      else if (!val_f32 && fac_f32) e = eager_round_bs<double, float>(g, st, ms, &eager_iters);
      else if (val_f32 && fac_f32) e = eager_round_bs<float, float>(g, st, ms, &eager_iters);
      else e = eager_round_bs<float, double>(g, st, ms, &eager_iters);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, g->args.s, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const double bnorm = sqrt(hs.bb);
    if (hs.status != ST_OK || hs.bb == 0.0) break;
    if (hs.cont != 0) break;   // should not happen: the loop ended with the condition set
    if (sqrt(hs.tt) <= tol * bnorm) break;
    if (restarts >= max_restarts) {
      hs.status = ST_NO_CONV;
      break;
    }
    ++restarts;
    // next round: keep the iteration count, clear the round flags
    CgScalars nxt = hs;
    nxt.done = 0;
    nxt.xupd = 0;
    nxt.pupd = 0;
    nxt.cont = 0;
    nxt.cnt[0] = nxt.cnt[1] = nxt.cnt[2] = nxt.cnt[3] = 0u;
    e = cudaMemcpyAsync(g->args.s, &nxt, sizeof(nxt), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host copy source is on the stack
    if (e != cudaSuccess) return e;
  }
  res->status = hs.status;
  res->iterations = hs.it;
  res->restarts = restarts;
  res->rel_residual = hs.bb > 0.0 ? sqrt(hs.rr) / sqrt(hs.bb) : 0.0;
  res->true_rel_residual = hs.bb > 0.0 ? sqrt(hs.tt) / sqrt(hs.bb) : 0.0;
  for (int i = 0; i < 3; ++i) res->kernel_us[i] = eager_iters ? 1000.0 * ms[i] / eager_iters : 0.0;
  return cudaSuccess;
}

}  // namespace pc

// Persistent block-Jacobi preconditioned CG: the whole iteration runs in one cooperative
// launch.  Per step there are three grid-wide synchronisations:
//   A  q = A p (rows split by rows+nnz), partial p.q          -> allreduce -> alpha
//   B  r -= alpha q; z = M^{-1} r per warp unit; r.z, r.r     -> allreduce -> beta, ||r||
//   C  x += alpha p; p = z + beta p                           -> barrier
// (x's update is deferred from A/B to C; on convergence it is applied before exit.)
// The scalar recurrences follow Hestenes-Stiefel PCG exactly:
//   alpha = rho / p.q,  beta = rho' / rho,  stop when ||r|| <= tol ||b||,
// followed by the true residual b - A x and at most max_restarts restarts from x.
// All reductions are fixed-order, so a solve is bit-reproducible run to run.
//
// Streaming.  Inside a phase every warp works through its own sequence of chunks (32 CSR
// rows in A, one warp unit in B) with a private two-stage pipeline: lane 0 moves the
// chunk's read-only data (row-pointer/column/value windows, or the unit's M^{-1} block)
// global -> shared memory with bulk asynchronous copies that complete on the warp's
// mbarriers, one chunk ahead.  There is no CTA-wide synchronisation inside a phase, so the
// warps of an SM drift apart and FP64-pipe work of some overlaps the gathers and copies
// of others.  Vector operands (written by this kernel) are read with L2-coherent loads.
#pragma once

#include "pc_kernels.cuh"
#include "pc_tma.cuh"

// Build-time tuning knobs: minimum resident CTAs per SM (register budget) and whether the
// phases are separate device functions (kernel-level state is then saved once per phase
// and each phase gets the whole register budget).
#ifndef PCG_MIN_CTAS
#define PCG_MIN_CTAS 4
#endif
#ifdef PCG_PHASE_NOINLINE
#define PCG_PHASE_ATTR __device__ __noinline__
#else
#define PCG_PHASE_ATTR __device__ __forceinline__
#endif

namespace pc {

enum { SPMV_Q = 0, SPMV_RES = 1, SPMV_INIT = 2 };

struct PcgCtx {
  uint64_t* mbar;        // this warp's PCG_NSTW mbarriers
  unsigned char* stage;  // this warp's stages
  int32_t* chunkE;       // CSR offset at the start of each SpMV chunk of this CTA
  double* sm;
  int* flag;
  uint32_t parity;       // per-stage phase bits (warp-uniform)
  int bar;
  int64_t sa0, sa1, u0, u1, row0, row1;
  int nch;               // SpMV chunks of this CTA
  bool table;            // chunk table in shared memory
};

// Optional phase trace: CTA 0 records the time at kernel start and after every grid
// barrier (entry k = after barrier k, entry 0 = start).
__device__ __forceinline__ void trace_mark(const PcgArgs& a, const PcgCtx& c) {
  if (a.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && c.bar < a.trace_len)
    a.trace[c.bar] = globaltimer_ns();
}

__device__ __forceinline__ unsigned char* wstage_ptr(const PcgArgs& a, const PcgCtx& c, int s) {
  return c.stage + (size_t)s * a.sp.wstage;
}

// All lanes wait (bounded) for stage s; warp-uniform result.  The stage's parity flips
// only on success.
__device__ __forceinline__ bool warp_stage_wait(const PcgArgs& a, PcgCtx& c, int s) {
  const bool ok = mbar_wait_bounded(&c.mbar[s], (c.parity >> s) & 1u, a.budget);
  const bool all = __all_sync(FULL, ok);
  if (all) c.parity ^= 1u << s;
  else if ((threadIdx.x & 31) == 0 && atomicCAS(&a.gs->status, 0, ST_TIMEOUT) == 0) a.gs->where = -1;
  return all;
}

// After a timeout: lane 0 waits (bounded) for the copies of chunks j .. j+NSTW-1 that
// this warp issued and that are still in flight.
__device__ __forceinline__ void warp_drain(const PcgArgs& a, PcgCtx& c, int j, int nj) {
  if ((threadIdx.x & 31) != 0) return;
  for (int t = j; t < nj && t < j + PCG_NSTW; ++t) {
    const int s = t % PCG_NSTW;
    if (mbar_wait_bounded(&c.mbar[s], (c.parity >> s) & 1u, a.budget)) c.parity ^= 1u << s;
  }
}

__device__ __forceinline__ void chunk_bounds(const PcgArgs& a, const PcgCtx& c, int k, int64_t& r0, int64_t& r1,
                                             int64_t& e0, int64_t& e1) {
  r0 = c.sa0 + (int64_t)k * PCG_CHUNK;
  r1 = min(r0 + PCG_CHUNK, c.sa1);
  if (c.table) {
    e0 = c.chunkE[k];
    e1 = c.chunkE[k + 1];
  } else {
    e0 = __ldg(a.rp + r0);
    e1 = __ldg(a.rp + r1);
  }
}

// Lane 0: SpMV chunk k into stage s.
template <typename VT>
__device__ __forceinline__ void issue_chunk(const PcgArgs& a, const PcgCtx& c, int k, int s) {
  int64_t r0, r1, e0, e1;
  chunk_bounds(a, c, k, r0, r1, e0, e1);
  uint64_t* m = &c.mbar[s];
  if (e1 - e0 > a.sp.tnnz) {
    mbar_arrive_expect_tx(m, 0);   // direct chunk: read from global memory
    return;
  }
  const Window wr = make_window(a.rp, 4, r0, r1 + 1, a.lay.n + 1);
  const Window wc = make_window(a.ci, 4, e0, e1, a.nnz);
  const Window wv = make_window(a.va, (int)sizeof(VT), e0, e1, a.nnz);
  unsigned char* st = wstage_ptr(a, c, s);
  mbar_arrive_expect_tx(m, wr.bytes + wc.bytes + wv.bytes);
  if (wr.bytes) bulk_g2s(st, window_src(a.rp, 4, wr), wr.bytes, m);
  if (wc.bytes) bulk_g2s(st + a.sp.off_col, window_src(a.ci, 4, wc), wc.bytes, m);
  if (wv.bytes) bulk_g2s(st + a.sp.off_val, window_src(a.va, (int)sizeof(VT), wv), wv.bytes, m);
}

// Lane 0: M^{-1} of warp unit u into stage s.
template <typename FT>
__device__ __forceinline__ void issue_unit(const PcgArgs& a, const PcgCtx& c, int64_t u, int s) {
  const int64_t uM = unit_elems_minv(a.lay);
  const uint32_t bytes = (uint32_t)(uM * (int64_t)sizeof(FT));
  uint64_t* m = &c.mbar[s];
  mbar_arrive_expect_tx(m, bytes);
  bulk_g2s(wstage_ptr(a, c, s), reinterpret_cast<const FT*>(a.minv) + u * uM, bytes, m);
}

// Per-lane state of one SpMV chunk between "prefetch" (stage landed, first gathers
// issued) and "compute" (products, store).
struct ChunkState {
  int64_t row;
  int32_t rs;
  int32_t cnt;
  int32_t wmax;
  int32_t kind;     // 0 empty, 1 staged, 2 direct (too many entries for a stage)
  bool valid;
  double aux;       // p_row (SPMV_Q) or b_row
  double xv[8];     // gathered operands of the row's first 8 entries
};

// Wait for chunk j's stage, read its row pointers and first column indices from shared
// memory and issue the gathers of the first 8 entries.  Returns false on timeout.
template <int MODE, typename VT>
__device__ __forceinline__ bool spmv_prefetch(const PcgArgs& a, PcgCtx& c, int j, ChunkState& cs) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const double* src = MODE == SPMV_Q ? a.p : a.x;
  int64_t r0, r1, e0, e1;
  chunk_bounds(a, c, warp + j * PCG_NW, r0, r1, e0, e1);
  cs.row = r0 + lane;
  cs.valid = cs.row < r1;
  cs.aux = 0.0;
  if (cs.valid) cs.aux = MODE == SPMV_Q ? ld_vec(a.p + cs.row) : __ldg(a.b + cs.row);
  if (!warp_stage_wait(a, c, j % PCG_NSTW)) return false;
  cs.kind = e1 <= e0 ? 0 : (e1 - e0 > a.sp.tnnz ? 2 : 1);
  cs.rs = (int32_t)e0;
  cs.cnt = 0;
  cs.wmax = 0;
  if (cs.kind == 1) {
    const Window wr = make_window(a.rp, 4, r0, r1 + 1, a.lay.n + 1);
    const Window wc = make_window(a.ci, 4, e0, e1, a.nnz);
    const unsigned char* st = wstage_ptr(a, c, j % PCG_NSTW);
    const int32_t* srp = reinterpret_cast<const int32_t*>(st);
    const int32_t* scol = reinterpret_cast<const int32_t*>(st + a.sp.off_col);
    if (cs.valid) {
      const int64_t row = cs.row;
      cs.rs = (row >= wr.lo && row < wr.hi) ? srp[row - wr.lo] : __ldg(a.rp + row);
      const int32_t re = (row + 1 >= wr.lo && row + 1 < wr.hi) ? srp[row + 1 - wr.lo] : __ldg(a.rp + row + 1);
      cs.cnt = re - cs.rs;
    }
    cs.wmax = __reduce_max_sync(FULL, cs.cnt);
    const int last = max(cs.cnt, 1) - 1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int32_t kk = cs.rs + min(q, last);
      const int32_t cc = (kk >= wc.lo && kk < wc.hi) ? scol[kk - wc.lo] : ld_stream(a.ci + kk);
      cs.xv[q] = ld_vec(src + cc);
    }
  }
  return true;
}

// Entries 8.. of rows longer than 8 (out of line so the pipelined common path keeps its
// registers).
template <typename VT>
__device__ __noinline__ double spmv_tail(const PcgArgs& a, const double* src, const int32_t* scol, const VT* sval,
                                         Window wc, Window wv, int32_t rs, int32_t cnt, int32_t wmax, double acc) {
  const VT* gval = reinterpret_cast<const VT*>(a.va);
  const int last = max(cnt, 1) - 1;
  for (int k0 = 8; k0 < wmax; k0 += 8) {
    int32_t cc[8];
    VT vv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int32_t kk = rs + min(k0 + q, last);
      cc[q] = (kk >= wc.lo && kk < wc.hi) ? scol[kk - wc.lo] : ld_stream(a.ci + kk);
      vv[q] = (kk >= wv.lo && kk < wv.hi) ? sval[kk - wv.lo] : ld_stream(gval + kk);
    }
    double xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) xv[q] = ld_vec(src + cc[q]);
    const int rem = wmax - k0;   // warp-uniform
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q < rem) {
        const double pr = fma(from_ft(vv[q]), xv[q], acc);
        acc = (k0 + q < cnt) ? pr : acc;
      }
    }
  }
  return acc;
}

template <typename VT>
__device__ __noinline__ double spmv_row_direct(const PcgArgs& a, const double* src, int64_t row) {
  return spmv_row<VT, true>(a.rp, a.ci, reinterpret_cast<const VT*>(a.va), src, row);
}

// Products of chunk j (stage still resident), then the phase's store and dot term.
template <int MODE, typename VT>
__device__ __forceinline__ void spmv_compute(const PcgArgs& a, PcgCtx& c, int j, const ChunkState& cs,
                                             double& acc_dot) {
  const int warp = threadIdx.x >> 5;
  const double* src = MODE == SPMV_Q ? a.p : a.x;
  const VT* gval = reinterpret_cast<const VT*>(a.va);
  double acc = 0.0;
  if (cs.kind == 2) {
    if (cs.valid) acc = spmv_row_direct<VT>(a, src, cs.row);
  } else if (cs.kind == 1) {
    int64_t r0, r1, e0, e1;
    chunk_bounds(a, c, warp + j * PCG_NW, r0, r1, e0, e1);
    const Window wc = make_window(a.ci, 4, e0, e1, a.nnz);
    const Window wv = make_window(a.va, (int)sizeof(VT), e0, e1, a.nnz);
    const unsigned char* st = wstage_ptr(a, c, j % PCG_NSTW);
    const int32_t* scol = reinterpret_cast<const int32_t*>(st + a.sp.off_col);
    const VT* sval = reinterpret_cast<const VT*>(st + a.sp.off_val);
    const int last = max(cs.cnt, 1) - 1;
    // Warp-uniform trip count: a product slot is issued only if some lane of the warp
    // needs it (a fully masked FP64 instruction still costs FP64-pipe time).
    const int rem0 = cs.wmax;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q < rem0) {
        const int32_t kk = cs.rs + min(q, last);
        const VT v = (kk >= wv.lo && kk < wv.hi) ? sval[kk - wv.lo] : ld_stream(gval + kk);
        const double pr = fma(from_ft(v), cs.xv[q], acc);
        acc = (q < cs.cnt) ? pr : acc;
      }
    }
    if (cs.wmax > 8)   // rows longer than 8 entries (kept out of line: rare for stencils)
      acc = spmv_tail<VT>(a, src, scol, sval, wc, wv, cs.rs, cs.cnt, cs.wmax, acc);
  }
  if (cs.valid) {
    if (MODE == SPMV_Q) {
      st_vec(a.q + cs.row, acc);
      acc_dot = fma(cs.aux, acc, acc_dot);
    } else {
      const double ri = cs.aux - acc;
      st_vec(a.r + cs.row, ri);
      acc_dot = MODE == SPMV_RES ? fma(ri, ri, acc_dot) : fma(cs.aux, cs.aux, acc_dot);
    }
  }
}

// SpMV phase over this CTA's rows (chunk k to warp k mod NW).  MODE:
//   SPMV_Q    q = A p,      returns sum p_i q_i
//   SPMV_RES  r = b - A x,  returns sum r_i^2
//   SPMV_INIT r = b - A x,  returns sum b_i^2
template <int MODE, typename VT>
PCG_PHASE_ATTR bool spmv_phase(const PcgArgs& a, PcgCtx& c, double& out) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nj = c.nch > warp ? (c.nch - warp + PCG_NW - 1) / PCG_NW : 0;   // chunks of this warp
  double acc_dot = 0.0;
  if (lane == 0)
    for (int j = 0; j < nj && j < PCG_NSTW; ++j) issue_chunk<VT>(a, c, warp + j * PCG_NW, j);
  ChunkState cs;
  for (int j = 0; j < nj; ++j) {
    if (!spmv_prefetch<MODE, VT>(a, c, j, cs)) {
      warp_drain(a, c, j, min(nj, j + PCG_NSTW));
      break;
    }
    spmv_compute<MODE, VT>(a, c, j, cs, acc_dot);
    __syncwarp();
    if (lane == 0 && j + PCG_NSTW < nj) issue_chunk<VT>(a, c, warp + (j + PCG_NSTW) * PCG_NW, j % PCG_NSTW);
  }
  double v[1] = {acc_dot};
  if (!grid_allreduce<1>(v, a.part, a.gs, a.budget, c.sm, c.flag, c.bar++)) return false;
  trace_mark(a, c);
  out = v[0];
  return true;
}

// Preconditioner phase over this CTA's warp units (unit u0 + warp + j*NW to warp `warp`),
// RESTART: z = M^{-1} r, p = z; otherwise r -= alpha q, z = M^{-1} r.
// Returns r.z and r.r.
template <bool RESTART, typename FT, int BS>
PCG_PHASE_ATTR bool precond_phase(const PcgArgs& a, PcgCtx& c, double alpha, double& rz, double& rr) {
  const Layout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t uM = unit_elems_minv(L);
  const int64_t mine = c.u1 - c.u0 > warp ? (c.u1 - c.u0 - warp + PCG_NW - 1) / PCG_NW : 0;
  const int nj = (int)mine;
  const bool staged = a.sp.fac_smem != 0;
  // row slots per lane: 1 for blocks of <= 32 rows (known at compile time when BS > 0)
  constexpr int NSLOT = (BS > 0 && BS <= 32) ? 1 : 2;
  const int nslot = NSLOT == 1 ? 1 : L.S;
  double v0 = 0.0, v1 = 0.0;
  if (staged && lane == 0)
    for (int j = 0; j < nj && j < PCG_NSTW; ++j) issue_unit<FT>(a, c, c.u0 + warp + (int64_t)j * PCG_NW, j);
  // vector operands of the current and the next unit: r (and q) per row slot
  double cr[2] = {0.0, 0.0}, cq[2] = {0.0, 0.0};
  auto load_rq = [&](int64_t u, double (&r)[2], double (&q)[2]) {
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t >= nslot) break;
      bool vld;
      const int rh = unit_row(L, lane, t, vld);
      const int64_t row = u * L.U + rh;
      if (vld && row < L.n) {
        r[t] = ld_vec(a.r + row);
        if (!RESTART) q[t] = ld_vec(a.q + row);
      }
    }
  };
  for (int j = 0; j < nj; ++j) {
    const int s = j % PCG_NSTW;
    const int64_t u = c.u0 + warp + (int64_t)j * PCG_NW;
    load_rq(u, cr, cq);
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
      if (ok[t]) rv[t] = RESTART ? cr[t] : fma(-alpha, cq[t], cr[t]);
    }
    if (staged) {
      if (!warp_stage_wait(a, c, s)) {
        warp_drain(a, c, j, min(nj, j + PCG_NSTW));
        break;
      }
      unit_apply_inv<FT, BS, true>(L, reinterpret_cast<const FT*>(wstage_ptr(a, c, s)), lane, rv, zv);
    } else {
      unit_apply_inv<FT, BS, false>(L, reinterpret_cast<const FT*>(a.minv) + u * uM, lane, rv, zv);
    }
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t >= nslot) break;
      if (!ok[t]) continue;
      if (!RESTART) st_vec(a.r + rows[t], rv[t]);
      st_vec(a.z + rows[t], zv[t]);
      if (RESTART) st_vec(a.p + rows[t], zv[t]);
      v0 = fma(rv[t], zv[t], v0);
      v1 = fma(rv[t], rv[t], v1);
    }
    __syncwarp();
    if (staged && lane == 0 && j + PCG_NSTW < nj) issue_unit<FT>(a, c, u + (int64_t)PCG_NSTW * PCG_NW, s);
  }
  double v[2] = {v0, v1};
  if (!grid_allreduce<2>(v, a.part, a.gs, a.budget, c.sm, c.flag, c.bar++)) return false;
  trace_mark(a, c);
  rz = v[0];
  rr = v[1];
  return true;
}

template <typename VT, typename FT, int BS>
__global__ void __launch_bounds__(PCG_BLOCK, PCG_MIN_CTAS) pcg_kernel(const __grid_constant__ PcgArgs a) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ double sm[2 * 32];
  __shared__ int flag[4];
  const Layout& L = a.lay;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int G = gridDim.x;
  const int cta = blockIdx.x;
  const int64_t n = L.n;
  PcgCtx c;
  c.mbar = reinterpret_cast<uint64_t*>(dsm) + warp * PCG_NSTW;
  c.chunkE = reinterpret_cast<int32_t*>(dsm + 256);
  c.stage = dsm + 256 + PCG_TCAP * 4 + (size_t)warp * PCG_NSTW * a.sp.wstage;
  c.sm = sm;
  c.flag = flag;
  c.parity = 0u;
  c.bar = 0;
  const int64_t upc = (L.n_units + G - 1) / G;
  c.u0 = min((int64_t)cta * upc, L.n_units);
  c.u1 = min(c.u0 + upc, L.n_units);
  c.row0 = min(c.u0 * L.U, n);
  c.row1 = min(c.u1 * L.U, n);
  c.sa0 = a.split[cta];
  c.sa1 = a.split[cta + 1];
  c.nch = (int)((c.sa1 - c.sa0 + PCG_CHUNK - 1) / PCG_CHUNK);
  c.table = c.nch + 1 <= PCG_TCAP;
  if (lane == 0) {
    for (int s = 0; s < PCG_NSTW; ++s) mbar_init(&c.mbar[s], 1);
    mbar_fence_init();
  }
  if (c.table)
    for (int t = tid; t <= c.nch; t += blockDim.x)
      c.chunkE[t] = __ldg(a.rp + min(c.sa0 + (int64_t)t * PCG_CHUNK, c.sa1));
  __syncthreads();
  const double tol = a.tol;
  trace_mark(a, c);

  // ---- r = b - A x, ||b||^2
  double bb;
  if (!spmv_phase<SPMV_INIT, VT>(a, c, bb)) return;
  const double bnorm = sqrt(bb);
  if (bb == 0.0) {
    for (int64_t row = c.row0 + tid; row < c.row1; row += blockDim.x) st_vec(a.x + row, 0.0);
    if (cta == 0 && tid == 0) {
      a.out->status = ST_OK;
      a.out->iterations = 0;
      a.out->restarts = 0;
      a.out->rel_residual = 0.0;
      a.out->true_rel_residual = 0.0;
    }
    return;
  }

  int it = 0, restarts = 0, status = ST_OK;
  double rho = 0.0, rr = 0.0, tt = 0.0;
  for (;;) {
    // ---- (re)start: z = M^{-1} r, p = z, rho = r.z, rr = r.r
    if (!precond_phase<true, FT, BS>(a, c, 0.0, rho, rr)) return;
    bool conv = sqrt(rr) <= tol * bnorm;
    while (!conv) {
      if (it >= a.max_iter) {
        status = ST_NO_CONV;
        break;
      }
      if (!(rho > 0.0) || !isfinite(rho)) {
        status = ST_BREAKDOWN;
        break;
      }
      // ---- A: q = A p, p.q
      double pq;
      if (!spmv_phase<SPMV_Q, VT>(a, c, pq)) return;
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = ST_BREAKDOWN;
        break;
      }
      const double alpha = rho / pq;
      // ---- B: r -= alpha q; z = M^{-1} r; r.z, r.r
      double rz;
      if (!precond_phase<false, FT, BS>(a, c, alpha, rz, rr)) return;
      ++it;
      if (sqrt(rr) <= tol * bnorm) {
        for (int64_t row = c.row0 + tid; row < c.row1; row += blockDim.x)
          st_vec(a.x + row, fma(alpha, ld_vec(a.p + row), ld_vec(a.x + row)));
        if (!grid_allreduce<0>(nullptr, a.part, a.gs, a.budget, sm, flag, c.bar++)) return;
        trace_mark(a, c);
        conv = true;
        break;
      }
      const double beta = rz / rho;
      rho = rz;
      // ---- C: x += alpha p; p = z + beta p  (4 rows per thread in flight)
      for (int64_t base = c.row0 + tid; base < c.row1; base += 4 * (int64_t)blockDim.x) {
        double pv[4], xv[4], zv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t row = min(base + t * (int64_t)blockDim.x, c.row1 - 1);
          pv[t] = ld_vec(a.p + row);
          xv[t] = ld_vec(a.x + row);
          zv[t] = ld_vec(a.z + row);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t row = base + t * (int64_t)blockDim.x;
          if (row < c.row1) {
            st_vec(a.x + row, fma(alpha, pv[t], xv[t]));
            st_vec(a.p + row, fma(beta, pv[t], zv[t]));
          }
        }
      }
      if (!grid_allreduce<0>(nullptr, a.part, a.gs, a.budget, sm, flag, c.bar++)) return;
      trace_mark(a, c);
    }
    // ---- true residual r = b - A x
    if (!spmv_phase<SPMV_RES, VT>(a, c, tt)) return;
    if (!conv) break;                         // breakdown / no convergence: report and stop
    if (sqrt(tt) <= tol * bnorm) break;       // converged
    if (restarts >= a.max_restarts) {
      status = ST_NO_CONV;
      break;
    }
    ++restarts;
  }
  if (cta == 0 && tid == 0) {
    a.out->status = status;
    a.out->iterations = it;
    a.out->restarts = restarts;
    a.out->rel_residual = sqrt(rr) / bnorm;
    a.out->true_rel_residual = sqrt(tt) / bnorm;
  }
}

template <typename VT, typename FT>
const void* pcg_fn(int bs) {
  switch (bs) {
    case 8: return (const void*)pcg_kernel<VT, FT, 8>;
    case 16: return (const void*)pcg_kernel<VT, FT, 16>;
    case 32: return (const void*)pcg_kernel<VT, FT, 32>;
    case 64: return (const void*)pcg_kernel<VT, FT, 64>;
    default: return (const void*)pcg_kernel<VT, FT, 0>;
  }
}

template <typename VT, typename FT>
cudaError_t launch_pcg_t(const PcgArgs& a, int grid, int block, cudaStream_t st) {
  void* args[] = {const_cast<PcgArgs*>(&a)};
  const void* fn = pcg_fn<VT, FT>(a.lay.bs);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, a.sp.total);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, (size_t)a.sp.total, st);
}

template <typename VT, typename FT>
cudaError_t pcg_occupancy_t(const Layout& L, int block, int smem, int* ctas) {
  const void* fn = pcg_fn<VT, FT>(L.bs);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, block, (size_t)smem);
}

}  // namespace pc

// Batched block-Jacobi PCG: many independent SPD systems of uneven size, each with its own
// block size, set up (Sec. 3.2-3.3) and solved (Hestenes-Stiefel PCG, Sec. 3.7 residual)
// inside ONE persistent cooperative kernel launch that is captured in a CUDA graph.
//
// Work distribution.  The host scheduler gives every system a team of T co-resident CTAs
// (T a power of two, sized by the system's estimated work) and lays the teams out as
// consecutive "slots" in order of decreasing work per slot.  Each CTA of the persistent
// grid takes the next slot from a device counter, runs its share of that system (a
// contiguous range of warp units / rows) to completion and takes the next slot.  Teams
// synchronise through their own release/acquire counter; because slots are handed out in
// increasing order and every CTA is resident, the lowest unfinished team always has all of
// its members, so the waits cannot deadlock.  Every wait has a cycle budget after which the
// launch records PC_ERR_TIMEOUT and all waits give up.
//
// Reductions are fixed-order: warp xor tree, CTA sum, then each member adds the team's
// partials in rank order, so every member holds the same bits and reaches the same
// decisions (convergence, breakdown, restart) without a broadcast.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pc.h"
#include "pc_kernels.cuh"
#include "pc_tune.h"
#include "pc_setup_unit.cuh"

namespace pc {
namespace {

constexpr int BT = 512;   // threads per CTA
constexpr int BNW = BT / 32;

struct BSys {
  int64_t row0;   // first row in the concatenated arrays
  int64_t fac0;   // first factor element of the system
  int32_t n;      // rows
  int32_t bs;     // block size
  int32_t team;   // CTAs on this system
  int32_t slot0;  // first queue slot of the team
};

struct BArgs {
  const BSys* sys;
  const int32_t* slot_sys;   // queue slot -> system
  int32_t n_sys, n_slots;
  const int32_t* rp;         // global row pointers (global nnz offsets)
  const int32_t* ci;         // local column indices
  const double* va;
  const double* b;
  double* x;
  double *r, *z, *p, *q;     // workspace vectors, one entry per row
  void* minv;                // M^{-1} of every system, unit layout, FT
  double* part;              // [slot][2][4] team partial sums
  unsigned* cnt;             // [n_sys] team barrier counters
  unsigned long long* fail;  // [n_sys] smallest failing block (all ones: none)
  unsigned* queue;           // next slot
  int* err;                  // first launch-wide error (timeout)
  int32_t* o_status;         // [n_sys]
  int32_t* o_iters;          // [n_sys]
  int32_t* o_restarts;       // [n_sys]
  double* o_relres;          // [n_sys] true relative residual
  double tol, pivot_tol;
  int32_t max_iter, max_restarts;
  long long budget;
  int32_t setup_warps;       // warps per CTA with a shared-memory setup slot
  int32_t slot_bytes;        // shared memory per setup slot
  unsigned long long* prof;  // null, or PH_N phase accumulators (profiling mode)
  int32_t smem_bytes;        // dynamic shared memory of a CTA
  int32_t tc;                // FP32 factors: M^{-1} formed on the tensor cores (PC_PREC_TF32)
};

struct Team {
  int s, rank, T, slot0;
  unsigned phase;   // team barriers passed
  unsigned nred;    // team reductions done (partial-buffer parity)
};

// Launch-wide pointers and constants the phases need, copied once per CTA into shared
// memory (the phases are out-of-line functions; handing them the kernel parameter block
// by reference would make the compiler copy it to local memory).
struct Env {
  const int32_t* ci;
  const double* va;
  double* part;
  unsigned* cnt;
  unsigned long long* fail;
  int* err;
  long long budget;
  double tol, pivot_tol;
  int32_t max_iter, max_restarts;
  int32_t setup_warps, slot_bytes, smem_bytes;
  unsigned long long* prof;   // null, or per-phase nanoseconds summed over CTAs (profiling mode)
  int32_t tc;                 // FP32 factors: M^{-1} formed on the tensor cores (PC_PREC_TF32)
};

// Profiling mode: thread 0 of every CTA adds the time since its previous mark to a phase
// accumulator (globaltimer, ns).  Phases: 0 setup, 1 start (x0 = 0 pass), 2 SpMV,
// 3 unit pass (r, x, z), 4 p update, 5 true residual, 6 reductions and team waits,
// 7 queue and idle.
enum { PH_SETUP = 0, PH_START, PH_SPMV, PH_UNITS, PH_PUPD, PH_TRUE, PH_SYNC, PH_IDLE, PH_N };

__device__ __forceinline__ void prof_mark(const Env& e, int ph, unsigned long long& last) {
  if (e.prof != nullptr && threadIdx.x == 0) {
    const unsigned long long now = globaltimer_ns();
    atomicAdd(e.prof + ph, now - last);
    last = now;
  }
}

__device__ __forceinline__ double* part_at(const Env& e, int slot, unsigned parity) {
  return e.part + ((size_t)slot * 2 + (parity & 1u)) * 4;
}

// All CTAs of the team arrive; false if the wait ran out of budget or another wait did.
// The first wait of a team also covers its formation: a member may have to wait until the
// last member's CTA has finished its previous system, so it gets a longer budget.
__device__ __forceinline__ bool team_sync(const Env& e, Team& t, int* flag) {
  __syncthreads();
  if (t.T == 1) return true;
  if (threadIdx.x == 0) {
    const unsigned target = (t.phase + 1u) * (unsigned)t.T;
    red_release_add_u32(&e.cnt[t.s], 1u);
    const long long t0 = clock64();
    const long long limit = t.phase == 0 ? 16 * e.budget : e.budget;
    int good = 1;
    while ((int)(ld_acquire_u32(&e.cnt[t.s]) - target) < 0) {
      if (ld_volatile_i32(e.err) != 0 || clock64() - t0 > limit) {
        atomicCAS(e.err, 0, ST_TIMEOUT);
        good = 0;
        break;
      }
    }
    *flag = good;
  }
  __syncthreads();
  t.phase++;
  return *flag != 0;
}

// Sum of NV values over the team, identical bits in every thread of every member.
template <int NV>
__device__ __forceinline__ bool team_allreduce(const Env& e, Team& t, double* v, double* red, int* flag) {
  block_sum<NV>(v, red);
  if (t.T == 1) return true;
  const unsigned par = t.nred++;
  if (threadIdx.x == 0) {
    double* mine = part_at(e, t.slot0 + t.rank, par);
#pragma unroll
    for (int i = 0; i < NV; ++i) __stcg(mine + i, v[i]);
  }
  if (!team_sync(e, t, flag)) return false;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double acc = 0.0;
    for (int m = 0; m < t.T; ++m) acc += __ldcg(part_at(e, t.slot0 + m, par) + i);
    v[i] = acc;
  }
  return true;
}

// Row of the system's CSR: sum_e val[e] * x[col[e]] in storage order.  The trip count is
// the warp's longest row (all lanes run every chunk; shorter rows are masked), so the
// whole warp must call it.  x may have been written by other CTAs of the team before the
// last team barrier: that barrier's release (writer) -> acquire (thread 0 here) ->
// bar.sync chain orders those stores before these plain coherent loads, so the gathers
// may use L1 (never the read-only .nc path, which assumes data constant for the launch).
__device__ __forceinline__ double brow(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const double* __restrict__ va, const double* x, int64_t row, bool valid,
                                       int32_t s_idle) {
  const int32_t s0 = valid ? __ldg(rp + row) : s_idle;
  const int32_t e = valid ? __ldg(rp + row + 1) : s_idle;
  const int32_t cnt = e - s0;
  const int32_t s = cnt > 0 ? s0 : s_idle;   // an empty row loads (and ignores) a valid entry
  const int32_t wmax = __reduce_max_sync(FULL, cnt);
  double acc = 0.0;
  for (int32_t k0 = 0; k0 < wmax; k0 += 8) {
    int32_t c[8];
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int32_t k = s + min(k0 + t, max(cnt, 1) - 1);
      c[t] = __ldg(ci + k);
      v[t] = __ldg(va + k);
    }
    double xv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) xv[t] = x[c[t]];
    const int rem = wmax - k0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < rem) {
        const double pr = fma(v[t], xv[t], acc);
        acc = (k0 + t < cnt) ? pr : acc;
      }
    }
  }
  return acc;
}

// Staged rows: a warp copies the contiguous entry range of its 32 consecutive rows into its
// own shared-memory slice with coalesced loads, then every lane walks its row there.  With
// one row per lane and direct loads, each load instruction touches about one cache line per
// few lanes; staged, it touches one per 32 entries.  Only the gathers of x stay global.
constexpr int STAGE_CAP = 512;                                    // entries per warp slice
constexpr int STAGE_BYTES = STAGE_CAP * (int)(sizeof(double) + sizeof(int32_t));

__device__ __forceinline__ double brow_staged(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              const double* __restrict__ va, const double* x, int64_t row, bool valid,
                                              int32_t s_idle, unsigned char* slice) {
  const int lane = threadIdx.x & 31;
  const int32_t s0 = valid ? __ldg(rp + row) : 0;
  const int32_t e = valid ? __ldg(rp + row + 1) : 0;
  const int32_t cnt = e - s0;
  const int32_t wmax = __reduce_max_sync(FULL, cnt);
  if (wmax == 0) return 0.0;
  // rows of the warp are consecutive: the range starts at lane 0's first entry
  const int32_t e0 = __shfl_sync(FULL, s0, 0);
  const int32_t e1 = (int32_t)__reduce_max_sync(FULL, (unsigned)(valid ? e : 0));
  const int32_t T = e1 - e0;
  if (T > STAGE_CAP) return brow(rp, ci, va, x, row, valid, s_idle);
  double* sva = reinterpret_cast<double*>(slice);
  int32_t* sci = reinterpret_cast<int32_t*>(slice + STAGE_CAP * sizeof(double));
  for (int32_t k = lane; k < T; k += 32) {
    sci[k] = __ldg(ci + e0 + k);
    sva[k] = __ldg(va + e0 + k);
  }
  __syncwarp();
  const int32_t off = cnt > 0 ? s0 - e0 : 0;   // an empty or idle row reads (and ignores) entry 0
  double acc = 0.0;
  for (int32_t k0 = 0; k0 < wmax; k0 += 8) {
    int32_t c[8];
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int32_t k = off + min(k0 + t, max(cnt, 1) - 1);
      c[t] = sci[k];
      v[t] = sva[k];
    }
    double xv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) xv[t] = x[c[t]];
    const int rem = wmax - k0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < rem) {
        const double pr = fma(v[t], xv[t], acc);
        acc = (k0 + t < cnt) ? pr : acc;
      }
    }
  }
  __syncwarp();   // the slice is refilled by the next group
  return acc;
}

enum { U_INIT = 0, U_ITER = 1, U_RESTART = 2 };

// CTA-uniform description of this member's share of one system.  It lives in shared
// memory and the phases below are out-of-line functions, so that no phase carries the
// others' state in registers.
struct SysCtx {
  const int32_t* rp;   // the system's row pointers (global nnz offsets)
  const double* b;
  double *x, *r, *z, *p, *q;
  const void* Mf;      // the system's M^{-1} (FT)
  Layout L;
  int64_t u0, u1;      // member's warp units
  int64_t rl, rh;      // member's rows
  int32_t s_idle;      // a valid entry index of the system (loaded by idle lanes)
  int32_t s;           // system index
};

struct D2 {
  double a, b;
};

// Setup of the member's units: extraction + block Cholesky + M^{-1} (setup_unit).
template <typename FT>
__device__ __noinline__ void phase_setup(const Env& e, const SysCtx& c, unsigned char* dsm) {
  const int warp = threadIdx.x >> 5;
  const Layout L = c.L;
  // as many warps as this system's block size allows in the CTA's shared memory
  const int slot = (int)((setup_unit_smem(L, sizeof(FT)) + 15) & ~(size_t)15);
  int nw = e.smem_bytes / slot;
  nw = nw < BNW ? nw : BNW;
  nw = nw > e.setup_warps ? nw : e.setup_warps;
  if (warp >= nw) return;
  FT* As = reinterpret_cast<FT*>(dsm + (size_t)warp * slot);
  FT* Xs = As + (size_t)L.U * (L.bs + 1);
  FT* Mf = reinterpret_cast<FT*>(const_cast<void*>(c.Mf));
  const int64_t uM = unit_elems_minv(L);
  if constexpr (sizeof(FT) == 4) {
    if (e.tc) {
      for (int64_t u = c.u0 + warp; u < c.u1; u += nw)
        setup_unit<double, FT, FT, true>(L, u, c.rp, e.ci, e.va, e.pivot_tol, Mf + u * uM, nullptr, As, Xs,
                                         threadIdx.x & 31, &e.fail[c.s]);
      return;
    }
  }
  for (int64_t u = c.u0 + warp; u < c.u1; u += nw)
    setup_unit<double, FT, FT>(L, u, c.rp, e.ci, e.va, e.pivot_tol, Mf + u * uM, nullptr, As, Xs, threadIdx.x & 31,
                           &e.fail[c.s]);
}

// q = A p over the member's rows; returns this thread's share of p.q.
__device__ __noinline__ double phase_spmv(const Env& e, const SysCtx& c, unsigned char* dsm) {
  double pq = 0.0;
  const int64_t rl = c.rl, rh = c.rh;
  unsigned char* slice = dsm + (size_t)(threadIdx.x >> 5) * STAGE_BYTES;
  for (int64_t base = rl; base < rh; base += BT) {
    const int64_t row = base + threadIdx.x;
    const bool valid = row < rh;
    const double qi = brow_staged(c.rp, e.ci, e.va, c.p, row, valid, c.s_idle, slice);
    if (valid) {
      c.q[row] = qi;
      pq = fma(c.p[row], qi, pq);
    }
  }
  return pq;
}

// t = b - A x over the member's rows, stored in r; returns this thread's share of t.t.
__device__ __noinline__ double phase_true_residual(const Env& e, const SysCtx& c, unsigned char* dsm) {
  double tt = 0.0;
  const int64_t rl = c.rl, rh = c.rh;
  unsigned char* slice = dsm + (size_t)(threadIdx.x >> 5) * STAGE_BYTES;
  for (int64_t base = rl; base < rh; base += BT) {
    const int64_t row = base + threadIdx.x;
    const bool valid = row < rh;
    const double ax = brow_staged(c.rp, e.ci, e.va, c.x, row, valid, c.s_idle, slice);
    if (valid) {
      const double ti = __ldg(c.b + row) - ax;
      c.r[row] = ti;
      tt = fma(ti, ti, tt);
    }
  }
  return tt;
}

// p = z + beta p over the member's rows.
__device__ __noinline__ void phase_p_update(const SysCtx& c, double beta) {
  double* p = c.p;
  const double* z = c.z;
  for (int64_t row = c.rl + threadIdx.x; row < c.rh; row += BT) p[row] = fma(beta, p[row], z[row]);
}

// Warp-unit pass over the member's units: r update (U_ITER: r -= alpha q, x += alpha p),
// z = M^{-1} r, p = z (U_INIT / U_RESTART; U_INIT also sets x = 0, r = b), and this
// thread's shares of r.z and r.r.
template <typename FT, int BS, int MODE>
__device__ __noinline__ D2 phase_units(const SysCtx& c, double alpha) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const Layout L = c.L;
  const int64_t uM = unit_elems_minv(L);
  const FT* Mf = reinterpret_cast<const FT*>(c.Mf);
  double* xs = c.x;
  double* rs = c.r;
  double* zs = c.z;
  double* ps = c.p;
  const double* qs = c.q;
  double v0 = 0.0, v1 = 0.0;
  for (int64_t u = c.u0 + warp; u < c.u1; u += BNW) {
    double rv[2] = {0.0, 0.0}, zv[2];
    int64_t rows[2];
    bool ok[2] = {false, false};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (t >= L.S) break;
      bool vld;
      const int rh = unit_row(L, lane, t, vld);
      rows[t] = u * L.U + rh;
      ok[t] = vld && rows[t] < L.n;
      if (ok[t]) {
        if (MODE == U_INIT) rv[t] = __ldg(c.b + rows[t]);
        else if (MODE == U_RESTART) rv[t] = rs[rows[t]];
        else rv[t] = fma(-alpha, qs[rows[t]], rs[rows[t]]);
      }
    }
    unit_apply_inv<FT, BS, false>(L, Mf + u * uM, lane, rv, zv);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (t >= L.S || !ok[t]) continue;
      const int64_t row = rows[t];
      if (MODE == U_INIT) {
        xs[row] = 0.0;
        rs[row] = rv[t];
      } else if (MODE == U_ITER) {
        xs[row] = fma(alpha, ps[row], xs[row]);
        rs[row] = rv[t];
      }
      zs[row] = zv[t];
      if (MODE != U_ITER) ps[row] = zv[t];
      v0 = fma(rv[t], zv[t], v0);
      v1 = fma(rv[t], rv[t], v1);
    }
  }
  return D2{v0, v1};
}

// One member's share of one system: setup of its units, then PCG with true-residual
// restarts.  Every member takes the same decisions (identical reduced bits).
template <typename FT, int BS>
__device__ __noinline__ void solve_system(const Env& e, const SysCtx& c, Team t, unsigned char* dsm,
                                          double* red, int* flag, int32_t* o_status, int32_t* o_iters,
                                          int32_t* o_restarts, double* o_relres) {
  int status = ST_OK, it = 0, restarts = 0;
  double relres = -1.0;   // -1: not computed (setup failure, timeout)
  unsigned long long last = e.prof != nullptr && threadIdx.x == 0 ? globaltimer_ns() : 0ull;

  phase_setup<FT>(e, c, dsm);
  __syncthreads();
  prof_mark(e, PH_SETUP, last);

  // x0 = 0: r = b, z = M^{-1} r, p = z; ||b||^2, rho = r.z
  double v[2];
  {
    const D2 d = phase_units<FT, BS, U_INIT>(c, 0.0);
    v[0] = d.b;
    v[1] = d.a;
  }
  prof_mark(e, PH_START, last);
  const bool ok0 = team_allreduce<2>(e, t, v, red, flag);
  prof_mark(e, PH_SYNC, last);
  if (!ok0) {
    status = ST_TIMEOUT;
  } else if (*(volatile unsigned long long*)&e.fail[t.s] != ~0ull) {
    status = ST_NOT_SPD;
  } else if (v[0] == 0.0) {
    relres = 0.0;   // b = 0: x = 0 is exact
  } else {
    const double bnorm = sqrt(v[0]);
    double rho = v[1];
    double rr = v[0];
    for (;;) {
      // CG iterations until the recurrence residual meets the tolerance
      while (!(sqrt(rr) <= e.tol * bnorm)) {
        if (it >= e.max_iter) {
          status = ST_NO_CONV;
          break;
        }
        if (!(rho > 0.0) || !isfinite(rho)) {
          status = ST_BREAKDOWN;
          break;
        }
        double pq[1] = {phase_spmv(e, c, dsm)};
        prof_mark(e, PH_SPMV, last);
        const bool ok1 = team_allreduce<1>(e, t, pq, red, flag);
        prof_mark(e, PH_SYNC, last);
        if (!ok1) {
          status = ST_TIMEOUT;
          break;
        }
        if (!(pq[0] > 0.0) || !isfinite(pq[0])) {
          status = ST_BREAKDOWN;
          break;
        }
        const double alpha = rho / pq[0];
        const D2 d = phase_units<FT, BS, U_ITER>(c, alpha);
        double w[2] = {d.a, d.b};
        prof_mark(e, PH_UNITS, last);
        const bool ok2 = team_allreduce<2>(e, t, w, red, flag);
        prof_mark(e, PH_SYNC, last);
        if (!ok2) {
          status = ST_TIMEOUT;
          break;
        }
        ++it;
        rr = w[1];
        if (sqrt(rr) <= e.tol * bnorm) break;
        const double beta = w[0] / rho;
        rho = w[0];
        phase_p_update(c, beta);
        prof_mark(e, PH_PUPD, last);
        const bool ok3 = team_sync(e, t, flag);
        prof_mark(e, PH_SYNC, last);
        if (!ok3) {
          status = ST_TIMEOUT;
          break;
        }
      }
      if (status == ST_TIMEOUT) break;
      // True residual t = b - A x (kept in r for a restart); also reported when the
      // iteration stopped without convergence.  Every exit from the loop above follows a
      // team barrier that came after the last x update, so the gathers of x are safe.
      double tv[1] = {phase_true_residual(e, c, dsm)};
      prof_mark(e, PH_TRUE, last);
      const bool ok4 = team_allreduce<1>(e, t, tv, red, flag);
      prof_mark(e, PH_SYNC, last);
      if (!ok4) {
        status = ST_TIMEOUT;
        break;
      }
      relres = sqrt(tv[0]) / bnorm;
      if (status != ST_OK) break;
      if (sqrt(tv[0]) <= e.tol * bnorm) break;
      if (restarts >= e.max_restarts) {
        status = ST_NO_CONV;
        break;
      }
      ++restarts;
      __syncthreads();
      const D2 d = phase_units<FT, BS, U_RESTART>(c, 0.0);
      double w[2] = {d.a, d.b};
      if (!team_allreduce<2>(e, t, w, red, flag)) {
        status = ST_TIMEOUT;
        break;
      }
      rho = w[0];
      rr = w[1];
    }
  }
  if (status == ST_TIMEOUT) relres = -1.0;
  if (t.rank == 0 && threadIdx.x == 0) {
    o_status[t.s] = status;
    o_iters[t.s] = it;
    o_restarts[t.s] = restarts;
    o_relres[t.s] = relres;
  }
  __syncthreads();
}

template <typename FT>
__global__ void __launch_bounds__(BT, 2) batched_kernel(const __grid_constant__ BArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[2 * 32];
  __shared__ SysCtx ctx;
  __shared__ Env env;
  __shared__ int s_slot;
  __shared__ int flag;
  if (threadIdx.x == 0) {
    env.ci = a.ci;
    env.va = a.va;
    env.part = a.part;
    env.cnt = a.cnt;
    env.fail = a.fail;
    env.err = a.err;
    env.budget = a.budget;
    env.tol = a.tol;
    env.pivot_tol = a.pivot_tol;
    env.max_iter = a.max_iter;
    env.max_restarts = a.max_restarts;
    env.setup_warps = a.setup_warps;
    env.slot_bytes = a.slot_bytes;
    env.prof = a.prof;
    env.smem_bytes = a.smem_bytes;
    env.tc = a.tc;
  }
  unsigned long long idle_from = a.prof != nullptr && threadIdx.x == 0 ? globaltimer_ns() : 0ull;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_slot = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int slot = s_slot;
    if (slot >= a.n_slots) break;
    if (a.prof != nullptr && threadIdx.x == 0) atomicAdd(a.prof + PH_IDLE, globaltimer_ns() - idle_from);
    const int s = __ldg(a.slot_sys + slot);
    const BSys d = a.sys[s];
    Team t;
    t.s = s;
    t.T = d.team;
    t.slot0 = d.slot0;
    t.rank = slot - d.slot0;
    t.phase = 0;
    t.nred = 0;
    if (d.n == 0) {
      if (t.rank == 0 && threadIdx.x == 0) {
        a.o_status[s] = ST_OK;
        a.o_iters[s] = 0;
        a.o_restarts[s] = 0;
        a.o_relres[s] = 0.0;
      }
      continue;
    }
    if (threadIdx.x == 0) {
      SysCtx& c = ctx;
      c.L = make_layout(d.n, d.bs);
      c.u0 = c.L.n_units * t.rank / t.T;
      c.u1 = c.L.n_units * (t.rank + 1) / t.T;
      c.rl = c.u0 * c.L.U < c.L.n ? c.u0 * c.L.U : c.L.n;
      c.rh = c.u1 * c.L.U < c.L.n ? c.u1 * c.L.U : c.L.n;
      c.rp = a.rp + d.row0;
      c.b = a.b + d.row0;
      c.x = a.x + d.row0;
      c.r = a.r + d.row0;
      c.z = a.z + d.row0;
      c.p = a.p + d.row0;
      c.q = a.q + d.row0;
      c.Mf = sizeof(FT) == 4 ? (const void*)(reinterpret_cast<const float*>(a.minv) + d.fac0)
                             : (const void*)(reinterpret_cast<const double*>(a.minv) + d.fac0);
      c.s_idle = __ldg(c.rp);
      c.s = s;
    }
    __syncthreads();
    switch (d.bs) {
      case 4: solve_system<FT, 4>(env, ctx, t, dsm, red, &flag, a.o_status, a.o_iters, a.o_restarts, a.o_relres); break;
      case 8: solve_system<FT, 8>(env, ctx, t, dsm, red, &flag, a.o_status, a.o_iters, a.o_restarts, a.o_relres); break;
      case 16: solve_system<FT, 16>(env, ctx, t, dsm, red, &flag, a.o_status, a.o_iters, a.o_restarts, a.o_relres); break;
      case 32: solve_system<FT, 32>(env, ctx, t, dsm, red, &flag, a.o_status, a.o_iters, a.o_restarts, a.o_relres); break;
      case 64: solve_system<FT, 64>(env, ctx, t, dsm, red, &flag, a.o_status, a.o_iters, a.o_restarts, a.o_relres); break;
      default: solve_system<FT, 0>(env, ctx, t, dsm, red, &flag, a.o_status, a.o_iters, a.o_restarts, a.o_relres); break;
    }
    if (a.prof != nullptr && threadIdx.x == 0) idle_from = globaltimer_ns();
  }
}

// Resets the launch's counters (part of the captured graph).
__global__ void batched_reset(unsigned* queue, int* err, unsigned* cnt, unsigned long long* fail, int n_sys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *queue = 0u;
    *err = 0;
  }
  for (int s = i; s < n_sys; s += gridDim.x * blockDim.x) {
    cnt[s] = 0u;
    fail[s] = ~0ull;
  }
}

// CSR checks of the concatenated batch: row pointers non-decreasing and inside [0, nnz],
// every local column index inside its system, columns strictly increasing within a row and
// the diagonal stored.  bad[0] counts violations.
__global__ void batched_validate(const int64_t* __restrict__ sys_row, int n_sys, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, int64_t nnz, unsigned* bad) {
  const int s = blockIdx.x;
  if (s >= n_sys) return;
  const int64_t r0 = sys_row[s], r1 = sys_row[s + 1];
  const int32_t n = (int32_t)(r1 - r0);
  unsigned nbad = 0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const int32_t e0 = rp[row], e1 = rp[row + 1];
    if (e0 < 0 || e1 < e0 || (int64_t)e1 > nnz) {
      ++nbad;
      continue;
    }
    const int32_t lr = (int32_t)(row - r0);   // the row's local index (its diagonal column)
    int32_t prev = -1;
    bool diag = false;
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t c = ci[e];
      if (c < 0 || c >= n || c <= prev) ++nbad;   // out of range, or not strictly increasing
      diag = diag || c == lr;
      prev = c;
    }
    if (!diag) ++nbad;
  }
  if (nbad) atomicAdd(bad, nbad);
}

}  // namespace
}  // namespace pc

// ------------------------------------------------------------------ host side
using pc::BSys;

struct pc_batch_handle {
  int32_t n_sys = 0;
  int64_t n_rows = 0, nnz = 0;
  int32_t prec = 0;
  bool fac_f32 = false;
  int grid = 0, ctas_per_sm = 0, team_max = 0;
  int n_slots = 0;
  pc::BArgs args{};
  int smem = 0;
  // device memory (library-owned)
  BSys* sys = nullptr;
  int32_t* slot_sys = nullptr;
  double* work = nullptr;   // r, z, p, q
  void* minv = nullptr;
  double* part = nullptr;
  unsigned* cnt = nullptr;
  unsigned long long* fail = nullptr;
  unsigned* misc = nullptr;   // queue, err, bad
  int32_t* o_restarts = nullptr;
  unsigned long long* prof = nullptr;   // PC_BATCH_PROFILE=1: phase accumulators
  int32_t* d_status = nullptr;
  int32_t* d_iters = nullptr;
  double* d_relres = nullptr;
  // host copies
  std::vector<BSys> hsys;
  std::vector<int32_t> hslot;
  // captured launch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  double g_tol = -1.0;
  int32_t g_max_iter = -1;
};

namespace {

pc_status bfrom(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
}

#define PCB_TRY(expr)                          \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) return bfrom(_e);   \
  } while (0)

template <typename T>
pc_status balloc(T** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    return bfrom(e);
  }
  return PC_OK;
}

long long batch_budget() {
  const char* e = getenv("PC_WAIT_BUDGET");
  if (e) {
    const long long v = atoll(e);
    if (v > 0) return v;
  }
  return 4000000000LL;
}

int g_batch_ctas_per_sm = 0;   // 0: occupancy maximum
int g_batch_team_max = 0;      // 0: default
double g_batch_split = 0.0;    // 0: default slots-per-CTA target
int g_batch_setup_kb = 0;      // 0: default shared-memory budget for setup slots (KB)

// Launch shape chosen by pc_batch_autotune for a batch signature on a device with sms SMs.
struct Tuned {
  int32_t n_sys;
  int64_t n_rows, nnz;
  int32_t prec, sms;
  int32_t ctas_per_sm, team_max, setup_kb;
  double split;
};
std::mutex g_tuned_mu;
std::vector<Tuned> g_tuned;

bool same_batch(const Tuned& a, const Tuned& b) {
  return a.n_sys == b.n_sys && a.n_rows == b.n_rows && a.nnz == b.nnz && a.prec == b.prec && a.sms == b.sms;
}

void put_tuned(const Tuned& t) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  for (Tuned& e : g_tuned)
    if (same_batch(e, t)) {
      e = t;
      return;
    }
  g_tuned.push_back(t);
}

bool find_tuned(const pc_batch* B, int32_t prec, Tuned* out) {
  pc::tune_autoload();
  Tuned k{};
  k.n_sys = B->n_sys;
  k.n_rows = B->n_rows;
  k.nnz = B->nnz;
  k.prec = prec;
  k.sms = pc::current_sms();
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  for (const Tuned& t : g_tuned)
    if (same_batch(t, k)) {
      *out = t;
      return true;
    }
  return false;
}

}  // namespace

namespace pc {

bool batch_tune_parse(const std::map<std::string, std::string>& kv) {
  auto num = [&](const char* k, double* v) {
    auto it = kv.find(k);
    if (it == kv.end() || it->second.empty()) return false;
    char* end = nullptr;
    *v = strtod(it->second.c_str(), &end);
    return end != it->second.c_str() && *end == '\0' && std::isfinite(*v);
  };
  double ns, nr, nz, pr, sm, occ, team, kb, split;
  if (!num("n_sys", &ns) || !num("n_rows", &nr) || !num("nnz", &nz) || !num("prec", &pr) || !num("sms", &sm) ||
      !num("ctas_per_sm", &occ) || !num("team_max", &team) || !num("setup_kb", &kb) || !num("split", &split))
    return false;
  if (ns < 1 || nr < 1 || nz < 0 || pr < 0 || pr > 2 || occ < 0 || occ > 64 || team < 1 || team > 1024 || kb < 1 ||
      kb > 228 || !(split > 0.0) || split > 64.0)
    return false;
  Tuned t{(int32_t)ns, (int64_t)nr, (int64_t)nz, (int32_t)pr, (int32_t)sm, (int32_t)occ, (int32_t)team, (int32_t)kb,
          split};
  put_tuned(t);
  return true;
}

void batch_tune_lines(std::string& out) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  char buf[512];
  for (const Tuned& t : g_tuned) {
    snprintf(buf, sizeof buf,
             "{\"kind\": \"batch\", \"n_sys\": %d, \"n_rows\": %lld, \"nnz\": %lld, \"prec\": %d, \"sms\": %d, "
             "\"ctas_per_sm\": %d, \"team_max\": %d, \"setup_kb\": %d, \"split\": %.6g}\n",
             t.n_sys, (long long)t.n_rows, (long long)t.nnz, t.prec, t.sms, t.ctas_per_sm, t.team_max, t.setup_kb,
             t.split);
    out += buf;
  }
}

}  // namespace pc

extern "C" {

void pc_batch_set_tuning(int32_t ctas_per_sm, int32_t team_max, double slots_per_cta) {
  g_batch_ctas_per_sm = ctas_per_sm > 0 ? ctas_per_sm : 0;
  g_batch_team_max = team_max > 0 ? team_max : 0;
  g_batch_split = slots_per_cta > 0.0 ? slots_per_cta : 0.0;
}

void pc_batch_set_setup_smem(int32_t kb) { g_batch_setup_kb = kb > 0 ? kb : 0; }

void pc_batch_clear_tuned(void) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  g_tuned.clear();
}

int32_t pc_batch_schedule(int32_t n_sys, const int64_t* n_rows, const int64_t* nnz, const int32_t* block_size,
                          int32_t n_ctas, int32_t team_max, double slots_per_cta, int32_t* team, int32_t* slot0,
                          int32_t* order) {
  if (n_sys < 1 || !n_rows || !nnz || !block_size || n_ctas < 1 || team_max < 1 || !team || !slot0 || !order)
    return -1;
  // Estimated cost of a system: bytes per CG iteration (CSR, factor, ~11 vector streams)
  // times an iteration count that grows like N^(1/3) (PCG iterations ~ sqrt(kappa) and
  // kappa ~ N^(2/3) for meshes and geometric graphs in 3D).
  std::vector<double> w(n_sys);
  double total = 0.0;
  for (int s = 0; s < n_sys; ++s) {
    if (n_rows[s] < 0 || nnz[s] < 0 || block_size[s] < 1 || block_size[s] > 64) return -1;
    const double n = (double)n_rows[s];
    const double fac = (double)(block_size[s] / 2 + 1) * 4.0;
    w[s] = (12.0 * (double)nnz[s] + (88.0 + fac) * n) * std::cbrt(std::max(n, 1.0));
    total += w[s];
  }
  const double target = total / (std::max(slots_per_cta, 0.25) * (double)n_ctas);
  std::vector<double> per_slot(n_sys);
  for (int s = 0; s < n_sys; ++s) {
    const int bs = block_size[s];
    const int64_t U = bs <= 32 ? (32 / bs) * bs : bs;
    const int64_t units = (n_rows[s] + U - 1) / U;
    int T = 1;
    while (T * 2 <= team_max && T * 2 <= n_ctas && (double)(T * 2) * target <= w[s] && units >= (int64_t)T * 2 * 4)
      T *= 2;
    team[s] = T;
    per_slot[s] = w[s] / T;
  }
  for (int s = 0; s < n_sys; ++s) order[s] = s;
  // Larger teams first (they form while the grid is still free), then longest slot first.
  std::stable_sort(order, order + n_sys, [&](int a, int b) {
    if (team[a] != team[b]) return team[a] > team[b];
    return per_slot[a] > per_slot[b];
  });
  int32_t k = 0;
  for (int i = 0; i < n_sys; ++i) {
    slot0[order[i]] = k;
    k += team[order[i]];
  }
  return k;
}

pc_status pc_batch_destroy(pc_batch_handle* h) {
  if (!h) return PC_OK;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  void* ptrs[] = {h->sys, h->slot_sys, h->work, h->minv, h->part, h->cnt, h->fail, h->misc, h->o_restarts,
                  h->d_status, h->d_iters, h->d_relres, h->prof};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
  return PC_OK;
}

pc_status pc_batch_create(const pc_batch* B, int32_t prec, double pivot_tol, void* stream, pc_batch_handle** out) {
  if (out) *out = nullptr;
  if (!B || !out || B->n_sys < 1 || B->n_rows < 0 || B->nnz < 1 || B->nnz >= (int64_t)INT32_MAX || !B->sys_row ||
      !B->row_ptr || !B->col_idx || !B->val || !B->block_size || B->max_block_size < 1 || B->max_block_size > 64 ||
      (prec != PC_PREC_FP64 && prec != PC_PREC_FP32 && prec != PC_PREC_TF32) || !(pivot_tol >= 0.0))
    return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int n_sys = B->n_sys;
  std::vector<int64_t> srow(n_sys + 1);
  std::vector<int32_t> hbs(n_sys);
  std::vector<int32_t> hrp(n_sys + 1);
  PCB_TRY(cudaMemcpyAsync(srow.data(), B->sys_row, sizeof(int64_t) * (n_sys + 1), cudaMemcpyDeviceToHost, st));
  PCB_TRY(cudaMemcpyAsync(hbs.data(), B->block_size, sizeof(int32_t) * n_sys, cudaMemcpyDeviceToHost, st));
  PCB_TRY(cudaStreamSynchronize(st));
  if (srow[0] != 0 || srow[n_sys] != B->n_rows) return PC_ERR_INVALID_ARG;
  for (int s = 0; s < n_sys; ++s) {
    if (srow[s + 1] < srow[s] || srow[s + 1] - srow[s] >= (int64_t)INT32_MAX) return PC_ERR_INVALID_ARG;
    if (hbs[s] < 1 || hbs[s] > B->max_block_size) return PC_ERR_INVALID_ARG;
  }
  for (int s = 0; s <= n_sys; ++s)
    PCB_TRY(cudaMemcpyAsync(&hrp[s], B->row_ptr + srow[s], sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  PCB_TRY(cudaStreamSynchronize(st));
  if (hrp[0] != 0 || (int64_t)hrp[n_sys] != B->nnz) return PC_ERR_INVALID_ARG;
  for (int s = 0; s < n_sys; ++s)
    if (hrp[s + 1] < hrp[s] || (srow[s + 1] > srow[s] && hrp[s + 1] == hrp[s])) return PC_ERR_INVALID_ARG;

  pc_batch_handle* h = new pc_batch_handle();
  h->n_sys = n_sys;
  h->n_rows = B->n_rows;
  h->nnz = B->nnz;
  h->prec = prec;
  h->fac_f32 = prec != PC_PREC_FP64;
  const size_t fts = h->fac_f32 ? sizeof(float) : sizeof(double);
  pc_status ps = PC_OK;
#define PCB_CHECK(expr)            \
  do {                             \
    ps = (expr);                   \
    if (ps != PC_OK) {             \
      pc_batch_destroy(h);         \
      return ps;                   \
    }                              \
  } while (0)
#define PCB_CUDA(expr) PCB_CHECK(bfrom(expr))

  // validation of the concatenated CSR on the device
  PCB_CHECK(balloc(&h->misc, 4 * sizeof(unsigned)));
  PCB_CUDA(cudaMemsetAsync(h->misc, 0, 4 * sizeof(unsigned), st));
  pc::batched_validate<<<n_sys, 256, 0, st>>>(B->sys_row, n_sys, B->row_ptr, B->col_idx, B->nnz, h->misc + 2);
  PCB_CUDA(cudaGetLastError());
  unsigned bad = 0;
  PCB_CUDA(cudaMemcpyAsync(&bad, h->misc + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  PCB_CUDA(cudaStreamSynchronize(st));
  if (bad) PCB_CHECK(PC_ERR_INVALID_ARG);

  // shared memory: setup slots large enough for every block size up to the maximum (the
  // need is not monotone in bs: U = 32 rows for bs <= 32 only when bs divides 32), as
  // many slots as fit in the budget
  size_t need = 0;
  for (int bsz = 1; bsz <= B->max_block_size; ++bsz)
    need = std::max(need, pc::setup_unit_smem(pc::make_layout(64, bsz), fts));
  const int slot_bytes = (int)((need + 15) & ~(size_t)15);
  Tuned tuned{};
  const Tuned* tu = (g_batch_ctas_per_sm || g_batch_team_max || g_batch_split > 0.0 || g_batch_setup_kb)
                        ? nullptr
                        : (find_tuned(B, prec, &tuned) ? &tuned : nullptr);
  const int setup_kb = g_batch_setup_kb ? g_batch_setup_kb : (tu ? tu->setup_kb : 70);
  const int budget = setup_kb * 1024;
  int setup_warps = std::max(1, std::min(pc::BNW, budget / slot_bytes));
  // the same dynamic shared memory holds the setup slots, then the SpMV warp slices
  h->smem = std::max(setup_warps * slot_bytes, pc::BNW * pc::STAGE_BYTES);
  const void* fn = h->fac_f32 ? (const void*)pc::batched_kernel<float> : (const void*)pc::batched_kernel<double>;
  PCB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem));
  int occ = 0;
  PCB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, pc::BT, (size_t)h->smem));
  if (occ < 1) PCB_CHECK(PC_ERR_CUDA);
  const int want_occ = g_batch_ctas_per_sm ? g_batch_ctas_per_sm : (tu ? tu->ctas_per_sm : 0);
  if (want_occ > 0 && want_occ < occ) occ = want_occ;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  h->ctas_per_sm = occ;
  h->grid = occ * std::max(sms, 1);

  // schedule
  std::vector<int64_t> nr(n_sys), nz(n_sys);
  for (int s = 0; s < n_sys; ++s) {
    nr[s] = srow[s + 1] - srow[s];
    nz[s] = (int64_t)hrp[s + 1] - hrp[s];
  }
  std::vector<int32_t> team(n_sys), slot0(n_sys), order(n_sys);
  h->team_max = g_batch_team_max > 0 ? g_batch_team_max : (tu ? tu->team_max : 32);
  const double split = g_batch_split > 0.0 ? g_batch_split : (tu ? tu->split : 2.0);
  const int n_slots = pc_batch_schedule(n_sys, nr.data(), nz.data(), hbs.data(), h->grid, h->team_max, split,
                                        team.data(), slot0.data(), order.data());
  if (n_slots < 1) PCB_CHECK(PC_ERR_INVALID_ARG);
  h->n_slots = n_slots;
  h->hsys.resize(n_sys);
  h->hslot.resize(n_slots);
  int64_t fac = 0;
  for (int s = 0; s < n_sys; ++s) {
    const pc::Layout L = pc::make_layout(nr[s], hbs[s]);
    BSys& d = h->hsys[s];
    d.row0 = srow[s];
    d.fac0 = fac;
    d.n = (int32_t)nr[s];
    d.bs = hbs[s];
    d.team = team[s];
    d.slot0 = slot0[s];
    fac += L.n_units * pc::unit_elems_minv(L);
    for (int m = 0; m < team[s]; ++m) h->hslot[slot0[s] + m] = s;
  }

  // device memory
  PCB_CHECK(balloc(&h->sys, sizeof(BSys) * n_sys));
  PCB_CHECK(balloc(&h->slot_sys, sizeof(int32_t) * n_slots));
  PCB_CHECK(balloc(&h->work, sizeof(double) * 4 * (size_t)std::max<int64_t>(B->n_rows, 1)));
  PCB_CHECK(balloc(&h->minv, fts * (size_t)std::max<int64_t>(fac, 1)));
  PCB_CHECK(balloc(&h->part, sizeof(double) * 8 * (size_t)n_slots));
  PCB_CHECK(balloc(&h->cnt, sizeof(unsigned) * n_sys));
  PCB_CHECK(balloc(&h->fail, sizeof(unsigned long long) * n_sys));
  PCB_CHECK(balloc(&h->o_restarts, sizeof(int32_t) * n_sys));
  PCB_CHECK(balloc(&h->d_status, sizeof(int32_t) * n_sys));
  PCB_CHECK(balloc(&h->d_iters, sizeof(int32_t) * n_sys));
  PCB_CHECK(balloc(&h->d_relres, sizeof(double) * n_sys));
  {
    const char* pe = getenv("PC_BATCH_PROFILE");
    if (pe && pe[0] == '1') {
      PCB_CHECK(balloc(&h->prof, sizeof(unsigned long long) * pc::PH_N));
      PCB_CUDA(cudaMemsetAsync(h->prof, 0, sizeof(unsigned long long) * pc::PH_N, st));
    }
  }
  PCB_CUDA(cudaMemcpyAsync(h->sys, h->hsys.data(), sizeof(BSys) * n_sys, cudaMemcpyHostToDevice, st));
  PCB_CUDA(cudaMemcpyAsync(h->slot_sys, h->hslot.data(), sizeof(int32_t) * n_slots, cudaMemcpyHostToDevice, st));
  PCB_CUDA(cudaStreamSynchronize(st));   // host vectors are the copy sources

  pc::BArgs& a = h->args;
  memset(&a, 0, sizeof(a));
  a.sys = h->sys;
  a.slot_sys = h->slot_sys;
  a.n_sys = n_sys;
  a.n_slots = n_slots;
  a.rp = B->row_ptr;
  a.ci = B->col_idx;
  a.va = B->val;
  const int64_t nr_all = std::max<int64_t>(B->n_rows, 1);
  a.r = h->work;
  a.z = h->work + nr_all;
  a.p = h->work + 2 * nr_all;
  a.q = h->work + 3 * nr_all;
  a.minv = h->minv;
  a.part = h->part;
  a.cnt = h->cnt;
  a.fail = h->fail;
  a.queue = h->misc;
  a.err = reinterpret_cast<int*>(h->misc + 1);
  a.o_status = h->d_status;
  a.o_iters = h->d_iters;
  a.o_restarts = h->o_restarts;
  a.o_relres = h->d_relres;
  a.pivot_tol = pivot_tol;
  a.tc = prec == PC_PREC_TF32 ? 1 : 0;
  a.max_restarts = 3;
  a.budget = batch_budget();
  a.setup_warps = setup_warps;
  a.slot_bytes = slot_bytes;
  a.prof = h->prof;
  a.smem_bytes = h->smem;
  *out = h;
  return PC_OK;
#undef PCB_CUDA
#undef PCB_CHECK
}

static cudaError_t batch_launch(pc_batch_handle* h, cudaStream_t st) {
  // the dynamic shared-memory limit is per function: another handle may have lowered it
  cudaError_t ae = cudaFuncSetAttribute(h->fac_f32 ? (const void*)pc::batched_kernel<float>
                                                   : (const void*)pc::batched_kernel<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem);
  if (ae != cudaSuccess) return ae;
  pc::batched_reset<<<std::max(1, std::min(1024, (h->n_sys + 255) / 256)), 256, 0, st>>>(
      h->misc, reinterpret_cast<int*>(h->misc + 1), h->cnt, h->fail, h->n_sys);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)h->grid);
  cfg.blockDim = dim3(pc::BT);
  cfg.dynamicSmemBytes = (size_t)h->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (h->fac_f32) return cudaLaunchKernelEx(&cfg, pc::batched_kernel<float>, h->args);
  return cudaLaunchKernelEx(&cfg, pc::batched_kernel<double>, h->args);
}

static cudaError_t batch_capture(pc_batch_handle* h, cudaStream_t st) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = batch_launch(h, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) {
      h->graph = g;
      e = cudaGraphInstantiate(&h->exec, g, 0);
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  (void)st;
  return e;
}

static pc_status batch_solve_impl(pc_batch_handle* h, const double* b, double* x, double tol, int32_t max_iter,
                                  int32_t* iters, int32_t* status, double* relres, pc_solve_info* info,
                                  void* stream);

pc_status pc_batch_solve(pc_batch_handle* h, const double* b, double* x, double tol, int32_t max_iter,
                         int32_t* iters, int32_t* status, double* relres, pc_solve_info* info, void* stream) {
  nvtxRangePushA("pc_batch_solve");
  const pc_status ret = batch_solve_impl(h, b, x, tol, max_iter, iters, status, relres, info, stream);
  nvtxRangePop();
  return ret;
}

static pc_status batch_solve_impl(pc_batch_handle* h, const double* b, double* x, double tol, int32_t max_iter,
                                  int32_t* iters, int32_t* status, double* relres, pc_solve_info* info,
                                  void* stream) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->failed_block = -1;
  }
  if (!h || (!b && h->n_rows > 0) || (!x && h->n_rows > 0) || !(tol >= 0.0) || max_iter < 0)
    return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  h->args.b = b;
  h->args.x = x;
  h->args.tol = tol;
  h->args.max_iter = max_iter;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PCB_TRY(cudaEventCreate(&e0));
  PCB_TRY(cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  const bool same = h->exec && h->g_b == b && h->g_x == x && h->g_tol == tol && h->g_max_iter == max_iter;
  if (!same) {
    e = batch_capture(h, st);
    h->graph_ok = e == cudaSuccess;
    if (h->graph_ok) {
      h->g_b = b;
      h->g_x = x;
      h->g_tol = tol;
      h->g_max_iter = max_iter;
    } else {
      cudaGetLastError();
      h->exec = nullptr;
    }
  }
  cudaEventRecord(e0, st);
  if (h->graph_ok) e = cudaGraphLaunch(h->exec, st);
  else e = batch_launch(h, st);
  cudaEventRecord(e1, st);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->misc + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  std::vector<int32_t> hs(h->n_sys), hi(h->n_sys), hr(h->n_sys);
  std::vector<double> hrel(h->n_sys);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), h->d_status, sizeof(int32_t) * h->n_sys, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hi.data(), h->d_iters, sizeof(int32_t) * h->n_sys, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hr.data(), h->o_restarts, sizeof(int32_t) * h->n_sys, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hrel.data(), h->d_relres, sizeof(double) * h->n_sys, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && iters) e = cudaMemcpyAsync(iters, h->d_iters, sizeof(int32_t) * h->n_sys, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && status)
    e = cudaMemcpyAsync(status, h->d_status, sizeof(int32_t) * h->n_sys, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && relres)
    e = cudaMemcpyAsync(relres, h->d_relres, sizeof(double) * h->n_sys, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return bfrom(e);
  pc_status out = PC_OK;
  int max_it = 0, max_rs = 0;
  double worst = 0.0;
  for (int s = 0; s < h->n_sys; ++s) {
    max_it = std::max(max_it, hi[s]);
    max_rs = std::max(max_rs, hr[s]);
    worst = std::max(worst, hrel[s]);
    if (out == PC_OK && hs[s] != pc::ST_OK) {
      out = hs[s] == pc::ST_NOT_SPD   ? PC_ERR_NOT_SPD
            : hs[s] == pc::ST_BREAKDOWN ? PC_ERR_BREAKDOWN
            : hs[s] == pc::ST_NO_CONV   ? PC_ERR_NO_CONVERGENCE
            : hs[s] == pc::ST_TIMEOUT   ? PC_ERR_TIMEOUT
                                        : PC_ERR_CUDA;
      if (info) info->failed_block = s;
    }
  }
  if (err == pc::ST_TIMEOUT) out = PC_ERR_TIMEOUT;
  if (info) {
    info->status = out;
    info->iterations = max_it;
    info->restarts = max_rs;
    info->rel_residual = worst;
    info->true_rel_residual = worst;
    info->setup_ms = 0.0;
    info->solve_ms = ms;
    info->grid_ctas = h->grid;
    info->block_size = 0;
    info->prec = h->prec;
    info->reserved = h->graph_ok ? 1 : 0;
  }
  return out;
}

int32_t pc_batch_info(const pc_batch_handle* h, int32_t* out, int32_t max_entries) {
  if (!h || !out || max_entries < 1) return 0;
  const int32_t vals[] = {h->grid, h->ctas_per_sm, h->n_slots, h->team_max, h->smem, h->args.setup_warps,
                          h->graph_ok ? 1 : 0};
  const int32_t k = std::min<int32_t>(max_entries, (int32_t)(sizeof(vals) / sizeof(vals[0])));
  for (int32_t i = 0; i < k; ++i) out[i] = vals[i];
  return k;
}

int32_t pc_batch_profile(const pc_batch_handle* h, uint64_t* out, int32_t max_entries) {
  if (!h || !h->prof || !out || max_entries < 1) return 0;
  unsigned long long v[pc::PH_N];
  if (cudaMemcpy(v, h->prof, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int32_t k = std::min<int32_t>(max_entries, (int32_t)pc::PH_N);
  for (int32_t i = 0; i < k; ++i) out[i] = v[i];
  return k;
}

int32_t pc_batch_teams(const pc_batch_handle* h, int32_t* team, int32_t* slot0) {
  if (!h) return 0;
  for (int s = 0; s < h->n_sys; ++s) {
    if (team) team[s] = h->hsys[s].team;
    if (slot0) slot0[s] = h->hsys[s].slot0;
  }
  return h->n_sys;
}

pc_status pc_batch_autotune(const pc_batch* B, int32_t prec, const double* b, double tol, int32_t max_iter,
                            int32_t max_trials, void* stream, double* best_ms, int32_t* best_cfg) {
  if (!B || !b || !(tol >= 0.0) || max_iter < 0) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* x = nullptr;
  pc_status ps = balloc(&x, sizeof(double) * (size_t)std::max<int64_t>(B->n_rows, 1));
  if (ps != PC_OK) return ps;
  // Candidate launch shapes: CTAs per SM (0 = occupancy maximum), team limit, slots per CTA
  // of the scheduler, and the shared memory given to setup slots (setup warps per CTA).
  struct Cand {
    int occ, team, kb;
    double split;
  };
  std::vector<Cand> cands;
  // the measured best on the 512-system RGG batch (team limit 4, 8 slots per CTA) comes first
  for (int occ : {0, 1})
    for (int team : {4, 8, 32})
      for (double split : {8.0, 4.0, 2.0})
        for (int kb : {70, 140}) cands.push_back({occ, team, kb, split});
  const int saved_occ = g_batch_ctas_per_sm, saved_team = g_batch_team_max, saved_kb = g_batch_setup_kb;
  const double saved_split = g_batch_split;
  double best = 1e300;
  Cand bc{0, 32, 70, 2.0};
  int trials = 0;
  pc_status out = PC_OK;
  for (const Cand& c : cands) {
    if (max_trials > 0 && trials >= max_trials) break;
    g_batch_ctas_per_sm = c.occ;
    g_batch_team_max = c.team;
    g_batch_split = c.split;
    g_batch_setup_kb = c.kb;
    pc_batch_handle* h = nullptr;
    pc_status s = pc_batch_create(B, prec, 0.0, stream, &h);
    if (s != PC_OK) {
      if (s == PC_ERR_INVALID_ARG) {
        out = s;
        break;
      }
      continue;   // e.g. a shared-memory budget the device cannot give
    }
    pc_solve_info info;
    // first call captures the graph; the second is timed
    s = pc_batch_solve(h, b, x, tol, max_iter, nullptr, nullptr, nullptr, &info, stream);
    if (s == PC_OK || s == PC_ERR_NO_CONVERGENCE)
      s = pc_batch_solve(h, b, x, tol, max_iter, nullptr, nullptr, nullptr, &info, stream);
    pc_batch_destroy(h);
    ++trials;
    if (s != PC_OK && s != PC_ERR_NO_CONVERGENCE) {
      out = s;
      break;
    }
    if (info.solve_ms < best) {
      best = info.solve_ms;
      bc = c;
    }
  }
  g_batch_ctas_per_sm = saved_occ;
  g_batch_team_max = saved_team;
  g_batch_split = saved_split;
  g_batch_setup_kb = saved_kb;
  cudaStreamSynchronize(st);
  cudaFree(x);
  if (out != PC_OK) return out;
  if (best_ms) *best_ms = best;
  if (best_cfg) {
    best_cfg[0] = bc.occ;
    best_cfg[1] = bc.team;
    best_cfg[2] = (int32_t)(bc.split * 1000.0);
    best_cfg[3] = bc.kb;
  }
  Tuned t{B->n_sys, B->n_rows, B->nnz, prec, pc::current_sms(), bc.occ, bc.team, bc.kb, bc.split};
  put_tuned(t);
  return pc::tune_save_env();
}

pc_status pcg_solve_batched(const pc_batch* B, const double* b, double* x, double tol, int32_t max_iter,
                            int32_t prec, int32_t* iters, int32_t* status, double* relres, pc_solve_info* info,
                            void* stream) {
  pc_batch_handle* h = nullptr;
  pc_status s = pc_batch_create(B, prec, 0.0, stream, &h);
  if (s != PC_OK) {
    if (info) {
      memset(info, 0, sizeof(*info));
      info->status = s;
      info->failed_block = -1;
    }
    return s;
  }
  s = pc_batch_solve(h, b, x, tol, max_iter, iters, status, relres, info, stream);
  pc_batch_destroy(h);
  return s;
}

}  // extern "C"

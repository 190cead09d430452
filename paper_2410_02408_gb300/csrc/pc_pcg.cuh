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
#pragma once

#include "pc_kernels.cuh"

namespace pc {

template <typename VT, typename FT, int BS>
__global__ void __launch_bounds__(256, 4) pcg_kernel(const PcgArgs a) {
  __shared__ double sm[2 * 32];
  __shared__ int flag[4];
  const Layout L = a.lay;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  const int G = gridDim.x;
  const int cta = blockIdx.x;
  const int64_t n = L.n;
  const VT* __restrict__ va = reinterpret_cast<const VT*>(a.va);
  const FT* __restrict__ Mf = reinterpret_cast<const FT*>(a.minv);
  const int64_t uM = unit_elems_minv(L);
  // unit range (phases B, C) and SpMV row range (phase A, residuals)
  const int64_t upc = (L.n_units + G - 1) / G;
  const int64_t u0 = min((int64_t)cta * upc, L.n_units);
  const int64_t u1 = min(u0 + upc, L.n_units);
  const int64_t row0 = min(u0 * L.U, n);
  const int64_t row1 = min(u1 * L.U, n);
  const int64_t sa0 = a.split[cta];
  const int64_t sa1 = a.split[cta + 1];
  const double tol = a.tol;
  int bar = 0;

  // ---- r = b - A x, ||b||^2
  double bb;
  {
    double v[1] = {0.0};
    for (int64_t row = sa0 + tid; row < sa1; row += blockDim.x) {
      const double ax = spmv_row<VT, true>(a.rp, a.ci, va, a.x, row);
      const double bi = __ldg(a.b + row);
      st_vec(a.r + row, bi - ax);
      v[0] = fma(bi, bi, v[0]);
    }
    if (!grid_allreduce<1>(v, a.part, a.gs, a.budget, sm, flag, bar++)) return;
    bb = v[0];
  }
  const double bnorm = sqrt(bb);
  if (bb == 0.0) {
    for (int64_t row = row0 + tid; row < row1; row += blockDim.x) st_vec(a.x + row, 0.0);
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
    {
      double v[2] = {0.0, 0.0};
      for (int64_t u = u0 + warp; u < u1; u += nw) {
        double rv[2], zv[2];
        int64_t rows[2];
        bool ok[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          bool valid;
          const int rh = unit_row(L, lane, s, valid);
          rows[s] = u * L.U + rh;
          ok[s] = valid && rows[s] < n;
          rv[s] = ok[s] ? ld_vec(a.r + rows[s]) : 0.0;
        }
        unit_apply_inv<FT, BS>(L, Mf + u * uM, lane, rv, zv);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if (!ok[s]) continue;
          st_vec(a.z + rows[s], zv[s]);
          st_vec(a.p + rows[s], zv[s]);
          v[0] = fma(rv[s], zv[s], v[0]);
          v[1] = fma(rv[s], rv[s], v[1]);
        }
      }
      if (!grid_allreduce<2>(v, a.part, a.gs, a.budget, sm, flag, bar++)) return;
      rho = v[0];
      rr = v[1];
    }
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
      {
        double v[1] = {0.0};
        for (int64_t row = sa0 + tid; row < sa1; row += blockDim.x) {
          const double qi = spmv_row<VT, true>(a.rp, a.ci, va, a.p, row);
          st_vec(a.q + row, qi);
          v[0] = fma(ld_vec(a.p + row), qi, v[0]);
        }
        if (!grid_allreduce<1>(v, a.part, a.gs, a.budget, sm, flag, bar++)) return;
        pq = v[0];
      }
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = ST_BREAKDOWN;
        break;
      }
      const double alpha = rho / pq;
      // ---- B: r -= alpha q; z = M^{-1} r; r.z, r.r
      double rz;
      {
        double v[2] = {0.0, 0.0};
        for (int64_t u = u0 + warp; u < u1; u += nw) {
          double rv[2], zv[2];
          int64_t rows[2];
          bool ok[2];
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            bool valid;
            const int rh = unit_row(L, lane, s, valid);
            rows[s] = u * L.U + rh;
            ok[s] = valid && rows[s] < n;
            rv[s] = ok[s] ? fma(-alpha, ld_vec(a.q + rows[s]), ld_vec(a.r + rows[s])) : 0.0;
          }
          unit_apply_inv<FT, BS>(L, Mf + u * uM, lane, rv, zv);
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            if (!ok[s]) continue;
            st_vec(a.r + rows[s], rv[s]);
            st_vec(a.z + rows[s], zv[s]);
            v[0] = fma(rv[s], zv[s], v[0]);
            v[1] = fma(rv[s], rv[s], v[1]);
          }
        }
        if (!grid_allreduce<2>(v, a.part, a.gs, a.budget, sm, flag, bar++)) return;
        rz = v[0];
        rr = v[1];
      }
      ++it;
      if (sqrt(rr) <= tol * bnorm) {
        for (int64_t row = row0 + tid; row < row1; row += blockDim.x)
          st_vec(a.x + row, fma(alpha, ld_vec(a.p + row), ld_vec(a.x + row)));
        if (!grid_allreduce<0>(nullptr, a.part, a.gs, a.budget, sm, flag, bar++)) return;
        conv = true;
        break;
      }
      const double beta = rz / rho;
      rho = rz;
      // ---- C: x += alpha p; p = z + beta p  (4 rows per thread in flight)
      for (int64_t base = row0 + tid; base < row1; base += 4 * (int64_t)blockDim.x) {
        double pv[4], xv[4], zv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t row = min(base + t * (int64_t)blockDim.x, row1 - 1);
          pv[t] = ld_vec(a.p + row);
          xv[t] = ld_vec(a.x + row);
          zv[t] = ld_vec(a.z + row);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t row = base + t * (int64_t)blockDim.x;
          if (row < row1) {
            st_vec(a.x + row, fma(alpha, pv[t], xv[t]));
            st_vec(a.p + row, fma(beta, pv[t], zv[t]));
          }
        }
      }
      if (!grid_allreduce<0>(nullptr, a.part, a.gs, a.budget, sm, flag, bar++)) return;
    }
    // ---- true residual r = b - A x
    {
      double v[1] = {0.0};
      for (int64_t row = sa0 + tid; row < sa1; row += blockDim.x) {
        const double ri = __ldg(a.b + row) - spmv_row<VT, true>(a.rp, a.ci, va, a.x, row);
        st_vec(a.r + row, ri);
        v[0] = fma(ri, ri, v[0]);
      }
      if (!grid_allreduce<1>(v, a.part, a.gs, a.budget, sm, flag, bar++)) return;
      tt = v[0];
    }
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
cudaError_t launch_pcg_t(const PcgArgs& a, int grid, int block, cudaStream_t st) {
  void* args[] = {const_cast<PcgArgs*>(&a)};
  const void* fn;
  switch (a.lay.bs) {
    case 8: fn = (const void*)pcg_kernel<VT, FT, 8>; break;
    case 16: fn = (const void*)pcg_kernel<VT, FT, 16>; break;
    case 32: fn = (const void*)pcg_kernel<VT, FT, 32>; break;
    case 64: fn = (const void*)pcg_kernel<VT, FT, 64>; break;
    default: fn = (const void*)pcg_kernel<VT, FT, 0>; break;
  }
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

template <typename VT, typename FT>
cudaError_t pcg_occupancy_t(const Layout& L, int block, int* ctas) {
  const void* fn;
  switch (L.bs) {
    case 8: fn = (const void*)pcg_kernel<VT, FT, 8>; break;
    case 16: fn = (const void*)pcg_kernel<VT, FT, 16>; break;
    case 32: fn = (const void*)pcg_kernel<VT, FT, 32>; break;
    case 64: fn = (const void*)pcg_kernel<VT, FT, 64>; break;
    default: fn = (const void*)pcg_kernel<VT, FT, 0>; break;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, block, 0);
}

}  // namespace pc

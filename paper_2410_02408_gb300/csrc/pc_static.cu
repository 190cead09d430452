// pcg_solve_noalloc: the block-Jacobi PCG solve of pcg_solve, for callers that must not
// allocate device memory.  Every piece of scratch the solve needs (block factors, CG
// vectors, reduction partials, row split, barrier words) is carved out of one
// file-scope device array of fixed size instead of coming from cudaMalloc.
//
// Host code never dereferences or passes the array's name to a kernel: in host code the
// symbol is only a host-side stand-in.  Its device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "pc.h"
#include "pc_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)PC_NOALLOC_SCRATCH_BYTES;

}  // namespace

// Shared by every call on a device; keeps the previous call's contents.
static __device__ __align__(256) unsigned char pc_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};

pc_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  cudaGetLastError();
  return PC_ERR_CUDA;
}

// Device address of the scratch array on the current device (looked up on first use).
pc_status scratch_base(unsigned char** base) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return to_status(e);
  if (dev < 0 || dev >= 64) return PC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, pc_noalloc_scratch);
    if (e != cudaSuccess || !p) return to_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_scratch_addr[dev] = p;
  }
  *base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return PC_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" pc_status pcg_solve_noalloc(const pc_csr* A, int32_t block_size, const double* b, double* x, double tol,
                                       int32_t max_iter, int32_t prec, pc_solve_info* info, void* stream) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->failed_block = -1;
  }
  if (!A || A->n <= 0 || A->n >= (int64_t)INT32_MAX || A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX ||
      !A->row_ptr || !A->col_idx || (A->nnz > 0 && !A->val) || (A->dtype != PC_F64 && A->dtype != PC_F32))
    return PC_ERR_INVALID_ARG;
  if (block_size < 1 || block_size > 64 || !b || !x || !(tol >= 0.0) || max_iter < 0) return PC_ERR_INVALID_ARG;
  if (prec != PC_PREC_FP64 && prec != PC_PREC_FP32 && prec != PC_PREC_TF32) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const pc::Layout L = pc::make_layout(A->n, block_size);
  const bool val_f32 = A->dtype == PC_F32;
  const bool fac_f32 = prec != PC_PREC_FP64;
  const size_t es = fac_f32 ? 4 : 8;

  // persistent grid and wait budget exactly as pcg_solve_h computes them
  const int block = pc::PCG_BLOCK;
  pc::PcgArgs a;
  a.lay = L;
  pc::pcg_plan(a, A->nnz, val_f32, fac_f32);
  int grid = 0;
  cudaError_t e = pc::persistent_grid(L, A->nnz, val_f32, fac_f32, &grid);
  if (e != cudaSuccess) return to_status(e);

  // carve the scratch: sizes first, so an oversized problem is rejected before any work.
  // The CG vectors sit at a stride of a multiple of 32 doubles (every vector and every
  // bulk-copied row window starts 16-byte aligned), with 64 doubles of tail padding.
  const size_t n = (size_t)A->n;
  const size_t vs = (n + 31) & ~(size_t)31;
  const size_t sz_minv = round256(es * (size_t)(L.n_units * pc::unit_elems_minv(L)));
  const size_t sz_linv = round256(es * (size_t)(L.n_units * pc::unit_elems_linv(L)));
  const size_t sz_fail = 256;
  const size_t sz_vec = round256(sizeof(double) * (4 * vs + 64));
  const size_t sz_part = round256(sizeof(double) * 4 * (size_t)grid);
  const size_t sz_split = round256(sizeof(int64_t) * (size_t)(grid + 1));
  const size_t sz_ctl = round256(sizeof(pc::GridSync) + sizeof(pc::PcgOut));
  const size_t total = sz_minv + sz_linv + sz_fail + sz_vec + sz_part + sz_split + sz_ctl;
  if (total > kScratchBytes) return PC_ERR_INVALID_ARG;

  unsigned char* base = nullptr;
  pc_status ps = scratch_base(&base);
  if (ps != PC_OK) return ps;
  unsigned char* cur = base;
  void* minv = cur;
  cur += sz_minv;
  void* linv = cur;
  cur += sz_linv;
  unsigned long long* failed_d = reinterpret_cast<unsigned long long*>(cur);
  cur += sz_fail;
  double* vec = reinterpret_cast<double*>(cur);
  cur += sz_vec;
  double* part = reinterpret_cast<double*>(cur);
  cur += sz_part;
  int64_t* split = reinterpret_cast<int64_t*>(cur);
  cur += sz_split;
  unsigned char* ctl = cur;

  // CSR structure check (the word is cleared by the launcher) before anything reads the matrix
  unsigned bad = 0u;
  e = pc::launch_validate_csr(A->n, A->nnz, A->row_ptr, A->col_idx, reinterpret_cast<unsigned*>(failed_d), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, failed_d, sizeof(bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  if (bad) return PC_ERR_INVALID_ARG;

  // setup: the failure word must start at all ones (the scratch keeps old contents)
  e = cudaMemsetAsync(failed_d, 0xff, sizeof(unsigned long long), st);
  pc::SetupArgs sa;
  sa.lay = L;
  sa.row_ptr = A->row_ptr;
  sa.col = A->col_idx;
  sa.val = A->val;
  sa.tol = 0.0;
  sa.minv = minv;
  sa.linv = linv;
  sa.failed = failed_d;
  if (e == cudaSuccess)
    e = prec == PC_PREC_TF32 ? pc::launch_setup_tf32(sa, val_f32, st) : pc::launch_setup(sa, val_f32, fac_f32, st);
  unsigned long long failed = ~0ull;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&failed, failed_d, sizeof(failed), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && failed != ~0ull && fac_f32) {
    // as in pc_setup: an FP32 pivot broke down, so every block is factored again in FP64
    // arithmetic (factors stored in FP32); NOT_SPD only if that fails too
    e = cudaMemsetAsync(failed_d, 0xff, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = pc::launch_setup_f64_store_f32(sa, val_f32, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&failed, failed_d, sizeof(failed), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return to_status(e);
  if (failed != ~0ull) {
    if (info) {
      info->status = PC_ERR_NOT_SPD;
      info->failed_block = (int32_t)failed;
    }
    return PC_ERR_NOT_SPD;
  }

  // solve: barrier words and outputs must start at zero
  e = pc::launch_split(A->n, A->nnz, A->row_ptr, grid, split, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(pc::GridSync) + sizeof(pc::PcgOut), st);
  a.rp = A->row_ptr;
  a.ci = A->col_idx;
  a.va = A->val;
  a.minv = minv;
  a.b = b;
  a.x = x;
  a.r = vec;
  a.z = vec + vs;
  a.p = vec + 2 * vs;
  a.q = vec + 3 * vs;
  a.part = part;
  a.split = split;
  a.gs = reinterpret_cast<pc::GridSync*>(ctl);
  a.out = reinterpret_cast<pc::PcgOut*>(ctl + sizeof(pc::GridSync));
  a.tol = tol;
  a.max_iter = max_iter;
  a.max_restarts = 3;
  a.budget = pc::wait_budget_cycles();
  a.trace = nullptr;
  a.trace_len = 0;
  if (e == cudaSuccess) e = pc::launch_pcg(a, val_f32, fac_f32, grid, block, st);
  unsigned char hostctl[sizeof(pc::GridSync) + sizeof(pc::PcgOut)];
  if (e == cudaSuccess) e = cudaMemcpyAsync(hostctl, ctl, sizeof(hostctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  pc::GridSync gs;
  pc::PcgOut out;
  memcpy(&gs, hostctl, sizeof(gs));
  memcpy(&out, hostctl + sizeof(gs), sizeof(out));
  const pc_status status = gs.status != 0 ? (pc_status)gs.status : (pc_status)out.status;
  if (info) {
    info->status = status;
    info->iterations = out.iterations;
    info->restarts = out.restarts;
    info->rel_residual = out.rel_residual;
    info->true_rel_residual = out.true_rel_residual;
    info->grid_ctas = grid;
    info->block_size = block_size;
    info->prec = prec;
  }
  return status;
}

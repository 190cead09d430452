// Complex Hermitian positive definite systems (Sec. 3.1 takes A Hermitian PD) through their
// real-equivalent form.
//
// Write z = u + i v and a_ij = b_ij + i c_ij.  With the unknowns interleaved as
// (u_0, v_0, u_1, v_1, ...), A z = f is the real system K y = g whose 2x2 block (i, j) is
// [[b, -c], [c, b]].  K is symmetric when A is Hermitian, and y^T K y = z^H A z, so K is SPD
// exactly when A is Hermitian PD, with the spectrum of A (each eigenvalue twice).
//
// The real-form block of a complex diagonal block A_kk (block size bs) is the real block K_kk of
// block size 2 bs, and the real form of the complex Cholesky factor L (lower triangular, real
// positive diagonal) is lower triangular with a positive diagonal and satisfies
// form(L) form(L)^T = form(L L^H) = K_kk; by uniqueness of the Cholesky factor it IS the
// Cholesky factor of K_kk.  Hence block-Jacobi on K with block size 2 bs is the complex
// block-Jacobi M = blockdiag(L_k L_k^H), and since every CG scalar of an HPD system is real
// (r^H z, p^H A p), PCG on K runs the complex PCG iteration for iteration.  The Lanczos
// tridiagonal of K from form(v0) is the complex one as well (alpha_j = q_j^H A q_j is real).
//
// So the complex path builds K on the device (one pass over the complex CSR) and runs the real
// kernels on it.  K stores every complex entry as four real entries, 48 bytes against the 20 of
// a complex CSR entry (16-byte value + 4-byte column index); the arithmetic is the same four real
// products per complex entry.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "pc.h"
#include "pc_kernels.cuh"

namespace pc {

// One thread per complex row i: real rows 2i (real parts) and 2i+1 (imaginary parts), each with
// two entries per complex entry, columns 2j and 2j+1 (so columns stay strictly increasing).
__global__ void __launch_bounds__(256) herm_real_form_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                             const int32_t* __restrict__ ci,
                                                             const double2* __restrict__ va, int32_t* __restrict__ krp,
                                                             int32_t* __restrict__ kci, double* __restrict__ kva) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e0 = __ldg(rp + i), e1 = __ldg(rp + i + 1);
    const int32_t len = e1 - e0;
    const int64_t r0 = 4 * (int64_t)e0;           // first entry of real row 2i
    const int64_t r1 = r0 + 2 * (int64_t)len;     // first entry of real row 2i+1
    krp[2 * i] = (int32_t)r0;
    krp[2 * i + 1] = (int32_t)r1;
    if (i == n - 1) krp[2 * n] = (int32_t)(4 * (int64_t)e1);
    for (int32_t t = 0; t < len; ++t) {
      const int32_t j = __ldg(ci + e0 + t);
      const double2 a = __ldg(va + e0 + t);   // (b, c): a = b + i c
      kci[r0 + 2 * t] = 2 * j;
      kva[r0 + 2 * t] = a.x;
      kci[r0 + 2 * t + 1] = 2 * j + 1;
      kva[r0 + 2 * t + 1] = -a.y;
      kci[r1 + 2 * t] = 2 * j;
      kva[r1 + 2 * t] = a.y;
      kci[r1 + 2 * t + 1] = 2 * j + 1;
      kva[r1 + 2 * t + 1] = a.x;
    }
  }
}

}  // namespace pc

namespace {

bool zcsr_ok(const pc_csr_z* A) {
  if (!A || A->n <= 0 || A->nnz < 0) return false;
  if (2 * A->n + 1 >= (int64_t)INT32_MAX || 4 * A->nnz >= (int64_t)INT32_MAX) return false;
  return A->row_ptr && A->col_idx && (A->nnz == 0 || A->val);
}

pc_status zstatus(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
}

// The real form of A in freshly allocated device memory (freed by release()).
struct RealForm {
  pc_csr K;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* va = nullptr;
  void release() {
    if (rp) cudaFree(rp);
    if (ci) cudaFree(ci);
    if (va) cudaFree(va);
    rp = nullptr;
    ci = nullptr;
    va = nullptr;
  }
};

pc_status build_real_form(const pc_csr_z* A, RealForm* f, cudaStream_t st) {
  // the complex CSR's structure is checked as for real matrices (its indices are read below)
  pc_csr S;
  memset(&S, 0, sizeof(S));
  S.n = A->n;
  S.nnz = A->nnz;
  S.row_ptr = A->row_ptr;
  S.col_idx = A->col_idx;
  S.val = A->val;
  S.dtype = PC_F64;
  uint32_t bad = 0;
  pc_status s = pc_csr_check(&S, &bad, st);
  if (s != PC_OK) return s;
  const int64_t kn = 2 * A->n, knz = 4 * A->nnz;
  cudaError_t e = cudaMalloc(&f->rp, sizeof(int32_t) * (size_t)(kn + 1));
  if (e == cudaSuccess) e = cudaMalloc(&f->ci, sizeof(int32_t) * (size_t)(knz > 0 ? knz : 1));
  if (e == cudaSuccess) e = cudaMalloc(&f->va, sizeof(double) * (size_t)(knz > 0 ? knz : 1));
  if (e != cudaSuccess) {
    f->release();
    return zstatus(e);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (A->n + 255) / 256;
  if (grid > (int64_t)(sms > 0 ? sms : 1) * 16) grid = (int64_t)(sms > 0 ? sms : 1) * 16;
  pc::herm_real_form_kernel<<<(unsigned)(grid > 0 ? grid : 1), 256, 0, st>>>(
      A->n, A->row_ptr, A->col_idx, reinterpret_cast<const double2*>(A->val), f->rp, f->ci, f->va);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    f->release();
    return zstatus(e);
  }
  memset(&f->K, 0, sizeof(f->K));
  f->K.n = kn;
  f->K.nnz = knz;
  f->K.row_ptr = f->rp;
  f->K.col_idx = f->ci;
  f->K.val = f->va;
  f->K.dtype = PC_F64;
  return PC_OK;
}

}  // namespace

extern "C" {

pc_status pc_hermitian_real_form(const pc_csr_z* A, int32_t* row_ptr, int32_t* col_idx, double* val, void* stream) {
  if (!zcsr_ok(A) || !row_ptr || !col_idx || (A->nnz > 0 && !val)) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  pc_csr S;
  memset(&S, 0, sizeof(S));
  S.n = A->n;
  S.nnz = A->nnz;
  S.row_ptr = A->row_ptr;
  S.col_idx = A->col_idx;
  S.val = A->val;
  S.dtype = PC_F64;
  pc_status s = pc_csr_check(&S, nullptr, st);
  if (s != PC_OK) return s;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (A->n + 255) / 256;
  if (grid > (int64_t)(sms > 0 ? sms : 1) * 16) grid = (int64_t)(sms > 0 ? sms : 1) * 16;
  pc::herm_real_form_kernel<<<(unsigned)(grid > 0 ? grid : 1), 256, 0, st>>>(
      A->n, A->row_ptr, A->col_idx, reinterpret_cast<const double2*>(A->val), row_ptr, col_idx, val);
  return zstatus(cudaGetLastError());
}

pc_status pcg_solve_z(const pc_csr_z* A, int32_t block_size, const double* b, double* x, double tol, int32_t max_iter,
                      int32_t prec, pc_solve_info* info, void* stream) {
  nvtxRangePushA("pcg_solve_z");
  if (info) {
    memset(info, 0, sizeof(*info));
    info->failed_block = -1;
  }
  pc_status s = PC_OK;
  if (!zcsr_ok(A) || block_size < 1 || block_size > 32 || !b || !x) s = PC_ERR_INVALID_ARG;
  RealForm f;
  if (s == PC_OK) s = build_real_form(A, &f, (cudaStream_t)stream);
  if (s == PC_OK) {
    s = pcg_solve(&f.K, 2 * block_size, b, x, tol, max_iter, prec, info, stream);
    if (info) info->block_size = block_size;   // failed_block: complex block k is real block k
    cudaStreamSynchronize((cudaStream_t)stream);
    f.release();
  } else if (info) {
    info->status = s;
  }
  nvtxRangePop();
  return s;
}

pc_status kappa_estimate_z(const pc_csr_z* A, int32_t block_size, int32_t max_steps, double tol, const double* v0,
                           int32_t reorth, pc_kappa_info* info, void* stream) {
  nvtxRangePushA("kappa_estimate_z");
  pc_status s = PC_OK;
  if (!zcsr_ok(A) || block_size < 0 || block_size > 32 || !v0) s = PC_ERR_INVALID_ARG;
  RealForm f;
  if (s == PC_OK) s = build_real_form(A, &f, (cudaStream_t)stream);
  if (s == PC_OK) {
    s = kappa_estimate(&f.K, 2 * block_size, max_steps, tol, v0, reorth, info, stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    f.release();
  } else if (info) {
    info->status = s;
  }
  nvtxRangePop();
  return s;
}

}  // extern "C"

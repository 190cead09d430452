// Block-Jacobi setup (Sec. 3.2-3.3) for one matrix: every warp factors warp units with
// setup_unit (extraction from CSR, block Cholesky, L^{-1}, M^{-1}); plus the dense
// extraction and factor read-back used for inspection.
#include "pc_kernels.cuh"
#include "pc_setup_unit.cuh"

namespace pc {

template <typename VT, typename FT, typename ST = FT, bool TC = false>
__global__ void __launch_bounds__(128) setup_kernel(SetupArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Layout L = a.lay;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  FT* As = reinterpret_cast<FT*>(smem_raw) + (size_t)warp * 2 * L.U * (L.bs + 1);
  FT* Xs = As + (size_t)L.U * (L.bs + 1);
  const VT* va = reinterpret_cast<const VT*>(a.val);
  ST* Mo = reinterpret_cast<ST*>(a.minv);
  ST* Lo = reinterpret_cast<ST*>(a.linv);
  const int64_t uM = unit_elems_minv(L), uL = unit_elems_linv(L);
  for (int64_t u = (int64_t)blockIdx.x * nw + warp; u < L.n_units; u += (int64_t)gridDim.x * nw)
    setup_unit<VT, FT, ST, TC>(L, u, a.row_ptr, a.col, va, a.tol, Mo + u * uM, Lo ? Lo + u * uL : nullptr, As, Xs,
                               lane, a.failed);
}

// Dense copy of the diagonal blocks (bit-exact value copy; rows past n are zero).
template <typename VT>
__global__ void extract_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const VT* __restrict__ va, int32_t bs, int64_t nrows_pad, double* __restrict__ out) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < nrows_pad;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = row / bs;
    const int i = (int)(row % bs);
    double* o = out + (k * bs + i) * bs;
    for (int j = 0; j < bs; ++j) o[j] = 0.0;
    if (row < n) {
      const int64_t bstart = k * bs;
      for (int32_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int64_t c = ci[e];
        if (c >= bstart && c < bstart + bs) o[c - bstart] = (double)va[e];
      }
    }
  }
}

// Unit layout -> dense blocks.  which = 0: L^{-1}; which = 1: M^{-1}.
template <typename FT>
__global__ void get_factor_kernel(Layout L, const FT* __restrict__ fac, int which, double* __restrict__ out) {
  const int bs = L.bs;
  const int64_t total = L.n_blocks * (int64_t)bs * bs;
  const int64_t uM = unit_elems_minv(L), uL = unit_elems_linv(L);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / ((int64_t)bs * bs);
    const int i = (int)((t / bs) % bs);
    const int j = (int)(t % bs);
    const int64_t u = k / L.G;
    const int g = (int)(k % L.G);
    double v;
    if (which == 0) {
      if (j > i) {
        v = 0.0;
      } else {
        const int rho = g * bs + i;
        v = (double)fac[u * uL + ((i - j) * L.S + rho / 32) * 32 + (rho & 31)];
      }
    } else {
      int d = j - i;
      if (d < 0) d += bs;
      int row = i;
      if (d > L.K) {
        d = i - j;
        if (d < 0) d += bs;
        row = j;
      }
      const int rho = g * bs + row;
      v = (double)fac[u * uM + (d * L.S + rho / 32) * 32 + (rho & 31)];
    }
    out[t] = v;
  }
}

// ------------------------------------------------------------------ launchers
template <typename VT, typename FT, typename ST = FT, bool TC = false>
static cudaError_t launch_setup_t(const SetupArgs& a, cudaStream_t st) {
  const Layout& L = a.lay;
  const size_t per_warp = (size_t)2 * L.U * (L.bs + 1) * sizeof(FT);
  int warps = 4;
  while (warps > 1 && per_warp * warps > 200 * 1024) --warps;
  const size_t smem = per_warp * warps;
  cudaError_t e =
      cudaFuncSetAttribute(setup_kernel<VT, FT, ST, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, setup_kernel<VT, FT, ST, TC>, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  int64_t need = (L.n_units + warps - 1) / warps;
  int64_t grid = (int64_t)sms * occ * 4;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  setup_kernel<VT, FT, ST, TC><<<(unsigned)grid, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_setup(const SetupArgs& a, bool val_f32, bool fac_f32, cudaStream_t st) {
  if (!val_f32 && !fac_f32) return launch_setup_t<double, double>(a, st);
  if (!val_f32 && fac_f32) return launch_setup_t<double, float>(a, st);
  if (val_f32 && fac_f32) return launch_setup_t<float, float>(a, st);
  return launch_setup_t<float, double>(a, st);
}

// FP32 arithmetic with M^{-1} = L^{-T} L^{-1} formed on the tensor cores (TF32 operands, FP32
// accumulation): the PC_PREC_TF32 setup.
cudaError_t launch_setup_tf32(const SetupArgs& a, bool val_f32, cudaStream_t st) {
  if (val_f32) return launch_setup_t<float, float, float, true>(a, st);
  return launch_setup_t<double, float, float, true>(a, st);
}

// FP64 arithmetic, FP32 stored factors: the fallback for blocks whose FP32 factorisation
// breaks down.
cudaError_t launch_setup_f64_store_f32(const SetupArgs& a, bool val_f32, cudaStream_t st) {
  if (val_f32) return launch_setup_t<float, double, float>(a, st);
  return launch_setup_t<double, double, float>(a, st);
}

cudaError_t launch_extract(int64_t n, const int32_t* rp, const int32_t* ci, const void* va, bool val_f32,
                           int32_t bs, double* out, cudaStream_t st) {
  const int64_t nb = (n + bs - 1) / bs;
  const int64_t rows = nb * bs;
  int64_t grid = (rows + 255) / 256;
  if (grid > 65535 * 8) grid = 65535 * 8;
  if (val_f32)
    extract_kernel<float><<<(unsigned)grid, 256, 0, st>>>(n, rp, ci, (const float*)va, bs, rows, out);
  else
    extract_kernel<double><<<(unsigned)grid, 256, 0, st>>>(n, rp, ci, (const double*)va, bs, rows, out);
  return cudaGetLastError();
}

cudaError_t launch_get_factor(const Layout& L, const void* fac, bool fac_f32, int which, double* out,
                              cudaStream_t st) {
  const int64_t total = L.n_blocks * (int64_t)L.bs * L.bs;
  int64_t grid = (total + 255) / 256;
  if (grid > 65535 * 8) grid = 65535 * 8;
  if (grid < 1) grid = 1;
  if (fac_f32)
    get_factor_kernel<float><<<(unsigned)grid, 256, 0, st>>>(L, (const float*)fac, which, out);
  else
    get_factor_kernel<double><<<(unsigned)grid, 256, 0, st>>>(L, (const double*)fac, which, out);
  return cudaGetLastError();
}

}  // namespace pc

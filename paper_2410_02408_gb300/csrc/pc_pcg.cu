// Instantiations of the persistent CG kernel for every (CSR value type, factor type)
// pair and the block sizes with unrolled apply paths (8, 16, 32, 64; others use the
// runtime-block-size path), plus its launch plan.
#include "pc_pcg.cuh"

namespace pc {

void pcg_plan(PcgArgs& a, int64_t nnz, bool val_f32, bool fac_f32) {
  a.nnz = nnz;
  a.tr = PCG_CHUNK;
  a.pad0 = 0;
  const int64_t unit_bytes = unit_elems_minv(a.lay) * (fac_f32 ? 4 : 8);
  a.sp = pcg_smem_plan(val_f32 ? 4 : 8, unit_bytes);
}

cudaError_t launch_pcg(const PcgArgs& a, bool val_f32, bool fac_f32, int grid, int block, cudaStream_t st) {
  if (block != PCG_BLOCK) return cudaErrorInvalidValue;
  if (!val_f32 && !fac_f32) return launch_pcg_t<double, double>(a, grid, block, st);
  if (!val_f32 && fac_f32) return launch_pcg_t<double, float>(a, grid, block, st);
  if (val_f32 && fac_f32) return launch_pcg_t<float, float>(a, grid, block, st);
  return launch_pcg_t<float, double>(a, grid, block, st);
}

cudaError_t pcg_occupancy(const Layout& L, bool val_f32, bool fac_f32, int block, int smem, int* ctas) {
  if (!val_f32 && !fac_f32) return pcg_occupancy_t<double, double>(L, block, smem, ctas);
  if (!val_f32 && fac_f32) return pcg_occupancy_t<double, float>(L, block, smem, ctas);
  if (val_f32 && fac_f32) return pcg_occupancy_t<float, float>(L, block, smem, ctas);
  return pcg_occupancy_t<float, double>(L, block, smem, ctas);
}

}  // namespace pc

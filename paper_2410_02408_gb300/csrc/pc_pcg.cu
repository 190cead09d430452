// Instantiations of the persistent CG kernel for every (CSR value type, factor type)
// pair and the block sizes with unrolled apply paths (8, 16, 32, 64; others use the
// runtime-block-size path).
#include "pc_pcg.cuh"

namespace pc {

cudaError_t launch_pcg(const PcgArgs& a, bool val_f32, bool fac_f32, int grid, int block, cudaStream_t st) {
  if (!val_f32 && !fac_f32) return launch_pcg_t<double, double>(a, grid, block, st);
  if (!val_f32 && fac_f32) return launch_pcg_t<double, float>(a, grid, block, st);
  if (val_f32 && fac_f32) return launch_pcg_t<float, float>(a, grid, block, st);
  return launch_pcg_t<float, double>(a, grid, block, st);
}

cudaError_t pcg_occupancy(const Layout& L, bool val_f32, bool fac_f32, int block, int* ctas) {
  if (!val_f32 && !fac_f32) return pcg_occupancy_t<double, double>(L, block, ctas);
  if (!val_f32 && fac_f32) return pcg_occupancy_t<double, float>(L, block, ctas);
  if (val_f32 && fac_f32) return pcg_occupancy_t<float, float>(L, block, ctas);
  return pcg_occupancy_t<float, double>(L, block, ctas);
}

}  // namespace pc

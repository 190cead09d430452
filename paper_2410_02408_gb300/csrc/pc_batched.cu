// Batched mode placeholder: replaced by the cluster-per-system persistent kernel.
#include "pc.h"
#include "pc_kernels.cuh"

extern "C" pc_status pc_batched_impl(const pc_batch*, const double*, double*, double, int32_t, int32_t, int32_t*,
                                     int32_t*, double*, pc_solve_info*, void*) {
  return PC_ERR_INVALID_ARG;
}

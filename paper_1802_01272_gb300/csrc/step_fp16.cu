// step_fp16.cu -- instantiations of the fused CTU step kernel for FP16 shifted
// storage (f - w rho_ref kept as half in memory, arithmetic in FP32).
#include "lbm_internal.h"

namespace ctulbm {

#include "step_select.cuh"

using Sel16 = StepSelect<float, __half>;

cudaError_t launch_step_f16(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s) {
  return Sel16::launch(a, maps, order, lim, vec, grid, smem, s);
}

void* step_kernel_ptr_f16(int order, int lim, bool vec, bool regu) {
  return Sel16::select(order, lim, vec, false, regu);
}

int step_occupancy_f16(int order, int lim, bool vec, bool regu, size_t smem) {
  return Sel16::occupancy(order, lim, vec, regu, smem);
}

}  // namespace ctulbm

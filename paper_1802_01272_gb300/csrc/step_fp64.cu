// step_fp64.cu -- instantiations of the fused CTU step kernel for double storage.
#include "lbm_internal.h"

namespace ctulbm {

#include "step_select.cuh"

using Sel64 = StepSelect<double, double>;

cudaError_t launch_step_f64(const StepArgs<double>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s) {
  return Sel64::launch(a, maps, order, lim, vec, grid, smem, s);
}

void* step_kernel_ptr_f64(int order, int lim, bool vec, bool regu) {
  return Sel64::select(order, lim, vec, false, regu);
}

int step_occupancy_f64(int order, int lim, bool vec, bool regu, size_t smem) {
  return Sel64::occupancy(order, lim, vec, regu, smem);
}

}  // namespace ctulbm

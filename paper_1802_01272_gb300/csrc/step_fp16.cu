// step_fp16.cu -- instantiations of the fused CTU step kernel for FP16 shifted
// storage (f - w rho_ref kept as half in memory, arithmetic in FP32).
#include "lbm_internal.h"

namespace ctulbm {

namespace {
template <int ORDER, int LIM, bool VEC>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&step_kernel<float, __half, ORDER, LIM, VEC>);
}

void* select(int order, int lim, bool vec) {
  if (order == 1) return vec ? kernel_ptr<1, 0, true>() : kernel_ptr<1, 0, false>();
  switch (lim) {
    case 1: return vec ? kernel_ptr<2, 1, true>() : kernel_ptr<2, 1, false>();
    case 2: return vec ? kernel_ptr<2, 2, true>() : kernel_ptr<2, 2, false>();
    default: return vec ? kernel_ptr<2, 0, true>() : kernel_ptr<2, 0, false>();
  }
}
}  // namespace

cudaError_t launch_step_f16(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s) {
  // the shared-memory attribute was set by step_occupancy_* when the handle was made
  void* fn = select(order, lim, vec);
  void* args[] = {const_cast<StepArgs<float>*>(&a), const_cast<RowMaps*>(&maps)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s);
}

void* step_kernel_ptr_f16(int order, int lim, bool vec) { return select(order, lim, vec); }

int step_occupancy_f16(int order, int lim, bool vec, size_t smem) {
  void* fn = select(order, lim, vec);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace ctulbm

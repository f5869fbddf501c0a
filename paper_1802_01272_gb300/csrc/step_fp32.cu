// step_fp32.cu -- instantiations of the fused CTU step kernel for float storage,
// single-lattice and batched.
#include "lbm_internal.h"

namespace ctulbm {

#include "step_select.cuh"

using Sel32 = StepSelect<float, float>;

cudaError_t launch_step_f32(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s) {
  return Sel32::launch(a, maps, order, lim, vec, grid, smem, s);
}

void* step_kernel_ptr_f32(int order, int lim, bool vec, bool regu) {
  return Sel32::select(order, lim, vec, false, regu);
}

int step_occupancy_f32(int order, int lim, bool vec, bool regu, size_t smem) {
  return Sel32::occupancy(order, lim, vec, regu, smem);
}

// Batched lattices always stage by tensor copies (lbm_step_many groups only
// lattices that have tensor maps).
namespace {
template <int ORDER, int LIM, bool REGU>
void* batch_ptr() {
  return reinterpret_cast<void*>(&step_batch_kernel<float, ORDER, LIM, true, REGU>);
}
template <bool REGU>
void* batch_by_scheme(int order, int lim) {
  if (order == 1) return batch_ptr<1, 0, REGU>();
  switch (lim) {
    case 1: return batch_ptr<2, 1, REGU>();
    case 2: return batch_ptr<2, 2, REGU>();
    default: return batch_ptr<2, 0, REGU>();
  }
}
void* select_batch(int order, int lim, bool regu) {
  return regu ? batch_by_scheme<true>(order, lim) : batch_by_scheme<false>(order, lim);
}
}  // namespace

static_assert(sizeof(BatchArgs<float>) <= 32764, "batched launch exceeds kernel parameter space");

cudaError_t launch_step_batch_f32(const BatchArgs<float>& b, int order, int lim, bool regu,
                                  int grid, size_t smem, cudaStream_t s) {
  void* fn = select_batch(order, lim, regu);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<BatchArgs<float>*>(&b)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s);
}

void* step_batch_kernel_ptr_f32(int order, int lim, bool regu) {
  return select_batch(order, lim, regu);
}

int step_batch_occupancy_f32(int order, int lim, bool regu, size_t smem) {
  void* fn = select_batch(order, lim, regu);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace ctulbm

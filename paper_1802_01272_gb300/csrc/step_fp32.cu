// step_fp32.cu -- instantiations of the fused CTU step kernel for float storage.
#include "lbm_internal.h"

namespace ctulbm {

namespace {
template <int ORDER, int LIM, bool VEC, bool DIAG>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&step_kernel<float, float, ORDER, LIM, VEC, DIAG>);
}

template <bool DIAG>
void* select_d(int order, int lim, bool vec) {
  if (order == 1) return vec ? kernel_ptr<1, 0, true, DIAG>() : kernel_ptr<1, 0, false, DIAG>();
  switch (lim) {
    case 1: return vec ? kernel_ptr<2, 1, true, DIAG>() : kernel_ptr<2, 1, false, DIAG>();
    case 2: return vec ? kernel_ptr<2, 2, true, DIAG>() : kernel_ptr<2, 2, false, DIAG>();
    default: return vec ? kernel_ptr<2, 0, true, DIAG>() : kernel_ptr<2, 0, false, DIAG>();
  }
}

// the variant with fused diagnostics is a separate kernel, so the plain step
// carries none of their instructions
void* select(int order, int lim, bool vec, bool diag) {
  return diag ? select_d<true>(order, lim, vec) : select_d<false>(order, lim, vec);
}
}  // namespace

cudaError_t launch_step_f32(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s) {
  // the shared-memory attribute was set by step_occupancy_* when the handle was made
  void* fn = select(order, lim, vec, a.diag_mass != nullptr);
  void* args[] = {const_cast<StepArgs<float>*>(&a), const_cast<RowMaps*>(&maps)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s);
}

void* step_kernel_ptr_f32(int order, int lim, bool vec) { return select(order, lim, vec, false); }

// Sets the shared-memory attribute of both variants (with and without fused
// diagnostics); returns the CTAs per SM both reach.
int step_occupancy_f32(int order, int lim, bool vec, size_t smem) {
  int occ = 1 << 30;
  for (int d = 0; d < 2; ++d) {
    void* fn = select(order, lim, vec, d == 1);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, smem) != cudaSuccess) return 0;
    occ = n < occ ? n : occ;
  }
  return occ;
}

namespace {
template <int ORDER, int LIM, bool VEC>
void* batch_ptr() {
  return reinterpret_cast<void*>(&step_batch_kernel<float, ORDER, LIM, VEC>);
}
void* select_batch(int order, int lim, bool vec) {
  if (order == 1) return vec ? batch_ptr<1, 0, true>() : batch_ptr<1, 0, false>();
  switch (lim) {
    case 1: return vec ? batch_ptr<2, 1, true>() : batch_ptr<2, 1, false>();
    case 2: return vec ? batch_ptr<2, 2, true>() : batch_ptr<2, 2, false>();
    default: return vec ? batch_ptr<2, 0, true>() : batch_ptr<2, 0, false>();
  }
}
}  // namespace

static_assert(sizeof(BatchArgs<float>) <= 32764, "batched launch exceeds kernel parameter space");

cudaError_t launch_step_batch_f32(const BatchArgs<float>& b, int order, int lim, bool vec, int grid,
                                  size_t smem, cudaStream_t s) {
  void* fn = select_batch(order, lim, vec);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<BatchArgs<float>*>(&b)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s);
}

int step_batch_occupancy_f32(int order, int lim, bool vec, size_t smem) {
  void* fn = select_batch(order, lim, vec);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace ctulbm

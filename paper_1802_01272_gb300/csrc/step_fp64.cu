// step_fp64.cu -- instantiations of the fused CTU step kernel for double storage.
#include "lbm_internal.h"

namespace ctulbm {

namespace {
template <int ORDER, int LIM, bool VEC, bool DIAG>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&step_kernel<double, double, ORDER, LIM, VEC, DIAG>);
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

cudaError_t launch_step_f64(const StepArgs<double>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s) {
  // the shared-memory attribute was set by step_occupancy_* when the handle was made
  void* fn = select(order, lim, vec, a.diag_mass != nullptr);
  void* args[] = {const_cast<StepArgs<double>*>(&a), const_cast<RowMaps*>(&maps)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s);
}

void* step_kernel_ptr_f64(int order, int lim, bool vec) { return select(order, lim, vec, false); }

// Sets the shared-memory attribute of both variants (with and without fused
// diagnostics); returns the CTAs per SM both reach.
int step_occupancy_f64(int order, int lim, bool vec, size_t smem) {
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

}  // namespace ctulbm

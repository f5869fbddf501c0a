// step_select.cuh -- launch-time selection of the step kernel instantiation
// for one storage type (included by step_fp32.cu, step_fp64.cu, step_fp16.cu
// inside namespace ctulbm): scheme (CTU1, CTU2 with the MC limiter or with a
// fixed limiter), staging (tensor copies or per-thread loads), fused
// diagnostics and the regularised collision are compile-time choices, so the
// plain step's loop carries no code for the others.
#pragma once

template <typename T, typename ST>
struct StepSelect {
  template <int ORDER, int LIM, bool VEC, bool DIAG, bool REGU>
  static void* ptr() {
    return reinterpret_cast<void*>(&step_kernel<T, ST, ORDER, LIM, VEC, DIAG, REGU>);
  }
  template <bool VEC, bool DIAG, bool REGU>
  static void* by_scheme(int order, int lim) {
    if (order == 1) return ptr<1, 0, VEC, DIAG, REGU>();
    switch (lim) {
      case 1: return ptr<2, 1, VEC, DIAG, REGU>();
      case 2: return ptr<2, 2, VEC, DIAG, REGU>();
      default: return ptr<2, 0, VEC, DIAG, REGU>();
    }
  }
  template <bool VEC>
  static void* by_mode(int order, int lim, bool diag, bool regu) {
    if (diag)
      return regu ? by_scheme<VEC, true, true>(order, lim) : by_scheme<VEC, true, false>(order, lim);
    return regu ? by_scheme<VEC, false, true>(order, lim) : by_scheme<VEC, false, false>(order, lim);
  }
  static void* select(int order, int lim, bool vec, bool diag, bool regu) {
    return vec ? by_mode<true>(order, lim, diag, regu) : by_mode<false>(order, lim, diag, regu);
  }
  static cudaError_t launch(const StepArgs<T>& a, const RowMaps& maps, int order, int lim, bool vec,
                            int grid, size_t smem, cudaStream_t s) {
    // the shared-memory attribute was set by occupancy() when the handle was made
    void* fn = select(order, lim, vec, a.diag_mass != nullptr, a.regularize != 0);
    void* args[] = {const_cast<StepArgs<T>*>(&a), const_cast<RowMaps*>(&maps)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s);
  }
  // Sets the shared-memory attribute of the plain and fused-diagnostics
  // variants; returns the CTAs per SM both reach (0 on error).
  static int occupancy(int order, int lim, bool vec, bool regu, size_t smem) {
    int occ = 1 << 30;
    for (int d = 0; d < 2; ++d) {
      void* fn = select(order, lim, vec, d == 1, regu);
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return 0;
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT, smem) != cudaSuccess) return 0;
      occ = n < occ ? n : occ;
    }
    return occ;
  }
};

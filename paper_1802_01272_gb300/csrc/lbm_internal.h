// lbm_internal.h -- launch interface between the C ABI (api.cu) and the
// kernels (step_fp32.cu, step_fp64.cu, aux.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"

namespace ctulbm {

// Parameters of the small per-node kernels (initialisation, conversion,
// moments, diagnostics).  Always FP64 on the host side.
struct AuxArgs {
  int Lx, Ly;
  long long plane;
  int storage64;     // 1: f is double, 0: f is float (shifted by w_k rho_ref)
  double rho_ref, Tt;
  double xi[16][2], w[16];
};

// One fused step kernel: returns cudaSuccess or the launch error.
// `maps` describe a.fin (RowMaps); they are read only when a.tma_ok.
cudaError_t launch_step_f32(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_step_f64(const StepArgs<double>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s);
// Several FP32 lattices in one launch (same scheme, limiter and column path).
cudaError_t launch_step_batch_f32(const BatchArgs<float>& b, int order, int lim, bool vec,
                                  int grid, size_t smem, cudaStream_t s);
int step_batch_occupancy_f32(int order, int lim, bool vec, size_t smem);
// Largest resident CTAs per SM for the selected step kernel (0 on error).
int step_occupancy_f32(int order, int lim, bool vec, size_t smem);
int step_occupancy_f64(int order, int lim, bool vec, size_t smem);

size_t step_smem_bytes(size_t elem);

// f = f^eq(rho, u) - w rho_ref from FP64 device fields.
cudaError_t launch_init_feq(const AuxArgs& a, void* f, const double* rho, const double* ux,
                            const double* uy, cudaStream_t s);
// FP64 [16][Ly][Lx] <-> storage.
cudaError_t launch_set_f(const AuxArgs& a, void* f, const double* src, cudaStream_t s);
cudaError_t launch_get_f(const AuxArgs& a, const void* f, double* dst, cudaStream_t s);
// rho, u of the stored f.
cudaError_t launch_moments(const AuxArgs& a, const void* f, double* rho, double* ux, double* uy,
                           cudaStream_t s);

// Diagnostics accumulators (device).
struct DiagAcc {
  double mass;
  double ring_sum;
  unsigned long long ring_n;
  unsigned long long nb, sx, sy, sxx, sxy, syy;
  unsigned long long rmin_key, rmax_key;  // order-preserving keys of FP64 rho
  double rho_center;
};
cudaError_t launch_diag(const AuxArgs& a, const void* f, double thr, double r_ring, DiagAcc* acc,
                        cudaStream_t s);
cudaError_t launch_hist(const AuxArgs& a, const void* f, int nbins, double lo, double hi,
                        unsigned long long* counts, cudaStream_t s);

}  // namespace ctulbm

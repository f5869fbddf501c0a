// lbm_internal.h -- launch interface between the C ABI (api.cu) and the
// kernels (step_fp32.cu, step_fp64.cu, aux.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"

namespace ctulbm {

enum { STORE_F32 = 0, STORE_F64 = 1, STORE_F16 = 2 };

// Parameters of the small per-node kernels (initialisation, conversion,
// moments, diagnostics).  Always FP64 on the host side.
struct AuxArgs {
  int Lx, Ly;
  long long plane;
  int storage;       // STORE_F32 / STORE_F16: f - w_k rho_ref as float / half; STORE_F64: f
  double rho_ref, Tt;
  double xi[16][2], w[16];
  float xif[16][2], wf[16];  // the same tables rounded to float on the host
};

// One fused step kernel: returns cudaSuccess or the launch error.  `vec`: the
// lattice has tensor maps (`maps`, for a.fin and a.fout) and stages by them.
cudaError_t launch_step_f32(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_step_f64(const StepArgs<double>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s);
// FP16 shifted storage, FP32 arithmetic (a.fin / a.fout hold half).
cudaError_t launch_step_f16(const StepArgs<float>& a, const RowMaps& maps, int order, int lim,
                            bool vec, int grid, size_t smem, cudaStream_t s);
// Several FP32 lattices in one launch (same scheme, limiter and collision;
// every lattice has tensor maps).
cudaError_t launch_step_batch_f32(const BatchArgs<float>& b, int order, int lim, bool regu,
                                  int grid, size_t smem, cudaStream_t s);
int step_batch_occupancy_f32(int order, int lim, bool regu, size_t smem);
// The batched kernel (for CUDA graph kernel nodes; its attribute is set by
// step_batch_occupancy_f32).
void* step_batch_kernel_ptr_f32(int order, int lim, bool regu);
// Largest resident CTAs per SM for the selected step kernel (0 on error).
int step_occupancy_f32(int order, int lim, bool vec, bool regu, size_t smem);
int step_occupancy_f64(int order, int lim, bool vec, bool regu, size_t smem);
int step_occupancy_f16(int order, int lim, bool vec, bool regu, size_t smem);
// The step kernel a launch_step_* call would run (for CUDA graph kernel nodes,
// whose parameters are (StepArgs, RowMaps) as in a direct launch).
void* step_kernel_ptr_f32(int order, int lim, bool vec, bool regu);
void* step_kernel_ptr_f64(int order, int lim, bool vec, bool regu);
void* step_kernel_ptr_f16(int order, int lim, bool vec, bool regu);

// Dynamic shared memory of the step kernel: staging ring in the storage type
// (stage_elem bytes per value), the other rings in the arithmetic type.
size_t step_smem_bytes(size_t stage_elem, size_t elem);

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

// aux.cu -- per-node kernels around the fused step: initialisation to f^eq
// (Eq. herfeq), FP64 <-> storage conversion, moments (Sec. II A) and the
// diagnostics of Sec. III B-C (mass, bubble-site sums of Eq. gyr, probe
// densities, density histogram).
#include "lbm_internal.h"

namespace ctulbm {

namespace {

constexpr int BS = 256;

__device__ __forceinline__ double load_f(const void* f, int storage64, long long idx) {
  return storage64 ? static_cast<const double*>(f)[idx]
                   : (double)static_cast<const float*>(f)[idx];
}

__device__ __forceinline__ void store_f(void* f, int storage64, long long idx, double v) {
  if (storage64)
    static_cast<double*>(f)[idx] = v;
  else
    static_cast<float*>(f)[idx] = (float)v;
}

// Eq. (herfeq) with the storage shift w_k rho_ref removed.
__device__ void feq_shifted(const AuxArgs& a, double rho, double ux, double uy, double* out) {
  const double T = a.Tt, u2 = ux * ux + uy * uy;
  for (int k = 0; k < 16; ++k) {
    const double xx = a.xi[k][0], xy = a.xi[k][1];
    const double cu = xx * ux + xy * uy, x2 = xx * xx + xy * xy;
    const double p = 1.0 + cu + 0.5 * (cu * cu - u2 + (T - 1.0) * (x2 - 2.0)) +
                     cu / 6.0 * (cu * cu - 3.0 * u2 + 3.0 * (T - 1.0) * (x2 - 4.0));
    out[k] = a.w[k] * (rho * p - a.rho_ref);
  }
}

__global__ void init_feq_kernel(const AuxArgs a, void* f, const double* rho, const double* ux,
                                const double* uy) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  double fe[16];
  feq_shifted(a, rho[q], ux[q], uy[q], fe);
  for (int k = 0; k < 16; ++k) store_f(f, a.storage64, k * a.plane + q, fe[k]);
}

__global__ void set_f_kernel(const AuxArgs a, void* f, const double* src) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  for (int k = 0; k < 16; ++k)
    store_f(f, a.storage64, k * a.plane + q, src[k * a.plane + q] - a.w[k] * a.rho_ref);
}

__global__ void get_f_kernel(const AuxArgs a, const void* f, double* dst) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  for (int k = 0; k < 16; ++k)
    dst[k * a.plane + q] = load_f(f, a.storage64, k * a.plane + q) + a.w[k] * a.rho_ref;
}

__device__ __forceinline__ void node_moments(const AuxArgs& a, const void* f, long long q,
                                             double& rho, double& mx, double& my) {
  double d = 0.0;
  mx = my = 0.0;
  for (int k = 0; k < 16; ++k) {
    const double v = load_f(f, a.storage64, k * a.plane + q);
    d += v;
    mx += v * a.xi[k][0];
    my += v * a.xi[k][1];
  }
  rho = a.rho_ref + d;  // sum_k w_k = 1 and sum_k w_k xi_k = 0 undo the shift
}

__global__ void moments_kernel(const AuxArgs a, const void* f, double* rho, double* ux,
                               double* uy) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  double r, mx, my;
  node_moments(a, f, q, r, mx, my);
  rho[q] = r;
  ux[q] = mx / r;
  uy[q] = my / r;
}

// order-preserving 64-bit key of a double
__device__ __forceinline__ unsigned long long dkey(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void diag_kernel(const AuxArgs a, const void* f, double thr, double r_ring,
                            DiagAcc* acc) {
  double mass = 0.0, ring = 0.0;
  unsigned long long nring = 0, nb = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
  unsigned long long kmin = ~0ULL, kmax = 0ULL;
  const double cx = a.Lx / 2.0, cy = a.Ly / 2.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.plane;
       q += (long long)gridDim.x * blockDim.x) {
    double rho, mx, my;
    node_moments(a, f, q, rho, mx, my);
    const unsigned long long i = (unsigned long long)(q % a.Lx), j = (unsigned long long)(q / a.Lx);
    mass += rho;
    const unsigned long long key = dkey(rho);
    kmin = min(kmin, key);
    kmax = max(kmax, key);
    if (rho < thr) {
      nb += 1;
      sx += i;
      sy += j;
      sxx += i * i;
      sxy += i * j;
      syy += j * j;
    }
    const double dr = hypot((double)i - cx, (double)j - cy) - r_ring;
    if (fabs(dr) < 0.5) {
      ring += rho;
      nring += 1;
    }
    if ((long long)i == a.Lx / 2 && (long long)j == a.Ly / 2) acc->rho_center = rho;
  }
  mass = warp_sum(mass);
  ring = warp_sum(ring);
  nring = warp_sum(nring);
  nb = warp_sum(nb);
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  sxx = warp_sum(sxx);
  sxy = warp_sum(sxy);
  syy = warp_sum(syy);
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_down_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_down_sync(0xffffffffu, kmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc->mass, mass);
    atomicAdd(&acc->ring_sum, ring);
    atomicAdd(&acc->ring_n, nring);
    atomicAdd(&acc->nb, nb);
    atomicAdd(&acc->sx, sx);
    atomicAdd(&acc->sy, sy);
    atomicAdd(&acc->sxx, sxx);
    atomicAdd(&acc->sxy, sxy);
    atomicAdd(&acc->syy, syy);
    atomicMin(&acc->rmin_key, kmin);
    atomicMax(&acc->rmax_key, kmax);
  }
}

__global__ void hist_kernel(const AuxArgs a, const void* f, int nbins, double lo, double hi,
                            unsigned long long* counts) {
  extern __shared__ unsigned int sh[];
  const bool priv = nbins <= 8192;
  if (priv)
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.plane;
       q += (long long)gridDim.x * blockDim.x) {
    double rho, mx, my;
    node_moments(a, f, q, rho, mx, my);
    const double t = (rho - lo) / (hi - lo) * nbins;
    if (t >= 0.0 && t < (double)nbins) {
      const int b = (int)t;
      if (priv)
        atomicAdd(&sh[b], 1u);
      else
        atomicAdd(&counts[b], 1ULL);
    }
  }
  __syncthreads();
  if (priv)
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
      if (sh[b]) atomicAdd(&counts[b], (unsigned long long)sh[b]);
}

unsigned grid_for(long long n) { return (unsigned)((n + BS - 1) / BS); }

}  // namespace

cudaError_t launch_init_feq(const AuxArgs& a, void* f, const double* rho, const double* ux,
                            const double* uy, cudaStream_t s) {
  init_feq_kernel<<<grid_for(a.plane), BS, 0, s>>>(a, f, rho, ux, uy);
  return cudaGetLastError();
}

cudaError_t launch_set_f(const AuxArgs& a, void* f, const double* src, cudaStream_t s) {
  set_f_kernel<<<grid_for(a.plane), BS, 0, s>>>(a, f, src);
  return cudaGetLastError();
}

cudaError_t launch_get_f(const AuxArgs& a, const void* f, double* dst, cudaStream_t s) {
  get_f_kernel<<<grid_for(a.plane), BS, 0, s>>>(a, f, dst);
  return cudaGetLastError();
}

cudaError_t launch_moments(const AuxArgs& a, const void* f, double* rho, double* ux, double* uy,
                           cudaStream_t s) {
  moments_kernel<<<grid_for(a.plane), BS, 0, s>>>(a, f, rho, ux, uy);
  return cudaGetLastError();
}

cudaError_t launch_diag(const AuxArgs& a, const void* f, double thr, double r_ring, DiagAcc* acc,
                        cudaStream_t s) {
  unsigned g = grid_for(a.plane);
  if (g > 4096) g = 4096;
  diag_kernel<<<g, BS, 0, s>>>(a, f, thr, r_ring, acc);
  return cudaGetLastError();
}

cudaError_t launch_hist(const AuxArgs& a, const void* f, int nbins, double lo, double hi,
                        unsigned long long* counts, cudaStream_t s) {
  unsigned g = grid_for(a.plane);
  if (g > 2048) g = 2048;
  const size_t sh = nbins <= 8192 ? sizeof(unsigned int) * nbins : 0;
  hist_kernel<<<g, BS, sh, s>>>(a, f, nbins, lo, hi, counts);
  return cudaGetLastError();
}

size_t step_smem_bytes(size_t elem) {
  return elem * ((size_t)FR * 16 * SREG + 6 * (size_t)MR * REG + (size_t)NODE_W * REG +
                 (size_t)REG_W * REG);
}

}  // namespace ctulbm

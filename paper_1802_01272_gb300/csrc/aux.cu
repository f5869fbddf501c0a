// aux.cu -- per-node kernels around the fused step: initialisation to f^eq
// (Eq. herfeq), FP64 <-> storage conversion, moments (Sec. II A) and the
// diagnostics of Sec. III B-C (mass, bubble-site sums of Eq. gyr, probe
// densities, density histogram).
#include <type_traits>

#include "lbm_internal.h"

namespace ctulbm {

namespace {

constexpr int BS = 256;

// Arithmetic type of a storage type: double for double, float for float and half.
template <typename S>
struct Comp {
  using type = float;
};
template <>
struct Comp<double> {
  using type = double;
};

// Velocity table in the arithmetic precision, loaded once per thread.  The
// float table comes rounded from the host, so the one-node-per-thread kernels
// do no double -> float conversions (GB300's FP64 path is narrow).
template <typename T>
struct Vel {
  T x[16], y[16], w[16];
  __device__ explicit Vel(const AuxArgs& a) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x[k] = a.xi[k][0];
      y[k] = a.xi[k][1];
      w[k] = a.w[k];
    }
  }
};
template <>
struct Vel<float> {
  float x[16], y[16], w[16];
  __device__ explicit Vel(const AuxArgs& a) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x[k] = a.xif[k][0];
      y[k] = a.xif[k][1];
      w[k] = a.wf[k];
    }
  }
};

// Eq. (herfeq) with the storage shift w_k rho_ref removed:
// f^eq - w rho_ref = w [ (rho - rho_ref) + rho (P_k - 1) ],
// P_k - 1 = xi.u + [(xi.u)^2 - u^2 + (T-1)(xi^2-2)]/2 + xi.u [(xi.u)^2 - 3u^2 + 3(T-1)(xi^2-4)]/6
template <typename S>
__global__ void init_feq_kernel(const AuxArgs a, S* f, const double* rho, const double* ux,
                                const double* uy) {
  using T = typename Comp<S>::type;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  const Vel<T> v(a);
  const T r = (T)rho[q], drho = (T)(rho[q] - a.rho_ref), u = (T)ux[q], w = (T)uy[q];
  const T Tm1 = (T)(a.Tt - 1.0), u2 = u * u + w * w;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const T cu = v.x[k] * u + v.y[k] * w, x2 = v.x[k] * v.x[k] + v.y[k] * v.y[k];
    const T pm1 = cu + T(0.5) * (cu * cu - u2 + Tm1 * (x2 - T(2))) +
                  cu / T(6) * (cu * cu - T(3) * u2 + T(3) * Tm1 * (x2 - T(4)));
    f[k * a.plane + q] = to_store<S, T>(v.w[k] * (drho + r * pm1));
  }
}

template <typename S>
__global__ void set_f_kernel(const AuxArgs a, S* f, const double* src) {
  using T = typename Comp<S>::type;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  for (int k = 0; k < 16; ++k)
    f[k * a.plane + q] = to_store<S, T>((T)(src[k * a.plane + q] - a.w[k] * a.rho_ref));
}

template <typename S>
__global__ void get_f_kernel(const AuxArgs a, const S* f, double* dst) {
  using T = typename Comp<S>::type;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  for (int k = 0; k < 16; ++k)
    dst[k * a.plane + q] = (double)from_store<S, T>(f[k * a.plane + q]) + a.w[k] * a.rho_ref;
}

// rho - rho_ref = sum_k f_k and rho u = sum_k f_k xi_k of the stored (shifted) f
template <typename S, typename T>
__device__ __forceinline__ void node_moments(const AuxArgs& a, const Vel<T>& v, const S* f,
                                             long long q, T& drho, T& mx, T& my) {
  drho = mx = my = T(0);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const T fv = from_store<S, T>(f[k * a.plane + q]);
    drho += fv;
    mx += fv * v.x[k];
    my += fv * v.y[k];
  }
}

template <typename S>
__global__ void moments_kernel(const AuxArgs a, const S* f, double* rho, double* ux, double* uy) {
  using T = typename Comp<S>::type;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.plane) return;
  const Vel<T> v(a);
  T d, mx, my;
  node_moments(a, v, f, q, d, mx, my);
  const T r = (T)a.rho_ref + d;
  rho[q] = (double)r;
  ux[q] = (double)(mx / r);
  uy[q] = (double)(my / r);
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

// Ring membership |dist - r_ring| < 1/2 tested exactly on integers:
// (2r-1)^2 < (2i - Lx)^2 + (2j - Ly)^2 < (2r+1)^2.
template <typename S>
__global__ void diag_kernel(const AuxArgs a, const S* f, double thr, double r_ring, DiagAcc* acc) {
  using T = typename Comp<S>::type;
  const Vel<T> v(a);
  double mass = 0.0, ring = 0.0;
  unsigned long long nring = 0, nb = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
  unsigned long long kmin = ~0ULL, kmax = 0ULL;
  const double rin = fmax(2.0 * r_ring - 1.0, 0.0), rout = 2.0 * r_ring + 1.0;
  const double rin2 = 2.0 * r_ring - 1.0 > 0.0 ? rin * rin : -1.0, rout2 = rout * rout;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.plane;
       q += (long long)gridDim.x * blockDim.x) {
    T d, mx, my;
    node_moments(a, v, f, q, d, mx, my);
    const double rho = a.rho_ref + (double)d;
    const long long i = q % a.Lx, j = q / a.Lx;
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
    const long long di = 2 * i - a.Lx, dj = 2 * j - a.Ly;
    const double d2 = (double)(di * di + dj * dj);
    if (d2 > rin2 && d2 < rout2) {
      ring += rho;
      nring += 1;
    }
    if (i == a.Lx / 2 && j == a.Ly / 2) acc->rho_center = rho;
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

template <typename S>
__global__ void hist_kernel(const AuxArgs a, const S* f, int nbins, double lo, double hi,
                            unsigned long long* counts) {
  using T = typename Comp<S>::type;
  extern __shared__ unsigned int sh[];
  const Vel<T> v(a);
  const bool priv = nbins <= 8192;
  if (priv)
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.plane;
       q += (long long)gridDim.x * blockDim.x) {
    T d, mx, my;
    node_moments(a, v, f, q, d, mx, my);
    const double rho = a.rho_ref + (double)d;
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

// Calls fn(typed f) with f cast to the storage type of a.storage.
template <typename F>
cudaError_t by_storage(const AuxArgs& a, const void* f, F fn) {
  switch (a.storage) {
    case STORE_F64: fn(static_cast<const double*>(f)); break;
    case STORE_F16: fn(static_cast<const __half*>(f)); break;
    default: fn(static_cast<const float*>(f)); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_init_feq(const AuxArgs& a, void* f, const double* rho, const double* ux,
                            const double* uy, cudaStream_t s) {
  return by_storage(a, f, [&](auto p) {
    using S = std::remove_const_t<std::remove_pointer_t<decltype(p)>>;
    init_feq_kernel<S><<<grid_for(a.plane), BS, 0, s>>>(a, const_cast<S*>(p), rho, ux, uy);
  });
}

cudaError_t launch_set_f(const AuxArgs& a, void* f, const double* src, cudaStream_t s) {
  return by_storage(a, f, [&](auto p) {
    using S = std::remove_const_t<std::remove_pointer_t<decltype(p)>>;
    set_f_kernel<S><<<grid_for(a.plane), BS, 0, s>>>(a, const_cast<S*>(p), src);
  });
}

cudaError_t launch_get_f(const AuxArgs& a, const void* f, double* dst, cudaStream_t s) {
  return by_storage(a, f, [&](auto p) {
    get_f_kernel<<<grid_for(a.plane), BS, 0, s>>>(a, p, dst);
  });
}

cudaError_t launch_moments(const AuxArgs& a, const void* f, double* rho, double* ux, double* uy,
                           cudaStream_t s) {
  return by_storage(a, f, [&](auto p) {
    moments_kernel<<<grid_for(a.plane), BS, 0, s>>>(a, p, rho, ux, uy);
  });
}

cudaError_t launch_diag(const AuxArgs& a, const void* f, double thr, double r_ring, DiagAcc* acc,
                        cudaStream_t s) {
  unsigned g = grid_for(a.plane);
  if (g > 4096) g = 4096;
  return by_storage(a, f, [&](auto p) { diag_kernel<<<g, BS, 0, s>>>(a, p, thr, r_ring, acc); });
}

cudaError_t launch_hist(const AuxArgs& a, const void* f, int nbins, double lo, double hi,
                        unsigned long long* counts, cudaStream_t s) {
  unsigned g = grid_for(a.plane);
  if (g > 2048) g = 2048;
  const size_t sh = nbins <= 8192 ? sizeof(unsigned int) * nbins : 0;
  return by_storage(a, f, [&](auto p) {
    hist_kernel<<<g, BS, sh, s>>>(a, p, nbins, lo, hi, counts);
  });
}

size_t step_smem_bytes(size_t stage_elem, size_t elem) {
  const size_t elems = (size_t)FROWS * FRS + 4 * (size_t)MROWS * MP;  // f*, drho, ux, uy, phi
  // + 128 bytes to align the staging ring (which also holds the output tiles)
  // for tensor copies; the fused diagnostics' bubble-site sums, the staging
  // slots' mbarriers and the CTA's wait-abort flag
  const size_t scol = stage_elem == 2 ? scol_of<__half>() : scol_of<float>();
  return 128 + stage_elem * (size_t)NSLOT * RPI * 16 * scol +
         elem * elems + 6 * sizeof(unsigned long long) + NSLOT * sizeof(unsigned long long) +
         2 * sizeof(int);
}

}  // namespace ctulbm

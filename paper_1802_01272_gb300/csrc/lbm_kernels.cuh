// lbm_kernels.cuh -- device code of the CTU lattice Boltzmann time step for
// GB300 (sm_103a), after arXiv:1802.01272 (Sofonea et al.).
//
// One step, as Sec. II C splits Eq. (eBGK): advection of each f_k over its
// upwind-corner stencil (CTU1, Eq. ctueq; CTU2 with the MC limiter,
// Sec. II C 2), then on the advected f*: rho, u, g (Eq. eder with Eq. evdw,
// 25-point stencils: fourth-order gradient of p^i - p^w, isotropic gradient of
// the 9-point Laplacian), f^eq (Eq. herfeq), F_k (Eq. herforce), BGK
// relaxation (optionally regularised, Eq. ereg), and the density reservoir of
// Sec. III A.
//
// Kernel layout (step_kernel): a CTA owns a strip of TW = 56 output columns
// [56 s, 56 s + 56) and streams down a range of rows, RPI = 4 rows per
// iteration.  Its 256 threads are (velocity k, group g of four columns) over a
// 64-column region [56 s - 4, 56 s + 60): the strip, the two-column halo where
// rho* is needed for the force stencil, and two more columns that complete the
// four-column groups.  Strips start on 32-byte sectors, so every output sector
// is written whole by one warp store (a partly written sector would cost a
// DRAM read-modify-write).  Warps hold one sign quadrant (sgn xi_x, sgn xi_y), so
// the upwind side of every stencil is a compile-time constant inside a warp.
// Per iteration of four rows a0 .. a0+3 the CTA
//   L   issues cp.async copies of the f^n rows of the NEXT iteration into a
//       shared staging ring (one iteration of look-ahead hides DRAM latency);
//   P1  advects rows a0..a0+3 of every plane from the staging ring (the CTU2
//       jumps, limited corrections and their differences of the previous rows
//       live in registers) into a ring of advected rows f*;
//   P2  one thread per node: rho*, u*, p^i - p^w of rows a0..a0+3;
//   P3  one thread per node: 9-point Laplacian of rho* on rows a0-1..a0+2;
//   P4  one thread per node on rows a0-2..a0+1: gradients (5x5 of p^i - p^w,
//       3x3 of the Laplacian) -> g, the collision coefficients, then all 16
//       planes relaxed and stored
//       (coalesced 128-byte warp stores per plane).
// Four CTA barriers per four rows.  Global memory is read once per step for
// f^n (halo columns of neighbouring strips are L2 hits) and written once.
#pragma once

#include <cuda.h>  // CUtensorMap (type only)
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ctulbm {

constexpr int NG = 16;          // four-column groups in a strip region
constexpr int REG = 4 * NG;     // region columns: output strip plus 4 columns per side
constexpr int TW = REG - 8;     // output columns per strip (56: strips start on 32-byte sectors)
constexpr int XOFF = 4;         // region column of the strip's first output column
constexpr int NT = 16 * NG;     // threads per CTA
constexpr int RPI = 4;          // rows per pipeline iteration
constexpr int SG = NG + 2;      // staging groups per plane row: region plus one group per side
constexpr int SCOL = 4 * SG;    // staging columns per plane row
constexpr int SROWS = 3 * RPI;  // staging ring rows: three batches of RPI rows (the batch read,
                                // the last row of the one before, the batch being loaded)
constexpr int FROWS = 8;        // advected-row ring (power of two)
constexpr int MROWS = 8;        // moment rings (power of two)
constexpr int WARMUP = 5;       // pipeline rows before the first output row of a segment

// Per-velocity constants, computed on the host in FP64 and rounded to T.
template <typename T>
struct VelConst {
  T xi_x, xi_y, w;
  T c00, c10, c01, c11;     // Eq. (ctueq) corner weights (1-cx)(1-cy), cx(1-cy), cy(1-cx), cx cy
  T a1, a2, b1, b2;         // CTU2 correction weights acting on half-limited jumps
  T omA, Ak, omB, Bk;       // omega*A_k, A_k, omega*B_k, B_k; A_k=(T-1)(xi^2-2)/2, B_k=(T-1)(xi^2-4)/2
  T gbot, gtop;             // wall ghost-row values (storage variable)
  T r2xx, r2xy, r2yy, r3xxx, r3xxy, r3xyy, r3yyy;  // Eq. (ereg) weights, 1/n! folded in
};

// Per-class constants of the collision (class = velocity group of Table I).
template <typename T>
struct ClassConst {
  T omA, Ak, omB, Bk, w;
};

template <typename T>
struct StepArgs {
  const void* fin;          // f^n, [16][Ly][Lx] in the storage type (float, double or half)
  void* fout;               // f^{n+1}
  int Lx, Ly;
  long long plane;          // Lx * Ly
  int nstrip;
  int row_block;            // rows per work item
  long long items;          // work items: ceil(Ly / row_block) * nstrip, row-block major
  unsigned long long* sched;  // [2]: next item, CTAs done (reset by the last CTA)
  // fused diagnostics of the state after this step (null: off): FP64 mass,
  // bubble sites rho < diag_thr and their exact integer moment sums
  double* diag_mass;
  unsigned long long* diag_sums;  // [6]: nb, sx, sy, sxx, sxy, syy
  T diag_thr;
  int walls, reservoir, regularize;
  T rho_ref, Tt, a, b, kappa, inv_ds, inv_ds2, dt, omega, one_m_omega, om2, om6;
  T rho_ext, rbc2, cxc, cyc;
  unsigned int* err;         // bit 0: non-finite or non-positive rho; bit 1: a wait timed out
  int tma_ok;               // the launch's tensor map describes fin (interior strips use it)
  T xlo, xhi;               // |xi| components sqrt(3 - sqrt 6), sqrt(3 + sqrt 6)
  ClassConst<T> cls[4];     // groups (lo,lo), (hi,lo), (lo,hi), (hi,hi)
  VelConst<T> v[16];
};

// f^n as a 3-D tensor (x, plane, row) for tensor copies of staged rows:
// m[0] copies boxes of SCOL columns x 16 planes x RPI rows, m[1] single rows.
struct RowMaps {
  CUtensorMap m[2];
};

constexpr int MAXB = 16;  // lattices per batched launch (kernel parameter space)

template <typename T>
struct BatchArgs {
  int count;
  unsigned long long* sched;       // [2] work counter and done counter
  long long item_start[MAXB + 1];  // prefix sums of the lattices' work items
  StepArgs<T> L[MAXB];
};

// ---------------------------------------------------------------- helpers
// Storage of f (float, double, or half for FP16 shifted storage) and the
// arithmetic type T: conversions on load and store.
template <typename S, typename T>
__device__ __forceinline__ T from_store(S v) {
  return (T)v;
}
template <>
__device__ __forceinline__ float from_store<__half, float>(__half v) {
  return __half2float(v);
}
template <typename S, typename T>
__device__ __forceinline__ S to_store(T v) {
  return (S)v;
}
template <>
__device__ __forceinline__ __half to_store<__half, float>(float v) {
  return __float2half_rn(v);
}
__device__ __forceinline__ float flip_sign(float v, float s) {
  return __int_as_float(__float_as_int(v) ^ (__float_as_int(s) & 0x80000000));
}
__device__ __forceinline__ double flip_sign(double v, double s) {
  return __longlong_as_double(__double_as_longlong(v) ^
                              (__double_as_longlong(s) & (long long)0x8000000000000000ULL));
}

__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(fmin(a, b), c); }
// Reciprocal in FP32: the hardware approximation (relative error below 2^-22),
// enough for u = (rho u)/rho and the pressure and force terms, which enter the
// update multiplied by dt; FP64 keeps the correctly rounded division.
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Half of the limited jump R * Psi(Ru / R) of Sec. II C 2.  For the MC limiter,
// with a = |R| and b = sgn(R) Ru, R Psi = sgn(R) max(0, min((a+b)/2, 2a, 2b)),
// which needs no division and is 0 at R = 0 (where Psi's argument is undefined).
template <int LIM, typename T>
__device__ __forceinline__ T half_limited(T R, T Ru) {
  if constexpr (LIM == 1) {
    return T(0);
  } else if constexpr (LIM == 2) {
    return T(0.5) * R;
  } else {
    T a = fabs(R);
    T b = flip_sign(Ru, R);
    T m = min3(T(0.25) * (a + b), a, b);
    m = fmax(m, T(0));
    return copysign(m, R);
  }
}

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

template <typename T>
__device__ __forceinline__ void sload4(const T* p, T* v) {
  if constexpr (sizeof(T) == 4) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    double2 t0 = reinterpret_cast<const double2*>(p)[0];
    double2 t1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
  }
}

// Twelve consecutive staged values (16-byte aligned for float/double, 8-byte
// for half) converted to the arithmetic type.
template <typename S, typename T>
__device__ __forceinline__ void sload12(const S* p, T* v) {
  if constexpr (sizeof(S) == 2) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const uint2 u = reinterpret_cast<const uint2*>(p)[m];
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
      v[4 * m] = a.x; v[4 * m + 1] = a.y; v[4 * m + 2] = b.x; v[4 * m + 3] = b.y;
    }
  } else {
    sload4(p, v);
    sload4(p + 4, v + 4);
    sload4(p + 8, v + 8);
  }
}

// ------------------------------------------------------ advection state
// Columns: the thread owns group columns 0..3.  f keeps five columns C5 =
// {own, own - sgn_x} (relative -1..3 for sgn_x > 0, else 0..4), loaded from
// the staged row.  Jumps, limited corrections and their differences are kept
// for the own four columns only: the value a stencil needs one column beyond
// the group is the neighbouring group's, taken from the adjacent lane (the 16
// groups of a velocity sit on 16 consecutive lanes).  At the two region edges
// that lane holds nothing useful; those columns (region 0 and 63) feed only
// rho* outside the stencils of the strip's outputs.
template <typename T>
struct AdvState {
  T F0[5], F1[5];  // f on row a and on the y-upwind row a - sgn_y
  T RY[4];         // sgn_y > 0: R^y(a);  sgn_y < 0: R^y(a+1)
  T SY[4];         // half-limited S^y(a)
  T A0[4], A1[4];  // x-differences of half-limited S^x on row a and on row a - sgn_y
};

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// One advection row for velocity k of quadrant (SX, SY).  `v` holds the newly
// loaded row (a+1 if SY > 0, a+2 if SY < 0) at relative columns -4..7.  All 32
// lanes of the warp must call it together (it exchanges neighbour columns).
template <int SX, int SY, int ORDER, int LIM, typename T>
__device__ __forceinline__ void advect_row(AdvState<T>& s, const T* v, const VelConst<T>& c,
                                           T* out) {
  constexpr int B5 = SX > 0 ? -1 : 0;  // relative column of C5[0]
  T Fn[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) Fn[m] = v[4 + B5 + m];

  T Bv[4], Bu = T(0), An[4];
  if constexpr (ORDER == 2) {
    T RYn[4], SYn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int mo = i - B5;
      if constexpr (SY > 0) {
        RYn[i] = Fn[mo] - s.F0[mo];                   // R^y(a+1)
        SYn[i] = half_limited<LIM>(RYn[i], s.RY[i]);  // S^y(a+1), upwind R^y(a)
      } else {
        RYn[i] = Fn[mo] - s.F1[mo];                   // R^y(a+2)
        SYn[i] = half_limited<LIM>(s.RY[i], RYn[i]);  // S^y(a+1), upwind R^y(a+2)
      }
      Bv[i] = SYn[i] - s.SY[i];                       // S^y(a+1) - S^y(a)
      s.RY[i] = RYn[i];
      s.SY[i] = SYn[i];
    }
    // B one column upwind in x: the neighbouring group's edge column
    if constexpr (SX > 0) Bu = shfl_up1(Bv[3]); else Bu = shfl_dn1(Bv[0]);
    // x direction on the new row: R^x(c) = f(c) - f(c-1)
    T RX[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) RX[j] = v[3 + j] - v[2 + j];  // RX[j] = R^x(j-1)
    T SXh[5];
#pragma unroll
    for (int m = 0; m < 4; ++m) SXh[m] = half_limited<LIM>(RX[m + 1], RX[m + 1 - SX]);
    SXh[4] = shfl_dn1(SXh[0]);                         // column 4 = next group's column 0
#pragma unroll
    for (int i = 0; i < 4; ++i) An[i] = SXh[i + 1] - SXh[i];
  }

  // output row a
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int mo = i - B5;       // own column in C5
    const int mu = i - SX - B5;  // x-upwind column in C5
    T u1 = c.c00 * s.F0[mo] + c.c10 * s.F0[mu] + c.c01 * s.F1[mo] + c.c11 * s.F1[mu];
    if constexpr (ORDER == 2) {
      const int iu = i - SX;     // x-upwind column among the own four (or the neighbour's)
      const T bu = (iu >= 0 && iu < 4) ? Bv[iu >= 0 && iu < 4 ? iu : 0] : Bu;
      u1 -= c.a1 * s.A0[i] + c.a2 * s.A1[i];
      u1 -= c.b1 * Bv[i] + c.b2 * bu;
    }
    out[i] = u1;
  }

  // shift the row history
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    if constexpr (SY > 0) {
      s.F1[m] = s.F0[m];
      s.F0[m] = Fn[m];
    } else {
      s.F0[m] = s.F1[m];
      s.F1[m] = Fn[m];
    }
  }
  if constexpr (ORDER == 2) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if constexpr (SY > 0) {
        s.A1[i] = s.A0[i];
        s.A0[i] = An[i];
      } else {
        s.A0[i] = s.A1[i];
        s.A1[i] = An[i];
      }
    }
  }
}

#include "step_kernel_body.cuh"

}  // namespace ctulbm

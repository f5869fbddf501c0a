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
// [56 s, 56 s + 56) and streams down a range of rows, 4 rows per iteration.
// Its 256 threads are (velocity k, group g of four columns) over a 64-column
// region [56 s - 4, 56 s + 60): the strip, the two columns of rho* halo the
// force stencil needs on each side, and two more that complete the groups.
// Warps hold one sign quadrant (sgn xi_x, sgn xi_y), so the upwind side of
// every stencil is a compile-time constant inside a warp.  Iteration i takes
// the staged rows n = B_i .. B_i + 3 of f^n (one tensor copy of 68 columns x
// 16 planes x 4 rows into one of two staging slots, issued by a producer
// thread whose warp has no collision work at the end of the previous
// iteration's advection) and
//   P1  advects them (every quadrant emits the rows n - 2, two rows behind
//       the staged one) into a six-row ring of advected rows f*;
//   P2  one thread per node: rho* - rho_ref, u*, p^i - p^w of those rows;
//   P4  224 threads, one per output node, two rows further back (warp w:
//       columns 8w .. 8w+7 of the four rows): the 5x5 force stencils -> g
//       (the Laplacian composed into the gradient of kappa lap rho), f^eq +
//       dt F_k, relaxation of all 16 planes into a plane-major output tile in
//       the staging slot P1 has consumed, which one thread writes to f^{n+1}
//       with a tensor store at the start of the next iteration.
// Three CTA barriers per four rows; three CTAs per SM; every shared-memory
// offset inside an iteration is a compile-time constant from a per-thread
// base.  f^n is read from HBM once per step (the halo columns of
// neighbouring strips are L2 hits) and f^{n+1} written once.
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
constexpr int RPI = 4;          // rows per pipeline iteration (one staged batch)
// Staging columns per plane row: the region plus the advection halo.  A thread
// of column group g reads staging columns 4g + 2 .. 4g + 8 (s_x > 0 uses
// 4g + 2 .. 4g + 7); column 68 is needed only by the last group of s_x < 0,
// whose results there (region columns 62, 63) feed no output.  68 columns
// are whole 16-byte chunks for float and double; half rows need 72.
template <typename ST>
constexpr int scol_of() {
  return sizeof(ST) == 2 ? 72 : 68;
}
constexpr int NSLOT = 2;        // staging ring: the batch being read, the next being loaded
static_assert(TW <= 68, "an output tile [16][RPI][TW] fits in a staging slot");
constexpr int PRODUCER = NT - 32;  // the thread that issues tensor copies and stores (warp 7,
                                   // which has no node in the collision phase)
constexpr int FROWS = 6;        // advected-row ring f*: rows B - 4 .. B + 1 of an iteration
constexpr int MROWS = 8;        // moment rings (power of two)
constexpr int P4T = RPI * TW;   // collision threads: one per output node of an iteration
// Padded pitches: the collision's warps read 4 rows x 8 columns of the rings;
// row strides of 8 mod 32 words put the four rows on distinct banks.
constexpr int MP = REG + 8;           // moment rings: words per row
constexpr int FRS = 16 * REG + 8;     // advected-row ring: words per row (16 planes of REG)
constexpr int WARM = 2;         // iterations of a segment before its first output row

// Per-velocity constants, computed on the host in FP64 and rounded to T.
template <typename T>
struct VelConst {
  T xi_x, xi_y, w;
  T cx, cy;                 // Courant numbers |xi_x| dt/ds, |xi_y| dt/ds
  T ax;                     // lam |xi_x| (1 - cx): weight of the x-difference of half-limited S^x
  T by0, by1;               // -lam |xi_y| (1 - cy) (1 - cx), -lam |xi_y| (1 - cy) cx (S^y terms)
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
  T rho_ref, Tt, a, b, omega, one_m_omega, om2, om6;
  // force stencils with dt/ds (and kappa) folded in: g dt/ds = ir * (gradient
  // of p^i - p^w) + kappa * (gradient of the Laplacian)
  T gw1, gw2, gw3, gw4;     // (4/9, 1/9, 1/18, 1/72) dt/ds
  // kappa D_h(9-point Laplacian) composed into one 5x5 stencil: weights of
  // q(+-1, b) - q(-+1, b) for |b| = 0, 1, 2 and of q(+-2, b) - q(-+2, b),
  // (-1, -1/18, 1/18, 1/4, 1/9, 1/72) kappa dt/ds^3
  T kw[6];
  T rho_ext, rbc2, cxc, cyc;
  unsigned int* err;         // bit 0: non-finite or non-positive rho; bit 1: a wait timed out
  int tma_in;               // the tensor maps describe fin (interior strips stage by tensor copies)
  int tma_out;              // the store maps describe fout (tiles leave by tensor stores)
  T xlo, xhi;               // |xi| components sqrt(3 - sqrt 6), sqrt(3 + sqrt 6)
  ClassConst<T> cls[4];     // groups (lo,lo), (hi,lo), (lo,hi), (hi,hi)
  VelConst<T> v[16];
};

// f^n as a 3-D tensor (x, plane, row): m[0] loads boxes of scol_of<ST>()
// columns x 16 planes x RPI rows of fin, m[1] single rows; f^{n+1} as (x, row, plane):
// m[2] stores tiles of TW columns x RPI rows x 16 planes into fout.
struct RowMaps {
  CUtensorMap m[3];
};

constexpr int MAXB = 12;  // lattices per batched launch (kernel parameter space)

template <typename T>
struct BatchArgs {
  int count;
  unsigned long long* sched;       // [2] work counter and done counter
  long long item_start[MAXB + 1];  // prefix sums of the lattices' work items
  StepArgs<T> L[MAXB];
  RowMaps maps[MAXB];
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
__device__ __forceinline__ double flip_sign(double v, double s) {
  return __longlong_as_double(__double_as_longlong(v) ^
                              (__double_as_longlong(s) & (long long)0x8000000000000000ULL));
}

// Reciprocal in FP32: the hardware approximation (relative error below 2^-22),
// enough for u = (rho u)/rho and the pressure and force terms, which enter the
// update multiplied by dt; FP64 keeps the correctly rounded division.
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// min(|a|, |b|) carrying the sign sgn(a) sgn(b) (one instruction on sm_86+).
__device__ __forceinline__ float min_xorsign_abs(float a, float b) {
  float r;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Half of the limited jump R Psi(Ru / R) of Sec. II C 2 (Ru the upwind jump).
// For the MC limiter Psi = max(0, min((1 + th)/2, 2, 2 th)) this is the
// three-way minmod of R, Ru and (R + Ru)/4: the one of least magnitude when
// all three share a sign, else 0 -- no division, and 0 at R = 0 where the
// limiter's argument is undefined.  FP32: u = minmod(R, Ru) as sgn(R) sgn(Ru)
// min(|R|, |Ru|) clamped at 0, then min(u, |h|) with the sign of h = (R + Ru)/4,
// which is sgn(R) whenever u > 0.
template <int LIM>
__device__ __forceinline__ float half_limited(float R, float Ru) {
  if constexpr (LIM == 1) {
    return 0.0f;
  } else if constexpr (LIM == 2) {
    return 0.5f * R;
  } else {
    const float h = 0.25f * (R + Ru);
    const float u = fmaxf(min_xorsign_abs(R, Ru), 0.0f);
    return min_xorsign_abs(u, h);
  }
}
template <int LIM>
__device__ __forceinline__ double half_limited(double R, double Ru) {
  if constexpr (LIM == 1) {
    return 0.0;
  } else if constexpr (LIM == 2) {
    return 0.5 * R;
  } else {
    const double a = fabs(R);
    const double b = flip_sign(Ru, R);  // sgn(R) Ru
    double m = fmin(fmin(0.25 * (a + b), a), b);
    m = fmax(m, 0.0);
    return copysign(m, R);
  }
}

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// n consecutive staged values from shared memory (16-byte aligned start for
// n = 4, 8-byte for n = 2; half: 8- and 4-byte), converted to T.
template <typename S, typename T, int N>
__device__ __forceinline__ void sload(const S* p, T* v) {
  if constexpr (sizeof(S) == 4) {
    if constexpr (N == 4) {
      const float4 t = *reinterpret_cast<const float4*>(p);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (N == 2) {
      const float2 t = *reinterpret_cast<const float2*>(p);
      v[0] = t.x; v[1] = t.y;
    } else {
      v[0] = *p;
    }
  } else if constexpr (sizeof(S) == 8) {
#pragma unroll
    for (int m = 0; m < N / 2; ++m) {
      const double2 t = reinterpret_cast<const double2*>(p)[m];
      v[2 * m] = t.x; v[2 * m + 1] = t.y;
    }
    if constexpr (N & 1) v[N - 1] = p[N - 1];
  } else {
    if constexpr (N == 4) {
      const uint2 u = *reinterpret_cast<const uint2*>(p);
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else if constexpr (N == 2) {
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(p));
      v[0] = a.x; v[1] = a.y;
    } else {
      v[0] = __half2float(*p);
    }
  }
}

// ------------------------------------------------------ advection state
// A thread advects four columns of one plane.  Row history, for its own
// columns: f and R^y of the last staged row, the last S^y, and Z of the last
// two rows, Z = f - c_x (f - f_upwind) - ax dS^x the x part of the update
// (CTU1's x-weights and the limited x correction in one number per node).
// Output row j = Z(j) + c_y (Z(j - s_y) - Z(j)) + by0 dS^y(i) + by1 dS^y(i - s_x),
// with dS^x = S^x(i+1) - S^x(i), dS^y = S^y(j+1) - S^y(j) (Sec. II C 2,
// collected per node).  A value a stencil needs one column beyond the group
// is the neighbouring group's, taken from the adjacent lane (a velocity's 16
// groups sit on 16 consecutive lanes).  At the two region edges that lane
// holds nothing useful; those columns (region 0 and 63) feed only rho*
// outside the stencils of the strip's outputs.
template <typename T>
struct AdvState {
  T Fp[4];   // f(n - 1)
  T Ryp[4];  // R^y(n - 1)
  T Syp[4];  // s_y > 0: S^y(n - 1);  s_y < 0: S^y(n - 2)
  T Z1[4];   // Z(n - 1)
  T Z2[4];   // Z(n - 2)
  T pend[4]; // s_y > 0: output row n - 2, computed one staged row earlier
};

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// One staged row n of velocity k in quadrant (SX, SY): `srow` points at the
// thread's group start (own column 0) in the staged row, `out` receives the
// advected row n - 2 (four values).  All 32 lanes of the warp must call it
// together (it exchanges neighbour columns).
template <int SX, int SY, int ORDER, int LIM, typename T, typename ST>
__device__ __forceinline__ void advect_row(AdvState<T>& s, const ST* srow, const VelConst<T>& c,
                                           T* out) {
  // f of the staged row at columns -2..3 (SX > 0) or -1..4 (SX < 0): F[m] is
  // column m - 2 resp. m - 1
  T F[6];
  if constexpr (SX > 0) {
    sload<ST, T, 2>(srow - 2, F);
    sload<ST, T, 4>(srow, F + 2);
  } else {
    sload<ST, T, 1>(srow - 1, F);
    sload<ST, T, 4>(srow, F + 1);
    sload<ST, T, 1>(srow + 4, F + 5);
  }
  constexpr int O = SX > 0 ? 2 : 1;  // index of own column 0 in F

  // x direction: R^x(i) = f(i) - f(i-1), S^x(i) = half-limited R^x(i) with the
  // upwind jump R^x(i - s_x); Z = f(i) - c_x (f(i) - f(i - s_x)) - ax dS^x(i)
  T Z[4];
  if constexpr (ORDER == 2) {
    T R[5];  // SX > 0: R^x(-1..3);  SX < 0: R^x(0..4)
#pragma unroll
    for (int m = 0; m < 5; ++m) R[m] = F[m + 1] - F[m];
    T S[5];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if constexpr (SX > 0)
        S[i] = half_limited<LIM>(R[i + 1], R[i]);
      else
        S[i] = half_limited<LIM>(R[i], R[i + 1]);
    }
    S[4] = shfl_dn1(S[0]);  // S^x(4): the next group's column 0
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T dS = S[i + 1] - S[i];
      // f(i) - f(i - s_x) = s_x R^x(i) for s_x > 0, -R^x(i+1) for s_x < 0
      const T X = SX > 0 ? fma(-c.cx, R[i + 1], F[O + i]) : fma(c.cx, R[i + 1], F[O + i]);
      Z[i] = fma(-c.ax, dS, X);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T Rx = SX > 0 ? F[O + i] - F[O + i - 1] : F[O + i + 1] - F[O + i];
      Z[i] = SX > 0 ? fma(-c.cx, Rx, F[O + i]) : fma(c.cx, Rx, F[O + i]);
    }
  }

  // y direction and the output row
  T o[4];
  if constexpr (ORDER == 2) {
    T Ry[4], Sy[4], dSy[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Ry[i] = F[O + i] - s.Fp[i];  // R^y(n)
      if constexpr (SY > 0) {
        Sy[i] = half_limited<LIM>(Ry[i], s.Ryp[i]);  // S^y(n), upwind R^y(n - 1)
      } else {
        Sy[i] = half_limited<LIM>(s.Ryp[i], Ry[i]);  // S^y(n - 1), upwind R^y(n)
      }
      dSy[i] = Sy[i] - s.Syp[i];  // SY > 0: dS^y(n - 1);  SY < 0: dS^y(n - 2)
    }
    // dS^y one column upwind in x: the neighbouring group's edge column
    const T du = SX > 0 ? shfl_up1(dSy[3]) : shfl_dn1(dSy[0]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T dsu = SX > 0 ? (i > 0 ? dSy[i - 1] : du) : (i < 3 ? dSy[i + 1] : du);
      // SY > 0: output row n - 1 from Z(n - 1), Z(n - 2); SY < 0: row n - 2
      // from Z(n - 2), Z(n - 1)
      const T Zi = SY > 0 ? s.Z1[i] : s.Z2[i];
      const T Zu = SY > 0 ? s.Z2[i] : s.Z1[i];
      T v = fma(c.cy, Zu - Zi, Zi);
      v = fma(c.by0, dSy[i], v);
      o[i] = fma(c.by1, dsu, v);
      s.Ryp[i] = Ry[i];
      s.Syp[i] = Sy[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T Zi = SY > 0 ? s.Z1[i] : s.Z2[i];
      const T Zu = SY > 0 ? s.Z2[i] : s.Z1[i];
      o[i] = fma(c.cy, Zu - Zi, Zi);
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if constexpr (SY > 0) {
      out[i] = s.pend[i];
      s.pend[i] = o[i];
    } else {
      out[i] = o[i];
    }
    s.Fp[i] = F[O + i];
    s.Z2[i] = s.Z1[i];
    s.Z1[i] = Z[i];
  }
}

// ------------------------------------------- packed FP32 advection (FP32 and FP16 storage)
// The same row update on column pairs (0, 1) and (2, 3) held as float2: every
// operation whose operands are whole pairs runs as one packed FP32x2
// instruction (sm_100+), which issues once for two lanes' worth of work; the
// jumps R^x (pairs shifted by one column), the limiters (min/max have no
// packed form) and the neighbour-shifted terms stay scalar.  Numerically each
// component is the scalar operation (round to nearest), except h^x, taken as
// (f(i) - f(i-2))/4 for s_x > 0 (the same quantity as (R^x(i) + R^x(i-1))/4).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
        "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
// the same pair operations on FP64 pairs, component by component
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 dup2(double v) { return make_double2(v, v); }
template <typename T>
struct PairOf {
  using type = float2;
  static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <>
struct PairOf<double> {
  using type = double2;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

// the MC half-limited jump with h = (R + Ru)/4 given (see half_limited)
template <int LIM>
__device__ __forceinline__ float mc_half(float R, float Ru, float h) {
  if constexpr (LIM == 1) {
    return 0.0f;
  } else if constexpr (LIM == 2) {
    return 0.5f * R;
  } else {
    return min_xorsign_abs(fmaxf(min_xorsign_abs(R, Ru), 0.0f), h);
  }
}

struct AdvState2 {
  float2 Fp[2], Ryp[2], Syp[2], Z1[2], Z2[2], pend[2];  // as AdvState, column pairs
};

// per-thread constant pairs of the packed row update
struct VelPairs {
  float2 ncx, nax, cy, by0, q;  // (-/+)c_x (sign of -s_x), -ax, c_y, by0, 1/4
  float by1;
};
template <int SX>
__device__ __forceinline__ VelPairs vel_pairs(const VelConst<float>& c) {
  VelPairs v;
  v.ncx = dup2(SX > 0 ? -c.cx : c.cx);
  v.nax = dup2(-c.ax);
  v.cy = dup2(c.cy);
  v.by0 = dup2(c.by0);
  v.q = dup2(0.25f);
  v.by1 = c.by1;
  return v;
}

template <typename ST>
__device__ __forceinline__ float2 sload2(const ST* p) {
  if constexpr (sizeof(ST) == 4) return *reinterpret_cast<const float2*>(p);
  else return __half22float2(*reinterpret_cast<const __half2*>(p));
}
template <typename ST>
__device__ __forceinline__ void sload4p(const ST* p, float2& a, float2& b) {
  if constexpr (sizeof(ST) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
  } else {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  }
}

template <int SX, int SY, int ORDER, int LIM, typename ST>
__device__ __forceinline__ void advect_row2(AdvState2& s, const ST* srow, const VelPairs& c,
                                            float* out) {
  float2 B0, B1;  // columns (0, 1), (2, 3)
  sload4p<ST>(srow, B0, B1);
  float2 Z[2];
  if constexpr (SX > 0) {
    const float2 A = sload2<ST>(srow - 2);  // columns (-2, -1)
    const float R_1 = A.y - A.x, R0 = B0.x - A.y, R1 = B0.y - B0.x;
    const float R2 = B1.x - B0.y, R3 = B1.y - B1.x;
    const float2 X01 = fma2(c.ncx, make_float2(R0, R1), B0);
    const float2 X23 = fma2(c.ncx, make_float2(R2, R3), B1);
    if constexpr (ORDER == 2) {
      const float2 h01 = mul2(c.q, sub2(B0, A)), h23 = mul2(c.q, sub2(B1, B0));
      const float S0 = mc_half<LIM>(R0, R_1, h01.x), S1 = mc_half<LIM>(R1, R0, h01.y);
      const float S2 = mc_half<LIM>(R2, R1, h23.x), S3 = mc_half<LIM>(R3, R2, h23.y);
      const float S4 = shfl_dn1(S0);
      Z[0] = fma2(c.nax, make_float2(S1 - S0, S2 - S1), X01);
      Z[1] = fma2(c.nax, make_float2(S3 - S2, S4 - S3), X23);
    } else {
      Z[0] = X01;
      Z[1] = X23;
    }
  } else {
    const float a = from_store<ST, float>(srow[-1]), e = from_store<ST, float>(srow[4]);
    const float R0 = B0.x - a, R1 = B0.y - B0.x, R2 = B1.x - B0.y;
    const float R3 = B1.y - B1.x, R4 = e - B1.y;
    const float2 X01 = fma2(c.ncx, make_float2(R1, R2), B0);
    const float2 X23 = fma2(c.ncx, make_float2(R3, R4), B1);
    if constexpr (ORDER == 2) {
      const float S0 = mc_half<LIM>(R0, R1, 0.25f * (R0 + R1));
      const float S1 = mc_half<LIM>(R1, R2, 0.25f * (R1 + R2));
      const float S2 = mc_half<LIM>(R2, R3, 0.25f * (R2 + R3));
      const float S3 = mc_half<LIM>(R3, R4, 0.25f * (R3 + R4));
      const float S4 = shfl_dn1(S0);
      Z[0] = fma2(c.nax, make_float2(S1 - S0, S2 - S1), X01);
      Z[1] = fma2(c.nax, make_float2(S3 - S2, S4 - S3), X23);
    } else {
      Z[0] = X01;
      Z[1] = X23;
    }
  }

  float2 o[2];
  const float2 Bn[2] = {B0, B1};
  if constexpr (ORDER == 2) {
    float2 Ry[2], Sy[2], dSy[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      Ry[m] = sub2(Bn[m], s.Fp[m]);
      const float2 hy = mul2(c.q, add2(Ry[m], s.Ryp[m]));
      if constexpr (SY > 0)
        Sy[m] = make_float2(mc_half<LIM>(Ry[m].x, s.Ryp[m].x, hy.x),
                            mc_half<LIM>(Ry[m].y, s.Ryp[m].y, hy.y));
      else
        Sy[m] = make_float2(mc_half<LIM>(s.Ryp[m].x, Ry[m].x, hy.x),
                            mc_half<LIM>(s.Ryp[m].y, Ry[m].y, hy.y));
      dSy[m] = sub2(Sy[m], s.Syp[m]);
    }
    // dS^y one column upwind in x
    float2 dsu[2];
    if constexpr (SX > 0) {
      const float du = shfl_up1(dSy[1].y);
      dsu[0] = make_float2(du, dSy[0].x);
      dsu[1] = make_float2(dSy[0].y, dSy[1].x);
    } else {
      const float du = shfl_dn1(dSy[0].x);
      dsu[0] = make_float2(dSy[0].y, dSy[1].x);
      dsu[1] = make_float2(dSy[1].y, du);
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const float2 Zi = SY > 0 ? s.Z1[m] : s.Z2[m];
      const float2 Zu = SY > 0 ? s.Z2[m] : s.Z1[m];
      float2 v = fma2(c.cy, sub2(Zu, Zi), Zi);
      v = fma2(c.by0, dSy[m], v);
      o[m] = make_float2(fmaf(c.by1, dsu[m].x, v.x), fmaf(c.by1, dsu[m].y, v.y));
      s.Ryp[m] = Ry[m];
      s.Syp[m] = Sy[m];
    }
  } else {
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const float2 Zi = SY > 0 ? s.Z1[m] : s.Z2[m];
      const float2 Zu = SY > 0 ? s.Z2[m] : s.Z1[m];
      o[m] = fma2(c.cy, sub2(Zu, Zi), Zi);
    }
  }

#pragma unroll
  for (int m = 0; m < 2; ++m) {
    if constexpr (SY > 0) {
      out[2 * m] = s.pend[m].x;
      out[2 * m + 1] = s.pend[m].y;
      s.pend[m] = o[m];
    } else {
      out[2 * m] = o[m].x;
      out[2 * m + 1] = o[m].y;
    }
    s.Fp[m] = Bn[m];
    s.Z2[m] = s.Z1[m];
    s.Z1[m] = Z[m];
  }
}

// the advection state of the arithmetic type: FP32 packs column pairs
template <typename T>
struct AdvSel {
  using State = AdvState<T>;
};
template <>
struct AdvSel<float> {
  using State = AdvState2;
};

#include "step_kernel_body.cuh"

}  // namespace ctulbm

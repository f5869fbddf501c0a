// lbm_kernels.cuh -- device code of the CTU lattice Boltzmann time step for
// GB300 (sm_103a), after arXiv:1802.01272 (Sofonea et al.).
//
// One step, as Sec. II C splits Eq. (eBGK): advection of each f_k over its
// upwind-corner stencil (CTU1, Eq. ctueq; CTU2 with the MC limiter,
// Sec. II C 2), then on the advected f*: rho, u, g (Eq. eder with Eq. evdw,
// isotropic 25-point stencil), f^eq (Eq. herfeq), F_k (Eq. herforce), BGK
// relaxation (optionally regularised, Eq. ereg), and the density reservoir of
// Sec. III A.
//
// Kernel layout (step_kernel): a CTA owns a strip of TW = 60 output columns
// and streams down a range of rows.  Its 256 threads are (velocity k, group g
// of four columns) over a 64-column region = the strip plus a two-column halo
// on each side (rho* is needed there for the force stencil).  Warps hold one
// sign quadrant (sgn xi_x, sgn xi_y), so the upwind side of every stencil is a
// compile-time constant inside a warp.  For each row a the CTA
//   P1  advects row a of every plane (the CTU2 jumps, limited corrections and
//       their differences of the previous rows live in registers) into a ring
//       of advected rows in shared memory;
//   P2  sums the 16 planes of row a: rho*, u*, p^i - p^w;
//   P3  takes the 9-point Laplacian of rho* on row a-1 and, on row c = a-3,
//       the isotropic gradients -> g, and per-node collision coefficients;
//   P4  relaxes row c of every plane and stores it (coalesced 16-byte stores).
// Global memory is read once per step for f^n (halo re-reads hit L1/L2) and
// written once for f^{n+1}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ctulbm {

constexpr int NG = 16;          // four-column groups in a strip region
constexpr int REG = 4 * NG;     // region columns: output strip plus 2 halo columns per side
constexpr int TW = REG - 4;     // output columns per strip
constexpr int NT = 16 * NG;     // threads per CTA
constexpr int FR = 5;           // rows of advected f kept in shared memory
constexpr int SREG = REG + 8;   // padded plane row: 16-byte aligned, and the four
                                // plane-interleaved moment partial sums hit distinct banks
constexpr int MR = 5;           // rows of rho*, u*, phi, lap kept
constexpr int NODE_W = 9;       // per-node collision words
constexpr int REG_W = 7;        // per-node non-equilibrium moments (regularisation)
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

template <typename T>
struct StepArgs {
  const T* fin;
  T* fout;
  int Lx, Ly;
  long long plane;          // Lx * Ly
  int nstrip;
  long long rows_total;     // nstrip * Ly
  long long rows_per_cta;
  int walls, reservoir, regularize;
  T rho_ref, Tt, a, b, kappa, inv_ds, inv_ds2, dt, omega, one_m_omega, om2, om6;
  T rho_ext, rbc2, cxc, cyc;
  unsigned int* err;
  VelConst<T> v[16];
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float flip_sign(float v, float s) {
  return __int_as_float(__float_as_int(v) ^ (__float_as_int(s) & 0x80000000));
}
__device__ __forceinline__ double flip_sign(double v, double s) {
  return __longlong_as_double(__double_as_longlong(v) ^
                              (__double_as_longlong(s) & (long long)0x8000000000000000ULL));
}

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
    T m = fmin(fmin(T(0.25) * (a + b), a), b);
    m = fmax(m, T(0));
    return copysign(m, R);
  }
}

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

template <typename T>
__device__ __forceinline__ void load4(const T* p, T* v);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float* v) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* p, double* v) {
  double2 t0 = __ldg(reinterpret_cast<const double2*>(p));
  double2 t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}
template <typename T>
__device__ __forceinline__ void store4(T* p, const T* v);
template <>
__device__ __forceinline__ void store4<float>(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4<double>(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
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

// ------------------------------------------------------ advection state
// Columns: the thread owns group columns 0..3.  CTU keeps five columns C5 =
// {own, own - sgn_x}: for sgn_x > 0 relative columns -1..3, else 0..4.
template <typename T>
struct AdvState {
  T F0[5], F1[5];  // f on row a and on the y-upwind row a - sgn_y
  T RY[5];         // sgn_y > 0: R^y(a);  sgn_y < 0: R^y(a+1)
  T SY[5];         // half-limited S^y(a)
  T A0[4], A1[4];  // x-differences of half-limited S^x on row a and on row a - sgn_y
};

// One advection row for velocity k of quadrant (SX, SY).  `v` holds the newly
// loaded row (a+1 if SY > 0, a+2 if SY < 0) at relative columns -4..7.
template <int SX, int SY, int ORDER, int LIM, typename T>
__device__ __forceinline__ void advect_row(AdvState<T>& s, const T* v, const VelConst<T>& c,
                                           T* out) {
  constexpr int B5 = SX > 0 ? -1 : 0;  // relative column of C5[0]
  T Fn[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) Fn[m] = v[4 + B5 + m];

  T Bv[5], An[4];
  if constexpr (ORDER == 2) {
    T RYn[5], SYn[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      if constexpr (SY > 0) {
        RYn[m] = Fn[m] - s.F0[m];                     // R^y(a+1)
        SYn[m] = half_limited<LIM>(RYn[m], s.RY[m]);  // S^y(a+1), upwind R^y(a)
      } else {
        RYn[m] = Fn[m] - s.F1[m];                     // R^y(a+2)
        SYn[m] = half_limited<LIM>(s.RY[m], RYn[m]);  // S^y(a+1), upwind R^y(a+2)
      }
      Bv[m] = SYn[m] - s.SY[m];                       // S^y(a+1) - S^y(a)
      s.RY[m] = RYn[m];
      s.SY[m] = SYn[m];
    }
    // x direction on the new row: R^x(c) = f(c) - f(c-1) for c in -1..5
    T RX[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) RX[j] = v[3 + j] - v[2 + j];  // RX[j] = R^x(j-1)
    T SXh[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) SXh[m] = half_limited<LIM>(RX[m + 1], RX[m + 1 - SX]);
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
      u1 -= c.a1 * s.A0[i] + c.a2 * s.A1[i];
      u1 -= c.b1 * Bv[mo] + c.b2 * Bv[mu];
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

// ---------------------------------------------------------------- kernel
template <typename T, int ORDER, int LIM, bool VEC>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    step_kernel(const __grid_constant__ StepArgs<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_fs = reinterpret_cast<T*>(smem_raw);   // [FR][16][SREG] advected f*
  T* s_rho = s_fs + FR * 16 * SREG;           // [MR][REG]
  T* s_drho = s_rho + MR * REG;
  T* s_ux = s_drho + MR * REG;
  T* s_uy = s_ux + MR * REG;
  T* s_phi = s_uy + MR * REG;
  T* s_lap = s_phi + MR * REG;
  T* s_node = s_lap + MR * REG;               // [NODE_W][REG] for row c
  T* s_reg = s_node + NODE_W * REG;           // [REG_W][REG] for row c

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;                          // sign quadrant of the warp
  const int g = ((warp >> 2) << 3) | (lane & 7);   // column group 0..15
  const int k = ((lane >> 3) << 2) | q;            // velocity
  const VelConst<T> vc = P.v[k];
  const int Lx = P.Lx, Ly = P.Ly;
  const int lag = (q == 0 || q == 1) ? 1 : 2;      // sgn_y > 0 for quadrants 0, 1
  const T* fin_k = P.fin + (long long)k * P.plane;
  T xip[4], yip[4];                                // velocities summed by this thread in P2
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    xip[j] = P.v[(tid & 3) + 4 * j].xi_x;
    yip[j] = P.v[(tid & 3) + 4 * j].xi_y;
  }
  T* fout_k = P.fout + (long long)k * P.plane;

  long long r0 = (long long)blockIdx.x * P.rows_per_cta;
  const long long r1 = min(r0 + P.rows_per_cta, P.rows_total);

  while (r0 < r1) {
    const int strip = (int)(r0 / Ly);
    const int ys = (int)(r0 % Ly);
    const int ye = (int)min((long long)Ly, (long long)ys + (r1 - r0));
    r0 += ye - ys;

    const int gx0 = strip * TW + 4 * g;   // first global column (unwrapped) of this group
    const int x0 = strip * TW + 2;        // first output column of the strip (unwrapped)
    int colL = 0, colC = 0, colR = 0;
    if (VEC) {
      colL = wrapi(gx0 - 4, Lx);
      colC = wrapi(gx0, Lx);
      colR = wrapi(gx0 + 4, Lx);
    }

    AdvState<T> st;
#pragma unroll
    for (int m = 0; m < 5; ++m) st.F0[m] = st.F1[m] = st.RY[m] = st.SY[m] = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) st.A0[i] = st.A1[i] = T(0);

    for (int a = ys - WARMUP; a <= ye + 2; ++a) {
      // ---------------- P1: advect row a of plane k
      {
        T v[12];
        const int rl = a + lag;
        if (P.walls && (rl < 0 || rl >= Ly)) {
          const T gv = rl < 0 ? vc.gbot : vc.gtop;
#pragma unroll
          for (int j = 0; j < 12; ++j) v[j] = gv;
        } else {
          const T* row = fin_k + (long long)wrapi(rl, Ly) * Lx;
          if (VEC) {
            load4<T>(row + colL, v);
            load4<T>(row + colC, v + 4);
            load4<T>(row + colR, v + 8);
          } else {
#pragma unroll
            for (int j = 0; j < 12; ++j) v[j] = __ldg(row + wrapi(gx0 - 4 + j, Lx));
          }
        }
        T out[4];
        switch (q) {
          case 0: advect_row<+1, +1, ORDER, LIM>(st, v, vc, out); break;
          case 1: advect_row<-1, +1, ORDER, LIM>(st, v, vc, out); break;
          case 2: advect_row<-1, -1, ORDER, LIM>(st, v, vc, out); break;
          default: advect_row<+1, -1, ORDER, LIM>(st, v, vc, out); break;
        }
        if (P.walls && (a < 0 || a >= Ly)) {  // ghost rows keep f^eq(rho_ext, u_wall)
          const T gv = a < 0 ? vc.gbot : vc.gtop;
#pragma unroll
          for (int i = 0; i < 4; ++i) out[i] = gv;
        }
        T* dst = s_fs + ((a + 10) % FR) * 16 * SREG + k * SREG + 4 * g;
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(dst) = make_float4(out[0], out[1], out[2], out[3]);
        } else {
          reinterpret_cast<double2*>(dst)[0] = make_double2(out[0], out[1]);
          reinterpret_cast<double2*>(dst)[1] = make_double2(out[2], out[3]);
        }
      }
      __syncthreads();

      // ---------------- P2: moments of row a over the region
      {
        const int col = tid >> 2, part = tid & 3;   // part sums planes part, part+4, part+8, part+12
        const T* src = s_fs + ((a + 10) % FR) * 16 * SREG + col;
        T d = 0, mx = 0, my = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T fv = src[(part + 4 * j) * SREG];
          d += fv;
          mx += fv * xip[j];
          my += fv * yip[j];
        }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
          d += __shfl_xor_sync(0xffffffffu, d, o);
          mx += __shfl_xor_sync(0xffffffffu, mx, o);
          my += __shfl_xor_sync(0xffffffffu, my, o);
        }
        if (part == 0) {
          const int sl = ((a + 10) % MR) * REG + col;
          const T rho = P.rho_ref + d;
          const T ir = T(1) / rho;
          s_rho[sl] = rho;
          s_drho[sl] = d;
          s_ux[sl] = mx * ir;
          s_uy[sl] = my * ir;
          // p^i - p^w = rho T - [rho T/(1 - b rho) - a rho^2]   (Eqs. eder, evdw)
          s_phi[sl] = rho * P.Tt - (rho * P.Tt / (T(1) - P.b * rho) - P.a * rho * rho);
        }
      }
      __syncthreads();

      // ---------------- P3: Laplacian on row a-1; g and collision coefficients on row c = a-3
      const int c = a - 3;
      if (tid < REG - 2) {
        const int col = tid + 1, r = a - 1;
        const T* R0 = s_rho + ((r + 10) % MR) * REG + col;
        const T* Rm = s_rho + ((r + 9) % MR) * REG + col;
        const T* Rp = s_rho + ((r + 11) % MR) * REG + col;
        const T nn = R0[-1] + R0[1] + Rm[0] + Rp[0];
        const T dg = Rm[-1] + Rm[1] + Rp[-1] + Rp[1];
        s_lap[((r + 10) % MR) * REG + col] =
            (T(2) / T(3) * nn + dg / T(6) - T(10) / T(3) * R0[0]) * P.inv_ds2;
      } else if (tid >= 64 && tid < 64 + TW && c >= ys && c < ye) {
        const int col = tid - 64 + 2;
        const int sc = ((c + 10) % MR) * REG + col;
        const int sm = ((c + 9) % MR) * REG + col;
        const int sp = ((c + 11) % MR) * REG + col;
        // isotropic gradient: [ (q(+1,0)-q(-1,0))/3 + (diagonal differences)/12 ] / ds
        const T px = ((s_phi[sc + 1] - s_phi[sc - 1]) / T(3) +
                      (s_phi[sp + 1] - s_phi[sp - 1] + s_phi[sm + 1] - s_phi[sm - 1]) / T(12));
        const T py = ((s_phi[sp] - s_phi[sm]) / T(3) +
                      (s_phi[sp + 1] - s_phi[sm + 1] + s_phi[sp - 1] - s_phi[sm - 1]) / T(12));
        const T lx = ((s_lap[sc + 1] - s_lap[sc - 1]) / T(3) +
                      (s_lap[sp + 1] - s_lap[sp - 1] + s_lap[sm + 1] - s_lap[sm - 1]) / T(12));
        const T ly = ((s_lap[sp] - s_lap[sm]) / T(3) +
                      (s_lap[sp + 1] - s_lap[sm + 1] + s_lap[sp - 1] - s_lap[sm - 1]) / T(12));
        const T rho = s_rho[sc], ux = s_ux[sc], uy = s_uy[sc];
        const T gx = (px / rho + P.kappa * lx) * P.inv_ds;
        const T gy = (py / rho + P.kappa * ly) * P.inv_ds;
        const T gdx = P.dt * gx, gdy = P.dt * gy;
        const T e = T(1) - T(0.5) * (ux * ux + uy * uy);
        const T h = gdx * ux + gdy * uy;
        s_node[0 * REG + col] = rho;
        s_node[1 * REG + col] = ux;
        s_node[2 * REG + col] = uy;
        s_node[3 * REG + col] = gdx;
        s_node[4 * REG + col] = gdy;
        s_node[5 * REG + col] = P.omega * s_drho[sc] / rho + P.omega * (e - T(1)) - h;
        s_node[6 * REG + col] = e - P.Tt + T(1);
        s_node[7 * REG + col] = P.omega * e - h;
        T scale = T(1);
        if (P.reservoir) {
          const int xg = wrapi(x0 + col - 2, Lx);
          const T dx = T(xg) - P.cxc, dy = T(c) - P.cyc;
          if (dx * dx + dy * dy > P.rbc2) scale = P.rho_ext / rho;
        }
        s_node[8 * REG + col] = scale;
        if (!(rho > T(0)) || !(rho < T(1e30))) atomicOr(P.err, 1u);
        if (P.regularize) {
          // non-equilibrium moments A2 = sum f xi xi - rho(uu + T 1),
          // A3 = sum f xi xi xi - rho(uuu + T sym(u 1)); the shift adds rho_ref to sum f xi xi
          const T* fr = s_fs + ((c + 10) % FR) * 16 * SREG + col;
          T m2xx = 0, m2xy = 0, m2yy = 0, m3xxx = 0, m3xxy = 0, m3xyy = 0, m3yyy = 0;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            const T fv = fr[kk * SREG], x = P.v[kk].xi_x, y = P.v[kk].xi_y;
            m2xx += fv * x * x;
            m2xy += fv * x * y;
            m2yy += fv * y * y;
            m3xxx += fv * x * x * x;
            m3xxy += fv * x * x * y;
            m3xyy += fv * x * y * y;
            m3yyy += fv * y * y * y;
          }
          const T Tt = P.Tt;
          s_reg[0 * REG + col] = m2xx + P.rho_ref - rho * (ux * ux + Tt);
          s_reg[1 * REG + col] = m2xy - rho * ux * uy;
          s_reg[2 * REG + col] = m2yy + P.rho_ref - rho * (uy * uy + Tt);
          s_reg[3 * REG + col] = m3xxx - rho * (ux * ux * ux + T(3) * Tt * ux);
          s_reg[4 * REG + col] = m3xxy - rho * (ux * ux * uy + Tt * uy);
          s_reg[5 * REG + col] = m3xyy - rho * (ux * uy * uy + Tt * ux);
          s_reg[6 * REG + col] = m3yyy - rho * (uy * uy * uy + T(3) * Tt * uy);
        }
      }
      __syncthreads();

      // ---------------- P4: relax row c of plane k and store it
      if (c >= ys && c < ye) {
        T fs[4];
        sload4(s_fs + ((c + 10) % FR) * 16 * SREG + k * SREG + 4 * g, fs);
        T nw[NODE_W][4];
#pragma unroll
        for (int w = 0; w < NODE_W; ++w) sload4(s_node + w * REG + 4 * g, nw[w]);
        T res[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const T rho = nw[0][m], ux = nw[1][m], uy = nw[2][m];
          const T gdx = nw[3][m], gdy = nw[4][m];
          const T cu = vc.xi_x * ux + vc.xi_y * uy;        // xi . u
          const T D = vc.xi_x * gdx + vc.xi_y * gdy;       // dt xi . g
          const T K0 = (nw[5][m] + vc.omA) + D * (nw[6][m] + vc.Ak);
          const T K1 = nw[7][m] + vc.omB + D;
          const T K2 = T(0.5) * D + P.om2;
          // (omega f^eq + dt F_k - omega w rho_ref) / (w rho), a cubic in xi.u
          const T poly = K0 + cu * (K1 + cu * (K2 + cu * P.om6));
          const T wr = vc.w * rho;
          T base = fs[m];
          if (P.regularize) {
            T rg[REG_W];
#pragma unroll
            for (int j = 0; j < REG_W; ++j) rg[j] = s_reg[j * REG + 4 * g + m];
            const T e = T(1) - T(0.5) * (ux * ux + uy * uy);
            // f^eq - w rho_ref = w [ (rho - rho_ref) + rho (P_k - 1) ]
            const T pm1 = (e - T(1) + vc.Ak) + cu * ((e + vc.Bk) + cu * (T(0.5) + cu / T(6)));
            const T feqs = vc.w * ((rho - P.rho_ref) + rho * pm1);
            const T fneq = vc.w * (vc.r2xx * rg[0] + vc.r2xy * rg[1] + vc.r2yy * rg[2] +
                                   vc.r3xxx * rg[3] + vc.r3xxy * rg[4] + vc.r3xyy * rg[5] +
                                   vc.r3yyy * rg[6]);
            base = feqs + fneq;
          }
          T fn = P.one_m_omega * base + wr * poly;
          if (P.reservoir) {
            const T s = nw[8][m];
            fn = s * fn + vc.w * P.rho_ref * (s - T(1));
          }
          res[m] = fn;
        }
        T* dst_row = fout_k + (long long)c * Lx;
        const bool full = VEC && g > 0 && g < NG - 1 && (x0 + 4 * g - 2 + 3) < Lx + 2;
        if (full) {
          store4<T>(dst_row + colC, res);
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int o = 4 * g + m - 2;               // output index in the strip
            if (o >= 0 && o < TW && x0 + o < Lx + 2) dst_row[wrapi(x0 + o, Lx)] = res[m];
          }
        }
      }
    }
  }
}

}  // namespace ctulbm

/*
 * ctu_oracle.h -- FP64 CPU oracle of the CTU lattice Boltzmann time step
 * (Sofonea et al., "Corner transport upwind lattice Boltzmann model for
 * bubble cavitation", arXiv:1802.01272).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark call this code.  It shares nothing with the
 * CUDA library: its own velocity table, its own equations, its own layout.
 *
 * Distribution layout: f[k][j][i], k = 0..15, j = 0..Ly-1 (y), i = 0..Lx-1 (x).
 */
#ifndef CTU_ORACLE_H
#define CTU_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_LIM_MC = 0, ORC_LIM_ZERO = 1, ORC_LIM_ONE = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_SHEAR_WALLS = 1 };

typedef struct orc_params {
  int32_t Lx, Ly;
  double a, b, kappa, T;      /* p^w = rho T/(1 - b rho) - a rho^2 (Eq. evdw: a = 9/8, b = 1/3) */
  double tau, dt, ds;
  int32_t ctu_order;          /* 1: Eq. ctueq, 2: flux-limited CTU2 (Sec. II C 2) */
  int32_t limiter;            /* ORC_LIM_* */
  int32_t regularize;         /* 1: Eq. ereg before every step */
  int32_t boundary;           /* ORC_BC_* */
  double shear_rate;          /* gamma_dot; u_w = gamma_dot * Ly * ds / 2 */
  double rho_ext;             /* wall ghost / reservoir density */
  int32_t reservoir;          /* 1: rescale f outside R_BC before every step */
  int32_t a2_full;            /* 0: a^(2) = rho(uu + (T-1) 1); 1: a^(2) = sum_k f_k H2(xi_k) */
} orc_params;

typedef struct orc_diag {
  double mass;                /* sum of rho over the lattice */
  double nb;                  /* number of nodes with rho < threshold */
  double sx, sy, sxx, sxy, syy; /* sums of i, j, i*i, i*j, j*j over those nodes */
  double rho_center;          /* rho at node (Lx/2, Ly/2) */
  double rho_ring;            /* mean rho over nodes at distance r_ring +- 0.5 from (Lx/2, Ly/2) */
  double rho_min, rho_max;
} orc_diag;

void orc_velocity_set(double* xi /* [16][2] */, double* w /* [16] */);
double orc_pw(const orc_params* p, double rho);
void orc_feq(const orc_params* p, double rho, double ux, double uy, double* out /*16*/);
void orc_force(const orc_params* p, double rho, double ux, double uy, double gx, double gy,
               const double* a2 /* xx, xy, yy or NULL for the equilibrium a^(2) */,
               double* out /*16*/);
void orc_init_feq(const orc_params* p, const double* rho, const double* ux, const double* uy,
                  double* f);
void orc_moments(const orc_params* p, const double* f, double* rho, double* ux, double* uy);
void orc_accel(const orc_params* p, const double* f, double* gx, double* gy);
void orc_regularize(const orc_params* p, double* f);
void orc_reservoir(const orc_params* p, double* f);
int orc_step(const orc_params* p, double* f, int64_t nsteps);
void orc_diagnostics(const orc_params* p, const double* f, double threshold, double r_ring,
                     orc_diag* out);
void orc_histogram(const orc_params* p, const double* f, int32_t nbins, double lo, double hi,
                   int64_t* counts);
double orc_limiter(int32_t limiter, double theta);

#ifdef __cplusplus
}
#endif
#endif

/*
 * ctu_oracle.c -- plain, slow FP64 CPU oracle of one time step of the
 * third-order, 16-velocity, isothermal van der Waals lattice Boltzmann model
 * advanced with the corner transport upwind schemes of arXiv:1802.01272.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the library.
 *
 * Every quantity is computed the way the paper writes it, node by node:
 *   - velocity set and weights ............ Table I
 *   - f^eq ................................ Eq. (herfeq)
 *   - force term F_k ...................... Eq. (herforce), a^(2) read as the
 *                                           equilibrium a^(2) = rho(uu + (T-1)1)
 *   - acceleration g ...................... Eq. (eder) with the vdW pressure of
 *                                           Eq. (evdw); 25-point (5x5) stencils:
 *                                           a fourth-order gradient of p^i - p^w,
 *                                           and grad(lap rho) from an isotropic
 *                                           3x3 gradient of the 9-point Laplacian
 *                                           (the paper gives no weights)
 *   - CTU1 ................................ Eq. (ctueq), four-node product form
 *   - CTU2 ................................ Sec. II C 2: jumps R, limited
 *                                           corrections S (MC limiter), fluxes F, G
 *                                           and the conservative update
 *   - regularisation ...................... Eq. (ereg)
 *   - density reservoir ................... Sec. III A (rescale outside R_BC)
 *   - sheared permeable walls ............. Sec. III C (ghost rows of f^eq)
 *   - gyration-tensor sums ................ Eq. (gyr)
 *
 * Readings where the paper is garbled or silent (all listed in the design
 * notes): S^y's limiter argument uses R^y (the printed R^x is a misprint);
 * the transverse jump in F_{i+1/2,j} sits in the upwind column
 * i + (1 - sgn_x)/2; the step is split as Sec. II C says, advection first and
 * then collision + force evaluated on the advected f (the printed CTU2 update
 * leaves the collision's f without a time level; Table II's viscosities,
 * T (tau - dt/2) plus the CTU1 numerical part, hold only for this order);
 * at R = 0 the limited correction is 0; the reservoir rescale acts on f at
 * the end of every step, before the next one starts (Sec. III A); the
 * regularisation replaces the advected f by f^eq + fhat^neq inside the
 * collision.
 *
 * Parity of the force stencil and of a^(2) against the paper itself is
 * pinned only indirectly (convergence order, isotropy, and on the GPU the
 * coexistence densities and critical radius the paper reports), since the
 * paper prints neither the stencil weights nor the label of a^(2).
 */
#include "ctu_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- Table I: the 16 velocities and weights ----------------------------
 * Cartesian components are roots of H^4: +-sqrt(3 - sqrt 6), +-sqrt(3 + sqrt 6).
 * Order inside each group of four: (+,+), (-,+), (-,-), (+,-).             */
void orc_velocity_set(double* xi, double* w) {
  const double s6 = sqrt(6.0);
  const double lo = sqrt(3.0 - s6), hi = sqrt(3.0 + s6);
  const double mag[4][2] = {{lo, lo}, {hi, lo}, {lo, hi}, {hi, hi}};
  const double wt[4] = {(5.0 + 2.0 * s6) / 48.0, 1.0 / 48.0, 1.0 / 48.0,
                        (5.0 - 2.0 * s6) / 48.0};
  const double sg[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
  for (int g = 0; g < 4; ++g)
    for (int s = 0; s < 4; ++s) {
      int k = 4 * g + s;
      xi[2 * k + 0] = sg[s][0] * mag[g][0];
      xi[2 * k + 1] = sg[s][1] * mag[g][1];
      w[k] = wt[g];
    }
}

static double XI[16][2], W[16];
static int tables_ready = 0;
/* OpenMP over rows only pays off on lattices of a few thousand nodes or more */
#define PAR(p) ((size_t)(p)->Lx * (size_t)(p)->Ly >= 16384)
static void tables(void) {
  if (!tables_ready) {
    orc_velocity_set(&XI[0][0], W);
    tables_ready = 1;
  }
}

/* ---- Eq. (evdw) with general a, b ---------------------------------------- */
double orc_pw(const orc_params* p, double rho) {
  return rho * p->T / (1.0 - p->b * rho) - p->a * rho * rho;
}

/* ---- Eq. (herfeq) --------------------------------------------------------- */
void orc_feq(const orc_params* p, double rho, double ux, double uy, double* out) {
  tables();
  const double T = p->T, u2 = ux * ux + uy * uy;
  for (int k = 0; k < 16; ++k) {
    double xu = XI[k][0] * ux + XI[k][1] * uy;
    double xi2 = XI[k][0] * XI[k][0] + XI[k][1] * XI[k][1];
    double second = 0.5 * (xu * xu - u2 + (T - 1.0) * (xi2 - 2.0));
    double third = xu / 6.0 * (xu * xu - 3.0 * u2 + 3.0 * (T - 1.0) * (xi2 - 4.0));
    out[k] = W[k] * rho * (1.0 + xu + second + third);
  }
}

/* H2_ab(xi) = xi_a xi_b - delta_ab */
static double H2(int a, int b, const double* x) { return x[a] * x[b] - (a == b ? 1.0 : 0.0); }
/* H3_abc(xi) = xi_a xi_b xi_c - xi_a d_bc - xi_b d_ac - xi_c d_ab */
static double H3(int a, int b, int c, const double* x) {
  return x[a] * x[b] * x[c] - x[a] * (b == c) - x[b] * (a == c) - x[c] * (a == b);
}

/* ---- Eq. (herforce) ------------------------------------------------------
 * F_k = w rho { xi.g + (xi.g)(xi.u) - g.u + 1/(2 rho) a2 : [(xi.g) H2(xi) - 2 g xi] } */
void orc_force(const orc_params* p, double rho, double ux, double uy, double gx, double gy,
               const double* a2in, double* out) {
  tables();
  double a2[2][2];
  if (a2in) {
    a2[0][0] = a2in[0];
    a2[0][1] = a2[1][0] = a2in[1];
    a2[1][1] = a2in[2];
  } else {
    const double u[2] = {ux, uy};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) a2[a][b] = rho * (u[a] * u[b] + (a == b ? p->T - 1.0 : 0.0));
  }
  const double g[2] = {gx, gy};
  const double gu = gx * ux + gy * uy;
  for (int k = 0; k < 16; ++k) {
    const double* x = XI[k];
    double xg = x[0] * gx + x[1] * gy;
    double xu = x[0] * ux + x[1] * uy;
    double c1 = 0.0, c2 = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        c1 += a2[a][b] * H2(a, b, x);
        c2 += a2[a][b] * g[a] * x[b];
      }
    out[k] = W[k] * rho * (xg + xg * xu - gu + (xg * c1 - 2.0 * c2) / (2.0 * rho));
  }
}

/* ---- lattice access --------------------------------------------------------
 * Periodic in x always.  In y: periodic, or the sheared permeable walls of
 * Sec. III C, whose ghost rows j in {-2,-1} and {Ly, Ly+1} hold f^eq at
 * rho_ext with velocities (-u_w, 0) and (+u_w, 0).                         */
typedef struct {
  const orc_params* p;
  const double* f;
  double ghost_bot[16], ghost_top[16];
} lattice;

static double wall_velocity(const orc_params* p) { return p->shear_rate * p->Ly * p->ds / 2.0; }

static void lattice_init(lattice* L, const orc_params* p, const double* f) {
  L->p = p;
  L->f = f;
  if (p->boundary == ORC_BC_SHEAR_WALLS) {
    double uw = wall_velocity(p);
    orc_feq(p, p->rho_ext, -uw, 0.0, L->ghost_bot);
    orc_feq(p, p->rho_ext, +uw, 0.0, L->ghost_top);
  }
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

static double fget(const lattice* L, int k, int i, int j) {
  const orc_params* p = L->p;
  i = wrap(i, p->Lx);
  if (p->boundary == ORC_BC_SHEAR_WALLS) {
    if (j < 0) return L->ghost_bot[k];
    if (j >= p->Ly) return L->ghost_top[k];
  } else {
    j = wrap(j, p->Ly);
  }
  return L->f[((size_t)k * p->Ly + j) * p->Lx + i];
}

static double rho_at(const lattice* L, int i, int j) {
  double s = 0.0;
  for (int k = 0; k < 16; ++k) s += fget(L, k, i, j);
  return s;
}

/* ---- moments (rho = sum f, rho u = sum f xi) ---------------------------- */
void orc_moments(const orc_params* p, const double* f, double* rho, double* ux, double* uy) {
  tables();
  const size_t n = (size_t)p->Lx * p->Ly;
#pragma omp parallel for schedule(static) if (PAR(p))
  for (long q = 0; q < (long)n; ++q) {
    double r = 0.0, mx = 0.0, my = 0.0;
    for (int k = 0; k < 16; ++k) {
      double v = f[(size_t)k * n + q];
      r += v;
      mx += v * XI[k][0];
      my += v * XI[k][1];
    }
    rho[q] = r;
    ux[q] = mx / r;
    uy[q] = my / r;
  }
}

void orc_init_feq(const orc_params* p, const double* rho, const double* ux, const double* uy,
                  double* f) {
  const size_t n = (size_t)p->Lx * p->Ly;
  for (size_t q = 0; q < n; ++q) {
    double fe[16];
    orc_feq(p, rho[q], ux[q], uy[q], fe);
    for (int k = 0; k < 16; ++k) f[(size_t)k * n + q] = fe[k];
  }
}

/* ---- Eq. (eder): g = grad(p^i - p^w)/rho + kappa grad(lap rho) -----------
 * Sec. II B computes both terms on 25-point stencils, chosen there because
 * large stencils make the interface more isotropic and the coexistence
 * densities more accurate.  The weights are not printed; the ones used here:
 *
 * Isotropic 3x3 gradient D_h (error (ds^2/6) grad lap q, the same in every
 * direction):
 *   d_x q = [ (q(i+1,j) - q(i-1,j))/3
 *           + (q(i+1,j+1) - q(i-1,j+1) + q(i+1,j-1) - q(i-1,j-1))/12 ] / ds
 * Fourth-order gradient on the 5x5 square, the Richardson combination
 * (4 D_h - D_2h)/3 of D_h at spacings ds and 2 ds, which cancels that error:
 *   d_x q = [ 4/9 (q(i+1,j) - q(i-1,j))
 *           + 1/9 (q(i+1,j+1) - q(i-1,j+1) + q(i+1,j-1) - q(i-1,j-1))
 *           - 1/18 (q(i+2,j) - q(i-2,j))
 *           - 1/72 (q(i+2,j+2) - q(i-2,j+2) + q(i+2,j-2) - q(i-2,j-2)) ] / ds
 *   (on a planar profile it is the five-point fourth-order difference
 *    [8 (q(+1) - q(-1)) - (q(+2) - q(-2))] / 12)
 * Isotropic 9-point Laplacian:
 *   lap q = [ 2/3 (4 nearest) + 1/6 (4 diagonal) - 10/3 q(i,j) ] / ds^2
 * grad(p^i - p^w) takes the fourth-order gradient; grad(lap rho) the 3x3
 * gradient of the Laplacian, which composes to the 5x5 square as well.    */
typedef struct {
  int Lx, nrow, j0; /* rows j0 .. j0+nrow-1 */
  double* v;
} rowfield;

static double rf(const rowfield* r, int i, int j) {
  return r->v[(size_t)(j - r->j0) * r->Lx + wrap(i, r->Lx)];
}

static void grad_iso(const rowfield* q, int i, int j, double ds, double* gx, double* gy) {
  *gx = ((rf(q, i + 1, j) - rf(q, i - 1, j)) / 3.0 +
         (rf(q, i + 1, j + 1) - rf(q, i - 1, j + 1) + rf(q, i + 1, j - 1) - rf(q, i - 1, j - 1)) /
             12.0) / ds;
  *gy = ((rf(q, i, j + 1) - rf(q, i, j - 1)) / 3.0 +
         (rf(q, i + 1, j + 1) - rf(q, i + 1, j - 1) + rf(q, i - 1, j + 1) - rf(q, i - 1, j - 1)) /
             12.0) / ds;
}

static void grad_4th(const rowfield* q, int i, int j, double ds, double* gx, double* gy) {
  *gx = (4.0 / 9.0 * (rf(q, i + 1, j) - rf(q, i - 1, j)) +
         1.0 / 9.0 *
             (rf(q, i + 1, j + 1) - rf(q, i - 1, j + 1) + rf(q, i + 1, j - 1) - rf(q, i - 1, j - 1)) -
         1.0 / 18.0 * (rf(q, i + 2, j) - rf(q, i - 2, j)) -
         1.0 / 72.0 *
             (rf(q, i + 2, j + 2) - rf(q, i - 2, j + 2) + rf(q, i + 2, j - 2) - rf(q, i - 2, j - 2))) /
        ds;
  *gy = (4.0 / 9.0 * (rf(q, i, j + 1) - rf(q, i, j - 1)) +
         1.0 / 9.0 *
             (rf(q, i + 1, j + 1) - rf(q, i + 1, j - 1) + rf(q, i - 1, j + 1) - rf(q, i - 1, j - 1)) -
         1.0 / 18.0 * (rf(q, i, j + 2) - rf(q, i, j - 2)) -
         1.0 / 72.0 *
             (rf(q, i + 2, j + 2) - rf(q, i + 2, j - 2) + rf(q, i - 2, j + 2) - rf(q, i - 2, j - 2))) /
        ds;
}

static double lap_iso(const rowfield* q, int i, int j, double ds) {
  double nn = rf(q, i + 1, j) + rf(q, i - 1, j) + rf(q, i, j + 1) + rf(q, i, j - 1);
  double dg = rf(q, i + 1, j + 1) + rf(q, i - 1, j + 1) + rf(q, i + 1, j - 1) + rf(q, i - 1, j - 1);
  return (2.0 / 3.0 * nn + dg / 6.0 - 10.0 / 3.0 * rf(q, i, j)) / (ds * ds);
}

/* Fills gx, gy for rows 0..Ly-1 (and rho for rows -2..Ly+1 in rho_ext_rows). */
static void accel_field(const lattice* L, double* gx, double* gy) {
  const orc_params* p = L->p;
  const int Lx = p->Lx, Ly = p->Ly;
  rowfield rho = {Lx, Ly + 4, -2, malloc(sizeof(double) * Lx * (Ly + 4))};
  rowfield phi = {Lx, Ly + 4, -2, malloc(sizeof(double) * Lx * (Ly + 4))};
  rowfield lap = {Lx, Ly + 2, -1, malloc(sizeof(double) * Lx * (Ly + 2))};
#pragma omp parallel for schedule(static) if (PAR(p))
  for (int j = -2; j < Ly + 2; ++j)
    for (int i = 0; i < Lx; ++i) rho.v[(size_t)(j + 2) * Lx + i] = rho_at(L, i, j);
#pragma omp parallel for schedule(static) if (PAR(p))
  for (int j = -2; j < Ly + 2; ++j)
    for (int i = 0; i < Lx; ++i) {
      double r = rf(&rho, i, j);
      phi.v[(size_t)(j + 2) * Lx + i] = r * p->T - orc_pw(p, r); /* p^i - p^w */
      if (j >= -1 && j < Ly + 1) lap.v[(size_t)(j + 1) * Lx + i] = lap_iso(&rho, i, j, p->ds);
    }
#pragma omp parallel for schedule(static) if (PAR(p))
  for (int j = 0; j < Ly; ++j)
    for (int i = 0; i < Lx; ++i) {
      double px, py, lx, ly;
      grad_4th(&phi, i, j, p->ds, &px, &py);
      grad_iso(&lap, i, j, p->ds, &lx, &ly);
      double r = rf(&rho, i, j);
      gx[(size_t)j * Lx + i] = px / r + p->kappa * lx;
      gy[(size_t)j * Lx + i] = py / r + p->kappa * ly;
    }
  free(rho.v);
  free(phi.v);
  free(lap.v);
}

void orc_accel(const orc_params* p, const double* f, double* gx, double* gy) {
  tables();
  lattice L;
  lattice_init(&L, p, f);
  accel_field(&L, gx, gy);
}

/* ---- Sec. II C 2: jumps, MC limiter, limited corrections, fluxes ---------- */
double orc_limiter(int32_t limiter, double theta) {
  if (limiter == ORC_LIM_ZERO) return 0.0;
  if (limiter == ORC_LIM_ONE) return 1.0;
  /* monotonized centred limiter: max{0, min[(1+theta)/2, 2, 2 theta]} */
  double m = fmin(fmin(0.5 * (1.0 + theta), 2.0), 2.0 * theta);
  return fmax(0.0, m);
}

static int sgn(double v) { return v >= 0.0 ? 1 : -1; }

static double Rx(const lattice* L, int k, int i, int j) {
  return fget(L, k, i, j) - fget(L, k, i - 1, j);
}
static double Ry(const lattice* L, int k, int i, int j) {
  return fget(L, k, i, j) - fget(L, k, i, j - 1);
}

static double Sx(const lattice* L, int k, int i, int j) {
  const orc_params* p = L->p;
  double ax = fabs(XI[k][0]);
  double r = Rx(L, k, i, j);
  if (r == 0.0) return 0.0;
  double theta = Rx(L, k, i - sgn(XI[k][0]), j) / r;
  return 0.5 * ax * (1.0 - p->dt / p->ds * ax) * r * orc_limiter(p->limiter, theta);
}
static double Sy(const lattice* L, int k, int i, int j) {
  const orc_params* p = L->p;
  double ay = fabs(XI[k][1]);
  double r = Ry(L, k, i, j);
  if (r == 0.0) return 0.0;
  double theta = Ry(L, k, i, j - sgn(XI[k][1])) / r;
  return 0.5 * ay * (1.0 - p->dt / p->ds * ay) * r * orc_limiter(p->limiter, theta);
}

/* F_{k, i+1/2, j} */
static double flux_x(const lattice* L, int k, int i, int j) {
  const orc_params* p = L->p;
  const double xx = XI[k][0], xy = XI[k][1], lam = p->dt / p->ds;
  const int ux = (1 - sgn(xx)) / 2, uy = (1 - sgn(xy)) / 2; /* 0 or 1 */
  return fget(L, k, i + ux, j) * xx + Sx(L, k, i + 1, j) -
         0.5 * lam * xx * xy * Ry(L, k, i + ux, j + uy) +
         lam * xx * (Sy(L, k, i + ux, j) - Sy(L, k, i + ux, j + 1));
}

/* G_{k, i, j+1/2} */
static double flux_y(const lattice* L, int k, int i, int j) {
  const orc_params* p = L->p;
  const double xx = XI[k][0], xy = XI[k][1], lam = p->dt / p->ds;
  const int ux = (1 - sgn(xx)) / 2, uy = (1 - sgn(xy)) / 2;
  return fget(L, k, i, j + uy) * xy + Sy(L, k, i, j + 1) -
         0.5 * lam * xx * xy * Rx(L, k, i + ux, j + uy) +
         lam * xy * (Sx(L, k, i, j + uy) - Sx(L, k, i + 1, j + uy));
}

/* Eq. (ctueq): advected value from the four upwind-corner nodes */
static double ctu1(const lattice* L, int k, int i, int j) {
  const orc_params* p = L->p;
  const double ds = p->ds, dt = p->dt;
  const double ax = fabs(XI[k][0]), ay = fabs(XI[k][1]);
  const int sx = sgn(XI[k][0]), sy = sgn(XI[k][1]);
  return (fget(L, k, i, j) * (ds - ax * dt) * (ds - ay * dt) +
          fget(L, k, i - sx, j) * ax * (ds - ay * dt) * dt +
          fget(L, k, i, j - sy) * ay * (ds - ax * dt) * dt +
          fget(L, k, i - sx, j - sy) * ax * ay * dt * dt) /
         (ds * ds);
}

/* ---- Eq. (ereg): f <- f^eq + w [ H2:A2/2! + H3:A3/3! ] with A_n = sum f^neq xi^n */
static void regularize_node(const orc_params* p, double* fk) {
  double rho = 0.0, mx = 0.0, my = 0.0, fe[16];
  for (int k = 0; k < 16; ++k) {
    rho += fk[k];
    mx += fk[k] * XI[k][0];
    my += fk[k] * XI[k][1];
  }
  orc_feq(p, rho, mx / rho, my / rho, fe);
  double A2[2][2] = {{0, 0}, {0, 0}}, A3[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  for (int k = 0; k < 16; ++k) {
    double ne = fk[k] - fe[k];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        A2[a][b] += ne * XI[k][a] * XI[k][b];
        for (int c = 0; c < 2; ++c) A3[a][b][c] += ne * XI[k][a] * XI[k][b] * XI[k][c];
      }
  }
  for (int k = 0; k < 16; ++k) {
    double s2 = 0.0, s3 = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        s2 += H2(a, b, XI[k]) * A2[a][b];
        for (int c = 0; c < 2; ++c) s3 += H3(a, b, c, XI[k]) * A3[a][b][c];
      }
    fk[k] = fe[k] + W[k] * (s2 / 2.0 + s3 / 6.0);
  }
}

void orc_regularize(const orc_params* p, double* f) {
  tables();
  const size_t n = (size_t)p->Lx * p->Ly;
#pragma omp parallel for schedule(static) if (PAR(p))
  for (long q = 0; q < (long)n; ++q) {
    double fk[16];
    for (int k = 0; k < 16; ++k) fk[k] = f[(size_t)k * n + q];
    regularize_node(p, fk);
    for (int k = 0; k < 16; ++k) f[(size_t)k * n + q] = fk[k];
  }
}

/* ---- Sec. III A: outside R_BC = [L/2 - 1/(2 ds)] ds, f <- f rho_ext / rho ---- */
static double rbc_nodes(const orc_params* p) {
  int L = p->Lx < p->Ly ? p->Lx : p->Ly;
  return L / 2.0 - 1.0 / (2.0 * p->ds);
}

void orc_reservoir(const orc_params* p, double* f) {
  const size_t n = (size_t)p->Lx * p->Ly;
  const double r0 = rbc_nodes(p), cx = p->Lx / 2.0, cy = p->Ly / 2.0;
#pragma omp parallel for schedule(static) if (PAR(p))
  for (int j = 0; j < p->Ly; ++j)
    for (int i = 0; i < p->Lx; ++i) {
      if (hypot(i - cx, j - cy) <= r0) continue;
      size_t q = (size_t)j * p->Lx + i;
      double rho = 0.0;
      for (int k = 0; k < 16; ++k) rho += f[(size_t)k * n + q];
      double s = p->rho_ext / rho;
      for (int k = 0; k < 16; ++k) f[(size_t)k * n + q] *= s;
    }
}

/* ---- one full step ---------------------------------------------------------
 * Sec. II C splits Eq. (eBGK) into two explicit steps: first the advection
 * (left-hand side), then the collision and force (right-hand side):
 *   f*      = f^n - dt/ds [F_{i+1/2} - F_{i-1/2} + G_{j+1/2} - G_{j-1/2}]   (CTU2)
 *           or Eq. (ctueq)                                                 (CTU1)
 *   f^{n+1} = f* - dt/tau (f* - f^eq) + dt F_k
 * with rho, u, g, f^eq and F_k taken from the advected f*.  With
 * regularisation, f* is first replaced by f^eq + fhat^neq (Eq. ereg), so
 *   f^{n+1} = f^eq + (1 - dt/tau) fhat^neq + dt F_k.                       */
static void collide_node(const orc_params* p, const double* fs, double gx, double gy,
                         double* out) {
  double rho = 0.0, mx = 0.0, my = 0.0;
  for (int k = 0; k < 16; ++k) {
    rho += fs[k];
    mx += fs[k] * XI[k][0];
    my += fs[k] * XI[k][1];
  }
  double ux = mx / rho, uy = my / rho;
  double fe[16], Fk[16], fr[16];
  orc_feq(p, rho, ux, uy, fe);
  if (p->a2_full) {
    double a2[3] = {0, 0, 0};
    for (int k = 0; k < 16; ++k) {
      a2[0] += fs[k] * H2(0, 0, XI[k]);
      a2[1] += fs[k] * H2(0, 1, XI[k]);
      a2[2] += fs[k] * H2(1, 1, XI[k]);
    }
    orc_force(p, rho, ux, uy, gx, gy, a2, Fk);
  } else {
    orc_force(p, rho, ux, uy, gx, gy, NULL, Fk);
  }
  for (int k = 0; k < 16; ++k) fr[k] = fs[k];
  if (p->regularize) regularize_node(p, fr);
  const double om = p->dt / p->tau;
  for (int k = 0; k < 16; ++k) out[k] = fr[k] - om * (fr[k] - fe[k]) + p->dt * Fk[k];
}

static void one_step(const orc_params* p, const double* f, double* fn) {
  const int Lx = p->Lx, Ly = p->Ly;
  const size_t n = (size_t)Lx * Ly;
  const double lam = p->dt / p->ds;
  double* fs = malloc(sizeof(double) * 16 * n);
  lattice L;
  lattice_init(&L, p, f);
  /* advection of every velocity over its upwind corner stencil */
#pragma omp parallel for schedule(static) if (PAR(p))
  for (int j = 0; j < Ly; ++j)
    for (int i = 0; i < Lx; ++i)
      for (int k = 0; k < 16; ++k) {
        double v;
        if (p->ctu_order == 1)
          v = ctu1(&L, k, i, j);
        else
          v = fget(&L, k, i, j) - lam * (flux_x(&L, k, i, j) - flux_x(&L, k, i - 1, j) +
                                         flux_y(&L, k, i, j) - flux_y(&L, k, i, j - 1));
        fs[((size_t)k * Ly + j) * Lx + i] = v;
      }
  /* g from the advected density (ghost rows keep f^eq at rho_ext) */
  lattice Ls;
  lattice_init(&Ls, p, fs);
  double* gx = malloc(sizeof(double) * n);
  double* gy = malloc(sizeof(double) * n);
  accel_field(&Ls, gx, gy);
#pragma omp parallel for schedule(static) if (PAR(p))
  for (long q = 0; q < (long)n; ++q) {
    double a[16], b[16];
    for (int k = 0; k < 16; ++k) a[k] = fs[(size_t)k * n + q];
    collide_node(p, a, gx[q], gy[q], b);
    for (int k = 0; k < 16; ++k) fn[(size_t)k * n + q] = b[k];
  }
  free(fs);
  free(gx);
  free(gy);
}

int orc_step(const orc_params* p, double* f, int64_t nsteps) {
  tables();
  if (p->Lx < 1 || p->Ly < 1 || (p->ctu_order != 1 && p->ctu_order != 2)) return -1;
  const size_t n = (size_t)p->Lx * p->Ly;
  double* tmp = malloc(sizeof(double) * 16 * n);
  if (!tmp) return -2;
  for (int64_t s = 0; s < nsteps; ++s) {
    one_step(p, f, tmp);
    memcpy(f, tmp, sizeof(double) * 16 * n);
    if (p->reservoir) orc_reservoir(p, f);
  }
  free(tmp);
  return 0;
}

/* ---- diagnostics: mass, bubble sums for Eq. (gyr), probe densities ------- */
void orc_diagnostics(const orc_params* p, const double* f, double threshold, double r_ring,
                     orc_diag* out) {
  const int Lx = p->Lx, Ly = p->Ly;
  const size_t n = (size_t)Lx * Ly;
  memset(out, 0, sizeof(*out));
  out->rho_min = INFINITY;
  out->rho_max = -INFINITY;
  double ring = 0.0, nring = 0.0;
  const double cx = Lx / 2.0, cy = Ly / 2.0;
  for (int j = 0; j < Ly; ++j)
    for (int i = 0; i < Lx; ++i) {
      size_t q = (size_t)j * Lx + i;
      double rho = 0.0;
      for (int k = 0; k < 16; ++k) rho += f[(size_t)k * n + q];
      out->mass += rho;
      out->rho_min = fmin(out->rho_min, rho);
      out->rho_max = fmax(out->rho_max, rho);
      if (rho < threshold) {
        out->nb += 1.0;
        out->sx += i;
        out->sy += j;
        out->sxx += (double)i * i;
        out->sxy += (double)i * j;
        out->syy += (double)j * j;
      }
      if (fabs(hypot(i - cx, j - cy) - r_ring) < 0.5) {
        ring += rho;
        nring += 1.0;
      }
      if (i == Lx / 2 && j == Ly / 2) out->rho_center = rho;
    }
  out->rho_ring = nring > 0 ? ring / nring : NAN;
}

void orc_histogram(const orc_params* p, const double* f, int32_t nbins, double lo, double hi,
                   int64_t* counts) {
  const size_t n = (size_t)p->Lx * p->Ly;
  memset(counts, 0, sizeof(int64_t) * nbins);
  for (size_t q = 0; q < n; ++q) {
    double rho = 0.0;
    for (int k = 0; k < 16; ++k) rho += f[(size_t)k * n + q];
    double t = (rho - lo) / (hi - lo) * nbins;
    if (t >= 0.0 && t < nbins) counts[(int)t] += 1;
  }
}

// api.cu -- the C ABI declared in include/ctulbm.h.
//
// Host-side duties: parameter validation (CFL of Sec. II C 1, density range of
// Eq. evdw), per-velocity constants in FP64 (Table I, Eqs. ctueq, herfeq,
// ereg), launch geometry of the persistent step kernel, sticky error state,
// and the small host finishing step of the diagnostics (eigenvalues of the
// 2x2 gyration tensor, Eq. gyr).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>

#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "ctulbm.h"
#include "lbm_internal.h"

using namespace ctulbm;

struct lbm_handle {
  lbm_params p;
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t elem = 4;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned int* d_err = nullptr;
  unsigned long long* d_sched = nullptr;  // work-item counters of the step kernel
  DiagAcc* d_acc = nullptr;
  double* d_work = nullptr;       // 3 planes of FP64 for moments / init staging
  size_t work_elems = 0;
  int64_t steps = 0;
  int sticky = LBM_OK;
  int grid = 0;
  int nstrip = 0;
  int row_block = 256;
  bool vec = false;
  size_t smem = 0;
  double xi[16][2], w[16];
  StepArgs<float> a32;
  StepArgs<double> a64;
  // tensor maps of the step from f[c] to f[1 - c]: loads of f[c] (RPI-row and
  // 1-row staging boxes), stores of output tiles into f[1 - c]
  RowMaps tmap[2];
  // CUDA graphs of GRAPH_STEPS consecutive steps starting from f[0] / f[1]
  // (built on first use, rebuilt when the launch geometry changes)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  AuxArgs aux;
};

namespace {

void velocity_table(double xi[16][2], double w[16]) {
  const double s6 = std::sqrt(6.0);
  const double lo = std::sqrt(3.0 - s6), hi = std::sqrt(3.0 + s6);
  const double mag[4][2] = {{lo, lo}, {hi, lo}, {lo, hi}, {hi, hi}};
  const double wt[4] = {(5.0 + 2.0 * s6) / 48.0, 1.0 / 48.0, 1.0 / 48.0, (5.0 - 2.0 * s6) / 48.0};
  const double sg[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
  for (int m = 0; m < 4; ++m)
    for (int s = 0; s < 4; ++s) {
      xi[4 * m + s][0] = sg[s][0] * mag[m][0];
      xi[4 * m + s][1] = sg[s][1] * mag[m][1];
      w[4 * m + s] = wt[m];
    }
}

// Eq. (herfeq) in FP64 on the host (wall ghost rows).
void feq_host(const lbm_params& p, const double xi[16][2], const double w[16], double rho,
              double ux, double uy, double* out) {
  const double T = p.T, u2 = ux * ux + uy * uy;
  for (int k = 0; k < 16; ++k) {
    const double cu = xi[k][0] * ux + xi[k][1] * uy;
    const double x2 = xi[k][0] * xi[k][0] + xi[k][1] * xi[k][1];
    out[k] = w[k] * rho *
             (1.0 + cu + 0.5 * (cu * cu - u2 + (T - 1.0) * (x2 - 2.0)) +
              cu / 6.0 * (cu * cu - 3.0 * u2 + 3.0 * (T - 1.0) * (x2 - 4.0)));
  }
}

// The driver's tensor-map encoder, resolved once through the runtime (the
// library does not link the driver library itself).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// f [16][Ly][Lx] as a 3-D tensor ordered (x, plane, row), read in boxes of
// `cols` columns x 16 planes x `rows` rows: a box is [rows][16][cols] in
// shared memory (consecutive rows of the staging ring).  False when the
// encoder is unavailable or rejects the layout (the kernel then stages every
// strip by per-thread copies).
bool encode_row_map(void* base, size_t elem, int Lx, int Ly, int cols, int rows,
                    CUtensorMap* out) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || Lx < cols || Ly < rows) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Lx, 16, (cuuint64_t)Ly};
  const cuuint64_t strides[2] = {(cuuint64_t)Lx * (cuuint64_t)Ly * elem, (cuuint64_t)Lx * elem};
  const cuuint32_t box[3] = {(cuuint32_t)cols, 16, (cuuint32_t)rows};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType type = elem == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return enc(out, type, 3,
             base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// f [16][Ly][Lx] as a 3-D tensor ordered (x, row, plane), written in tiles of
// TW columns x RPI rows x 16 planes: a tile is [16][RPI][TW] in shared memory
// (the collision's plane-major output tile).  False when the encoder is
// unavailable or rejects the layout (the kernel then stores per thread).
bool encode_tile_map(void* base, size_t elem, int Lx, int Ly, CUtensorMap* out) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || Lx < TW || Ly < RPI) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Lx, (cuuint64_t)Ly, 16};
  const cuuint64_t strides[2] = {(cuuint64_t)Lx * elem, (cuuint64_t)Lx * (cuuint64_t)Ly * elem};
  const cuuint32_t box[3] = {(cuuint32_t)TW, (cuuint32_t)RPI, 16};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType type = elem == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return enc(out, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int set_err(lbm_handle* h, int code) {
  if (h && h->sticky == LBM_OK) h->sticky = code;
  return code;
}

int cuda_check(lbm_handle* h, cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  return set_err(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA);
}

double rho_ref_of(const lbm_params& p) { return p.precision == LBM_FP64 ? 0.0 : p.rho_ref; }

// FP32 keeps the relaxation exactly balanced: omega is put on the 2^-24 grid,
// so that 1 - omega is exact in FP32.  Rounding the two separately would leave
// (1 - omega) + omega 2e-8 off 1, a systematic damping of every deviation by
// that much per step (it shows as +2% in the decay rate of a shear wave over
// 2e5 steps).  FP64 keeps the exact value.
double snap(double v, bool fp32) {
  return fp32 ? std::ldexp(std::nearbyint(std::ldexp(v, 24)), -24) : v;
}

template <typename T>
void fill_step_args(lbm_handle* h, StepArgs<T>& a) {
  const lbm_params& p = h->p;
  const bool f32 = sizeof(T) == 4;
  const double lam = p.dt / p.ds, om = snap(p.dt / p.tau, f32), rr = rho_ref_of(p);
  a.Lx = p.Lx;
  a.Ly = p.Ly;
  a.plane = (long long)p.Lx * p.Ly;
  a.nstrip = h->nstrip;
  a.row_block = h->row_block;
  a.items = (long long)((p.Ly + h->row_block - 1) / h->row_block) * h->nstrip;
  a.sched = h->d_sched;
  a.diag_mass = nullptr;
  a.diag_sums = nullptr;
  a.diag_thr = (T)0;
  a.walls = p.boundary == LBM_BC_SHEAR_WALLS;
  a.reservoir = p.reservoir;
  a.regularize = p.regularize;
  a.rho_ref = (T)rr;
  a.Tt = (T)p.T;
  a.a = (T)p.a;
  a.b = (T)p.b;
  // force stencils (Eq. eder): the fourth-order gradient (4 D_h - D_2h)/3 of
  // p^i - p^w and the isotropic gradient D_h of the 9-point Laplacian, with
  // dt/ds (and kappa) folded into the weights
  a.gw1 = (T)(4.0 / 9.0 * lam);
  a.gw2 = (T)(1.0 / 9.0 * lam);
  a.gw3 = (T)(1.0 / 18.0 * lam);
  a.gw4 = (T)(1.0 / 72.0 * lam);
  // D_h (weights 1/3 axial, 1/12 diagonal) applied to the 9-point Laplacian
  // (2/3, 1/6, -10/3) / ds^2 is the 5x5 stencil W(a, b) = -W(-a, b) =
  // W(a, -b) with W(1, 0) = -1, W(1, 1) = -1/18, W(1, 2) = 1/18, W(2, 0) = 1/4,
  // W(2, 1) = 1/9, W(2, 2) = 1/72 (units 1/ds^3; W(0, b) = 0)
  {
    const double kl = p.kappa * lam / (p.ds * p.ds);
    const double w[6] = {-1.0, -1.0 / 18.0, 1.0 / 18.0, 0.25, 1.0 / 9.0, 1.0 / 72.0};
    for (int i = 0; i < 6; ++i) a.kw[i] = (T)(w[i] * kl);
  }
  a.omega = (T)om;
  a.one_m_omega = (T)(1.0 - om);
  a.om2 = (T)(0.5 * om);
  a.om6 = (T)(om / 6.0);
  a.rho_ext = (T)p.rho_ext;
  const int Lmin = p.Lx < p.Ly ? p.Lx : p.Ly;
  const double rbc = Lmin / 2.0 - 1.0 / (2.0 * p.ds);
  a.rbc2 = (T)(rbc > 0 ? rbc * rbc : 0.0);
  a.cxc = (T)(p.Lx / 2.0);
  a.cyc = (T)(p.Ly / 2.0);
  a.err = h->d_err;
  a.xlo = (T)std::sqrt(3.0 - std::sqrt(6.0));
  a.xhi = (T)std::sqrt(3.0 + std::sqrt(6.0));
  for (int grp = 0; grp < 4; ++grp) {
    const int k = 4 * grp;
    const double x2 = h->xi[k][0] * h->xi[k][0] + h->xi[k][1] * h->xi[k][1];
    const double Ak = (p.T - 1.0) * (x2 - 2.0) / 2.0, Bk = (p.T - 1.0) * (x2 - 4.0) / 2.0;
    a.cls[grp].omA = (T)(om * Ak);
    a.cls[grp].Ak = (T)Ak;
    a.cls[grp].omB = (T)(om * Bk);
    a.cls[grp].Bk = (T)Bk;
    a.cls[grp].w = (T)h->w[k];
  }
  double gb[16], gt[16];
  const double uw = p.shear_rate * p.Ly * p.ds / 2.0;
  feq_host(p, h->xi, h->w, p.rho_ext, -uw, 0.0, gb);
  feq_host(p, h->xi, h->w, p.rho_ext, +uw, 0.0, gt);
  for (int k = 0; k < 16; ++k) {
    const double x = h->xi[k][0], y = h->xi[k][1];
    const double ax = std::fabs(x), ay = std::fabs(y);
    const double cx = lam * ax, cy = lam * ay;
    const double hx = 0.5 * ax * (1.0 - cx), hy = 0.5 * ay * (1.0 - cy);
    const double x2 = x * x + y * y;
    const double Ak = (p.T - 1.0) * (x2 - 2.0) / 2.0, Bk = (p.T - 1.0) * (x2 - 4.0) / 2.0;
    VelConst<T>& v = a.v[k];
    v.xi_x = (T)x;
    v.xi_y = (T)y;
    v.w = (T)h->w[k];
    // CTU2 per node (Sec. II C 2 collected): with Z(j) = f - c_x (f - f(i - s_x))
    // - 2 lam hx dS^x(j), the update is Z(j) + c_y (Z(j - s_y) - Z(j))
    // - 2 lam hy [(1 - c_x) dS^y(i) + c_x dS^y(i - s_x)] on the kernel's
    // half-limited jumps (hence the factors 2).  The interpolations
    // f + c (g - f) return f exactly for g = f, so the CTU1 weights of a
    // uniform state sum to 1 in any precision.
    v.cx = (T)cx;
    v.cy = (T)cy;
    v.ax = (T)(2.0 * lam * hx);
    v.by0 = (T)(-2.0 * lam * hy * (1.0 - cx));
    v.by1 = (T)(-2.0 * lam * hy * cx);
    v.gbot = (T)(gb[k] - h->w[k] * rr);
    v.gtop = (T)(gt[k] - h->w[k] * rr);
    // Eq. (ereg): w [ H2:A2 / 2! + H3:A3 / 3! ] over the independent components
    v.r2xx = (T)(0.5 * (x * x - 1.0));
    v.r2xy = (T)(x * y);
    v.r2yy = (T)(0.5 * (y * y - 1.0));
    v.r3xxx = (T)((x * x * x - 3.0 * x) / 6.0);
    v.r3xxy = (T)(0.5 * (x * x * y - y));
    v.r3xyy = (T)(0.5 * (x * y * y - x));
    v.r3yyy = (T)((y * y * y - 3.0 * y) / 6.0);
  }
}

int validate(const lbm_params* p) {
  if (!p) return LBM_ERR_INVALID_ARG;
  if (p->Lx < 1 || p->Ly < 1) return LBM_ERR_INVALID_ARG;
  if ((long long)p->Lx * p->Ly > (1LL << 31) - 1) return LBM_ERR_INVALID_ARG;
  if (p->velset != LBM_VEL_D2Q16_H3) return LBM_ERR_UNSUPPORTED;
  if (p->ctu_order != 1 && p->ctu_order != 2) return LBM_ERR_INVALID_ARG;
  if (p->limiter < 0 || p->limiter > 2) return LBM_ERR_INVALID_ARG;
  if (p->boundary != LBM_BC_PERIODIC && p->boundary != LBM_BC_SHEAR_WALLS)
    return LBM_ERR_INVALID_ARG;
  if (p->precision != LBM_FP64 && p->precision != LBM_FP32_SHIFTED &&
      p->precision != LBM_FP16_SHIFTED)
    return LBM_ERR_UNSUPPORTED;
  if (p->regularize != 0 && p->regularize != 1) return LBM_ERR_INVALID_ARG;
  if (p->reservoir != 0 && p->reservoir != 1) return LBM_ERR_INVALID_ARG;
  if (!(p->tau > 0) || !(p->dt > 0) || !(p->ds > 0) || !(p->T > 0)) return LBM_ERR_INVALID_ARG;
  if (!(p->dt / p->tau < 2.0)) return LBM_ERR_INVALID_ARG;       // explicit relaxation stability
  if (!(p->kappa >= 0) || !(p->a >= 0) || !(p->b >= 0)) return LBM_ERR_INVALID_ARG;
  const double vmax = std::sqrt(3.0 + std::sqrt(6.0));
  if (vmax * p->dt > p->ds) return LBM_ERR_CFL;                   // Sec. II C 1
  if (p->boundary == LBM_BC_SHEAR_WALLS || p->reservoir) {
    if (!(p->rho_ext > 0) || (p->b > 0 && !(p->rho_ext * p->b < 1.0))) return LBM_ERR_DENSITY_RANGE;
  }
  if (!std::isfinite(p->shear_rate)) return LBM_ERR_INVALID_ARG;
  if (p->precision != LBM_FP64 && !std::isfinite(p->rho_ref)) return LBM_ERR_INVALID_ARG;
  return LBM_OK;
}

// Host finishing of a diagnostics record: centroid and Eq. (gyr) shape from
// the exact integer sums; probe fields only when the full reduction ran.
void finish_diag(const DiagAcc& acc, bool full, lbm_diag* out) {
  auto unkey = [](unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ULL) ? (k & ~0x8000000000000000ULL) : ~k;
    double v;
    std::memcpy(&v, &b, sizeof(v));
    return v;
  };
  std::memset(out, 0, sizeof(*out));
  out->mass = acc.mass;
  out->nb = (int64_t)acc.nb;
  out->sx = (int64_t)acc.sx;
  out->sy = (int64_t)acc.sy;
  out->sxx = (int64_t)acc.sxx;
  out->sxy = (int64_t)acc.sxy;
  out->syy = (int64_t)acc.syy;
  out->rho_center = full ? acc.rho_center : NAN;
  out->rho_ring = full && acc.ring_n ? acc.ring_sum / (double)acc.ring_n : NAN;
  out->rho_min = full ? unkey(acc.rmin_key) : NAN;
  out->rho_max = full ? unkey(acc.rmax_key) : NAN;
  if (acc.nb >= 1) {
    const double nb = (double)acc.nb;
    out->cx = (double)acc.sx / nb;
    out->cy = (double)acc.sy / nb;
  }
  if (acc.nb >= 2) {
    // Eq. (gyr): T = <r r> - <r><r>, from exact integer sums
    const double nb = (double)acc.nb;
    const double txx = (double)acc.sxx / nb - out->cx * out->cx;
    const double txy = (double)acc.sxy / nb - out->cx * out->cy;
    const double tyy = (double)acc.syy / nb - out->cy * out->cy;
    const double mean = 0.5 * (txx + tyy);
    const double rad = std::sqrt(0.25 * (txx - tyy) * (txx - tyy) + txy * txy);
    const double lM = mean + rad, lm = mean - rad;
    out->a = 2.0 * std::sqrt(lM > 0 ? lM : 0.0);
    out->b = 2.0 * std::sqrt(lm > 0 ? lm : 0.0);
    out->D = (out->a + out->b) > 0 ? (out->a - out->b) / (out->a + out->b) : 0.0;
    out->theta = 0.5 * std::atan2(2.0 * txy, txx - tyy);  // major-axis angle to x
  }
}

int check_device_error(lbm_handle* h) {
  unsigned int e = 0;
  if (cudaMemcpyAsync(&e, h->d_err, sizeof(e), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return set_err(h, LBM_ERR_CUDA);
  if (e & 1u) set_err(h, LBM_ERR_NONFINITE);
  if (e & 2u) set_err(h, LBM_ERR_TIMEOUT);
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_default_params(lbm_params* p, int32_t Lx, int32_t Ly) {
  if (!p) return LBM_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->Lx = Lx;
  p->Ly = Ly;
  p->velset = LBM_VEL_D2Q16_H3;
  p->a = 9.0 / 8.0;
  p->b = 1.0 / 3.0;
  p->kappa = 1e-4;
  p->T = 0.9;
  p->tau = 1e-3;
  p->dt = 1e-4;
  p->ds = 1.0 / 256.0;
  p->ctu_order = 2;
  p->limiter = LBM_LIM_MC;
  p->regularize = 0;
  p->boundary = LBM_BC_PERIODIC;
  p->shear_rate = 0.0;
  p->rho_ext = 1.0;
  p->reservoir = 0;
  p->precision = LBM_FP32_SHIFTED;
  p->rho_ref = 1.0;
  return LBM_OK;
}

int lbm_create(const lbm_params* p, void* cuda_stream, lbm_handle** out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  int v = validate(p);
  if (v != LBM_OK) return v;
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return LBM_ERR_OOM;
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return LBM_ERR_CUDA;
  }
  h->elem = p->precision == LBM_FP64 ? 8 : (p->precision == LBM_FP16_SHIFTED ? 2 : 4);
  velocity_table(h->xi, h->w);
  const size_t plane = (size_t)p->Lx * p->Ly;
  const size_t bytes = 16 * plane * h->elem;
  h->work_elems = 3 * plane;
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&h->f[0], bytes)) != cudaSuccess ||
      (e = cudaMalloc(&h->f[1], bytes)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_err, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_acc, sizeof(DiagAcc))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_sched, 2 * sizeof(unsigned long long))) != cudaSuccess) {
    lbm_destroy(h);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
  }
  cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), h->stream);
  cudaMemsetAsync(h->d_sched, 0, 2 * sizeof(unsigned long long), h->stream);

  // tensor maps: rows of f^n staged by tensor copies (row strides and the
  // staging window's start must be 16-byte multiples: Lx a multiple of 4
  // values, 8 for half), output tiles stored by tensor stores
  std::memset(h->tmap, 0, sizeof(h->tmap));
  bool tin = (p->Lx % (h->elem == 2 ? 8 : 4)) == 0, tout = tin;
  const int scol = h->elem == 2 ? scol_of<__half>() : scol_of<float>();
  for (int i = 0; i < 2; ++i) {
    tin = tin && encode_row_map(h->f[i], h->elem, p->Lx, p->Ly, scol, RPI, &h->tmap[i].m[0]) &&
          encode_row_map(h->f[i], h->elem, p->Lx, p->Ly, scol, 1, &h->tmap[i].m[1]);
    tout = tout && encode_tile_map(h->f[1 - i], h->elem, p->Lx, p->Ly, &h->tmap[i].m[2]);
  }
  h->vec = tin;  // else every strip stages by per-thread loads

  // launch geometry: strips of TW output columns, rows split evenly over a
  // persistent grid of (SMs x resident CTAs), at least 48 rows per CTA
  h->nstrip = (p->Lx + TW - 1) / TW;
  h->smem = step_smem_bytes(h->elem, h->elem == 8 ? 8 : 4);
  const int lim = p->ctu_order == 1 ? 0 : p->limiter;
  const bool regu = p->regularize != 0;
  int occ = h->elem == 4   ? step_occupancy_f32(p->ctu_order, lim, h->vec, regu, h->smem)
            : h->elem == 2 ? step_occupancy_f16(p->ctu_order, lim, h->vec, regu, h->smem)
                           : step_occupancy_f64(p->ctu_order, lim, h->vec, regu, h->smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (occ < 1 || nsm < 1) {
    lbm_destroy(h);
    return LBM_ERR_CUDA;
  }
  // work items: row blocks of up to 256 rows x strips; blocks shrink (down to
  // 96 rows, where the 7-row pipeline warm-up still costs < 8 %) when a
  // lattice would leave the grid with fewer than ~3 items per CTA.  A lattice
  // too small to give every CTA one 96-row item is latency-bound: its blocks
  // shrink further (down to 16 rows), trading warm-up work for a shorter row
  // loop per CTA.
  const long long rows_total = (long long)h->nstrip * p->Ly;
  const long long grid_max = (long long)nsm * occ;
  long long rb = rows_total / (3 * grid_max);
  rb = rb < 96 ? 96 : (rb > 256 ? 256 : rb);
  if (rows_total < 96 * grid_max) {
    const long long fill = (rows_total + grid_max - 1) / grid_max;
    rb = fill < 16 ? 16 : fill;
  }
  h->row_block = (int)rb;
  const long long items = (long long)((p->Ly + rb - 1) / rb) * h->nstrip;
  h->grid = (int)(items < grid_max ? items : grid_max);
  if (h->elem == 8)
    fill_step_args<double>(h, h->a64);
  else
    fill_step_args<float>(h, h->a32);
  h->a32.tma_in = h->a64.tma_in = tin;
  h->a32.tma_out = h->a64.tma_out = tout;
  AuxArgs& x = h->aux;
  x.Lx = p->Lx;
  x.Ly = p->Ly;
  x.plane = (long long)plane;
  x.storage = h->elem == 8 ? STORE_F64 : (h->elem == 2 ? STORE_F16 : STORE_F32);
  x.rho_ref = rho_ref_of(*p);
  x.Tt = p->T;
  std::memcpy(x.xi, h->xi, sizeof(h->xi));
  std::memcpy(x.w, h->w, sizeof(h->w));
  for (int k = 0; k < 16; ++k) {
    x.xif[k][0] = (float)h->xi[k][0];
    x.xif[k][1] = (float)h->xi[k][1];
    x.wf[k] = (float)h->w[k];
  }
  *out = h;
  return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& g : h->graph)
    if (g) cudaGraphExecDestroy(g);
  cudaFree(h->f[0]);
  cudaFree(h->f[1]);
  cudaFree(h->d_err);
  cudaFree(h->d_acc);
  cudaFree(h->d_sched);
  cudaFree(h->d_work);
  delete h;
}

static int ensure_work(lbm_handle* h) {
  if (h->d_work) return LBM_OK;
  if (cudaMalloc(&h->d_work, sizeof(double) * h->work_elems) != cudaSuccess)
    return set_err(h, LBM_ERR_OOM);
  return LBM_OK;
}

int lbm_init_rho_u_device(lbm_handle* h, const double* rho, const double* ux, const double* uy) {
  if (!h || !rho || !ux || !uy) return LBM_ERR_INVALID_ARG;
  h->cur = 0;
  h->steps = 0;
  return cuda_check(h, launch_init_feq(h->aux, h->f[0], rho, ux, uy, h->stream));
}

int lbm_init_rho_u(lbm_handle* h, const double* rho, const double* ux, const double* uy) {
  if (!h || !rho || !ux || !uy) return LBM_ERR_INVALID_ARG;
  int r = ensure_work(h);
  if (r) return r;
  const size_t n = (size_t)h->aux.plane, b = n * sizeof(double);
  double* d = h->d_work;
  if (cuda_check(h, cudaMemcpyAsync(d, rho, b, cudaMemcpyHostToDevice, h->stream)) ||
      cuda_check(h, cudaMemcpyAsync(d + n, ux, b, cudaMemcpyHostToDevice, h->stream)) ||
      cuda_check(h, cudaMemcpyAsync(d + 2 * n, uy, b, cudaMemcpyHostToDevice, h->stream)))
    return h->sticky;
  r = lbm_init_rho_u_device(h, d, d + n, d + 2 * n);
  if (r) return r;
  return cuda_check(h, cudaStreamSynchronize(h->stream));
}

int lbm_set_f_device(lbm_handle* h, const double* f) {
  if (!h || !f) return LBM_ERR_INVALID_ARG;
  h->cur = 0;
  h->steps = 0;
  return cuda_check(h, launch_set_f(h->aux, h->f[0], f, h->stream));
}

int lbm_get_f_device(lbm_handle* h, double* f) {
  if (!h || !f) return LBM_ERR_INVALID_ARG;
  return cuda_check(h, launch_get_f(h->aux, h->f[h->cur], f, h->stream));
}

// Host transfers stage through a device FP64 buffer of 16 planes, taken from
// the idle ping-pong buffer when the storage is FP64-sized, else allocated.
static int with_f64_stage(lbm_handle* h, double** stage, bool* owned) {
  *owned = false;
  if (h->elem == 8) {
    *stage = static_cast<double*>(h->f[1 - h->cur]);
    return LBM_OK;
  }
  if (cudaMalloc(stage, sizeof(double) * 16 * (size_t)h->aux.plane) != cudaSuccess)
    return set_err(h, LBM_ERR_OOM);
  *owned = true;
  return LBM_OK;
}

int lbm_set_f(lbm_handle* h, const double* f) {
  if (!h || !f) return LBM_ERR_INVALID_ARG;
  double* st;
  bool owned;
  h->cur = 0;  // the stage may be buffer 1
  int r = with_f64_stage(h, &st, &owned);
  if (r) return r;
  const size_t b = sizeof(double) * 16 * (size_t)h->aux.plane;
  r = cuda_check(h, cudaMemcpyAsync(st, f, b, cudaMemcpyHostToDevice, h->stream));
  if (!r) r = lbm_set_f_device(h, st);
  if (!r) r = cuda_check(h, cudaStreamSynchronize(h->stream));
  if (owned) cudaFree(st);
  return r;
}

int lbm_get_f(lbm_handle* h, double* f) {
  if (!h || !f) return LBM_ERR_INVALID_ARG;
  double* st;
  bool owned;
  int r = with_f64_stage(h, &st, &owned);
  if (r) return r;
  const size_t b = sizeof(double) * 16 * (size_t)h->aux.plane;
  r = lbm_get_f_device(h, st);
  if (!r) r = cuda_check(h, cudaMemcpyAsync(f, st, b, cudaMemcpyDeviceToHost, h->stream));
  if (!r) r = cuda_check(h, cudaStreamSynchronize(h->stream));
  if (owned) cudaFree(st);
  return r;
}

namespace {

constexpr int GRAPH_STEPS = 16;  // steps per graph launch (even: the buffers come back)

// One step launch from f[c] to f[1 - c].
cudaError_t launch_one(lbm_handle* h, int c, int lim) {
  if (h->elem != 8) {
    h->a32.fin = h->f[c];
    h->a32.fout = h->f[1 - c];
    return (h->elem == 4 ? launch_step_f32 : launch_step_f16)(
        h->a32, h->tmap[c], h->p.ctu_order, lim, h->vec, h->grid, h->smem, h->stream);
  }
  h->a64.fin = static_cast<const double*>(h->f[c]);
  h->a64.fout = static_cast<double*>(h->f[1 - c]);
  return launch_step_f64(h->a64, h->tmap[c], h->p.ctu_order, lim, h->vec, h->grid, h->smem,
                         h->stream);
}

// A graph of GRAPH_STEPS step kernels chained in order, starting from f[c]:
// one graph launch replaces GRAPH_STEPS kernel launches (small lattices are
// bound by launch overhead).  Built with explicit kernel nodes, so it works
// on any stream, the legacy default stream included.  nullptr on failure.
cudaGraphExec_t build_graph(lbm_handle* h, int c, int lim) {
  const bool f32 = h->elem != 8;
  const bool regu = h->p.regularize != 0;
  void* fn = h->elem == 8   ? step_kernel_ptr_f64(h->p.ctu_order, lim, h->vec, regu)
             : h->elem == 4 ? step_kernel_ptr_f32(h->p.ctu_order, lim, h->vec, regu)
                            : step_kernel_ptr_f16(h->p.ctu_order, lim, h->vec, regu);
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return nullptr;
  cudaGraphNode_t prev = nullptr;
  bool ok = true;
  for (int s = 0; s < GRAPH_STEPS && ok; ++s) {
    const int cc = (c + s) & 1;
    StepArgs<float> a32 = h->a32;
    StepArgs<double> a64 = h->a64;
    a32.fin = h->f[cc];
    a32.fout = h->f[1 - cc];
    a64.fin = static_cast<const double*>(h->f[cc]);
    a64.fout = static_cast<double*>(h->f[1 - cc]);
    RowMaps maps = h->tmap[cc];
    void* args[2] = {f32 ? static_cast<void*>(&a32) : static_cast<void*>(&a64), &maps};
    cudaKernelNodeParams kp{};
    kp.func = fn;
    kp.gridDim = dim3(h->grid);
    kp.blockDim = dim3(NT);
    kp.sharedMemBytes = (unsigned)h->smem;
    kp.kernelParams = args;  // copied into the node
    cudaGraphNode_t node = nullptr;
    ok = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp) ==
         cudaSuccess;
    prev = node;
  }
  cudaGraphExec_t ex = nullptr;
  if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  cudaGraphDestroy(g);
  return ex;
}

void drop_graphs(lbm_handle* h) {
  for (auto& g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

}  // namespace

int lbm_step(lbm_handle* h, int64_t n) {
  if (!h || n < 0) return LBM_ERR_INVALID_ARG;
  const int lim = h->p.ctu_order == 1 ? 0 : h->p.limiter;
  // whole blocks of GRAPH_STEPS steps by graph launches when there are two or more
  if (n >= 2 * GRAPH_STEPS) {
    cudaGraphExec_t& g = h->graph[h->cur];
    if (!g) g = build_graph(h, h->cur, lim);
    if (g) {
      for (; n >= GRAPH_STEPS; n -= GRAPH_STEPS) {
        const cudaError_t e = cudaGraphLaunch(g, h->stream);
        if (e != cudaSuccess) return cuda_check(h, e);
        h->steps += GRAPH_STEPS;  // an even count: h->cur is unchanged
      }
    }
  }
  for (int64_t s = 0; s < n; ++s) {
    const cudaError_t e = launch_one(h, h->cur, lim);
    if (e != cudaSuccess) return cuda_check(h, e);
    h->cur ^= 1;
    h->steps += 1;
  }
  return LBM_OK;
}

int lbm_set_launch(lbm_handle* h, int32_t row_block, int32_t ctas_per_sm) {
  if (!h || row_block < 1 || ctas_per_sm < 0) return LBM_ERR_INVALID_ARG;
  const int lim = h->p.ctu_order == 1 ? 0 : h->p.limiter;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  const bool regu = h->p.regularize != 0;
  const int occ =
      h->elem == 4   ? step_occupancy_f32(h->p.ctu_order, lim, h->vec, regu, h->smem)
      : h->elem == 2 ? step_occupancy_f16(h->p.ctu_order, lim, h->vec, regu, h->smem)
                     : step_occupancy_f64(h->p.ctu_order, lim, h->vec, regu, h->smem);
  if (nsm < 1 || occ < 1) return set_err(h, LBM_ERR_CUDA);
  if (ctas_per_sm > occ) return LBM_ERR_INVALID_ARG;
  if (ctas_per_sm == 0) ctas_per_sm = occ;
  const long long items = (long long)((h->p.Ly + row_block - 1) / row_block) * h->nstrip;
  const long long gmax = (long long)nsm * ctas_per_sm;
  h->row_block = row_block;
  h->grid = (int)(items < gmax ? items : gmax);
  h->a32.row_block = h->a64.row_block = row_block;
  h->a32.items = h->a64.items = items;
  drop_graphs(h);  // built for the old geometry
  return LBM_OK;
}

int lbm_tune(lbm_handle* h, int32_t steps_per_trial, lbm_kernel_info* out) {
  if (!h || steps_per_trial < 1) return LBM_ERR_INVALID_ARG;
  const int lim = h->p.ctu_order == 1 ? 0 : h->p.limiter;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  const bool regu = h->p.regularize != 0;
  const int occ =
      h->elem == 4   ? step_occupancy_f32(h->p.ctu_order, lim, h->vec, regu, h->smem)
      : h->elem == 2 ? step_occupancy_f16(h->p.ctu_order, lim, h->vec, regu, h->smem)
                     : step_occupancy_f64(h->p.ctu_order, lim, h->vec, regu, h->smem);
  if (nsm < 1 || occ < 1) return set_err(h, LBM_ERR_CUDA);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_err(h, LBM_ERR_CUDA);
  }
  auto apply = [&](int rb, int ctas) {
    const long long items = (long long)((h->p.Ly + rb - 1) / rb) * h->nstrip;
    const long long gmax = (long long)nsm * ctas;
    h->row_block = rb;
    h->grid = (int)(items < gmax ? items : gmax);
    h->a32.row_block = h->a64.row_block = rb;
    h->a32.items = h->a64.items = items;
  };
  // one trial: n real steps with geometry (rb, ctas), GPU time in ms
  int r = LBM_OK;
  auto trial = [&](int rb, int ctas, int n, float* ms) -> bool {
    apply(rb, ctas);
    cudaEventRecord(e0, h->stream);
    for (int s = 0; s < n; ++s) {
      const cudaError_t e = launch_one(h, h->cur, lim);
      if (e != cudaSuccess) {
        r = cuda_check(h, e);
        return false;
      }
      h->cur ^= 1;
      h->steps += 1;
    }
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) {
      r = set_err(h, LBM_ERR_CUDA);
      return false;
    }
    return true;
  };
  const int cur_rb = h->row_block;
  int cur_c = (int)((h->grid + nsm - 1) / nsm);
  cur_c = cur_c < 1 ? 1 : (cur_c > occ ? occ : cur_c);
  // the current geometry sets the trial length: at least ~1 ms of GPU time
  float ms = 0.0f;
  int steps = steps_per_trial;
  if (trial(cur_rb, cur_c, steps_per_trial, &ms) && ms > 0.0f && ms < 1.0f) {
    const float want = steps_per_trial / ms;
    steps = want > 1000.0f ? 1000 : (int)want + 1;
  }
  float best = 0.0f;
  int best_rb = cur_rb, best_c = cur_c;
  if (r == LBM_OK && trial(cur_rb, cur_c, steps, &best)) {
    const int rbs[] = {16, 32, 64, 96, 128, 192, 256, 384, 512, 1024};
    for (int ctas = 1; ctas <= occ && r == LBM_OK; ++ctas) {
      for (int rb : rbs) {
        if (rb > 16 && rb >= 2 * h->p.Ly) break;  // one block covers the lattice already
        if (rb == cur_rb && ctas == cur_c) continue;
        if (!trial(rb, ctas, steps, &ms)) break;
        if (ms < best) {
          best = ms;
          best_rb = rb;
          best_c = ctas;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply(best_rb, best_c);
  drop_graphs(h);  // built for the old geometry
  if (out) lbm_get_kernel_info(h, out);
  return r;
}

int lbm_step_many(lbm_handle* const* handles, int32_t count, int64_t n) {
  if (!handles || count < 1 || n < 0) return LBM_ERR_INVALID_ARG;
  lbm_handle* h0 = handles[0];
  if (!h0) return LBM_ERR_INVALID_ARG;
  const int lim0 = h0->p.ctu_order == 1 ? 0 : h0->p.limiter;
  for (int i = 0; i < count; ++i) {
    lbm_handle* h = handles[i];
    if (!h || h->stream != h0->stream || h->device != h0->device) return LBM_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) return LBM_ERR_INVALID_ARG;  // each lattice once
  }
  // Lattices that cannot share a launch (FP64 or FP16 storage, another scheme,
  // limiter or collision, no tensor maps) step on their own.
  lbm_handle* group[MAXB];
  int ng = 0;
  auto flush = [&](int64_t steps) -> int {
    if (ng == 0) return LBM_OK;
    if (ng == 1) {  // a lattice alone: the single-lattice path (graph launches, small parameters)
      ng = 0;
      return lbm_step(group[0], steps);
    }
    int grid_max = 0;
    {
      int occ = step_batch_occupancy_f32(h0->p.ctu_order, lim0, h0->p.regularize != 0,
                                         group[0]->smem);
      int nsm = 0;
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h0->device);
      grid_max = occ * nsm;
      if (grid_max < 1) return set_err(h0, LBM_ERR_CUDA);
    }
    std::unique_ptr<BatchArgs<float>> bp(new (std::nothrow) BatchArgs<float>());
    if (!bp) return set_err(h0, LBM_ERR_OOM);
    BatchArgs<float>& b = *bp;  // ~23 KB, copied into the launch's parameter space
    long long total = 0;
    b.count = ng;
    b.sched = h0->d_sched;
    // lattices share the launch, so each keeps row blocks of at least 96 rows
    // (its own may be shorter: sized to fill the GPU alone)
    int rbs[MAXB];
    long long its[MAXB];
    for (int i = 0; i < ng; ++i) {
      const StepArgs<float>& a = group[i]->a32;
      rbs[i] = a.row_block < 96 ? (a.Ly < 96 ? a.Ly : 96) : a.row_block;
      its[i] = (long long)((a.Ly + rbs[i] - 1) / rbs[i]) * a.nstrip;
      b.item_start[i] = total;
      total += its[i];
    }
    b.item_start[ng] = total;
    const int g = (int)(total < grid_max ? total : grid_max);
    const bool regu = h0->p.regularize != 0;
    // the arguments of the batched step `s` steps ahead of the lattices' state
    auto args_for = [&](int s) {
      for (int i = 0; i < ng; ++i) {
        lbm_handle* h = group[i];
        const int c = (h->cur + s) & 1;
        b.L[i] = h->a32;
        b.L[i].row_block = rbs[i];
        b.L[i].items = its[i];
        b.L[i].fin = static_cast<const float*>(h->f[c]);
        b.L[i].fout = static_cast<float*>(h->f[1 - c]);
        b.maps[i] = h->tmap[c];
      }
    };
    auto advance = [&](int64_t k) {
      for (int i = 0; i < ng; ++i) {
        group[i]->cur = (int)((group[i]->cur + k) & 1);
        group[i]->steps += k;
      }
    };
    // long runs: GRAPH_STEPS batched steps per graph launch (built for this
    // group, explicit kernel nodes, so any stream works)
    if (steps >= 3 * GRAPH_STEPS) {
      cudaGraph_t gr = nullptr;
      cudaGraphExec_t ex = nullptr;
      bool ok = cudaGraphCreate(&gr, 0) == cudaSuccess;
      cudaGraphNode_t prev = nullptr;
      void* fn = step_batch_kernel_ptr_f32(h0->p.ctu_order, lim0, regu);
      for (int s = 0; s < GRAPH_STEPS && ok; ++s) {
        args_for(s);
        void* kargs[1] = {&b};
        cudaKernelNodeParams kp{};
        kp.func = fn;
        kp.gridDim = dim3(g);
        kp.blockDim = dim3(NT);
        kp.sharedMemBytes = (unsigned)group[0]->smem;
        kp.kernelParams = kargs;  // copied into the node
        cudaGraphNode_t node = nullptr;
        ok = cudaGraphAddKernelNode(&node, gr, prev ? &prev : nullptr, prev ? 1 : 0, &kp) ==
             cudaSuccess;
        prev = node;
      }
      if (ok) ok = cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
      if (gr) cudaGraphDestroy(gr);
      if (ok) {
        for (; steps >= GRAPH_STEPS; steps -= GRAPH_STEPS) {
          const cudaError_t e = cudaGraphLaunch(ex, h0->stream);
          if (e != cudaSuccess) {
            cudaGraphExecDestroy(ex);
            return cuda_check(h0, e);
          }
          advance(GRAPH_STEPS);  // an even count: every lattice's buffer parity returns
        }
        cudaGraphExecDestroy(ex);
      } else if (ex) {
        cudaGraphExecDestroy(ex);
      }
    }
    for (int64_t s = 0; s < steps; ++s) {
      args_for(0);
      cudaError_t e = launch_step_batch_f32(b, h0->p.ctu_order, lim0, regu, g, group[0]->smem,
                                            h0->stream);
      if (e != cudaSuccess) return cuda_check(h0, e);
      advance(1);
    }
    ng = 0;
    return LBM_OK;
  };
  for (int i = 0; i < count; ++i) {
    lbm_handle* h = handles[i];
    const int lim = h->p.ctu_order == 1 ? 0 : h->p.limiter;
    const bool batchable = h->elem == 4 && h->vec && h->p.ctu_order == h0->p.ctu_order &&
                           h->p.regularize == h0->p.regularize &&
                           lim == lim0;
    if (!batchable) {
      int r = lbm_step(h, n);
      if (r) return r;
      continue;
    }
    group[ng++] = h;
    if (ng == MAXB) {
      int r = flush(n);
      if (r) return r;
    }
  }
  return flush(n);
}

int lbm_step_diag(lbm_handle* h, int64_t n, double threshold, lbm_diag* out) {
  if (!h || !out || n < 1) return LBM_ERR_INVALID_ARG;
  int r = lbm_step(h, n - 1);
  if (r) return r;
  DiagAcc acc;
  std::memset(&acc, 0, sizeof(acc));
  if (cuda_check(h, cudaMemsetAsync(h->d_acc, 0, sizeof(DiagAcc), h->stream))) return h->sticky;
  const int lim = h->p.ctu_order == 1 ? 0 : h->p.limiter;
  cudaError_t e;
  if (h->elem != 8) {
    StepArgs<float> a = h->a32;
    a.fin = h->f[h->cur];
    a.fout = h->f[1 - h->cur];
    a.diag_mass = &h->d_acc->mass;
    a.diag_sums = &h->d_acc->nb;
    a.diag_thr = (float)threshold;
    e = (h->elem == 4 ? launch_step_f32 : launch_step_f16)(a, h->tmap[h->cur], h->p.ctu_order, lim,
                                                           h->vec, h->grid, h->smem, h->stream);
  } else {
    StepArgs<double> a = h->a64;
    a.fin = static_cast<const double*>(h->f[h->cur]);
    a.fout = static_cast<double*>(h->f[1 - h->cur]);
    a.diag_mass = &h->d_acc->mass;
    a.diag_sums = &h->d_acc->nb;
    a.diag_thr = threshold;
    e = launch_step_f64(a, h->tmap[h->cur], h->p.ctu_order, lim, h->vec, h->grid, h->smem,
                        h->stream);
  }
  if (e != cudaSuccess) return cuda_check(h, e);
  h->cur ^= 1;
  h->steps += 1;
  if (cuda_check(h, cudaMemcpyAsync(&acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost,
                                    h->stream)) ||
      cuda_check(h, cudaStreamSynchronize(h->stream)))
    return h->sticky;
  finish_diag(acc, false, out);
  return lbm_sync(h);
}

int lbm_moments_device(lbm_handle* h, double* rho, double* ux, double* uy) {
  if (!h || !rho || !ux || !uy) return LBM_ERR_INVALID_ARG;
  return cuda_check(h, launch_moments(h->aux, h->f[h->cur], rho, ux, uy, h->stream));
}

int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy) {
  if (!h || !rho || !ux || !uy) return LBM_ERR_INVALID_ARG;
  int r = ensure_work(h);
  if (r) return r;
  const size_t n = (size_t)h->aux.plane, b = n * sizeof(double);
  double* d = h->d_work;
  r = lbm_moments_device(h, d, d + n, d + 2 * n);
  if (r) return r;
  if (cuda_check(h, cudaMemcpyAsync(rho, d, b, cudaMemcpyDeviceToHost, h->stream)) ||
      cuda_check(h, cudaMemcpyAsync(ux, d + n, b, cudaMemcpyDeviceToHost, h->stream)) ||
      cuda_check(h, cudaMemcpyAsync(uy, d + 2 * n, b, cudaMemcpyDeviceToHost, h->stream)) ||
      cuda_check(h, cudaStreamSynchronize(h->stream)))
    return h->sticky;
  return lbm_sync(h);
}

int lbm_diagnostics(lbm_handle* h, double threshold, double r_ring, lbm_diag* out) {
  if (!h || !out) return LBM_ERR_INVALID_ARG;
  DiagAcc acc;
  std::memset(&acc, 0, sizeof(acc));
  acc.rmin_key = ~0ULL;
  acc.rho_center = NAN;
  if (cuda_check(h, cudaMemcpyAsync(h->d_acc, &acc, sizeof(acc), cudaMemcpyHostToDevice,
                                    h->stream)) ||
      cuda_check(h, launch_diag(h->aux, h->f[h->cur], threshold, r_ring, h->d_acc, h->stream)) ||
      cuda_check(h, cudaMemcpyAsync(&acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost,
                                    h->stream)) ||
      cuda_check(h, cudaStreamSynchronize(h->stream)))
    return h->sticky;
  finish_diag(acc, true, out);
  return lbm_sync(h);
}

int lbm_histogram(lbm_handle* h, int32_t nbins, double lo, double hi, int64_t* counts) {
  if (!h || !counts || nbins < 1 || nbins > 65536 || !(hi > lo)) return LBM_ERR_INVALID_ARG;
  unsigned long long* d = nullptr;
  const size_t b = sizeof(unsigned long long) * nbins;
  if (cudaMalloc(&d, b) != cudaSuccess) return set_err(h, LBM_ERR_OOM);
  int r = LBM_OK;
  if (cuda_check(h, cudaMemsetAsync(d, 0, b, h->stream)) ||
      cuda_check(h, launch_hist(h->aux, h->f[h->cur], nbins, lo, hi, d, h->stream)) ||
      cuda_check(h, cudaMemcpyAsync(counts, d, b, cudaMemcpyDeviceToHost, h->stream)) ||
      cuda_check(h, cudaStreamSynchronize(h->stream)))
    r = h->sticky;
  cudaFree(d);
  if (r) return r;
  return lbm_sync(h);
}

int lbm_sync(lbm_handle* h) {
  if (!h) return LBM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) set_err(h, LBM_ERR_CUDA);
  check_device_error(h);
  const int r = h->sticky;
  h->sticky = LBM_OK;
  if (r == LBM_ERR_NONFINITE) cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), h->stream);
  return r;
}

int lbm_get_kernel_info(const lbm_handle* h, lbm_kernel_info* out) {
  if (!h || !out) return LBM_ERR_INVALID_ARG;
  out->grid = h->grid;
  out->threads = NT;
  out->smem_bytes = (int32_t)h->smem;
  out->strips = h->nstrip;
  out->row_block = h->row_block;
  out->tensor_copies = h->elem == 8 ? h->a64.tma_in : h->a32.tma_in;
  return LBM_OK;
}

int64_t lbm_step_count(const lbm_handle* h) { return h ? h->steps : -1; }

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "success";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_CFL: return "CFL condition violated: max |xi| dt > ds";
    case LBM_ERR_DENSITY_RANGE: return "density outside (0, 1/b)";
    case LBM_ERR_UNSUPPORTED: return "unsupported option";
    case LBM_ERR_OOM: return "device allocation failed";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_NONFINITE: return "non-finite or non-positive density after a step";
    case LBM_ERR_DEVICE_BOUNDS: return "device index check failed";
    case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown error";
  }
}

}  // extern "C"

/*
 * ctulbm.h -- C ABI of the GB300 (sm_103a) library for the time step of the
 * third-order, 16-velocity, isothermal van der Waals lattice Boltzmann model
 * advanced with corner transport upwind (CTU) schemes, after Sofonea,
 * Biciusca, Busuioc, Ambrus, Gonnella and Lamura, "Corner transport upwind
 * lattice Boltzmann model for bubble cavitation" (arXiv:1802.01272).
 *
 * One time step (Sec. II C splits Eq. eBGK into two explicit steps):
 *   1. advection of every f_k over its upwind corner stencil, CTU1
 *      (Eq. ctueq) or CTU2 (jumps R, MC-limited corrections S, fluxes F, G of
 *      Sec. II C 2);
 *   2. on the advected f: rho, u (Sec. II A), the van der Waals acceleration
 *      g (Eq. eder, vdW pressure Eq. evdw; the 25-point stencils of Sec. II B:
 *      a fourth-order 5x5 gradient of p^i - p^w and the isotropic 3x3
 *      gradient of the 9-point Laplacian of rho),
 *      f^eq (Eq. herfeq), F_k (Eq. herforce) and the BGK relaxation
 *      f <- f - dt/tau (f - f^eq) + dt F_k, optionally regularised (Eq. ereg);
 *   3. optionally the density reservoir of Sec. III A (rescale f outside R_BC).
 * Boundaries: periodic, or the sheared permeable walls of Sec. III C (ghost
 * rows j in {-2,-1} and {Ly, Ly+1} hold f^eq(rho_ext, (-+u_w, 0))), periodic
 * in x.
 *
 * Conventions for every entry point:
 *  - Return 0 on success or a negative LBM_ERR_* code.  A handle keeps the
 *    first error of an asynchronous launch (sticky) until lbm_sync() or a
 *    synchronising call returns it; nothing aborts, traps or exits.
 *  - Host arrays are FP64, owned by the caller, row-major: scalar fields
 *    [Ly][Lx] (x fastest), distributions [16][Ly][Lx].  They are read or
 *    written before the call returns.
 *  - "_device" variants take FP64 device pointers on the handle's device with
 *    the same layout; they are stream-ordered on the handle's stream.
 *  - The library owns all other device memory: allocated in lbm_create,
 *    freed in lbm_destroy.
 *  - Velocity order k = 0..15: groups of four with |xi| = (lo,lo), (hi,lo),
 *    (lo,hi), (hi,hi), lo = sqrt(3 - sqrt 6), hi = sqrt(3 + sqrt 6), weights
 *    (5+2 sqrt6)/48, 1/48, 1/48, (5-2 sqrt6)/48 (Table I); inside a group the
 *    signs (+,+), (-,+), (-,-), (+,-).
 */
#ifndef CTULBM_H
#define CTULBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1)   /* null pointer, bad size or enum value */
#define LBM_ERR_CFL (-2)           /* max_k |xi_k,a| dt > ds (Sec. II C 1) */
#define LBM_ERR_DENSITY_RANGE (-3) /* rho outside (0, 1/b) where the EOS is defined */
#define LBM_ERR_UNSUPPORTED (-4)   /* valid but not built: e.g. another velocity set */
#define LBM_ERR_OOM (-5)           /* device allocation failed */
#define LBM_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define LBM_ERR_NONFINITE (-7)     /* a step produced rho <= 0 or a non-finite rho */
#define LBM_ERR_DEVICE_BOUNDS (-8) /* a device-side index check failed (checked builds) */
#define LBM_ERR_TIMEOUT (-9)       /* a bounded device wait gave up */

/* ---- enumerations ------------------------------------------------------------ */
#define LBM_VEL_D2Q16_H3 0         /* the 16-velocity third-order set of Table I */
#define LBM_LIM_MC 0               /* monotonized centred limiter (Sec. II C 2) */
#define LBM_LIM_ZERO 1             /* Psi = 0: CTU2 reduces to CTU1 (test hook) */
#define LBM_LIM_ONE 2              /* Psi = 1: unlimited, Lax-Wendroff type (test hook) */
#define LBM_BC_PERIODIC 0
#define LBM_BC_SHEAR_WALLS 1       /* Sec. III C */
#define LBM_FP64 0                 /* f stored and computed in FP64 */
#define LBM_FP32_SHIFTED 1         /* f - w_k rho_ref stored and computed in FP32 */
#define LBM_FP16_SHIFTED 2         /* f - w_k rho_ref stored in FP16 (IEEE half), computed
                                      in FP32: half the memory traffic of FP32 storage,
                                      ~5e-4 relative rounding of the stored deviations per
                                      step (no counterpart in the paper, which computes in
                                      double precision) */

/* ---- parameters -------------------------------------------------------------
 * Defaults (lbm_default_params): a = 9/8, b = 1/3, kappa = 1e-4, T = 0.9,
 * tau = 1e-3, dt = 1e-4, ds = 1/256, CTU2 with the MC limiter, periodic,
 * FP32_SHIFTED with rho_ref = 1 (Sec. II D-E and III A).                   */
typedef struct lbm_params {
  int32_t Lx, Ly;          /* lattice nodes, each >= 1; the fast path wants Lx % 4 == 0
                              (Lx % 8 == 0 for FP16 storage) and Lx >= 72 */
  int32_t velset;          /* LBM_VEL_D2Q16_H3 */
  double a, b, kappa, T;   /* p^w = rho T/(1 - b rho) - a rho^2 (Eq. evdw); kappa of Eq. eder; T/T_c */
  double tau, dt, ds;      /* relaxation time, time step, lattice spacing */
  int32_t ctu_order;       /* 1 (Eq. ctueq) or 2 (Sec. II C 2) */
  int32_t limiter;         /* LBM_LIM_* (CTU2 only) */
  int32_t regularize;      /* 0 or 1: Eq. ereg inside the collision */
  int32_t boundary;        /* LBM_BC_* */
  double shear_rate;       /* gamma_dot of Sec. III C; wall speed u_w = gamma_dot Ly ds / 2 */
  double rho_ext;          /* density of the wall ghost rows and of the reservoir */
  int32_t reservoir;       /* 0 or 1: after every step, f <- f rho_ext/rho outside
                              R_BC = min(Lx,Ly)/2 - 1/(2 ds) nodes from (Lx/2, Ly/2) */
  int32_t precision;       /* LBM_FP64 | LBM_FP32_SHIFTED | LBM_FP16_SHIFTED */
  double rho_ref;          /* shift of the FP32 / FP16 storage (ignored in FP64) */
} lbm_params;

/* Diagnostics record (Sec. III B-C).  Bubble sites are nodes with
 * rho < threshold (the paper uses (rho_V + rho_L)/2).  Integer sums are exact.
 * a, b, D, theta follow Eq. (gyr): a = 2 sqrt(Lambda_M), b = 2 sqrt(Lambda_m),
 * D = (a-b)/(a+b), theta = angle of the major eigenvector to the x axis.      */
typedef struct lbm_diag {
  double mass;                 /* sum of rho over the lattice (FP64) */
  int64_t nb;                  /* bubble sites */
  int64_t sx, sy;              /* sums of i and j over bubble sites */
  int64_t sxx, sxy, syy;       /* sums of i*i, i*j, j*j over bubble sites */
  double rho_center;           /* rho at node (Lx/2, Ly/2) */
  double rho_ring;             /* mean rho over nodes within 0.5 of distance r_ring from (Lx/2, Ly/2) */
  double rho_min, rho_max;
  double cx, cy;               /* bubble centroid (nodes) */
  double a, b, D, theta;       /* shape from the gyration tensor; 0 if nb < 2 */
} lbm_diag;

typedef struct lbm_handle lbm_handle;

/* Fill *p with the defaults above for an Lx x Ly lattice. */
int lbm_default_params(lbm_params* p, int32_t Lx, int32_t Ly);

/* Validate *p (CFL, tau > 0, dt/tau < 2, 0 < rho_ext < 1/b when used, enums),
 * select the device current on the calling thread, allocate two ping-pong
 * buffers of 16 Lx Ly values plus small work areas, and bind the handle to
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * The distributions are uninitialised until lbm_init_rho_u or lbm_set_f. */
int lbm_create(const lbm_params* p, void* cuda_stream, lbm_handle** out);

/* Free every device allocation of the handle (synchronises its stream). NULL is a no-op. */
void lbm_destroy(lbm_handle* h);

/* f_k = f_k^eq(rho, u) (Eq. herfeq) at every node, from FP64 fields [Ly][Lx]:
 * host arrays (copied, then the stream is synchronised), or device arrays
 * for the _device variant (asynchronous; the caller keeps them alive until
 * the stream reaches this call).  The caller owns the arrays.  Resets the
 * step count. */
int lbm_init_rho_u(lbm_handle* h, const double* rho, const double* ux, const double* uy);
int lbm_init_rho_u_device(lbm_handle* h, const double* rho, const double* ux, const double* uy);

/* Copy distributions in or out, FP64 [16][Ly][Lx] in velocity order
 * (converted to/from the storage precision and layout); host variants
 * synchronise the stream, _device variants take device pointers and are
 * asynchronous.  lbm_set_f* resets the step count. */
int lbm_set_f(lbm_handle* h, const double* f);
int lbm_get_f(lbm_handle* h, double* f);
int lbm_set_f_device(lbm_handle* h, const double* f);
int lbm_get_f_device(lbm_handle* h, double* f);

/* Advance n >= 0 steps on the handle's stream (asynchronous; one fused kernel
 * per step).  From 32 steps on, whole blocks of 16 steps go out as one CUDA
 * graph launch (built on first use per handle; the same kernels, in order). */
int lbm_step(lbm_handle* h, int64_t n);

/* Advance n >= 1 steps and return the diagnostics of the final state, reduced
 * inside the last step's kernel (no extra pass over f): mass, bubble sites
 * rho < threshold, their integer moment sums and the Eq. (gyr) shape.
 * rho_center, rho_ring, rho_min and rho_max are NaN (use lbm_diagnostics).
 * Synchronises the stream. */
int lbm_step_diag(lbm_handle* h, int64_t n, double threshold, lbm_diag* out);

/* Advance `count` distinct lattices n >= 0 steps together (parameter sweeps,
 * many small jobs).  FP32-shifted lattices with Lx % 4 == 0 and the same
 * scheme and limiter as handles[0] share one fused launch per step, up to 16
 * per launch: their rows are split evenly over one persistent grid, which
 * keeps the GPU full when each lattice alone would not.  Other lattices step
 * on their own.  Every node goes through the same sequence of operations as in
 * lbm_step; the batched kernel is compiled separately, so FP32 results agree
 * with stepping alone to rounding (the compiler may fuse multiply-adds
 * differently), FP64 lattices step alone and agree exactly; a lattice alone in
 * its group takes lbm_step's path (graph launches).  All handles must share
 * one device and one stream (handles[0]'s); asynchronous like lbm_step.
 * Returns LBM_ERR_INVALID_ARG for a null or repeated handle or a stream
 * mismatch. */
int lbm_step_many(lbm_handle* const* handles, int32_t count, int64_t n);

/* rho, u = (sum_k f_k, sum_k f_k xi_k / rho) of the current state, FP64 [Ly][Lx].
 * The host version synchronises the stream. */
int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy);
int lbm_moments_device(lbm_handle* h, double* rho, double* ux, double* uy);

/* Reduction of the current state into *out (FP64 accumulators, exact integer sums);
 * synchronises the stream. */
int lbm_diagnostics(lbm_handle* h, double threshold, double r_ring, lbm_diag* out);

/* counts[b] = number of nodes with lo + b (hi-lo)/nbins <= rho < lo + (b+1)(hi-lo)/nbins;
 * 1 <= nbins <= 65536; synchronises the stream. */
int lbm_histogram(lbm_handle* h, int32_t nbins, double lo, double hi, int64_t* counts);

/* ---- allocation-free histogram (the paper has no counterpart) ----------------
 * Same counts as lbm_histogram, for distributions the caller holds in device
 * memory, without allocating anything.  It exists for callers that cannot
 * call cudaMalloc or any allocating routine: services whose device memory is
 * owned by another allocator or fully budgeted in advance, loops that cannot
 * afford the device synchronisation an allocation may imply, and callers
 * that keep f in their own buffers with no lbm_handle.  (lbm_histogram
 * allocates a device counts buffer on every call.)
 *   f_device : device pointer on the current device (another device returns
 *              LBM_ERR_INVALID_ARG), [16][Ly][Lx], FP64 f when precision is LBM_FP64,
 *              float (f - w_k rho_ref) when it is LBM_FP32_SHIFTED, IEEE half
 *              (f - w_k rho_ref) when it is LBM_FP16_SHIFTED
 *   nbins    : 1 .. LBM_NOALLOC_MAX_BINS; more returns LBM_ERR_INVALID_ARG
 *   counts   : host array of nbins int64, filled before return (the call
 *              synchronises cuda_stream); bins as in lbm_histogram
 * The bins are counted in one fixed device array of LBM_NOALLOC_MAX_BINS x 8
 * bytes, declared at file scope in the library: every device that loads the
 * library holds it until the process exits.  Each call zeroes the bins it
 * uses before counting; the array keeps the last call's counts afterwards.
 * All calls share that array, so calls that overlap on the GPU (different
 * streams or threads) race: issue them one after another.  The first call on
 * a device looks up the array's device address (once per device, with that
 * device current) and keeps it while the library is loaded, so the device's
 * context must not be reset (cudaDeviceReset) in between; make that first
 * call before any stream capture begins.
 * Returns LBM_ERR_INVALID_ARG for bad arguments, LBM_ERR_CUDA if a CUDA call
 * fails. */
#define LBM_NOALLOC_MAX_BINS 4096
int lbm_histogram_noalloc(const void* f_device, int32_t Lx, int32_t Ly, int32_t precision,
                          double rho_ref, int32_t nbins, double lo, double hi, void* cuda_stream,
                          int64_t* counts);

/* Wait for the handle's stream and return (then clear) its sticky error. */
int lbm_sync(lbm_handle* h);

/* Number of steps taken since the last init / set. */
int64_t lbm_step_count(const lbm_handle* h);

/* ---- batch server -----------------------------------------------------------
 * Continuous batching of many independent lattices (parameter sweeps over T,
 * shear rate, rho_ext: no counterpart in the paper, which runs one lattice at
 * a time).  A worker thread owned by the server admits submitted jobs in
 * submission order while their device footprint fits max_bytes and advances
 * resident jobs together (one batched launch per step for FP32 lattices with
 * the same scheme, lbm_step_many): each tick the jobs with the least work
 * left, as many as fill the GPU, while the others wait resident (short jobs
 * are not slowed to the pace of the largest lattice); it records each job's
 * diagnostics every diag_every steps and at its end, copies its final rho, u
 * to host memory and frees its device memory at once.  Jobs run to completion; a job's result
 * equals the one it has alone to FP32 rounding (exactly in FP64).
 *
 *   max_bytes   device memory the server may hold for jobs (each job needs
 *               32 x sizeof(storage) + 24 bytes per node)
 *   chunk_steps largest number of steps between two scheduling decisions
 *   cuda_stream stream for all of the server's work (NULL: the server creates
 *               its own); the device current at lbm_batch_create is used
 * All lbm_batch_* calls are thread-safe.  Returns LBM_ERR_INVALID_ARG for a
 * null argument, max_bytes = 0 or chunk_steps < 1, LBM_ERR_CUDA or
 * LBM_ERR_OOM if the stream or thread cannot be made. */
typedef struct lbm_batch lbm_batch;

#define LBM_JOB_PENDING 0          /* submitted, waiting for device memory */
#define LBM_JOB_ACTIVE 1           /* resident and stepping */
#define LBM_JOB_DONE 2             /* finished; final fields held on the host until fetched */
#define LBM_JOB_FAILED 3           /* error holds the cause (e.g. LBM_ERR_NONFINITE) */

typedef struct lbm_job_result {
  int32_t status;          /* LBM_JOB_* */
  int32_t error;           /* LBM_OK or the code that failed the job */
  int64_t steps_done, nsteps;
  int64_t diag_step;       /* step of `diag` (-1: no record yet) */
  double t_submit, t_start, t_finish;  /* seconds since lbm_batch_create (-1: not yet) */
  lbm_diag diag;           /* last diagnostics record, as lbm_diagnostics (r_ring = 0) */
} lbm_job_result;

typedef struct lbm_batch_info {
  int64_t pending, active, done, failed;
  int64_t used_bytes;      /* device bytes held by resident jobs */
  int64_t node_updates;    /* lattice nodes x steps advanced so far */
  int64_t launches;        /* lbm_step_many calls made by the worker */
} lbm_batch_info;

int lbm_batch_create(size_t max_bytes, int32_t chunk_steps, void* cuda_stream, lbm_batch** out);
/* Stops the worker after the step in flight, frees every job and the server. */
void lbm_batch_destroy(lbm_batch* b);
/* Queue a job.  rho, ux, uy: host FP64 [Ly][Lx], copied before return.
 * nsteps >= 1; diag_every >= 0 (0: a record at the end only); threshold:
 * bubble-site threshold of the records.  Returns the job id (>= 0) or
 * LBM_ERR_INVALID_ARG / the code lbm_create would return for these params,
 * LBM_ERR_OOM when the job alone exceeds max_bytes. */
int64_t lbm_batch_submit(lbm_batch* b, const lbm_params* p, const double* rho, const double* ux,
                         const double* uy, int64_t nsteps, int64_t diag_every, double threshold);
/* Current state of a job (LBM_ERR_INVALID_ARG for an unknown id). */
int lbm_batch_poll(lbm_batch* b, int64_t job, lbm_job_result* out);
/* Block until the job is DONE or FAILED (job = -1: every submitted job) or
 * timeout_s passes (< 0: no limit); LBM_ERR_TIMEOUT on timeout. */
int lbm_batch_wait(lbm_batch* b, int64_t job, double timeout_s, lbm_job_result* out);
/* Copy a DONE job's final rho, ux, uy (host FP64 [Ly][Lx], any may be NULL)
 * and release them; later fetches return LBM_ERR_INVALID_ARG. */
int lbm_batch_fetch(lbm_batch* b, int64_t job, double* rho, double* ux, double* uy);
int lbm_batch_get_info(lbm_batch* b, lbm_batch_info* out);

/* Launch geometry of the handle's fused step kernel (no counterpart in the
 * paper: for tuning, benchmarking and tests).
 *   grid          CTAs of the persistent launch (SMs x resident CTAs at most)
 *   threads       threads per CTA
 *   smem_bytes    dynamic shared memory per CTA
 *   strips        strips of 56 output columns across x
 *   row_block     rows per work item (work items = strips x row blocks)
 *   tensor_copies 1 when strips away from the periodic x seam stage f^n rows
 *                 with tensor (TMA) copies, 0 when every strip uses per-thread
 *                 16-byte copies (Lx not a multiple of 4, or Lx < 72)
 * Returns LBM_ERR_INVALID_ARG for a null argument; the handle is not touched. */
typedef struct lbm_kernel_info {
  int32_t grid, threads, smem_bytes, strips, row_block, tensor_copies;
} lbm_kernel_info;
int lbm_get_kernel_info(const lbm_handle* h, lbm_kernel_info* out);

/* Autotune the launch geometry of the handle's step kernel (no counterpart in
 * the paper): times steps_per_trial steps for each candidate row-block height
 * (16 .. 1024 rows, up to about twice Ly) and each number of resident CTAs
 * per SM, then keeps the fastest.  The trial steps are real steps of the run
 * (lbm_step_count grows by their number); the results of a step do not depend
 * on the launch geometry.  `out` (may be NULL) receives the chosen geometry.
 * Synchronises the handle's stream.  Returns LBM_ERR_INVALID_ARG for a null
 * handle or steps_per_trial < 1, LBM_ERR_CUDA if a launch or event fails. */
int lbm_tune(lbm_handle* h, int32_t steps_per_trial, lbm_kernel_info* out);

/* Set the launch geometry explicitly (e.g. one that lbm_tune chose earlier for
 * the same lattice size): row blocks of row_block rows, at most ctas_per_sm
 * resident CTAs per SM (0: as many as the kernel's resources allow on this
 * device).  Results do not depend on it.  No counterpart in the paper.
 * Returns LBM_ERR_INVALID_ARG for a null handle, row_block < 1 or
 * ctas_per_sm < 0 or above what the kernel's resources allow; LBM_ERR_CUDA if
 * the device cannot be queried. */
int lbm_set_launch(lbm_handle* h, int32_t row_block, int32_t ctas_per_sm);

/* Measured compute peaks of the current device (no counterpart in the paper:
 * the denominators of the compute rooflines a benchmark reports beside the
 * HBM one).  Runs two short probe kernels on cuda_stream (NULL: the legacy
 * default stream) and synchronises it:
 *   fp32_flops : FP32 FMA throughput, flop/s (independent FFMA chains)
 *   issue_rate : warp-instructions issued per second over the whole GPU, with
 *                independent chains alternating a 3-input FP32 min and an
 *                FP32 add (the ALU and FMA pipes the step kernel uses most)
 * Allocates and frees a probe buffer of (SMs x 2048) floats.  Returns
 * LBM_ERR_INVALID_ARG for a null output, LBM_ERR_OOM or LBM_ERR_CUDA. */
int lbm_measure_peaks(void* cuda_stream, double* fp32_flops, double* issue_rate);

/* Static description of a code. */
const char* lbm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CTULBM_H */

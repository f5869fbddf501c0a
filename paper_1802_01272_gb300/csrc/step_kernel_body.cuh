// step_kernel_body.cuh -- the fused CTU step kernel (included by lbm_kernels.cuh
// inside namespace ctulbm).  See the layout notes at the top of lbm_kernels.cuh.

// ------------------------------------- tensor copies, stores and mbarriers
// A staged batch (RPI rows of scol_of<ST>() columns x 16 planes) arrives by one
// tensor copy into a ring slot laid out [RPI][16][columns]; completion is
// counted in bytes on the slot's mbarrier, and every wait on it is bounded in
// time.  The collision's output tile [16][RPI][TW] is written into the slot
// whose batch P1 has consumed and leaves by one tensor store.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase `parity` of `bar` to complete, for at most `ns`
// nanoseconds; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > ns) return false;
  }
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// One tensor copy of rows y.. of the (x, plane, row) tensor into `dst`.
__device__ __forceinline__ void tma_load_rows(void* dst, const CUtensorMap* map, int x, int y,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(0), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// One tensor store of the tile at `src` to rows y.. of the (x, row, plane) tensor.
__device__ __forceinline__ void tma_store_rows(const CUtensorMap* map, int x, int y,
                                               const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
          map),
      "r"(x), "r"(y), "r"(0), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// at most N committed store groups may still be reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// every committed store group has completed (its writes are performed)
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ int mod_pos(int a, int n) {  // a mod n for a > -n*1024
  return (a + n * 1024) % n;
}

// Shared-memory layout: the staging ring and the output tiles in the storage
// type ST, the rings of advected rows and moments in the arithmetic type T,
// then ints.  All moment rings are indexed by lattice row mod MROWS.
template <typename T, typename ST>
struct Smem {
  static constexpr int SCOL = scol_of<ST>();
  // [NSLOT][RPI][16][SCOL] f^n rows of the strip, with the advection halo.
  // Once P1 has consumed a slot's batch, the slot holds that iteration's
  // f^{n+1} tile [16][RPI][TW] (plane-major) until its tensor store has read
  // it; the producer waits for that before it arms the slot's next copy.
  ST* stage;
  T* fs;      // [FROWS][FRS] advected f*: 16 planes of REG per row, padded
  T* drho;    // [MROWS][MP] rho* - rho_ref
  T* ux;
  T* uy;
  T* phi;     // p^i - p^w
  unsigned long long* dsums;  // [6] fused diagnostics: per-CTA bubble-site sums
  unsigned long long* bar;    // [NSLOT] mbarriers of the staging slots
  int* abort;                 // a bounded wait of this CTA timed out: stop waiting
  __device__ Smem(unsigned char* raw) {
    // tensor copies need 128-byte aligned tiles; the allocation has the slack
    raw += (128u - ((unsigned)__cvta_generic_to_shared(raw) & 127u)) & 127u;
    stage = reinterpret_cast<ST*>(raw);
    T* p = reinterpret_cast<T*>(stage + NSLOT * RPI * 16 * SCOL);
    fs = p;
    p += FROWS * FRS;
    drho = p;
    ux = drho + MROWS * MP;
    uy = ux + MROWS * MP;
    phi = uy + MROWS * MP;
    dsums = reinterpret_cast<unsigned long long*>(phi + MROWS * MP);  // 8-byte aligned
    bar = dsums + 6;
    abort = reinterpret_cast<int*>(bar + NSLOT);
  }
};

// Per-thread staging (lattices without tensor maps) and wall ghost rows: a
// staged row holds 16 planes x CH chunks of EPC values; thread t handles
// chunks t, t + NT, ..., so its (plane, column) slots are fixed for a segment.
template <typename T, typename ST>
struct StageSlots {
  static constexpr int SCOL = scol_of<ST>();
  static constexpr int CH = SCOL * (int)sizeof(ST) / 16;  // 16-byte chunks per plane row
  static constexpr int EPC = 16 / (int)sizeof(ST);         // elements per chunk
  static constexpr int PER_ROW = 16 * CH;
  static constexpr int NS = (PER_ROW + NT - 1) / NT;      // chunks per thread per row
  int dst[NS];        // element offset inside a staged row
  __device__ StageSlots() {
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      const int c = threadIdx.x + NT * m;
      const int k = c / CH, ch = c - (c / CH) * CH;
      dst[m] = k * SCOL + ch * EPC;
    }
  }
};

// Wall ghost row (constant per plane) into a staged row.
template <typename T, typename ST>
__device__ __forceinline__ void stage_ghost_row(const StepArgs<T>& P, const StageSlots<T, ST>& sl,
                                                ST* srow, bool bottom) {
  using SS = StageSlots<T, ST>;
#pragma unroll
  for (int m = 0; m < SS::NS; ++m) {
    const int c = threadIdx.x + NT * m;
    if (c < SS::PER_ROW) {
      const int k = c / SS::CH;
      const ST gv = to_store<ST, T>(bottom ? P.v[k].gbot : P.v[k].gtop);
#pragma unroll
      for (int e = 0; e < SS::EPC; ++e) srow[sl.dst[m] + e] = gv;
    }
  }
}

// Staged batch g (rows r0 .. r0+RPI-1, staging columns x0 .. x0+SCOL-1) lives
// in ring slot g % NSLOT; every batch arrives once on that slot's mbarrier
// (with the byte count of its tensor copies, zero otherwise), so the phase it
// completes has parity (g / NSLOT) & 1.
__device__ __forceinline__ unsigned slot_of(unsigned g) { return g % NSLOT; }
__device__ __forceinline__ unsigned parity_of(unsigned g) { return (g / NSLOT) & 1u; }

// Wall ghost rows of batch g (constant per plane), written by all threads.
template <typename T, typename ST>
__device__ __forceinline__ void ghost_rows(const StepArgs<T>& P, const Smem<T, ST>& S,
                                           const StageSlots<T, ST>& sl, int r0, unsigned g) {
  constexpr int SCOL = Smem<T, ST>::SCOL;
  if (!(P.walls && (r0 < 0 || r0 + RPI > P.Ly))) return;
  ST* base = S.stage + slot_of(g) * (RPI * 16 * SCOL);
  for (int r = 0; r < RPI; ++r) {
    const int row = r0 + r;
    if (row < 0 || row >= P.Ly) stage_ghost_row<T, ST>(P, sl, base + r * 16 * SCOL, row < 0);
  }
  // these generic writes precede later tensor copies into the same slot
  fence_proxy_async();
}

// Tensor copies of batch g, issued by the producer thread: one copy when the
// batch lies inside the lattice in y, else one per row (periodic wrap in y;
// wall ghost rows skipped).  Columns outside [0, Lx) arrive as zeros and
// seam_fixup replaces them.  After a timed-out wait nothing more is armed or
// issued: no copy can then be in flight except the batches armed before
// (drain_copies waits for them).
template <typename T, typename ST>
__device__ __forceinline__ void arm_tma(const StepArgs<T>& P, const Smem<T, ST>& S,
                                        const CUtensorMap* tm, int x0, int r0, unsigned g,
                                        unsigned& gi) {
  constexpr int SCOL = Smem<T, ST>::SCOL;
  constexpr unsigned ROW_BYTES = 16u * SCOL * (unsigned)sizeof(ST);
  if (*reinterpret_cast<volatile int*>(S.abort)) return;
  gi = g + 1u;
  const int Ly = P.Ly;
  ST* base = S.stage + slot_of(g) * (RPI * 16 * SCOL);
  unsigned long long* bar = S.bar + slot_of(g);
  if (r0 >= 0 && r0 + RPI <= Ly) {
    mbar_arrive_expect_tx(bar, RPI * ROW_BYTES);
    tma_load_rows(base, tm, x0, r0, bar);
  } else {
    unsigned bytes = 0;
    for (int r = 0; r < RPI; ++r)
      if (!(P.walls && (r0 + r < 0 || r0 + r >= Ly))) bytes += ROW_BYTES;
    mbar_arrive_expect_tx(bar, bytes);
    for (int r = 0; r < RPI; ++r) {
      const int row = r0 + r;
      if (P.walls && (row < 0 || row >= Ly)) continue;
      tma_load_rows(base + r * 16 * SCOL, tm + 1, x0, wrapi(row, Ly), bar);
    }
  }
}

// Lattices without tensor maps: every thread loads its chunks of batch g,
// wrapping in x and y; the producer arms the slot's barrier with no bytes.
template <typename T, typename ST>
__device__ __forceinline__ void load_scalar(const StepArgs<T>& P, const Smem<T, ST>& S,
                                            const StageSlots<T, ST>& sl, int x0, int r0,
                                            unsigned g, unsigned& gi) {
  using SS = StageSlots<T, ST>;
  constexpr int SCOL = Smem<T, ST>::SCOL;
  const int Ly = P.Ly;
  ST* base = S.stage + slot_of(g) * (RPI * 16 * SCOL);
  for (int r = 0; r < RPI; ++r) {
    const int row = r0 + r;
    if (P.walls && (row < 0 || row >= Ly)) continue;
    ST* srow = base + r * 16 * SCOL;
    const ST* frow = static_cast<const ST*>(P.fin) + (long long)wrapi(row, Ly) * P.Lx;
#pragma unroll
    for (int m = 0; m < SS::NS; ++m) {
      const int c = threadIdx.x + NT * m;
      if (c < SS::PER_ROW) {
        const int k = c / SS::CH, ch = c - k * SS::CH;
        const ST* fk = frow + (long long)k * P.plane;
#pragma unroll
        for (int e = 0; e < SS::EPC; ++e)
          srow[sl.dst[m] + e] = __ldg(fk + wrapi(x0 + ch * SS::EPC + e, P.Lx));
      }
    }
  }
  if (threadIdx.x == PRODUCER && !*reinterpret_cast<volatile int*>(S.abort)) {
    gi = g + 1u;
    mbar_arrive_expect_tx(S.bar + slot_of(g), 0u);
  }
}

// Every thread waits for staged batch g (bounded); per-thread loads also need
// the CTA barrier that makes the other threads' values visible.  A timeout
// sets error bit 1 and records the batch (abort = g + 1): the CTA stops
// waiting and issuing, its results are void.
template <bool VEC, typename T, typename SM>
__device__ __forceinline__ void wait_batch(const StepArgs<T>& P, const SM& S, unsigned g) {
  if (!*reinterpret_cast<volatile int*>(S.abort)) {
    if (!mbar_wait_bounded(S.bar + slot_of(g), parity_of(g), 1000000000ULL)) {
      *reinterpret_cast<volatile int*>(S.abort) = (int)(g + 1u);
      atomicOr(P.err, 2u);
    }
  }
  if (!VEC) __syncthreads();
}

// A strip at the periodic x seam: the tensor copy of batch g filled its
// staging columns outside [0, Lx) with zeros; each is replaced by its periodic
// image, loaded by the threads once the copy has landed (the left seam has 8
// such columns, the right one up to SCOL - 9 with Lx >= SCOL).  The columns
// come in 16-byte groups (Lx and the staging window's start are multiples of
// the group), every thread issues all of its loads before it stores any, and
// ghost rows, constant in x, are already complete.
template <typename T, typename ST>
__device__ __forceinline__ void seam_fixup(const StepArgs<T>& P, const Smem<T, ST>& S, int x0,
                                           int r0, unsigned g) {
  constexpr int SCOL = Smem<T, ST>::SCOL;
  constexpr int EPV = 16 / (int)sizeof(ST);  // values per 16-byte group
  constexpr int MAXV = (RPI * 16 * (SCOL / EPV) + NT - 1) / NT;  // groups per thread, at most
  const int Lx = P.Lx, Ly = P.Ly;
  const int nl = x0 < 0 ? -x0 / EPV : 0;                  // left: groups [0, nl)
  const int hs = (Lx - x0) / EPV;                          // right: groups [hs, SCOL / EPV)
  const int n = nl + (hs < SCOL / EPV ? SCOL / EPV - hs : 0);
  ST* base = S.stage + slot_of(g) * (RPI * 16 * SCOL);
  const ST* fin = static_cast<const ST*>(P.fin);
  uint4 v[MAXV];
  int at[MAXV];
#pragma unroll
  for (int m = 0; m < MAXV; ++m) {
    const int e = threadIdx.x + m * NT;
    at[m] = -1;
    if (e < RPI * 16 * n) {
      const int r = e / (16 * n), rem = e - r * (16 * n), k = rem / n, jj = rem - k * n;
      const int row = r0 + r;
      if (!(P.walls && (row < 0 || row >= Ly))) {
        const int j = (jj < nl ? jj : hs + (jj - nl)) * EPV;  // staging column
        const int x = wrapi(x0 + j, Lx);
        v[m] = __ldg(reinterpret_cast<const uint4*>(
            fin + (long long)k * P.plane + (long long)wrapi(row, Ly) * Lx + x));
        at[m] = (r * 16 + k) * SCOL + j;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < MAXV; ++m)
    if (at[m] >= 0) *reinterpret_cast<uint4*>(base + at[m]) = v[m];
  fence_proxy_async();  // before later tensor copies into the slot
  __syncthreads();
}

// P1 for one warp quadrant: the RPI staged rows of the batch in slot `sbase`,
// advected rows to the f* ring at `fbase` (thread's plane and group).
template <int SX, int SY, int ORDER, int LIM, typename T, typename ST>
__device__ __forceinline__ void advect_batch(typename AdvSel<T>::State& st, const VelConst<T>& vc,
                                             const ST* sbase, T* fa, T* fb) {
  // rows 0, 1 of the batch go to ring rows fa, fa + FRS; rows 2, 3 to fb, fb + FRS
  constexpr int SCOL = scol_of<ST>();
  if constexpr (sizeof(T) == 4) {
    const VelPairs vp = vel_pairs<SX>(vc);
#pragma unroll
    for (int r = 0; r < RPI; ++r) {
      float out[4];
      advect_row2<SX, SY, ORDER, LIM>(st, sbase + r * (16 * SCOL), vp, out);
      *reinterpret_cast<float4*>((r < 2 ? fa : fb) + (r & 1) * FRS) =
          make_float4(out[0], out[1], out[2], out[3]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < RPI; ++r) {
      T out[4];
      advect_row<SX, SY, ORDER, LIM>(st, sbase + r * (16 * SCOL), vc, out);
      T* dst = (r < 2 ? fa : fb) + (r & 1) * FRS;
      reinterpret_cast<double2*>(dst)[0] = make_double2(out[0], out[1]);
      reinterpret_cast<double2*>(dst)[1] = make_double2(out[2], out[3]);
    }
  }
}

// dt g / ds at one node (Eq. eder) from the moment rings; R[b + 2] is the ring
// offset (column included) of the node's row + b, b = -2 .. 2.
//  * grad(p^i - p^w): the fourth-order 5x5 gradient, the combination
//    (4 D_h - D_2h)/3 of the isotropic 3x3 gradient D_h at spacings ds and 2 ds;
//  * kappa grad(lap rho*): D_h of the isotropic 9-point Laplacian, the two
//    composed into one 5x5 stencil and applied to rho* - rho_ref (the
//    Laplacian of a constant vanishes), so no Laplacian row is kept.
// The y components read the x stencils transposed: each (x, y) pair of
// differences is one pair operation (packed FP32x2 in FP32).
template <typename T>
__device__ __forceinline__ void force_dt(const StepArgs<T>& P, const T* ph, const T* dq,
                                         const int (&R)[5], T ir, T& gdx, T& gdy) {
  using V = typename PairOf<T>::type;
  auto PH = [&](int a, int b) { return ph[R[b + 2] + a]; };
  auto Q = [&](int a, int b) { return dq[R[b + 2] + a]; };
  // x: F(a, b) - F(-a, b); y: F(b, a) - F(b, -a)
  auto dPH = [&](int a, int b) {
    return sub2(PairOf<T>::make(PH(a, b), PH(b, a)), PairOf<T>::make(PH(-a, b), PH(b, -a)));
  };
  auto dQ = [&](int a, int b) {
    return sub2(PairOf<T>::make(Q(a, b), Q(b, a)), PairOf<T>::make(Q(-a, b), Q(b, -a)));
  };
  const V t1 = dPH(1, 0), t2 = add2(dPH(1, 1), dPH(1, -1));
  const V t3 = dPH(2, 0), t4 = add2(dPH(2, 2), dPH(2, -2));
  const V pg = fma2(dup2(P.gw1), t1,
                    fma2(dup2(P.gw2), t2, fma2(dup2(-P.gw3), t3, mul2(dup2(-P.gw4), t4))));
  const V u0 = dQ(1, 0), u1 = add2(dQ(1, 1), dQ(1, -1)), u2 = add2(dQ(1, 2), dQ(1, -2));
  const V v0 = dQ(2, 0), v1 = add2(dQ(2, 1), dQ(2, -1)), v2 = add2(dQ(2, 2), dQ(2, -2));
  const V lg = fma2(dup2(P.kw[0]), u0,
               fma2(dup2(P.kw[1]), u1,
               fma2(dup2(P.kw[2]), u2,
               fma2(dup2(P.kw[3]), v0, fma2(dup2(P.kw[4]), v1, mul2(dup2(P.kw[5]), v2))))));
  const V g = fma2(dup2(ir), pg, lg);
  gdx = g.x;
  gdy = g.y;
}

// One row segment [ys, ye) of one strip of one lattice.  Every node's update
// uses the same arithmetic in the same order whatever the segment boundaries,
// so results do not depend on how the rows are split over CTAs or lattices.
//
// Iteration i consumes staged batch B_i = ys - 4 + 4 i .. +3 and, in the same
// iteration, P1 writes f* of rows B_i - 2 .., P2 their moments, P4 the outputs
// of rows B_i - 4 .. = ys + 4 (i - WARM) ..; the f* ring keeps rows by
// (row - ys) mod 6, the moment rings by (row - ys + 6) mod 8; three CTA
// barriers per iteration.  The tile of P4(i) is written into the staging slot
// that batch B_i has left and leaves by a tensor store that the producer
// issues at the start of iteration i + 1 (or after the loop), after the
// barrier that ends P4(i); the slot's next batch is armed once that store has
// read it.
template <typename T, typename ST, int ORDER, int LIM, bool VEC, bool DIAG, bool REGU>
__device__ __forceinline__ void run_segment(const StepArgs<T>& P, const Smem<T, ST>& S, int strip,
                                            int ys, int ye, const CUtensorMap* tm, unsigned& gb,
                                            unsigned& gi, double& dmass) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // P1 layout: a warp = one sign quadrant x two velocity groups x 16 column
  // groups, so column neighbours are adjacent lanes
  const int q = warp & 3;                                       // sign quadrant of the warp
  const int g = lane & 15;                                      // column group 0..15
  const int k = ((((warp >> 2) << 1) | (lane >> 4)) << 2) | q;  // velocity of this thread
  const VelConst<T> vc = P.v[k];
  const int Lx = P.Lx, Ly = P.Ly;

  // the tiles of the previous segment's last iterations may still be leaving
  // from the staging slots: the producer waits for their reads before anyone
  // writes a slot again
  if (VEC && P.tma_out && tid == PRODUCER) bulk_wait_read<0>();
  __syncthreads();  // previous segment done with the rings and the slots

  typename AdvSel<T>::State st;
  memset(&st, 0, sizeof(st));

  constexpr int SCOL = Smem<T, ST>::SCOL;
  const StageSlots<T, ST> slots;
  // first staging column (region column -4); the strips at the periodic x
  // seam get their wrapped columns from seam_fixup
  const int x0 = strip * TW - XOFF - 4;
  const bool seam = VEC && (x0 < 0 || x0 + SCOL > Lx);
  const bool producer = tid == PRODUCER;
  const bool tstore = VEC && P.tma_out;  // (the maps of both directions exist together)
  const int nit = WARM + (ye - ys + RPI - 1) / RPI;
  const unsigned g0 = gb;

  // per-thread bases: P1 (plane k, group g), P2 (node row r2, column c2),
  // P4 (row r4, output column)
  const ST* p1_src = S.stage + k * SCOL + 4 * g + 4;
  T* p1_dst = S.fs + k * REG + 4 * g;
  const int r2 = tid >> 6, c2 = tid & 63;
  const bool p4_on = tid < P4T;
  const int r4 = lane >> 3, o4 = 8 * warp + (lane & 7);  // row, output column of the strip
  const int c4 = XOFF + o4, x4 = strip * TW + o4;

  // batches g0 and g0 + 1 before the loop (both slots are free); in
  // iteration it >= 1 the producer issues the tensor copies of batch g0 + it + 1
  // at the end of P1 and all threads write its ghost rows after that barrier
  // (per-thread staging: loads and ghost rows of batch g0 + it + 1 in L)
  ghost_rows<T, ST>(P, S, slots, ys - 4, g0);
  if constexpr (VEC) {
    if (nit > 1) ghost_rows<T, ST>(P, S, slots, ys, g0 + 1);
    if (producer) {
      arm_tma<T, ST>(P, S, tm, x0, ys - 4, g0, gi);
      if (nit > 1) arm_tma<T, ST>(P, S, tm, x0, ys, g0 + 1, gi);
    }
  } else {
    load_scalar<T, ST>(P, S, slots, x0, ys - 4, g0, gi);
  }

  T dseg = T(0);  // fused diagnostics: mass of this thread's nodes (rho - rho_ref)
  int nseg = 0;
  int f6 = 0;  // f* ring row of row B - 2 (rows are kept mod FROWS = 6): 4 it mod 6
  for (int it = 0; it < nit; ++it) {
    const unsigned gcur = g0 + (unsigned)it;
    const int B = ys - 4 + RPI * it;  // first staged row of this iteration
    // ---------------- L: the previous iteration's output tile leaves from
    // its slot (its writes were fenced before the barrier that ended that
    // iteration); the next batch's ghost rows (and loads); wait for this batch
    if (tstore && producer) {
      const int row0 = ys + RPI * (it - 1 - WARM);  // rows of the previous iteration's P4
      if (it - 1 >= WARM && row0 + RPI <= ye) {       // (a partial batch is stored per thread)
        tma_store_rows(tm + 2, strip * TW, row0, S.stage + slot_of(gcur - 1) * (RPI * 16 * SCOL));
        bulk_commit();
      }
    }
    if constexpr (!VEC) {
      if (it + 1 < nit) {
        ghost_rows<T, ST>(P, S, slots, B + RPI, gcur + 1);
        load_scalar<T, ST>(P, S, slots, x0, B + RPI, gcur + 1, gi);
      }
    }
    wait_batch<VEC>(P, S, gcur);
    if (seam) seam_fixup<T, ST>(P, S, x0, B, gcur);

    // ---------------- P1: advect the staged batch into f* rows B - 2 ..
    {
      const ST* sb = p1_src + slot_of(gcur) * (RPI * 16 * SCOL);
      T* fa = p1_dst + f6 * FRS;                       // ring rows f6, f6 + 1
      T* fb = p1_dst + (f6 == 4 ? 0 : f6 + 2) * FRS;  // and f6 + 2, f6 + 3 (mod 6)
      switch (q) {
        case 0: advect_batch<+1, +1, ORDER, LIM>(st, vc, sb, fa, fb); break;
        case 1: advect_batch<-1, +1, ORDER, LIM>(st, vc, sb, fa, fb); break;
        case 2: advect_batch<-1, -1, ORDER, LIM>(st, vc, sb, fa, fb); break;
        default: advect_batch<+1, -1, ORDER, LIM>(st, vc, sb, fa, fb); break;
      }
      // wall ghost rows keep f^eq(rho_ext, u_wall)
      if (P.walls && (B - 2 < 0 || B + 2 > Ly)) {
#pragma unroll
        for (int r = 0; r < RPI; ++r) {
          const int a = B - 2 + r;
          if (a < 0 || a >= Ly) {
            const T gv = a < 0 ? vc.gbot : vc.gtop;
            T* dst = (r < 2 ? fa : fb) + (r & 1) * FRS;
#pragma unroll
            for (int m = 0; m < 4; ++m) dst[m] = gv;
          }
        }
      }
    }
    // the producer issues batch it + 1 into the other slot once the store of
    // the previous iteration's tile (issued in L) has read it
    if constexpr (VEC) {
      if (producer && it >= 1 && it + 1 < nit) {
        if (tstore) bulk_wait_read<0>();
        arm_tma<T, ST>(P, S, tm, x0, B + RPI, gcur + 1, gi);
      }
    }
    __syncthreads();
    if constexpr (VEC) {
      if (it >= 1 && it + 1 < nit) ghost_rows<T, ST>(P, S, slots, B + RPI, gcur + 1);
    }

    // ---------------- P2: moments of rows B - 2 .., one thread per node
    if (it >= 1) {
      const int sl = (it & 1) * RPI + r2;
      const T* src = S.fs + (f6 + r2 < 6 ? f6 + r2 : f6 + r2 - 6) * FRS + c2;
      T f[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) f[kk] = src[kk * REG];
      // velocity order: k = 4*group + sign, groups (lo,lo),(hi,lo),(lo,hi),(hi,hi),
      // signs (+,+),(-,+),(-,-),(+,-): per group A = f(++) - f(--), B = f(-+) - f(+-)
      T d[4], sx[4], sy[4];
#pragma unroll
      for (int gg = 0; gg < 4; ++gg) {
        const T* fg = f + 4 * gg;
        T A, Bm, s02, s13;
        if constexpr (sizeof(T) == 4) {  // (f0 +- f2, f1 +- f3) as packed pairs
          const float2 a = make_float2(fg[0], fg[1]), b = make_float2(fg[2], fg[3]);
          const float2 sp = add2(a, b), sm = sub2(a, b);
          s02 = sp.x; s13 = sp.y; A = sm.x; Bm = sm.y;
        } else {
          s02 = fg[0] + fg[2]; s13 = fg[1] + fg[3]; A = fg[0] - fg[2]; Bm = fg[1] - fg[3];
        }
        sx[gg] = A - Bm;
        sy[gg] = A + Bm;
        d[gg] = s02 + s13;
      }
      const T dr = (d[0] + d[1]) + (d[2] + d[3]);
      const T rho = P.rho_ref + dr;
      const T ir = rcp(rho);
      const int m = sl * MP + c2;
      S.drho[m] = dr;
      if constexpr (sizeof(T) == 4) {  // (rho ux, rho uy) and u as packed pairs
        const float2 mlo = add2(make_float2(sx[0], sy[0]), make_float2(sx[2], sy[1]));
        const float2 mhi = add2(make_float2(sx[1], sy[2]), make_float2(sx[3], sy[3]));
        const float2 u = mul2(fma2(dup2(P.xlo), mlo, mul2(dup2(P.xhi), mhi)), dup2(ir));
        S.ux[m] = u.x;
        S.uy[m] = u.y;
      } else {
        const T mx = P.xlo * (sx[0] + sx[2]) + P.xhi * (sx[1] + sx[3]);
        const T my = P.xlo * (sy[0] + sy[1]) + P.xhi * (sy[2] + sy[3]);
        S.ux[m] = mx * ir;
        S.uy[m] = my * ir;
      }
      // p^i - p^w = rho T - [rho T/(1 - b rho) - a rho^2]   (Eqs. eder, evdw)
      const T rT = rho * P.Tt;
      S.phi[m] = fma(P.a * rho, rho, rT - rT * rcp(T(1) - P.b * rho));
    }
    __syncthreads();

    // ---------------- P4: g, collision of all planes, output tile (rows B - 4 ..)
    if (it >= WARM && p4_on) {
      const int c = B - 4 + r4;  // lattice row
      T rho_post = T(-1);        // post-step density of this thread's node, if it has one
      if (c < ye && x4 < Lx) {
        const int s0 = ((it & 1) * RPI + r4 + 6) & 7;
        const int sc = s0 * MP + c4;
        const int sm = ((s0 + 7) & 7) * MP + c4;
        const int sp = ((s0 + 1) & 7) * MP + c4;
        const int s2m = ((s0 + 6) & 7) * MP + c4;
        const int s2p = ((s0 + 2) & 7) * MP + c4;
        const int R[5] = {s2m, sm, sc, sp, s2p};
        const T drho = S.drho[sc], ux = S.ux[sc], uy = S.uy[sc];
        const T rho = P.rho_ref + drho;  // as in P2
        const T ir = rcp(rho);
        T gdx, gdy;  // dt xi.g components: dt g
        force_dt<T>(P, S.phi, S.drho, R, ir, gdx, gdy);
        if (!(rho > T(0)) || !(rho < T(1e30))) atomicOr(P.err, 1u);
        const T e = T(1) - T(0.5) * (ux * ux + uy * uy);
        const T h = gdx * ux + gdy * uy;
        const T p0 = P.omega * drho * ir + P.omega * (e - T(1)) - h;
        const T p1 = e - P.Tt + T(1);
        const T p2 = P.omega * e - h;
        const T lo = P.xlo, hi = P.xhi;
        const T mxu[2] = {lo * ux, hi * ux}, myu[2] = {lo * uy, hi * uy};
        const T mxg[2] = {lo * gdx, hi * gdx}, myg[2] = {lo * gdy, hi * gdy};

        T f[16];
        const int fr = f6 + 4 + r4;  // f* ring row of lattice row c
        const T* src = S.fs + (fr < 6 ? fr : fr - 6) * FRS + c4;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) f[kk] = src[kk * REG];

        if constexpr (REGU) {
          // Eq. (ereg): replace f* by f^eq + w [H2:A2/2 + H3:A3/6], A_n = sum f^neq xi^n
          T m2xx = 0, m2xy = 0, m2yy = 0, m3xxx = 0, m3xxy = 0, m3xyy = 0, m3yyy = 0;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            const T x = P.v[kk].xi_x, y = P.v[kk].xi_y, fv = f[kk];
            m2xx += fv * x * x;
            m2xy += fv * x * y;
            m2yy += fv * y * y;
            m3xxx += fv * x * x * x;
            m3xxy += fv * x * x * y;
            m3xyy += fv * x * y * y;
            m3yyy += fv * y * y * y;
          }
          const T Tt = P.Tt;
          const T A2xx = m2xx + P.rho_ref - rho * (ux * ux + Tt);
          const T A2xy = m2xy - rho * ux * uy;
          const T A2yy = m2yy + P.rho_ref - rho * (uy * uy + Tt);
          const T A3xxx = m3xxx - rho * (ux * ux * ux + T(3) * Tt * ux);
          const T A3xxy = m3xxy - rho * (ux * ux * uy + Tt * uy);
          const T A3xyy = m3xyy - rho * (ux * uy * uy + Tt * ux);
          const T A3yyy = m3yyy - rho * (uy * uy * uy + T(3) * Tt * uy);
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            const VelConst<T>& v = P.v[kk];
            const ClassConst<T>& cl = P.cls[kk >> 2];
            const T cu = v.xi_x * ux + v.xi_y * uy;
            // f^eq - w rho_ref = w [ (rho - rho_ref) + rho (P_k - 1) ]
            const T pm1 = (e - T(1) + cl.Ak) + cu * ((e + cl.Bk) + cu * (T(0.5) + cu / T(6)));
            const T feqs = v.w * (drho + rho * pm1);
            const T fneq = v.w * (v.r2xx * A2xx + v.r2xy * A2xy + v.r2yy * A2yy +
                                  v.r3xxx * A3xxx + v.r3xxy * A3xxy + v.r3xyy * A3xyy +
                                  v.r3yyy * A3yyy);
            f[kk] = feqs + fneq;
          }
        }

        // f^{n+1} = (1 - omega) f* + w rho poly; opposite velocities (sign
        // patterns s and s + 2) differ only in the sign of xi.u and xi.g: the
        // cubic splits into even and odd parts E and O, poly(+-) = E +- O
        T outv[16];
        if constexpr (sizeof(T) == 4) {
          // FP32: the two sign patterns (+,+), (-,+) of a group as one packed
          // pair (their xi.u differ in the sign of the x term), the same
          // operations per component as the scalar form below
          const float2 rho2 = dup2(rho), p0_2 = dup2(p0), p1_2 = dup2(p1), p2_2 = dup2(p2);
          const float2 ux2 = dup2(ux), uy2 = dup2(uy), gx2 = dup2(gdx), gy2 = dup2(gdy);
          const float2 apm[2] = {mul2(make_float2(lo, -lo), ux2), mul2(make_float2(hi, -hi), ux2)};
          const float2 bb[2] = {mul2(dup2(lo), uy2), mul2(dup2(hi), uy2)};
          const float2 gpm[2] = {mul2(make_float2(lo, -lo), gx2), mul2(make_float2(hi, -hi), gx2)};
          const float2 gb[2] = {mul2(dup2(lo), gy2), mul2(dup2(hi), gy2)};
          const float2 s1 = dup2(P.one_m_omega), om2 = dup2(P.om2), om6 = dup2(P.om6);
#pragma unroll
          for (int grp = 0; grp < 4; ++grp) {
            const ClassConst<T>& cl = P.cls[grp];
            const int ix = grp & 1, iy = grp >> 1;
            const float2 P0 = add2(p0_2, dup2(cl.omA)), P1 = add2(p1_2, dup2(cl.Ak));
            const float2 K1c = add2(p2_2, dup2(cl.omB));
            const float2 sw = mul2(dup2(cl.w), rho2), nsw = mul2(dup2(-cl.w), rho2);
            const float2 cu = add2(bb[iy], apm[ix]);  // xi.u of (+,+), (-,+)
            const float2 D = add2(gb[iy], gpm[ix]);   // dt xi.g
            const float2 c2 = mul2(cu, cu);
            const float2 E = fma2(c2, om2, fma2(cu, D, P0));
            const float2 O = fma2(cu, fma2(c2, om6, K1c), mul2(D, fma2(c2, dup2(0.5f), P1)));
            const float2 Q = mul2(sw, E);
            const float2 op = fma2(s1, make_float2(f[4 * grp], f[4 * grp + 1]), fma2(sw, O, Q));
            const float2 om = fma2(s1, make_float2(f[4 * grp + 2], f[4 * grp + 3]), fma2(nsw, O, Q));
            outv[4 * grp] = op.x;
            outv[4 * grp + 1] = op.y;
            outv[4 * grp + 2] = om.x;
            outv[4 * grp + 3] = om.y;
          }
        } else {
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
          const ClassConst<T>& cl = P.cls[grp];
          const int ix = grp & 1, iy = grp >> 1;  // magnitude index (0 lo, 1 hi) in x, y
          const T P0 = p0 + cl.omA, P1 = p1 + cl.Ak, K1c = p2 + cl.omB, sw = cl.w * rho;
#pragma unroll
          for (int sgn = 0; sgn < 2; ++sgn) {
            const int kk = 4 * grp + sgn;
            const bool nx = sgn == 1;
            const T cu = (nx ? -mxu[ix] : mxu[ix]) + myu[iy];  // xi.u
            const T D = (nx ? -mxg[ix] : mxg[ix]) + myg[iy];   // dt xi.g
            // poly = K0 + cu (K1 + cu (K2 + cu om/6)) with K0 = D P1 + P0,
            // K1 = K1c + D, K2 = D/2 + om/2: the cubic in xi.u of
            // (omega f^eq + dt F_k - omega w rho_ref) / (w rho)
            const T c2 = cu * cu;
            const T E = c2 * P.om2 + (cu * D + P0);
            const T O = cu * (c2 * P.om6 + K1c) + D * (c2 * T(0.5) + P1);
            const T Q = sw * E;
            outv[kk] = fma(P.one_m_omega, f[kk], fma(sw, O, Q));
            outv[kk + 2] = fma(P.one_m_omega, f[kk + 2], fma(-sw, O, Q));
          }
        }
        }
        rho_post = rho;  // the collision conserves mass
        if (P.reservoir) {
          // Sec. III A: outside R_BC the node is rescaled to rho_ext: f -> s f,
          // stored deviation s (f - w rho_ref) + w rho_ref (s - 1)
          const T dx = T(x4) - P.cxc, dy = T(c) - P.cyc;
          if (dx * dx + dy * dy > P.rbc2) {
            const T s = P.rho_ext * ir;
            rho_post = s * rho;
#pragma unroll
            for (int kk = 0; kk < 16; ++kk)
              outv[kk] = fma(s, outv[kk], P.cls[kk >> 2].w * P.rho_ref * (s - T(1)));
          }
        }
        if (tstore && B + RPI - 4 <= ye) {  // a full batch: the tile
          ST* dst = S.stage + slot_of(gcur) * (RPI * 16 * SCOL) + r4 * TW + o4;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) dst[kk * (RPI * TW)] = to_store<ST, T>(outv[kk]);
        } else {
          ST* dst = static_cast<ST*>(P.fout) + (long long)c * Lx + x4;
          const long long pl = P.plane;
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) dst[kk * pl] = to_store<ST, T>(outv[kk]);
        }
      }
      if (DIAG) {  // fused diagnostics: mass per thread, bubble sites per warp
        const bool on = rho_post >= T(0);
        const bool in = on && rho_post < P.diag_thr;
        if (on) {
          dseg += rho_post - P.rho_ref;
          ++nseg;
        }
        if (__ballot_sync(0xffffffffu, in)) {  // bubble sites are rare: sum them only here
          const unsigned long long ii = in ? (unsigned long long)x4 : 0ULL;
          const unsigned long long jj = in ? (unsigned long long)c : 0ULL;
          unsigned long long v[6] = {in ? 1ULL : 0ULL, ii, jj, ii * ii, ii * jj, jj * jj};
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int t = 0; t < 6; ++t) v[t] += __shfl_down_sync(0xffffffffu, v[t], o);
          }
          if (lane == 0) {
#pragma unroll
            for (int t = 0; t < 6; ++t) atomicAdd(&S.dsums[t], v[t]);
          }
        }
      }
    }
    if (tstore) fence_proxy_async();  // the tile's generic writes before its tensor store
    __syncthreads();
    f6 = f6 >= 2 ? f6 - 2 : f6 + 4;
  }
  // the last tile of the segment
  if (tstore && producer) {
    const int row0 = ys + RPI * (nit - 1 - WARM);
    if (row0 + RPI <= ye) {
      tma_store_rows(tm + 2, strip * TW, row0,
                     S.stage + slot_of(g0 + (unsigned)(nit - 1)) * (RPI * 16 * SCOL));
      bulk_commit();
    }
  }
  gb = g0 + (unsigned)nit;
  if (DIAG) dmass += (double)dseg + (double)P.rho_ref * (double)nseg;
}

// Work items are (row block, strip) pairs claimed from a device counter: first
// the strips at the periodic x seam (slower: they complete their staging
// window by hand), so that they do not end up as the launch's tail, then the
// others in row-block-major order, so that CTAs running at the same time work
// on the same rows of neighbouring strips and the halo columns they share and
// the output lines they both write meet in L2.  The last CTA to finish resets
// the counters, so the next launch (or a replay of a captured graph) starts
// from zero.
__device__ __forceinline__ void item_coords(long long item, int nstrip, long long nrb, int& strip,
                                            long long& rb) {
  if (nstrip < 3) {
    rb = item / nstrip;
    strip = (int)(item - rb * nstrip);
  } else if (item < 2 * nrb) {
    rb = item >> 1;
    strip = (item & 1) ? nstrip - 1 : 0;
  } else {
    const long long j = item - 2 * nrb;
    rb = j / (nstrip - 2);
    strip = 1 + (int)(j - rb * (nstrip - 2));
  }
}
__device__ __forceinline__ long long claim_item(unsigned long long* sched, long long* s_item) {
  __syncthreads();  // everyone has read the previous item
  if (threadIdx.x == 0) *s_item = (long long)atomicAdd(&sched[0], 1ULL);
  __syncthreads();
  return *s_item;
}
__device__ __forceinline__ void retire_cta(unsigned long long* sched) {
  if (threadIdx.x == 0) {
    const unsigned long long done = atomicAdd(&sched[1], 1ULL);
    if (done == gridDim.x - 1) {
      sched[0] = 0ULL;
      sched[1] = 0ULL;
    }
  }
}

// Before the CTA leaves: every tensor store has completed, and every staged
// batch it armed has landed.  Normally all were waited for; after a timed-out
// wait (abort = first such batch + 1) the batches from that one up to the
// last armed may still be in flight into this CTA's shared memory, and the
// producer waits for each again, bounded, so that no copy outlives the CTA
// unless the copy engine itself is stuck.
template <typename SM>
__device__ __forceinline__ void drain_copies(const SM& S, unsigned armed) {
  if (threadIdx.x == PRODUCER) {
    bulk_wait_all();
    const int a = *reinterpret_cast<volatile int*>(S.abort);
    if (a > 0)
      for (unsigned b = (unsigned)(a - 1); b < armed; ++b)
        mbar_wait_bounded(S.bar + slot_of(b), parity_of(b), 2000000000ULL);
  }
}

__device__ __forceinline__ void init_cta_barriers(unsigned long long* dsums,
                                                  unsigned long long* bar, int* abort) {
  if (threadIdx.x == 0) {
    for (int t = 0; t < 6; ++t) dsums[t] = 0ULL;
    *abort = 0;
    for (int b = 0; b < NSLOT; ++b) mbar_init(bar + b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
}

// DIAG: fuse the diagnostics of the state after the step (P.diag_mass and
// P.diag_sums receive them); REGU: the regularised collision (Eq. ereg).  Both
// are separate instantiations, so that the plain step carries none of their
// instructions (cold code in the loop body costs instruction fetch).
template <typename T, typename ST, int ORDER, int LIM, bool VEC, bool DIAG, bool REGU>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1)
    step_kernel(const __grid_constant__ StepArgs<T> P, const __grid_constant__ RowMaps maps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Smem<T, ST> S(smem_raw);
  __shared__ long long s_item;
  init_cta_barriers(S.dsums, S.bar, S.abort);
  const CUtensorMap* tm = maps.m;
  unsigned gb = 0;     // staged batches of this CTA so far (slot g % NSLOT)
  unsigned gi = 0;     // the producer: batches armed on the mbarriers
  double dmass = 0.0;  // fused diagnostics: this thread's mass over all its segments
  for (;;) {
    const long long item = claim_item(P.sched, &s_item);
    if (item >= P.items) break;
    int strip;
    long long rb;
    item_coords(item, P.nstrip, P.items / P.nstrip, strip, rb);
    const int ys = (int)(rb * P.row_block);
    const int ye = min(P.Ly, ys + P.row_block);
    run_segment<T, ST, ORDER, LIM, VEC, DIAG, REGU>(P, S, strip, ys, ye, tm, gb, gi, dmass);
  }
  if (DIAG) {
    // one warp sum and one global add per warp for the mass; claim_item's
    // barrier after the last claim orders every warp's shared site sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmass += __shfl_down_sync(0xffffffffu, dmass, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(P.diag_mass, dmass);
    if (threadIdx.x == 0)
      for (int t = 0; t < 6; ++t) atomicAdd(&P.diag_sums[t], S.dsums[t]);
  }
  drain_copies(S, gi);
  retire_cta(P.sched);
}

// Several lattices advanced by one launch: their work items are concatenated
// and claimed from one counter; each lattice brings its own tensor maps.
template <typename T, int ORDER, int LIM, bool VEC, bool REGU>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1)
    step_batch_kernel(const __grid_constant__ BatchArgs<T> B) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Smem<T, T> S(smem_raw);
  __shared__ long long s_item;
  init_cta_barriers(S.dsums, S.bar, S.abort);
  int i = 0;
  unsigned gb = 0, gi = 0;
  double dmass = 0.0;  // unused: batched launches carry no fused diagnostics
  for (;;) {
    const long long item = claim_item(B.sched, &s_item);
    if (item >= B.item_start[B.count]) break;
    while (B.item_start[i + 1] <= item) ++i;
    const StepArgs<T>& P = B.L[i];
    const long long local = item - B.item_start[i];
    int strip;
    long long rb;
    item_coords(local, P.nstrip, P.items / P.nstrip, strip, rb);
    const int ys = (int)(rb * P.row_block);
    const int ye = min(P.Ly, ys + P.row_block);
    run_segment<T, T, ORDER, LIM, VEC, false, REGU>(P, S, strip, ys, ye, B.maps[i].m, gb, gi, dmass);
  }
  drain_copies(S, gi);
  retire_cta(B.sched);
}

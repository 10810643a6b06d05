// sm_103a kernels of the PDHG hot path.
//
//  packed_spmv_kernel one warp per slot of a lane-packed sparse matrix (rows of A for
//                     A x, rows of A^T -- the CSC copy -- for A^T y; layout in internal.h).
//                     Each lane sums its own rows in stored order with one FMA per stored
//                     nonzero: a GB300 SM issues 2 FP64 FMA lanes per clock and a warp FP64
//                     instruction holds its sub-partition's unit for 64 cycles whatever its
//                     active lanes, so no FP64 work runs lane-divergent.  The row results
//                     feed an epilogue:
//                       PrimalEpi  the primal step of Section 2.2 / Algorithm 1 step 1 and the
//                                  Halpern step of Appendix B.1 (K-A);
//                       DualEpi    the dual step of Section 2.2 / Algorithm 1 step 2 and the
//                                  Halpern step (K-B);
//                       StoreEpi   plain output (KKT products, power iteration, A x / A^T y).
//  finish_long_kernel rows longer than a lane: their pieces added in piece order, epilogue.
//  reduce_*_kernel    per-row / per-column terms of the relative KKT error (Appendix B.4)
//                     and of the fixed-point residual (Appendix D.2.1), block partials in a
//                     fixed order (deterministic, no floating-point atomics).
//  control_kernel     one block: final sums, KKT, restart test (Appendix B.2), PID primal
//                     weight (Appendix B.3), trace record, next Halpern weights, and the
//                     CUDA-graph loop condition.
//  apply_kernel       after a check: restart (anchor and iterate <- PDHG output) or the
//                     Halpern step of the check iteration.
//  fused_body_kernel, cluster_body_kernel
//                     a small LP's whole graph body (K iterations) in one launch of one
//                     block or of one thread-block cluster, from the same device code.
//  access_probe_kernel the packed kernels' memory accesses without their arithmetic (the
//                     roofline's access ceilings).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "../../include/dpdlp.h"
#include "internal.h"

namespace pdhg {

// ---------------------------------------------------------------- small device helpers
// Clamp written with comparisons so that a NaN input stays NaN (fmin/fmax would drop it
// and hide a diverged iterate from the non-finite check).
__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// The same clamp without FP64 instructions, for the iteration epilogues (GB300 issues about
// two FP64 operations per clock per SM, and the epilogues share that pipe with one FMA per
// stored nonzero).  Doubles compare as integers after mapping their bit patterns to keys
// that grow with the value (negative values: magnitude bits flipped).  A NaN input is
// returned unchanged, as clampd does; for any other input the result equals clampd's value
// (only the sign of a zero result may differ: -0 sorts below +0 here).
#ifndef DPDLP_INT_CLAMP
#define DPDLP_INT_CLAMP 1
#endif
__device__ __forceinline__ long long order_key(long long b) {
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double clampd_int(double v, double lo, double hi) {
#if DPDLP_INT_CLAMP
  const long long bv = __double_as_longlong(v);
  const long long kv = order_key(bv);
  if ((bv & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) return v;  // NaN
  return kv < order_key(__double_as_longlong(lo)) ? lo
                                                 : (kv > order_key(__double_as_longlong(hi)) ? hi : v);
#else
  return clampd(v, lo, hi);
#endif
}

__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Matrix values and indices are read once per pass and are larger than L2: stream them
// with an evict-first L2 policy so the gathered vectors (x_bar, y) stay L2-resident.
#ifndef DPDLP_STREAM_NOALLOC
#define DPDLP_STREAM_NOALLOC 0
#endif
#if DPDLP_STREAM_NOALLOC
#define DPDLP_LDS_L1 ".L1::no_allocate"
#else
#define DPDLP_LDS_L1 ""
#endif
__device__ __forceinline__ double2 ld_stream(const double2* p, unsigned long long pol) {
  double2 r;
  asm("ld.global.nc" DPDLP_LDS_L1 ".L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
      : "=d"(r.x), "=d"(r.y)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float4 ld_stream(const float4* p, unsigned long long pol) {
  float4 r;
  asm("ld.global.nc" DPDLP_LDS_L1 ".L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p, unsigned long long pol) {
  uint4 r;
  asm("ld.global.nc" DPDLP_LDS_L1 ".L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ int4 ld_stream(const int4* p, unsigned long long pol) {
  int4 r;
  asm("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(pol));
  return r;
}

// L2 priority hints for the per-row vectors (DPDLP_L2_HINTS, off: measured 3 % slower on the
// power-law LP): vectors that the next kernel
// gathers at random (x_bar, y) are written and gathered evict-last so they stay in L2;
// vectors only streamed once per launch are read and written evict-first.
#ifndef DPDLP_L2_HINTS
#define DPDLP_L2_HINTS 0
#endif
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ double ld_once(const double* p) {
#if DPDLP_L2_HINTS
  double r;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(l2_evict_first_policy()));
  return r;
#else
  return *p;
#endif
}
__device__ __forceinline__ void st_once(double* p, double v) {
#if DPDLP_L2_HINTS
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(l2_evict_first_policy()) : "memory");
#else
  *p = v;
#endif
}
__device__ __forceinline__ void st_keep(double* p, double v) {
#if DPDLP_L2_HINTS
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(l2_evict_last_policy()) : "memory");
#else
  *p = v;
#endif
}

// Deterministic block sum (fixed xor-butterfly inside warps, fixed order across warps).
// The result is valid in thread 0.  `buf` holds TPB/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* buf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) buf[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < TPB / 32 ? buf[l] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  An iteration kernel
// launched with the programmatic-serialization attribute may start while the kernel before
// it drains: its blocks load what no earlier kernel writes (slot descriptors, the first
// index batches), then pdl_wait() blocks until every earlier kernel has finished and its
// writes are visible.  Each block calls pdl_trigger() at its start, so the next kernel is
// released once all of this kernel's blocks are resident.  Launched without the attribute
// (plain products, the timing path) both instructions do nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

// Store v at shared-memory address p (a generic pointer into this CTA's shared memory) of
// every CTA 0 .. ncta-1 of the thread-block cluster, through distributed shared memory.
__device__ __forceinline__ void st_cluster_all(double* p, double v, unsigned ncta) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  for (unsigned c = 0; c < ncta; ++c) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(c));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(r), "d"(v) : "memory");
  }
}

// ---------------------------------------------------------------- epilogues
// An epilogue turns finished row sums into outputs: `apply_direct(row, sums)`.

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of the 128-byte lines that hold elements [r0, r0 + nr) of NA double arrays
// (256-byte aligned allocations), spread over the lanes of a warp.
template <int NA>
__device__ __forceinline__ void prefetch_rows(const double* const (&arr)[NA], int r0, int nr,
                                              int lane) {
  if (nr <= 0) return;
  const long long l0 = ((long long)r0 * 8) >> 7, l1 = ((long long)(r0 + nr) * 8 - 1) >> 7;
  const int nl = (int)(l1 - l0 + 1);
  for (int t = lane; t < NA * nl; t += LANES) {
    const int a = t / nl;
    const double* base = arr[0];
#pragma unroll
    for (int k = 1; k < NA; ++k)
      if (a == k) base = arr[k];
    prefetch_l2(reinterpret_cast<const char*>(base) + ((l0 + t - a * nl) << 7));
  }
}

struct StoreEpi1 {
  static constexpr bool kTunable = false;
  static constexpr bool kListable = true;
  double* out0;
  const InstScalars* itab;  // nullptr: every row; else rows of running instances only
  int listed;               // walk the active-slot list (batches)
  __device__ bool begin() { return true; }
  __device__ bool all_slots() const { return !listed; }
  __device__ bool inst(int i) { return !itab || itab[i].status == -1; }
  __device__ void prepare(int) {}
  __device__ void prefetch(int, int, int) {}
  __device__ bool fp32() const { return false; }  // KKT and step-size products: FP64 values
  __device__ void apply_direct(int r, const double* s) { out0[r] = s[0]; }
  __device__ void apply_rows(int r0, int nr, int lane, const double (*sr)[MAX_SLOT_ROWS]) {
    for (int r = lane; r < nr; r += LANES) {
      out0[r0 + r] = sr[0][r];
    }
  }
  struct Row {};
  __device__ Row load_row(int) const { return Row{}; }
  __device__ Row load_row_fixed(int) const { return Row{}; }
  __device__ void load_row_moving(int, Row&) const {}
  __device__ void apply_loaded(int r, const double* v, const Row&) { apply_direct(r, v); }
};
struct StoreEpi2 {
  static constexpr bool kTunable = false;
  static constexpr bool kListable = true;
  double *out0, *out1;
  const InstScalars* itab;
  int listed;
  __device__ bool begin() { return true; }
  __device__ bool all_slots() const { return !listed; }
  __device__ bool inst(int i) { return !itab || itab[i].status == -1; }
  __device__ void prepare(int) {}
  __device__ void prefetch(int, int, int) {}
  __device__ bool fp32() const { return false; }
  __device__ void apply_direct(int r, const double* s) {
    out0[r] = s[0];
    out1[r] = s[1];
  }
  __device__ void apply_rows(int r0, int nr, int lane, const double (*sr)[MAX_SLOT_ROWS]) {
    for (int r = lane; r < nr; r += LANES) {
      out0[r0 + r] = sr[0][r];
      out1[r0 + r] = sr[1][r];
    }
  }
  struct Row {};
  __device__ Row load_row(int) const { return Row{}; }
  __device__ Row load_row_fixed(int) const { return Row{}; }
  __device__ void load_row_moving(int, Row&) const {}
  __device__ void apply_loaded(int r, const double* v, const Row&) { apply_direct(r, v); }
};

// Per-iteration scalars read from device memory by the fused epilogues: the global part
// (iteration limit, check iteration) once per launch, the instance part once per slot.
struct IterScalars {
  double step, inv_step, two_step, w1, w0, gamma;
  int check, halpern, gamma_one, fp32;
};

__device__ __forceinline__ bool load_global(const DevScalars* sc, IterPlan p, IterScalars& o) {
  if (p.force_regular) {
    o.check = 0;
  } else {
    const long long T = sc->T_base + p.i;
    if (T >= sc->max_iter) return false;  // past the iteration limit inside this body
    o.check = (T + 1 == sc->T_check);
  }
  o.gamma = sc->gamma;
  o.halpern = sc->halpern;
  o.gamma_one = (sc->gamma == 1.0);
  return true;
}

// Instance part, in two steps for a batch: whether the instance still runs and which
// values its products use (before the lane sums), then its step sizes and Halpern weights
// (after them, so they are not held in registers across the sums).
__device__ __forceinline__ bool load_inst_mode(const InstScalars* tab, int inst, IterPlan p,
                                               IterScalars& o) {
  const InstScalars& I = tab[inst];
  if (p.idle) return false;                                // timing an idle launch
  if (I.status != -1 && !p.force_regular) return false;  // converged instance: skip its rows
  o.fp32 = I.spmv_fp32;
  return true;
}

__device__ __forceinline__ void load_inst_steps(const InstScalars* tab, const double* wtab,
                                                int inst, IterPlan p, bool primal,
                                                IterScalars& o) {
  const InstScalars& I = tab[inst];
  o.step = primal ? I.tau : I.sigma;
  o.inv_step = I.inv_sigma;
  o.two_step = 2.0 * o.step;
  o.w1 = wtab[(size_t)inst * 2 * KMAX + p.i];
  o.w0 = wtab[(size_t)inst * 2 * KMAX + KMAX + p.i];
}

// Primal step per column j, given s = (A^T y)_j:
//   x^ = proj_X(x - tau (c - s)),  x_bar = 2 x^ - x,
//   Halpern: x <- w1 ((1+gamma) x^ - gamma x) + w0 x0   (with gamma = 1 the reflected point
//   is x_bar itself), regular iterations;
//   check iteration: keep x = x^k, store x^ and dx = x^k - x^.
// Bcast: x_bar is a shared-memory vector copied in every CTA of a cluster (the cluster
// form of the fused body); each new x_bar_j is stored into all ncta copies.
template <bool Single, bool QP = false, bool Bcast = false>
struct PrimalEpi {
  static constexpr bool kTunable = true;
  static constexpr bool kListable = !Single;  // one LP never uses the active-slot list
  const DevScalars* sc;
  const InstScalars* itab;
  const double* wtab;
  IterPlan plan;
  int listed;  // batches: walk the active-slot list (all slots when timing)
  const double *c, *lv, *uv, *x0;
  double *x, *xbar, *xh, *dx;
  const double* qd;  // diagonal of Q of a diagonal QP (nullptr: an LP)
  IterScalars q;
  unsigned ncta = 0;  // Bcast: CTAs of the cluster
  // Single: one instance, whose scalars are loaded once per launch in begin()
  __device__ bool begin() {
    if (!Single) return load_global(sc, plan, q);
    // all loads issued before the first branch, so they overlap
    const int st = itab[0].status;
    q.fp32 = itab[0].spmv_fp32;
    load_inst_steps(itab, wtab, 0, plan, true, q);
    const bool go = load_global(sc, plan, q);
    return go && (st == -1 || plan.force_regular);
  }
  __device__ bool inst(int i) { return Single || load_inst_mode(itab, i, plan, q); }
  __device__ bool all_slots() const { return !listed || plan.force_regular; }
  __device__ void prepare(int i) {
    if (!Single) load_inst_steps(itab, wtab, i, plan, true, q);
  }
  __device__ void prefetch(int r0, int nr, int lane) {
    const double* const a[5] = {c, lv, uv, x, x0};
    prefetch_rows<5>(a, r0, nr, lane);
  }
  __device__ bool fp32() const { return q.fp32 != 0; }
  // anchor value x0_j is read only when used (Halpern, not a check iteration)
  __device__ bool need_anchor() const { return q.halpern && !q.check; }
  __device__ void step(int j, double s, double cj, double lvj, double uvj, double xj,
                       double x0j) {
    double t = fma(-q.step, cj - s, xj);
    // diagonal QP: the minimum of 1/2 Q_jj x^2 + (c_j - s) x + (x - x_j)^2 / (2 tau) over the
    // box is the clamped x = (x_j - tau (c_j - s)) / (1 + tau Q_jj)  (Eq. primal_update)
    if constexpr (QP) t = t / fma(q.step, ld_once(qd + j), 1.0);
    const double xhj = clampd_int(t, lvj, uvj);
    const double xb = fma(2.0, xhj, -xj);
    if constexpr (Bcast) st_cluster_all(xbar + j, xb, ncta);
    else st_keep(xbar + j, xb);
    if (q.check) {
      xh[j] = xhj;
      dx[j] = xj - xhj;
    } else if (q.halpern) {
      const double r = q.gamma_one ? xb : fma(1.0 + q.gamma, xhj, -q.gamma * xj);
      st_once(x + j, fma(q.w1, r, q.w0 * x0j));
    } else {
      x[j] = xhj;
    }
  }
  __device__ void apply_direct(int j, const double* s) {
    step(j, s[0], ld_once(c + j), ld_once(lv + j), ld_once(uv + j), ld_once(x + j),
         need_anchor() ? ld_once(x0 + j) : 0.0);
  }
  // the row's inputs loaded ahead of its product (long-row pass), then the step
  struct Row {
    double a[5];
  };
  __device__ Row load_row(int j) const {
    Row r = load_row_fixed(j);
    load_row_moving(j, r);
    return r;
  }
  // the inputs no kernel of a graph body writes (the anchor changes only at checks), and the
  // one the iterations do (x)
  __device__ Row load_row_fixed(int j) const {
    Row r;
    r.a[0] = ld_once(c + j);
    r.a[1] = ld_once(lv + j);
    r.a[2] = ld_once(uv + j);
    r.a[3] = 0.0;
    r.a[4] = need_anchor() ? ld_once(x0 + j) : 0.0;
    return r;
  }
  __device__ void load_row_moving(int j, Row& r) const { r.a[3] = ld_once(x + j); }
  __device__ void apply_loaded(int j, const double* s, const Row& r) {
    step(j, s[0], r.a[0], r.a[1], r.a[2], r.a[3], r.a[4]);
  }
  // Epilogue of a slot's rows r0 + r (r = lane + 32 k < nr): every load first, then the
  // updates, so the loads of all rows are in flight together.
  __device__ void apply_rows(int r0, int nr, int lane, const double (*sr)[MAX_SLOT_ROWS]) {
    constexpr int R = MAX_SLOT_ROWS / LANES;
    double cj[R], lj[R], uj[R], xj[R], aj[R];
    const bool na = need_anchor();
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < nr) {
        const int j = r0 + r;
        cj[k] = ld_once(c + j);
        lj[k] = ld_once(lv + j);
        uj[k] = ld_once(uv + j);
        xj[k] = ld_once(x + j);
        aj[k] = na ? ld_once(x0 + j) : 0.0;
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < nr) step(r0 + r, sr[0][r], cj[k], lj[k], uj[k], xj[k], aj[k]);
    }
  }
  // The fused bodies' epilogue: the slot's row inputs from the block's shared copy (field f of
  // row r at rc[f * fs + r]: c, lv, uv, x0, x, and for a QP the diagonal of Q), the updates
  // to the global rows r0 + r with step()'s arithmetic; a regular iteration's new x also goes
  // to the copy, which the next iteration reads.
  __device__ void apply_rows_copied(int r0, int nr, int lane, const double (*sr)[MAX_SLOT_ROWS],
                                    double* rc, int fs) {
    constexpr int R = MAX_SLOT_ROWS / LANES;
    const bool na = need_anchor();
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < nr) {
        const int j = r0 + r;
        const double xj = rc[4 * fs + r], x0j = na ? rc[3 * fs + r] : 0.0;
        double t = fma(-q.step, rc[r] - sr[0][r], xj);
        if constexpr (QP) t = t / fma(q.step, rc[5 * fs + r], 1.0);
        const double xhj = clampd_int(t, rc[fs + r], rc[2 * fs + r]);
        const double xb = fma(2.0, xhj, -xj);
        if constexpr (Bcast) st_cluster_all(xbar + j, xb, ncta);
        else st_keep(xbar + j, xb);
        if (q.check) {
          xh[j] = xhj;
          dx[j] = xj - xhj;
        } else {
          double xn = xhj;
          if (q.halpern) {
            const double rr = q.gamma_one ? xb : fma(1.0 + q.gamma, xhj, -q.gamma * xj);
            xn = fma(q.w1, rr, q.w0 * x0j);
          }
          st_once(x + j, xn);
          rc[4 * fs + r] = xn;
        }
      }
    }
  }
};

// Dual step per row i, given z = (A x_bar)_i:
//   w = y / sigma - z,  d = w - proj_{-S}(w),  y^ = sigma d,  -S_i = [lo_i, hi_i] = [-uc_i, -lc_i];
//   Halpern: y <- w1 ((1+gamma) y^ - gamma y) + w0 y0, with gamma = 1 evaluated as
//   w1 (2 sigma d - y) + w0 y0; check iteration: keep y = y^k, store y^.
// Mirror: 1 = every new y_i is also written to the shared copy ys (the fused body), 2 = to
// the shared copy ys of every CTA of a cluster (the cluster form of the fused body).
template <bool Single, int Mirror = 0>
struct DualEpi {
  static constexpr bool kTunable = true;
  static constexpr bool kListable = !Single;  // one LP never uses the active-slot list
  const DevScalars* sc;
  const InstScalars* itab;
  const double* wtab;
  IterPlan plan;
  int listed;  // batches: walk the active-slot list (all slots when timing)
  const double *lo, *hi, *y0;
  double *y, *yh;
  IterScalars q;
  double* ys;  // Mirror: the shared copy of y
  unsigned ncta = 0;  // Mirror 2: CTAs of the cluster
  // Single: one instance, whose scalars are loaded once per launch in begin()
  __device__ bool begin() {
    if (!Single) return load_global(sc, plan, q);
    // all loads issued before the first branch, so they overlap
    const int st = itab[0].status;
    q.fp32 = itab[0].spmv_fp32;
    load_inst_steps(itab, wtab, 0, plan, false, q);
    const bool go = load_global(sc, plan, q);
    return go && (st == -1 || plan.force_regular);
  }
  __device__ bool inst(int i) { return Single || load_inst_mode(itab, i, plan, q); }
  __device__ bool all_slots() const { return !listed || plan.force_regular; }
  __device__ void prepare(int i) {
    if (!Single) load_inst_steps(itab, wtab, i, plan, false, q);
  }
  __device__ void prefetch(int r0, int nr, int lane) {
    const double* const a[4] = {lo, hi, y, y0};
    prefetch_rows<4>(a, r0, nr, lane);
  }
  __device__ bool fp32() const { return q.fp32 != 0; }
  __device__ bool need_anchor() const { return q.halpern && !q.check; }
  __device__ void step(int i, double s, double loi, double hii, double yi, double y0i) {
    const double w = fma(yi, q.inv_step, -s);
    const double d = w - clampd_int(w, loi, hii);
    if (q.check) {
      yh[i] = q.step * d;
    } else if (q.halpern) {
      double r;
      if (q.gamma_one) {
        r = fma(q.two_step, d, -yi);
      } else {
        r = fma(1.0 + q.gamma, q.step * d, -q.gamma * yi);
      }
      const double yn = fma(q.w1, r, q.w0 * y0i);
      st_keep(y + i, yn);
      mirror(i, yn);
    } else {
      st_keep(y + i, q.step * d);
      mirror(i, q.step * d);
    }
  }
  __device__ void mirror(int i, double v) {
    if constexpr (Mirror == 1) ys[i] = v;
    if constexpr (Mirror == 2) st_cluster_all(ys + i, v, ncta);
  }
  __device__ void apply_direct(int i, const double* s) {
    step(i, s[0], ld_once(lo + i), ld_once(hi + i), ld_once(y + i),
         need_anchor() ? ld_once(y0 + i) : 0.0);
  }
  struct Row {
    double a[4];
  };
  __device__ Row load_row(int i) const {
    Row r = load_row_fixed(i);
    load_row_moving(i, r);
    return r;
  }
  __device__ Row load_row_fixed(int i) const {
    Row r;
    r.a[0] = ld_once(lo + i);
    r.a[1] = ld_once(hi + i);
    r.a[2] = 0.0;
    r.a[3] = need_anchor() ? ld_once(y0 + i) : 0.0;
    return r;
  }
  __device__ void load_row_moving(int i, Row& r) const { r.a[2] = ld_once(y + i); }
  __device__ void apply_loaded(int i, const double* s, const Row& r) {
    step(i, s[0], r.a[0], r.a[1], r.a[2], r.a[3]);
  }
  __device__ void apply_rows(int r0, int nr, int lane, const double (*sr)[MAX_SLOT_ROWS]) {
    constexpr int R = MAX_SLOT_ROWS / LANES;
    double lj[R], hj[R], yj[R], aj[R];
    const bool na = need_anchor();
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < nr) {
        const int i = r0 + r;
        lj[k] = ld_once(lo + i);
        hj[k] = ld_once(hi + i);
        yj[k] = ld_once(y + i);
        aj[k] = na ? ld_once(y0 + i) : 0.0;
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < nr) step(r0 + r, sr[0][r], lj[k], hj[k], yj[k], aj[k]);
    }
  }
  // The fused bodies' epilogue: the slot's row inputs from the block's shared copy (lo, hi,
  // y0 at rc[f * fs + r]) and y from the shared mirror ys, then step().
  __device__ void apply_rows_copied(int r0, int nr, int lane, const double (*sr)[MAX_SLOT_ROWS],
                                    double* rc, int fs) {
    static_assert(Mirror >= 1, "y is read from the shared mirror");
    constexpr int R = MAX_SLOT_ROWS / LANES;
    const bool na = need_anchor();
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < nr)
        step(r0 + r, sr[0][r], rc[r], rc[fs + r], ys[r0 + r], na ? rc[2 * fs + r] : 0.0);
    }
  }
};

// ---------------------------------------------------------------- packed SpMV
// Build-time tuning knobs (defaults are the measured best; see the profiles):
//   DPDLP_PK_MIN_BLOCKS  resident blocks per SM the register allocation targets
//   DPDLP_GATHER_NOALLOC gather x[col] without allocating in L1 (random, no reuse there)
//   DPDLP_PK_BATCH       stored entries per pipeline stage of a lane (4 or 8)
//   DPDLP_STREAM_NOALLOC stream matrix values and indices without allocating in L1
#ifndef DPDLP_PK_MIN_BLOCKS
#define DPDLP_PK_MIN_BLOCKS 8
#endif
#ifndef DPDLP_GATHER_NOALLOC
#define DPDLP_GATHER_NOALLOC 0
#endif
#ifndef DPDLP_PK_BATCH
#define DPDLP_PK_BATCH 4
#endif
#ifndef DPDLP_STREAM_NOALLOC
#define DPDLP_STREAM_NOALLOC 0
#endif
//   DPDLP_HOIST_SLOT     load the slot descriptor before the launch scalars are checked
//   DPDLP_EPI_PREFETCH   prefetch the slot rows' epilogue vectors into L2 at slot start
#ifndef DPDLP_HOIST_SLOT
#define DPDLP_HOIST_SLOT 1
#endif
#ifndef DPDLP_EPI_PREFETCH
#define DPDLP_EPI_PREFETCH 0
#endif
//   DPDLP_HOIST_IDX      issue the first two index batches at kernel entry
//   DPDLP_EPI_BATCH      epilogue loads of all of a lane's rows before any update
#ifndef DPDLP_HOIST_IDX
#define DPDLP_HOIST_IDX 0
#endif
static_assert(LANE_ITEMS % DPDLP_PK_BATCH == 0 && LANE_ITEMS / DPDLP_PK_BATCH >= 2,
              "a lane holds at least two pipeline batches (both are loaded before the sums)");
static_assert(DPDLP_PK_BATCH % 4 == 0,
              "indices (and FP32 values) of a batch are read four at a time with 16-byte loads");
#ifndef DPDLP_EPI_BATCH
#define DPDLP_EPI_BATCH 1
#endif


template <int NV>
struct GatherVecs {
  const double* x[NV];
};

// Coh: the gathered vector is written earlier in the same launch (fused small-LP body), so
// it is read with a coherent load instead of the read-only path.
template <bool Coh = false>
__device__ __forceinline__ double gather(const double* p) {
  if constexpr (Coh) return *p;
#if DPDLP_L2_HINTS && !DPDLP_GATHER_NOALLOC
  double r;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(l2_evict_last_policy()));
  return r;
#elif DPDLP_GATHER_NOALLOC
  double r;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(r) : "l"(p));
  return r;
#else
  return __ldg(p);
#endif
}

// Values and indices of batch b (positions B*b .. B*b+B-1) of this lane: 16-byte loads,
// each covering 512 contiguous bytes across the warp.  FP64 values are stored in pairs per
// lane, FP32 values and indices in fours.  Gen: plain (generic) loads, for a copy of the
// slot in shared memory; otherwise streaming global loads with the given L2 policy.
template <typename V>
struct Vals;
template <>
struct Vals<double> {
  using vec = double2;
  static __device__ __forceinline__ const double2* base(const DevPacked& M, size_t off, int lane) {
    return reinterpret_cast<const double2*>(M.val + off) + lane;
  }
  template <int B, bool Gen = false>
  static __device__ __forceinline__ void load(const double2* vp, int b, double (&v)[B],
                                              unsigned long long pol) {
#pragma unroll
    for (int q = 0; q < B / 2; ++q) {
      const double2* a = vp + ((B / 2) * b + q) * LANES;
      const double2 d = Gen ? *a : ld_stream(a, pol);
      v[2 * q] = d.x;
      v[2 * q + 1] = d.y;
    }
  }
  static __device__ __forceinline__ double widen(double v) { return v; }
};
template <>
struct Vals<float> {
  using vec = float4;
  static __device__ __forceinline__ const float4* base(const DevPacked& M, size_t off, int lane) {
    return reinterpret_cast<const float4*>(M.val32 + off) + lane;
  }
  template <int B, bool Gen = false>
  static __device__ __forceinline__ void load(const float4* vp, int b, float (&v)[B],
                                              unsigned long long pol) {
#pragma unroll
    for (int q = 0; q < B / 4; ++q) {
      const float4* a = vp + ((B / 4) * b + q) * LANES;
      const float4 d = Gen ? *a : ld_stream(a, pol);
      v[4 * q] = d.x;
      v[4 * q + 1] = d.y;
      v[4 * q + 2] = d.z;
      v[4 * q + 3] = d.w;
    }
  }
  // Exact float -> double for normal floats and zero (the only values the packing stores
  // in FP32 mode), with integer operations: rebias the exponent (+896) and shift the
  // fraction into place.  Keeps the conversion off the FP64 unit.
  static __device__ __forceinline__ double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned long long mag = b & 0x7fffffffu;
    const unsigned long long d = mag ? ((mag + (896ull << 23)) << 29) : 0ull;
    return __longlong_as_double((long long)(d | ((unsigned long long)(b & 0x80000000u) << 32)));
  }
};

template <int B, bool Gen = false>
__device__ __forceinline__ void load_idx(const uint4* ip, int b, uint32_t (&c)[B],
                                         unsigned long long pol) {
#pragma unroll
  for (int q = 0; q < B / 4; ++q) {
    const uint4* a = ip + ((B / 4) * b + q) * LANES;
    const uint4 d = Gen ? *a : ld_stream(a, pol);
    c[4 * q] = d.x;
    c[4 * q + 1] = d.y;
    c[4 * q + 2] = d.z;
    c[4 * q + 3] = d.w;
  }
}

// The 32 stored nonzeros of one lane, summed in order with one FMA each (products formed
// in FP64 from values of type V); at every end flag the finished sum goes to the slot's row
// sums (short rows) or to the piece array (long-row pieces).  Three-stage pipeline of
// batches: indices two batches ahead, values and the x[col] gathers one batch ahead, so
// gathers are in flight while the FMA chain runs.  Gen: the slot's values and indices are a
// copy in shared memory (M.val / M.idx point there).
template <typename V, int NV, int B, bool Coh = false, bool Gen = false>
__device__ __forceinline__ void lane_sums(const DevPacked& M, const GatherVecs<NV>& g, size_t off,
                                          int lane, int rl, int pid,
                                          double (*srow)[MAX_SLOT_ROWS], const uint4* ip,
                                          unsigned long long pol, uint32_t (&c0)[B],
                                          uint32_t (&c1)[B]) {
  constexpr int NB = LANE_ITEMS / B;
  const auto* vp = Vals<V>::base(M, off, lane);
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  V v0[B];
  double x0v[NV][B];
  Vals<V>::template load<B, Gen>(vp, 0, v0, pol);
#pragma unroll
  for (int j = 0; j < B; ++j) {
#pragma unroll
    for (int k = 0; k < NV; ++k) x0v[k][j] = gather<Coh>(g.x[k] + (c0[j] & IDX_MASK));
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    uint32_t c2[B];
    V v1[B];
    double x1v[NV][B];
    if (b + 2 < NB) load_idx<B, Gen>(ip, b + 2, c2, pol);
    if (b + 1 < NB) {
      Vals<V>::template load<B, Gen>(vp, b + 1, v1, pol);
#pragma unroll
      for (int j = 0; j < B; ++j) {
#pragma unroll
        for (int k = 0; k < NV; ++k) x1v[k][j] = gather<Coh>(g.x[k] + (c1[j] & IDX_MASK));
      }
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const double a = Vals<V>::widen(v0[j]);
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = fma(a, x0v[k][j], acc[k]);
      if (c0[j] & END_BIT) {
        if (c0[j] & PIECE_BIT) {
#pragma unroll
          for (int k = 0; k < NV; ++k) M.piece_sum[(size_t)k * M.npieces + pid] = acc[k];
          ++pid;
        } else {
#pragma unroll
          for (int k = 0; k < NV; ++k) srow[k][rl] = acc[k];
          ++rl;
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
      }
    }
    if (b + 1 < NB) {  // rotate the pipeline
#pragma unroll
      for (int j = 0; j < B; ++j) {
        c0[j] = c1[j];
        v0[j] = v1[j];
#pragma unroll
        for (int k = 0; k < NV; ++k) x0v[k][j] = x1v[k][j];
        if (b + 2 < NB) c1[j] = c2[j];
      }
    }
  }
}

// Whether this launch times an idle iteration (no instance running).
template <class Epi>
__device__ __forceinline__ bool idle_launch(const Epi& epi) {
  if constexpr (Epi::kTunable) return epi.plan.idle != 0;
  return false;
}

// Whether this launch is an iteration kernel launched as a programmatic dependent.
template <class Epi>
__device__ __forceinline__ bool launched_dependent(const Epi& epi) {
  if constexpr (Epi::kTunable) return epi.plan.pdl != 0;
  return false;
}

// One warp per slot, PK_WARPS slots per block, no block-level barrier: the lanes sum their
// rows (lane_sums), then apply the epilogue to the slot's short rows, one row per lane.
// W slots (warps) per block; the register cap keeps the same number of resident warps per
// SM for every W (W * min-blocks = PK_WARPS * DPDLP_PK_MIN_BLOCKS).
template <int NV, int W, class Epi>
__global__ void __launch_bounds__(W * LANES, (DPDLP_PK_MIN_BLOCKS * PK_WARPS) / W)
    packed_spmv_kernel(DevPacked M, GatherVecs<NV> g, Epi epi_in) {
  __shared__ double srow[W][NV][MAX_SLOT_ROWS];
  Epi epi = epi_in;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * W + w;
  constexpr int B = DPDLP_PK_BATCH;
  const size_t off = (size_t)s * SLOT_ITEMS;
  const uint4* ip = reinterpret_cast<const uint4*>(M.idx + off) + lane;
  const unsigned long long pol = l2_evict_first_policy();
  uint32_t c0[B], c1[B];
  // with programmatic dependent launch the first index batches (which no kernel writes)
  // load before the wait, while the previous kernel drains
  const bool early_idx = DPDLP_HOIST_IDX || launched_dependent(epi);
  if (early_idx && s < M.nslots) {
    load_idx<B>(ip, 0, c0, pol);
    load_idx<B>(ip, 1, c1, pol);
  }
#if DPDLP_HOIST_SLOT
  // the slot's descriptors are loaded while the launch scalars are in flight
  SlotDesc sd{0, 0, 0, 0};
  LaneMeta lm{0, 0};
  if (s < M.nslots) {
    sd = M.slots[s];
    lm = M.lanes[(size_t)s * LANES + lane];
  }
  pdl_trigger();
  pdl_wait();
  if (!epi.begin()) return;   // uniform over the launch
  if (s >= M.nslots) return;  // uniform over the warp
#else
  pdl_trigger();
  pdl_wait();
  if (!epi.begin()) return;
  if (s >= M.nslots) return;
  const SlotDesc sd = M.slots[s];
  const LaneMeta lm = M.lanes[(size_t)s * LANES + lane];
#endif
  if (!epi.inst(sd.inst)) return;  // uniform over the warp: instance scalars, or converged
#if DPDLP_EPI_PREFETCH
  epi.prefetch(sd.row_base, sd.nrows, lane);
#endif
  if (!early_idx) {
    load_idx<B>(ip, 0, c0, pol);
    load_idx<B>(ip, 1, c1, pol);
  }
  if (epi.fp32() && M.val32)  // uniform over the warp
    lane_sums<float, NV, B>(M, g, off, lane, lm.row_local, lm.piece_base, srow[w], ip, pol, c0, c1);
  else
    lane_sums<double, NV, B>(M, g, off, lane, lm.row_local, lm.piece_base, srow[w], ip, pol, c0, c1);
  __syncwarp();
  epi.prepare(sd.inst);
#if DPDLP_EPI_BATCH
  epi.apply_rows(sd.row_base, sd.nrows, lane, srow[w]);
#else
  for (int r = lane; r < sd.nrows; r += LANES) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = srow[w][k][r];
    epi.apply_direct(sd.row_base + r, v);
  }
#endif
}

// Sum of piece sums k = q, q + step, q + 2 step, ... < q1 of vector `v`, added in that order.
// The piece ids and then the sums are loaded PIECE_BATCH at a time before they are added,
// so a row's loads overlap instead of forming a chain of dependent round trips; the order
// of the additions is that of the plain loop.
// L2: read the sums from L2 (ld.global.cg), for sums another SM of the cluster wrote.
constexpr int PIECE_BATCH = 8;
// Piece ids of the batch starting at q (q, q + step, ...; -1 past q1).
__device__ __forceinline__ void piece_ids(const DevPacked& M, int q, int q1, int step,
                                          int (&pid)[PIECE_BATCH]) {
#pragma unroll
  for (int u = 0; u < PIECE_BATCH; ++u) {
    const int qq = q + u * step;
    pid[u] = qq < q1 ? M.long_piece[qq] : -1;
  }
}
// The same sum with the first batch's ids already loaded (`first`, from piece_ids(q)).
template <bool L2 = false>
__device__ __forceinline__ double strided_piece_sum_from(const DevPacked& M, int k, int q, int q1,
                                                         int step, const int (&first)[PIECE_BATCH]) {
  const double* ps = M.piece_sum + (size_t)k * M.npieces;
  double a = 0.0;
  int pid[PIECE_BATCH];
#pragma unroll
  for (int u = 0; u < PIECE_BATCH; ++u) pid[u] = first[u];
  for (; q < q1; q += PIECE_BATCH * step) {
    double v[PIECE_BATCH];
#pragma unroll
    for (int u = 0; u < PIECE_BATCH; ++u)
      v[u] = pid[u] >= 0 ? (L2 ? __ldcg(ps + pid[u]) : ps[pid[u]]) : 0.0;
    const int qn = q + PIECE_BATCH * step;
    if (qn < q1) piece_ids(M, qn, q1, step, pid);  // the next batch's ids during these loads
#pragma unroll
    for (int u = 0; u < PIECE_BATCH; ++u)
      if (q + u * step < q1) a += v[u];  // the batch's pieces in order (pid is the next batch's)
  }
  return a;
}
template <bool L2 = false>
__device__ __forceinline__ double strided_piece_sum(const DevPacked& M, int k, int q, int q1,
                                                    int step) {
  int first[PIECE_BATCH];
  piece_ids(M, q, q1, step, first);
  return strided_piece_sum_from<L2>(M, k, q, q1, step, first);
}

// Long rows: add each row's pieces, then its epilogue.  Rows come longest first: the first
// nlong_block rows get a thread block each, the next nlong_warp rows a warp each (fixed
// strided sums and fixed reduction trees), the rest a thread each (pieces in order).
// Resident blocks per SM the register allocation targets: on the power-law LP the pass's
// ~880 blocks fit one wave from 6 blocks per SM (at most 40 registers; 56 without the
// bound, 4 blocks per SM: 1.44 waves).  Measured on one GB300, the pass added to the dual
// slot kernel: 13.7 us at 6 blocks per SM, 13.2-13.7 at 4, 16.4 at 8 (32 registers, spills):
// its cost is its dependent loads and its launch, not waves.
#ifndef DPDLP_LONG_MIN_BLOCKS
#define DPDLP_LONG_MIN_BLOCKS 6
#endif
// DPDLP_LONG_PDL  launch the pass as a programmatic dependent of the slot kernel (measured:
// 13.7 us per pass with, 16.2 without)
#ifndef DPDLP_LONG_PDL
#define DPDLP_LONG_PDL 1
#endif
template <int NV, class Epi>
__global__ void __launch_bounds__(TPB, DPDLP_LONG_MIN_BLOCKS) finish_long_kernel(DevPacked M, Epi epi_in) {
  __shared__ double red[TPB / 32];
  Epi epi = epi_in;
  pdl_trigger();
  // Before waiting for the kernel that wrote the pieces, load what no kernel of a graph body
  // writes: the scalars and the anchor (checks only), the rows' indices, piece ranges, first
  // piece ids and fixed step inputs.  The row's iterate (x or y, written by the previous
  // iteration's pass, which with programmatic launches may still be running) and the piece
  // sums load after the wait.
  const bool go = epi.begin();  // uniform over the launch
  const int nb = M.nlong_block, nw = M.nlong_warp;
  const int wblocks = (nw + TPB / 32 - 1) / (TPB / 32);
  int b = blockIdx.x;
  double v[NV];
  int first[PIECE_BATCH];
  if (b < nb) {
    const int i = b;
    const bool act = go && epi.inst(M.long_inst[i]);  // uniform over the block
    const int row = M.long_row[i];
    const int q0 = M.long_ptr[i], q1 = M.long_ptr[i + 1];
    piece_ids(M, q0 + threadIdx.x, q1, TPB, first);
    typename Epi::Row in{};
    if (act && threadIdx.x == 0) in = epi.load_row_fixed(row);
    pdl_wait();  // the pieces come from the kernel before
    if (!act) return;
    if (threadIdx.x == 0) epi.load_row_moving(row, in);  // in flight during the sums
#pragma unroll
    for (int k = 0; k < NV; ++k)
      v[k] = block_sum(strided_piece_sum_from(M, k, q0 + threadIdx.x, q1, TPB, first), red);
    if (threadIdx.x == 0) {
      epi.prepare(M.long_inst[i]);
      epi.apply_loaded(row, v, in);
    }
    return;
  }
  b -= nb;
  if (b < wblocks) {
    const int i = nb + b * (TPB / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nb + nw) {
      pdl_wait();
      return;
    }
    const bool act = go && epi.inst(M.long_inst[i]);  // uniform over the warp
    const int row = M.long_row[i];
    const int q0 = M.long_ptr[i], q1 = M.long_ptr[i + 1];
    piece_ids(M, q0 + lane, q1, LANES, first);
    typename Epi::Row in{};
    if (act && lane == 0) in = epi.load_row_fixed(row);
    pdl_wait();
    if (!act) return;
    if (lane == 0) epi.load_row_moving(row, in);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = strided_piece_sum_from(M, k, q0 + lane, q1, LANES, first);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      v[k] = a;
    }
    if (lane == 0) {
      epi.prepare(M.long_inst[i]);
      epi.apply_loaded(row, v, in);
    }
    return;
  }
  b -= wblocks;
  const int i = nb + nw + b * TPB + threadIdx.x;
  if (i >= M.nlong) {
    pdl_wait();
    return;
  }
  const bool act = go && epi.inst(M.long_inst[i]);
  const int row = M.long_row[i];
  const int q0 = M.long_ptr[i], q1 = M.long_ptr[i + 1];
  piece_ids(M, q0, q1, 1, first);
  typename Epi::Row in{};
  if (act) in = epi.load_row_fixed(row);
  pdl_wait();
  if (!act) return;
  epi.load_row_moving(row, in);
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = strided_piece_sum_from(M, k, q0, q1, 1, first);
  epi.prepare(M.long_inst[i]);
  epi.apply_loaded(row, v, in);
}

// Batches: a persistent form of the same slot computation.  One wave of resident blocks
// walks the list of slots of running instances (rebuilt at every check), so once most
// instances have converged an iteration costs what the running ones need, not a launch
// over every slot of the batch.  all_slots() (timing, plain products) walks every slot.
// The persistent loop needs more registers than one slot per warp: 6 resident blocks (80
// registers) measured faster than 8 (64 registers, spills).
#ifndef DPDLP_LIST_MIN_BLOCKS
#define DPDLP_LIST_MIN_BLOCKS 6
#endif
#ifndef DPDLP_LIST_PERSISTENT
#define DPDLP_LIST_PERSISTENT 1
#endif
template <int NV, int W, class Epi>
__global__ void __launch_bounds__(W * LANES, (DPDLP_LIST_MIN_BLOCKS * PK_WARPS) / W)
    packed_list_kernel(DevPacked M, GatherVecs<NV> g, Epi epi_in) {
  __shared__ double srow[W][NV][MAX_SLOT_ROWS];
  Epi epi = epi_in;
  pdl_trigger();
  pdl_wait();  // the slot list and scalars come from the kernels before
  if (!epi.begin()) return;  // uniform over the launch
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = idle_launch(epi) ? 0 : epi.all_slots() ? M.nslots : *M.nactive;
  // with every instance running the list is the identity (instances keep their order and
  // own consecutive slots): no indirection then
  const bool all = total == M.nslots;
  constexpr int B = DPDLP_PK_BATCH;
  const unsigned long long pol = l2_evict_first_policy();
  for (int k = blockIdx.x * W + w; k < total; k += gridDim.x * W) {  // uniform over the warp
    const int s = all ? k : M.active[k];
    const SlotDesc sd = M.slots[s];
    const LaneMeta lm = M.lanes[(size_t)s * LANES + lane];
    if (!epi.inst(sd.inst)) continue;
    const size_t off = (size_t)s * SLOT_ITEMS;
    const uint4* ip = reinterpret_cast<const uint4*>(M.idx + off) + lane;
    uint32_t c0[B], c1[B];
    load_idx<B>(ip, 0, c0, pol);
    load_idx<B>(ip, 1, c1, pol);
    if (epi.fp32() && M.val32)
      lane_sums<float, NV, B>(M, g, off, lane, lm.row_local, lm.piece_base, srow[w], ip, pol, c0, c1);
    else
      lane_sums<double, NV, B>(M, g, off, lane, lm.row_local, lm.piece_base, srow[w], ip, pol, c0, c1);
    __syncwarp();
    epi.prepare(sd.inst);
    epi.apply_rows(sd.row_base, sd.nrows, lane, srow[w]);
    __syncwarp();  // the warp's row sums are read before its next slot writes them
  }
}

static int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

#ifndef DPDLP_BATCH_LIST
#define DPDLP_BATCH_LIST 1
#endif

// A launch, as a programmatic dependent of the previous work in the stream when `pdl`.
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s,
                            bool pdl, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class Epi>
static bool pdl_of(const Epi& epi) {
  if constexpr (Epi::kTunable) return epi.plan.pdl != 0;
  return false;
}
template <class Epi>
static bool slots_only_of(const Epi& epi) {
  if constexpr (Epi::kTunable) return epi.plan.slots_only != 0;
  return false;
}

template <int NV, int W, class Epi>
static cudaError_t launch_slots(const DevPacked& M, GatherVecs<NV> g, Epi epi, cudaStream_t s) {
  const bool pdl = pdl_of(epi);
  if constexpr (Epi::kListable && DPDLP_BATCH_LIST) {
    if (M.active && epi.listed) {
      const int most = (DPDLP_LIST_MIN_BLOCKS * PK_WARPS) / W;  // resident blocks per SM
      const int want = M.list_warps_per_sm > 0 ? M.list_warps_per_sm / W : most;
      const int resident = sm_count() * (want < 1 ? 1 : (want > most ? most : want));
      // few slots active: a grid of about one warp per possible active slot (the warps still
      // stride over however many there are, so any count is walked correctly)
      const int few = epi.listed == 2 && M.list_few_slots > 0 ? (M.list_few_slots + W - 1) / W : 0;
      const int need = few > 0 ? few : (M.nslots + W - 1) / W;
      const int grid = DPDLP_LIST_PERSISTENT && need > resident ? resident : need;
      return launch_k(packed_list_kernel<NV, W, Epi>, grid, W * LANES, s, pdl, M, g, epi);
    }
  }
  return launch_k(packed_spmv_kernel<NV, W, Epi>, (M.nslots + W - 1) / W, W * LANES, s, pdl, M, g,
                  epi);
}

// Iteration kernels (Epi::kTunable) run with the orientation's chosen slots per block;
// the plain products of the checks and the power iteration use PK_WARPS.
template <int NV, class Epi>
static cudaError_t launch_packed(const DevPacked& M, GatherVecs<NV> g, Epi epi, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (M.nslots > 0) {
    if constexpr (Epi::kTunable) {
      switch (M.cta_slots) {
        case 2: e = launch_slots<NV, 2>(M, g, epi, s); break;
        case 8: e = launch_slots<NV, 8>(M, g, epi, s); break;
        default: e = launch_slots<NV, 4>(M, g, epi, s); break;
      }
    } else {
      e = launch_slots<NV, PK_WARPS>(M, g, epi, s);
    }
  }
  if (e == cudaSuccess && M.nlong > 0 && !slots_only_of(epi)) {
    const int rest = M.nlong - M.nlong_block - M.nlong_warp;
    const int grid = M.nlong_block + (M.nlong_warp + TPB / 32 - 1) / (TPB / 32) + (rest + TPB - 1) / TPB;
    e = launch_k(finish_long_kernel<NV, Epi>, grid, TPB, s, pdl_of(epi) && DPDLP_LONG_PDL, M, epi);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_primal(const DevPacked& csc, const DevVecs& v, const DevScalars* sc,
                          IterPlan p, cudaStream_t s) {
  GatherVecs<1> g{{v.y}};
  if (v.q) {  // a diagonal QP: the prox step divides by 1 + tau Q_jj
    if (v.ninst == 1)
      return launch_packed<1>(csc, g, PrimalEpi<true, true>{sc, v.inst, v.wtab, p, 0, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, v.q, {}}, s);
    return launch_packed<1>(csc, g, PrimalEpi<false, true>{sc, v.inst, v.wtab, p, p.list, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, v.q, {}}, s);
  }
  if (v.ninst == 1)
    return launch_packed<1>(csc, g, PrimalEpi<true>{sc, v.inst, v.wtab, p, 0, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, nullptr, {}}, s);
  return launch_packed<1>(csc, g, PrimalEpi<false>{sc, v.inst, v.wtab, p, p.list, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, nullptr, {}}, s);
}

cudaError_t launch_dual(const DevPacked& csr, const DevVecs& v, const DevScalars* sc,
                        IterPlan p, cudaStream_t s) {
  GatherVecs<1> g{{v.xbar}};
  if (v.ninst == 1)
    return launch_packed<1>(csr, g, DualEpi<true>{sc, v.inst, v.wtab, p, 0, v.lo, v.hi, v.y0, v.y, v.yh, {}}, s);
  return launch_packed<1>(csr, g, DualEpi<false>{sc, v.inst, v.wtab, p, p.list, v.lo, v.hi, v.y0, v.y, v.yh, {}}, s);
}

cudaError_t launch_spmv(const DevPacked& M, const double* x0, const double* x1, double* out0,
                        double* out1, cudaStream_t s, const InstScalars* running) {
  const int listed = running != nullptr;
  if (x1) {
    GatherVecs<2> g{{x0, x1}};
    return launch_packed<2>(M, g, StoreEpi2{out0, out1, running, listed}, s);
  }
  GatherVecs<1> g{{x0}};
  return launch_packed<1>(M, g, StoreEpi1{out0, running, listed}, s);
}

// ---------------------------------------------------------------- access probes
// The packed kernels' memory accesses per stored entry without their arithmetic, to place
// the iteration kernels against what their access pattern allows (the roofline's ceilings):
//   mode 0  the index stream and the x[col] gathers (random 8-byte gathers, each its own
//           32-byte L2 sector: the gather ceiling of this layout);
//   mode 1  mode 0 plus the value stream (every load the product makes per stored entry);
//   mode 2  the index and value streams without gathers (the coalesced-stream ceiling);
//   mode 3  mode 1 plus the epilogue's per-row vector loads and stores (every memory access
//           of the iteration kernel's slots, the `ProbeRows` vectors).
// Same slots, warps, cache policies and pipeline depth as packed_spmv_kernel, and launched
// as it is (a programmatic dependent that loads its first index batches before the wait).
// Loaded words are folded with integer xor (no FP64 work) and the fold is stored only if it
// equals a constant it practically never takes, so every load stays live; mode 3 stores
// its folds into the epilogue's output vectors (the caller keeps a copy of them).
struct ProbeRows {
  const double* ld[5];  // the epilogue's per-row inputs (nld of them)
  double* st[2];        // its per-row outputs (nst of them)
  int nld, nst;
};
template <int Mode>
__global__ void __launch_bounds__(PK_TPB, DPDLP_PK_MIN_BLOCKS)
    access_probe_kernel(DevPacked M, const double* __restrict__ x, ProbeRows E,
                        unsigned long long* sink) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * PK_WARPS + w;
  if (s >= M.nslots) return;  // uniform over the warp
  constexpr int B = DPDLP_PK_BATCH;
  constexpr int NB = LANE_ITEMS / B;
  const size_t off = (size_t)s * SLOT_ITEMS;
  const uint4* ip = reinterpret_cast<const uint4*>(M.idx + off) + lane;
  const double2* vp = Vals<double>::base(M, off, lane);
  const unsigned long long pol = l2_evict_first_policy();
  unsigned long long acc = 0;
  uint32_t c0[B], c1[B];
  load_idx<B>(ip, 0, c0, pol);
  load_idx<B>(ip, 1, c1, pol);
  pdl_trigger();
  pdl_wait();
  unsigned long long g0[B];
  double v0[B];
  if (Mode >= 1) Vals<double>::load<B>(vp, 0, v0, pol);
#pragma unroll
  for (int j = 0; j < B; ++j)
    g0[j] = Mode == 2 ? c0[j] : (unsigned long long)__double_as_longlong(__ldg(x + (c0[j] & IDX_MASK)));
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    uint32_t c2[B];
    unsigned long long g1[B];
    double v1[B];
    if (b + 2 < NB) load_idx<B>(ip, b + 2, c2, pol);
    if (b + 1 < NB) {
      if (Mode >= 1) Vals<double>::load<B>(vp, b + 1, v1, pol);
#pragma unroll
      for (int j = 0; j < B; ++j)
        g1[j] = Mode == 2 ? c1[j]
                          : (unsigned long long)__double_as_longlong(__ldg(x + (c1[j] & IDX_MASK)));
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      acc ^= g0[j];
      if (Mode >= 1) acc ^= (unsigned long long)__double_as_longlong(v0[j]);
    }
    if (b + 1 < NB) {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        g0[j] = g1[j];
        v0[j] = v1[j];
        c1[j] = c2[j];
      }
    }
  }
  if (Mode == 3) {  // the epilogue's rows as apply_rows reads them: every load, then stores
    const SlotDesc sd = M.slots[s];
    constexpr int R = MAX_SLOT_ROWS / LANES;
    unsigned long long f[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      f[k] = 0;
      if (r < sd.nrows)
        for (int q = 0; q < E.nld; ++q)
          f[k] ^= (unsigned long long)__double_as_longlong(ld_once(E.ld[q] + sd.row_base + r));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane + k * LANES;
      if (r < sd.nrows)
        for (int q = 0; q < E.nst; ++q)
          st_once(E.st[q] + sd.row_base + r, __longlong_as_double((long long)(f[k] ^ acc)));
    }
  }
  if (acc == 0x9e3779b97f4a7c15ull) sink[0] = acc;
}

cudaError_t launch_access_probe(const DevPacked& M, const double* x, int mode,
                                const DevVecs& v, bool primal, bool pdl,
                                unsigned long long* sink, cudaStream_t s) {
  if (M.nslots <= 0) return cudaSuccess;
  const int grid = (M.nslots + PK_WARPS - 1) / PK_WARPS;
  // the rows' vectors of a regular (Halpern) iteration's epilogue: PrimalEpi reads c, the
  // bounds, x and the anchor and writes x_bar and x; DualEpi reads the -S box, y and the
  // anchor and writes y
  const ProbeRows E = primal ? ProbeRows{{v.c, v.lv, v.uv, v.x, v.x0}, {v.xbar, v.x}, 5, 2}
                             : ProbeRows{{v.lo, v.hi, v.y, v.y0, nullptr}, {v.y, nullptr}, 4, 1};
  cudaError_t e;
  switch (mode) {
    case 0: e = launch_k(access_probe_kernel<0>, grid, PK_TPB, s, pdl, M, x, E, sink); break;
    case 1: e = launch_k(access_probe_kernel<1>, grid, PK_TPB, s, pdl, M, x, E, sink); break;
    case 2: e = launch_k(access_probe_kernel<2>, grid, PK_TPB, s, pdl, M, x, E, sink); break;
    case 3: e = launch_k(access_probe_kernel<3>, grid, PK_TPB, s, pdl, M, x, E, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ---------------------------------------------------------------- fused body (small LPs)
// On a small LP an iteration costs launch latency, not bandwidth: its two products touch
// a few hundred kilobytes.  fused_body_kernel runs every iteration of a graph body in one
// thread block of FB_WARPS warps, phases separated by block barriers: the primal slots
// (one warp per slot, slots strided over the warps), the long columns, the dual slots, the
// long rows.  Each phase is the device code of the separate kernels (lane_sums, the
// epilogues, finish_long_kernel's row classes with the same reduction trees), so the
// sums, their order and hence the results are bitwise those of the separate launches.  One
// SM's L2 bandwidth bounds this form, and most of its traffic would be the random gathers
// (one 32-byte sector per 8-byte value), so the gathered vectors live in shared memory: x_bar
// only there, y in global memory and mirrored there.  Gathers read them with plain
// (coherent) loads, and the block barriers order every write before its reads.
static_assert(!DPDLP_L2_HINTS, "the fused body stores x_bar through a shared-memory pointer");
constexpr int FB_WARPS = 16;
constexpr int FB_TPB = FB_WARPS * LANES;
constexpr int FB_MAX_CLUSTER = 8;     // CTAs of the cluster form (the portable cluster size)
constexpr int FB_SLOTS_PER_CTA = 2;   // automatic cluster size: about this many slots per CTA
constexpr int FB_SINGLE_MAX_SLOTS = 6;  // automatic: one CTA up to this many slots per copy

// A CTA's copy of its slots of one packed orientation in shared memory (the slots rank,
// rank + C, rank + 2 C, ... of a C-CTA cluster, in that order): values, indices, lane
// metadata and descriptors, filled once per launch and read by every iteration of the body
// (the matrix does not change inside a graph body).  FP32 values are not copied: that form
// reads the global slot.
struct SlotCache {
  double* val;      // SLOT_ITEMS per cached slot, the global layout
  uint32_t* idx;    // likewise
  LaneMeta* lanes;  // LANES per cached slot
  SlotDesc* desc;
  // the epilogue's row inputs of the cached slots: field f of row r of cached slot k at
  // rows[f * fs + k * MAX_SLOT_ROWS + r] (primal: c, lv, uv, x0, x, Q diagonal; dual: lo, hi,
  // y0); none of them changes inside a body but x, which the epilogue keeps current
  double* rows;
  int fs;
};
// Bytes of the copies of one slot (values, indices, lane metadata, descriptor), and of its
// rows' epilogue inputs (ROW_FIELDS_PRIMAL / _DUAL fields).
constexpr size_t SLOT_CACHE_BYTES = SLOT_ITEMS * (sizeof(double) + sizeof(uint32_t)) +
                                    LANES * sizeof(LaneMeta) + sizeof(SlotDesc);
constexpr int ROW_FIELDS_PRIMAL = 6, ROW_FIELDS_DUAL = 3;
constexpr size_t ROW_COPY_BYTES = MAX_SLOT_ROWS * sizeof(double);
// Carves the copies of kc primal and kr dual slots out of shared memory at `base` (16-byte
// aligned).
__device__ __forceinline__ void carve_slot_caches(char* base, int kc, int kr, SlotCache& cc,
                                                  SlotCache& cr) {
  cc.val = reinterpret_cast<double*>(base);
  cr.val = cc.val + (size_t)kc * SLOT_ITEMS;
  cc.idx = reinterpret_cast<uint32_t*>(cr.val + (size_t)kr * SLOT_ITEMS);
  cr.idx = cc.idx + (size_t)kc * SLOT_ITEMS;
  cc.lanes = reinterpret_cast<LaneMeta*>(cr.idx + (size_t)kr * SLOT_ITEMS);
  cr.lanes = cc.lanes + (size_t)kc * LANES;
  cc.desc = reinterpret_cast<SlotDesc*>(cr.lanes + (size_t)kr * LANES);
  cr.desc = cc.desc + kc;
  cc.rows = reinterpret_cast<double*>(cr.desc + kr);
  cc.fs = kc * MAX_SLOT_ROWS;
  cr.rows = cc.rows + (size_t)ROW_FIELDS_PRIMAL * cc.fs;
  cr.fs = kr * MAX_SLOT_ROWS;
}
// Every thread of the CTA copies the epilogue inputs `src[0..nf)` of the rows of this CTA's
// slots of M into c.rows.
__device__ __forceinline__ void fill_row_copies(const DevPacked& M, const SlotCache& c,
                                                const double* const* src, int nf, int rank,
                                                int C) {
  const int nk = rank < M.nslots ? (M.nslots - rank + C - 1) / C : 0;
  for (int t = threadIdx.x; t < nk * MAX_SLOT_ROWS; t += blockDim.x) {
    const int k = t / MAX_SLOT_ROWS, r = t % MAX_SLOT_ROWS;
    const SlotDesc d = M.slots[rank + C * k];
    if (r < d.nrows)
      for (int f = 0; f < nf; ++f) c.rows[(size_t)f * c.fs + t] = src[f][d.row_base + r];
  }
}
// Every thread of the CTA copies (16 bytes at a time) this CTA's slots of M.
__device__ __forceinline__ void fill_slot_cache(const DevPacked& M, const SlotCache& c, int rank,
                                                int C) {
  const int nk = rank < M.nslots ? (M.nslots - rank + C - 1) / C : 0;
  constexpr int V16 = SLOT_ITEMS * (int)sizeof(double) / 16, I16 = SLOT_ITEMS * (int)sizeof(uint32_t) / 16;
  constexpr int L16 = LANES * (int)sizeof(LaneMeta) / 16;
  for (int t = threadIdx.x; t < nk * V16; t += blockDim.x) {
    const int k = t / V16, u = t % V16;
    reinterpret_cast<uint4*>(c.val + (size_t)k * SLOT_ITEMS)[u] =
        reinterpret_cast<const uint4*>(M.val + (size_t)(rank + C * k) * SLOT_ITEMS)[u];
  }
  for (int t = threadIdx.x; t < nk * I16; t += blockDim.x) {
    const int k = t / I16, u = t % I16;
    reinterpret_cast<uint4*>(c.idx + (size_t)k * SLOT_ITEMS)[u] =
        reinterpret_cast<const uint4*>(M.idx + (size_t)(rank + C * k) * SLOT_ITEMS)[u];
  }
  for (int t = threadIdx.x; t < nk * L16; t += blockDim.x) {
    const int k = t / L16, u = t % L16;
    reinterpret_cast<uint4*>(c.lanes + (size_t)k * LANES)[u] =
        reinterpret_cast<const uint4*>(M.lanes + (size_t)(rank + C * k) * LANES)[u];
  }
  for (int k = threadIdx.x; k < nk; k += blockDim.x) c.desc[k] = M.slots[rank + C * k];
}

// One product-and-step phase over this CTA's slots of M (the packed_spmv_kernel body): CTA
// `rank` of C takes the slots rank, rank + C, ..., its warps striding over them.  Cache: the
// slots are read from this CTA's shared-memory copy.
template <bool Cache, class Epi>
__device__ __forceinline__ void body_slots(const DevPacked& M, const SlotCache& cache,
                                           const GatherVecs<1>& g, Epi& epi,
                                           double (*srow)[MAX_SLOT_ROWS], int w, int lane,
                                           int rank, int C) {
  constexpr int B = DPDLP_PK_BATCH;
  const unsigned long long pol = l2_evict_first_policy();
  DevPacked Mv = M;  // the view the FP64 product reads: the copy when cached
  if constexpr (Cache) {
    Mv.val = cache.val;
    Mv.idx = cache.idx;
  }
  for (int k = w, s = rank + C * w; s < M.nslots; k += FB_WARPS, s += C * FB_WARPS) {
    // uniform over the warp
    const SlotDesc sd = Cache ? cache.desc[k] : M.slots[s];
    const LaneMeta lm = Cache ? cache.lanes[(size_t)k * LANES + lane] : M.lanes[(size_t)s * LANES + lane];
    uint32_t c0[B], c1[B];
    if (epi.fp32() && M.val32) {  // FP32 values: the global slot
      const size_t off = (size_t)s * SLOT_ITEMS;
      const uint4* ip = reinterpret_cast<const uint4*>(M.idx + off) + lane;
      load_idx<B>(ip, 0, c0, pol);
      load_idx<B>(ip, 1, c1, pol);
      lane_sums<float, 1, B, true>(M, g, off, lane, lm.row_local, lm.piece_base, srow, ip, pol, c0, c1);
    } else {
      const size_t off = (size_t)(Cache ? k : s) * SLOT_ITEMS;
      const uint4* ip = reinterpret_cast<const uint4*>(Mv.idx + off) + lane;
      load_idx<B, Cache>(ip, 0, c0, pol);
      load_idx<B, Cache>(ip, 1, c1, pol);
      lane_sums<double, 1, B, true, Cache>(Mv, g, off, lane, lm.row_local, lm.piece_base, srow, ip,
                                           pol, c0, c1);
    }
    __syncwarp();
    epi.prepare(sd.inst);
    if constexpr (Cache)
      epi.apply_rows_copied(sd.row_base, sd.nrows, lane, srow, cache.rows + (size_t)k * MAX_SLOT_ROWS,
                            cache.fs);
    else
      epi.apply_rows(sd.row_base, sd.nrows, lane, srow);
    __syncwarp();  // the row sums are read before the warp's next slot writes them
  }
}

// The long rows of M with finish_long_kernel's warp-class and thread-class sums (an LP that
// fits the fused body has no block-class rows: one would need more than 8,192 entries, so
// the other orientation would have more than FUSED_MAX_SLOTS slots).
template <class Epi>
__device__ __forceinline__ void fused_long(const DevPacked& M, Epi& epi, int w, int lane) {
  const int nw = M.nlong_warp;
  for (int i = w; i < nw; i += FB_WARPS) {  // uniform over the warp
    const int row = M.long_row[i];
    typename Epi::Row in{};
    if (lane == 0) in = epi.load_row(row);
    double a = strided_piece_sum(M, 0, M.long_ptr[i] + lane, M.long_ptr[i + 1], LANES);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    double v[1];
    v[0] = a;
    if (lane == 0) epi.apply_loaded(row, v, in);
  }
  for (int i = nw + (int)threadIdx.x; i < M.nlong; i += FB_TPB) {
    const int row = M.long_row[i];
    const typename Epi::Row in = epi.load_row(row);
    const double a = strided_piece_sum(M, 0, M.long_ptr[i], M.long_ptr[i + 1], 1);
    double v[1];
    v[0] = a;
    epi.apply_loaded(row, v, in);
  }
}

// Per-body constants of one LP in shared memory: the solver and instance scalars and the
// Halpern weights of the body's K iterations (same layout as the global table), which the
// epilogues read at every phase; only the check and control kernels between bodies change
// them.
struct BodyConsts {
  DevScalars sc;
  InstScalars inst;
  double w[2 * KMAX];
};
__device__ __forceinline__ void load_body_consts(BodyConsts& b, const DevScalars* sc,
                                                 const InstScalars* itab, const double* wtab, int K) {
  if (threadIdx.x == 0) {
    b.sc = *sc;
    b.inst = itab[0];
  }
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    b.w[t] = wtab[t];
    b.w[KMAX + t] = wtab[KMAX + t];
  }
}
template <class Epi>
__device__ __forceinline__ void use_body_consts(Epi& e, const BodyConsts& b) {
  e.sc = &b.sc;
  e.itab = &b.inst;
  e.wtab = b.w;
}

// Offset of the slot copies in the dynamic shared memory, after y and x_bar (16-byte aligned).
__host__ __device__ inline size_t fb_cache_offset(int rows_total) {
  return ((size_t)rows_total * sizeof(double) + 15) / 16 * 16;
}

template <class PEpi, bool Cache>
__global__ void __launch_bounds__(FB_TPB, 1)
    fused_body_kernel(DevPacked Mc, DevPacked Mr, PEpi pe_in, DualEpi<true, 1> de_in, int K,
                      int kc, int kr) {
  __shared__ double srow[FB_WARPS][1][MAX_SLOT_ROWS];
  extern __shared__ __align__(16) double fb_vecs[];  // y [m], x_bar [n], (Cache) slot copies
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = Mr.rows, n = Mc.rows;
  double* ys = fb_vecs;
  double* xs = fb_vecs + m;
  __shared__ BodyConsts consts;
  load_body_consts(consts, pe_in.sc, pe_in.itab, pe_in.wtab, K);
  SlotCache cc{}, cr{};
  if constexpr (Cache) {
    carve_slot_caches(reinterpret_cast<char*>(fb_vecs) + fb_cache_offset(m + n), kc, kr, cc, cr);
    fill_slot_cache(Mc, cc, 0, 1);
    fill_slot_cache(Mr, cr, 0, 1);
    const double* const ps[ROW_FIELDS_PRIMAL] = {pe_in.c, pe_in.lv, pe_in.uv, pe_in.x0, pe_in.x, pe_in.qd};
    const double* const ds[ROW_FIELDS_DUAL] = {de_in.lo, de_in.hi, de_in.y0};
    fill_row_copies(Mc, cc, ps, pe_in.qd ? 6 : 5, 0, 1);
    fill_row_copies(Mr, cr, ds, ROW_FIELDS_DUAL, 0, 1);
  }
  for (int i = threadIdx.x; i < m; i += FB_TPB) ys[i] = de_in.y[i];
  __syncthreads();
  // x_bar lives only in shared memory (nothing after the body reads it); y is written to
  // global memory and mirrored here
  const GatherVecs<1> gp{{ys}}, gd{{xs}};
  for (int i = 0; i < K; ++i) {
    // the scalars read by begin() change only at checks, so every thread takes the same
    // branch, and once the iteration limit is passed it stays passed
    PEpi pe = pe_in;
    pe.plan.i = i;
    pe.xbar = xs;
    use_body_consts(pe, consts);
    if (!pe.begin()) break;
    body_slots<Cache>(Mc, cc, gp, pe, srow[w], w, lane, 0, 1);
    __syncthreads();
    if (Mc.nlong > 0) {
      fused_long(Mc, pe, w, lane);
      __syncthreads();
    }
    DualEpi<true, 1> de = de_in;
    de.plan.i = i;
    de.ys = ys;
    use_body_consts(de, consts);
    if (!de.begin()) break;
    body_slots<Cache>(Mr, cr, gd, de, srow[w], w, lane, 0, 1);
    __syncthreads();
    if (Mr.nlong > 0) {
      fused_long(Mr, de, w, lane);
      __syncthreads();
    }
  }
}

// ---- cluster form: the same body spread over the CTAs of a thread-block cluster
// One CTA bounds the single-block body by its SM's FP64 issue rate (about two FMAs per
// clock) once an LP has more than a few slots.  Here C CTAs (one per SM) share the work:
// CTA r takes the slots r, r + C, ... (its warps striding over them) and every C-th long row.
// Each CTA keeps full shared-memory copies of x_bar and y for its gathers; a new x_bar_j or
// y_i is stored into all C copies through distributed shared memory, and cluster barriers
// separate the phases (and order the piece sums of long rows, which cross SMs through L2).
// Each slot's lane sums, each epilogue and each long row's sum are the same code as the
// separate launches, so results are bitwise theirs.
template <class Epi>
__device__ __forceinline__ void cluster_long(const DevPacked& M, Epi& epi, int w, int lane,
                                             int rank, int C) {
  const int nw = M.nlong_warp;
  for (int i = rank * FB_WARPS + w; i < nw; i += C * FB_WARPS) {  // uniform over the warp
    const int row = M.long_row[i];
    typename Epi::Row in{};
    if (lane == 0) in = epi.load_row(row);
    double a = strided_piece_sum<true>(M, 0, M.long_ptr[i] + lane, M.long_ptr[i + 1], LANES);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    double v[1];
    v[0] = a;
    if (lane == 0) epi.apply_loaded(row, v, in);
  }
  for (int i = nw + rank * FB_TPB + (int)threadIdx.x; i < M.nlong; i += C * FB_TPB) {
    const int row = M.long_row[i];
    const typename Epi::Row in = epi.load_row(row);
    double v[1];
    v[0] = strided_piece_sum<true>(M, 0, M.long_ptr[i], M.long_ptr[i + 1], 1);
    epi.apply_loaded(row, v, in);
  }
}

// Pieces written to global memory by this cluster's lanes become visible to the CTAs that
// finish the long rows.
__device__ __forceinline__ void cluster_sync_pieces(cooperative_groups::cluster_group& cl) {
  __threadfence();
  cl.sync();
}

template <class PEpi, bool Cache>
__global__ void __launch_bounds__(FB_TPB, 1)
    cluster_body_kernel(DevPacked Mc, DevPacked Mr, PEpi pe_in, DualEpi<true, 2> de_in, int K,
                        int kc, int kr) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  __shared__ double srow[FB_WARPS][1][MAX_SLOT_ROWS];
  // y [m], then x_bar [n]: this CTA's copies (same offsets in every CTA), then (Cache) the
  // copies of this CTA's slots
  extern __shared__ __align__(16) double fb_vecs[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = Mr.rows, n = Mc.rows;
  double* ys = fb_vecs;
  double* xs = fb_vecs + m;
  __shared__ BodyConsts consts;
  load_body_consts(consts, pe_in.sc, pe_in.itab, pe_in.wtab, K);
  SlotCache cc{}, cr{};
  if constexpr (Cache) {
    carve_slot_caches(reinterpret_cast<char*>(fb_vecs) + fb_cache_offset(m + n), kc, kr, cc, cr);
    fill_slot_cache(Mc, cc, rank, C);
    fill_slot_cache(Mr, cr, rank, C);
    const double* const ps[ROW_FIELDS_PRIMAL] = {pe_in.c, pe_in.lv, pe_in.uv, pe_in.x0, pe_in.x, pe_in.qd};
    const double* const ds[ROW_FIELDS_DUAL] = {de_in.lo, de_in.hi, de_in.y0};
    fill_row_copies(Mc, cc, ps, pe_in.qd ? 6 : 5, rank, C);
    fill_row_copies(Mr, cr, ds, ROW_FIELDS_DUAL, rank, C);
  }
  for (int i = threadIdx.x; i < m; i += FB_TPB) ys[i] = de_in.y[i];
  cl.sync();  // every CTA of the cluster runs before any stores into another's copies
  const GatherVecs<1> gp{{ys}}, gd{{xs}};
  for (int i = 0; i < K; ++i) {
    // begin() reads scalars that change only at checks: every CTA takes the same branch
    PEpi pe = pe_in;
    pe.plan.i = i;
    pe.xbar = xs;
    pe.ncta = (unsigned)C;
    use_body_consts(pe, consts);
    if (!pe.begin()) break;
    body_slots<Cache>(Mc, cc, gp, pe, srow[w], w, lane, rank, C);
    if (Mc.nlong > 0) {
      cluster_sync_pieces(cl);
      cluster_long(Mc, pe, w, lane, rank, C);
    }
    cl.sync();  // x_bar complete in every copy
    DualEpi<true, 2> de = de_in;
    de.plan.i = i;
    de.ys = ys;
    de.ncta = (unsigned)C;
    use_body_consts(de, consts);
    if (!de.begin()) break;
    body_slots<Cache>(Mr, cr, gd, de, srow[w], w, lane, rank, C);
    if (Mr.nlong > 0) {
      cluster_sync_pieces(cl);
      cluster_long(Mr, de, w, lane, rank, C);
    }
    cl.sync();  // y complete in every copy
  }
  cl.sync();  // no CTA exits while another may still store into its shared memory
  (void)n;
}

// x_bar and y in shared memory: at most FB_VEC_MAX entries together; with the slot copies
// at most FB_DYN_CACHE_MAX bytes of dynamic shared memory (a block may hold 227 KB; the
// static row sums and the body constants take about 32 KB)
constexpr int FB_VEC_MAX = 20480;
constexpr int FB_DYN_MAX = FB_VEC_MAX * (int)sizeof(double);
constexpr int FB_DYN_CACHE_MAX = 192 * 1024;
static_assert(FB_DYN_CACHE_MAX + FB_WARPS * MAX_SLOT_ROWS * sizeof(double) + sizeof(BodyConsts) <=
                  227 * 1024,
              "slot copies, vectors, row sums and body constants fit one block's shared memory");

bool fused_body_fits(const DevPacked& csc, const DevPacked& csr, int ninst, int max_slots) {
  return ninst == 1 && max_slots <= FUSED_MAX_SLOTS && csc.nslots <= max_slots &&
         csr.nslots <= max_slots && csc.nlong_block == 0 && csr.nlong_block == 0 &&
         (long long)csc.rows + csr.rows <= FB_VEC_MAX;
}

template <class Kern>
static cudaError_t set_dyn_smem(Kern kernel, int bytes, cudaError_t e) {
  return e != cudaSuccess ? e
                          : cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t fused_body_prepare() {
  cudaError_t e = cudaSuccess;
  e = set_dyn_smem(fused_body_kernel<PrimalEpi<true>, false>, FB_DYN_MAX, e);
  e = set_dyn_smem(fused_body_kernel<PrimalEpi<true, true>, false>, FB_DYN_MAX, e);
  e = set_dyn_smem(cluster_body_kernel<PrimalEpi<true, false, true>, false>, FB_DYN_MAX, e);
  e = set_dyn_smem(cluster_body_kernel<PrimalEpi<true, true, true>, false>, FB_DYN_MAX, e);
  e = set_dyn_smem(fused_body_kernel<PrimalEpi<true>, true>, FB_DYN_CACHE_MAX, e);
  e = set_dyn_smem(fused_body_kernel<PrimalEpi<true, true>, true>, FB_DYN_CACHE_MAX, e);
  e = set_dyn_smem(cluster_body_kernel<PrimalEpi<true, false, true>, true>, FB_DYN_CACHE_MAX, e);
  e = set_dyn_smem(cluster_body_kernel<PrimalEpi<true, true, true>, true>, FB_DYN_CACHE_MAX, e);
  return e;
}

// Automatic size, measured on one GB300 with the shared-memory copies (us per iteration,
// n = 2m, 8 nonzeros per column): one CTA is fastest up to about 6 slots per copy
// (latency-bound: 7.9 us at 2-3 slots, 9.2 for two CTAs, 11.8 separate); beyond that one
// SM's FP64 rate bounds it and a cluster with about two slots per CTA wins (8 slots: 10.2,
// 10.0 with two CTAs, 12.6 separate; 16: 9.5 against 12.3; 32: 10.5 against 13.0); its two
// barriers per iteration cost about 3.5 us, so from about 50 slots the separate launches
// win (48: 13.1 against 13.5; 64: 14.6 against 13.7).
int fused_cluster_ctas(const DevPacked& csc, const DevPacked& csr, int requested) {
  if (requested >= 1) return requested > FB_MAX_CLUSTER ? FB_MAX_CLUSTER : requested;
  const int slots = csc.nslots > csr.nslots ? csc.nslots : csr.nslots;
  if (slots <= FB_SINGLE_MAX_SLOTS) return 1;
  const int c = (slots + FB_SLOTS_PER_CTA - 1) / FB_SLOTS_PER_CTA;
  return c > FB_MAX_CLUSTER ? FB_MAX_CLUSTER : c;
}

template <class PEpi, bool Cache>
static cudaError_t launch_cluster(const DevPacked& csc, const DevPacked& csr, PEpi pe,
                                  DualEpi<true, 2> de, int K, int C, size_t dyn, int kc, int kr,
                                  cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(FB_TPB);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cluster_body_kernel<PEpi, Cache>, csc, csr, pe, de, K, kc, kr);
}

template <class PEpi>
static cudaError_t launch_single(const DevPacked& csc, const DevPacked& csr, PEpi pe,
                                 DualEpi<true, 1> de, int K, bool cache, size_t dyn, int kc,
                                 int kr, cudaStream_t s) {
  if (cache)
    fused_body_kernel<PEpi, true><<<1, FB_TPB, dyn, s>>>(csc, csr, pe, de, K, kc, kr);
  else
    fused_body_kernel<PEpi, false><<<1, FB_TPB, dyn, s>>>(csc, csr, pe, de, K, kc, kr);
  return cudaGetLastError();
}

cudaError_t launch_body_fused(const DevPacked& csc, const DevPacked& csr, const DevVecs& v,
                              const DevScalars* sc, int K, int cluster, int slot_cache,
                              cudaStream_t s) {
  if (v.ninst != 1 || csc.rows + csr.rows > FB_VEC_MAX) return cudaErrorInvalidValue;
  const IterPlan p{0, 0, 0};
  const int C = cluster > 1 ? (cluster > FB_MAX_CLUSTER ? FB_MAX_CLUSTER : cluster) : 1;
  // the slots of CTA 0 (the most of any CTA) copied into shared memory, when they fit
  const int kc = (csc.nslots + C - 1) / C, kr = (csr.nslots + C - 1) / C;
  const size_t cached = fb_cache_offset(csc.rows + csr.rows) + (size_t)(kc + kr) * SLOT_CACHE_BYTES +
                        (size_t)(ROW_FIELDS_PRIMAL * kc + ROW_FIELDS_DUAL * kr) * ROW_COPY_BYTES;
  const bool cache = slot_cache && cached <= (size_t)FB_DYN_CACHE_MAX;
  const size_t dyn = cache ? cached : (size_t)(csc.rows + csr.rows) * sizeof(double);
  if (C > 1) {
    const DualEpi<true, 2> de{sc, v.inst, v.wtab, p, 0, v.lo, v.hi, v.y0, v.y, v.yh, {}, nullptr, 0};
    const PrimalEpi<true, true, true> pq{sc, v.inst, v.wtab, p, 0, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, v.q, {}, 0};
    const PrimalEpi<true, false, true> pl{sc, v.inst, v.wtab, p, 0, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, nullptr, {}, 0};
    if (v.q)
      return cache ? launch_cluster<PrimalEpi<true, true, true>, true>(csc, csr, pq, de, K, C, dyn, kc, kr, s)
                   : launch_cluster<PrimalEpi<true, true, true>, false>(csc, csr, pq, de, K, C, dyn, kc, kr, s);
    return cache ? launch_cluster<PrimalEpi<true, false, true>, true>(csc, csr, pl, de, K, C, dyn, kc, kr, s)
                 : launch_cluster<PrimalEpi<true, false, true>, false>(csc, csr, pl, de, K, C, dyn, kc, kr, s);
  }
  const DualEpi<true, 1> de{sc, v.inst, v.wtab, p, 0, v.lo, v.hi, v.y0, v.y, v.yh, {}, nullptr};
  if (v.q)
    return launch_single(csc, csr, PrimalEpi<true, true>{sc, v.inst, v.wtab, p, 0, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, v.q, {}}, de, K, cache, dyn, kc, kr, s);
  return launch_single(csc, csr, PrimalEpi<true>{sc, v.inst, v.wtab, p, 0, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, nullptr, {}}, de, K, cache, dyn, kc, kr, s);
}

// ---------------------------------------------------------------- check reductions
// One thread block per reduction chunk (at most RED_CHUNK consecutive rows or columns of
// one instance); instances that are no longer running contribute zeros.

// Row terms at (x^, y^): [0] (Ax^ - proj_S(Ax^))^2, [1] the p(-y^; lc, uc) term,
// [2] (y^k - y^)^2, [3] (A dx)_i (y^k - y^)_i, [4] (y^ - y0)^2.
__global__ void __launch_bounds__(TPB) reduce_rows_kernel(DevVecs v) {
  __shared__ double buf[TPB / 32];
  const int4 ch = v.chunk_rows[blockIdx.x];  // {instance, start, length, -}
  double q[NRED] = {0, 0, 0, 0, 0, 0};
  if (v.inst[ch.x].status == -1) {
    for (int i = ch.y + threadIdx.x; i < ch.y + ch.z; i += TPB) {
      const double lc = -v.hi[i], uc = -v.lo[i];
      const double ax = v.axh[i];
      double d = ax - clampd(ax, lc, uc);
      if (v.row_w) d *= v.row_w[i];  // residual of the original LP (preconditioned solve)
      q[0] = fma(d, d, q[0]);
      const double yh = v.yh[i];
      double p = 0.0;  // u (-y)^+ - l (-y)^-, a term vanishing when its multiplier is 0
      if (yh < 0.0) p = uc * (-yh);
      if (yh > 0.0) p = -(lc * yh);
      q[1] += p;
      const double dy = v.y[i] - yh;
      q[2] = fma(dy, dy, q[2]);
      q[3] = fma(v.adx[i], dy, q[3]);
      const double ya = yh - v.y0[i];
      q[4] = fma(ya, ya, q[4]);
    }
  }
#pragma unroll
  for (int k = 0; k < NRED; ++k) {
    const double s = block_sum(q[k], buf);
    if (threadIdx.x == 0) v.red_rows[blockIdx.x * NRED + k] = s;
  }
}

// Column terms at (x^, y^) with the instance's current tau: g = c + Q x^ - A^T y^ (Q = 0
// for an LP), xt = x^ - tau g, px = proj_X(xt): [0] (px - x^)^2, [1] (px - xt) x^
// (= tau s_j x^_j), [2] c x^, [3] dx^2, [4] (x^ - x0)^2, [5] Q_jj x^_j^2.
__global__ void __launch_bounds__(TPB) reduce_cols_kernel(DevVecs v) {
  __shared__ double buf[TPB / 32];
  const int4 ch = v.chunk_cols[blockIdx.x];
  double q[NRED] = {0, 0, 0, 0, 0, 0};
  const InstScalars& I = v.inst[ch.x];
  if (I.status == -1) {
    const double tau = I.tau;
    for (int j = ch.y + threadIdx.x; j < ch.y + ch.z; j += TPB) {
      const double xhj = v.xh[j];
      double g = v.c[j] - v.aty[j];
      if (v.q) {
        const double qx = v.q[j] * xhj;
        g += qx;
        q[5] = fma(qx, xhj, q[5]);
      }
      const double xt = fma(-tau, g, xhj);
      const double px = clampd(xt, v.lv[j], v.uv[j]);
      double d = px - xhj;
      if (v.col_w) d *= v.col_w[j];
      q[0] = fma(d, d, q[0]);
      q[1] = fma(px - xt, xhj, q[1]);
      q[2] = fma(v.c[j], xhj, q[2]);
      const double dx = v.dx[j];
      q[3] = fma(dx, dx, q[3]);
      const double xa = xhj - v.x0[j];
      q[4] = fma(xa, xa, q[4]);
    }
  }
#pragma unroll
  for (int k = 0; k < NRED; ++k) {
    const double s = block_sum(q[k], buf);
    if (threadIdx.x == 0) v.red_cols[blockIdx.x * NRED + k] = s;
  }
}

// Restart criteria of Appendix B.2 (0 none, 1 sufficient, 2 necessary, 3 artificial).
__device__ int restart_kind(double r, double r_anchor, double r_prev, bool first, long long k,
                            long long T, const DevScalars& s) {
  if (r <= s.beta_s * r_anchor) return 1;
  if (!first && r <= s.beta_n * r_anchor && r > r_prev) return 2;
  if ((double)k >= s.beta_a * (double)T) return 3;
  return 0;
}

// Sum of one instance's chunk partials of quantity k, in a fixed order.
__device__ double inst_sum(const double* part, const int32_t* inst_chunk, int inst, int k,
                           double* buf) {
  double a = 0.0;
  for (int c = inst_chunk[inst] + threadIdx.x; c < inst_chunk[inst + 1]; c += TPB)
    a += part[c * NRED + k];
  return block_sum(a, buf);
}

// Control step of one instance (one thread block per instance): KKT errors (Section 2.2),
// the fixed-point residual of the restart test, the restart decision (Appendix B.2), the
// PID primal weight (Appendix B.3), the mixed-precision switch, the trace entry and the
// Halpern weights of the next graph body.  Global bookkeeping follows in finalize_kernel.
__global__ void __launch_bounds__(TPB) control_kernel(DevVecs v, const DevScalars* sc) {
  __shared__ double buf[TPB / 32];
  __shared__ double S[2][NRED];
  __shared__ long long kb_next;
  const int inst = blockIdx.x;
  InstScalars& I = v.inst[inst];
  const DevScalars& s = *sc;
  const bool running = I.status == -1;  // uniform over the block
  if (running) {
    for (int k = 0; k < NRED; ++k) {
      const double a = inst_sum(v.red_rows, v.inst_chunk_rows, inst, k, buf);
      const double b = inst_sum(v.red_cols, v.inst_chunk_cols, inst, k, buf);
      if (threadIdx.x == 0) {
        S[0][k] = a;
        S[1][k] = b;
      }
    }
  }
  const long long T = s.T_check;
  if (threadIdx.x == 0) {
    const long long k_after = I.k_base + (T - s.T_base);
    int kind = 0;
    const int mode_used = I.spmv_fp32;
    const double omega = I.omega;
    long long k_next = k_after;
    if (running) {
      const double tau = I.tau, eta = I.eta;
      const double* R = S[0];
      const double* C = S[1];
      const double r_p = sqrt(R[0]) / (1.0 + I.bnorm);
      const double r_d = sqrt(C[0]) / tau / (1.0 + I.cnorm);
      const double obj_p = C[2] + 0.5 * C[5];  // C[5] = x^T Q x (0 for an LP)
      const double obj_d = -R[1] + C[1] / tau - 0.5 * C[5];
      const double r_g = fabs(obj_p - obj_d) / (1.0 + fmax(fabs(obj_p), fabs(obj_d)));
      const double rsq = (omega / eta) * C[3] + (1.0 / (eta * omega)) * R[2] + 2.0 * R[3];
      const double r = sqrt(fmax(0.0, rsq));
      I.r_p = r_p; I.r_d = r_d; I.r_g = r_g; I.obj_p = obj_p; I.obj_d = obj_d; I.r_fp = r;
      I.iterations = T;
      if (I.spmv_fp32 && s.fp32_switch) {  // mixed precision: FP64 values once the error is
        const double kk = fmax(r_p, fmax(r_d, r_g));  // small enough or stops halving
        if (kk <= s.fp32_switch_tol) {
          I.spmv_fp32 = 0;
        } else if (kk <= 0.5 * I.best_kkt) {
          I.best_kkt = kk;
          I.stall_checks = 0;
        } else if (kk <= 100.0 * s.fp32_switch_tol && ++I.stall_checks >= s.fp32_stall_limit) {
          I.spmv_fp32 = 0;  // stalled near the floor the FP32 values set
        }
      }
      bool finite = isfinite(r) && isfinite(r_p) && isfinite(r_d) && isfinite(r_g);
      for (int k = 0; k < NRED; ++k) finite = finite && isfinite(R[k]) && isfinite(C[k]);
      if (!finite) {
        I.status = 2;
        I.apply_mode = 2;
      } else if (fmax(r_p, fmax(r_d, r_g)) <= s.eps) {
        I.status = 0;
        I.apply_mode = 2;
      } else {
        const bool first = !I.has_anchor;
        if (first) {
          I.r_anchor = r;
          I.r_prev = r;
          I.has_anchor = 1;
        }
        if (s.sched_len > 0) {
          kind = s.checks < s.sched_len ? (int)v.sched[(size_t)inst * s.sched_len + s.checks] : 0;
        } else if (s.restart_enabled) {
          kind = restart_kind(r, I.r_anchor, I.r_prev, first, k_after, T, s);
        }
        I.r_prev = r;
        if (kind) {
          I.restarts += 1;
          if (s.pid_enabled) {
            const double d_x = sqrt(C[4]), d_y = sqrt(R[4]);
            if (d_x > 0.0 && d_y > 0.0 && isfinite(d_x) && isfinite(d_y)) {
              const double so = sqrt(omega);
              const double e = log((so * d_x) / (d_y / so));
              I.e_sum += e;
              const double de = I.has_e_prev ? (e - I.e_prev) : 0.0;
              const double lw = log(omega) - (s.kp * e + s.ki * I.e_sum + s.kd * de);
              I.omega = exp(lw);
              I.e_prev = e;
              I.has_e_prev = 1;
            }
          }
          I.tau = I.eta / I.omega;
          I.sigma = I.eta * I.omega;
          I.inv_sigma = 1.0 / I.sigma;
          I.has_anchor = 0;
          k_next = 0;
          I.apply_mode = 1;
        } else {
          const double kc = (double)(k_after - 1);
          I.w1_check = (kc + 1.0) / (kc + 2.0);
          I.w0_check = 1.0 / (kc + 2.0);
          I.apply_mode = 0;
        }
        I.status = T >= s.max_iter ? 1 : -1;
      }
      I.k_base = k_next;
    } else {
      I.apply_mode = 2;
    }
    kb_next = k_next;
    if (s.trace_cap > 0) {
      dpdlp_trace_t* tr =
          static_cast<dpdlp_trace_t*>(v.trace) + ((s.trace_count + inst) % s.trace_cap);
      tr->T = T;
      tr->k = k_after;
      tr->r_primal = I.r_p;
      tr->r_dual = I.r_d;
      tr->r_gap = I.r_g;
      tr->obj_p = I.obj_p;
      tr->obj_d = I.obj_d;
      tr->r_fp = I.r_fp;
      tr->omega = omega;
      tr->restart = kind;
      tr->spmv_mode = mode_used;
      tr->inst = inst;
      tr->status = I.status;
    }
  }
  __syncthreads();
  if (!running) return;
  const double kb = (double)kb_next;
  double* w = v.wtab + (size_t)inst * 2 * KMAX;
  for (int i = threadIdx.x; i < s.K; i += TPB) {
    w[i] = (kb + i + 1.0) / (kb + i + 2.0);
    w[KMAX + i] = 1.0 / (kb + i + 2.0);
  }
}

// Global bookkeeping after the instances' control steps: the iteration counter, the check
// and trace counters, the batch status and the conditional of the device-side loop (it
// continues while any instance is running).
__global__ void __launch_bounds__(TPB) finalize_kernel(DevVecs v, DevScalars* sc,
                                                       unsigned long long cond, int use_cond) {
  __shared__ int nrun, worst;
  if (threadIdx.x == 0) {
    nrun = 0;
    worst = 0;
  }
  __syncthreads();
  int cnt = 0, wst = 0;
  for (int i = threadIdx.x; i < v.ninst; i += TPB) {
    const int st = v.inst[i].status;
    if (st == -1) ++cnt;
    else wst = st > wst ? st : wst;
  }
  atomicAdd(&nrun, cnt);  // integer sum and max: the result does not depend on the order
  atomicMax(&worst, wst);
  __syncthreads();
  if (threadIdx.x == 0) {
    DevScalars& s = *sc;
    const long long T = s.T_check;
    s.T_base = T;
    s.checks += 1;
    if (s.trace_cap > 0) s.trace_count += v.ninst;
    s.running = nrun;
    s.status = nrun > 0 ? -1 : worst;
    if (nrun > 0) s.T_check = T + s.K < s.max_iter ? T + s.K : s.max_iter;
    if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, nrun > 0 ? 1u : 0u);
  }
}

// Halpern step (or restart) at the check iteration, per element with its instance's mode.
__global__ void __launch_bounds__(TPB) apply_kernel(DevVecs v, const DevScalars* sc) {
  const int id = blockIdx.x * TPB + threadIdx.x;
  const double gamma = sc->gamma;
  const bool g1 = (gamma == 1.0), hal = sc->halpern != 0;
  if (id < v.n) {
    const InstScalars& I = v.inst[v.ninst == 1 ? 0 : v.inst_of_col[id]];
    const int mode = I.apply_mode;
    const double xh = v.xh[id];
    if (mode == 1) {
      v.x[id] = xh;
      v.x0[id] = xh;
    } else if (mode == 2) {
    } else if (hal) {
      const double xj = v.x[id];
      const double r = g1 ? fma(2.0, xh, -xj) : fma(1.0 + gamma, xh, -gamma * xj);
      v.x[id] = fma(I.w1_check, r, I.w0_check * v.x0[id]);
    } else {
      v.x[id] = xh;
    }
  }
  if (id < v.m) {
    const InstScalars& I = v.inst[v.ninst == 1 ? 0 : v.inst_of_row[id]];
    const int mode = I.apply_mode;
    const double yh = v.yh[id];
    if (mode == 1) {
      v.y[id] = yh;
      v.y0[id] = yh;
    } else if (mode == 2) {
    } else if (hal) {
      const double yi = v.y[id];
      const double r = g1 ? fma(2.0, yh, -yi) : fma(1.0 + gamma, yh, -gamma * yi);
      v.y[id] = fma(I.w1_check, r, I.w0_check * v.y0[id]);
    } else {
      v.y[id] = yh;
    }
  }
}

cudaError_t launch_check(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                         DevScalars* sc, unsigned long long cond_handle, int use_cond,
                         cudaStream_t s) {
  cudaError_t e;
  const InstScalars* running = v.ninst > 1 ? v.inst : nullptr;  // batches: running rows only
  if ((e = launch_spmv(csr, v.xh, v.dx, v.axh, v.adx, s, running)) != cudaSuccess) return e;
  if ((e = launch_spmv(csc, v.yh, nullptr, v.aty, nullptr, s, running)) != cudaSuccess) return e;
  if (v.g_rows > 0) reduce_rows_kernel<<<v.g_rows, TPB, 0, s>>>(v);
  if (v.g_cols > 0) reduce_cols_kernel<<<v.g_cols, TPB, 0, s>>>(v);
  control_kernel<<<v.ninst, TPB, 0, s>>>(v, sc);
  finalize_kernel<<<1, TPB, 0, s>>>(v, sc, cond_handle, use_cond);
  const int len = v.n > v.m ? v.n : v.m;
  if (len > 0) apply_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(v, sc);
  if (v.ninst > 1) return launch_compact(csr, csc, v, s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- active-slot lists
// Exclusive prefix sum over a block (fixed order); *total receives the block's sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* sm, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < TPB / 32; ++k) {
      const int t = sm[k];
      sm[k] = acc;
      acc += t;
    }
    sm[TPB / 32] = acc;
  }
  __syncthreads();
  const int r = sm[w] + x - v;
  *total = sm[TPB / 32];
  __syncthreads();
  return r;
}

// act_off[o][i]: first entry of instance i in orientation o's list (o = 0 rows of A, 1 rows
// of A^T), counting the slots of running instances only; the list lengths go to nactive.
__global__ void __launch_bounds__(TPB) active_offsets_kernel(DevVecs v, const int32_t* soff_r,
                                                             const int32_t* soff_c, int32_t* nact_r,
                                                             int32_t* nact_c) {
  __shared__ int sm[TPB / 32 + 1];
  const int N = v.ninst;
  int carry_r = 0, carry_c = 0;
  for (int base = 0; base < N; base += TPB) {
    const int i = base + threadIdx.x;
    const bool run = i < N && v.inst[i].status == -1;
    const int cr = run ? soff_r[i + 1] - soff_r[i] : 0;
    const int cc = run ? soff_c[i + 1] - soff_c[i] : 0;
    int tr, tc;
    const int er = block_exclusive_scan(cr, sm, &tr);
    const int ec = block_exclusive_scan(cc, sm, &tc);
    if (i < N) {
      v.act_off[i] = carry_r + er;
      v.act_off[N + 1 + i] = carry_c + ec;
    }
    carry_r += tr;
    carry_c += tc;
  }
  if (threadIdx.x == 0) {
    v.act_off[N] = carry_r;
    v.act_off[2 * N + 1] = carry_c;
    *nact_r = carry_r;
    *nact_c = carry_c;
  }
}

// One block per instance: a running instance's slot ids go to its place in the list.
__global__ void __launch_bounds__(TPB) active_fill_kernel(DevVecs v, const int32_t* soff,
                                                          const int32_t* off, int32_t* active) {
  const int i = blockIdx.x;
  if (v.inst[i].status != -1) return;
  const int first = soff[i], count = soff[i + 1] - soff[i], base = off[i];
  for (int t = threadIdx.x; t < count; t += TPB) active[base + t] = first + t;
}

__host__ __device__ int select_form_of(long long active, long long total, double fraction, int few) {
  if (few > 0 && active <= few) return 2;
  return (double)active < fraction * (double)total ? 1 : 0;
}

int select_form(long long active, long long total, double fraction, int few) {
  return select_form_of(active, total, fraction, few);
}

__global__ void select_kernel(const int32_t* nact_r, int nslots_r, const int32_t* nact_c,
                              int nslots_c, unsigned long long handle, double fraction, int few) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const long long active = (long long)*nact_r + *nact_c, total = (long long)nslots_r + nslots_c;
  cudaGraphSetConditional((cudaGraphConditionalHandle)handle,
                          (unsigned)select_form_of(active, total, fraction, few));
}

cudaError_t launch_select(const DevPacked& csr, const DevPacked& csc, unsigned long long handle,
                          double fraction, int few, cudaStream_t s) {
  select_kernel<<<1, 32, 0, s>>>(csr.nactive, csr.nslots, csc.nactive, csc.nslots, handle,
                                 fraction, few);
  return cudaGetLastError();
}

int list_max_warps_per_sm() { return DPDLP_LIST_MIN_BLOCKS * PK_WARPS; }

cudaError_t launch_compact(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                           cudaStream_t s) {
  if (!csr.active || !csc.active) return cudaSuccess;
  active_offsets_kernel<<<1, TPB, 0, s>>>(v, csr.slot_off, csc.slot_off, csr.nactive, csc.nactive);
  active_fill_kernel<<<v.ninst, TPB, 0, s>>>(v, csr.slot_off, v.act_off, csr.active);
  active_fill_kernel<<<v.ninst, TPB, 0, s>>>(v, csc.slot_off, v.act_off + v.ninst + 1, csc.active);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- start point, vectors
__global__ void fill_start_kernel(DevVecs v, int fresh_x, int fresh_y) {
  const int id = blockIdx.x * TPB + threadIdx.x;
  if (id < v.n) {
    const double x = fresh_x ? clampd(0.0, v.lv[id], v.uv[id]) : v.x[id];  // proj_X(0)
    v.x[id] = x;
    v.x0[id] = x;
    v.xh[id] = x;
  }
  if (id < v.m) {
    const double y = fresh_y ? 0.0 : v.y[id];
    v.y[id] = y;
    v.y0[id] = y;
    v.yh[id] = y;
  }
}

cudaError_t launch_fill_start(const DevVecs& v, int fresh_x, int fresh_y, cudaStream_t s) {
  const int len = v.n > v.m ? v.n : v.m;
  if (len == 0) return cudaSuccess;
  fill_start_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(v, fresh_x, fresh_y);
  return cudaGetLastError();
}

__global__ void gather_kernel(const double* in, const int32_t* perm, const double* scale,
                              double* out, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) out[i] = scale ? in[perm[i]] * scale[i] : in[perm[i]];
}
__global__ void scatter_kernel(const double* in, const int32_t* perm, const double* scale,
                               double* out, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) out[perm[i]] = scale ? in[i] * scale[i] : in[i];
}
__global__ void fill_kernel(double* p, double val, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) p[i] = val;
}

cudaError_t launch_gather(const double* in, const int32_t* perm, const double* scale,
                          double* out, int len, cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  gather_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(in, perm, scale, out, len);
  return cudaGetLastError();
}
cudaError_t launch_scatter(const double* in, const int32_t* perm, const double* scale,
                           double* out, int len, cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  scatter_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(in, perm, scale, out, len);
  return cudaGetLastError();
}
cudaError_t launch_fill(double* p, double val, int len, cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  fill_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(p, val, len);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- power iteration
// Per-instance sums of squares: one block per reduction chunk, then one block per instance.
__global__ void __launch_bounds__(TPB) sumsq_kernel(const double* a, const int4* chunks,
                                                    double* part) {
  __shared__ double buf[TPB / 32];
  const int4 ch = chunks[blockIdx.x];
  double q = 0.0;
  for (int i = ch.y + threadIdx.x; i < ch.y + ch.z; i += TPB) q = fma(a[i], a[i], q);
  q = block_sum(q, buf);
  if (threadIdx.x == 0) part[blockIdx.x] = q;
}

__global__ void __launch_bounds__(TPB) power_finish_kernel(DevVecs v) {
  __shared__ double buf[TPB / 32];
  const int inst = blockIdx.x;
  double a = 0.0;
  for (int c = v.inst_chunk_rows[inst] + threadIdx.x; c < v.inst_chunk_rows[inst + 1]; c += TPB)
    a += v.red_rows[c];
  a = block_sum(a, buf);
  double b = 0.0;
  for (int c = v.inst_chunk_cols[inst] + threadIdx.x; c < v.inst_chunk_cols[inst + 1]; c += TPB)
    b += v.red_cols[c];
  b = block_sum(b, buf);
  if (threadIdx.x == 0) {
    double* pw = v.pw + 4 * inst;
    pw[0] = a;
    pw[1] = sqrt(b);
    pw[2] = pw[1] > 0.0 ? 1.0 / pw[1] : 0.0;
  }
}

__global__ void scale_kernel(double* vv, const double* u, const double* pw, const int32_t* inst_of,
                             int single, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) vv[i] = u[i] * pw[4 * (single ? 0 : inst_of[i]) + 2];
}

cudaError_t launch_power_round(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                               double* vec_v, double* vec_w, double* vec_u, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_spmv(csr, vec_v, nullptr, vec_w, nullptr, s, nullptr)) != cudaSuccess) return e;
  if ((e = launch_spmv(csc, vec_w, nullptr, vec_u, nullptr, s, nullptr)) != cudaSuccess) return e;
  // partials live in the check-reduction buffers (NRED doubles per chunk)
  if (v.g_rows > 0) sumsq_kernel<<<v.g_rows, TPB, 0, s>>>(vec_w, v.chunk_rows, v.red_rows);
  if (v.g_cols > 0) sumsq_kernel<<<v.g_cols, TPB, 0, s>>>(vec_u, v.chunk_cols, v.red_cols);
  power_finish_kernel<<<v.ninst, TPB, 0, s>>>(v);
  if (v.n > 0)
    scale_kernel<<<(v.n + TPB - 1) / TPB, TPB, 0, s>>>(vec_v, vec_u, v.pw, v.inst_of_col,
                                                       v.ninst == 1, v.n);
  return cudaGetLastError();
}

}  // namespace pdhg

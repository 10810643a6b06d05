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

// ---------------------------------------------------------------- epilogues
// An epilogue turns finished row sums into outputs: `apply_direct(row, sums)`.

struct StoreEpi1 {
  double* out0;
  __device__ bool begin() { return true; }
  __device__ bool fp32() const { return false; }  // KKT and step-size products: FP64 values
  __device__ void apply_direct(int r, const double* s) { out0[r] = s[0]; }
};
struct StoreEpi2 {
  double *out0, *out1;
  __device__ bool begin() { return true; }
  __device__ bool fp32() const { return false; }
  __device__ void apply_direct(int r, const double* s) {
    out0[r] = s[0];
    out1[r] = s[1];
  }
};

// Per-iteration scalars read from device memory by the fused epilogues.
struct IterScalars {
  double step, inv_step, two_step, w1, w0, gamma;
  int check, halpern, gamma_one, fp32;
};

__device__ __forceinline__ bool load_iter(const DevScalars* sc, IterPlan p, bool primal,
                                          IterScalars& o) {
  if (p.force_regular) {
    o.check = 0;
  } else {
    const long long T = sc->T_base + p.i;
    if (T >= sc->max_iter) return false;  // past the iteration limit inside this body
    o.check = (T + 1 == sc->T_check);
  }
  o.step = primal ? sc->tau : sc->sigma;
  o.inv_step = sc->inv_sigma;
  o.two_step = 2.0 * o.step;
  o.w1 = sc->w1[p.i];
  o.w0 = sc->w0[p.i];
  o.gamma = sc->gamma;
  o.halpern = sc->halpern;
  o.gamma_one = (sc->gamma == 1.0);
  o.fp32 = sc->spmv_fp32;
  return true;
}

// Primal step per column j, given s = (A^T y)_j:
//   x^ = proj_X(x - tau (c - s)),  x_bar = 2 x^ - x,
//   Halpern: x <- w1 ((1+gamma) x^ - gamma x) + w0 x0   (with gamma = 1 the reflected point
//   is x_bar itself), regular iterations;
//   check iteration: keep x = x^k, store x^ and dx = x^k - x^.
struct PrimalEpi {
  const DevScalars* sc;
  IterPlan plan;
  const double *c, *lv, *uv, *x0;
  double *x, *xbar, *xh, *dx;
  IterScalars q;
  __device__ bool begin() { return load_iter(sc, plan, true, q); }
  __device__ bool fp32() const { return q.fp32 != 0; }
  __device__ void step(int j, double s, double cj, double lvj, double uvj, double xj,
                       const double* x0p) {
    const double xhj = clampd(fma(-q.step, cj - s, xj), lvj, uvj);
    const double xb = fma(2.0, xhj, -xj);
    st_keep(xbar + j, xb);
    if (q.check) {
      xh[j] = xhj;
      dx[j] = xj - xhj;
    } else if (q.halpern) {
      const double r = q.gamma_one ? xb : fma(1.0 + q.gamma, xhj, -q.gamma * xj);
      st_once(x + j, fma(q.w1, r, q.w0 * ld_once(x0p)));
    } else {
      x[j] = xhj;
    }
  }
  __device__ void apply_direct(int j, const double* s) {
    step(j, s[0], ld_once(c + j), ld_once(lv + j), ld_once(uv + j), ld_once(x + j), x0 + j);
  }
};

// Dual step per row i, given z = (A x_bar)_i:
//   w = y / sigma - z,  d = w - proj_{-S}(w),  y^ = sigma d,  -S_i = [lo_i, hi_i] = [-uc_i, -lc_i];
//   Halpern: y <- w1 ((1+gamma) y^ - gamma y) + w0 y0, with gamma = 1 evaluated as
//   w1 (2 sigma d - y) + w0 y0; check iteration: keep y = y^k, store y^.
struct DualEpi {
  const DevScalars* sc;
  IterPlan plan;
  const double *lo, *hi, *y0;
  double *y, *yh;
  IterScalars q;
  __device__ bool begin() { return load_iter(sc, plan, false, q); }
  __device__ bool fp32() const { return q.fp32 != 0; }
  __device__ void step(int i, double s, double loi, double hii, double yi, const double* y0p) {
    const double w = fma(yi, q.inv_step, -s);
    const double d = w - clampd(w, loi, hii);
    if (q.check) {
      yh[i] = q.step * d;
    } else if (q.halpern) {
      double r;
      if (q.gamma_one) {
        r = fma(q.two_step, d, -yi);
      } else {
        r = fma(1.0 + q.gamma, q.step * d, -q.gamma * yi);
      }
      st_keep(y + i, fma(q.w1, r, q.w0 * ld_once(y0p)));
    } else {
      st_keep(y + i, q.step * d);
    }
  }
  __device__ void apply_direct(int i, const double* s) {
    step(i, s[0], ld_once(lo + i), ld_once(hi + i), ld_once(y + i), y0 + i);
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

template <int NV>
struct GatherVecs {
  const double* x[NV];
};

__device__ __forceinline__ double gather(const double* p) {
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
// lane, FP32 values and indices in fours.
template <typename V>
struct Vals;
template <>
struct Vals<double> {
  using vec = double2;
  static __device__ __forceinline__ const double2* base(const DevPacked& M, size_t off, int lane) {
    return reinterpret_cast<const double2*>(M.val + off) + lane;
  }
  template <int B>
  static __device__ __forceinline__ void load(const double2* vp, int b, double (&v)[B],
                                              unsigned long long pol) {
#pragma unroll
    for (int q = 0; q < B / 2; ++q) {
      const double2 d = ld_stream(vp + ((B / 2) * b + q) * LANES, pol);
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
  template <int B>
  static __device__ __forceinline__ void load(const float4* vp, int b, float (&v)[B],
                                              unsigned long long pol) {
#pragma unroll
    for (int q = 0; q < B / 4; ++q) {
      const float4 d = ld_stream(vp + ((B / 4) * b + q) * LANES, pol);
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

template <int B>
__device__ __forceinline__ void load_idx(const uint4* ip, int b, uint32_t (&c)[B],
                                         unsigned long long pol) {
#pragma unroll
  for (int q = 0; q < B / 4; ++q) {
    const uint4 d = ld_stream(ip + ((B / 4) * b + q) * LANES, pol);
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
// gathers are in flight while the FMA chain runs.
template <typename V, int NV>
__device__ __forceinline__ void lane_sums(const DevPacked& M, const GatherVecs<NV>& g, size_t off,
                                          int lane, int rl, int pid,
                                          double (*srow)[MAX_SLOT_ROWS]) {
  constexpr int B = DPDLP_PK_BATCH;
  constexpr int NB = LANE_ITEMS / B;
  const auto* vp = Vals<V>::base(M, off, lane);
  const uint4* ip = reinterpret_cast<const uint4*>(M.idx + off) + lane;
  const unsigned long long pol = l2_evict_first_policy();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  uint32_t c0[B], c1[B];
  V v0[B];
  double x0v[NV][B];
  load_idx<B>(ip, 0, c0, pol);
  if (NB > 1) load_idx<B>(ip, 1, c1, pol);
  Vals<V>::template load<B>(vp, 0, v0, pol);
#pragma unroll
  for (int j = 0; j < B; ++j) {
#pragma unroll
    for (int k = 0; k < NV; ++k) x0v[k][j] = gather(g.x[k] + (c0[j] & IDX_MASK));
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    uint32_t c2[B];
    V v1[B];
    double x1v[NV][B];
    if (b + 2 < NB) load_idx<B>(ip, b + 2, c2, pol);
    if (b + 1 < NB) {
      Vals<V>::template load<B>(vp, b + 1, v1, pol);
#pragma unroll
      for (int j = 0; j < B; ++j) {
#pragma unroll
        for (int k = 0; k < NV; ++k) x1v[k][j] = gather(g.x[k] + (c1[j] & IDX_MASK));
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

// One warp per slot, PK_WARPS slots per block, no block-level barrier: the lanes sum their
// rows (lane_sums), then apply the epilogue to the slot's short rows, one row per lane.
template <int NV, class Epi>
__global__ void __launch_bounds__(PK_TPB, DPDLP_PK_MIN_BLOCKS) packed_spmv_kernel(DevPacked M, GatherVecs<NV> g, Epi epi_in) {
  __shared__ double srow[PK_WARPS][NV][MAX_SLOT_ROWS];
  Epi epi = epi_in;
  if (!epi.begin()) return;  // uniform over the launch
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * PK_WARPS + w;
  if (s >= M.nslots) return;  // uniform over the warp
  const SlotDesc sd = M.slots[s];
  const LaneMeta lm = M.lanes[(size_t)s * LANES + lane];
  const size_t off = (size_t)s * SLOT_ITEMS;
  if (epi.fp32() && M.val32)  // uniform over the launch
    lane_sums<float, NV>(M, g, off, lane, lm.row_local, lm.piece_base, srow[w]);
  else
    lane_sums<double, NV>(M, g, off, lane, lm.row_local, lm.piece_base, srow[w]);
  __syncwarp();
  for (int r = lane; r < sd.nrows; r += LANES) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = srow[w][k][r];
    epi.apply_direct(sd.row_base + r, v);
  }
}

// Long rows: add each row's pieces, then its epilogue.  Rows come longest first: the first
// nlong_block rows get a thread block each, the next nlong_warp rows a warp each (fixed
// strided sums and fixed reduction trees), the rest a thread each (pieces in order).
template <int NV, class Epi>
__global__ void __launch_bounds__(TPB) finish_long_kernel(DevPacked M, Epi epi_in) {
  __shared__ double red[TPB / 32];
  Epi epi = epi_in;
  if (!epi.begin()) return;
  const int nb = M.nlong_block, nw = M.nlong_warp;
  const int wblocks = (nw + TPB / 32 - 1) / (TPB / 32);
  int b = blockIdx.x;
  double v[NV];
  if (b < nb) {
    const int i = b;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int q = M.long_ptr[i] + threadIdx.x; q < M.long_ptr[i + 1]; q += TPB)
        a += M.piece_sum[(size_t)k * M.npieces + M.long_piece[q]];
      v[k] = block_sum(a, red);
    }
    if (threadIdx.x == 0) epi.apply_direct(M.long_row[i], v);
    return;
  }
  b -= nb;
  if (b < wblocks) {
    const int i = nb + b * (TPB / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nb + nw) return;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int q = M.long_ptr[i] + lane; q < M.long_ptr[i + 1]; q += LANES)
        a += M.piece_sum[(size_t)k * M.npieces + M.long_piece[q]];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      v[k] = a;
    }
    if (lane == 0) epi.apply_direct(M.long_row[i], v);
    return;
  }
  b -= wblocks;
  const int i = nb + nw + b * TPB + threadIdx.x;
  if (i >= M.nlong) return;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = 0.0;
    for (int q = M.long_ptr[i]; q < M.long_ptr[i + 1]; ++q)
      a += M.piece_sum[(size_t)k * M.npieces + M.long_piece[q]];
    v[k] = a;
  }
  epi.apply_direct(M.long_row[i], v);
}

template <int NV, class Epi>
static cudaError_t launch_packed(const DevPacked& M, GatherVecs<NV> g, Epi epi, cudaStream_t s) {
  if (M.nslots > 0)
    packed_spmv_kernel<NV, Epi><<<(M.nslots + PK_WARPS - 1) / PK_WARPS, PK_TPB, 0, s>>>(M, g, epi);
  if (M.nlong > 0) {
    const int rest = M.nlong - M.nlong_block - M.nlong_warp;
    const int grid = M.nlong_block + (M.nlong_warp + TPB / 32 - 1) / (TPB / 32) + (rest + TPB - 1) / TPB;
    finish_long_kernel<NV, Epi><<<grid, TPB, 0, s>>>(M, epi);
  }
  return cudaGetLastError();
}

cudaError_t launch_primal(const DevPacked& csc, const DevVecs& v, const DevScalars* sc,
                          IterPlan p, cudaStream_t s) {
  PrimalEpi e{sc, p, v.c, v.lv, v.uv, v.x0, v.x, v.xbar, v.xh, v.dx, {}};
  GatherVecs<1> g{{v.y}};
  return launch_packed<1>(csc, g, e, s);
}

cudaError_t launch_dual(const DevPacked& csr, const DevVecs& v, const DevScalars* sc,
                        IterPlan p, cudaStream_t s) {
  DualEpi e{sc, p, v.lo, v.hi, v.y0, v.y, v.yh, {}};
  GatherVecs<1> g{{v.xbar}};
  return launch_packed<1>(csr, g, e, s);
}

cudaError_t launch_spmv(const DevPacked& M, const double* x0, const double* x1, double* out0,
                        double* out1, cudaStream_t s) {
  if (x1) {
    GatherVecs<2> g{{x0, x1}};
    return launch_packed<2>(M, g, StoreEpi2{out0, out1}, s);
  }
  GatherVecs<1> g{{x0}};
  return launch_packed<1>(M, g, StoreEpi1{out0}, s);
}

// ---------------------------------------------------------------- check reductions
int reduction_grid(int len) {
  const int g = (len + 4095) / 4096;
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

// Row terms at (x^, y^): [0] (Ax^ - proj_S(Ax^))^2, [1] the p(-y^; lc, uc) term,
// [2] (y^k - y^)^2, [3] (A dx)_i (y^k - y^)_i, [4] (y^ - y0)^2.
__global__ void __launch_bounds__(TPB) reduce_rows_kernel(DevVecs v, int m) {
  __shared__ double buf[TPB / 32];
  double q[NRED] = {0, 0, 0, 0, 0};
  for (int i = blockIdx.x * TPB + threadIdx.x; i < m; i += gridDim.x * TPB) {
    const double lc = -v.hi[i], uc = -v.lo[i];
    const double ax = v.axh[i];
    const double d = ax - clampd(ax, lc, uc);
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
#pragma unroll
  for (int k = 0; k < NRED; ++k) {
    const double s = block_sum(q[k], buf);
    if (threadIdx.x == 0) v.red_rows[blockIdx.x * NRED + k] = s;
  }
}

// Column terms at (x^, y^) with the current tau: g = c - A^T y^, xt = x^ - tau g,
// px = proj_X(xt): [0] (px - x^)^2, [1] (px - xt) x^ (= tau s_j x^_j), [2] c x^,
// [3] dx^2, [4] (x^ - x0)^2.
__global__ void __launch_bounds__(TPB) reduce_cols_kernel(DevVecs v, int n, const DevScalars* sc) {
  __shared__ double buf[TPB / 32];
  const double tau = sc->tau;
  double q[NRED] = {0, 0, 0, 0, 0};
  for (int j = blockIdx.x * TPB + threadIdx.x; j < n; j += gridDim.x * TPB) {
    const double xhj = v.xh[j];
    const double g = v.c[j] - v.aty[j];
    const double xt = fma(-tau, g, xhj);
    const double px = clampd(xt, v.lv[j], v.uv[j]);
    const double d = px - xhj;
    q[0] = fma(d, d, q[0]);
    q[1] = fma(px - xt, xhj, q[1]);
    q[2] = fma(v.c[j], xhj, q[2]);
    const double dx = v.dx[j];
    q[3] = fma(dx, dx, q[3]);
    const double xa = xhj - v.x0[j];
    q[4] = fma(xa, xa, q[4]);
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

__global__ void __launch_bounds__(TPB) control_kernel(DevVecs v, DevScalars* sc,
                                                      unsigned long long cond, int use_cond) {
  __shared__ double buf[TPB / 32];
  __shared__ double S[2][NRED];
  __shared__ long long kb_next;
  for (int k = 0; k < NRED; ++k) {
    double a = 0.0;
    for (int gi = threadIdx.x; gi < v.g_rows; gi += TPB) a += v.red_rows[gi * NRED + k];
    a = block_sum(a, buf);
    double b = 0.0;
    for (int gi = threadIdx.x; gi < v.g_cols; gi += TPB) b += v.red_cols[gi * NRED + k];
    b = block_sum(b, buf);
    if (threadIdx.x == 0) {
      S[0][k] = a;
      S[1][k] = b;
    }
  }
  if (threadIdx.x == 0) {
    DevScalars& s = *sc;
    const double tau = s.tau, omega = s.omega, eta = s.eta;
    const double* R = S[0];
    const double* C = S[1];
    const double r_p = sqrt(R[0]) / (1.0 + s.bnorm);
    const double r_d = sqrt(C[0]) / tau / (1.0 + s.cnorm);
    const double obj_p = C[2];
    const double obj_d = -R[1] + C[1] / tau;
    const double r_g = fabs(obj_p - obj_d) / (1.0 + fmax(fabs(obj_p), fabs(obj_d)));
    const double rsq = (omega / eta) * C[3] + (1.0 / (eta * omega)) * R[2] + 2.0 * R[3];
    const double r = sqrt(fmax(0.0, rsq));
    const long long T = s.T_check;
    const long long k_after = s.k_base + (T - s.T_base);
    const long long check_idx = s.checks;
    s.checks += 1;
    s.r_p = r_p; s.r_d = r_d; s.r_g = r_g; s.obj_p = obj_p; s.obj_d = obj_d; s.r_fp = r;
    const int mode_used = s.spmv_fp32;
    if (s.spmv_fp32 && s.fp32_switch) {  // mixed precision: FP64 values once the error is
      const double kk = fmax(r_p, fmax(r_d, r_g));  // small enough or stops halving
      if (kk <= s.fp32_switch_tol) {
        s.spmv_fp32 = 0;
      } else if (kk <= 0.5 * s.best_kkt) {
        s.best_kkt = kk;
        s.stall_checks = 0;
      } else if (kk <= 100.0 * s.fp32_switch_tol && ++s.stall_checks >= s.fp32_stall_limit) {
        s.spmv_fp32 = 0;  // stalled near the floor the FP32 values set
      }
    }
    bool finite = isfinite(r) && isfinite(r_p) && isfinite(r_d) && isfinite(r_g);
    for (int k = 0; k < NRED; ++k) finite = finite && isfinite(R[k]) && isfinite(C[k]);
    int kind = 0;
    unsigned go = 0;
    long long k_next = k_after;
    s.T_base = T;
    if (!finite) {
      s.status = 2;
      s.apply_mode = 2;
    } else if (fmax(r_p, fmax(r_d, r_g)) <= s.eps) {
      s.status = 0;
      s.apply_mode = 2;
    } else {
      const bool first = !s.has_anchor;
      if (first) {
        s.r_anchor = r;
        s.r_prev = r;
        s.has_anchor = 1;
      }
      const int8_t* sched = v.sched;
      if (s.sched_len > 0) {
        kind = check_idx < s.sched_len ? (int)sched[check_idx] : 0;
      } else if (s.restart_enabled) {
        kind = restart_kind(r, s.r_anchor, s.r_prev, first, k_after, T, s);
      }
      s.r_prev = r;
      if (kind) {
        s.restarts += 1;
        if (s.pid_enabled) {
          const double d_x = sqrt(C[4]), d_y = sqrt(R[4]);
          if (d_x > 0.0 && d_y > 0.0 && isfinite(d_x) && isfinite(d_y)) {
            const double so = sqrt(omega);
            const double e = log((so * d_x) / (d_y / so));
            s.e_sum += e;
            const double de = s.has_e_prev ? (e - s.e_prev) : 0.0;
            const double lw = log(omega) - (s.kp * e + s.ki * s.e_sum + s.kd * de);
            s.omega = exp(lw);
            s.e_prev = e;
            s.has_e_prev = 1;
          }
        }
        s.tau = s.eta / s.omega;
        s.sigma = s.eta * s.omega;
        s.inv_sigma = 1.0 / s.sigma;
        s.has_anchor = 0;
        k_next = 0;
        s.apply_mode = 1;
      } else {
        const double kc = (double)(k_after - 1);
        s.w1_check = (kc + 1.0) / (kc + 2.0);
        s.w0_check = 1.0 / (kc + 2.0);
        s.apply_mode = 0;
      }
      if (T >= s.max_iter) {
        s.status = 1;
      } else {
        s.status = -1;
        go = 1;
        s.T_check = T + s.K < s.max_iter ? T + s.K : s.max_iter;
      }
    }
    s.k_base = k_next;
    kb_next = k_next;
    if (s.trace_cap > 0) {
      dpdlp_trace_t* tr = static_cast<dpdlp_trace_t*>(v.trace) + (s.trace_count % s.trace_cap);
      tr->T = T;
      tr->k = k_after;
      tr->r_primal = r_p;
      tr->r_dual = r_d;
      tr->r_gap = r_g;
      tr->obj_p = obj_p;
      tr->obj_d = obj_d;
      tr->r_fp = r;
      tr->omega = omega;
      tr->restart = kind;
      tr->spmv_mode = mode_used;
      s.trace_count += 1;
    }
    if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, go);
  }
  __syncthreads();
  const double kb = (double)kb_next;
  for (int i = threadIdx.x; i < sc->K; i += TPB) {
    sc->w1[i] = (kb + i + 1.0) / (kb + i + 2.0);
    sc->w0[i] = 1.0 / (kb + i + 2.0);
  }
}

__global__ void __launch_bounds__(TPB) apply_kernel(DevVecs v, const DevScalars* sc) {
  const int mode = sc->apply_mode;
  if (mode == 2) return;
  const int id = blockIdx.x * TPB + threadIdx.x;
  const double w1 = sc->w1_check, w0 = sc->w0_check, gamma = sc->gamma;
  const bool g1 = (gamma == 1.0), hal = sc->halpern != 0;
  if (id < v.n) {
    const double xh = v.xh[id];
    if (mode == 1) {
      v.x[id] = xh;
      v.x0[id] = xh;
    } else if (hal) {
      const double xj = v.x[id];
      const double r = g1 ? fma(2.0, xh, -xj) : fma(1.0 + gamma, xh, -gamma * xj);
      v.x[id] = fma(w1, r, w0 * v.x0[id]);
    } else {
      v.x[id] = xh;
    }
  }
  if (id < v.m) {
    const double yh = v.yh[id];
    if (mode == 1) {
      v.y[id] = yh;
      v.y0[id] = yh;
    } else if (hal) {
      const double yi = v.y[id];
      const double r = g1 ? fma(2.0, yh, -yi) : fma(1.0 + gamma, yh, -gamma * yi);
      v.y[id] = fma(w1, r, w0 * v.y0[id]);
    } else {
      v.y[id] = yh;
    }
  }
}

cudaError_t launch_check(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                         DevScalars* sc, unsigned long long cond_handle, int use_cond,
                         cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_spmv(csr, v.xh, v.dx, v.axh, v.adx, s)) != cudaSuccess) return e;
  if ((e = launch_spmv(csc, v.yh, nullptr, v.aty, nullptr, s)) != cudaSuccess) return e;
  if (v.m > 0) {
    reduce_rows_kernel<<<v.g_rows, TPB, 0, s>>>(v, v.m);
  } else {
    cudaMemsetAsync(v.red_rows, 0, sizeof(double) * NRED * v.g_rows, s);
  }
  if (v.n > 0) {
    reduce_cols_kernel<<<v.g_cols, TPB, 0, s>>>(v, v.n, sc);
  } else {
    cudaMemsetAsync(v.red_cols, 0, sizeof(double) * NRED * v.g_cols, s);
  }
  control_kernel<<<1, TPB, 0, s>>>(v, sc, cond_handle, use_cond);
  const int len = v.n > v.m ? v.n : v.m;
  if (len > 0) apply_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(v, sc);
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

__global__ void gather_kernel(const double* in, const int32_t* perm, double* out, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) out[i] = in[perm[i]];
}
__global__ void scatter_kernel(const double* in, const int32_t* perm, double* out, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) out[perm[i]] = in[i];
}
__global__ void fill_kernel(double* p, double val, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) p[i] = val;
}

cudaError_t launch_gather(const double* in, const int32_t* perm, double* out, int len,
                          cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  gather_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(in, perm, out, len);
  return cudaGetLastError();
}
cudaError_t launch_scatter(const double* in, const int32_t* perm, double* out, int len,
                           cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  scatter_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(in, perm, out, len);
  return cudaGetLastError();
}
cudaError_t launch_fill(double* p, double val, int len, cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  fill_kernel<<<(len + TPB - 1) / TPB, TPB, 0, s>>>(p, val, len);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- power iteration
__global__ void __launch_bounds__(TPB) sumsq_kernel(const double* a, int len, double* part) {
  __shared__ double buf[TPB / 32];
  double q = 0.0;
  for (int i = blockIdx.x * TPB + threadIdx.x; i < len; i += gridDim.x * TPB) q = fma(a[i], a[i], q);
  q = block_sum(q, buf);
  if (threadIdx.x == 0) part[blockIdx.x] = q;
}

__global__ void __launch_bounds__(TPB) power_finish_kernel(const double* pw_part, int gw,
                                                           const double* pu_part, int gu,
                                                           double* pw) {
  __shared__ double buf[TPB / 32];
  double a = 0.0;
  for (int i = threadIdx.x; i < gw; i += TPB) a += pw_part[i];
  a = block_sum(a, buf);
  double b = 0.0;
  for (int i = threadIdx.x; i < gu; i += TPB) b += pu_part[i];
  b = block_sum(b, buf);
  if (threadIdx.x == 0) {
    pw[0] = a;
    pw[1] = sqrt(b);
    pw[2] = pw[1] > 0.0 ? 1.0 / pw[1] : 0.0;
  }
}

__global__ void scale_kernel(double* v, const double* u, const double* pw, int len) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < len) v[i] = u[i] * pw[2];
}

cudaError_t launch_power_round(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                               double* vec_v, double* vec_w, double* vec_u, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_spmv(csr, vec_v, nullptr, vec_w, nullptr, s)) != cudaSuccess) return e;
  if ((e = launch_spmv(csc, vec_w, nullptr, vec_u, nullptr, s)) != cudaSuccess) return e;
  const int gw = reduction_grid(v.m), gu = reduction_grid(v.n);
  // partials live in the check-reduction buffers (at least 1024 * NRED doubles each)
  sumsq_kernel<<<gw, TPB, 0, s>>>(vec_w, v.m, v.red_rows);
  sumsq_kernel<<<gu, TPB, 0, s>>>(vec_u, v.n, v.red_cols);
  power_finish_kernel<<<1, TPB, 0, s>>>(v.red_rows, gw, v.red_cols, gu, v.pw);
  if (v.n > 0) scale_kernel<<<(v.n + TPB - 1) / TPB, TPB, 0, s>>>(vec_v, vec_u, v.pw, v.n);
  return cudaGetLastError();
}

}  // namespace pdhg

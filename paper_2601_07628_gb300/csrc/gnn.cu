// Warm-start network (include/dpdlp_gnn.h): forward and backward kernels and the C ABI.
//
// Four kinds of kernel carry the whole network:
//   spmm_*            sparse aggregation over A's pattern, H = 64 features per node (a warp
//                     per row, two features per lane, sums in stored order; a block of 16
//                     warps per row longer than 64 entries, chunk sums added in order);
//   linear_mma_kernel relu(X1 W1^T + X2 W2^T + b) of the 64 x 64 layers on the tensor
//                     cores (mma.sync BF16, FP32 accumulation, FP32 activations split into
//                     BF16 hi + lo); linear_kernel the same on the FP32 pipe for the 8-wide
//                     input encoders;
//   linear_bwd_mma_kernel the ReLU mask and the products with W1 and W2 for the backward
//                     pass (the mask alone for the encoders);
//   wgrad_mma_kernel, wgrad8_mma_kernel  weight and bias gradients dZ^T X on the tensor cores
//                     as fixed per-block partial sums, added in block order by
//                     reduce_partials_kernel.
// No floating-point atomics anywhere: every result is bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/dpdlp.h"
#include "../../include/dpdlp_gnn.h"

namespace {

constexpr int H = DPDLP_GNN_HIDDEN;
constexpr int F = DPDLP_GNN_FEATURES;
constexpr int L = DPDLP_GNN_ROUNDS;
constexpr int TPB = 256;
constexpr int TILE = 64;   // rows per block of the dense kernels
constexpr int WG_BLOCKS = 304;  // blocks of the weight-gradient reductions (2 per SM)

// Offsets of the parameter blocks in the flat vector (order of dpdlp_gnn.h).
struct Layout {
  int64_t Ev, ev, Ec, ec;
  int64_t Uc[L], Vc[L], bc[L], Uv[L], Vv[L], bv[L];
  int64_t wx, bx, wy, by, total;
  Layout() {
    int64_t o = 0;
    auto take = [&](int64_t k) {
      const int64_t r = o;
      o += k;
      return r;
    };
    Ev = take(H * F);
    ev = take(H);
    Ec = take(H * F);
    ec = take(H);
    for (int l = 0; l < L; ++l) {
      Uc[l] = take(H * H);
      Vc[l] = take(H * H);
      bc[l] = take(H);
      Uv[l] = take(H * H);
      Vv[l] = take(H * H);
      bv[l] = take(H);
    }
    wx = take(H);
    bx = take(1);
    wy = take(H);
    by = take(1);
    total = o;
  }
};
const Layout LAY;

// ---------------------------------------------------------------- kernels
// Sum over entries k0 .. k1-1 of val[k] * in[idx[k]][2 lane .. 2 lane + 1], added in stored
// order; SPMM_BATCH entries at a time (indices and values, then the gathers, all in flight
// together).
constexpr int SPMM_BATCH = 8;
constexpr int SPMM_LONG = 64;        // rows with more entries: a thread block per row
constexpr int SPMM_LONG_WARPS = 16;  // warps of that block, each a contiguous chunk
__device__ __forceinline__ float2 spmm_range(int64_t k0, int64_t k1, const int* __restrict__ idx,
                                             const float* __restrict__ val,
                                             const float* __restrict__ in, int lane) {
  float2 acc = make_float2(0.f, 0.f);
  int jn[SPMM_BATCH];
  float an[SPMM_BATCH];
#pragma unroll
  for (int u = 0; u < SPMM_BATCH; ++u) {
    jn[u] = k0 + u < k1 ? idx[k0 + u] : -1;
    an[u] = k0 + u < k1 ? val[k0 + u] : 0.f;
  }
  for (int64_t k = k0; k < k1; k += SPMM_BATCH) {
    int j[SPMM_BATCH];
    float a[SPMM_BATCH];
    float2 h[SPMM_BATCH];
#pragma unroll
    for (int u = 0; u < SPMM_BATCH; ++u) {
      j[u] = jn[u];
      a[u] = an[u];
    }
#pragma unroll
    for (int u = 0; u < SPMM_BATCH; ++u)
      h[u] = j[u] >= 0 ? reinterpret_cast<const float2*>(in + (size_t)j[u] * H)[lane]
                       : make_float2(0.f, 0.f);
    // the next batch's indices and values load while these gathers are in flight
    const int64_t kn = k + SPMM_BATCH;
#pragma unroll
    for (int u = 0; u < SPMM_BATCH; ++u) {
      jn[u] = kn + u < k1 ? idx[kn + u] : -1;
      an[u] = kn + u < k1 ? val[kn + u] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < SPMM_BATCH; ++u) {
      if (j[u] < 0) break;
      acc.x = fmaf(a[u], h[u].x, acc.x);
      acc.y = fmaf(a[u], h[u].y, acc.y);
    }
  }
  return acc;
}

__device__ __forceinline__ void spmm_store(float* out, int r, int lane, float2 acc, int accumulate) {
  float2* o = reinterpret_cast<float2*>(out + (size_t)r * H) + lane;
  if (accumulate) {
    const float2 p = *o;
    acc.x += p.x;
    acc.y += p.y;
  }
  *o = acc;
}

// out[r][:] (=|+=) sum_k val[k] * in[idx[k]][:] over row r's stored entries, in order: eight
// lanes per row (four rows per warp), eight features per lane, each feature summed by one
// lane in stored order.  Rows longer than SPMM_LONG are left to spmm_long_kernel.
constexpr int SPMM_ROW_LANES = 8;
__global__ void __launch_bounds__(TPB) spmm_kernel(int rows, const int64_t* __restrict__ ptr,
                                                   const int* __restrict__ idx,
                                                   const float* __restrict__ val,
                                                   const float* __restrict__ in, float* out,
                                                   int accumulate) {
  const size_t t = blockIdx.x * (size_t)TPB + threadIdx.x;
  const int r = (int)(t / SPMM_ROW_LANES), sl = (int)(t % SPMM_ROW_LANES);
  if (r >= rows) return;
  const int64_t k0 = ptr[r], k1 = ptr[r + 1];
  if (k1 - k0 > SPMM_LONG) return;
  float acc[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) acc[f] = 0.f;
  constexpr int BATCH = 4;
  for (int64_t k = k0; k < k1; k += BATCH) {
    int j[BATCH];
    float a[BATCH];
    float4 h0[BATCH], h1[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      j[u] = k + u < k1 ? idx[k + u] : -1;
      a[u] = k + u < k1 ? val[k + u] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const float4* src = reinterpret_cast<const float4*>(in + (size_t)(j[u] < 0 ? 0 : j[u]) * H) + 2 * sl;
      h0[u] = j[u] >= 0 ? src[0] : make_float4(0.f, 0.f, 0.f, 0.f);
      h1[u] = j[u] >= 0 ? src[1] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      if (j[u] < 0) break;
      acc[0] = fmaf(a[u], h0[u].x, acc[0]);
      acc[1] = fmaf(a[u], h0[u].y, acc[1]);
      acc[2] = fmaf(a[u], h0[u].z, acc[2]);
      acc[3] = fmaf(a[u], h0[u].w, acc[3]);
      acc[4] = fmaf(a[u], h1[u].x, acc[4]);
      acc[5] = fmaf(a[u], h1[u].y, acc[5]);
      acc[6] = fmaf(a[u], h1[u].z, acc[6]);
      acc[7] = fmaf(a[u], h1[u].w, acc[7]);
    }
  }
  float4* o = reinterpret_cast<float4*>(out + (size_t)r * H) + 2 * sl;
  if (accumulate) {
    const float4 p0 = o[0], p1 = o[1];
    acc[0] += p0.x; acc[1] += p0.y; acc[2] += p0.z; acc[3] += p0.w;
    acc[4] += p1.x; acc[5] += p1.y; acc[6] += p1.z; acc[7] += p1.w;
  }
  o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}
int spmm_blocks(int rows) { return (int)(((size_t)rows * SPMM_ROW_LANES + TPB - 1) / TPB); }

// The long rows (list `longs`): a block per row; warp w sums the w-th of SPMM_LONG_WARPS
// contiguous chunks of the row's entries in order, then the chunk sums are added in chunk
// order.  Fixed order: reproducible.
__global__ void __launch_bounds__(SPMM_LONG_WARPS * 32) spmm_long_kernel(
    const int* __restrict__ longs, const int64_t* __restrict__ ptr, const int* __restrict__ idx,
    const float* __restrict__ val, const float* __restrict__ in, float* out, int accumulate) {
  __shared__ float2 part[SPMM_LONG_WARPS][32];
  const int r = longs[blockIdx.x];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = ptr[r], k1 = ptr[r + 1];
  const int64_t len = k1 - k0, chunk = (len + SPMM_LONG_WARPS - 1) / SPMM_LONG_WARPS;
  const int64_t a = k0 + w * chunk, b = a + chunk < k1 ? a + chunk : k1;
  part[w][lane] = a < b ? spmm_range(a, b, idx, val, in, lane) : make_float2(0.f, 0.f);
  __syncthreads();
  if (w == 0) {
    float2 acc = part[0][lane];
    for (int q = 1; q < SPMM_LONG_WARPS; ++q) {
      acc.x += part[q][lane].x;
      acc.y += part[q][lane].y;
    }
    spmm_store(out, r, lane, acc, accumulate);
  }
}

// Stage a 64-row tile of an N x K row-major matrix into shared memory (rows past N read 0).
template <int K>
__device__ __forceinline__ void stage_rows(float (*S)[K + 1], const float* X, int r0, int N) {
  for (int e = threadIdx.x; e < TILE * K; e += TPB) {
    const int rr = e / K, kk = e % K;
    S[rr][kk] = (r0 + rr < N) ? X[(size_t)(r0 + rr) * K + kk] : 0.f;
  }
}

// Stage a BF16 weight matrix W[H][K] widened to FP32.
template <int K>
__device__ __forceinline__ void stage_weights(float (*S)[H + 1], const __nv_bfloat16* W) {
  for (int e = threadIdx.x; e < H * K; e += TPB) S[e / K][e % K] = __bfloat162float(W[e]);
}

// out = relu(X1 W1^T + X2 W2^T + b) on a 64-row tile; thread (rg, cg) owns rows
// 4 rg .. 4 rg + 3 and columns 4 cg .. 4 cg + 3.
template <int K1, bool HAS2>
__global__ void __launch_bounds__(TPB) linear_kernel(int N, const float* __restrict__ X1,
                                                     const __nv_bfloat16* __restrict__ W1,
                                                     const float* __restrict__ X2,
                                                     const __nv_bfloat16* __restrict__ W2,
                                                     const float* __restrict__ b, float* out) {
  __shared__ float Xs[TILE][H + 1];
  __shared__ float Ws[H][H + 1];
  const int r0 = blockIdx.x * TILE;
  const int t = threadIdx.x, rg = t >> 4, cg = t & 15;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  stage_rows<K1>(reinterpret_cast<float(*)[K1 + 1]>(&Xs[0][0]), X1, r0, N);
  stage_weights<K1>(Ws, W1);
  __syncthreads();
  {
    const float(*S)[K1 + 1] = reinterpret_cast<const float(*)[K1 + 1]>(&Xs[0][0]);
#pragma unroll 8
    for (int k = 0; k < K1; ++k) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = S[rg * 4 + i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = Ws[cg * 4 + j][k];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
  }
  if (HAS2) {
    __syncthreads();
    stage_rows<H>(Xs, X2, r0, N);
    stage_weights<H>(Ws, W2);
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < H; ++k) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Xs[rg * 4 + i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = Ws[cg * 4 + j][k];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + rg * 4 + i;
    if (row >= N) continue;
    float4 v;
    v.x = fmaxf(acc[i][0] + b[cg * 4 + 0], 0.f);
    v.y = fmaxf(acc[i][1] + b[cg * 4 + 1], 0.f);
    v.z = fmaxf(acc[i][2] + b[cg * 4 + 2], 0.f);
    v.w = fmaxf(acc[i][3] + b[cg * 4 + 3], 0.f);
    reinterpret_cast<float4*>(out + (size_t)row * H)[cg] = v;
  }
}

// ---------------------------------------------------------------- tensor-core dense layers
// The 64 x 64 layers run on the tensor cores: mma.sync m16n8k16, BF16 operands, FP32
// accumulation.  Weights are BF16 already.  Activations are FP32; each is split into
// hi = bf16(v) and lo = bf16(v - hi), and a product with a weight is taken as hi*w + lo*w
// (both exact in FP32), which keeps 16 significant bits of v.  In the weight gradient both
// operands are FP32 activations: dZ^T X is taken as Zhi Xhi + Zhi Xlo + Zlo Xhi.
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4):
//   A (16 x 16, row-major)  a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]
//   B (16 x 8, k-major)     b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C (16 x 8, FP32)        c0, c1 = C[g][2t], C[g][2t+1];  c2, c3 = C[g+8][2t], C[g+8][2t+1]
// (a register holds two BF16, the lower column / row index in the low half).
constexpr int MMA_WARPS = 8;                     // warps per block, 16 rows each
constexpr int MMA_ROWS = MMA_WARPS * 16;         // rows per block of the dense kernels
// Resident blocks per SM of the persistent dense kernels: they are bound by load latency
// (ncu: long-scoreboard stalls, DRAM 17-20 % busy at two blocks per SM), so the register
// budget is set for three.
constexpr int MMA_BLOCKS_PER_SM = 3;
constexpr int WPAD = H + 8;                      // shared row stride (BF16): conflict-free fragments

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat162 v) {
  return *reinterpret_cast<uint32_t*>(&v);
}

// hi and lo BF16 pairs of two FP32 values (the first in the low half)
__device__ __forceinline__ void split2(float2 v, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const float2 hf = __bfloat1622float2(h);
  hi = pack_bf16(h);
  lo = pack_bf16(__floats2bfloat162_rn(v.x - hf.x, v.y - hf.y));
}

// Stage W[H][H] (BF16) as S[n][k] = W[n][k] (transpose = false) or W[k][n] (true), eight
// weights per 16-byte load, every thread's loads issued before its stores (W is 16-byte
// aligned: each weight block of the parameter vector starts at a multiple of 8 entries).
__device__ __forceinline__ void stage_w_bf16(__nv_bfloat16 (*S)[WPAD], const __nv_bfloat16* W,
                                             bool transpose) {
  constexpr int V = H * H / 8, PER = V / (MMA_WARPS * 32);  // 512 vectors, 2 per thread
  const uint4* W4 = reinterpret_cast<const uint4*>(W);
  uint4 v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) v[u] = __ldg(W4 + threadIdx.x + u * MMA_WARPS * 32);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int q = threadIdx.x + u * MMA_WARPS * 32, r = (8 * q) / H, c = (8 * q) % H;
    if (!transpose) {
      *reinterpret_cast<uint4*>(&S[r][c]) = v[u];
    } else {
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v[u]);
#pragma unroll
      for (int j = 0; j < 8; ++j) S[c + j][r] = e[j];
    }
  }
}
static_assert((H * H / 8) % (MMA_WARPS * 32) == 0, "weight staging: whole vectors per thread");
static_assert((WPAD * 2) % 16 == 0, "weight staging: 16-byte aligned shared rows");

// B fragments of n-tile j, k-step kk from S[n][k]
__device__ __forceinline__ void b_frag(const __nv_bfloat16 (*S)[WPAD], int j, int kk, int g,
                                       int t, uint32_t& b0, uint32_t& b1) {
  b0 = *reinterpret_cast<const uint32_t*>(&S[8 * j + g][16 * kk + 2 * t]);
  b1 = *reinterpret_cast<const uint32_t*>(&S[8 * j + g][16 * kk + 2 * t + 8]);
}

// The four FP32 pairs behind the A fragment of k-step kk of the 16-row tile at row r0 of
// X[N][H] (rows >= N: 0), in fragment order.
__device__ __forceinline__ void a_frag_load(const float* X, int r0, int N, int kk, int g, int t,
                                            float2 (&v)[4]) {
  const int ra = r0 + g, rb = r0 + g + 8, c = 16 * kk + 2 * t;
  const float2 z = make_float2(0.f, 0.f);
  v[0] = ra < N ? *reinterpret_cast<const float2*>(X + (size_t)ra * H + c) : z;
  v[1] = rb < N ? *reinterpret_cast<const float2*>(X + (size_t)rb * H + c) : z;
  v[2] = ra < N ? *reinterpret_cast<const float2*>(X + (size_t)ra * H + c + 8) : z;
  v[3] = rb < N ? *reinterpret_cast<const float2*>(X + (size_t)rb * H + c + 8) : z;
}

// out = relu(X1 W1^T + X2 W2^T + b) for X1, X2 [N][H], W1, W2 [H][H]: each warp one 16-row
// tile, all 64 output columns (8 n-tiles), both products into the same accumulators.
__global__ void __launch_bounds__(MMA_WARPS * 32, MMA_BLOCKS_PER_SM) linear_mma_kernel(
    int N, const float* __restrict__ X1, const __nv_bfloat16* __restrict__ W1,
    const float* __restrict__ X2, const __nv_bfloat16* __restrict__ W2,
    const float* __restrict__ b, float* out) {
  __shared__ __align__(16) __nv_bfloat16 S1[H][WPAD];
  __shared__ __align__(16) __nv_bfloat16 S2[H][WPAD];
  stage_w_bf16(S1, W1, false);
  stage_w_bf16(S2, W2, false);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // persistent over row tiles: the weights are staged once per block
  for (int tile = blockIdx.x; tile * MMA_ROWS < N; tile += gridDim.x) {
  const int r0 = tile * MMA_ROWS + w * 16;
  if (r0 >= N) break;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  float2 v[2][H / 16][4];  // the warp's 16 rows of X1 and X2, all loads in flight together
#pragma unroll
  for (int kk = 0; kk < H / 16; ++kk) {
    a_frag_load(X1, r0, N, kk, g, t, v[0][kk]);
    a_frag_load(X2, r0, N, kk, g, t, v[1][kk]);
  }
#pragma unroll
  for (int which = 0; which < 2; ++which) {
    const __nv_bfloat16(*S)[WPAD] = which ? S2 : S1;
#pragma unroll
    for (int kk = 0; kk < H / 16; ++kk) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) split2(v[which][kk][q], hi[q], lo[q]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b0, b1;
        b_frag(S, j, kk, g, t, b0, b1);
        mma_bf16(acc[j], hi, b0, b1);
        mma_bf16(acc[j], lo, b0, b1);
      }
    }
  }
  const int ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = 8 * j + 2 * t;
    const float b0 = b[c], b1 = b[c + 1];
    if (ra < N)
      *reinterpret_cast<float2*>(out + (size_t)ra * H + c) =
          make_float2(fmaxf(acc[j][0] + b0, 0.f), fmaxf(acc[j][1] + b1, 0.f));
    if (rb < N)
      *reinterpret_cast<float2*>(out + (size_t)rb * H + c) =
          make_float2(fmaxf(acc[j][2] + b0, 0.f), fmaxf(acc[j][3] + b1, 0.f));
  }
  }
}

// Backward of out = relu(X1 W1^T + X2 W2^T + b): dZ = dOut * [out > 0] (stored), then
// dX1 = dZ W1 and dX2 = dZ W2 ([N][H] each) on the tensor cores.
__global__ void __launch_bounds__(MMA_WARPS * 32, MMA_BLOCKS_PER_SM) linear_bwd_mma_kernel(
    int N, const float* __restrict__ dOut, const float* __restrict__ Hout,
    const __nv_bfloat16* __restrict__ W1, const __nv_bfloat16* __restrict__ W2, float* dZ,
    float* dX1, float* dX2) {
  __shared__ __align__(16) __nv_bfloat16 S1[H][WPAD];
  __shared__ __align__(16) __nv_bfloat16 S2[H][WPAD];
  const bool products = W1 != nullptr;  // without weights: the ReLU mask only (dZ)
  if (products) {
    stage_w_bf16(S1, W1, true);  // B[o][k] = W[o][k] read as S[n = k][o]
    stage_w_bf16(S2, W2, true);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // persistent over row tiles: the weights are staged once per block
  for (int tile = blockIdx.x; tile * MMA_ROWS < N; tile += gridDim.x) {
  const int r0 = tile * MMA_ROWS + w * 16;
  if (r0 >= N) break;
  const int ra = r0 + g, rb = r0 + g + 8;
  float2 dv[H / 16][4], hv[H / 16][4];  // every load of the warp's rows before any store
#pragma unroll
  for (int kk = 0; kk < H / 16; ++kk) {
    a_frag_load(dOut, r0, N, kk, g, t, dv[kk]);
    a_frag_load(Hout, r0, N, kk, g, t, hv[kk]);
  }
  uint32_t hi[H / 16][4], lo[H / 16][4];
#pragma unroll
  for (int kk = 0; kk < H / 16; ++kk) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = (q & 1) ? rb : ra;
      const int c = 16 * kk + 2 * t + ((q & 2) ? 8 : 0);
      const float2 d = dv[kk][q], h = hv[kk][q];
      const float2 z = make_float2(h.x > 0.f ? d.x : 0.f, h.y > 0.f ? d.y : 0.f);
      if (r < N) *reinterpret_cast<float2*>(dZ + (size_t)r * H + c) = z;
      split2(z, hi[kk][q], lo[kk][q]);
    }
  }
  if (!products) continue;
#pragma unroll
  for (int which = 0; which < 2; ++which) {
    float* dX = which ? dX2 : dX1;
    const __nv_bfloat16(*S)[WPAD] = which ? S2 : S1;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
#pragma unroll
    for (int kk = 0; kk < H / 16; ++kk) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t b0, b1;
        b_frag(S, j, kk, g, t, b0, b1);
        mma_bf16(acc[j], hi[kk], b0, b1);
        mma_bf16(acc[j], lo[kk], b0, b1);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t;
      if (ra < N) *reinterpret_cast<float2*>(dX + (size_t)ra * H + c) = make_float2(acc[j][0], acc[j][1]);
      if (rb < N) *reinterpret_cast<float2*>(dX + (size_t)rb * H + c) = make_float2(acc[j][2], acc[j][3]);
    }
  }
  }
}

// Weight gradients dW1 = dZ^T X1, dW2 = dZ^T X2 (H x H each) and the bias gradient sum_r dZ[r]
// of one layer on the tensor cores: partial[block] = [dW1 | dW2 | bias] (2 H H + H floats,
// the parameter order of a round) over the block's 64-row tiles (tiles t = block, block +
// grid, ...), added in block order by reduce_partials_kernel.  Each tile is staged transposed
// in shared memory as BF16 hi / lo pairs: ZT[o][r] once, then X1T[k][r] and X2T[k][r] in turn
// through the same buffer.  Warp w owns the output rows o = 16 (w % 4) .. + 15 and the
// n-tiles 4 (w / 4) .. + 3 of both products.
constexpr int WG_TILE = 64;
constexpr int WG_PAIRS = WG_TILE / 2 / 4;  // row pairs per staging thread (4 threads per column)
__device__ __forceinline__ void wg_stage(__nv_bfloat16 (*Th)[WPAD], __nv_bfloat16 (*Tl)[WPAD],
                                         const float* __restrict__ X, int r0, int N, int col,
                                         int pr, float* colsum) {
  float a[WG_PAIRS], b[WG_PAIRS];
#pragma unroll
  for (int u = 0; u < WG_PAIRS; ++u) {  // every load first
    const int ra = r0 + 2 * (pr + 4 * u), rb = ra + 1;
    a[u] = ra < N ? X[(size_t)ra * H + col] : 0.f;
    b[u] = rb < N ? X[(size_t)rb * H + col] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < WG_PAIRS; ++u) {
    const int p = pr + 4 * u;
    if (colsum) {
      *colsum += a[u];
      *colsum += b[u];
    }
    uint32_t h, l;
    split2(make_float2(a[u], b[u]), h, l);
    *reinterpret_cast<uint32_t*>(&Th[col][2 * p]) = h;
    *reinterpret_cast<uint32_t*>(&Tl[col][2 * p]) = l;
  }
}

__device__ __forceinline__ void wg_mma(const __nv_bfloat16 (*ZTh)[WPAD], const __nv_bfloat16 (*ZTl)[WPAD],
                                       const __nv_bfloat16 (*XTh)[WPAD], const __nv_bfloat16 (*XTl)[WPAD],
                                       int mt, int nh, int g, int t, float (&acc)[4][4]) {
#pragma unroll
  for (int kk = 0; kk < WG_TILE / 16; ++kk) {
    uint32_t ah[4], al[4];
    const int o = 16 * mt + g, c = 16 * kk + 2 * t;
    ah[0] = *reinterpret_cast<const uint32_t*>(&ZTh[o][c]);
    ah[1] = *reinterpret_cast<const uint32_t*>(&ZTh[o + 8][c]);
    ah[2] = *reinterpret_cast<const uint32_t*>(&ZTh[o][c + 8]);
    ah[3] = *reinterpret_cast<const uint32_t*>(&ZTh[o + 8][c + 8]);
    al[0] = *reinterpret_cast<const uint32_t*>(&ZTl[o][c]);
    al[1] = *reinterpret_cast<const uint32_t*>(&ZTl[o + 8][c]);
    al[2] = *reinterpret_cast<const uint32_t*>(&ZTl[o][c + 8]);
    al[3] = *reinterpret_cast<const uint32_t*>(&ZTl[o + 8][c + 8]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 8 * (4 * nh + j) + g;
      const uint32_t bh0 = *reinterpret_cast<const uint32_t*>(&XTh[k][c]);
      const uint32_t bh1 = *reinterpret_cast<const uint32_t*>(&XTh[k][c + 8]);
      const uint32_t bl0 = *reinterpret_cast<const uint32_t*>(&XTl[k][c]);
      const uint32_t bl1 = *reinterpret_cast<const uint32_t*>(&XTl[k][c + 8]);
      mma_bf16(acc[j], ah, bh0, bh1);
      mma_bf16(acc[j], ah, bl0, bl1);
      mma_bf16(acc[j], al, bh0, bh1);
    }
  }
}

__device__ __forceinline__ void wg_store(float* p, int mt, int nh, int g, int t,
                                         const float (&acc)[4][4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = 8 * (4 * nh + j) + 2 * t, o = 16 * mt + g;
    *reinterpret_cast<float2*>(p + (size_t)o * H + k) = make_float2(acc[j][0], acc[j][1]);
    *reinterpret_cast<float2*>(p + (size_t)(o + 8) * H + k) = make_float2(acc[j][2], acc[j][3]);
  }
}

constexpr int WG_STRIDE = 2 * H * H + H;  // floats per block partial
__global__ void __launch_bounds__(MMA_WARPS * 32) wgrad_mma_kernel(int N,
                                                                  const float* __restrict__ dZ,
                                                                  const float* __restrict__ X1,
                                                                  const float* __restrict__ X2,
                                                                  float* __restrict__ partial) {
  __shared__ __align__(16) __nv_bfloat16 ZTh[H][WPAD], ZTl[H][WPAD], XTh[H][WPAD], XTl[H][WPAD];
  __shared__ float bsum[4][H];
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int mt = w & 3, nh = w >> 2;
  const int col = tid & (H - 1), pr = tid >> 6;  // staging: column, first row pair
  float acc1[4][4], acc2[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc1[j][q] = acc2[j][q] = 0.f;
  float bacc = 0.f;
  for (int tile = blockIdx.x; tile * WG_TILE < N; tile += gridDim.x) {
    const int r0 = tile * WG_TILE;
    __syncthreads();  // the previous tile's fragments are read
    wg_stage(ZTh, ZTl, dZ, r0, N, col, pr, &bacc);
    wg_stage(XTh, XTl, X1, r0, N, col, pr, nullptr);
    __syncthreads();
    wg_mma(ZTh, ZTl, XTh, XTl, mt, nh, g, t, acc1);
    __syncthreads();  // X1's fragments are read
    wg_stage(XTh, XTl, X2, r0, N, col, pr, nullptr);
    __syncthreads();
    wg_mma(ZTh, ZTl, XTh, XTl, mt, nh, g, t, acc2);
  }
  float* p = partial + (size_t)blockIdx.x * WG_STRIDE;
  wg_store(p, mt, nh, g, t, acc1);
  wg_store(p + H * H, mt, nh, g, t, acc2);
  bsum[pr][col] = bacc;
  __syncthreads();
  if (tid < H) p[2 * H * H + tid] = ((bsum[0][tid] + bsum[1][tid]) + bsum[2][tid]) + bsum[3][tid];
}

// The 8-wide input encoders' gradients: dW = dZ^T X (H x F) and the bias, partial[block] =
// [dW | bias] (H F + H floats), read by reduce_partials_kernel; one n8 tile, warps 0..3 own
// the output rows 16 w .. + 15, all warps stage.  Same BF16 splits as wgrad_mma_kernel.
__global__ void __launch_bounds__(MMA_WARPS * 32) wgrad8_mma_kernel(int N,
                                                                   const float* __restrict__ dZ,
                                                                   const float* __restrict__ X,
                                                                   float* __restrict__ partial) {
  __shared__ __align__(16) __nv_bfloat16 ZTh[H][WPAD], ZTl[H][WPAD], XTh[F][WPAD], XTl[F][WPAD];
  __shared__ float bsum[4][H];
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int col = tid & (H - 1), pr = tid >> 6;
  const int c8 = tid & (F - 1), p8 = tid / F;  // X staging: column, row pair (256 = 8 x 32)
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  for (int tile = blockIdx.x; tile * WG_TILE < N; tile += gridDim.x) {
    const int r0 = tile * WG_TILE;
    __syncthreads();
    wg_stage(ZTh, ZTl, dZ, r0, N, col, pr, &bacc);
    {
      const int ra = r0 + 2 * p8, rb = ra + 1;
      const float xa = ra < N ? X[(size_t)ra * F + c8] : 0.f;
      const float xb = rb < N ? X[(size_t)rb * F + c8] : 0.f;
      uint32_t h, l;
      split2(make_float2(xa, xb), h, l);
      *reinterpret_cast<uint32_t*>(&XTh[c8][2 * p8]) = h;
      *reinterpret_cast<uint32_t*>(&XTl[c8][2 * p8]) = l;
    }
    __syncthreads();
    if (w < 4) {
#pragma unroll
      for (int kk = 0; kk < WG_TILE / 16; ++kk) {
        uint32_t ah[4], al[4];
        const int o = 16 * w + g, c = 16 * kk + 2 * t;
        ah[0] = *reinterpret_cast<const uint32_t*>(&ZTh[o][c]);
        ah[1] = *reinterpret_cast<const uint32_t*>(&ZTh[o + 8][c]);
        ah[2] = *reinterpret_cast<const uint32_t*>(&ZTh[o][c + 8]);
        ah[3] = *reinterpret_cast<const uint32_t*>(&ZTh[o + 8][c + 8]);
        al[0] = *reinterpret_cast<const uint32_t*>(&ZTl[o][c]);
        al[1] = *reinterpret_cast<const uint32_t*>(&ZTl[o + 8][c]);
        al[2] = *reinterpret_cast<const uint32_t*>(&ZTl[o][c + 8]);
        al[3] = *reinterpret_cast<const uint32_t*>(&ZTl[o + 8][c + 8]);
        const uint32_t bh0 = *reinterpret_cast<const uint32_t*>(&XTh[g][c]);
        const uint32_t bh1 = *reinterpret_cast<const uint32_t*>(&XTh[g][c + 8]);
        const uint32_t bl0 = *reinterpret_cast<const uint32_t*>(&XTl[g][c]);
        const uint32_t bl1 = *reinterpret_cast<const uint32_t*>(&XTl[g][c + 8]);
        mma_bf16(acc, ah, bh0, bh1);
        mma_bf16(acc, ah, bl0, bl1);
        mma_bf16(acc, al, bh0, bh1);
      }
    }
  }
  float* pp = partial + (size_t)blockIdx.x * (H * F + H);
  if (w < 4) {
    const int o = 16 * w + g, k = 2 * t;
    *reinterpret_cast<float2*>(pp + (size_t)o * F + k) = make_float2(acc[0], acc[1]);
    *reinterpret_cast<float2*>(pp + (size_t)(o + 8) * F + k) = make_float2(acc[2], acc[3]);
  }
  bsum[pr][col] = bacc;
  __syncthreads();
  if (tid < H) pp[H * F + tid] = ((bsum[0][tid] + bsum[1][tid]) + bsum[2][tid]) + bsum[3][tid];
}

// grad[e] += sum over blocks g of partial[g * stride + e], e < len: a block takes 32
// consecutive e and RP_SLICES slices of g (slice q: g = q, q + RP_SLICES, ... in order, loads
// batched), then adds the slices' sums in slice order.  Fixed order: reproducible.
constexpr int RP_E = 32, RP_SLICES = 8, RP_BATCH = 8;
__global__ void __launch_bounds__(RP_E * RP_SLICES) reduce_partials_kernel(
    int G, int len, int stride, const float* __restrict__ partial, float* grad) {
  __shared__ float part[RP_SLICES][RP_E];
  const int ex = threadIdx.x % RP_E, q = threadIdx.x / RP_E;
  const int e = blockIdx.x * RP_E + ex;
  float acc = 0.f;
  if (e < len) {
    for (int g = q; g < G; g += RP_SLICES * RP_BATCH) {
      float v[RP_BATCH];
#pragma unroll
      for (int u = 0; u < RP_BATCH; ++u) {
        const int gg = g + u * RP_SLICES;
        v[u] = gg < G ? partial[(size_t)gg * stride + e] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < RP_BATCH; ++u)
        if (g + u * RP_SLICES < G) acc += v[u];
    }
  }
  part[q][ex] = acc;
  __syncthreads();
  if (q == 0 && e < len) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < RP_SLICES; ++k) s += part[k][ex];
    grad[e] += s;
  }
}
int reduce_grid(int len) { return (len + RP_E - 1) / RP_E; }

// out[r] = Hm[r] . w + b (warp per row, fixed shuffle tree).
__global__ void __launch_bounds__(TPB) head_kernel(int N, const float* __restrict__ Hm,
                                                   const __nv_bfloat16* __restrict__ w,
                                                   const float* __restrict__ b, float* out) {
  const int r = (int)((blockIdx.x * (size_t)TPB + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= N) return;
  const float2 h = reinterpret_cast<const float2*>(Hm + (size_t)r * H)[lane];
  float p = fmaf(h.x, __bfloat162float(w[2 * lane]), h.y * __bfloat162float(w[2 * lane + 1]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  if (lane == 0) out[r] = p + b[0];
}

// d[r] = 2 (out[r] - t[r]) / N, dH[r][:] = d[r] w, loss_part[block] = sum (out - t)^2 / N.
__global__ void __launch_bounds__(TPB) head_bwd_kernel(int N, const float* __restrict__ out,
                                                       const float* __restrict__ tgt,
                                                       const __nv_bfloat16* __restrict__ w,
                                                       float* __restrict__ d, float* dH,
                                                       float* __restrict__ loss_part) {
  __shared__ float ls[TPB / 32];
  const int r = (int)((blockIdx.x * (size_t)TPB + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  float l = 0.f;
  if (r < N) {
    const float e = out[r] - tgt[r];
    const float dr = 2.f * e / (float)N;
    reinterpret_cast<float2*>(dH + (size_t)r * H)[lane] =
        make_float2(dr * __bfloat162float(w[2 * lane]), dr * __bfloat162float(w[2 * lane + 1]));
    if (lane == 0) {
      d[r] = dr;
      l = e * e / (float)N;
    }
  }
  if (lane == 0) ls[wi] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < TPB / 32; ++k) s += ls[k];
    loss_part[blockIdx.x] = s;
  }
}

// partial[block][k] = sum over the block's rows of d[r] Hm[r][k] (k < H), [H] = sum d[r].
// Thread (rg, c) of the 4 x 64 threads sums, over the block's tiles, the rows r = tile
// start + rg, + 4, ... of d[r] Hm[r][c] (and thread c = 0 also d[r], the bias gradient), the
// rows' loads batched; the four row groups are then added in order.  Fixed order.
constexpr int HW_GROUPS = TPB / H;  // 4 row groups of 64 columns
__global__ void __launch_bounds__(TPB) head_wgrad_kernel(int N, const float* __restrict__ d,
                                                         const float* __restrict__ Hm,
                                                         float* __restrict__ partial) {
  __shared__ float part[HW_GROUPS][H + 1];
  const int c = threadIdx.x % H, rg = threadIdx.x / H;
  constexpr int BATCH = 4;
  float acc = 0.f, bacc = 0.f;
  for (int tile = blockIdx.x; tile * TILE < N; tile += gridDim.x) {
    const int r1 = min(N, (tile + 1) * TILE);
    for (int r = tile * TILE + rg; r < r1; r += HW_GROUPS * BATCH) {
      float dv[BATCH], hv[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int rr = r + u * HW_GROUPS;
        dv[u] = rr < r1 ? d[rr] : 0.f;
        hv[u] = rr < r1 ? Hm[(size_t)rr * H + c] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        if (r + u * HW_GROUPS >= r1) break;
        acc = fmaf(dv[u], hv[u], acc);
        bacc += dv[u];
      }
    }
  }
  part[rg][c] = acc;
  if (c == 0) part[rg][H] = bacc;
  __syncthreads();
  if (threadIdx.x <= H) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < HW_GROUPS; ++k) s += part[k][threadIdx.x];
    partial[(size_t)blockIdx.x * (H + 1) + threadIdx.x] = s;
  }
}

// *out = sum of parts[0 .. G) in FP64: thread t adds parts t, t + SP_THREADS, ... in order
// (loads batched), then a fixed tree over the threads.
constexpr int SP_THREADS = 1024;
__global__ void __launch_bounds__(SP_THREADS) sum_parts_kernel(int G, const float* __restrict__ parts,
                                                               double* out) {
  __shared__ double red[SP_THREADS / 32];
  double s = 0.0;
  constexpr int BATCH = 8;
  for (int g = threadIdx.x; g < G; g += SP_THREADS * BATCH) {
    float v[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int gg = g + u * SP_THREADS;
      v[u] = gg < G ? parts[gg] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) s += (double)v[u];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < SP_THREADS / 32; ++k) t += red[k];
    *out = t;
  }
}

// Adam's step scalars [lr, beta1, beta2, eps, 1 - beta1^step, 1 - beta2^step] are read from
// device memory, so a captured training step can be replayed with new ones.
constexpr int ADAM_SCALARS = 6;
__global__ void adam_kernel(int64_t P, float* theta, float* grad, float* m1, float* m2,
                            const float* __restrict__ sc, __nv_bfloat16* wbf) {
  const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (i >= P) return;
  const float lr = sc[0], b1 = sc[1], b2 = sc[2], eps = sc[3], bc1 = sc[4], bc2 = sc[5];
  const float g = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float v = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  const float th = theta[i] - lr * (a / bc1) / (sqrtf(v / bc2) + eps);
  theta[i] = th;
  wbf[i] = __float2bfloat16_rn(th);
  grad[i] = 0.f;
}

__global__ void to_bf16_kernel(int64_t P, const float* theta, __nv_bfloat16* wbf) {
  const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (i < P) wbf[i] = __float2bfloat16_rn(theta[i]);
}

}  // namespace

// ---------------------------------------------------------------- handle
struct dpdlp_gnn {
  int device = 0;
  cudaStream_t stream = nullptr;
  // backward: the weight gradients (the users of `partial`) run on a second stream beside the
  // data-gradient chain; ev_z* are recorded after a dZ buffer is written (main stream),
  // ev_w* after the gradient pass that reads it (side stream)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_zv = nullptr, ev_zc = nullptr, ev_wv = nullptr, ev_wc = nullptr;
  // a whole training step (forward, backward, Adam) captured once per graph and replayed
  cudaGraphExec_t step_exec = nullptr;
  float* adam_sc = nullptr;  // [ADAM_SCALARS] on the device
  float adam_host[8] = {};
  std::string err;
  int ptr_dev = 0;
  int n = 0, m = 0;
  bool graph = false, fwd_done = false;
  std::vector<void*> allocs;  // graph-dependent buffers
  // A (m rows): R values (row-normalised) and Ct values (A D_c^-1, for C^T in backward);
  // A^T (n rows): C values (column-normalised) and Rt values (A^T D_r^-1, for R^T)
  int64_t *a_ptr = nullptr, *t_ptr = nullptr;
  int *a_long = nullptr, *t_long = nullptr;  // rows longer than SPMM_LONG of A and of A^T
  int na_long = 0, nt_long = 0;
  int *a_idx = nullptr, *t_idx = nullptr;
  float *a_R = nullptr, *a_Ct = nullptr, *t_C = nullptr, *t_Rt = nullptr;
  float *Fv = nullptr, *Fc = nullptr, *tx = nullptr, *ty = nullptr;
  float* hv[L + 1] = {};
  float* hc[L + 1] = {};
  float* gv[L] = {};
  float* gc[L] = {};
  float *xhat = nullptr, *yhat = nullptr;
  float *dhv[2] = {}, *dhc[2] = {}, *dzv = nullptr, *dzc = nullptr, *dgv = nullptr, *dgc = nullptr;
  float *dx = nullptr, *dy = nullptr, *loss_part = nullptr;
  double* loss_d = nullptr;
  // parameters (graph-independent)
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *partial = nullptr;
  __nv_bfloat16* wbf = nullptr;
};

namespace {

int gfail(dpdlp_gnn* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  return code;
}

#define GCK(call)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return gfail(g, e_ == cudaErrorMemoryAllocation ? DPDLP_ERR_OOM : DPDLP_ERR_CUDA, \
                   std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

template <class T>
int galloc(dpdlp_gnn* g, T** p, size_t count) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, (count > 0 ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return gfail(g, DPDLP_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  g->allocs.push_back(*p);
  return 0;
}

void free_graph_buffers(dpdlp_gnn* g) {
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->step_exec) cudaGraphExecDestroy(g->step_exec);
  g->step_exec = nullptr;
  for (void* p : g->allocs) cudaFree(p);
  g->allocs.clear();
  g->graph = false;
  g->fwd_done = false;
}

int blocks_for_rows(int rows) { return (rows + TILE - 1) / TILE; }
// persistent dense kernels: at most MMA_BLOCKS_PER_SM blocks per SM, each looping over
// 128-row tiles
int mma_blocks(int rows) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int tiles = (rows + MMA_ROWS - 1) / MMA_ROWS, most = MMA_BLOCKS_PER_SM * sms;
  return tiles < most ? (tiles > 0 ? tiles : 1) : most;
}
int warp_blocks(int rows) { return (int)(((size_t)rows * 32 + TPB - 1) / TPB); }
int wg_grid(int rows) {
  const int b = blocks_for_rows(rows);
  return b < WG_BLOCKS ? (b > 0 ? b : 1) : WG_BLOCKS;
}

cudaMemcpyKind in_kind(const dpdlp_gnn* g) {
  return g->ptr_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind out_kind(const dpdlp_gnn* g) {
  return g->ptr_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// weight gradient of one layer: grad[off .. off + H*K) += dZ^T X and, with_bias, the next
// H entries (the bias that follows the weight in the parameter order) += column sums of dZ
// out (=|+=) the aggregation over A's rows (transpose = false) or A^T's rows with the value
// array `val`: a warp per short row, a block per long row.
void spmm(dpdlp_gnn* g, bool transpose, const float* val, const float* in, float* out,
          int accumulate) {
  const int rows = transpose ? g->n : g->m;
  if (rows == 0) return;
  const int64_t* ptr = transpose ? g->t_ptr : g->a_ptr;
  const int* idx = transpose ? g->t_idx : g->a_idx;
  spmm_kernel<<<spmm_blocks(rows), TPB, 0, g->stream>>>(rows, ptr, idx, val, in, out, accumulate);
  const int nl = transpose ? g->nt_long : g->na_long;
  if (nl > 0)
    spmm_long_kernel<<<nl, SPMM_LONG_WARPS * 32, 0, g->stream>>>(transpose ? g->t_long : g->a_long,
                                                                ptr, idx, val, in, out, accumulate);
}

// both weight gradients and the bias gradient of a round's layer: grad[off ..) += [dZ^T X1 |
// dZ^T X2 | column sums of dZ] (the parameter order U, V, b)
int add_wgrad2(dpdlp_gnn* g, int N, const float* dZ, const float* X1, const float* X2, int64_t off) {
  const int G = wg_grid(N);
  wgrad_mma_kernel<<<G, MMA_WARPS * 32, 0, g->side>>>(N, dZ, X1, X2, g->partial);
  reduce_partials_kernel<<<reduce_grid(WG_STRIDE), RP_E * RP_SLICES, 0, g->side>>>(
      G, WG_STRIDE, WG_STRIDE, g->partial, g->grad + off);
  GCK(cudaGetLastError());
  return 0;
}

// an input encoder's weight and bias gradients: grad[off ..) += [dZ^T X | column sums of dZ]
int add_wgrad8(dpdlp_gnn* g, int N, const float* dZ, const float* X, int64_t off) {
  const int G = wg_grid(N);
  const int stride = H * F + H;
  const int len = stride;
  wgrad8_mma_kernel<<<G, MMA_WARPS * 32, 0, g->side>>>(N, dZ, X, g->partial);
  reduce_partials_kernel<<<reduce_grid(len), RP_E * RP_SLICES, 0, g->side>>>(G, len, stride, g->partial,
                                                                      g->grad + off);
  GCK(cudaGetLastError());
  return 0;
}

// The forward pass's kernels on g->stream (no copies, no synchronization).
int enqueue_forward(dpdlp_gnn* g) {
  const int n = g->n, m = g->m;
  cudaStream_t s = g->stream;
  const float* th = g->theta;
  const __nv_bfloat16* w = g->wbf;
  if (n) linear_kernel<F, false><<<blocks_for_rows(n), TPB, 0, s>>>(n, g->Fv, w + LAY.Ev, nullptr, nullptr, th + LAY.ev, g->hv[0]);
  if (m) linear_kernel<F, false><<<blocks_for_rows(m), TPB, 0, s>>>(m, g->Fc, w + LAY.Ec, nullptr, nullptr, th + LAY.ec, g->hc[0]);
  for (int l = 0; l < L; ++l) {
    if (m) {
      spmm(g, false, g->a_R, g->hv[l], g->gc[l], 0);
      linear_mma_kernel<<<mma_blocks(m), MMA_WARPS * 32, 0, s>>>(m, g->hc[l], w + LAY.Uc[l], g->gc[l], w + LAY.Vc[l], th + LAY.bc[l], g->hc[l + 1]);
    }
    if (n) {
      spmm(g, true, g->t_C, g->hc[l + 1], g->gv[l], 0);
      linear_mma_kernel<<<mma_blocks(n), MMA_WARPS * 32, 0, s>>>(n, g->hv[l], w + LAY.Uv[l], g->gv[l], w + LAY.Vv[l], th + LAY.bv[l], g->hv[l + 1]);
    }
  }
  if (n) head_kernel<<<warp_blocks(n), TPB, 0, s>>>(n, g->hv[L], w + LAY.wx, th + LAY.bx, g->xhat);
  if (m) head_kernel<<<warp_blocks(m), TPB, 0, s>>>(m, g->hc[L], w + LAY.wy, th + LAY.by, g->yhat);
  GCK(cudaGetLastError());
  return 0;
}

// The backward pass's kernels (targets already in g->tx, g->ty): the data-gradient chain on
// g->stream, the weight gradients on g->side, joined back into g->stream at the end.
int enqueue_backward(dpdlp_gnn* g) {
  const int n = g->n, m = g->m;
  cudaStream_t s = g->stream;
  const __nv_bfloat16* w = g->wbf;
  int cv = 0, cc = 0;  // dhv[cv], dhc[cc]: gradients of the current hv, hc (the heads write all rows)
  const int gx = n ? warp_blocks(n) : 0, gy = m ? warp_blocks(m) : 0;
  // The weight gradients run on g->side, in order (they share `partial`); before the main
  // stream rewrites a dZ buffer it waits for the side pass that reads it.
  cudaStream_t side = g->side;
  GCK(cudaEventRecord(g->ev_zv, s));  // the side stream starts after the targets are in
  GCK(cudaStreamWaitEvent(side, g->ev_zv, 0));
  if (n) {
    head_bwd_kernel<<<gx, TPB, 0, s>>>(n, g->xhat, g->tx, w + LAY.wx, g->dx, g->dhv[0], g->loss_part);
    GCK(cudaEventRecord(g->ev_zv, s));
    GCK(cudaStreamWaitEvent(side, g->ev_zv, 0));
    const int G = wg_grid(n);
    head_wgrad_kernel<<<G, TPB, 0, side>>>(n, g->dx, g->hv[L], g->partial);
    reduce_partials_kernel<<<reduce_grid(H + 1), RP_E * RP_SLICES, 0, side>>>(G, H + 1, H + 1, g->partial, g->grad + LAY.wx);
  }
  if (m) {
    head_bwd_kernel<<<gy, TPB, 0, s>>>(m, g->yhat, g->ty, w + LAY.wy, g->dy, g->dhc[0], g->loss_part + gx);
    GCK(cudaEventRecord(g->ev_zc, s));
    GCK(cudaStreamWaitEvent(side, g->ev_zc, 0));
    const int G = wg_grid(m);
    head_wgrad_kernel<<<G, TPB, 0, side>>>(m, g->dy, g->hc[L], g->partial);
    reduce_partials_kernel<<<reduce_grid(H + 1), RP_E * RP_SLICES, 0, side>>>(G, H + 1, H + 1, g->partial, g->grad + LAY.wy);
  }
  GCK(cudaEventRecord(g->ev_wv, side));
  GCK(cudaEventRecord(g->ev_wc, side));
  sum_parts_kernel<<<1, SP_THREADS, 0, s>>>(gx + gy, g->loss_part, g->loss_d);
  int rc;
  for (int l = L - 1; l >= 0; --l) {
    // variable update of round l: hv[l+1] = relu(hv[l] Uv^T + gv[l] Vv^T + bv), gv = C hc[l+1]
    if (n) {
      GCK(cudaStreamWaitEvent(s, g->ev_wv, 0));  // the previous pass over dzv is done
      linear_bwd_mma_kernel<<<mma_blocks(n), MMA_WARPS * 32, 0, s>>>(n, g->dhv[cv], g->hv[l + 1], w + LAY.Uv[l], w + LAY.Vv[l], g->dzv, g->dhv[1 - cv], g->dgv);
      GCK(cudaEventRecord(g->ev_zv, s));
      GCK(cudaStreamWaitEvent(side, g->ev_zv, 0));
      if ((rc = add_wgrad2(g, n, g->dzv, g->hv[l], g->gv[l], LAY.Uv[l]))) return rc;
      GCK(cudaEventRecord(g->ev_wv, side));
      if (m) spmm(g, false, g->a_Ct, g->dgv, g->dhc[cc], 1);
      cv = 1 - cv;
    }
    // constraint update of round l: hc[l+1] = relu(hc[l] Uc^T + gc[l] Vc^T + bc), gc = R hv[l]
    if (m) {
      GCK(cudaStreamWaitEvent(s, g->ev_wc, 0));  // the previous pass over dzc is done
      linear_bwd_mma_kernel<<<mma_blocks(m), MMA_WARPS * 32, 0, s>>>(m, g->dhc[cc], g->hc[l + 1], w + LAY.Uc[l], w + LAY.Vc[l], g->dzc, g->dhc[1 - cc], g->dgc);
      GCK(cudaEventRecord(g->ev_zc, s));
      GCK(cudaStreamWaitEvent(side, g->ev_zc, 0));
      if ((rc = add_wgrad2(g, m, g->dzc, g->hc[l], g->gc[l], LAY.Uc[l]))) return rc;
      GCK(cudaEventRecord(g->ev_wc, side));
      if (n) spmm(g, true, g->t_Rt, g->dgc, g->dhv[cv], 1);
      cc = 1 - cc;
    }
  }
  if (n) {
    GCK(cudaStreamWaitEvent(s, g->ev_wv, 0));
    linear_bwd_mma_kernel<<<mma_blocks(n), MMA_WARPS * 32, 0, s>>>(n, g->dhv[cv], g->hv[0], nullptr, nullptr, g->dzv, nullptr, nullptr);
    GCK(cudaEventRecord(g->ev_zv, s));
    GCK(cudaStreamWaitEvent(side, g->ev_zv, 0));
    if ((rc = add_wgrad8(g, n, g->dzv, g->Fv, LAY.Ev))) return rc;
  }
  if (m) {
    GCK(cudaStreamWaitEvent(s, g->ev_wc, 0));
    linear_bwd_mma_kernel<<<mma_blocks(m), MMA_WARPS * 32, 0, s>>>(m, g->dhc[cc], g->hc[0], nullptr, nullptr, g->dzc, nullptr, nullptr);
    GCK(cudaEventRecord(g->ev_zc, s));
    GCK(cudaStreamWaitEvent(side, g->ev_zc, 0));
    if ((rc = add_wgrad8(g, m, g->dzc, g->Fc, LAY.Ec))) return rc;
  }
  GCK(cudaEventRecord(g->ev_wv, side));  // every gradient is in before the backward returns
  GCK(cudaStreamWaitEvent(s, g->ev_wv, 0));
  GCK(cudaGetLastError());
  return 0;
}

int enqueue_adam(dpdlp_gnn* g) {
  const int64_t P = LAY.total;
  adam_kernel<<<(unsigned)((P + TPB - 1) / TPB), TPB, 0, g->stream>>>(P, g->theta, g->grad, g->m1,
                                                                      g->m2, g->adam_sc, g->wbf);
  GCK(cudaGetLastError());
  return 0;
}

// Adam's step scalars into the device buffer the adam kernel reads (stream-ordered).
int set_adam_scalars(dpdlp_gnn* g, double lr, double beta1, double beta2, double eps, int64_t step) {
  float* h = g->adam_host;
  h[0] = (float)lr;
  h[1] = (float)beta1;
  h[2] = (float)beta2;
  h[3] = (float)eps;
  h[4] = (float)(1.0 - std::pow(beta1, (double)step));
  h[5] = (float)(1.0 - std::pow(beta2, (double)step));
  GCK(cudaMemcpyAsync(g->adam_sc, h, ADAM_SCALARS * sizeof(float), cudaMemcpyHostToDevice, g->stream));
  return 0;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

int64_t dpdlp_gnn_param_count(void) { return LAY.total; }

int dpdlp_gnn_create(dpdlp_gnn_t** out, int device) {
  if (!out) return DPDLP_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return DPDLP_ERR_INVALID;
  for (int l = 0; l < L; ++l)  // the dense kernels stage weights with 16-byte loads
    if (LAY.Uc[l] % 8 || LAY.Vc[l] % 8 || LAY.Uv[l] % 8 || LAY.Vv[l] % 8) return DPDLP_ERR_INVALID;
  dpdlp_gnn* g = new (std::nothrow) dpdlp_gnn();
  if (!g) return DPDLP_ERR_OOM;
  g->device = device;
  const size_t P = (size_t)LAY.total;
  const size_t part = (size_t)WG_BLOCKS * WG_STRIDE;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_zv, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_zc, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_wv, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_wc, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&g->theta, P * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&g->grad, P * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&g->m1, P * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&g->m2, P * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&g->wbf, P * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&g->partial, part * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&g->adam_sc, ADAM_SCALARS * sizeof(float)) != cudaSuccess) {
    dpdlp_gnn_destroy(g);
    return DPDLP_ERR_CUDA;
  }
  cudaMemset(g->theta, 0, P * sizeof(float));
  cudaMemset(g->grad, 0, P * sizeof(float));
  cudaMemset(g->m1, 0, P * sizeof(float));
  cudaMemset(g->m2, 0, P * sizeof(float));
  cudaMemset(g->wbf, 0, P * sizeof(__nv_bfloat16));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    dpdlp_gnn_destroy(g);
    return DPDLP_ERR_CUDA;
  }
  *out = g;
  return 0;
}

void dpdlp_gnn_destroy(dpdlp_gnn_t* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  free_graph_buffers(g);
  void* ps[] = {g->theta, g->grad, g->m1, g->m2, g->wbf, g->partial, g->adam_sc};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (g->side) cudaStreamSynchronize(g->side);
  cudaEvent_t evs[] = {g->ev_zv, g->ev_zc, g->ev_wv, g->ev_wc};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (g->side) cudaStreamDestroy(g->side);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

const char* dpdlp_gnn_last_error(const dpdlp_gnn_t* g) { return g ? g->err.c_str() : "null handle"; }

int dpdlp_gnn_set_ptr_mode(dpdlp_gnn_t* g, int device) {
  if (!g || (device != 0 && device != 1)) return DPDLP_ERR_INVALID;
  g->ptr_dev = device;
  return 0;
}

int dpdlp_gnn_set_params(dpdlp_gnn_t* g, const float* params, int64_t count) {
  if (!g || !params || count != LAY.total) return gfail(g, DPDLP_ERR_INVALID, "params: count must be dpdlp_gnn_param_count()");
  GCK(cudaSetDevice(g->device));
  const size_t P = (size_t)LAY.total;
  GCK(cudaMemcpyAsync(g->theta, params, P * sizeof(float), cudaMemcpyHostToDevice, g->stream));
  GCK(cudaMemsetAsync(g->grad, 0, P * sizeof(float), g->stream));
  GCK(cudaMemsetAsync(g->m1, 0, P * sizeof(float), g->stream));
  GCK(cudaMemsetAsync(g->m2, 0, P * sizeof(float), g->stream));
  to_bf16_kernel<<<(unsigned)((P + TPB - 1) / TPB), TPB, 0, g->stream>>>((int64_t)P, g->theta, g->wbf);
  GCK(cudaGetLastError());
  GCK(cudaStreamSynchronize(g->stream));
  return 0;
}

int dpdlp_gnn_get_params(dpdlp_gnn_t* g, float* params, int64_t count) {
  if (!g || !params || count != LAY.total) return gfail(g, DPDLP_ERR_INVALID, "params: count must be dpdlp_gnn_param_count()");
  GCK(cudaSetDevice(g->device));
  GCK(cudaMemcpyAsync(params, g->theta, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
  GCK(cudaStreamSynchronize(g->stream));
  return 0;
}

int dpdlp_gnn_get_grads(dpdlp_gnn_t* g, float* grads, int64_t count) {
  if (!g || !grads || count != LAY.total) return gfail(g, DPDLP_ERR_INVALID, "grads: count must be dpdlp_gnn_param_count()");
  GCK(cudaSetDevice(g->device));
  GCK(cudaMemcpyAsync(grads, g->grad, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
  GCK(cudaStreamSynchronize(g->stream));
  return 0;
}

int dpdlp_gnn_zero_grads(dpdlp_gnn_t* g) {
  if (!g) return DPDLP_ERR_INVALID;
  GCK(cudaSetDevice(g->device));
  GCK(cudaMemsetAsync(g->grad, 0, (size_t)LAY.total * sizeof(float), g->stream));
  GCK(cudaStreamSynchronize(g->stream));
  return 0;
}

int dpdlp_gnn_set_graph(dpdlp_gnn_t* g, int32_t n, int32_t m, const int64_t* row_ptr,
                        const int32_t* col_idx, const double* val) {
  if (!g || n < 0 || m < 0 || !row_ptr) return gfail(g, DPDLP_ERR_INVALID, "graph: invalid arguments");
  const int64_t nnz = row_ptr[m];
  if (row_ptr[0] != 0 || nnz < 0 || (nnz > 0 && (!col_idx || !val)) || nnz > (int64_t)1 << 31)
    return gfail(g, DPDLP_ERR_INVALID, "graph: invalid row pointers");
  for (int i = 0; i < m; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return gfail(g, DPDLP_ERR_INVALID, "graph: row pointers decrease");
  for (int64_t k = 0; k < nnz; ++k)
    if (col_idx[k] < 0 || col_idx[k] >= n || !std::isfinite(val[k]))
      return gfail(g, DPDLP_ERR_INVALID, "graph: column index out of range or non-finite value");
  GCK(cudaSetDevice(g->device));
  free_graph_buffers(g);
  g->n = n;
  g->m = m;
  // row and column sums of |A|, then the four value arrays
  std::vector<double> rs(m, 0.0), cs(n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      rs[i] += std::fabs(val[k]);
      cs[col_idx[k]] += std::fabs(val[k]);
    }
  for (auto& v : rs) v = v > 1.0 ? v : 1.0;
  for (auto& v : cs) v = v > 1.0 ? v : 1.0;
  std::vector<float> aR(nnz), aCt(nnz);
  for (int i = 0; i < m; ++i)
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      aR[k] = (float)(val[k] / rs[i]);
      aCt[k] = (float)(val[k] / cs[col_idx[k]]);
    }
  // A^T by a stable counting sort (entries of a column in row order)
  std::vector<int64_t> tptr(n + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) ++tptr[col_idx[k] + 1];
  for (int j = 0; j < n; ++j) tptr[j + 1] += tptr[j];
  std::vector<int32_t> tidx(nnz);
  std::vector<float> tC(nnz), tRt(nnz);
  {
    std::vector<int64_t> pos(tptr.begin(), tptr.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        const int j = col_idx[k];
        const int64_t q = pos[j]++;
        tidx[q] = i;
        tC[q] = (float)(val[k] / cs[j]);
        tRt[q] = (float)(val[k] / rs[i]);
      }
  }
  std::vector<int> along, tlong;
  for (int i = 0; i < m; ++i)
    if (row_ptr[i + 1] - row_ptr[i] > SPMM_LONG) along.push_back(i);
  for (int j = 0; j < n; ++j)
    if (tptr[j + 1] - tptr[j] > SPMM_LONG) tlong.push_back(j);
  int rc;
  const size_t nH = (size_t)n * H, mH = (size_t)m * H;
  if ((rc = galloc(g, &g->a_long, along.size())) || (rc = galloc(g, &g->t_long, tlong.size())))
    return rc;
  g->na_long = (int)along.size();
  g->nt_long = (int)tlong.size();
  if ((rc = galloc(g, &g->a_ptr, m + 1)) || (rc = galloc(g, &g->t_ptr, n + 1)) ||
      (rc = galloc(g, &g->a_idx, nnz)) || (rc = galloc(g, &g->t_idx, nnz)) ||
      (rc = galloc(g, &g->a_R, nnz)) || (rc = galloc(g, &g->a_Ct, nnz)) ||
      (rc = galloc(g, &g->t_C, nnz)) || (rc = galloc(g, &g->t_Rt, nnz)))
    return rc;
  for (int l = 0; l <= L; ++l)
    if ((rc = galloc(g, &g->hv[l], nH)) || (rc = galloc(g, &g->hc[l], mH))) return rc;
  for (int l = 0; l < L; ++l)
    if ((rc = galloc(g, &g->gv[l], nH)) || (rc = galloc(g, &g->gc[l], mH))) return rc;
  if ((rc = galloc(g, &g->dhv[0], nH)) || (rc = galloc(g, &g->dhv[1], nH)) ||
      (rc = galloc(g, &g->dhc[0], mH)) || (rc = galloc(g, &g->dhc[1], mH)) ||
      (rc = galloc(g, &g->dzv, nH)) || (rc = galloc(g, &g->dzc, mH)) ||
      (rc = galloc(g, &g->dgv, nH)) || (rc = galloc(g, &g->dgc, mH)) ||
      (rc = galloc(g, &g->xhat, n)) || (rc = galloc(g, &g->yhat, m)) ||
      (rc = galloc(g, &g->dx, n)) || (rc = galloc(g, &g->dy, m)) ||
      (rc = galloc(g, &g->tx, n)) || (rc = galloc(g, &g->ty, m)) ||
      (rc = galloc(g, &g->Fv, (size_t)n * F)) || (rc = galloc(g, &g->Fc, (size_t)m * F)) ||
      (rc = galloc(g, &g->loss_part, warp_blocks(n) + warp_blocks(m) + 1)) ||
      (rc = galloc(g, &g->loss_d, 1)))
    return rc;
  auto up = [&](void* d, const void* h, size_t bytes) {
    return bytes ? cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  GCK(up(g->a_ptr, row_ptr, (m + 1) * sizeof(int64_t)));
  GCK(up(g->t_ptr, tptr.data(), (n + 1) * sizeof(int64_t)));
  GCK(up(g->a_idx, col_idx, nnz * sizeof(int32_t)));
  GCK(up(g->t_idx, tidx.data(), nnz * sizeof(int32_t)));
  GCK(up(g->a_R, aR.data(), nnz * sizeof(float)));
  GCK(up(g->a_Ct, aCt.data(), nnz * sizeof(float)));
  GCK(up(g->t_C, tC.data(), nnz * sizeof(float)));
  GCK(up(g->t_Rt, tRt.data(), nnz * sizeof(float)));
  GCK(up(g->a_long, along.data(), along.size() * sizeof(int)));
  GCK(up(g->t_long, tlong.data(), tlong.size() * sizeof(int)));
  g->graph = true;
  return 0;
}

int dpdlp_gnn_set_features(dpdlp_gnn_t* g, const float* fv, const float* fc) {
  if (!g || (g->n && !fv) || (g->m && !fc)) return gfail(g, DPDLP_ERR_INVALID, "features: NULL array");
  if (!g->graph) return gfail(g, DPDLP_ERR_NOT_LOADED, "no graph set");
  GCK(cudaSetDevice(g->device));
  if (g->n) GCK(cudaMemcpyAsync(g->Fv, fv, (size_t)g->n * F * sizeof(float), in_kind(g), g->stream));
  if (g->m) GCK(cudaMemcpyAsync(g->Fc, fc, (size_t)g->m * F * sizeof(float), in_kind(g), g->stream));
  g->fwd_done = false;
  return 0;
}

int dpdlp_gnn_forward(dpdlp_gnn_t* g, float* x_hat, float* y_hat) {
  if (!g) return DPDLP_ERR_INVALID;
  if (!g->graph) return gfail(g, DPDLP_ERR_NOT_LOADED, "no graph set");
  GCK(cudaSetDevice(g->device));
  int rc;
  if ((rc = enqueue_forward(g))) return rc;
  const int n = g->n, m = g->m;
  cudaStream_t s = g->stream;
  if (x_hat && n) GCK(cudaMemcpyAsync(x_hat, g->xhat, n * sizeof(float), out_kind(g), s));
  if (y_hat && m) GCK(cudaMemcpyAsync(y_hat, g->yhat, m * sizeof(float), out_kind(g), s));
  GCK(cudaStreamSynchronize(s));
  g->fwd_done = true;
  return 0;
}

int dpdlp_gnn_backward(dpdlp_gnn_t* g, const float* tx, const float* ty, double* loss) {
  if (!g || (g->n && !tx) || (g->m && !ty)) return gfail(g, DPDLP_ERR_INVALID, "backward: NULL target");
  if (!g->graph || !g->fwd_done) return gfail(g, DPDLP_ERR_INVALID, "backward needs a forward pass first");
  GCK(cudaSetDevice(g->device));
  const int n = g->n, m = g->m;
  cudaStream_t s = g->stream;
  if (n) GCK(cudaMemcpyAsync(g->tx, tx, n * sizeof(float), in_kind(g), s));
  if (m) GCK(cudaMemcpyAsync(g->ty, ty, m * sizeof(float), in_kind(g), s));
  int rc;
  if ((rc = enqueue_backward(g))) return rc;
  double lv = 0.0;
  GCK(cudaMemcpyAsync(&lv, g->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s));
  GCK(cudaStreamSynchronize(s));
  if (loss) *loss = lv;
  return 0;
}

int dpdlp_gnn_adam(dpdlp_gnn_t* g, double lr, double beta1, double beta2, double eps,
                   int64_t step) {
  if (!g || step < 1 || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) ||
      !(eps > 0))
    return gfail(g, DPDLP_ERR_INVALID, "adam: invalid hyper-parameters");
  GCK(cudaSetDevice(g->device));
  int rc;
  if ((rc = set_adam_scalars(g, lr, beta1, beta2, eps, step)) || (rc = enqueue_adam(g))) return rc;
  GCK(cudaStreamSynchronize(g->stream));
  return 0;
}

int dpdlp_gnn_train_step(dpdlp_gnn_t* g, const float* fv, const float* fc, const float* tx,
                         const float* ty, double lr, double beta1, double beta2, double eps,
                         int64_t step, double* loss) {
  if (!g || step < 1 || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) ||
      !(eps > 0))
    return gfail(g, DPDLP_ERR_INVALID, "train_step: invalid hyper-parameters");
  if (!g->graph) return gfail(g, DPDLP_ERR_NOT_LOADED, "no graph set");
  const int n = g->n, m = g->m;
  if ((n && (!fv || !tx)) || (m && (!fc || !ty)))
    return gfail(g, DPDLP_ERR_INVALID, "train_step: NULL features or targets");
  GCK(cudaSetDevice(g->device));
  cudaStream_t s = g->stream;
  if (n) GCK(cudaMemcpyAsync(g->Fv, fv, (size_t)n * F * sizeof(float), in_kind(g), s));
  if (m) GCK(cudaMemcpyAsync(g->Fc, fc, (size_t)m * F * sizeof(float), in_kind(g), s));
  if (n) GCK(cudaMemcpyAsync(g->tx, tx, n * sizeof(float), in_kind(g), s));
  if (m) GCK(cudaMemcpyAsync(g->ty, ty, m * sizeof(float), in_kind(g), s));
  int rc;
  if ((rc = set_adam_scalars(g, lr, beta1, beta2, eps, step))) return rc;
  if (!g->step_exec) {  // capture forward, backward (both streams) and Adam once per graph
    cudaGraph_t graph = nullptr;
    GCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_forward(g);
    if (!rc) rc = enqueue_backward(g);
    if (!rc) rc = enqueue_adam(g);
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    GCK(e);
    const cudaError_t ei = cudaGraphInstantiate(&g->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    GCK(ei);
  }
  GCK(cudaGraphLaunch(g->step_exec, s));
  g->fwd_done = true;
  if (loss) {
    double lv = 0.0;
    GCK(cudaMemcpyAsync(&lv, g->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    *loss = lv;
  }
  return 0;
}

}  // extern "C"

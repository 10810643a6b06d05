// dpdlp_csr_spmv_noalloc: y = A x for a plain CSR matrix in device memory, allocating
// nothing.
//
// Some callers cannot allocate device memory at the point where they need a product:
// frameworks whose own pool has reserved the device's memory and forbid allocations behind
// its back, and latency-critical loops that must not stall on the allocator (cudaMalloc and
// cudaFree may synchronize the device).  For them this entry point keeps its only scratch
// -- the partial sums of rows that cross thread-block boundaries -- in one file-scope
// device array of fixed size, reserved once per device when the library is loaded and held
// until the process exits.
//
// Work split: the nonzeros are cut into P equal parts (P <= NA_MAX_PARTS), one thread block
// per part.  A block owns the rows that start inside its part and sums them completely,
// except its last row when that row runs into later parts: then it writes that row's
// partial sum to y and every later part the row covers leaves its share in the scratch
// array.  A second launch adds those shares to y in part order, so results do not depend
// on scheduling and reruns are bitwise identical.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dpdlp.h"

namespace {

constexpr int NA_TPB = 256;
constexpr int NA_MAX_PARTS = 16384;
constexpr int NA_PART_NNZ = 4096;                                   // target nonzeros per part
constexpr long long NA_MAX_NNZ = (long long)NA_MAX_PARTS * 65536;   // 2^30 nonzeros

struct NoAllocScratch {
  double carry[NA_MAX_PARTS];   // share of the row that part p continues (if any)
  int carry_row[NA_MAX_PARTS];  // that row, or -1
};

// 192 KB per device, shared by every call on that device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Smallest r in [0, m] with rp[r] >= key (rp[m] = nnz >= key).
__device__ int first_ge(const int32_t* rp, int m, long long key) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)rp[mid] >= key) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(NA_TPB)
noalloc_parts_kernel(int m, long long nnz, int P, long long S, const int32_t* __restrict__ rp,
                     const int32_t* __restrict__ ci, const double* __restrict__ val,
                     const double* __restrict__ x, double* __restrict__ y, NoAllocScratch* sc) {
  __shared__ int rows[2];
  const int p = blockIdx.x;
  const long long e0 = (long long)p * S;
  const long long e1 = e0 + S < nnz ? e0 + S : nnz;
  if (threadIdx.x == 0) {
    rows[0] = first_ge(rp, m, e0);
    rows[1] = (p == P - 1) ? m : first_ge(rp, m, e1);
  }
  __syncthreads();
  const int R0 = rows[0], R1 = rows[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    // leading share: item e0 belongs to a row that started in an earlier part
    const bool lead = R0 > 0 && e0 < nnz && (long long)rp[R0] > e0;
    double s = 0.0;
    if (lead) {
      const long long end = (long long)rp[R0] < e1 ? (long long)rp[R0] : e1;
      for (long long e = e0 + lane; e < end; e += 32) s = fma(val[e], x[ci[e]], s);
      s = warp_sum(s);
    }
    if (lane == 0) {
      sc->carry[p] = lead ? s : 0.0;
      sc->carry_row[p] = lead ? R0 - 1 : -1;
    }
  }
  for (int r = R0 + warp; r < R1; r += NA_TPB / 32) {
    const long long a = rp[r];
    const long long b = (long long)rp[r + 1] < e1 ? (long long)rp[r + 1] : e1;
    double s = 0.0;
    for (long long e = a + lane; e < b; e += 32) s = fma(val[e], x[ci[e]], s);
    s = warp_sum(s);
    if (lane == 0) y[r] = s;  // partial when the row runs past e1; finished below
  }
}

__global__ void __launch_bounds__(NA_TPB)
noalloc_fixup_kernel(int m, long long nnz, int P, long long S, const int32_t* __restrict__ rp,
                     double* __restrict__ y, const NoAllocScratch* sc) {
  const int p = blockIdx.x * NA_TPB + threadIdx.x;
  if (p >= P) return;
  const long long e0 = (long long)p * S;
  const long long e1 = e0 + S < nnz ? e0 + S : nnz;
  const int R0 = first_ge(rp, m, e0);
  const int R1 = (p == P - 1) ? m : first_ge(rp, m, e1);
  if (R1 <= R0) return;
  const int r = R1 - 1;  // the part's last row
  if ((long long)rp[r + 1] <= e1) return;
  double s = y[r];
  for (int q = p + 1; q < P && sc->carry_row[q] == r; ++q) s += sc->carry[q];
  y[r] = s;
}

std::mutex g_scratch_mu;
NoAllocScratch* g_scratch_ptr[64] = {};  // device address of the array, per device ordinal

// Device address of the scratch array on the current device, looked up once per device and
// kept for the life of the process (a device reset would make it stale; the header says so).
cudaError_t scratch_address(int dev, NoAllocScratch** out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int dpdlp_csr_spmv_noalloc(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr,
                                      const int32_t* col_idx, const double* val, const double* x,
                                      double* y, void* cuda_stream) {
  if (m < 0 || n < 0 || nnz < 0) return DPDLP_ERR_INVALID;
  if (nnz > NA_MAX_NNZ) return DPDLP_ERR_TOO_LARGE;
  if (m == 0) return 0;
  if (!row_ptr || !y || (nnz > 0 && (!col_idx || !val || !x))) return DPDLP_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPDLP_ERR_CUDA;
  NoAllocScratch* sc = nullptr;
  if (scratch_address(dev, &sc) != cudaSuccess) return DPDLP_ERR_CUDA;
  long long P = (nnz + NA_PART_NNZ - 1) / NA_PART_NNZ;
  if (P < 1) P = 1;
  if (P > NA_MAX_PARTS) P = NA_MAX_PARTS;
  long long S = (nnz + P - 1) / P;
  if (S < 1) S = 1;
  P = nnz > 0 ? (nnz + S - 1) / S : 1;  // no empty part
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  noalloc_parts_kernel<<<(int)P, NA_TPB, 0, s>>>(m, nnz, (int)P, S, row_ptr, col_idx, val, x, y, sc);
  noalloc_fixup_kernel<<<(int)((P + NA_TPB - 1) / NA_TPB), NA_TPB, 0, s>>>(m, nnz, (int)P, S, row_ptr, y, sc);
  return cudaGetLastError() == cudaSuccess ? 0 : DPDLP_ERR_CUDA;
}

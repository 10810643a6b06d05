// Internal declarations shared by the host preprocessing, the kernels and the C ABI layer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace pdhg {

// Thread-block shape of every tiled SpMV kernel: 256 threads, each summing 32 consecutive
// nonzeros (four batches of 8 loaded with 16-byte vector loads), so one tile holds at most
// 8192 nonzeros and 768 rows (nonzero-aware partitioning of Section 4.3, applied to thread
// blocks instead of devices).  Small matrices get smaller tiles so that every SM has work.
constexpr int TPB = 256;
constexpr int BATCH = 8;
constexpr int NBATCH = 4;
constexpr int IPT = BATCH * NBATCH;
constexpr int TILE_NNZ = TPB * IPT;
constexpr int MAX_TILE_ROWS = 768;
constexpr int KMAX = 1024;  // largest check period (iterations per graph body)
constexpr int NRED = 5;     // quantities per check reduction (rows and columns)

// One tile of a row-major sparse matrix (CSR of A, or CSR of A^T for the column pass).
// Short tile: whole rows [r0, r1) (at most MAX_TILE_ROWS) whose nonzeros [e0, e1) fit in
// TILE_NNZ; e0 is a multiple of BATCH.  Long tile: chunk `chunk` of `nchunks` of the single row r0 (r1 = r0+1)
// that is longer than a tile; `slot` indexes the chunk-partial array (slot + chunk) and
// `lrow` the per-row arrival counter.  slot < 0 marks a short tile.
struct Tile {
  int r0, r1, e0, e1;
  int slot, lrow, chunk, nchunks;
};

// Host copy of one tiled orientation.  Every tile starts at a BATCH-aligned offset: the
// padding between tiles is stored as explicit zero entries appended to the tile's last row
// (value 0, column = that row's last column, or 0), so row pointers stay a plain CSR.
struct HostTiled {
  int rows = 0, cols = 0;
  std::vector<int32_t> ptr;  // rows + 1, offsets into the padded arrays
  std::vector<int32_t> idx;  // padded length + TILE_NNZ tail
  std::vector<double> val;
  std::vector<Tile> tiles;
  int long_rows = 0;     // rows split over several tiles
  int long_chunks = 0;   // total chunks of those rows
  int64_t nnz_padded = 0;
};

// Device copy of one tiled orientation plus the scratch of its long-row combine.
struct DevTiled {
  int rows = 0, cols = 0;
  int32_t* ptr = nullptr;
  int32_t* idx = nullptr;
  double* val = nullptr;
  Tile* tiles = nullptr;
  int ntiles = 0;
  double* lr_partial = nullptr;  // 2 * long_chunks (room for two vectors)
  unsigned* lr_count = nullptr;  // long_rows arrival counters, zero between launches
  int long_rows = 0, long_chunks = 0;
};

// Solver scalars resident in device memory.  The control kernel updates them at every
// check; the iteration kernels only read them.  The host writes them at the start of a
// solve and reads them at the end.
struct DevScalars {
  long long T_base;    // total iterations before the current graph body
  long long k_base;    // iterations since the last restart, before the current body
  long long T_check;   // total iteration count at the end of the current body's check
  long long max_iter;
  double tau, sigma, inv_sigma, omega, eta, gamma, eps;
  double beta_s, beta_n, beta_a, kp, ki, kd;
  double bnorm, cnorm;
  int K, halpern, restart_enabled, pid_enabled;
  // epoch and PID state
  double r_anchor, r_prev, e_sum, e_prev;
  int has_anchor, has_e_prev;
  long long restarts, checks;
  // results of the last check
  double r_p, r_d, r_g, obj_p, obj_d, r_fp;
  int status;       // -1 running, 0 converged, 1 iteration limit, 2 non-finite
  int apply_mode;   // what the apply kernel does: 0 Halpern step, 1 restart, 2 nothing
  double w1_check, w0_check;  // Halpern weights of the check iteration
  int sched_len;    // forced restart schedule length (0: off)
  int trace_cap;
  long long trace_count;
  double w1[KMAX], w0[KMAX];  // Halpern weights (k+1)/(k+2), 1/(k+2) of each body iteration
};

// Device vectors of one LP (internal, permuted index order).
struct DevVecs {
  int n = 0, m = 0;
  double *c = nullptr, *lv = nullptr, *uv = nullptr;  // [n]
  double *lo = nullptr, *hi = nullptr;                // [m]: the box -S = [-uc, -lc]
  double *x = nullptr, *x0 = nullptr, *xbar = nullptr, *xh = nullptr, *dx = nullptr;  // [n]
  double *aty = nullptr;                               // [n]
  double *y = nullptr, *y0 = nullptr, *yh = nullptr;   // [m]
  double *axh = nullptr, *adx = nullptr;               // [m]
  double *red_rows = nullptr, *red_cols = nullptr;     // reduction partials [G][NRED]
  int g_rows = 1, g_cols = 1;
  int32_t *perm_col = nullptr, *perm_row = nullptr;    // internal index -> caller index
  double *tmp_n = nullptr, *tmp_m = nullptr, *tmp_n2 = nullptr;  // scratch vectors
  double *pw = nullptr;                                // power-iteration scalars [4]
  int8_t* sched = nullptr;                             // forced schedule
  void* trace = nullptr;                               // dpdlp_trace_t ring
};

// ---------------------------------------------------------------- host preprocessing
// Validate a CSR matrix; returns an empty string or an error description.
std::string validate_csr(int rows, int cols, const int64_t* ptr, const int32_t* idx,
                         const double* val);
// Block-wise random permutation of 0..len-1 in blocks of `block` (Section 4.2): full
// blocks are shuffled by a SplitMix64-driven Fisher-Yates, order inside a block is kept,
// a trailing partial block stays last.  Returns new index -> old index.
std::vector<int32_t> block_permutation(int len, int block, uint64_t seed, bool enabled);
// Apply row and column permutations (new -> old) to a CSR matrix; columns sorted per row.
void permute_csr(int rows, int cols, const int64_t* ptr, const int32_t* idx, const double* val,
                 const std::vector<int32_t>& prow, const std::vector<int32_t>& pcol,
                 std::vector<int64_t>& optr, std::vector<int32_t>& oidx, std::vector<double>& oval);
// CSR of the transpose by a stable counting sort (entries of a column in row order).
void transpose_csr(int rows, int cols, const std::vector<int64_t>& ptr,
                   const std::vector<int32_t>& idx, const std::vector<double>& val,
                   std::vector<int64_t>& tptr, std::vector<int32_t>& tidx,
                   std::vector<double>& tval);
// Tiles and padded arrays of one orientation.
// tile_cap: largest tile in nonzeros (0 = automatic: TILE_NNZ, smaller for small matrices).
void build_tiled(int rows, int cols, const std::vector<int64_t>& ptr,
                 const std::vector<int32_t>& idx, const std::vector<double>& val, HostTiled& out,
                 int tile_cap = 0);

// ---------------------------------------------------------------- kernel launchers
struct IterPlan {
  int i;              // iteration index inside the graph body
  int force_regular;  // 1: run as a regular iteration regardless of the scalars (timing)
};

cudaError_t launch_primal(const DevTiled& csc, const DevVecs& v, const DevScalars* sc,
                          IterPlan p, cudaStream_t s);
cudaError_t launch_dual(const DevTiled& csr, const DevVecs& v, const DevScalars* sc,
                        IterPlan p, cudaStream_t s);
// out0 = M x0 (and out1 = M x1 when x1 != nullptr) for one tiled orientation M.
cudaError_t launch_spmv(const DevTiled& M, const double* x0, const double* x1, double* out0,
                        double* out1, cudaStream_t s);
cudaError_t launch_check(const DevTiled& csr, const DevTiled& csc, const DevVecs& v,
                         DevScalars* sc, unsigned long long cond_handle, int use_cond,
                         cudaStream_t s);
cudaError_t launch_fill_start(const DevVecs& v, int fresh_x, int fresh_y, cudaStream_t s);
cudaError_t launch_gather(const double* in, const int32_t* perm, double* out, int len,
                          cudaStream_t s);  // out[i] = in[perm[i]]
cudaError_t launch_scatter(const double* in, const int32_t* perm, double* out, int len,
                           cudaStream_t s);  // out[perm[i]] = in[i]
cudaError_t launch_fill(double* p, double v, int len, cudaStream_t s);
// One power-iteration round: w = A v, lam = w.w, u = A^T w, v = u / ||u||; pw[0] = lam,
// pw[1] = ||u||.
cudaError_t launch_power_round(const DevTiled& csr, const DevTiled& csc, const DevVecs& v,
                               double* vec_v, double* vec_w, double* vec_u, cudaStream_t s);
int reduction_grid(int len);

}  // namespace pdhg

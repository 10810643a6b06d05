// Internal declarations shared by the host preprocessing, the kernels and the C ABI layer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace pdhg {

// ---------------------------------------------------------------- packed sparse layout
// Both products (A x_bar over rows of A, A^T y over rows of A^T = columns of A) use one
// layout.  The rows of the matrix are packed, on the host, into warp lanes: a lane holds
// at most LANE_ITEMS nonzeros, made of whole short rows (at most LANE_ITEMS nonzeros) and
// pieces of long rows; 32 lanes form a slot that one warp processes.  Every lane sums its
// own rows sequentially, one FMA per stored nonzero, so rows never cross lanes, warps or
// blocks (the nonzero-aware partitioning of Section 4.3 taken down to the lane).  Pieces
// of long rows are finished by a second, lane-per-row pass that adds them in piece order.
constexpr int LANES = 32;
constexpr int LANE_ITEMS = 32;
constexpr int SLOT_ITEMS = LANES * LANE_ITEMS;
constexpr int MAX_SLOT_ROWS = 128;  // short rows per slot (shared-memory row sums)
#ifndef DPDLP_PK_WARPS
#define DPDLP_PK_WARPS 4
#endif
constexpr int PK_WARPS = DPDLP_PK_WARPS;  // slots per thread block of the packed kernels
constexpr int PK_TPB = PK_WARPS * LANES;
constexpr uint32_t END_BIT = 0x80000000u;    // last stored nonzero of a row or piece
constexpr uint32_t PIECE_BIT = 0x40000000u;  // ... and that segment is a long-row piece
constexpr uint32_t IDX_MASK = 0x3FFFFFFFu;   // column index (< 2^30)

// Long rows with more pieces than these get a thread block / a warp of the long-row pass.
constexpr int LONG_BLOCK_PIECES = 256;
constexpr int LONG_WARP_PIECES = 32;

// Thread-block size of the element-wise and reduction kernels.
constexpr int TPB = 256;
constexpr int KMAX = 1024;  // largest check period (iterations per graph body)
constexpr int NRED = 6;     // quantities per check reduction (rows and columns)

// Slot s: its short rows have the new indices [row_base, row_base + nrows); all belong to
// LP instance `inst` (a slot never mixes instances of a batch).
struct SlotDesc {
  int row_base, nrows, inst, pad;
};
// Lane l of a slot: slot-local index of its first short row, global id of its first piece.
struct LaneMeta {
  int row_local, piece_base;
};

// Host copy of one packed orientation.  Item (lane l, position p) of slot s is stored at
// val[s*SLOT_ITEMS + ((p/2)*LANES + l)*2 + p%2] and idx[s*SLOT_ITEMS + ((p/4)*LANES + l)*4 + p%4]
// (val32 like idx), so a warp reads a slot with 16-byte loads that cover 512 contiguous bytes.
struct HostPacked {
  int rows = 0, cols = 0;
  int nslots = 0, nshort = 0, nlong = 0, npieces = 0;
  int nlong_block = 0, nlong_warp = 0;  // leading long rows finished by a block / a warp
  std::vector<double> val;
  std::vector<float> val32;         // FP32 copy, stored like idx (groups of 4 per lane)
  bool fp32_exact_range = true;     // every value rounds to a normal float (or is zero)
  std::vector<uint32_t> idx;
  std::vector<SlotDesc> slots;
  std::vector<LaneMeta> lanes;
  std::vector<int32_t> long_row;    // new index of each long row
  std::vector<int32_t> long_inst;   // instance of each long row
  std::vector<int32_t> long_ptr;    // nlong + 1
  std::vector<int32_t> long_piece;  // piece ids of each long row, in row order
  int64_t stored = 0;               // nslots * SLOT_ITEMS
};

// Device copy of one packed orientation plus the per-piece partial sums.
struct DevPacked {
  int rows = 0, cols = 0, nslots = 0, nlong = 0, npieces = 0;
  int nlong_block = 0, nlong_warp = 0;
  int cta_slots = PK_WARPS;  // slots per block of this orientation's iteration kernel (2, 4, 8)
  int list_warps_per_sm = 0;  // resident warps per SM of the persistent list kernel (0: most)
  int list_few_slots = 0;     // a body with at most this many active slots (list mode 2) walks
                              // the lists with a grid of about this many warps
  const double* val = nullptr;
  const float* val32 = nullptr;  // FP32 copy of the values (nullptr: not representable)
  const uint32_t* idx = nullptr;
  const SlotDesc* slots = nullptr;
  const LaneMeta* lanes = nullptr;
  const int32_t* long_row = nullptr;
  const int32_t* long_inst = nullptr;
  const int32_t* long_ptr = nullptr;
  const int32_t* long_piece = nullptr;
  double* piece_sum = nullptr;  // 2 * npieces (room for two vectors)
  // batches: slots of the running instances, rebuilt at every check (nullptr for one LP)
  const int32_t* slot_off = nullptr;  // ninst + 1: instance i owns slots [slot_off[i], slot_off[i+1])
  int32_t* active = nullptr;          // nslots: slot ids of running instances, instance order
  int32_t* nactive = nullptr;         // 1: entries of active in use
};

// Row order chosen by the packing of one orientation (pre-order = after the block
// permutation): new_of_old[r] and old_of_new[r'].
struct PackPlan {
  std::vector<int32_t> new_of_old, old_of_new;
  // lane contents: segments (pre-order row, first item, count, piece id or -1)
  struct Seg {
    int32_t row, first, count, piece;
  };
  std::vector<int32_t> lane_ptr;  // per lane, into segs
  std::vector<Seg> segs;
  std::vector<SlotDesc> slots;
  std::vector<int32_t> slot_lanes;  // LANES entries per slot: lane index or -1 (empty lane)
  int nshort = 0, nlong = 0, npieces = 0;
  std::vector<int32_t> long_rows;   // pre-order index of each long row, longest first
  std::vector<int32_t> long_inst;   // instance of each long row
  std::vector<int32_t> long_ptr, long_piece;
};

// Solver scalars resident in device memory, in two parts.  All instances of a batch take
// their iterations together (one iteration counter); each has its own step sizes, primal
// weight, restart epoch and status.  The control kernel updates both at every check; the
// iteration kernels only read them.  The host writes them at the start of a solve and
// reads them at the end.
struct DevScalars {
  long long T_base;    // total iterations before the current graph body
  long long T_check;   // total iteration count at the end of the current body's check
  long long max_iter;
  double gamma, eps;
  double beta_s, beta_n, beta_a, kp, ki, kd;
  int K, halpern, restart_enabled, pid_enabled;
  int ninst;
  int running;         // instances still iterating
  long long checks;
  int status;          // -1 running, else the worst instance status (2 > 1 > 0)
  int sched_len;       // forced restart schedule length per instance (0: off)
  int trace_cap;
  long long trace_count;
  int fp32_switch;     // mixed precision: switch to FP64 values when the KKT error stalls
  int fp32_stall_limit;
  double fp32_switch_tol;
};

struct InstScalars {
  double tau, sigma, inv_sigma, omega, eta;
  double bnorm, cnorm;
  long long k_base;    // iterations since the instance's last restart, before the body
  long long iterations;  // total iterations the instance has taken
  double r_anchor, r_prev, e_sum, e_prev;
  int has_anchor, has_e_prev;
  long long restarts;
  double r_p, r_d, r_g, obj_p, obj_d, r_fp;
  int status;          // -1 running, 0 converged, 1 iteration limit, 2 non-finite
  int apply_mode;      // what the apply kernel does: 0 Halpern step, 1 restart, 2 nothing
  double w1_check, w0_check;  // Halpern weights of the check iteration
  int spmv_fp32;       // this instance's products use FP32 values
  int stall_checks;
  double best_kkt;
};

// Device vectors of one LP (internal, packed index order).
struct DevVecs {
  int n = 0, m = 0;
  double *c = nullptr, *lv = nullptr, *uv = nullptr;  // [n]
  double *lo = nullptr, *hi = nullptr;                // [m]: the box -S = [-uc, -lc]
  double *x = nullptr, *x0 = nullptr, *xbar = nullptr, *xh = nullptr, *dx = nullptr;  // [n]
  double *aty = nullptr;                               // [n]
  double *q = nullptr;                                 // [n] diagonal of Q (nullptr: an LP)
  double *y = nullptr, *y0 = nullptr, *yh = nullptr;   // [m]
  double *axh = nullptr, *adx = nullptr;               // [m]
  double *red_rows = nullptr, *red_cols = nullptr;     // reduction partials [chunks][NRED]
  const int4* chunk_rows = nullptr;                   // reduction chunks {inst, start, len, -}
  const int4* chunk_cols = nullptr;
  const int32_t* inst_chunk_rows = nullptr;           // ninst + 1: chunks of each instance
  const int32_t* inst_chunk_cols = nullptr;
  int g_rows = 1, g_cols = 1;                         // number of chunks
  const double* row_w = nullptr;                      // [m] KKT weights 1/D_r (nullptr: 1)
  const double* col_w = nullptr;                      // [n] KKT weights 1/D_c (nullptr: 1)
  const int32_t* inst_of_row = nullptr;               // [m]
  const int32_t* inst_of_col = nullptr;               // [n]
  InstScalars* inst = nullptr;                        // [ninst]
  double* wtab = nullptr;                             // [ninst][2][KMAX] Halpern weights
  int ninst = 1;
  int32_t* act_off = nullptr;                         // 2 (ninst + 1): offsets into the active lists
  int32_t *perm_col = nullptr, *perm_row = nullptr;    // internal index -> caller index
  double *tmp_n = nullptr, *tmp_m = nullptr, *tmp_n2 = nullptr;  // scratch vectors
  double *pw = nullptr;                                // power-iteration scalars [ninst][4]
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
// Optional diagonal preconditioning (the paper defines none): Ruiz infinity-norm passes,
// then one Pock-Chambolle pass (alpha = 1), every factor rounded to the nearest power of
// two so scaling is exact.  Scales val in place to D_r A D_c and returns D_r, D_c.
void precondition(int rows, int cols, const std::vector<int64_t>& ptr,
                  const std::vector<int32_t>& idx, std::vector<double>& val, int ruiz_passes,
                  bool pock_chambolle, std::vector<double>& dr, std::vector<double>& dc);
// Pack the rows of one orientation into lanes and slots (best-fit decreasing on row
// lengths); decides the new row order.
void plan_packing(int rows, const std::vector<int64_t>& ptr, PackPlan& plan);
// The same for a batch: rows [offsets[i], offsets[i+1]) are instance i; each instance is
// packed into slots of its own and keeps its row range in the new order.
void plan_packing_batch(int rows, const std::vector<int64_t>& ptr,
                        const std::vector<int32_t>& offsets, PackPlan& plan);
// Stored arrays of one orientation from its plan; column indices are mapped through the
// other orientation's new_of_old.
void build_packed(int rows, int cols, const std::vector<int64_t>& ptr,
                  const std::vector<int32_t>& idx, const std::vector<double>& val,
                  const PackPlan& plan, const std::vector<int32_t>& col_new_of_old,
                  HostPacked& out);
// A batch: padding and empty rows of instance i's slots gather offsets[i], the instance's
// own first entry of the gathered vector (its entry 0 when solved alone), not entry 0 of
// the stack, which belongs to instance 0.
void own_instance_zero_gathers(HostPacked& packed, const std::vector<int32_t>& offsets);

// ---------------------------------------------------------------- kernel launchers
struct IterPlan {
  int i;              // iteration index inside the graph body
  int force_regular;  // 1: run as a regular iteration regardless of the scalars (timing)
  int list;           // batches: 1 walk the active-slot list, 2 the same with a small grid
                      // (few slots active), 0 one launch over every slot
  int pdl;            // launch as a programmatic dependent of the previous kernel
  int idle;           // timing only: every instance counts as stopped (an empty slot list)
  int slots_only;     // timing only: the slot kernel without the long-row pass
};

cudaError_t launch_primal(const DevPacked& csc, const DevVecs& v, const DevScalars* sc,
                          IterPlan p, cudaStream_t s);
cudaError_t launch_dual(const DevPacked& csr, const DevVecs& v, const DevScalars* sc,
                        IterPlan p, cudaStream_t s);
// Small single LPs: all K iterations of a graph body in one launch of one thread block,
// bitwise equal to K pairs of launch_primal / launch_dual.  Applies when both orientations
// have at most max_slots (<= FUSED_MAX_SLOTS) slots and no block-class long rows.
constexpr int FUSED_MAX_SLOTS = 64;
bool fused_body_fits(const DevPacked& csc, const DevPacked& csr, int ninst, int max_slots);
// Sets the fused kernel's shared-memory limit; called before the first launch or capture.
cudaError_t fused_body_prepare();
// cluster > 1: the body spread over a thread-block cluster of that many CTAs (at most 8),
// bitwise the same results.  slot_cache: each CTA copies its slots into shared memory once
// per launch when they fit (bitwise the same results).
cudaError_t launch_body_fused(const DevPacked& csc, const DevPacked& csr, const DevVecs& v,
                              const DevScalars* sc, int K, int cluster, int slot_cache,
                              cudaStream_t s);
// CTAs of the cluster form: `requested` (>= 1), or 0 = about two slots per CTA, at most 8.
int fused_cluster_ctas(const DevPacked& csc, const DevPacked& csr, int requested);
// out0 = M x0 (and out1 = M x1 when x1 != nullptr) for one packed orientation M; with
// `running` (a batch's instance scalars) only the rows of running instances are computed.
cudaError_t launch_spmv(const DevPacked& M, const double* x0, const double* x1, double* out0,
                        double* out1, cudaStream_t s, const InstScalars* running);
cudaError_t launch_check(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                         DevScalars* sc, unsigned long long cond_handle, int use_cond,
                         cudaStream_t s);
// Batches: set the graph conditional `handle` (a switch over the body's three forms) to 2 when
// at most `few` slots are active (the lists, small grids), else 1 when fewer than `fraction`
// of the slots are active (the lists), else 0 (every slot).
cudaError_t launch_select(const DevPacked& csr, const DevPacked& csc, unsigned long long handle,
                          double fraction, int few, cudaStream_t s);
// The same choice on the host, from the active counts.
int select_form(long long active, long long total, double fraction, int few);
// Most resident warps per SM of the persistent list kernel (its register budget).
int list_max_warps_per_sm();
// Batches: rebuild both orientations' lists of slots of running instances.
cudaError_t launch_compact(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                           cudaStream_t s);
cudaError_t launch_fill_start(const DevVecs& v, int fresh_x, int fresh_y, cudaStream_t s);
// out[i] = in[perm[i]] * scale[i] (scale may be nullptr: 1)
cudaError_t launch_gather(const double* in, const int32_t* perm, const double* scale,
                          double* out, int len, cudaStream_t s);
// out[perm[i]] = in[i] * scale[i] (scale may be nullptr: 1)
cudaError_t launch_scatter(const double* in, const int32_t* perm, const double* scale,
                           double* out, int len, cudaStream_t s);
cudaError_t launch_fill(double* p, double v, int len, cudaStream_t s);
// Access probes of one packed orientation (no arithmetic, for the roofline): mode 0 the
// index stream and the gathers of x, mode 1 plus the value stream, mode 2 the streams only,
// mode 3 mode 1 plus the loads and stores of the epilogue's row vectors of `v` (primal: the
// A^T y orientation's; else the dual's), which it overwrites.
cudaError_t launch_access_probe(const DevPacked& M, const double* x, int mode,
                                const DevVecs& v, bool primal, bool pdl,
                                unsigned long long* sink, cudaStream_t s);
// One power-iteration round for every instance: w = A v, lam_i = w_i.w_i, u = A^T w,
// v_i = u_i / ||u_i||; pw[4 i] = lam_i, pw[4 i + 1] = ||u_i||.
cudaError_t launch_power_round(const DevPacked& csr, const DevPacked& csc, const DevVecs& v,
                               double* vec_v, double* vec_w, double* vec_u, cudaStream_t s);
// Reduction chunks of at most `chunk` consecutive elements inside one instance, as
// {inst, start, len, 0} quadruples; inst_chunk[i] .. inst_chunk[i+1] are instance i's.
void build_chunks(const std::vector<int32_t>& offsets, int chunk, std::vector<int32_t>& chunks,
                  std::vector<int32_t>& inst_chunk);
constexpr int RED_CHUNK = 4096;

}  // namespace pdhg

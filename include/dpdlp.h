/*
 * dpdlp.h -- C ABI of libdpdlp, a single-GPU (GB300, sm_103a) restarted reflected-Halpern
 * PDHG solver for sparse linear programs.
 *
 * The method is the PDLP iteration of "D-PDLP: Scaling PDLP to Distributed Multi-GPU
 * Systems" (arXiv 2601.07628), run on one device:
 *   - problem (Section 2.1, Eq. prob:primal):  min c^T x  s.t.  lc <= A x <= uc,
 *     lv <= x <= uv, with A sparse (m rows, n columns);
 *   - PDHG step (Section 2.2; Algorithm 1, steps 1-2):
 *       x^ = proj_X(x - tau (c - A^T y)),  z = A (2 x^ - x),
 *       y^ = y - sigma z - sigma proj_{-S}(y / sigma - z),   tau = eta/omega, sigma = eta*omega;
 *   - reflected Halpern step (Appendix B.1; Algorithm 1, step 3);
 *   - every check_every iterations: relative KKT error (Appendix B.4), fixed-point residual
 *     in the P-norm (Appendix B, D.2.1), adaptive restart (Appendix B.2) and the PID primal
 *     weight (Appendix B.3).
 * The paper's 2D device grid and its AllReduces are not used: everything runs on one GPU;
 * its block-wise random permutation (Section 4.2) and nonzero-aware partitioning
 * (Section 4.3) are used to balance nonzeros across thread blocks.
 *
 * Conventions for every entry point:
 *   - Return value: >= 0 on success (dpdlp_solve returns a solve status), < 0 an error code
 *     (DPDLP_ERR_*).  After an error, dpdlp_last_error(h) describes it.
 *   - Arrays are plain C arrays in the caller's index order (the library permutes
 *     internally and undoes it on output).  Sizes: n = number of variables (columns of A),
 *     m = number of rows.
 *   - Pointer location: dpdlp_load_lp, dpdlp_load_batch and dpdlp_set_row_bounds take
 *     HOST pointers.  Vector
 *     arguments of dpdlp_set_start, dpdlp_get_solution, dpdlp_get_state, dpdlp_set_state,
 *     dpdlp_apply_A and dpdlp_apply_AT are HOST pointers by default and DEVICE pointers
 *     (on the handle's device) after dpdlp_set_param(h, "ptr_mode_device", 1).
 *   - Ownership: inputs are copied; the caller keeps and frees its buffers.  Outputs are
 *     written into caller-owned buffers of the stated length.  The handle owns all device
 *     memory it allocates and frees it in dpdlp_destroy.
 *   - Concurrency: handles are independent; one handle must not be used from two host
 *     threads at once.  All device work of a handle is ordered on its stream.
 */
#ifndef DPDLP_H
#define DPDLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Solve status (non-negative return of dpdlp_solve). */
#define DPDLP_CONVERGED 0     /* max(r_primal, r_dual, r_gap) <= tol at a check */
#define DPDLP_MAX_ITER 1      /* iteration limit reached without convergence */
#define DPDLP_NUMERICAL 2     /* a non-finite iterate or residual was detected at a check */

/* Error codes (negative returns). */
#define DPDLP_ERR_INVALID (-1)    /* invalid argument: bad CSR, lv > uv, lc > uc, NaN input... */
#define DPDLP_ERR_OOM (-2)        /* device or host allocation failed */
#define DPDLP_ERR_CUDA (-3)       /* a CUDA runtime call failed */
#define DPDLP_ERR_NOT_LOADED (-4) /* no LP loaded on this handle */
#define DPDLP_ERR_TIMEOUT (-5)    /* reserved for a bounded device wait that gives up; this
                                     build has no device-side wait and never returns it */
#define DPDLP_ERR_TOO_LARGE (-6)  /* size beyond dpdlp_csr_spmv_noalloc's fixed scratch */

typedef struct dpdlp dpdlp_t; /* opaque solver handle, one LP per handle */

/* Convergence report of the last solve (Appendix B.4 quantities at the final check). */
typedef struct dpdlp_kkt {
  double r_primal;   /* ||Ax - proj_S(Ax)|| / (1 + ||[lc,uc]||_finite) */
  double r_dual;     /* ||proj_X(x - tau(c - A^T y)) - x|| / tau / (1 + ||c||) */
  double r_gap;      /* |obj_p - obj_d| / (1 + max(|obj_p|, |obj_d|)) */
  double obj_p;      /* c^T x */
  double obj_d;      /* -p(-y; lc, uc) + s^T x */
  double r_fp;       /* fixed-point residual ||z - PDHG(z)||_P at the final check */
  double omega;      /* primal weight */
  double eta;        /* step size */
  double tau, sigma; /* eta / omega, eta * omega */
  int64_t iterations;
  int64_t restarts;
  int64_t checks;
  int32_t status;    /* DPDLP_CONVERGED / DPDLP_MAX_ITER / DPDLP_NUMERICAL, -1 before a solve */
  int32_t spmv_mode; /* iteration products at the end: 0 FP64 values, 1 FP32 values */
} dpdlp_kkt_t;

/* One record per check and instance (a batch of N instances writes N records per check,
 * instance order, every instance every check), kept in a device ring of the last
 * trace_capacity records. */
typedef struct dpdlp_trace {
  int64_t T;        /* total iterations at the check */
  int64_t k;        /* iterations since the last restart, after this check's iteration */
  double r_primal, r_dual, r_gap, obj_p, obj_d;
  double r_fp;      /* fixed-point residual */
  double omega;     /* primal weight used by this check's iteration */
  int32_t restart;  /* 0 none, 1 sufficient decay, 2 necessary decay, 3 artificial */
  int32_t spmv_mode;/* values used by this check's iteration: 0 FP64, 1 FP32 */
  int32_t inst;     /* instance of a batch (0 for a single LP) */
  int32_t status;   /* the instance's status after the check (-1 still running) */
} dpdlp_trace_t;

/* Scalar part of a checkpoint (the vector part is x, y, x0, y0). */
typedef struct dpdlp_scalar_state {
  int64_t T, k, restarts, checks;
  double eta, omega;
  double r_anchor, r_prev; /* restart references; has_anchor = 0 means "unset" */
  double e_sum, e_prev;    /* PID integral and last error; has_e_prev = 0 means "unset" */
  int32_t has_anchor, has_e_prev;
  int32_t spmv_mode;       /* 1: iterations use the FP32 values (mixed precision) */
  int32_t stall_checks;    /* FP32 mode: checks since the KKT error last halved */
  double best_kkt;         /* FP32 mode: best KKT error so far */
} dpdlp_scalar_state_t;

/* Sizes and layout facts of the loaded LP. */
typedef struct dpdlp_info {
  int32_t n, m;
  int64_t nnz;
  int64_t nnz_padded_csr, nnz_padded_csc; /* stored entries of each packed copy, padding included */
  int32_t tiles_csr, tiles_csc;           /* warp slots (32 lanes x 32 stored entries) of each copy */
  int32_t long_rows, long_cols;           /* rows / columns longer than one lane (32 nonzeros) */
  int64_t device_bytes;
  double preprocess_ms;
  int32_t fused_body;  /* 1: each graph body (check_every iterations) runs as one launch of one
                          thread block (parameters fused_body, fused_max_slots); results are
                          bitwise those of the separate primal / dual launches */
  int32_t reserved;
} dpdlp_info_t;

/* Create a handle bound to CUDA device `device`.  Work goes to a stream the handle creates
 * unless dpdlp_set_stream supplies one.  Errors: DPDLP_ERR_INVALID (bad device),
 * DPDLP_ERR_CUDA, DPDLP_ERR_OOM. */
int dpdlp_create(dpdlp_t** h, int device);

/* Free the handle and every device buffer it owns.  Safe on NULL. */
void dpdlp_destroy(dpdlp_t* h);

/* Description of the last error on this handle ("" if none); valid until the next call. */
const char* dpdlp_last_error(const dpdlp_t* h);

/* Device allocator hook: every device buffer of the loaded LP (matrix copies, vectors,
 * scalars, trace) comes from alloc(bytes, ctx) and goes back through
 * release(ptr, bytes, ctx) instead of cudaMalloc / cudaFree -- for instance a framework's
 * caching allocator.  alloc returns memory on the handle's device aligned to 256 bytes
 * (else the load fails with DPDLP_ERR_INVALID), or NULL (DPDLP_ERR_OOM).  Setting an
 * allocator unloads the current LP (its memory goes back to the allocator it came from);
 * NULL, NULL restores cudaMalloc.  The library synchronises its stream before releasing. */
typedef void* (*dpdlp_alloc_fn)(size_t bytes, void* ctx);
typedef void (*dpdlp_release_fn)(void* ptr, size_t bytes, void* ctx);
int dpdlp_set_allocator(dpdlp_t* h, dpdlp_alloc_fn alloc, dpdlp_release_fn release, void* ctx);

/* Use `cuda_stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream) for
 * all later work of the handle; NULL restores the handle's own stream.  The caller keeps
 * the stream alive while the handle uses it. */
int dpdlp_set_stream(dpdlp_t* h, void* cuda_stream);

/* Load an LP (Section 2.1, Eq. prob:primal) from HOST arrays.
 *   c[n]                objective
 *   row_ptr[m+1]        CSR row pointers, row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz
 *   col_idx[nnz]        CSR column indices in [0, n)
 *   val[nnz]            CSR values (finite)
 *   b[m], ctype[m]      row type 0: lc = uc = b ('='), 1: lc = -inf, uc = b ('<='),
 *                       2: lc = b, uc = +inf ('>=').  Both may be NULL (rows free until
 *                       dpdlp_set_row_bounds).
 *   lv[n], uv[n]        variable bounds, -INFINITY / +INFINITY allowed, lv <= uv
 * Validates the input (DPDLP_ERR_INVALID on failure; 1 <= n and 0 <= m, both below 2^30:
 * an LP needs a variable, while m = 0 leaves only the bounds), then on the host applies
 * the optional block-wise random permutation (Section 4.2), builds the CSC copy of A,
 * packs the rows of both copies into warp lanes (nonzero-aware partitioning, Section 4.3,
 * at lane granularity), and copies everything to the device.  Replaces any LP loaded
 * before and resets the solver state. */
int dpdlp_load_lp(dpdlp_t* h, int32_t n, int32_t m, const double* c, const int64_t* row_ptr,
                  const int32_t* col_idx, const double* val, const double* b,
                  const double* lv, const double* uv, const int8_t* ctype);

/* Load a batch of `count` independent LPs into one handle (the batched solve of many
 * small and medium LPs; the instances iterate together in the same kernels).  The
 * arguments are those of dpdlp_load_lp for the block-diagonal LP that stacks the
 * instances, plus HOST ranges row_off[count+1] and col_off[count+1]: instance i owns rows
 * [row_off[i], row_off[i+1]) and columns [col_off[i], col_off[i+1]) (row_off[0] =
 * col_off[0] = 0, row_off non-decreasing, col_off increasing: every instance has at
 * least one variable, row_off[count] = m, col_off[count] = n), and every nonzero of its
 * rows must lie in its columns (else DPDLP_ERR_INVALID).  Each instance
 * gets its own step size (power iteration on its own block), primal weight, restart
 * epoch, PID state, mixed-precision switch and status; the iteration counter, the check
 * period and the parameters are shared.  An instance that converges stops iterating (its
 * rows are skipped) while the others continue; dpdlp_solve returns when none is running,
 * with the worst status (2 > 1 > 0).  The block permutation acts inside every instance
 * (instance i draws seeds perm_seed + 2i and perm_seed + 2i + 1), so count = 1 is
 * dpdlp_load_lp.  Checkpoints (dpdlp_get_state / dpdlp_set_state) hold a single LP. */
int dpdlp_load_batch(dpdlp_t* h, int32_t count, const int32_t* row_off, const int32_t* col_off,
                     int32_t n, int32_t m, const double* c, const int64_t* row_ptr,
                     const int32_t* col_idx, const double* val, const double* b,
                     const double* lv, const double* uv, const int8_t* ctype);

/* Per-instance step sizes eta[count] (HOST, count = the number of loaded instances) used
 * by the next fresh solve instead of the power iteration; count = 0 clears them.  The
 * "eta" parameter, when > 0, still takes precedence. */
int dpdlp_set_batch_eta(dpdlp_t* h, const double* eta, int32_t count);

/* Diagonal QP (Section "Extensions to Diagonal QPs"): objective 1/2 x^T diag(q) x + c^T x
 * with q[n] >= 0 finite (HOST array, caller order); q = NULL restores the LP.  The primal
 * step becomes the clamped minimum of the separable quadratic (Eq. primal_update),
 * x^ = proj_X((x - tau (c - A^T y)) / (1 + tau q)); KKT errors use the objective gradient
 * c + Q x^ - A^T y^ and the objectives carry the quadratic term.  Resets the solver
 * state; a later dpdlp_load_lp / dpdlp_load_batch clears it.  For a batch, q covers the
 * stacked variables (zeros for the instances that are LPs). */
int dpdlp_set_objective_diag(dpdlp_t* h, const double* q);

/* Replace the row bounds with general ranges lc[m] <= A x <= uc[m] (HOST arrays, +-inf
 * allowed, lc <= uc, no NaN).  Resets the solver state. */
int dpdlp_set_row_bounds(dpdlp_t* h, const double* lc, const double* uc);

/* Set a named parameter.  Keys (default):
 *   eta (0 = power iteration, 0.998 / sigma_max(A)), eta_safety (0.998), power_iters (200),
 *   power_tol (1e-8), omega0 (0 = ||c|| / ||b_finite||), gamma (1.0), halpern (1),
 *   check_every (64, 1..1024), restart (1), beta_sufficient (0.2), beta_necessary (0.8),
 *   beta_artificial (0.36), pid (1), pid_kp (0.99), pid_ki (0.01), pid_kd (0.0),
 *   block_permute (1), perm_block (256), perm_seed (1), use_graph (1),
 *   ptr_mode_device (0), resume (0: each solve starts from the start point; 1: continue
 *   from the current state), trace_capacity (4096), spmv_fp32 (0: FP64 matrix values;
 *   1: mixed precision -- the iteration products use an FP32 copy of A's values, formed
 *   and accumulated in FP64, until the KKT error reaches fp32_switch_tol (1e-6), or is below
 *   100 x fp32_switch_tol and fails to halve over fp32_stall_checks (64) consecutive checks,
 *   then FP64 values; 2: FP32 values
 *   throughout).  KKT, restart and step-size products always use FP64 values.  Needs every
 *   value of A to round to a normal float or zero, else the FP64 values are used.
 *   precond (0): 1 = solve the diagonally scaled LP D_r A D_c instead of A (the paper
 *   defines no preconditioning; this is an option): ruiz_passes (10) Ruiz infinity-norm
 *   passes, then, if pock_chambolle (1), one Pock-Chambolle pass (alpha = 1); every factor
 *   is a power of two, so scaling is exact.  Vectors at the boundary (start points,
 *   solutions, checkpoints, dpdlp_apply_A/AT) stay in the original variables; reported
 *   KKT errors and objectives are those of the original LP (primal and dual residual
 *   vectors of the scaled LP divided by D_r and D_c); eta, the initial omega and the
 *   restart metric belong to the scaled LP.  Load-time keys.
 *   cta_slots_primal, cta_slots_dual (4): warp slots per thread block of the primal (A^T y)
 *   and dual (A x_bar) iteration kernels, 2, 4 or 8 (64, 128 or 256 threads); a launch
 *   shape only, results do not depend on it (set by the autotuner).
 *   fused_body (1), fused_max_slots (48, at most 64), fused_cluster (0): a single LP whose
 *   packed copies have at most fused_max_slots warp slots each (a slot holds 1,024 stored
 *   nonzeros) runs each graph body -- check_every iterations -- as one launch instead of two
 *   or three launches per iteration: one thread block with block barriers between the
 *   primal and dual phases, or a thread-block cluster of fused_cluster CTAs (at most 8)
 *   that share the slots, exchange x_bar and y through distributed shared memory and
 *   synchronize with cluster barriers.  fused_cluster = 0 chooses: one CTA up to 6 slots per
 *   copy, else about two slots per CTA.  On a tiny LP an iteration costs launch latency;
 *   one SM's FP64 issue rate bounds a single block beyond a few slots.  The sums and their
 *   order are those of the separate launches, so results are bitwise the same in every
 *   form; fused_body = 0 always launches the kernels separately.  dpdlp_get_info reports
 *   which form the next solve takes.  fused_slot_cache (1): each block of that form copies
 *   its slots (values, indices, lane metadata) and their rows' epilogue inputs into shared
 *   memory once per launch, when they fit next to the shared copies of x_bar and y (192 KB
 *   in all), and every iteration of the body reads them there; same results.
 *   pdl (1): the iteration kernels launch as programmatic dependents of the kernel before
 *   them (they load what no kernel writes -- slot descriptors, first index batches -- while
 *   it drains, then wait for it); 0 = plain stream order.  Results do not depend on it.
 *   list_fraction (0.5, 0..2), list_warps_per_sm (0 = the most the list kernel's register
 *   budget allows), list_few_slots (256): batches only.  A graph body walks the lists of
 *   slots of running instances (a persistent kernel with list_warps_per_sm resident warps
 *   per SM) when fewer than list_fraction of all slots are active, else launches over every
 *   slot (stopped instances' warps exit at once); with at most list_few_slots active slots
 *   it walks the lists with grids of about that many warps (a few stragglers do not pay for
 *   launching a full grid each iteration).  Launch choices only; the first two are set by
 *   the autotuner.
 * Load-time keys (block_permute, perm_block, perm_seed, precond, ruiz_passes,
 * pock_chambolle, trace_capacity) take effect at the next dpdlp_load_lp /
 * dpdlp_load_batch.  Unknown key or out-of-range value: DPDLP_ERR_INVALID. */
int dpdlp_set_param(dpdlp_t* h, const char* key, double v);

/* Read a parameter's current value. */
int dpdlp_get_param(const dpdlp_t* h, const char* key, double* v);

/* Warm start: x0[n], y0[m] (host or device per ptr_mode_device; either may be NULL for the
 * default x = proj_X(0), y = 0).  The start stays set: every later solve that starts fresh
 * (not resumed) begins there, until the next dpdlp_set_start replaces it (NULL, NULL
 * restores the default start) or an LP is loaded. */
int dpdlp_set_start(dpdlp_t* h, const double* x0, const double* y0);

/* Run PDHG until max(r_primal, r_dual, r_gap) <= tol at a check, or until the total
 * iteration count reaches max_iter.  The loop runs on the device (one CUDA graph with a
 * conditional while node); the host waits once at the end.  Returns DPDLP_CONVERGED,
 * DPDLP_MAX_ITER or DPDLP_NUMERICAL, or an error code. */
int dpdlp_solve(dpdlp_t* h, double tol, int64_t max_iter);

/* The returned point: (x^, y^), the PDHG output at the final check, x[n] and y[m]
 * (either may be NULL). */
int dpdlp_get_solution(dpdlp_t* h, double* x, double* y);

/* Residuals and counters of the last solve (HOST struct).  For a batch: the largest
 * residuals, the summed objectives and restarts, instance 0's step sizes and weight, and
 * the batch status. */
int dpdlp_get_kkt(dpdlp_t* h, dpdlp_kkt_t* out);

/* Per-instance residuals and counters of the last solve into HOST out[count]; count must
 * equal the number of loaded instances.  `iterations` is the iteration count at the
 * instance's last check (where it converged, for a converged instance). */
int dpdlp_get_batch_kkt(dpdlp_t* h, dpdlp_kkt_t* out, int32_t count);

/* Copy up to `cap` trace records, oldest first, into HOST `out`; *count receives the number
 * copied. */
int dpdlp_get_trace(dpdlp_t* h, dpdlp_trace_t* out, int32_t cap, int32_t* count);

/* Checkpoint: the current iterate (x[n], y[m]), anchor (x0[n], y0[m]) and scalars.  After
 * dpdlp_set_state the next dpdlp_solve resumes from it and reproduces the uninterrupted
 * solve.  Vector pointers may be NULL to skip them (get) -- set needs all four. */
int dpdlp_get_state(dpdlp_t* h, double* x, double* y, double* x0, double* y0,
                    dpdlp_scalar_state_t* s);
int dpdlp_set_state(dpdlp_t* h, const double* x, const double* y, const double* x0,
                    const double* y0, const dpdlp_scalar_state_t* s);

/* Parity mode: restart decisions of checks 0..count-1 (0 none, 1..3 restart kinds) are
 * taken from `kinds` (HOST) instead of the restart test; checks past the schedule make no
 * restart.  The schedule stays in force for every later solve until count = 0 switches it
 * off (a fresh solve counts its checks from 0, a resumed one continues the count).  For a batch of N instances
 * count = N * L and kinds[i * L + c] is instance i's decision at check c (count not a
 * multiple of N: DPDLP_ERR_INVALID). */
int dpdlp_set_schedule(dpdlp_t* h, const int8_t* kinds, int32_t count);

/* Operator application with the solver's SpMV kernels: out[m] = A x[n], out[n] = A^T y[m]. */
int dpdlp_apply_A(dpdlp_t* h, const double* x, double* out);
int dpdlp_apply_AT(dpdlp_t* h, const double* y, double* out);

/* Time `reps` back-to-back launches of one iteration kernel ("primal": fused CSC SpMV +
 * primal update, "dual": fused CSR SpMV + dual update) on the handle's stream with CUDA
 * events, on the current state (the state is left as it was).  *avg_ms = mean duration of
 * one launch.  Needs a solve or dpdlp_set_start beforehand.  Other names:
 *   "primal_slots", "dual_slots": the same without the long-row pass (the slot kernel);
 *   "gather_primal", "access_primal", "stream_primal", "memory_primal" (and _dual):
 *   access probes of the orientation's product -- its index stream and x[col] gathers;
 *   plus its value stream; its two streams alone; the product's loads plus the loads and
 *   stores of the epilogue's row vectors (every access of the kernel's slots) -- without
 *   arithmetic (ceilings of the access pattern), launched like the kernels (programmatic
 *   dependents when the "pdl" parameter is on);
 *   "primal_list", "primal_idle", "primal_list_idle" (and dual_), batches only: the
 *   persistent kernel walking the list of every slot, a launch over every slot with all
 *   instances stopped, the list kernel over an empty list (costs the autotuner compares). */
int dpdlp_time_kernel(dpdlp_t* h, const char* which, int32_t reps, double* avg_ms);

/* Sizes and layout of the loaded LP. */
int dpdlp_get_info(dpdlp_t* h, dpdlp_info_t* out);

/* y[m] = A x[n] for a plain CSR matrix already in DEVICE memory, allocating nothing.
 * The paper has no counterpart: this is a service for callers that cannot allocate device
 * memory where they need the product -- frameworks whose own pool has reserved the
 * device's memory (a cudaMalloc behind its back fails or fragments it), and
 * latency-critical loops that must not stall on the allocator (cudaMalloc and cudaFree
 * may synchronize the device).
 *   row_ptr[m+1] (int32, row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz), col_idx[nnz]
 *   (int32 in [0, n)), val[nnz], x[n], y[m]: device pointers on the current device; the
 *   caller guarantees a valid CSR (it is not checked on the device).  In particular nnz
 *   must equal row_ptr[m]: a smaller nnz leaves the last rows with truncated sums.
 *   cuda_stream: a cudaStream_t or NULL; the call only enqueues work, y is ready when the
 *   stream reaches this point.
 * Scratch: one fixed array of 192 KB per device (static device storage, reserved when the
 * library is loaded and held until the process exits) for the partial sums of rows that
 * cross thread-block boundaries.  Every call on a device shares it, so calls that may run
 * concurrently on the GPU (different streams without ordering) race and must not overlap;
 * each call rewrites every slot it reads, so nothing needs clearing between calls.  The
 * first call on a device looks up the array's device address (once per device, with that
 * device current) and keeps it for the life of the process.  A device reset
 * (cudaDeviceReset) unloads the array and leaves the kept address stale: do not call this
 * entry point on a device after resetting it.
 * Limits: nnz <= 2^30 (DPDLP_ERR_TOO_LARGE beyond it); negative sizes or NULL pointers:
 * DPDLP_ERR_INVALID; a failed launch or lookup: DPDLP_ERR_CUDA.  Results are deterministic
 * (fixed summation order) and agree with dpdlp_apply_A to rounding. */
int dpdlp_csr_spmv_noalloc(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr,
                           const int32_t* col_idx, const double* val, const double* x, double* y,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DPDLP_H */

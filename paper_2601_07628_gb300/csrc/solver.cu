// C ABI of libdpdlp (declared in include/dpdlp.h): handle, load, solve loop, getters.
//
// The solve loop is one CUDA graph: a conditional WHILE node whose body holds
// check_every iterations (primal kernel, dual kernel) followed by the check kernels; the
// control kernel of the check sets the loop condition on the device, so the host waits
// once per solve.  With use_graph = 0 the same kernels are launched from a host loop that
// reads the status after every check.
//
// A handle holds a batch of independent LPs (a single LP is a batch of one): the matrix is
// block diagonal, every instance keeps its rows and columns in its own index range, has
// its own step sizes, primal weight, restart epoch and status, and all instances take
// their iterations in the same kernels.  Converged instances are skipped; the loop ends
// when no instance is running.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dpdlp.h"
#include "internal.h"

using namespace pdhg;

namespace {

struct Param {
  double value, lo, hi;
  bool integer;
};

std::map<std::string, Param> default_params() {
  return {
      {"eta", {0.0, 0.0, 1e300, false}},
      {"eta_safety", {0.998, 1e-6, 1.0, false}},
      {"power_iters", {200, 1, 100000, true}},
      {"power_tol", {1e-8, 0.0, 1.0, false}},
      {"omega0", {0.0, 0.0, 1e300, false}},
      {"gamma", {1.0, 0.0, 1.0, false}},
      {"halpern", {1, 0, 1, true}},
      {"check_every", {64, 1, KMAX, true}},
      {"restart", {1, 0, 1, true}},
      {"beta_sufficient", {0.2, 0.0, 1.0, false}},
      {"beta_necessary", {0.8, 0.0, 1.0, false}},
      {"beta_artificial", {0.36, 0.0, 1.0, false}},
      {"pid", {1, 0, 1, true}},
      {"pid_kp", {0.99, -1e3, 1e3, false}},
      {"pid_ki", {0.01, -1e3, 1e3, false}},
      {"pid_kd", {0.0, -1e3, 1e3, false}},
      {"block_permute", {1, 0, 1, true}},
      {"perm_block", {256, 1, 1 << 30, true}},
      {"perm_seed", {1, 0, 9007199254740992.0, true}},
      {"use_graph", {1, 0, 1, true}},
      {"pdl", {1, 0, 1, true}},
      {"ptr_mode_device", {0, 0, 1, true}},
      {"resume", {0, 0, 1, true}},
      {"trace_capacity", {4096, 0, 1 << 20, true}},
      {"spmv_fp32", {0, 0, 2, true}},
      {"fp32_switch_tol", {1e-6, 0.0, 1.0, false}},
      {"fp32_stall_checks", {64, 1, 1 << 30, true}},
      {"precond", {0, 0, 1, true}},
      {"ruiz_passes", {10, 0, 100, true}},
      {"pock_chambolle", {1, 0, 1, true}},
      {"list_fraction", {0.5, 0.0, 2.0, false}},
      {"list_warps_per_sm", {0, 0, 64, true}},
      {"list_few_slots", {256, 0, 1 << 20, true}},
      {"cta_slots_primal", {4, 2, 8, true}},
      {"cta_slots_dual", {4, 2, 8, true}},
      {"fused_body", {1, 0, 1, true}},
      {"fused_max_slots", {48, 1, FUSED_MAX_SLOTS, true}},
      {"fused_cluster", {0, 0, 8, true}},
      {"fused_slot_cache", {1, 0, 1, true}},
  };
}

}  // namespace

struct dpdlp {
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  std::map<std::string, Param> params = default_params();

  bool loaded = false;
  int n = 0, m = 0;
  int64_t nnz = 0;
  std::vector<int32_t> prow, pcol;  // internal index -> caller index
  std::vector<double> h_lc, h_uc;   // caller order
  DevPacked csr, csc;
  DevVecs v;
  double *xs = nullptr, *ys = nullptr;  // warm start (internal order)
  bool have_start_x = false, have_start_y = false;
  DevScalars* d_sc = nullptr;
  DevScalars h_sc{};
  int ninst = 1;
  std::vector<int32_t> row_off, col_off;    // instance ranges (caller = internal ranges)
  std::vector<InstScalars> h_inst;          // host mirror of the instance scalars
  std::vector<double> inst_bnorm, inst_cnorm;       // original LP (KKT denominators)
  std::vector<double> inst_bnorm_s, inst_cnorm_s;   // the LP PDHG runs on (initial omega)
  // diagonal preconditioning (internal order; empty / nullptr when off): the solver works
  // on D_r A D_c, x = D_c xs, y = D_r ys; every factor is a power of two
  std::vector<double> dr, dc;
  double *d_dr = nullptr, *d_dc = nullptr, *d_rw = nullptr, *d_cw = nullptr;
  double* d_q = nullptr;  // diagonal of Q (a diagonal QP), internal order
  std::vector<double> eta_inst;             // power-iteration step size per instance
  bool eta_valid = false;
  std::vector<double> eta_user;             // per-instance step sizes set by the caller
  bool pending_state = false;
  bool has_state = false;
  int trace_cap = 0;

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_K = -1;

  std::vector<std::pair<void*, size_t>> allocs;
  int64_t dev_bytes = 0;
  dpdlp_alloc_fn alloc_fn = nullptr;  // caller's allocator (nullptr: cudaMalloc)
  dpdlp_release_fn release_fn = nullptr;
  void* alloc_ctx = nullptr;
  dpdlp_info_t info{};

  double P(const char* k) const { return params.at(k).value; }
};

namespace {

int fail(dpdlp* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(h, e_ == cudaErrorMemoryAllocation ? DPDLP_ERR_OOM : DPDLP_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

template <class T>
int dalloc(dpdlp* h, T** p, size_t count) {
  *p = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  if (h->alloc_fn) {
    void* q = h->alloc_fn(bytes, h->alloc_ctx);
    if (!q) return fail(h, DPDLP_ERR_OOM, "the allocator hook returned NULL");
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      h->release_fn(q, bytes, h->alloc_ctx);
      return fail(h, DPDLP_ERR_INVALID, "the allocator hook returned memory not aligned to 256 bytes");
    }
    *p = static_cast<T*>(q);
  } else {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
      *p = nullptr;
      return fail(h, DPDLP_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
  }
  h->allocs.emplace_back(*p, bytes);
  h->dev_bytes += bytes;
  return 0;
}

// Releases one buffer of the handle's allocations; the caller has drained the stream and
// no captured graph refers to it.
void dfree(dpdlp* h, void* p) {
  for (size_t k = 0; k < h->allocs.size(); ++k) {
    if (h->allocs[k].first != p) continue;
    if (h->release_fn) h->release_fn(p, h->allocs[k].second, h->alloc_ctx);
    else cudaFree(p);
    h->dev_bytes -= (int64_t)h->allocs[k].second;
    h->allocs.erase(h->allocs.begin() + (std::ptrdiff_t)k);
    return;
  }
}

void free_graph(dpdlp* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  h->graph_K = -1;
}

void free_problem(dpdlp* h) {
  free_graph(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (const auto& a : h->allocs) {
    if (h->release_fn) h->release_fn(a.first, a.second, h->alloc_ctx);
    else cudaFree(a.first);
  }
  h->allocs.clear();
  h->dev_bytes = 0;
  h->csr = DevPacked{};
  h->csc = DevPacked{};
  h->v = DevVecs{};
  h->xs = h->ys = nullptr;
  h->d_sc = nullptr;
  h->d_dr = h->d_dc = h->d_rw = h->d_cw = nullptr;
  h->d_q = nullptr;
  h->dr.clear();
  h->dc.clear();
  h->loaded = false;
  h->eta_valid = false;
  h->pending_state = false;
  h->has_state = false;
  h->have_start_x = h->have_start_y = false;
}

int upload_packed(dpdlp* h, const HostPacked& H, DevPacked& D) {
  D.rows = H.rows;
  D.cols = H.cols;
  D.nslots = H.nslots;
  D.nlong = H.nlong;
  D.npieces = H.npieces;
  D.nlong_block = H.nlong_block;
  D.nlong_warp = H.nlong_warp;
  int rc;
  double *val, *psum;
  float* val32 = nullptr;
  uint32_t* idx;
  SlotDesc* slots;
  LaneMeta* lanes;
  int32_t *lrow, *linst, *lptr, *lpiece;
  if ((rc = dalloc(h, &val, H.val.size()))) return rc;
  if ((rc = dalloc(h, &idx, H.idx.size()))) return rc;
  if (H.fp32_exact_range && (rc = dalloc(h, &val32, H.val32.size()))) return rc;
  if ((rc = dalloc(h, &slots, H.slots.size()))) return rc;
  if ((rc = dalloc(h, &lanes, H.lanes.size()))) return rc;
  if ((rc = dalloc(h, &lrow, H.long_row.size()))) return rc;
  if ((rc = dalloc(h, &linst, H.long_inst.size()))) return rc;
  if ((rc = dalloc(h, &lptr, H.long_ptr.size()))) return rc;
  if ((rc = dalloc(h, &lpiece, H.long_piece.size()))) return rc;
  if ((rc = dalloc(h, &psum, 2 * (size_t)H.npieces))) return rc;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  CK(up(val, H.val.data(), H.val.size() * sizeof(double)));
  CK(up(idx, H.idx.data(), H.idx.size() * sizeof(uint32_t)));
  if (val32) CK(up(val32, H.val32.data(), H.val32.size() * sizeof(float)));
  CK(up(slots, H.slots.data(), H.slots.size() * sizeof(SlotDesc)));
  CK(up(lanes, H.lanes.data(), H.lanes.size() * sizeof(LaneMeta)));
  CK(up(lrow, H.long_row.data(), H.long_row.size() * sizeof(int32_t)));
  CK(up(linst, H.long_inst.data(), H.long_inst.size() * sizeof(int32_t)));
  CK(up(lptr, H.long_ptr.data(), H.long_ptr.size() * sizeof(int32_t)));
  CK(up(lpiece, H.long_piece.data(), H.long_piece.size() * sizeof(int32_t)));
  D.val = val;
  D.val32 = val32;
  D.idx = idx;
  D.slots = slots;
  D.lanes = lanes;
  D.long_row = lrow;
  D.long_inst = linst;
  D.long_ptr = lptr;
  D.long_piece = lpiece;
  D.piece_sum = psum;
  return 0;
}

template <class T>
std::vector<T> permuted(const T* src, const std::vector<int32_t>& p) {
  std::vector<T> out(p.size());
  for (size_t i = 0; i < p.size(); ++i) out[i] = src[p[i]];
  return out;
}

// ||[lc, uc]|| over finite entries of rows [r0, r1), an equality row counted once (reading
// of the r_primal denominator of Appendix B.4 and of the initial primal weight).
double bound_norm(const std::vector<double>& lc, const std::vector<double>& uc, int r0, int r1) {
  double s = 0.0;
  for (int i = r0; i < r1; ++i) {
    const bool lf = std::isfinite(lc[i]), uf = std::isfinite(uc[i]);
    if (lf && uf && lc[i] == uc[i]) {
      s += lc[i] * lc[i];
    } else {
      if (lf) s += lc[i] * lc[i];
      if (uf) s += uc[i] * uc[i];
    }
  }
  return std::sqrt(s);
}

// The -S box of the LP the solver iterates on (rows scaled by D_r when preconditioned),
// and the bound norms of the original and of the scaled LP.
int upload_row_bounds(dpdlp* h) {
  std::vector<double> lo(h->m), hi(h->m), lcs(h->h_lc), ucs(h->h_uc);
  for (int i = 0; i < h->m; ++i) {
    const int o = h->prow[i];
    if (!h->dr.empty()) {
      lcs[o] = h->h_lc[o] * h->dr[i];
      ucs[o] = h->h_uc[o] * h->dr[i];
    }
    lo[i] = -ucs[o];
    hi[i] = -lcs[o];
  }
  if (h->m) {
    CK(cudaMemcpy(h->v.lo, lo.data(), h->m * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->v.hi, hi.data(), h->m * sizeof(double), cudaMemcpyHostToDevice));
  }
  h->inst_bnorm.assign(h->ninst, 0.0);
  h->inst_bnorm_s.assign(h->ninst, 0.0);
  for (int i = 0; i < h->ninst; ++i) {
    h->inst_bnorm[i] = bound_norm(h->h_lc, h->h_uc, h->row_off[i], h->row_off[i + 1]);
    h->inst_bnorm_s[i] = bound_norm(lcs, ucs, h->row_off[i], h->row_off[i + 1]);
  }
  return 0;
}

bool ptr_device(const dpdlp* h) { return h->P("ptr_mode_device") != 0.0; }

// Caller vector (caller order, host or device) -> internal-order device vector `dst`.
int import_vec(dpdlp* h, const double* src, double* dst, const int32_t* perm, int len,
               double* staging, const double* scale) {
  if (len == 0) return 0;
  const double* dsrc = src;
  if (!ptr_device(h)) {
    CK(cudaMemcpyAsync(staging, src, len * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    dsrc = staging;
  }
  CK(launch_gather(dsrc, perm, scale, dst, len, h->stream));
  return 0;
}

// Internal-order device vector -> caller vector (caller order, host or device).
int export_vec(dpdlp* h, const double* src, double* dst, const int32_t* perm, int len,
               double* staging, const double* scale) {
  if (len == 0 || !dst) return 0;
  if (ptr_device(h)) {
    CK(launch_scatter(src, perm, scale, dst, len, h->stream));
  } else {
    CK(launch_scatter(src, perm, scale, staging, len, h->stream));
    CK(cudaMemcpyAsync(dst, staging, len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

// eta_i = eta_safety / sigma_max(A_i) for every instance i by power iteration on A_i^T A_i
// (start 1/sqrt(n_i), stop when the Rayleigh quotient changes by <= power_tol relatively,
// at most power_iters rounds); eta_i = 1 when A_i has no nonzeros.  The instances iterate
// together; each keeps the quotient of the round at which it stopped.
int compute_eta(dpdlp* h) {
  if (h->eta_valid) return 0;
  const int n = h->n, N = h->ninst;
  std::vector<double> lam(N, 0.0), lam_prev(N, 0.0);
  std::vector<char> done(N, 0);
  if (n > 0 && h->nnz > 0) {
    double* vv = h->v.tmp_n;
    double* ww = h->v.tmp_m;
    double* uu = h->v.tmp_n2;
    std::vector<double> start(n);
    for (int i = 0; i < N; ++i) {
      const int a = h->col_off[i], b = h->col_off[i + 1];
      for (int j = a; j < b; ++j) start[j] = 1.0 / std::sqrt((double)(b - a));
      if (a == b) done[i] = 1;
    }
    CK(cudaMemcpyAsync(vv, start.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const int iters = (int)h->P("power_iters");
    const double tol = h->P("power_tol");
    std::vector<double> pw(4 * (size_t)N);
    int left = 0;
    for (int i = 0; i < N; ++i) left += !done[i];
    for (int it = 0; it < iters && left > 0; ++it) {
      CK(launch_power_round(h->csr, h->csc, h->v, vv, ww, uu, h->stream));
      CK(cudaMemcpyAsync(pw.data(), h->v.pw, pw.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int i = 0; i < N; ++i) {
        if (done[i]) continue;
        lam[i] = pw[4 * i];
        if (pw[4 * i + 1] == 0.0 || lam[i] == 0.0 || std::fabs(lam[i] - lam_prev[i]) <= tol * lam[i]) {
          done[i] = 1;
          --left;
        } else {
          lam_prev[i] = lam[i];
        }
      }
    }
  }
  h->eta_inst.assign(N, 1.0);
  for (int i = 0; i < N; ++i) {
    const double s = std::sqrt(lam[i]);
    h->eta_inst[i] = s > 0.0 ? h->P("eta_safety") / s : 1.0;
  }
  h->eta_valid = true;
  return 0;
}

// Halpern weights of the next graph body for every instance, from its k_base.
int upload_weights(dpdlp* h) {
  const int K = h->h_sc.K;
  std::vector<double> w((size_t)h->ninst * 2 * KMAX, 0.0);
  for (int i = 0; i < h->ninst; ++i) {
    const double kb = (double)h->h_inst[i].k_base;
    double* wi = w.data() + (size_t)i * 2 * KMAX;
    for (int k = 0; k < K; ++k) {
      wi[k] = (kb + k + 1.0) / (kb + k + 2.0);
      wi[KMAX + k] = 1.0 / (kb + k + 2.0);
    }
  }
  CK(cudaMemcpyAsync(h->v.wtab, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

void copy_params(dpdlp* h, DevScalars& s) {
  s.gamma = h->P("gamma");
  s.halpern = (int)h->P("halpern");
  s.K = (int)h->P("check_every");
  s.restart_enabled = (int)h->P("restart");
  s.pid_enabled = (int)h->P("pid");
  s.beta_s = h->P("beta_sufficient");
  s.beta_n = h->P("beta_necessary");
  s.beta_a = h->P("beta_artificial");
  s.kp = h->P("pid_kp");
  s.ki = h->P("pid_ki");
  s.kd = h->P("pid_kd");
  s.ninst = h->ninst;
  s.trace_cap = h->trace_cap;
  s.fp32_switch = h->P("spmv_fp32") == 1.0;
  s.fp32_switch_tol = h->P("fp32_switch_tol");
  s.fp32_stall_limit = (int)h->P("fp32_stall_checks");
}

// Instance scalars at iteration 0 with step size eta and primal weight omega.
InstScalars fresh_inst(const dpdlp* h, int i, double eta, double omega, int fp32) {
  InstScalars I;
  std::memset(&I, 0, sizeof(I));
  I.eta = eta;
  I.omega = omega;
  I.tau = eta / omega;
  I.sigma = eta * omega;
  I.inv_sigma = 1.0 / I.sigma;
  I.bnorm = h->inst_bnorm[i];
  I.cnorm = h->inst_cnorm[i];
  I.status = -1;
  I.apply_mode = 2;
  I.spmv_fp32 = fp32;
  I.best_kkt = INFINITY;
  return I;
}

// Fresh start: x = proj_X(0) (or the warm start), y = 0 (or the warm start), anchor = start.
int init_fresh(dpdlp* h) {
  int rc;
  const double pe = h->P("eta");
  if (pe <= 0.0 && h->eta_user.empty() && (rc = compute_eta(h))) return rc;
  const double po = h->P("omega0");
  if (h->have_start_x && h->n)
    CK(cudaMemcpyAsync(h->v.x, h->xs, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h->have_start_y && h->m)
    CK(cudaMemcpyAsync(h->v.y, h->ys, h->m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(launch_fill_start(h->v, h->have_start_x ? 0 : 1, h->have_start_y ? 0 : 1, h->stream));
  DevScalars& s = h->h_sc;
  const int sched = s.sched_len;  // the forced schedule outlives a fresh start
  std::memset(&s, 0, sizeof(s));
  s.sched_len = sched;
  s.status = -1;
  const int fp32 = (h->P("spmv_fp32") >= 1.0 && h->csr.val32 && h->csc.val32) ? 1 : 0;
  h->h_inst.resize(h->ninst);
  for (int i = 0; i < h->ninst; ++i) {
    const double eta = pe > 0.0 ? pe : (!h->eta_user.empty() ? h->eta_user[i] : h->eta_inst[i]);
    const double cn = h->inst_cnorm_s[i], bn = h->inst_bnorm_s[i];  // of the LP iterated on
    const double omega = po > 0.0 ? po : ((cn > 0.0 && bn > 0.0) ? cn / bn : 1.0);
    h->h_inst[i] = fresh_inst(h, i, eta, omega, fp32);
  }
  h->has_state = true;
  return 0;
}

// A small single LP runs each graph body as one fused launch (same results, fewer launches):
// one thread block up to 6 slots per copy, a thread-block cluster beyond (fused_cluster_ctas);
// measured faster than the separate launches up to about 50 slots per copy (48: 13.1 against
// 13.5 us per iteration; 64: 14.6 against 13.7), hence fused_max_slots = 48 by default.
bool use_fused(const dpdlp* h) {
  return h->P("fused_body") != 0.0 &&
         fused_body_fits(h->csc, h->csr, h->ninst, (int)h->P("fused_max_slots"));
}

int build_graph(dpdlp* h, int K) {
  free_graph(h);
  CK(cudaGraphCreate(&h->graph, 0));
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, h->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  const int pdl = (int)h->P("pdl");
  // K iterations captured into graph g after `deps`
  auto capture_iters = [&](cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, int list) {
    cudaError_t e = cudaStreamBeginCaptureToGraph(h->cap_stream, g, deps, nullptr, ndeps, mode);
    for (int i = 0; i < K && e == cudaSuccess; ++i) {
      e = launch_primal(h->csc, h->v, h->d_sc, IterPlan{i, 0, list, pdl}, h->cap_stream);
      if (e == cudaSuccess) e = launch_dual(h->csr, h->v, h->d_sc, IterPlan{i, 0, list, pdl}, h->cap_stream);
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
    return e != cudaSuccess ? e : e2;
  };
  cudaError_t e = cudaSuccess;
  if (use_fused(h)) CK(fused_body_prepare());  // a function attribute, set outside the capture
  if (h->ninst == 1) {  // one capture: the iterations, then the check
    e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, mode);
    if (use_fused(h)) {
      if (e == cudaSuccess)
        e = launch_body_fused(h->csc, h->csr, h->v, h->d_sc, K,
                              fused_cluster_ctas(h->csc, h->csr, (int)h->P("fused_cluster")),
                              (int)h->P("fused_slot_cache"), h->cap_stream);
    } else {
      for (int i = 0; i < K && e == cudaSuccess; ++i) {
        e = launch_primal(h->csc, h->v, h->d_sc, IterPlan{i, 0, 0, pdl}, h->cap_stream);
        if (e == cudaSuccess) e = launch_dual(h->csr, h->v, h->d_sc, IterPlan{i, 0, 0, pdl}, h->cap_stream);
      }
    }
    if (e == cudaSuccess)
      e = launch_check(h->csr, h->csc, h->v, h->d_sc, (unsigned long long)handle, 1, h->cap_stream);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
    if (e == cudaSuccess) e = e2;
  } else {
    // a batch: a select kernel sets a SWITCH condition from the active-slot counts, then the
    // body's iterations launch over every slot (0), walk the lists (1) or walk them with small
    // grids when few slots are left (2), then the check
    cudaGraphConditionalHandle sel;
    CK(cudaGraphConditionalHandleCreate(&sel, body, 0, 0));
    e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, mode);
    if (e == cudaSuccess)
      e = launch_select(h->csr, h->csc, (unsigned long long)sel, h->P("list_fraction"),
                        (int)h->P("list_few_slots"), h->cap_stream);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
    if (e == cudaSuccess) e = e2;
    cudaGraphNode_t sel_node = nullptr, if_node = nullptr;
    if (e == cudaSuccess) {
      size_t nn = 1;
      CK(cudaGraphGetNodes(body, &sel_node, &nn));
      cudaGraphNodeParams ip{};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = sel;
      ip.conditional.type = cudaGraphCondTypeSwitch;
      ip.conditional.size = 3;
      CK(cudaGraphAddNode(&if_node, body, &sel_node, nullptr, 1, &ip));
      e = capture_iters(ip.conditional.phGraph_out[0], nullptr, 0, 0);
      if (e == cudaSuccess) e = capture_iters(ip.conditional.phGraph_out[1], nullptr, 0, 1);
      if (e == cudaSuccess) e = capture_iters(ip.conditional.phGraph_out[2], nullptr, 0, 2);
    }
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, &if_node, nullptr, 1, mode);
      if (e == cudaSuccess)
        e = launch_check(h->csr, h->csc, h->v, h->d_sc, (unsigned long long)handle, 1, h->cap_stream);
      const cudaError_t e3 = cudaStreamEndCapture(h->cap_stream, &captured);
      if (e == cudaSuccess) e = e3;
    }
  }
  if (e != cudaSuccess) return fail(h, DPDLP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  CK(cudaGraphInstantiate(&h->exec, h->graph, 0));
  h->graph_K = K;
  return 0;
}

int run_host_loop(dpdlp* h) {
  const int K = h->h_sc.K;
  if (use_fused(h)) CK(fused_body_prepare());
  const int pdl = (int)h->P("pdl");
  for (;;) {
    int list = 0;
    if (h->ninst > 1) {  // the same choice the graph's select kernel makes
      int32_t na[2] = {0, 0};
      CK(cudaMemcpyAsync(&na[0], h->csr.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(&na[1], h->csc.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      list = select_form(na[0] + na[1], (long long)h->csr.nslots + h->csc.nslots,
                         h->P("list_fraction"), (int)h->P("list_few_slots"));
    }
    if (use_fused(h)) {
      CK(launch_body_fused(h->csc, h->csr, h->v, h->d_sc, K,
                           fused_cluster_ctas(h->csc, h->csr, (int)h->P("fused_cluster")),
                           (int)h->P("fused_slot_cache"), h->stream));
    } else {
      for (int i = 0; i < K; ++i) {
        CK(launch_primal(h->csc, h->v, h->d_sc, IterPlan{i, 0, list, pdl}, h->stream));
        CK(launch_dual(h->csr, h->v, h->d_sc, IterPlan{i, 0, list, pdl}, h->stream));
      }
    }
    CK(launch_check(h->csr, h->csc, h->v, h->d_sc, 0ULL, 0, h->stream));
    int status = -1;
    CK(cudaMemcpyAsync(&status, &h->d_sc->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (status != -1) return 0;
  }
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

int dpdlp_create(dpdlp_t** out, int device) {
  if (!out) return DPDLP_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return DPDLP_ERR_INVALID;
  dpdlp* h = new (std::nothrow) dpdlp();
  if (!h) return DPDLP_ERR_OOM;
  h->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return DPDLP_ERR_CUDA;
  }
  h->stream = h->own_stream;
  *out = h;
  return 0;
}

void dpdlp_destroy(dpdlp_t* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  free_problem(h);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

const char* dpdlp_last_error(const dpdlp_t* h) { return h ? h->err.c_str() : "null handle"; }

int dpdlp_set_allocator(dpdlp_t* h, dpdlp_alloc_fn alloc, dpdlp_release_fn release, void* ctx) {
  if (!h || (alloc == nullptr) != (release == nullptr))
    return fail(h, DPDLP_ERR_INVALID, "allocator: give both functions or neither");
  cudaSetDevice(h->device);
  free_problem(h);  // buffers go back to the allocator they came from
  h->alloc_fn = alloc;
  h->release_fn = release;
  h->alloc_ctx = ctx;
  return 0;
}

int dpdlp_set_stream(dpdlp_t* h, void* s) {
  if (!h) return DPDLP_ERR_INVALID;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  h->stream = s ? (cudaStream_t)s : h->own_stream;
  return 0;
}

int dpdlp_set_param(dpdlp_t* h, const char* key, double v) {
  if (!h || !key) return DPDLP_ERR_INVALID;
  auto it = h->params.find(key);
  if (it == h->params.end()) return fail(h, DPDLP_ERR_INVALID, std::string("unknown parameter: ") + key);
  Param& p = it->second;
  if (!(v >= p.lo && v <= p.hi) || (p.integer && v != std::floor(v)))
    return fail(h, DPDLP_ERR_INVALID, std::string("value out of range for ") + key);
  const std::string k(key);
  if ((k == "cta_slots_primal" || k == "cta_slots_dual") && v != 2 && v != 4 && v != 8)
    return fail(h, DPDLP_ERR_INVALID, k + " must be 2, 4 or 8");
  if ((k == "check_every" || k == "cta_slots_primal" || k == "cta_slots_dual" ||
       k == "fused_body" || k == "fused_max_slots" || k == "fused_cluster" || k == "pdl" ||
       k == "fused_slot_cache" ||
       k == "list_fraction" || k == "list_few_slots" ||
       k == "list_warps_per_sm") && v != p.value)
    free_graph(h);  // the captured graph holds the launch shapes
  if (std::string(key) == "eta_safety" || std::string(key) == "power_iters" ||
      std::string(key) == "power_tol")
    h->eta_valid = false;
  p.value = v;
  h->csc.cta_slots = (int)h->P("cta_slots_primal");
  h->csr.cta_slots = (int)h->P("cta_slots_dual");
  h->csc.list_warps_per_sm = h->csr.list_warps_per_sm = (int)h->P("list_warps_per_sm");
  h->csc.list_few_slots = h->csr.list_few_slots = (int)h->P("list_few_slots");
  return 0;
}

int dpdlp_get_param(const dpdlp_t* h, const char* key, double* v) {
  if (!h || !key || !v) return DPDLP_ERR_INVALID;
  auto it = h->params.find(key);
  if (it == h->params.end()) return DPDLP_ERR_INVALID;
  *v = it->second.value;
  return 0;
}

}  // extern "C"

namespace {

// Loads `count` instances: instance i owns rows [row_off[i], row_off[i+1]) and columns
// [col_off[i], col_off[i+1]) of one block-diagonal matrix.
int load_impl(dpdlp* h, int32_t count, const int32_t* row_off, const int32_t* col_off,
              int32_t n, int32_t m, const double* c, const int64_t* row_ptr,
              const int32_t* col_idx, const double* val, const double* b, const double* lv,
              const double* uv, const int8_t* ctype) {
  CK(cudaSetDevice(h->device));
  const auto t0 = std::chrono::steady_clock::now();
  if (n < 0 || m < 0) return fail(h, DPDLP_ERR_INVALID, "negative dimension");
  if ((n > 0 && (!c || !lv || !uv)) || !row_ptr)
    return fail(h, DPDLP_ERR_INVALID, "NULL input array");
  if ((b == nullptr) != (ctype == nullptr))
    return fail(h, DPDLP_ERR_INVALID, "b and ctype must both be given or both be NULL");
  if (m > (int32_t)IDX_MASK) return fail(h, DPDLP_ERR_INVALID, "too many rows for the packed index format");
  if (count < 1 || !row_off || !col_off) return fail(h, DPDLP_ERR_INVALID, "invalid instance count or ranges");
  if (row_off[0] != 0 || col_off[0] != 0 || row_off[count] != m || col_off[count] != n)
    return fail(h, DPDLP_ERR_INVALID, "instance ranges must start at 0 and end at m and n");
  for (int i = 0; i < count; ++i) {
    if (row_off[i + 1] < row_off[i] || col_off[i + 1] < col_off[i])
      return fail(h, DPDLP_ERR_INVALID, "instance ranges must be non-decreasing");
    // An empty row is stored as one zero entry gathering column 0 of its instance, which
    // must exist (in the fused body's shared copies as much as in global memory).
    if (col_off[i + 1] == col_off[i])
      return fail(h, DPDLP_ERR_INVALID, "an LP (each instance of a batch) needs at least one variable");
  }
  std::string e = validate_csr(m, n, row_ptr, col_idx, val);
  if (!e.empty()) return fail(h, DPDLP_ERR_INVALID, e);
  for (int i = 0; i < count; ++i)
    for (int r = row_off[i]; r < row_off[i + 1]; ++r)
      for (int64_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q)
        if (col_idx[q] < col_off[i] || col_idx[q] >= col_off[i + 1])
          return fail(h, DPDLP_ERR_INVALID, "nonzero outside its instance's columns in row " +
                                                std::to_string(r));
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(c[j])) return fail(h, DPDLP_ERR_INVALID, "non-finite objective coefficient");
    if (std::isnan(lv[j]) || std::isnan(uv[j]) || lv[j] > uv[j] || lv[j] == INFINITY ||
        uv[j] == -INFINITY)
      return fail(h, DPDLP_ERR_INVALID, "invalid variable bounds at " + std::to_string(j));
  }
  std::vector<double> lc(m, -INFINITY), uc(m, INFINITY);
  if (ctype) {
    for (int i = 0; i < m; ++i) {
      if (!std::isfinite(b[i])) return fail(h, DPDLP_ERR_INVALID, "non-finite right-hand side");
      switch (ctype[i]) {
        case 0: lc[i] = b[i]; uc[i] = b[i]; break;
        case 1: uc[i] = b[i]; break;
        case 2: lc[i] = b[i]; break;
        default: return fail(h, DPDLP_ERR_INVALID, "constraint type must be 0, 1 or 2");
      }
    }
  }
  free_problem(h);
  h->n = n;
  h->m = m;
  h->nnz = row_ptr[m];
  h->h_lc = lc;
  h->h_uc = uc;
  h->ninst = count;
  h->row_off.assign(row_off, row_off + count + 1);
  h->col_off.assign(col_off, col_off + count + 1);
  h->eta_user.clear();
  // block permutation inside every instance (instance i draws seeds seed + 2i, seed + 2i + 1)
  const bool perm = h->P("block_permute") != 0.0;
  const int pb = (int)h->P("perm_block");
  const uint64_t seed = (uint64_t)h->P("perm_seed");
  h->prow.assign(m, 0);
  h->pcol.assign(n, 0);
  for (int i = 0; i < count; ++i) {
    const std::vector<int32_t> pr = block_permutation(row_off[i + 1] - row_off[i], pb, seed + 2 * (uint64_t)i, perm);
    const std::vector<int32_t> pc = block_permutation(col_off[i + 1] - col_off[i], pb, seed + 2 * (uint64_t)i + 1, perm);
    for (size_t k = 0; k < pr.size(); ++k) h->prow[row_off[i] + k] = row_off[i] + pr[k];
    for (size_t k = 0; k < pc.size(); ++k) h->pcol[col_off[i] + k] = col_off[i] + pc[k];
  }
  std::vector<int64_t> pptr, tptr;
  std::vector<int32_t> pidx, tidx;
  std::vector<double> pval, tval;
  permute_csr(m, n, row_ptr, col_idx, val, h->prow, h->pcol, pptr, pidx, pval);
  std::vector<double> drp, dcp;  // preconditioner factors, pre-packing order
  if (h->P("precond") != 0.0)
    precondition(m, n, pptr, pidx, pval, (int)h->P("ruiz_passes"), h->P("pock_chambolle") != 0.0,
                 drp, dcp);
  transpose_csr(m, n, pptr, pidx, pval, tptr, tidx, tval);
  // pack rows of A and rows of A^T into warp lanes; each packing fixes one index order
  PackPlan rplan, cplan;
  {  // the two orientations are planned independently: the columns on a second thread
    std::thread cols_thread([&] {
      if (count == 1) plan_packing(n, tptr, cplan);
      else plan_packing_batch(n, tptr, h->col_off, cplan);
    });
    if (count == 1) plan_packing(m, pptr, rplan);
    else plan_packing_batch(m, pptr, h->row_off, rplan);
    cols_thread.join();
  }
  HostPacked Hr, Hc;
  build_packed(m, n, pptr, pidx, pval, rplan, cplan.new_of_old, Hr);
  build_packed(n, m, tptr, tidx, tval, cplan, rplan.new_of_old, Hc);
  if (count > 1) {
    own_instance_zero_gathers(Hr, h->col_off);  // rows of A gather x_bar
    own_instance_zero_gathers(Hc, h->row_off);  // rows of A^T gather y
  }
  std::vector<int64_t>().swap(pptr);
  std::vector<int32_t>().swap(pidx);
  std::vector<double>().swap(pval);
  std::vector<int64_t>().swap(tptr);
  std::vector<int32_t>().swap(tidx);
  std::vector<double>().swap(tval);
  {  // internal index -> caller index: packing order after the block permutation
    std::vector<int32_t> pr(m), pc(n);
    for (int i = 0; i < m; ++i) pr[i] = h->prow[rplan.old_of_new[i]];
    for (int j = 0; j < n; ++j) pc[j] = h->pcol[cplan.old_of_new[j]];
    h->prow.swap(pr);
    h->pcol.swap(pc);
    if (!drp.empty() || !dcp.empty()) {
      h->dr.resize(m);
      h->dc.resize(n);
      for (int i = 0; i < m; ++i) h->dr[i] = drp[rplan.old_of_new[i]];
      for (int j = 0; j < n; ++j) h->dc[j] = dcp[cplan.old_of_new[j]];
    }
  }

  int rc;
  if ((rc = upload_packed(h, Hr, h->csr))) return rc;
  if ((rc = upload_packed(h, Hc, h->csc))) return rc;
  if (count > 1) {  // per-instance slot ranges and the active-slot lists of a batch
    for (int o = 0; o < 2; ++o) {
      const HostPacked& Hp = o == 0 ? Hr : Hc;
      DevPacked& D = o == 0 ? h->csr : h->csc;
      std::vector<int32_t> soff(count + 1, 0);
      for (const SlotDesc& d : Hp.slots) ++soff[d.inst + 1];
      for (int i = 0; i < count; ++i) soff[i + 1] += soff[i];
      int32_t *d_soff, *d_act, *d_nact;
      if ((rc = dalloc(h, &d_soff, count + 1)) || (rc = dalloc(h, &d_act, Hp.slots.size())) ||
          (rc = dalloc(h, &d_nact, 1)))
        return rc;
      CK(cudaMemcpy(d_soff, soff.data(), (count + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
      CK(cudaMemset(d_nact, 0, sizeof(int32_t)));
      D.slot_off = d_soff;
      D.active = d_act;
      D.nactive = d_nact;
    }
  }
  h->csc.cta_slots = (int)h->P("cta_slots_primal");
  h->csr.cta_slots = (int)h->P("cta_slots_dual");
  h->csc.list_warps_per_sm = h->csr.list_warps_per_sm = (int)h->P("list_warps_per_sm");
  h->csc.list_few_slots = h->csr.list_few_slots = (int)h->P("list_few_slots");
  DevVecs& v = h->v;
  v.n = n;
  v.m = m;
  v.ninst = count;
  double** nvecs[] = {&v.c, &v.lv, &v.uv, &v.x, &v.x0, &v.xbar, &v.xh, &v.dx, &v.aty,
                      &v.tmp_n, &v.tmp_n2, &h->xs};
  for (double** p : nvecs) {
    if ((rc = dalloc(h, p, n))) return rc;
    CK(cudaMemset(*p, 0, (n > 0 ? n : 2) * sizeof(double)));  // padding gathers read finite zeros
  }
  double** mvecs[] = {&v.lo, &v.hi, &v.y, &v.y0, &v.yh, &v.axh, &v.adx, &v.tmp_m, &h->ys};
  for (double** p : mvecs) {
    if ((rc = dalloc(h, p, m))) return rc;
    CK(cudaMemset(*p, 0, (m > 0 ? m : 2) * sizeof(double)));
  }
  // reduction chunks and the instance of every row and column
  std::vector<int32_t> chr, chc, icr, icc;
  build_chunks(h->row_off, RED_CHUNK, chr, icr);
  build_chunks(h->col_off, RED_CHUNK, chc, icc);
  v.g_rows = (int)chr.size() / 4;
  v.g_cols = (int)chc.size() / 4;
  std::vector<int32_t> ior(m), ioc(n);
  for (int i = 0; i < count; ++i) {
    for (int r = row_off[i]; r < row_off[i + 1]; ++r) ior[r] = i;
    for (int j = col_off[i]; j < col_off[i + 1]; ++j) ioc[j] = i;
  }
  int32_t *d_chr, *d_chc, *d_icr, *d_icc, *d_ior, *d_ioc;
  if ((rc = dalloc(h, &d_chr, chr.size()))) return rc;
  if ((rc = dalloc(h, &d_chc, chc.size()))) return rc;
  if ((rc = dalloc(h, &d_icr, icr.size()))) return rc;
  if ((rc = dalloc(h, &d_icc, icc.size()))) return rc;
  if ((rc = dalloc(h, &d_ior, m))) return rc;
  if ((rc = dalloc(h, &d_ioc, n))) return rc;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  CK(up(d_chr, chr.data(), chr.size() * sizeof(int32_t)));
  CK(up(d_chc, chc.data(), chc.size() * sizeof(int32_t)));
  CK(up(d_icr, icr.data(), icr.size() * sizeof(int32_t)));
  CK(up(d_icc, icc.data(), icc.size() * sizeof(int32_t)));
  CK(up(d_ior, ior.data(), ior.size() * sizeof(int32_t)));
  CK(up(d_ioc, ioc.data(), ioc.size() * sizeof(int32_t)));
  v.chunk_rows = reinterpret_cast<const int4*>(d_chr);
  v.chunk_cols = reinterpret_cast<const int4*>(d_chc);
  v.inst_chunk_rows = d_icr;
  v.inst_chunk_cols = d_icc;
  v.inst_of_row = d_ior;
  v.inst_of_col = d_ioc;
  const size_t gr = v.g_rows > 0 ? v.g_rows : 1, gc = v.g_cols > 0 ? v.g_cols : 1;
  if ((rc = dalloc(h, &v.red_rows, gr * NRED))) return rc;
  if ((rc = dalloc(h, &v.red_cols, gc * NRED))) return rc;
  if ((rc = dalloc(h, &v.perm_col, n))) return rc;
  if ((rc = dalloc(h, &v.perm_row, m))) return rc;
  if ((rc = dalloc(h, &v.pw, 4 * (size_t)count))) return rc;
  if ((rc = dalloc(h, &v.inst, count))) return rc;
  if ((rc = dalloc(h, &v.act_off, 2 * ((size_t)count + 1)))) return rc;
  if ((rc = dalloc(h, &v.wtab, (size_t)count * 2 * KMAX))) return rc;
  if ((rc = dalloc(h, &v.sched, 1))) return rc;
  h->trace_cap = (int)h->P("trace_capacity");
  if ((rc = dalloc(h, (dpdlp_trace_t**)&v.trace, h->trace_cap > 0 ? h->trace_cap : 1))) return rc;
  if ((rc = dalloc(h, &h->d_sc, 1))) return rc;
  const bool pre = !h->dr.empty();
  std::vector<double> cs_int;  // the cost vector the solver iterates with (internal order)
  if (n) {
    std::vector<double> tmp = permuted(c, h->pcol);
    if (pre)
      for (int j = 0; j < n; ++j) tmp[j] *= h->dc[j];
    cs_int = tmp;
    CK(cudaMemcpy(v.c, tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    tmp = permuted(lv, h->pcol);
    if (pre)
      for (int j = 0; j < n; ++j) tmp[j] /= h->dc[j];
    CK(cudaMemcpy(v.lv, tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    tmp = permuted(uv, h->pcol);
    if (pre)
      for (int j = 0; j < n; ++j) tmp[j] /= h->dc[j];
    CK(cudaMemcpy(v.uv, tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(v.perm_col, h->pcol.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  if (pre) {  // factors and their inverses (exact: powers of two) for the boundary and KKT
    std::vector<double> rw(m), cw(n);
    for (int i = 0; i < m; ++i) rw[i] = 1.0 / h->dr[i];
    for (int j = 0; j < n; ++j) cw[j] = 1.0 / h->dc[j];
    if ((rc = dalloc(h, &h->d_dr, m)) || (rc = dalloc(h, &h->d_dc, n)) ||
        (rc = dalloc(h, &h->d_rw, m)) || (rc = dalloc(h, &h->d_cw, n)))
      return rc;
    if (m) {
      CK(cudaMemcpy(h->d_dr, h->dr.data(), m * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_rw, rw.data(), m * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (n) {
      CK(cudaMemcpy(h->d_dc, h->dc.data(), n * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_cw, cw.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    }
    v.row_w = h->d_rw;
    v.col_w = h->d_cw;
  }
  if (m) CK(cudaMemcpy(v.perm_row, h->prow.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice));
  if ((rc = upload_row_bounds(h))) return rc;
  h->inst_cnorm.assign(count, 0.0);
  h->inst_cnorm_s.assign(count, 0.0);
  for (int i = 0; i < count; ++i) {
    double cs = 0.0, css = 0.0;
    for (int j = col_off[i]; j < col_off[i + 1]; ++j) {
      cs += c[j] * c[j];
      css += cs_int[j] * cs_int[j];  // instance ranges are the same in both orders
    }
    h->inst_cnorm[i] = std::sqrt(cs);
    h->inst_cnorm_s[i] = pre ? std::sqrt(css) : h->inst_cnorm[i];
  }
  h->loaded = true;
  const auto t1 = std::chrono::steady_clock::now();
  dpdlp_info_t& I = h->info;
  I.n = n;
  I.m = m;
  I.nnz = h->nnz;
  I.nnz_padded_csr = Hr.stored;
  I.nnz_padded_csc = Hc.stored;
  I.tiles_csr = Hr.nslots;
  I.tiles_csc = Hc.nslots;
  I.long_rows = Hr.nlong;
  I.long_cols = Hc.nlong;
  I.device_bytes = h->dev_bytes;
  I.preprocess_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  return 0;
}

}  // namespace

extern "C" {

int dpdlp_load_lp(dpdlp_t* h, int32_t n, int32_t m, const double* c, const int64_t* row_ptr,
                  const int32_t* col_idx, const double* val, const double* b, const double* lv,
                  const double* uv, const int8_t* ctype) {
  if (!h) return DPDLP_ERR_INVALID;
  const int32_t ro[2] = {0, m < 0 ? 0 : m}, co[2] = {0, n < 0 ? 0 : n};
  return load_impl(h, 1, ro, co, n, m, c, row_ptr, col_idx, val, b, lv, uv, ctype);
}

int dpdlp_load_batch(dpdlp_t* h, int32_t count, const int32_t* row_off, const int32_t* col_off,
                     int32_t n, int32_t m, const double* c, const int64_t* row_ptr,
                     const int32_t* col_idx, const double* val, const double* b,
                     const double* lv, const double* uv, const int8_t* ctype) {
  if (!h) return DPDLP_ERR_INVALID;
  return load_impl(h, count, row_off, col_off, n, m, c, row_ptr, col_idx, val, b, lv, uv, ctype);
}

int dpdlp_set_objective_diag(dpdlp_t* h, const double* q) {
  if (!h) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  if (q)
    for (int j = 0; j < h->n; ++j)
      if (!(q[j] >= 0.0) || !std::isfinite(q[j]))
        return fail(h, DPDLP_ERR_INVALID, "Q diagonal must be finite and >= 0 at " + std::to_string(j));
  CK(cudaStreamSynchronize(h->stream));
  free_graph(h);  // the captured kernels follow the LP / QP choice
  h->has_state = false;
  h->pending_state = false;
  if (!q) {
    h->v.q = nullptr;
    return 0;
  }
  if (!h->d_q) {
    int rc;
    if ((rc = dalloc(h, &h->d_q, h->n))) return rc;
  }
  std::vector<double> qi(h->n);  // internal order; the scaled LP's Q is D_c Q D_c
  for (int j = 0; j < h->n; ++j)
    qi[j] = q[h->pcol[j]] * (h->dc.empty() ? 1.0 : h->dc[j] * h->dc[j]);
  if (h->n) CK(cudaMemcpy(h->d_q, qi.data(), h->n * sizeof(double), cudaMemcpyHostToDevice));
  h->v.q = h->d_q;
  return 0;
}

int dpdlp_set_row_bounds(dpdlp_t* h, const double* lc, const double* uc) {
  if (!h || !lc || !uc) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  for (int i = 0; i < h->m; ++i)
    if (std::isnan(lc[i]) || std::isnan(uc[i]) || lc[i] > uc[i] || lc[i] == INFINITY ||
        uc[i] == -INFINITY)
      return fail(h, DPDLP_ERR_INVALID, "invalid row bounds at " + std::to_string(i));
  CK(cudaStreamSynchronize(h->stream));
  h->h_lc.assign(lc, lc + h->m);
  h->h_uc.assign(uc, uc + h->m);
  h->has_state = false;
  h->pending_state = false;
  return upload_row_bounds(h);
}

int dpdlp_set_start(dpdlp_t* h, const double* x0, const double* y0) {
  if (!h) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  int rc;
  h->have_start_x = x0 != nullptr;
  h->have_start_y = y0 != nullptr;
  if (x0 && (rc = import_vec(h, x0, h->xs, h->v.perm_col, h->n, h->v.tmp_n, h->d_cw))) return rc;
  if (y0 && (rc = import_vec(h, y0, h->ys, h->v.perm_row, h->m, h->v.tmp_m, h->d_rw))) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

int dpdlp_solve(dpdlp_t* h, double tol, int64_t max_iter) {
  if (!h) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  if (!(tol >= 0.0) || max_iter < 0) return fail(h, DPDLP_ERR_INVALID, "tol must be >= 0, max_iter >= 0");
  CK(cudaSetDevice(h->device));
  int rc;
  const bool resume = (h->P("resume") != 0.0 && h->has_state) || h->pending_state;
  if (!resume && (rc = init_fresh(h))) return rc;
  DevScalars& s = h->h_sc;
  copy_params(h, s);
  s.eps = tol;
  s.max_iter = max_iter;
  h->pending_state = false;
  for (InstScalars& I : h->h_inst) I.status = -1;  // a solve continues every instance
  if (s.T_base >= max_iter) {
    s.status = 1;
    for (InstScalars& I : h->h_inst) I.status = 1;
    s.running = 0;
    CK(cudaMemcpyAsync(h->d_sc, &s, sizeof(DevScalars), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->v.inst, h->h_inst.data(), h->ninst * sizeof(InstScalars),
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return 1;
  }
  s.status = -1;
  s.running = h->ninst;
  s.T_check = s.T_base + s.K < max_iter ? s.T_base + s.K : max_iter;
  if ((rc = upload_weights(h))) return rc;
  CK(cudaMemcpyAsync(h->d_sc, &s, sizeof(DevScalars), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->v.inst, h->h_inst.data(), h->ninst * sizeof(InstScalars),
                     cudaMemcpyHostToDevice, h->stream));
  CK(launch_compact(h->csr, h->csc, h->v, h->stream));  // a batch: every instance is running
  if (h->P("use_graph") != 0.0) {
    if (h->graph_K != s.K || !h->exec) {
      CK(cudaStreamSynchronize(h->stream));
      if ((rc = build_graph(h, s.K))) return rc;
    }
    CK(cudaGraphLaunch(h->exec, h->stream));
  } else {
    if ((rc = run_host_loop(h))) return rc;
  }
  CK(cudaMemcpyAsync(&s, h->d_sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_inst.data(), h->v.inst, h->ninst * sizeof(InstScalars),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return s.status;
}

int dpdlp_get_solution(dpdlp_t* h, double* x, double* y) {
  if (!h) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  int rc;
  if ((rc = export_vec(h, h->v.xh, x, h->v.perm_col, h->n, h->v.tmp_n, h->d_dc))) return rc;
  if ((rc = export_vec(h, h->v.yh, y, h->v.perm_row, h->m, h->v.tmp_m, h->d_dr))) return rc;
  return 0;
}

}  // extern "C"

namespace {

void inst_kkt(const dpdlp* h, int i, dpdlp_kkt_t* o) {
  const DevScalars& s = h->h_sc;
  const InstScalars& I = h->h_inst[i];
  o->r_primal = I.r_p;
  o->r_dual = I.r_d;
  o->r_gap = I.r_g;
  o->obj_p = I.obj_p;
  o->obj_d = I.obj_d;
  o->r_fp = I.r_fp;
  o->omega = I.omega;
  o->eta = I.eta;
  o->tau = I.tau;
  o->sigma = I.sigma;
  o->iterations = h->ninst == 1 ? s.T_base : I.iterations;
  o->restarts = I.restarts;
  o->checks = s.checks;
  o->status = I.status;
  o->spmv_mode = I.spmv_fp32;
}

}  // namespace

extern "C" {

int dpdlp_get_kkt(dpdlp_t* h, dpdlp_kkt_t* o) {
  if (!h || !o) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  std::memset(o, 0, sizeof(*o));
  o->status = -1;
  if (!h->has_state) return 0;
  inst_kkt(h, 0, o);
  if (h->ninst > 1) {  // batch: worst residuals, summed objectives and restarts
    for (int i = 1; i < h->ninst; ++i) {
      dpdlp_kkt_t k;
      inst_kkt(h, i, &k);
      o->r_primal = std::fmax(o->r_primal, k.r_primal);
      o->r_dual = std::fmax(o->r_dual, k.r_dual);
      o->r_gap = std::fmax(o->r_gap, k.r_gap);
      o->r_fp = std::fmax(o->r_fp, k.r_fp);
      o->obj_p += k.obj_p;
      o->obj_d += k.obj_d;
      o->restarts += k.restarts;
      o->spmv_mode = o->spmv_mode > k.spmv_mode ? o->spmv_mode : k.spmv_mode;
    }
    o->iterations = h->h_sc.T_base;
  }
  o->status = h->h_sc.status;
  return 0;
}

int dpdlp_get_batch_kkt(dpdlp_t* h, dpdlp_kkt_t* out, int32_t count) {
  if (!h || !out) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  if (count != h->ninst) return fail(h, DPDLP_ERR_INVALID, "count must equal the number of instances");
  for (int i = 0; i < count; ++i) {
    std::memset(&out[i], 0, sizeof(out[i]));
    out[i].status = -1;
    if (h->has_state) inst_kkt(h, i, &out[i]);
  }
  return 0;
}

int dpdlp_set_batch_eta(dpdlp_t* h, const double* eta, int32_t count) {
  if (!h || (count > 0 && !eta)) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  if (count == 0) {
    h->eta_user.clear();
    return 0;
  }
  if (count != h->ninst) return fail(h, DPDLP_ERR_INVALID, "count must equal the number of instances");
  for (int i = 0; i < count; ++i)
    if (!(eta[i] > 0.0) || !std::isfinite(eta[i])) return fail(h, DPDLP_ERR_INVALID, "eta must be positive and finite");
  h->eta_user.assign(eta, eta + count);
  return 0;
}

int dpdlp_get_trace(dpdlp_t* h, dpdlp_trace_t* out, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  const long long total = h->h_sc.trace_count;
  const long long avail = total < h->trace_cap ? total : h->trace_cap;
  const long long take = avail < cap ? avail : cap;
  std::vector<dpdlp_trace_t> ring(h->trace_cap > 0 ? h->trace_cap : 1);
  if (h->trace_cap > 0) {
    CK(cudaMemcpyAsync(ring.data(), h->v.trace, h->trace_cap * sizeof(dpdlp_trace_t),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  const long long first = total - avail;  // oldest record kept
  for (long long r = 0; r < take; ++r) out[r] = ring[(first + r) % h->trace_cap];
  *count = (int32_t)take;
  return 0;
}

int dpdlp_get_state(dpdlp_t* h, double* x, double* y, double* x0, double* y0,
                    dpdlp_scalar_state_t* st) {
  if (!h) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  if (!h->has_state) return fail(h, DPDLP_ERR_INVALID, "no solver state yet");
  if (h->ninst != 1) return fail(h, DPDLP_ERR_INVALID, "checkpoints hold a single LP, not a batch");
  CK(cudaSetDevice(h->device));
  int rc;
  if ((rc = export_vec(h, h->v.x, x, h->v.perm_col, h->n, h->v.tmp_n, h->d_dc))) return rc;
  if ((rc = export_vec(h, h->v.y, y, h->v.perm_row, h->m, h->v.tmp_m, h->d_dr))) return rc;
  if ((rc = export_vec(h, h->v.x0, x0, h->v.perm_col, h->n, h->v.tmp_n, h->d_dc))) return rc;
  if ((rc = export_vec(h, h->v.y0, y0, h->v.perm_row, h->m, h->v.tmp_m, h->d_dr))) return rc;
  if (st) {
    const InstScalars& s = h->h_inst[0];
    st->T = h->h_sc.T_base;
    st->k = s.k_base;
    st->restarts = s.restarts;
    st->checks = h->h_sc.checks;
    st->eta = s.eta;
    st->omega = s.omega;
    st->r_anchor = s.r_anchor;
    st->r_prev = s.r_prev;
    st->e_sum = s.e_sum;
    st->e_prev = s.e_prev;
    st->has_anchor = s.has_anchor;
    st->has_e_prev = s.has_e_prev;
    st->spmv_mode = s.spmv_fp32;
    st->stall_checks = s.stall_checks;
    st->best_kkt = s.best_kkt;
  }
  return 0;
}

int dpdlp_set_state(dpdlp_t* h, const double* x, const double* y, const double* x0,
                    const double* y0, const dpdlp_scalar_state_t* st) {
  if (!h || !st || (h->n && (!x || !x0)) || (h->m && (!y || !y0))) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  if (!(st->eta > 0.0) || !(st->omega > 0.0) || st->T < 0 || st->k < 0)
    return fail(h, DPDLP_ERR_INVALID, "invalid scalar state");
  if (h->ninst != 1) return fail(h, DPDLP_ERR_INVALID, "checkpoints hold a single LP, not a batch");
  CK(cudaSetDevice(h->device));
  int rc;
  if ((rc = import_vec(h, x, h->v.x, h->v.perm_col, h->n, h->v.tmp_n, h->d_cw))) return rc;
  if ((rc = import_vec(h, y, h->v.y, h->v.perm_row, h->m, h->v.tmp_m, h->d_rw))) return rc;
  if ((rc = import_vec(h, x0, h->v.x0, h->v.perm_col, h->n, h->v.tmp_n, h->d_cw))) return rc;
  if ((rc = import_vec(h, y0, h->v.y0, h->v.perm_row, h->m, h->v.tmp_m, h->d_rw))) return rc;
  if (h->n) CK(cudaMemcpyAsync(h->v.xh, h->v.x, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h->m) CK(cudaMemcpyAsync(h->v.yh, h->v.y, h->m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  DevScalars& g = h->h_sc;
  const int sched = g.sched_len;
  std::memset(&g, 0, sizeof(g));
  g.sched_len = sched;
  g.T_base = st->T;
  g.checks = st->checks;
  g.status = -1;
  h->h_inst.resize(1);
  InstScalars& s = h->h_inst[0];
  s = fresh_inst(h, 0, st->eta, st->omega,
                 (st->spmv_mode && h->csr.val32 && h->csc.val32) ? 1 : 0);
  s.k_base = st->k;
  s.restarts = st->restarts;
  s.r_anchor = st->r_anchor;
  s.r_prev = st->r_prev;
  s.e_sum = st->e_sum;
  s.e_prev = st->e_prev;
  s.has_anchor = st->has_anchor;
  s.has_e_prev = st->has_e_prev;
  s.stall_checks = st->stall_checks;
  s.best_kkt = st->best_kkt;
  s.iterations = st->T;
  h->has_state = true;
  h->pending_state = true;
  return 0;
}

int dpdlp_set_schedule(dpdlp_t* h, const int8_t* kinds, int32_t count) {
  if (!h || count < 0 || (count > 0 && !kinds)) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  if (count % h->ninst != 0)
    return fail(h, DPDLP_ERR_INVALID, "schedule length must be a multiple of the instance count");
  for (int i = 0; i < count; ++i)
    if (kinds[i] < 0 || kinds[i] > 3) return fail(h, DPDLP_ERR_INVALID, "restart kind must be 0..3");
  CK(cudaStreamSynchronize(h->stream));
  // a new schedule buffer replaces the old one; the captured graph holds the old pointer
  // (through DevVecs), so it is rebuilt
  free_graph(h);
  int rc;
  int8_t* fresh = nullptr;
  if ((rc = dalloc(h, &fresh, count > 0 ? count : 1))) return rc;
  if (count > 0) CK(cudaMemcpy(fresh, kinds, count, cudaMemcpyHostToDevice));
  dfree(h, h->v.sched);
  h->v.sched = fresh;
  h->h_sc.sched_len = count / h->ninst;  // per instance: kinds[i * len + check]
  return 0;
}

int dpdlp_apply_A(dpdlp_t* h, const double* x, double* out) {
  if (!h || (h->n && !x) || (h->m && !out)) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  int rc;
  if ((rc = import_vec(h, x, h->v.tmp_n2, h->v.perm_col, h->n, h->v.tmp_n, h->d_cw))) return rc;
  CK(launch_spmv(h->csr, h->v.tmp_n2, nullptr, h->v.axh, nullptr, h->stream, nullptr));
  return export_vec(h, h->v.axh, out, h->v.perm_row, h->m, h->v.tmp_m, h->d_rw);
}

int dpdlp_apply_AT(dpdlp_t* h, const double* y, double* out) {
  if (!h || (h->m && !y) || (h->n && !out)) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  CK(cudaSetDevice(h->device));
  int rc;
  if ((rc = import_vec(h, y, h->v.axh, h->v.perm_row, h->m, h->v.tmp_m, h->d_rw))) return rc;
  CK(launch_spmv(h->csc, h->v.axh, nullptr, h->v.tmp_n2, nullptr, h->stream, nullptr));
  return export_vec(h, h->v.tmp_n2, out, h->v.perm_col, h->n, h->v.tmp_n, h->d_cw);
}

int dpdlp_time_kernel(dpdlp_t* h, const char* which, int32_t reps, double* avg_ms) {
  if (!h || !which || reps <= 0 || !avg_ms) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  const std::string w(which);
  // the iteration kernels (*_slots: without the long-row pass), or an access probe of one
  // orientation's product (its loads without arithmetic): gather_* indices + gathers,
  // access_* plus values, stream_* the index and value streams only, memory_* access_* plus
  // the epilogue's row vectors
  int probe = -1;
  bool primal = w == "primal";
  // batches also time the iteration kernels as the solve may run them: walking the
  // active-slot lists (*_list), and with every instance stopped (*_idle, *_list_idle)
  // launched as the solve launches them (programmatic dependents when pdl is on)
  IterPlan p{0, 1, 0, (int)h->P("pdl"), 0};
  const std::string side0 = w.substr(0, w.find('_'));
  const std::string rest = w.find('_') == std::string::npos ? "" : w.substr(w.find('_') + 1);
  if ((side0 == "primal" || side0 == "dual") && rest == "slots") {
    primal = side0 == "primal";
    p.slots_only = 1;
  } else if ((side0 == "primal" || side0 == "dual") &&
             (rest == "list" || rest == "idle" || rest == "list_idle")) {
    if (h->ninst < 2) return fail(h, DPDLP_ERR_INVALID, "list and idle timings need a batch");
    primal = side0 == "primal";
    p.list = rest != "idle";
    p.idle = rest != "list";
  } else if (w != "primal" && w != "dual") {
    const size_t us = w.find('_');
    const std::string kind = us == std::string::npos ? w : w.substr(0, us);
    const std::string side = us == std::string::npos ? "" : w.substr(us + 1);
    probe = kind == "gather" ? 0 : kind == "access" ? 1 : kind == "stream" ? 2
          : kind == "memory" ? 3 : -1;
    if (probe < 0 || (side != "primal" && side != "dual"))
      return fail(h, DPDLP_ERR_INVALID,
                  "kernel must be primal, dual, primal_slots, dual_slots, or "
                  "gather_/access_/stream_/memory_ + primal or dual");
    primal = side == "primal";
  }
  if (!h->has_state) return fail(h, DPDLP_ERR_INVALID, "solve or set a start first");
  CK(cudaSetDevice(h->device));
  // keep the state: snapshot the vectors the kernels update in place
  if (h->n) CK(cudaMemcpyAsync(h->v.tmp_n, h->v.x, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h->m) CK(cudaMemcpyAsync(h->v.tmp_m, h->v.y, h->m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h->n) CK(cudaMemcpyAsync(h->v.tmp_n2, h->v.xbar, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->stream));
  for (int r = 0; r < reps; ++r) {
    if (probe >= 0) {
      // the primal product gathers y over the rows of A^T, the dual one x_bar over A
      CK(launch_access_probe(primal ? h->csc : h->csr, primal ? h->v.y : h->v.xbar, probe,
                             h->v, primal, p.pdl != 0,
                             reinterpret_cast<unsigned long long*>(h->v.pw), h->stream));
    } else if (primal) {
      CK(launch_primal(h->csc, h->v, h->d_sc, p, h->stream));
    } else {
      CK(launch_dual(h->csr, h->v, h->d_sc, p, h->stream));
    }
  }
  CK(cudaEventRecord(e1, h->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *avg_ms = (double)ms / reps;
  if (h->n) CK(cudaMemcpyAsync(h->v.x, h->v.tmp_n, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h->m) CK(cudaMemcpyAsync(h->v.y, h->v.tmp_m, h->m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (h->n) CK(cudaMemcpyAsync(h->v.xbar, h->v.tmp_n2, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

int dpdlp_get_info(dpdlp_t* h, dpdlp_info_t* out) {
  if (!h || !out) return DPDLP_ERR_INVALID;
  if (!h->loaded) return fail(h, DPDLP_ERR_NOT_LOADED, "no LP loaded");
  *out = h->info;
  out->device_bytes = h->dev_bytes;
  out->fused_body = use_fused(h) ? 1 : 0;
  out->reserved = 0;
  return 0;
}

}  // extern "C"

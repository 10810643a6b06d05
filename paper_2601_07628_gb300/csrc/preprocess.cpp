// Host preprocessing of an LP before it goes to the device (runs once per load).
//
//  * CSR validation.
//  * Block-wise random permutation of rows and columns (Section 4.2): contiguous blocks of
//    B indices (B = 256 by default) are shuffled, the order inside a block is kept.
//  * The CSC copy of A (the paper keeps both CSR and CSC in device memory so that A^T y
//    needs no atomics, Appendix E.2), built as the CSR of A^T by a stable counting sort.
//  * Optional diagonal preconditioning (Ruiz, Pock-Chambolle) with power-of-two factors.
//  * (packing.cpp) nonzero-aware partitioning (Section 4.3) down to warp lanes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "host_parallel.h"
#include "internal.h"

namespace pdhg {

std::string validate_csr(int rows, int cols, const int64_t* ptr, const int32_t* idx,
                         const double* val) {
  if (rows < 0 || cols < 0) return "negative dimension";
  if (!ptr) return "row_ptr is NULL";
  if (ptr[0] != 0) return "row_ptr[0] != 0";
  for (int r = 0; r < rows; ++r)
    if (ptr[r + 1] < ptr[r]) return "row_ptr not non-decreasing at row " + std::to_string(r);
  const int64_t nnz = ptr[rows];
  if (nnz > (int64_t)INT32_MAX / 2) return "too many nonzeros for 32-bit offsets";
  if (cols > (int)IDX_MASK) return "too many columns for the packed index format";
  if (nnz > 0 && (!idx || !val)) return "col_idx or val is NULL";
  for (int64_t e = 0; e < nnz; ++e) {
    if (idx[e] < 0 || idx[e] >= cols)
      return "column index out of range at entry " + std::to_string(e);
    if (!std::isfinite(val[e])) return "non-finite matrix value at entry " + std::to_string(e);
  }
  return "";
}

static inline uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

std::vector<int32_t> block_permutation(int len, int block, uint64_t seed, bool enabled) {
  std::vector<int32_t> p(len);
  std::iota(p.begin(), p.end(), 0);
  if (!enabled || block <= 0 || len <= block) return p;
  const int nfull = len / block;
  std::vector<int32_t> order(nfull);
  std::iota(order.begin(), order.end(), 0);
  uint64_t s = seed;
  for (int i = nfull - 1; i > 0; --i) {  // Fisher-Yates over whole blocks
    const int j = (int)(splitmix64(s) % (uint64_t)(i + 1));
    std::swap(order[i], order[j]);
  }
  for (int b = 0; b < nfull; ++b)
    for (int t = 0; t < block; ++t) p[(size_t)b * block + t] = order[b] * block + t;
  return p;  // the trailing partial block keeps its place
}

void permute_csr(int rows, int cols, const int64_t* ptr, const int32_t* idx, const double* val,
                 const std::vector<int32_t>& prow, const std::vector<int32_t>& pcol,
                 std::vector<int64_t>& optr, std::vector<int32_t>& oidx,
                 std::vector<double>& oval) {
  std::vector<int32_t> inv_col(cols);
  for (int j = 0; j < cols; ++j) inv_col[pcol[j]] = j;
  optr.assign(rows + 1, 0);
  for (int r = 0; r < rows; ++r) optr[r + 1] = optr[r] + (ptr[prow[r] + 1] - ptr[prow[r]]);
  const int64_t nnz = optr[rows];
  oidx.resize(nnz);
  oval.resize(nnz);
  // rows are independent: threads take ranges of new rows of about equal nonzeros
  run_parts(balanced_rows(rows, optr.data(), host_threads()), [&](int, int64_t r0, int64_t r1) {
    std::vector<std::pair<int32_t, double>> buf;
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t s = ptr[prow[r]], e = ptr[prow[r] + 1];
      buf.resize(e - s);
      bool sorted = true;
      for (int64_t k = s; k < e; ++k) {
        buf[k - s] = {inv_col[idx[k]], val[k]};
        if (k > s && buf[k - s].first < buf[k - s - 1].first) sorted = false;
      }
      if (!sorted)
        std::stable_sort(buf.begin(), buf.end(),
                         [](const std::pair<int32_t, double>& a,
                            const std::pair<int32_t, double>& b) { return a.first < b.first; });
      for (size_t k = 0; k < buf.size(); ++k) {
        oidx[optr[r] + k] = buf[k].first;
        oval[optr[r] + k] = buf[k].second;
      }
    }
  });
}

// Stable counting sort of the entries of a CSR matrix by column: tptr (cols + 1) gets the
// column offsets and emit(p, r, e) is called once per entry e (of row r) with its place p
// in column order, entries of a column in row order.  In parallel: each thread counts the
// columns of its own range of rows, a thread's entries of column j go after those of the
// earlier threads' rows, and each thread then places its rows in order -- the sequential
// placement exactly.
template <class Emit>
static void column_sort(int rows, int cols, const int64_t* ptr, const int32_t* idx,
                        std::vector<int64_t>& tptr, Emit&& emit) {
  const int64_t nnz = ptr[rows];
  tptr.assign(cols + 1, 0);
  // per-thread column counts cost threads x cols x 4 bytes: at most one thread per cols
  // nonzeros, and at most 512 MB of counts
  int T = (int)std::min<int64_t>(host_threads(), nnz / std::max(cols, 1));
  T = (int)std::min<int64_t>(T, ((int64_t)1 << 27) / std::max(cols, 1));
  if (nnz >= INT32_MAX) T = 1;  // the parallel form keeps positions in 32 bits
  if (T <= 1) {
    for (int64_t e = 0; e < nnz; ++e) tptr[idx[e] + 1]++;
    for (int j = 0; j < cols; ++j) tptr[j + 1] += tptr[j];
    std::vector<int64_t> pos(tptr.begin(), tptr.end() - 1);
    for (int r = 0; r < rows; ++r)
      for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) emit(pos[idx[e]]++, r, e);
    return;
  }
  const std::vector<int64_t> rb = balanced_rows(rows, ptr, T);
  T = (int)rb.size() - 1;
  std::vector<std::vector<int32_t>> cnt(T);
  run_parts(rb, [&](int t, int64_t r0, int64_t r1) {
    std::vector<int32_t>& c = cnt[t];
    c.assign(cols, 0);
    for (int64_t e = ptr[r0]; e < ptr[r1]; ++e) c[idx[e]]++;
  });
  for (int j = 0; j < cols; ++j) {
    int64_t a = 0;
    for (int t = 0; t < T; ++t) a += cnt[t][j];
    tptr[j + 1] = tptr[j] + a;
  }
  // counts -> first position of each thread's entries in each column
  run_parts(even_parts(cols, T), [&](int, int64_t j0, int64_t j1) {
    for (int64_t j = j0; j < j1; ++j) {
      int64_t p = tptr[j];
      for (int t = 0; t < T; ++t) {
        const int32_t c = cnt[t][j];
        cnt[t][j] = (int32_t)p;
        p += c;
      }
    }
  });
  run_parts(rb, [&](int t, int64_t r0, int64_t r1) {
    std::vector<int32_t>& pos = cnt[t];
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) emit((int64_t)pos[idx[e]]++, (int)r, e);
  });
}

void transpose_csr(int rows, int cols, const std::vector<int64_t>& ptr,
                   const std::vector<int32_t>& idx, const std::vector<double>& val,
                   std::vector<int64_t>& tptr, std::vector<int32_t>& tidx,
                   std::vector<double>& tval) {
  const int64_t nnz = ptr[rows];
  tidx.resize(nnz);
  tval.resize(nnz);
  column_sort(rows, cols, ptr.data(), idx.data(), tptr, [&](int64_t p, int r, int64_t e) {
    tidx[p] = r;
    tval[p] = val[e];
  });
}

// 2^k with k the integer nearest to log2(v) (v > 0 finite): v = f 2^e with 0.5 <= f < 1,
// and log2(v) rounds up to e exactly when f >= 2^-1/2.
static double pow2_nearest(double v) {
  int e = 0;
  const double f = std::frexp(v, &e);
  return std::ldexp(1.0, f >= std::sqrt(0.5) ? e : e - 1);
}

void precondition(int rows, int cols, const std::vector<int64_t>& ptr,
                  const std::vector<int32_t>& idx, std::vector<double>& val, int ruiz_passes,
                  bool pock_chambolle, std::vector<double>& dr, std::vector<double>& dc) {
  dr.assign(rows, 1.0);
  dc.assign(cols, 1.0);
  std::vector<double> rn(rows), cn(cols);
  // column lists of entry positions (entries of a column in row order), so that column
  // norms can be taken per column, on threads, in the order a row-by-row pass adds them
  std::vector<int64_t> cptr;
  std::vector<int64_t> cpos(ptr[rows]);
  column_sort(rows, cols, ptr.data(), idx.data(), cptr,
              [&](int64_t p, int, int64_t e) { cpos[p] = e; });
  const int T = host_threads();
  const std::vector<int64_t> rparts = balanced_rows(rows, ptr.data(), T);
  const std::vector<int64_t> cparts = balanced_rows(cols, cptr.data(), T);
  // row and column norms of |A|: the maximum (Ruiz) or the sum (Pock-Chambolle)
  auto norms = [&](bool sum) {
    run_parts(rparts, [&](int, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        double a = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
          a = sum ? a + std::fabs(val[k]) : std::max(a, std::fabs(val[k]));
        rn[i] = a;
      }
    });
    run_parts(cparts, [&](int, int64_t j0, int64_t j1) {
      for (int64_t j = j0; j < j1; ++j) {
        double a = 0.0;
        for (int64_t q = cptr[j]; q < cptr[j + 1]; ++q)
          a = sum ? a + std::fabs(val[cpos[q]]) : std::max(a, std::fabs(val[cpos[q]]));
        cn[j] = a;
      }
    });
  };
  auto apply = [&]() {  // factors from the norms rn, cn; scale the values and accumulate
    run_parts(even_parts(cols, T), [&](int, int64_t j0, int64_t j1) {
      for (int64_t j = j0; j < j1; ++j) {
        cn[j] = cn[j] > 0.0 ? pow2_nearest(1.0 / std::sqrt(cn[j])) : 1.0;
        dc[j] *= cn[j];
      }
    });
    run_parts(rparts, [&](int, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        rn[i] = rn[i] > 0.0 ? pow2_nearest(1.0 / std::sqrt(rn[i])) : 1.0;
        dr[i] *= rn[i];
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) val[k] = val[k] * rn[i] * cn[idx[k]];
      }
    });
  };
  for (int pass = 0; pass < ruiz_passes; ++pass) {
    norms(false);
    apply();
  }
  if (pock_chambolle) {
    norms(true);
    apply();
  }
}

}  // namespace pdhg

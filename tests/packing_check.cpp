// Host check of the lane packing (no GPU): reads a CSR matrix and a vector x from a binary
// file, packs the rows, replays what the warp lanes and the long-row pass compute from the
// stored arrays, and compares with a plain CSR product.  Also checks the structural
// invariants of the layout, the (threaded) transpose and row / column permutation against
// plain sequential definitions, and prints a hash of every output so that runs with
// different host thread counts (DPDLP_HOST_THREADS) can be compared.
// Prints "ok <stats> hash=<hex>" or "FAIL <reason>".
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace pdhg;

static int fail(const char* what, long a = 0, long b = 0) {
  std::printf("FAIL %s %ld %ld\n", what, a, b);
  return 1;
}

int main(int argc, char** argv) {
  if (argc == 5 && std::strcmp(argv[1], "--perm") == 0) {  // the block permutation alone
    const std::vector<int32_t> p =
        block_permutation(std::atoi(argv[2]), std::atoi(argv[3]), std::strtoull(argv[4], nullptr, 10), true);
    for (size_t i = 0; i < p.size(); ++i) std::printf("%d%c", p[i], i + 1 < p.size() ? ',' : '\n');
    if (p.empty()) std::printf("\n");
    return 0;
  }
  if (argc < 2) return fail("usage");
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return fail("open");
  int64_t hdr[3];
  if (std::fread(hdr, 8, 3, f) != 3) return fail("header");
  const int rows = (int)hdr[0], cols = (int)hdr[1];
  const int64_t nnz = hdr[2];
  std::vector<int64_t> ptr(rows + 1);
  std::vector<int32_t> idx(nnz);
  std::vector<double> val(nnz), x(cols);
  if (std::fread(ptr.data(), 8, rows + 1, f) != (size_t)rows + 1) return fail("ptr");
  if (nnz && std::fread(idx.data(), 4, nnz, f) != (size_t)nnz) return fail("idx");
  if (nnz && std::fread(val.data(), 8, nnz, f) != (size_t)nnz) return fail("val");
  if (cols && std::fread(x.data(), 8, cols, f) != (size_t)cols) return fail("x");
  std::fclose(f);

  auto parse_offsets = [](const char* q) {
    std::vector<int32_t> o;
    while (*q) {
      o.push_back((int32_t)std::strtol(q, (char**)&q, 10));
      if (*q == ',') ++q;
    }
    return o;
  };
  // optional argv[2]: instance row offsets (comma separated, first 0, last rows) -> batch
  std::vector<int32_t> offsets;
  if (argc > 2) {
    offsets = parse_offsets(argv[2]);
    if (offsets.size() < 2 || offsets.front() != 0 || offsets.back() != rows) return fail("offsets");
  }
  // optional argv[3] (a batch): the instances' column offsets; padding and empty rows then
  // gather their own instance's first column, as the solver packs a batch
  std::vector<int32_t> col_offsets;
  if (argc > 3) {
    col_offsets = parse_offsets(argv[3]);
    if (col_offsets.size() != offsets.size() || col_offsets.front() != 0 || col_offsets.back() != cols)
      return fail("column offsets");
  }
  PackPlan P;
  if (offsets.empty()) plan_packing(rows, ptr, P);
  else plan_packing_batch(rows, ptr, offsets, P);
  std::vector<int32_t> ident(cols);
  for (int j = 0; j < cols; ++j) ident[j] = j;
  HostPacked H;
  build_packed(rows, cols, ptr, idx, val, P, ident, H);
  if (!col_offsets.empty()) own_instance_zero_gathers(H, col_offsets);

  // permutation
  std::vector<int> seen(rows, 0);
  for (int r = 0; r < rows; ++r) {
    const int nr = P.new_of_old[r];
    if (nr < 0 || nr >= rows || seen[nr]++) return fail("new_of_old not a permutation", r, nr);
    if (P.old_of_new[nr] != r) return fail("old_of_new", r, nr);
  }
  // slots (in increasing row order, within the row budget) and long rows cover every row
  // exactly once; for one LP the slots come first and are consecutive
  std::vector<int> cover(rows, 0);
  int expect = 0;
  for (int s = 0; s < H.nslots; ++s) {
    const SlotDesc d = H.slots[s];
    if (d.row_base < expect || (offsets.empty() && d.row_base != expect))
      return fail("slot row_base", s, d.row_base);
    if (d.nrows > MAX_SLOT_ROWS) return fail("slot rows", s, d.nrows);
    for (int r = d.row_base; r < d.row_base + d.nrows; ++r) {
      if (r >= rows) return fail("slot past the rows", s, r);
      ++cover[r];
    }
    expect = d.row_base + d.nrows;
  }
  for (int i = 0; i < H.nlong; ++i) ++cover[H.long_row[i]];
  for (int r = 0; r < rows; ++r)
    if (cover[r] != 1) return fail("row not covered exactly once", r, cover[r]);
  if (H.nshort + H.nlong != rows) return fail("row counts", H.nshort, H.nlong);
  if (offsets.empty()) {
    for (int r = 0; r < rows; ++r) {
      const int64_t L = ptr[r + 1] - ptr[r];
      const bool is_long = L > LANE_ITEMS;
      if (is_long != (P.new_of_old[r] >= H.nshort)) return fail("long/short class", r, L);
    }
  } else {
    // a batch: rows keep their instance's range, slots and long rows know their instance
    auto inst_of = [&](int r) {
      int i = 0;
      while (offsets[i + 1] <= r) ++i;
      return i;
    };
    for (int r = 0; r < rows; ++r)
      if (inst_of(P.new_of_old[r]) != inst_of(r)) return fail("row left its instance", r, 0);
    for (int s = 0; s < H.nslots; ++s) {
      const SlotDesc d = H.slots[s];
      if (d.nrows && (inst_of(d.row_base) != d.inst || inst_of(d.row_base + d.nrows - 1) != d.inst))
        return fail("slot instance", s, d.inst);
    }
    for (int i = 0; i < H.nlong; ++i)
      if (inst_of(H.long_row[i]) != H.long_inst[i]) return fail("long row instance", i, 0);
    for (int i = 1; i < H.nlong; ++i)
      if (H.long_ptr[i + 1] - H.long_ptr[i] > H.long_ptr[i] - H.long_ptr[i - 1])
        return fail("long rows not longest first", i, 0);
    // every stored entry of an instance's slots, padding and empty rows included, gathers
    // a column of that instance (index 0 for an instance without columns)
    for (int s = 0; s < H.nslots && !col_offsets.empty(); ++s) {
      const int i = H.slots[s].inst;
      const bool own = col_offsets[i + 1] > col_offsets[i];
      for (int k = 0; k < SLOT_ITEMS; ++k) {
        const int c = (int)(H.idx[(size_t)s * SLOT_ITEMS + k] & IDX_MASK);
        if (own ? (c < col_offsets[i] || c >= col_offsets[i + 1]) : c != 0)
          return fail("gather outside its instance", s, c);
      }
    }
  }
  // replay the lanes
  std::vector<double> out(rows, NAN), piece(H.npieces, NAN);
  int64_t stored_flags = 0, stored_nonpad = 0;
  for (int s = 0; s < H.nslots; ++s) {
    for (int l = 0; l < LANES; ++l) {
      const LaneMeta lm = H.lanes[(size_t)s * LANES + l];
      int rl = lm.row_local, pid = lm.piece_base;
      double acc = 0.0;
      for (int p = 0; p < LANE_ITEMS; ++p) {
        const double v = H.val[(size_t)s * SLOT_ITEMS + ((p >> 1) * LANES + l) * 2 + (p & 1)];
        const uint32_t c = H.idx[(size_t)s * SLOT_ITEMS + ((p >> 2) * LANES + l) * 4 + (p & 3)];
        if ((c & IDX_MASK) >= (uint32_t)(cols > 0 ? cols : 1)) return fail("column range", s, l);
        if (v != 0.0) ++stored_nonpad;
        acc = std::fma(v, cols > 0 ? x[c & IDX_MASK] : 0.0, acc);
        if (c & END_BIT) {
          ++stored_flags;
          if (c & PIECE_BIT) {
            if (pid < 0 || pid >= H.npieces) return fail("piece id", s, pid);
            piece[pid++] = acc;
          } else {
            if (rl >= H.slots[s].nrows) return fail("row_local overflow", s, rl);
            out[H.slots[s].row_base + rl++] = acc;
          }
          acc = 0.0;
        }
      }
    }
  }
  for (int i = 0; i < H.nlong; ++i) {
    double a = 0.0;
    for (int q = H.long_ptr[i]; q < H.long_ptr[i + 1]; ++q) {
      const int pid = H.long_piece[q];
      if (pid < 0 || pid >= H.npieces || std::isnan(piece[pid])) return fail("long row piece", i, q);
      a += piece[pid];
    }
    out[H.long_row[i]] = a;
  }
  // compare with the plain product (rows in the new order)
  double maxrel = 0.0;
  int64_t nz_vals = 0;
  for (int r = 0; r < rows; ++r) {
    double ref = 0.0, mag = 0.0;
    for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) {
      ref = std::fma(val[e], x[idx[e]], ref);
      mag += std::fabs(val[e] * x[idx[e]]);
      if (val[e] != 0.0) ++nz_vals;
    }
    const double got = out[P.new_of_old[r]];
    if (std::isnan(got)) return fail("row not produced", r, 0);
    const double err = std::fabs(got - ref) / (mag > 0 ? mag : 1.0);
    if (err > maxrel) maxrel = err;
  }
  if (maxrel > 1e-13) return fail("product mismatch (1e-15 units)", (long)(maxrel * 1e15), 0);
  if (stored_nonpad != nz_vals) return fail("stored nonzeros", stored_nonpad, nz_vals);
  if (stored_flags != H.nshort + H.npieces) return fail("end flags", stored_flags, H.nshort + H.npieces);

  // transpose: a stable counting sort by column, written out plainly
  std::vector<int64_t> tptr, rptr(cols + 1, 0);
  std::vector<int32_t> tidx, ridx(nnz);
  std::vector<double> tval, rval(nnz);
  transpose_csr(rows, cols, ptr, idx, val, tptr, tidx, tval);
  for (int64_t e = 0; e < nnz; ++e) rptr[idx[e] + 1]++;
  for (int j = 0; j < cols; ++j) rptr[j + 1] += rptr[j];
  {
    std::vector<int64_t> next(rptr.begin(), rptr.end() - 1);
    for (int r = 0; r < rows; ++r)
      for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) {
        ridx[next[idx[e]]] = r;
        rval[next[idx[e]]++] = val[e];
      }
  }
  if (tptr != rptr || tidx != ridx ||
      std::memcmp(tval.data(), rval.data(), nnz * sizeof(double)) != 0)
    return fail("transpose");
  // permutation: new row r is old row prow[r], columns renamed and sorted (stable)
  const std::vector<int32_t> prow = block_permutation(rows, 3, 7, true);
  const std::vector<int32_t> pcol = block_permutation(cols, 5, 8, true);
  std::vector<int64_t> pptr;
  std::vector<int32_t> pidx;
  std::vector<double> pval;
  permute_csr(rows, cols, ptr.data(), idx.data(), val.data(), prow, pcol, pptr, pidx, pval);
  {
    std::vector<int32_t> inv(cols);
    for (int j = 0; j < cols; ++j) inv[pcol[j]] = j;
    int64_t k = 0;
    for (int r = 0; r < rows; ++r) {
      if (pptr[r] != k) return fail("permuted row_ptr", r, 0);
      std::vector<std::pair<int32_t, double>> row;
      for (int64_t e = ptr[prow[r]]; e < ptr[prow[r] + 1]; ++e) row.push_back({inv[idx[e]], val[e]});
      std::stable_sort(row.begin(), row.end(), [](const std::pair<int32_t, double>& a,
                                                  const std::pair<int32_t, double>& b) {
        return a.first < b.first;
      });
      for (const auto& q : row) {
        if (pidx[k] != q.first || std::memcmp(&pval[k], &q.second, sizeof(double)) != 0)
          return fail("permuted entry", r, (long)k);
        ++k;
      }
    }
    if (pptr[rows] != k) return fail("permuted nnz");
  }

  // preconditioning (10 Ruiz passes, then Pock-Chambolle) against the plain row-by-row loops
  std::vector<double> sval(val), dr, dc;
  precondition(rows, cols, ptr, idx, sval, 10, true, dr, dc);
  {
    std::vector<double> v(val), er(rows, 1.0), ec(cols, 1.0), rn(rows), cn(cols);
    auto p2 = [](double x) {  // the power of two nearest to x in log scale
      int e = 0;
      const double f = std::frexp(x, &e);
      return std::ldexp(1.0, f >= std::sqrt(0.5) ? e : e - 1);
    };
    for (int pass = 0; pass < 11; ++pass) {
      const bool sum = pass == 10;
      std::fill(rn.begin(), rn.end(), 0.0);
      std::fill(cn.begin(), cn.end(), 0.0);
      for (int r = 0; r < rows; ++r)
        for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) {
          const double a = std::fabs(v[e]);
          rn[r] = sum ? rn[r] + a : std::max(rn[r], a);
          cn[idx[e]] = sum ? cn[idx[e]] + a : std::max(cn[idx[e]], a);
        }
      for (int r = 0; r < rows; ++r) rn[r] = rn[r] > 0.0 ? p2(1.0 / std::sqrt(rn[r])) : 1.0;
      for (int j = 0; j < cols; ++j) cn[j] = cn[j] > 0.0 ? p2(1.0 / std::sqrt(cn[j])) : 1.0;
      for (int r = 0; r < rows; ++r)
        for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) v[e] = v[e] * rn[r] * cn[idx[e]];
      for (int r = 0; r < rows; ++r) er[r] *= rn[r];
      for (int j = 0; j < cols; ++j) ec[j] *= cn[j];
    }
    if (std::memcmp(v.data(), sval.data(), nnz * sizeof(double)) != 0 || er != dr || ec != dc)
      return fail("preconditioning");
    if (const char* path = std::getenv("PACKING_CHECK_SCALING")) {  // D_r then D_c, float64
      FILE* g = std::fopen(path, "wb");
      if (!g || std::fwrite(dr.data(), 8, dr.size(), g) != dr.size() ||
          std::fwrite(dc.data(), 8, dc.size(), g) != dc.size())
        return fail("scaling dump");
      std::fclose(g);
    }
  }

  unsigned long long h = 1469598103934665603ull;  // FNV-1a over every output
  auto mix = [&](const void* p, size_t b) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < b; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  };
  mix(H.val.data(), H.val.size() * sizeof(double));
  mix(H.val32.data(), H.val32.size() * sizeof(float));
  mix(H.idx.data(), H.idx.size() * sizeof(uint32_t));
  mix(H.slots.data(), H.slots.size() * sizeof(SlotDesc));
  mix(H.lanes.data(), H.lanes.size() * sizeof(LaneMeta));
  mix(H.long_row.data(), H.long_row.size() * sizeof(int32_t));
  mix(H.long_ptr.data(), H.long_ptr.size() * sizeof(int32_t));
  mix(H.long_piece.data(), H.long_piece.size() * sizeof(int32_t));
  mix(P.old_of_new.data(), P.old_of_new.size() * sizeof(int32_t));
  mix(tidx.data(), tidx.size() * sizeof(int32_t));
  mix(tval.data(), tval.size() * sizeof(double));
  mix(pidx.data(), pidx.size() * sizeof(int32_t));
  mix(pval.data(), pval.size() * sizeof(double));
  mix(sval.data(), sval.size() * sizeof(double));
  mix(dr.data(), dr.size() * sizeof(double));
  mix(dc.data(), dc.size() * sizeof(double));
  std::printf("ok slots=%d nshort=%d nlong=%d npieces=%d fill=%.4f maxrel=%.3g exact32=%d hash=%016llx\n",
              H.nslots, H.nshort, H.nlong, H.npieces,
              H.stored ? (double)nnz / (double)H.stored : 1.0, maxrel, (int)H.fp32_exact_range, h);
  return 0;
}

// Host check of the lane packing (no GPU): reads a CSR matrix and a vector x from a binary
// file, packs the rows, replays what the warp lanes and the long-row pass compute from the
// stored arrays, and compares with a plain CSR product.  Also checks the structural
// invariants of the layout.  Prints "ok <stats>" or "FAIL <reason>".
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

  // optional argv[2]: instance row offsets (comma separated, first 0, last rows) -> batch
  std::vector<int32_t> offsets;
  if (argc > 2) {
    const char* q = argv[2];
    while (*q) {
      offsets.push_back((int32_t)std::strtol(q, (char**)&q, 10));
      if (*q == ',') ++q;
    }
    if (offsets.size() < 2 || offsets.front() != 0 || offsets.back() != rows) return fail("offsets");
  }
  PackPlan P;
  if (offsets.empty()) plan_packing(rows, ptr, P);
  else plan_packing_batch(rows, ptr, offsets, P);
  std::vector<int32_t> ident(cols);
  for (int j = 0; j < cols; ++j) ident[j] = j;
  HostPacked H;
  build_packed(rows, cols, ptr, idx, val, P, ident, H);

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
  std::printf("ok slots=%d nshort=%d nlong=%d npieces=%d fill=%.4f maxrel=%.3g\n", H.nslots,
              H.nshort, H.nlong, H.npieces,
              H.stored ? (double)nnz / (double)H.stored : 1.0, maxrel);
  return 0;
}

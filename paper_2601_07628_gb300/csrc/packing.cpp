// Host packing of a sparse orientation into warp lanes (layout described in internal.h).
//
// Rows of at most LANE_ITEMS nonzeros ("short rows", empty rows counting as one stored
// zero) and the tails of longer rows are packed into lanes by best-fit decreasing: segments
// in decreasing length, each into the open lane whose free room fits it most tightly.
// The full LANE_ITEMS-nonzero pieces of long rows fill lanes of their own.  Lanes are then
// grouped 32 to a slot, at most MAX_SLOT_ROWS short rows per slot.  The short rows are
// renumbered in slot / lane / position order, so each slot's rows are consecutive and its
// row vectors are read with coalesced loads; long rows come after all short rows.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <numeric>
#include <utility>

#include "host_parallel.h"
#include "internal.h"

namespace pdhg {

void plan_packing(int rows, const std::vector<int64_t>& ptr, PackPlan& P) {
  P = PackPlan{};
  struct Seg {
    int32_t row, first, count, usage;
    bool piece;
  };
  std::vector<Seg> segs;
  segs.reserve(rows);
  std::vector<int32_t> to_fit;  // short rows and tails of long rows, in row order
  std::vector<int32_t> long_of_row(rows, -1);
  for (int r = 0; r < rows; ++r) {
    const int64_t L = ptr[r + 1] - ptr[r];
    if (L <= LANE_ITEMS) {
      segs.push_back({r, 0, (int32_t)L, (int32_t)std::max<int64_t>(L, 1), false});
      to_fit.push_back((int32_t)segs.size() - 1);
      continue;
    }
    long_of_row[r] = (int32_t)P.long_rows.size();
    P.long_rows.push_back(r);
    const int64_t f = L / LANE_ITEMS, t = L % LANE_ITEMS;
    for (int64_t k = 0; k < f; ++k)
      segs.push_back({r, (int32_t)(k * LANE_ITEMS), LANE_ITEMS, LANE_ITEMS, true});
    if (t > 0) {
      segs.push_back({r, (int32_t)(f * LANE_ITEMS), (int32_t)t, (int32_t)t, true});
      to_fit.push_back((int32_t)segs.size() - 1);
    }
  }
  // long rows ordered by length, longest first (stable), so the long-row pass can give the
  // longest rows a block or a warp each and keep similar rows together
  std::stable_sort(P.long_rows.begin(), P.long_rows.end(), [&](int32_t a, int32_t b) {
    return ptr[a + 1] - ptr[a] > ptr[b + 1] - ptr[b];
  });
  for (size_t i = 0; i < P.long_rows.size(); ++i) long_of_row[P.long_rows[i]] = (int32_t)i;
  // per lane: linked list of segments in insertion order, free room, short-row count
  std::vector<int32_t> head, tail, room, nrows_lane;
  std::vector<int32_t> next(segs.size(), -1);
  auto new_lane = [&]() {
    head.push_back(-1);
    tail.push_back(-1);
    room.push_back(LANE_ITEMS);
    nrows_lane.push_back(0);
    return (int32_t)head.size() - 1;
  };
  std::vector<int32_t> piece_lanes, bfd_lanes;
  for (size_t s = 0; s < segs.size(); ++s) {  // every full piece fills a lane of its own
    if (segs[s].piece && segs[s].count == LANE_ITEMS) {
      const int32_t lane = new_lane();
      head[lane] = tail[lane] = (int32_t)s;
      room[lane] = 0;
      piece_lanes.push_back(lane);
    }
  }
  {  // stable order by decreasing usage (1..LANE_ITEMS): one bucket per usage value
    std::vector<int32_t> start(LANE_ITEMS + 2, 0), sorted(to_fit.size());
    for (int32_t g : to_fit) ++start[LANE_ITEMS + 1 - segs[g].usage];
    for (int u = 1; u <= LANE_ITEMS + 1; ++u) start[u] += start[u - 1];
    for (int32_t g : to_fit) sorted[start[LANE_ITEMS - segs[g].usage]++] = g;
    to_fit.swap(sorted);
  }
  std::vector<std::vector<int32_t>> bucket(LANE_ITEMS);  // open lanes by free room 1..31
  for (int32_t s : to_fit) {
    const int u = segs[s].usage;
    int32_t lane = -1;
    for (int c = u; c < LANE_ITEMS && lane < 0; ++c) {
      if (!bucket[c].empty()) {
        lane = bucket[c].back();
        bucket[c].pop_back();
      }
    }
    if (lane < 0) {
      lane = new_lane();
      bfd_lanes.push_back(lane);
    }
    if (tail[lane] < 0) head[lane] = s; else next[tail[lane]] = s;
    tail[lane] = s;
    room[lane] -= u;
    if (!segs[s].piece) nrows_lane[lane] += 1;
    if (room[lane] > 0) bucket[room[lane]].push_back(lane);
  }
  // slots: best-fit lanes first while the short-row budget allows, piece lanes fill the rest
  size_t bi = 0, pi = 0;
  std::vector<int32_t> slot_lanes;
  while (bi < bfd_lanes.size() || pi < piece_lanes.size()) {
    int nl = 0, nr = 0;
    while (nl < LANES && bi < bfd_lanes.size() && nr + nrows_lane[bfd_lanes[bi]] <= MAX_SLOT_ROWS) {
      nr += nrows_lane[bfd_lanes[bi]];
      slot_lanes.push_back(bfd_lanes[bi++]);
      ++nl;
    }
    while (nl < LANES && pi < piece_lanes.size()) {
      slot_lanes.push_back(piece_lanes[pi++]);
      ++nl;
    }
    for (; nl < LANES; ++nl) slot_lanes.push_back(-1);
  }
  // numbering: short rows in slot / lane / position order, pieces likewise
  P.new_of_old.assign(rows, -1);
  const int nslots = (int)(slot_lanes.size() / LANES);
  P.slots.resize(nslots);
  P.slot_lanes = slot_lanes;
  P.lane_ptr.assign(head.size() + 1, 0);
  int32_t nshort = 0, npieces = 0;
  std::vector<int32_t> piece_of_seg(segs.size(), -1);
  for (int s = 0; s < nslots; ++s) {
    P.slots[s].inst = 0;
    P.slots[s].pad = 0;
    P.slots[s].row_base = nshort;
    for (int l = 0; l < LANES; ++l) {
      const int32_t lane = slot_lanes[(size_t)s * LANES + l];
      if (lane < 0) continue;
      for (int32_t g = head[lane]; g >= 0; g = next[g]) {
        if (segs[g].piece) piece_of_seg[g] = npieces++;
        else P.new_of_old[segs[g].row] = nshort++;
      }
    }
    P.slots[s].nrows = nshort - P.slots[s].row_base;
  }
  P.nshort = nshort;
  P.nlong = (int)P.long_rows.size();
  P.npieces = npieces;
  for (int i = 0; i < P.nlong; ++i) P.new_of_old[P.long_rows[i]] = nshort + i;
  P.old_of_new.assign(rows, 0);
  for (int r = 0; r < rows; ++r) P.old_of_new[P.new_of_old[r]] = r;
  // flattened lane contents (lanes in creation order)
  for (size_t lane = 0; lane < head.size(); ++lane) {
    int cnt = 0;
    for (int32_t g = head[lane]; g >= 0; g = next[g]) ++cnt;
    P.lane_ptr[lane + 1] = P.lane_ptr[lane] + cnt;
  }
  P.segs.resize(P.lane_ptr.back());
  for (size_t lane = 0; lane < head.size(); ++lane) {
    int k = P.lane_ptr[lane];
    for (int32_t g = head[lane]; g >= 0; g = next[g])
      P.segs[k++] = {segs[g].row, segs[g].first, segs[g].count, piece_of_seg[g]};
  }
  // pieces of each long row in row order
  P.long_inst.assign(P.nlong, 0);
  P.long_ptr.assign(P.nlong + 1, 0);
  for (int i = 0; i < P.nlong; ++i) {
    const int64_t L = ptr[P.long_rows[i] + 1] - ptr[P.long_rows[i]];
    P.long_ptr[i + 1] = P.long_ptr[i] + (int32_t)((L + LANE_ITEMS - 1) / LANE_ITEMS);
  }
  P.long_piece.assign(P.long_ptr.back(), -1);
  for (size_t g = 0; g < segs.size(); ++g) {
    if (!segs[g].piece) continue;
    const int32_t i = long_of_row[segs[g].row];
    P.long_piece[P.long_ptr[i] + segs[g].first / LANE_ITEMS] = piece_of_seg[g];
  }
}

void plan_packing_batch(int rows, const std::vector<int64_t>& ptr,
                        const std::vector<int32_t>& offsets, PackPlan& P) {
  P = PackPlan{};
  P.new_of_old.assign(rows, 0);
  P.old_of_new.assign(rows, 0);
  P.lane_ptr.assign(1, 0);
  std::vector<int32_t> lrow, linst, lcount;
  std::vector<std::vector<int32_t>> lpieces;
  const int ninst = (int)offsets.size() - 1;
  // the instances are planned independently (on threads, ranges of instances of about equal
  // nonzeros), then concatenated in instance order
  std::vector<PackPlan> plans(ninst);
  {
    std::vector<int64_t> inst_nnz(ninst + 1);
    for (int i = 0; i <= ninst; ++i) inst_nnz[i] = ptr[offsets[i]];
    run_parts(balanced_rows(ninst, inst_nnz.data(), host_threads()),
              [&](int, int64_t i0, int64_t i1) {
                for (int64_t i = i0; i < i1; ++i) {
                  const int off = offsets[i], len = offsets[i + 1] - offsets[i];
                  std::vector<int64_t> sub(len + 1);
                  for (int r = 0; r <= len; ++r) sub[r] = ptr[off + r] - ptr[off];
                  plan_packing(len, sub, plans[i]);
                }
              });
  }
  for (int i = 0; i < ninst; ++i) {
    const int off = offsets[i], len = offsets[i + 1] - offsets[i];
    const PackPlan Q = std::move(plans[i]);  // freed at the end of this instance
    const int32_t lane_off = (int32_t)P.lane_ptr.size() - 1;
    const int32_t seg_off = (int32_t)P.segs.size();
    const int32_t piece_off = P.npieces;
    for (int r = 0; r < len; ++r) {
      P.new_of_old[off + r] = off + Q.new_of_old[r];
      P.old_of_new[off + r] = off + Q.old_of_new[r];
    }
    for (size_t k = 1; k < Q.lane_ptr.size(); ++k) P.lane_ptr.push_back(seg_off + Q.lane_ptr[k]);
    for (const PackPlan::Seg& g : Q.segs)
      P.segs.push_back({g.row + off, g.first, g.count, g.piece >= 0 ? g.piece + piece_off : -1});
    for (int32_t l : Q.slot_lanes) P.slot_lanes.push_back(l >= 0 ? l + lane_off : -1);
    for (SlotDesc d : Q.slots) {
      d.row_base += off;
      d.inst = i;
      P.slots.push_back(d);
    }
    for (int k = 0; k < Q.nlong; ++k) {
      lrow.push_back(Q.long_rows[k] + off);
      linst.push_back(i);
      std::vector<int32_t> pcs;
      for (int q = Q.long_ptr[k]; q < Q.long_ptr[k + 1]; ++q) pcs.push_back(Q.long_piece[q] + piece_off);
      lpieces.push_back(pcs);
    }
    P.nshort += Q.nshort;
    P.npieces += Q.npieces;
  }
  // long rows of all instances, longest first (their new indices are already fixed)
  std::vector<int32_t> order(lrow.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return lpieces[a].size() > lpieces[b].size();
  });
  P.nlong = (int)lrow.size();
  P.long_ptr.assign(1, 0);
  for (int32_t k : order) {
    P.long_rows.push_back(lrow[k]);
    P.long_inst.push_back(linst[k]);
    for (int32_t q : lpieces[k]) P.long_piece.push_back(q);
    P.long_ptr.push_back((int32_t)P.long_piece.size());
  }
}

void build_packed(int rows, int cols, const std::vector<int64_t>& ptr,
                  const std::vector<int32_t>& idx, const std::vector<double>& val,
                  const PackPlan& P, const std::vector<int32_t>& col_new_of_old,
                  HostPacked& out) {
  out = HostPacked{};
  out.rows = rows;
  out.cols = cols;
  out.nslots = (int)P.slots.size();
  out.nshort = P.nshort;
  out.nlong = P.nlong;
  out.npieces = P.npieces;
  out.stored = (int64_t)out.nslots * SLOT_ITEMS;
  out.val.assign(out.stored, 0.0);  // padding: value 0, column 0, no flag
  out.val32.assign(out.stored, 0.0f);
  out.idx.assign(out.stored, 0u);
  out.slots = P.slots;
  out.lanes.assign((size_t)out.nslots * LANES, LaneMeta{0, 0});
  // global id of the first piece in each slot (pieces are numbered in slot / lane order),
  // so that slots can be filled independently
  std::vector<int32_t> slot_piece(out.nslots + 1, 0);
  for (int s = 0; s < out.nslots; ++s) {
    int32_t c = 0;
    for (int l = 0; l < LANES; ++l) {
      const int32_t lane = P.slot_lanes[(size_t)s * LANES + l];
      if (lane < 0) continue;
      for (int k = P.lane_ptr[lane]; k < P.lane_ptr[lane + 1]; ++k) c += P.segs[k].piece >= 0;
    }
    slot_piece[s + 1] = slot_piece[s] + c;
  }
  const std::vector<int64_t> parts = even_parts(out.nslots, host_threads());
  std::vector<char> exact(parts.size() - 1, 1);  // per part: every value fits FP32 exactly
  run_parts(parts, [&](int part, int64_t s0, int64_t s1) {
    bool ok = true;
    for (int64_t s = s0; s < s1; ++s) {
      double* sv = out.val.data() + (size_t)s * SLOT_ITEMS;
      uint32_t* si = out.idx.data() + (size_t)s * SLOT_ITEMS;
      float* sf = out.val32.data() + (size_t)s * SLOT_ITEMS;
      int32_t rows_before = 0, piece_counter = slot_piece[s];
      for (int l = 0; l < LANES; ++l) {
        LaneMeta& lm = out.lanes[(size_t)s * LANES + l];
        lm.row_local = rows_before;
        lm.piece_base = piece_counter;
        const int32_t lane = P.slot_lanes[(size_t)s * LANES + l];
        if (lane < 0) continue;
        int p = 0;
        auto put = [&](double v, uint32_t c) {
          sv[((p >> 1) * LANES + l) * 2 + (p & 1)] = v;
          si[((p >> 2) * LANES + l) * 4 + (p & 3)] = c;
          const float f = (float)v;
          if (v != 0.0 && !(std::isfinite(f) && std::fabs(f) >= FLT_MIN)) ok = false;
          sf[((p >> 2) * LANES + l) * 4 + (p & 3)] = f;
          ++p;
        };
        for (int k = P.lane_ptr[lane]; k < P.lane_ptr[lane + 1]; ++k) {
          const PackPlan::Seg& g = P.segs[k];
          const uint32_t end = END_BIT | (g.piece >= 0 ? PIECE_BIT : 0u);
          if (g.piece >= 0) ++piece_counter; else ++rows_before;
          if (g.count == 0) {  // empty row: one stored zero carries its end flag
            put(0.0, end);
            continue;
          }
          const int64_t e0 = ptr[g.row] + g.first;
          for (int q = 0; q < g.count; ++q) {
            const uint32_t c = (uint32_t)col_new_of_old[idx[e0 + q]];
            put(val[e0 + q], c | (q == g.count - 1 ? end : 0u));
          }
        }
      }
    }
    exact[part] = ok;
  });
  for (char e : exact) out.fp32_exact_range = out.fp32_exact_range && e;
  out.long_row.resize(P.nlong);
  for (int i = 0; i < P.nlong; ++i) out.long_row[i] = P.new_of_old[P.long_rows[i]];
  out.long_inst = P.long_inst;
  out.long_ptr = P.long_ptr;
  out.long_piece = P.long_piece;
  out.nlong_block = out.nlong_warp = 0;  // rows sorted by pieces: block rows, then warp rows
  for (int i = 0; i < P.nlong; ++i) {
    const int pieces = P.long_ptr[i + 1] - P.long_ptr[i];
    if (pieces > LONG_BLOCK_PIECES) ++out.nlong_block;
    else if (pieces > LONG_WARP_PIECES) ++out.nlong_warp;
  }
}

void build_chunks(const std::vector<int32_t>& offsets, int chunk, std::vector<int32_t>& chunks,
                  std::vector<int32_t>& inst_chunk) {
  chunks.clear();
  inst_chunk.assign(1, 0);
  const int ninst = (int)offsets.size() - 1;
  for (int i = 0; i < ninst; ++i) {
    for (int a = offsets[i]; a < offsets[i + 1]; a += chunk) {
      const int len = std::min(chunk, offsets[i + 1] - a);
      chunks.insert(chunks.end(), {i, a, len, 0});
    }
    inst_chunk.push_back((int32_t)(chunks.size() / 4));
  }
}

// Padding entries and the stored zero of an empty row gather entry 0 of the other
// orientation's vector (value 0 times a finite entry).  In a batch entry 0 belongs to
// instance 0, so a non-finite iterate there would reach the other instances' rows through
// 0 * inf = NaN.  Each slot of instance i instead gathers offsets[i], the instance's own
// first entry: its entry 0 in a solve of its own, so the batch still mirrors that solve.
// An entry of such a slot with index 0 is never a real nonzero unless offsets[i] is 0
// (load checks that nonzeros lie in their instance's range), when nothing changes.  An
// instance with no entries in that orientation keeps index 0.
void own_instance_zero_gathers(HostPacked& H, const std::vector<int32_t>& offsets) {
  run_parts(even_parts(H.nslots, host_threads()), [&](int, int64_t s0, int64_t s1) {
    for (int64_t s = s0; s < s1; ++s) {  // slots are independent
      const int inst = H.slots[s].inst;
      if (offsets[inst + 1] == offsets[inst]) continue;
      const uint32_t base = (uint32_t)offsets[inst];
      uint32_t* si = H.idx.data() + (size_t)s * SLOT_ITEMS;
      for (int k = 0; k < SLOT_ITEMS; ++k)
        if ((si[k] & IDX_MASK) == 0) si[k] |= base;
    }
  });
}

}  // namespace pdhg

// Host threads for the load-time preprocessing loops (row permutation, transpose, packed
// arrays).  Work is split into contiguous ranges, each output element is written by one
// thread with the value the sequential loop writes, so results do not depend on the number
// of threads.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <thread>
#include <vector>

namespace pdhg {

// Worker threads for the load: DPDLP_HOST_THREADS if set (1..64), else the machine's
// hardware threads, at most 16.
inline int host_threads() {
  if (const char* e = std::getenv("DPDLP_HOST_THREADS")) {
    const int v = std::atoi(e);
    if (v >= 1) return std::min(v, 64);
  }
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h, 16u));
}

// f(part, begin, end) for every range [bounds[p], bounds[p + 1]); part 0 runs on the
// calling thread, the others on threads of their own.
template <class F>
void run_parts(const std::vector<int64_t>& bounds, F&& f) {
  const int parts = (int)bounds.size() - 1;
  std::vector<std::thread> th;
  th.reserve(parts > 1 ? parts - 1 : 0);
  for (int p = 1; p < parts; ++p) th.emplace_back([&f, &bounds, p] { f(p, bounds[p], bounds[p + 1]); });
  if (parts > 0) f(0, bounds[0], bounds[1]);
  for (std::thread& t : th) t.join();
}

// Rows [0, rows) cut into at most `parts` consecutive ranges of about equal weight, the
// weight of row r being its nonzeros (prefix[r + 1] - prefix[r]) plus one.
inline std::vector<int64_t> balanced_rows(int rows, const int64_t* prefix, int parts) {
  std::vector<int64_t> b(1, 0);
  if (rows <= 0) {
    b.push_back(0);
    return b;
  }
  parts = std::max(1, std::min(parts, rows));
  const int64_t total = prefix[rows] - prefix[0] + rows;
  int64_t lo = 0;
  for (int p = 1; p < parts; ++p) {
    const int64_t target = total * p / parts;
    // first row r >= lo whose cumulative weight (prefix[r] - prefix[0] + r) reaches target
    int64_t a = lo, z = rows;
    while (a < z) {
      const int64_t mid = (a + z) / 2;
      if (prefix[mid] - prefix[0] + mid >= target) z = mid; else a = mid + 1;
    }
    if (a > lo && a < rows) {
      b.push_back(a);
      lo = a;
    }
  }
  b.push_back(rows);
  return b;
}

// [0, n) cut into at most `parts` ranges of equal length.
inline std::vector<int64_t> even_parts(int64_t n, int parts) {
  parts = (int)std::max<int64_t>(1, std::min<int64_t>(parts, n));
  std::vector<int64_t> b(parts + 1);
  for (int p = 0; p <= parts; ++p) b[p] = n * p / parts;
  return b;
}

}  // namespace pdhg

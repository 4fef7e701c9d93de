// parallel.h -- host thread helper of the plan builders (internal).
#pragma once
#include <algorithm>
#include <thread>
#include <vector>

namespace ompdart {

// f(t, lo, hi) for t < T over [0, n) split in T contiguous ranges, on up to
// `max_threads` host threads (the calling thread takes t = 0), no more than
// one per `min_per_thread` items; returns T
template <class F>
int parallel_ranges(int n, int min_per_thread, int max_threads, F f) {
  if (max_threads < 2 || n / std::max(1, min_per_thread) < 2) {  // small: no thread, no query
    f(0, 0, n);
    return 1;
  }
  static const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int T = std::max(1, std::min({hw, max_threads, n / std::max(1, min_per_thread)}));
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t)
    pool.emplace_back(f, t, (int)((long long)n * t / T), (int)((long long)n * (t + 1) / T));
  f(0, 0, (int)((long long)n / T));
  for (auto &x : pool) x.join();
  return T;
}

}  // namespace ompdart

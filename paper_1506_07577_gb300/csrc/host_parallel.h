// Host-side helpers of the library's set-up code (finalize, re-tiling):
// work split over host threads, and a stable radix order.
#pragma once

#include <algorithm>
#include <cstdint>
#include <exception>
#include <mutex>
#include <system_error>
#include <thread>
#include <vector>

namespace ebb {

// fn(lo, hi) runs over contiguous ranges covering [0, n), at least
// `min_chunk` items each, on up to 16 host threads (the calling thread takes
// the first range; a thread that cannot be started leaves its range to the
// caller).  fn must only write state of its own range.  An exception thrown
// by fn on any thread is rethrown on the calling thread once every range has
// finished or given up.
template <class F>
void parallel_ranges(int n, int min_chunk, F&& fn) {
  const int hw = (int)std::thread::hardware_concurrency();
  const int nth = std::max(1, std::min({hw > 0 ? hw : 1, 16, n / std::max(1, min_chunk)}));
  auto lo_of = [&](int i) { return (int)((long long)n * i / nth); };
  std::exception_ptr first_error;
  std::mutex error_mutex;
  auto guarded = [&](int lo, int hi) {
    try {
      fn(lo, hi);
    } catch (...) {
      std::lock_guard<std::mutex> lock(error_mutex);
      if (!first_error) first_error = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  std::vector<int> inline_ranges;
  for (int i = 1; i < nth; ++i) {
    try {
      th.emplace_back([&guarded, lo = lo_of(i), hi = lo_of(i + 1)] { guarded(lo, hi); });
    } catch (const std::system_error&) {
      inline_ranges.push_back(i);
    }
  }
  guarded(0, lo_of(1));
  for (int i : inline_ranges) guarded(lo_of(i), lo_of(i + 1));
  for (auto& t : th) t.join();
  if (first_error) std::rethrow_exception(first_error);
}

// Stable order of `key` (its low `bits` bits): order[i] = the index of the
// i-th smallest key, equal keys in index order (LSD radix sort, 11-bit
// digits).  With `order` non-empty on entry, that order is refined instead:
// the result sorts by key and keeps the given order among equal keys.
void radix_order(const std::vector<uint64_t>& key, int bits, std::vector<int>& order);

}  // namespace ebb

// sk_range_alloc.h -- first-fit range allocator of the serving arena and of
// its pinned host staging pool (host code only, no CUDA dependency).
//
// Manages the byte offsets [0, size) in 256-byte units. alloc(n) rounds n up
// to a whole number of units (at least one) and returns the lowest offset at
// which a free range holds it; release(off, n) returns a block and merges it
// with free neighbours, so free ranges stay maximal and a full release
// restores one range [0, size). Not thread-safe: the server calls it under
// its mutex.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace sk {

class RangeAlloc {
 public:
  static constexpr size_t UNIT = 256;

  void reset(size_t size) {
    free_.clear();
    free_[0] = size;
  }
  bool alloc(size_t n, size_t* off) {
    n = round_up(n ? n : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = round_up(n ? n : 1);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  // free ranges as (offset, bytes), in address order
  const std::map<size_t, size_t>& free_ranges() const { return free_; }

 private:
  static size_t round_up(size_t n) { return (n + UNIT - 1) / UNIT * UNIT; }
  std::map<size_t, size_t> free_;
};

}  // namespace sk

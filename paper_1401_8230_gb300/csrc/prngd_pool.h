// prngd_pool.h -- first-fit range allocator over [0, size) in 256-byte granules, with free
// neighbours merged on release: the bookkeeping of the serving loop's output pool (host code;
// the loop maps offsets onto one device allocation).
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <iterator>
#include <map>

namespace prngd_host {

class RangePool {
 public:
  static constexpr size_t kGranule = 256;
  static constexpr size_t kNone = SIZE_MAX;

  explicit RangePool(size_t size = 0) { reset(size); }

  // Forget every allocation; the whole range [0, size) is free (size rounded down to granules).
  void reset(size_t size) {
    free_.clear();
    size_ = size & ~(kGranule - 1);
    used_ = 0;
    if (size_) free_[0] = size_;
  }

  // Bytes an allocation of `bytes` takes: whole granules, at least one.
  static size_t footprint(size_t bytes) { return bytes <= kGranule ? kGranule : (bytes + kGranule - 1) & ~(kGranule - 1); }

  // Offset of the lowest free range that holds `bytes`, or kNone.
  size_t alloc(size_t bytes) {
    if (bytes > size_) return kNone;
    bytes = footprint(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_ += bytes;
        return off;
      }
    }
    return kNone;
  }

  // Return an allocation (`off` and the `bytes` it was made with); merges it with free
  // neighbours.
  void release(size_t off, size_t bytes) {
    bytes = footprint(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
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

  size_t used() const { return used_; }
  size_t size() const { return size_; }
  size_t free_ranges() const { return free_.size(); }
  // f(offset, length) for every free range, in address order.
  template <class F>
  void for_each_free(F f) const {
    for (const auto& kv : free_) f(kv.first, kv.second);
  }

 private:
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length of each free range
};

}  // namespace prngd_host

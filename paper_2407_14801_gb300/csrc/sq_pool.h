// Best-fit range allocator over one device slab (the serving memory pool).
// Host-only bookkeeping: offsets into [0, capacity) with 256-byte
// granularity, neighbouring free ranges merged on release.  Not thread-safe;
// the server serialises access with its mutex.
#pragma once
#include <cstdint>
#include <map>
#include <unordered_map>

namespace sq {

class RangePool {
 public:
  static constexpr uint64_t kAlign = 256;

  explicit RangePool(uint64_t capacity = 0) { reset(capacity); }

  void reset(uint64_t capacity) {
    cap_ = capacity & ~(kAlign - 1);
    used_ = 0;
    by_off_.clear();
    by_size_.clear();
    live_.clear();
    if (cap_) insert_free(0, cap_);
  }

  // Smallest free range that fits; returns false when none does.
  bool alloc(uint64_t bytes, uint64_t *off) {
    const uint64_t need = round(bytes ? bytes : 1);
    auto it = by_size_.lower_bound(need);
    if (it == by_size_.end()) return false;
    const uint64_t size = it->first, o = it->second;
    erase_free(o, size);
    if (size > need) insert_free(o + need, size - need);
    live_[o] = need;
    used_ += need;
    *off = o;
    return true;
  }

  // Releases a range returned by alloc; false if `off` is not live.
  bool release(uint64_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    uint64_t o = off, size = it->second;
    live_.erase(it);
    used_ -= size;
    auto nx = by_off_.find(o + size);  // merge with the following free range
    if (nx != by_off_.end()) {
      const uint64_t s2 = nx->second;
      erase_free(o + size, s2);
      size += s2;
    }
    auto pv = by_off_.lower_bound(o);  // and with the preceding one
    if (pv != by_off_.begin()) {
      --pv;
      if (pv->first + pv->second == o) {
        const uint64_t o2 = pv->first, s2 = pv->second;
        erase_free(o2, s2);
        o = o2;
        size += s2;
      }
    }
    insert_free(o, size);
    return true;
  }

  bool fits(uint64_t bytes) const {
    return !by_size_.empty() && by_size_.rbegin()->first >= round(bytes ? bytes : 1);
  }
  uint64_t capacity() const { return cap_; }
  uint64_t used() const { return used_; }
  uint64_t largest_free() const { return by_size_.empty() ? 0 : by_size_.rbegin()->first; }
  size_t free_ranges() const { return by_off_.size(); }
  size_t live_ranges() const { return live_.size(); }
  static uint64_t round(uint64_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

 private:
  void insert_free(uint64_t o, uint64_t s) {
    by_off_[o] = s;
    by_size_.emplace(s, o);
  }
  void erase_free(uint64_t o, uint64_t s) {
    by_off_.erase(o);
    auto r = by_size_.equal_range(s);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second == o) {
        by_size_.erase(it);
        break;
      }
  }
  uint64_t cap_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> by_off_;        // free: offset -> size
  std::multimap<uint64_t, uint64_t> by_size_;  // free: size -> offset
  std::unordered_map<uint64_t, uint64_t> live_;
};

}  // namespace sq

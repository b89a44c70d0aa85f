// range_alloc.h -- first-fit allocator of index ranges [0, cap), used for the
// device-polling server's partial slots (plain C++, no CUDA).
#pragma once

#include <stdint.h>

#include <iterator>
#include <map>

namespace scl {

class RangeAlloc {
  public:
    void init(uint32_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
    }
    // First fit; false if no free range of n indices exists.
    bool alloc(uint32_t n, uint32_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const uint32_t at = it->first + n, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    // Return [off, off + n); merges with free neighbours.
    void release(uint32_t off, uint32_t n) {
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t free_ranges() const { return free_.size(); }

  private:
    std::map<uint32_t, uint32_t> free_;   // offset -> length
};

}  // namespace scl

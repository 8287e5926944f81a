// gpz_arena.hpp -- first-fit allocator of offsets inside one device memory
// range of fixed capacity: the serving engine's admission budget.  Pure host
// code (no CUDA calls), so it can be tested without a GPU.
//
// Ranges are handed out 256-byte aligned (every size is rounded up).  Free
// ranges are kept sorted by offset and merged with their neighbours when a
// range is returned, so that memory released in any order coalesces back
// into one range.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>
#include <unordered_map>

namespace gpz {
namespace host {

class Arena {
   public:
    explicit Arena(uint64_t capacity, uint64_t align = 256) : align_(align) {
        capacity_ = capacity / align_ * align_;
        if (capacity_) free_[0] = capacity_;
    }

    uint64_t rounded(uint64_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }

    // First fit: the lowest free range that holds `bytes` (rounded up).
    // Returns false, changing nothing, when no free range is large enough.
    bool alloc(uint64_t bytes, uint64_t* offset) {
        const uint64_t need = rounded(bytes == 0 ? 1 : bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const uint64_t at = it->first, left = it->second - need;
            free_.erase(it);
            if (left) free_[at + need] = left;
            used_[at] = need;
            used_bytes_ += need;
            if (used_bytes_ > peak_) peak_ = used_bytes_;
            *offset = at;
            return true;
        }
        return false;
    }

    // Return the range that alloc() placed at `offset`; false if there is none.
    bool release(uint64_t offset) {
        auto u = used_.find(offset);
        if (u == used_.end()) return false;
        uint64_t at = offset, size = u->second;
        used_.erase(u);
        used_bytes_ -= size;
        auto next = free_.lower_bound(at);
        if (next != free_.end() && at + size == next->first) {  // merge with the following range
            size += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {  // merge with the preceding range
            auto prev = std::prev(next);
            if (prev->first + prev->second == at) {
                prev->second += size;
                return true;
            }
        }
        free_[at] = size;
        return true;
    }

    // Whether `bytes` could be allocated now.
    bool fits(uint64_t bytes) const { return largest_free() >= rounded(bytes == 0 ? 1 : bytes); }

    uint64_t largest_free() const {
        uint64_t m = 0;
        for (const auto& f : free_)
            if (f.second > m) m = f.second;
        return m;
    }
    uint64_t capacity() const { return capacity_; }
    uint64_t used_bytes() const { return used_bytes_; }
    uint64_t peak_bytes() const { return peak_; }
    size_t free_ranges() const { return free_.size(); }
    size_t live_ranges() const { return used_.size(); }

   private:
    uint64_t align_, capacity_ = 0, used_bytes_ = 0, peak_ = 0;
    std::map<uint64_t, uint64_t> free_;            // offset -> size
    std::unordered_map<uint64_t, uint64_t> used_;  // offset -> size
};

}  // namespace host
}  // namespace gpz

// arena.h -- the serving budget's allocator (host only, no CUDA).
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace qsim {

// First-fit allocator over [0, size) with 256-byte granularity; coalesces on free.
class Arena {
  public:
    void init(size_t size) { free_[0] = size; size_ = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                sizes_[*off] = bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t bytes = s->second;
        sizes_.erase(s);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            free_.erase(next);
        }
        auto nx = free_.lower_bound(off);
        if (nx != free_.begin()) {
            auto prev = std::prev(nx);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }
    size_t capacity() const { return size_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }
    // the free blocks and the allocated ones: offset -> length, ascending
    const std::map<size_t, size_t> &free_blocks() const { return free_; }
    const std::map<size_t, size_t> &allocated() const { return sizes_; }

  private:
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> sizes_;  // allocated offset -> length
    size_t used_ = 0, peak_ = 0, size_ = 0;
};

}  // namespace qsim

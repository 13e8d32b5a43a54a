// pool_alloc.h -- first-fit allocator of the serving queue's device pool
// (host code only: it hands out offsets; the queue adds them to the pool's
// base pointer).  Free space is a map offset -> length; a release merges the
// freed block with free neighbours on both sides.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace mps {

constexpr size_t kPoolAlign = 256;  // every block starts on a 256-byte boundary

inline size_t align_up(size_t x) { return (x + kPoolAlign - 1) / kPoolAlign * kPoolAlign; }

// First-fit allocator over [0, size) of the pool.
class PoolAllocator {
public:
    explicit PoolAllocator(size_t size) { free_[0] = size; }
    // Lowest-offset free block that holds `bytes` (rounded up to kPoolAlign);
    // false if none does.
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes;
                size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    // Returns a block given out by alloc (same offset and requested size).
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes ? bytes : 1);
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
    size_t free_blocks() const { return free_.size(); }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

}  // namespace mps

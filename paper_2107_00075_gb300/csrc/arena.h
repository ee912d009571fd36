// arena.h -- the coloring server's HBM arena bookkeeping (host only).
//
// First-fit allocation of byte ranges in [0, cap) with coalescing of free
// neighbours on release.  The server sizes one device buffer to the budget
// and admits a request only when alloc() finds room for its whole device
// footprint; the offsets it returns index into that buffer.  Plain C++ (no
// CUDA), so the host-side tests compile it on its own.
#pragma once
#include <cstddef>
#include <iterator>
#include <map>

namespace pgc {
namespace serve {

class Arena {
  public:
    void init(size_t cap) {
        cap_ = cap;
        free_.clear();
        if (cap) free_[0] = cap;
        used_ = 0;
    }
    // The lowest-offset free range that holds `bytes`; false if none does.
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    // Returns a range that alloc() handed out (same offset and size).
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t free_ranges() const { return free_.size(); }

  private:
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace serve
}  // namespace pgc

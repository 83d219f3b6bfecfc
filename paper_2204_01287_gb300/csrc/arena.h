// arena.h — first-fit range allocator of the serving loop's framebuffer and
// pinned image pools: offsets into [0, size), lengths rounded up to kAlign,
// neighbouring free ranges merged on release. Pure host code, not thread-safe
// (the serving loop calls it under its own mutex).
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace pcr {
namespace serve_detail {

constexpr uint64_t kAlign = 256;

inline uint64_t round_up(uint64_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

struct Arena {
    uint64_t size = 0;
    std::map<uint64_t, uint64_t> free_;   // offset -> length

    void init(uint64_t n) {
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    // The lowest free offset with room for n bytes (rounded up); false if none.
    bool alloc(uint64_t n, uint64_t& off) {
        n = round_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                uint64_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                return true;
            }
        }
        return false;
    }
    // Return [off, off + n) (n as given to alloc) and merge it with its free
    // neighbours.
    void release(uint64_t off, uint64_t n) {
        n = round_up(n);
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
};

}  // namespace serve_detail
}  // namespace pcr

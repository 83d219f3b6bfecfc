// Unit test of the serving loop's range allocator (arena.h) against a
// brute-force model: a bitmap of 256-byte units where alloc takes the first
// run of free units long enough. The arena keeps its free ranges fully merged,
// so both must pick the same offsets in any sequence of calls.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <utility>
#include <vector>

#include "arena.h"

using pcr::serve_detail::Arena;
using pcr::serve_detail::kAlign;

static int failures = 0;
#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);            \
            ++failures;                                                 \
        }                                                               \
    } while (0)

struct Model {
    std::vector<bool> used;
    explicit Model(uint64_t units) : used(units, false) {}
    bool alloc(uint64_t bytes, uint64_t& off) {
        const uint64_t n = (bytes + kAlign - 1) / kAlign;
        uint64_t run = 0;
        for (uint64_t u = 0; u < used.size(); ++u) {
            run = used[u] ? 0 : run + 1;
            if (n && run == n) {
                const uint64_t first = u + 1 - n;
                for (uint64_t k = first; k <= u; ++k) used[k] = true;
                off = first * kAlign;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        const uint64_t n = (bytes + kAlign - 1) / kAlign;
        for (uint64_t k = off / kAlign; k < off / kAlign + n; ++k) used[k] = false;
    }
};

int main() {
    {   // hand case: first fit, rounding, merging on release
        Arena a;
        a.init(16 * kAlign);
        uint64_t o0, o1, o2, o3;
        CHECK(a.alloc(1, o0) && o0 == 0);
        CHECK(a.alloc(300, o1) && o1 == kAlign);          // 2 units
        CHECK(a.alloc(kAlign, o2) && o2 == 3 * kAlign);
        a.release(o1, 300);
        CHECK(a.free_.size() == 2);                        // [1,3) and [4,16)
        CHECK(a.alloc(2 * kAlign, o3) && o3 == kAlign);    // back into the hole
        CHECK(!a.alloc(13 * kAlign, o3));                  // 12 units left, in one range
        CHECK(a.alloc(12 * kAlign, o3) && o3 == 4 * kAlign);
        CHECK(!a.alloc(1, o3));                            // full
        a.release(o0, 1);
        a.release(kAlign, 2 * kAlign);
        a.release(o2, kAlign);
        a.release(4 * kAlign, 12 * kAlign);
        CHECK(a.free_.size() == 1 && a.free_.begin()->first == 0 &&
              a.free_.begin()->second == 16 * kAlign);
    }
    {   // an empty pool holds nothing
        Arena a;
        a.init(0);
        uint64_t o;
        CHECK(!a.alloc(1, o));
    }
    {   // random sequences against the model
        std::mt19937_64 rng(12345);
        for (int trial = 0; trial < 200; ++trial) {
            const uint64_t units = 1 + rng() % 300;
            Arena a;
            a.init(units * kAlign);
            Model m(units);
            std::vector<std::pair<uint64_t, uint64_t>> live;
            for (int step = 0; step < 400; ++step) {
                if (live.empty() || rng() % 3 != 0) {
                    const uint64_t bytes = 1 + rng() % (kAlign * (1 + rng() % 24));
                    uint64_t oa = ~0ull, om = ~0ull;
                    const bool ra = a.alloc(bytes, oa), rm = m.alloc(bytes, om);
                    CHECK(ra == rm);
                    if (ra && rm) {
                        CHECK(oa == om);
                        live.push_back({oa, bytes});
                    }
                } else {
                    const size_t k = rng() % live.size();
                    a.release(live[k].first, live[k].second);
                    m.release(live[k].first, live[k].second);
                    live.erase(live.begin() + k);
                }
                // free ranges are disjoint, maximal and inside the pool
                uint64_t end = 0;
                bool first = true;
                for (auto& r : a.free_) {
                    CHECK(r.second > 0 && r.first + r.second <= units * kAlign);
                    CHECK(first || r.first > end);          // a gap: never adjacent
                    end = r.first + r.second;
                    first = false;
                }
                if (failures) return 1;
            }
            for (auto& l : live) a.release(l.first, l.second);
            CHECK(a.free_.size() == 1 && a.free_.begin()->second == units * kAlign);
            if (failures) return 1;
        }
    }
    if (failures) return 1;
    std::printf("arena ok\n");
    return 0;
}

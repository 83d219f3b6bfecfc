// encoder.cpp — host-side encoder (Sec. 3.1, Eq. 1, Listing 2), threaded.
//
// 1. Cloud box (binary32 min/max over all points).
// 2. 63-bit Morton code per point: q = floor(2^21 (p - cloudMin) / cloudSize)
//    per axis in binary64, clamped to [0, 2^21 - 1], bits interleaved with x
//    lowest.
// 3. Stable sort by code: one parallel MSD scatter on the top 16 code bits,
//    then an LSD radix sort of every bucket on the low 47 bits (buckets in
//    parallel). Ties keep input order, so the order is unique.
// 4. Batches of batch_size consecutive sorted points, binary32 box per batch
//    (size = max - min), Eq. 1 in binary64 per axis, and the 30-bit values
//    split into the low / medium / high words (x | y << 10 | z << 20).
// Coordinates must be finite: a NaN or an infinity is refused with PC_EINVAL.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "pc_internal.h"

namespace pcr {

unsigned hw_threads() {
    unsigned t = std::thread::hardware_concurrency();
    return t ? t : 1;
}

namespace {

template <class F>
void parallel_for(unsigned threads, uint64_t n, F&& f) {
    // f(thread_index, lo, hi) over a static split of [0, n)
    if (threads <= 1 || n < 2048) {
        f(0u, uint64_t(0), n);
        return;
    }
    std::vector<std::thread> pool;
    pool.reserve(threads);
    for (unsigned t = 0; t < threads; ++t) {
        uint64_t lo = n * t / threads, hi = n * (t + 1) / threads;
        pool.emplace_back([&f, t, lo, hi] { f(t, lo, hi); });
    }
    for (auto& th : pool) th.join();
}

template <class F>
void parallel_dynamic(unsigned threads, uint64_t n, uint64_t grain, F&& f) {
    // f(thread_index, lo, hi) over chunks of `grain` taken from a shared counter
    std::atomic<uint64_t> next{0};
    auto body = [&](unsigned t) {
        for (;;) {
            uint64_t lo = next.fetch_add(grain);
            if (lo >= n) break;
            f(t, lo, std::min(n, lo + grain));
        }
    };
    if (threads <= 1) {
        body(0);
        return;
    }
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < threads; ++t) pool.emplace_back(body, t);
    for (auto& th : pool) th.join();
}

// Spread the low 21 bits of v so that bit i lands on bit 3i.
inline uint64_t spread3(uint64_t v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x001F00000000FFFFull;
    v = (v | (v << 16)) & 0x001F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

struct MortonFrame {
    double lo[3], size[3];
    inline uint64_t code(const float* p) const {
        uint64_t q[3];
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            if (size[a] > 0.0) t = std::floor(2097152.0 * ((double)p[a] - lo[a]) / size[a]);
            t = t < 0.0 ? 0.0 : (t > 2097151.0 ? 2097151.0 : t);
            q[a] = (uint64_t)t;
        }
        return spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    }
};

// Eq. 1 in binary64 from binary32 inputs.
inline uint32_t fixed30(float v, float bmin, float bsize) {
    if (!(bsize > 0.0f)) return 0;
    double t = std::floor(1073741824.0 * ((double)v - (double)bmin) / (double)bsize);
    t = t < 0.0 ? 0.0 : (t > 1073741823.0 ? 1073741823.0 : t);
    return (uint32_t)t;
}

constexpr int kTopBits = 16;
constexpr int kLowBits = 63 - kTopBits;   // 47

// Stable LSD radix sort of (key, idx) on bits [0, kLowBits) of key.
void lsd_sort(uint64_t* key, uint32_t* idx, uint64_t m, std::vector<uint64_t>& tk,
              std::vector<uint32_t>& ti) {
    if (m < 2) return;
    if (m <= 48) {  // insertion sort: stable (moves only past strictly larger keys)
        for (uint64_t i = 1; i < m; ++i) {
            uint64_t k = key[i];
            uint32_t x = idx[i];
            uint64_t j = i;
            while (j > 0 && key[j - 1] > k) {
                key[j] = key[j - 1];
                idx[j] = idx[j - 1];
                --j;
            }
            key[j] = k;
            idx[j] = x;
        }
        return;
    }
    if (tk.size() < m) {
        tk.resize(m);
        ti.resize(m);
    }
    uint64_t* sk = key;
    uint32_t* si = idx;
    uint64_t* dk = tk.data();
    uint32_t* di = ti.data();
    for (int shift = 0; shift < kLowBits; shift += 8) {
        uint64_t cnt[256] = {0};
        for (uint64_t i = 0; i < m; ++i) cnt[(sk[i] >> shift) & 255]++;
        bool constant = false;
        for (int d = 0; d < 256; ++d)
            if (cnt[d] == m) constant = true;
        if (constant) continue;
        uint64_t off = 0;
        for (int d = 0; d < 256; ++d) {
            uint64_t c = cnt[d];
            cnt[d] = off;
            off += c;
        }
        for (uint64_t i = 0; i < m; ++i) {
            uint64_t p = cnt[(sk[i] >> shift) & 255]++;
            dk[p] = sk[i];
            di[p] = si[i];
        }
        std::swap(sk, dk);
        std::swap(si, di);
    }
    if (sk != key) {
        std::memcpy(key, sk, m * sizeof(uint64_t));
        std::memcpy(idx, si, m * sizeof(uint32_t));
    }
}

// Batches of batch_size consecutive points of the order idx: binary32 box,
// Eq. 1 and the word split (Sec. 3.1, Eq. 1, Listing 2).
void encode_batches(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
                    unsigned threads, const std::vector<uint32_t>& idx, pc_batch* batches,
                    uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color) {
    const uint64_t nbatch = (n + batch_size - 1) / batch_size;
    parallel_dynamic(threads, nbatch, 16, [&](unsigned, uint64_t blo, uint64_t bhi) {
        for (uint64_t b = blo; b < bhi; ++b) {
            uint64_t f = b * batch_size;
            uint64_t e = std::min<uint64_t>(n, f + batch_size);
            float mn[3], mx[3];
            for (int a = 0; a < 3; ++a) mn[a] = mx[a] = xyz[3 * (uint64_t)idx[f] + a];
            for (uint64_t j = f; j < e; ++j) {
                const float* p = &xyz[3 * (uint64_t)idx[j]];
                for (int a = 0; a < 3; ++a) {
                    if (p[a] < mn[a]) mn[a] = p[a];
                    if (p[a] > mx[a]) mx[a] = p[a];
                }
            }
            pc_batch& B = batches[b];
            for (int a = 0; a < 3; ++a) {
                B.min[a] = mn[a];
                B.size[a] = mx[a] - mn[a];
            }
            B.first = (uint32_t)f;
            B.count = (uint32_t)(e - f);
            for (uint64_t j = f; j < e; ++j) {
                const float* p = &xyz[3 * (uint64_t)idx[j]];
                uint32_t q0 = fixed30(p[0], B.min[0], B.size[0]);
                uint32_t q1 = fixed30(p[1], B.min[1], B.size[1]);
                uint32_t q2 = fixed30(p[2], B.min[2], B.size[2]);
                w1[j] = (q0 >> 20) | ((q1 >> 20) << 10) | ((q2 >> 20) << 20);
                w2[j] = ((q0 >> 10) & 1023u) | (((q1 >> 10) & 1023u) << 10) |
                        (((q2 >> 10) & 1023u) << 20);
                w3[j] = (q0 & 1023u) | ((q1 & 1023u) << 10) | ((q2 & 1023u) << 20);
                color[j] = rgba ? rgba[idx[j]] : 0u;
            }
        }
    });
}

}  // namespace

bool coords_finite(const float* xyz, uint64_t n, unsigned threads) {
    std::atomic<bool> ok{true};
    parallel_for(threads, 3 * n, [&](unsigned, uint64_t lo, uint64_t hi) {
        bool good = true;
        for (uint64_t i = lo; i < hi; ++i) good &= std::isfinite(xyz[i]);
        if (!good) ok = false;
    });
    return ok;
}

pc_status encode_host(const float* xyz, const uint32_t* rgba, uint64_t n,
                      uint32_t batch_size, unsigned threads, bool keep_order, pc_batch* batches,
                      uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color,
                      uint32_t* perm_out) {
    if (!xyz && n) return PC_EINVAL;
    if (batch_size == 0 || batch_size % 4 != 0) return PC_EINVAL;
    if (n >= 0xFFFFFFFFull) return PC_EINVAL;
    if (n == 0) return PC_OK;
    if (threads == 0) threads = hw_threads();
    threads = std::min<unsigned>(threads, 256);
    if (!coords_finite(xyz, n, threads)) return PC_EINVAL;   // Eq. 1 needs finite boxes
    std::vector<uint32_t> idx;
    if (keep_order) {
        try {
            idx.resize(n);
        } catch (...) {
            return PC_ENOMEM;
        }
        for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
        if (perm_out) std::memcpy(perm_out, idx.data(), n * sizeof(uint32_t));
        encode_batches(xyz, rgba, n, batch_size, threads, idx, batches, w1, w2, w3, color);
        return PC_OK;
    }

    // 1. cloud box
    std::vector<float> tlo(threads * 3), thi(threads * 3);
    std::vector<char> tused(threads, 0);
    parallel_for(threads, n, [&](unsigned t, uint64_t lo, uint64_t hi) {
        if (lo >= hi) return;
        float mn[3], mx[3];
        for (int a = 0; a < 3; ++a) mn[a] = mx[a] = xyz[3 * lo + a];
        for (uint64_t i = lo; i < hi; ++i)
            for (int a = 0; a < 3; ++a) {
                float v = xyz[3 * i + a];
                if (v < mn[a]) mn[a] = v;
                if (v > mx[a]) mx[a] = v;
            }
        for (int a = 0; a < 3; ++a) {
            tlo[3 * t + a] = mn[a];
            thi[3 * t + a] = mx[a];
        }
        tused[t] = 1;
    });
    float cmn[3], cmx[3];
    bool first = true;
    for (unsigned t = 0; t < threads; ++t) {
        if (!tused[t]) continue;
        for (int a = 0; a < 3; ++a) {
            if (first || tlo[3 * t + a] < cmn[a]) cmn[a] = tlo[3 * t + a];
            if (first || thi[3 * t + a] > cmx[a]) cmx[a] = thi[3 * t + a];
        }
        first = false;
    }
    MortonFrame fr;
    for (int a = 0; a < 3; ++a) {
        fr.lo[a] = (double)cmn[a];
        fr.size[a] = (double)cmx[a] - (double)cmn[a];
    }

    // 2.+3. MSD scatter on the top bits (codes computed twice to save memory)
    const uint64_t nb_top = 1ull << kTopBits;
    std::vector<uint64_t> keys;
    try {
        keys.resize(n);
        idx.resize(n);
    } catch (...) {
        return PC_ENOMEM;
    }
    // chunk the points into T contiguous ranges for a stable scatter
    const unsigned T = (unsigned)std::min<uint64_t>(threads, std::max<uint64_t>(1, n / 65536));
    std::vector<uint64_t> hist((uint64_t)T * nb_top, 0);
    parallel_for(T, n, [&](unsigned t, uint64_t lo, uint64_t hi) {
        uint64_t* h = &hist[(uint64_t)t * nb_top];
        for (uint64_t i = lo; i < hi; ++i) h[fr.code(&xyz[3 * i]) >> kLowBits]++;
    });
    std::vector<uint64_t> bucket_start(nb_top + 1, 0);
    {
        uint64_t off = 0;
        for (uint64_t d = 0; d < nb_top; ++d) {
            bucket_start[d] = off;
            for (unsigned t = 0; t < T; ++t) {
                uint64_t c = hist[(uint64_t)t * nb_top + d];
                hist[(uint64_t)t * nb_top + d] = off;
                off += c;
            }
        }
        bucket_start[nb_top] = off;
    }
    parallel_for(T, n, [&](unsigned t, uint64_t lo, uint64_t hi) {
        uint64_t* h = &hist[(uint64_t)t * nb_top];
        for (uint64_t i = lo; i < hi; ++i) {
            uint64_t c = fr.code(&xyz[3 * i]);
            uint64_t p = h[c >> kLowBits]++;
            keys[p] = c;
            idx[p] = (uint32_t)i;
        }
    });
    hist.clear();
    hist.shrink_to_fit();
    parallel_dynamic(threads, nb_top, 64, [&](unsigned, uint64_t lo, uint64_t hi) {
        std::vector<uint64_t> tk;
        std::vector<uint32_t> ti;
        for (uint64_t d = lo; d < hi; ++d) {
            uint64_t s = bucket_start[d], e = bucket_start[d + 1];
            lsd_sort(&keys[s], &idx[s], e - s, tk, ti);
        }
    });
    keys.clear();
    keys.shrink_to_fit();
    if (perm_out) std::memcpy(perm_out, idx.data(), n * sizeof(uint32_t));

    encode_batches(xyz, rgba, n, batch_size, threads, idx, batches, w1, w2, w3, color);
    return PC_OK;
}

}  // namespace pcr

// raster.cu — sm_103a kernels of the point rasterizer.
//
//   k_clear    visibility buffers <- all ones; scratch counters <- 0
//   k_cull     per batch and view: conservative frustum culling (Sec. 3.2) and
//              the precision k from the projected batch extent (Sec. 3.3);
//              surviving batches are appended, in segments of up to
//              kSegmentPoints points, to a draw list
//   k_raster   persistent warps take draw-list segments, load the k coordinate
//              words of 4 consecutive points with one 16-byte load per word
//              (Sec. 3.4), decode, project (Listing 1), do the non-atomic
//              early-depth test and atomicMin the 64-bit key; one pass serves
//              every view of the launch (Sec. 3.7)
//   k_resolve  visibility key -> colour of the winning point (Sec. 3.3)
//
// Bit-exactness: every float operation that decides a key or a pixel is an
// explicit round-to-nearest intrinsic in the same order as the CPU oracle's
// definition (decode x = min + float(X) * cell; c = ((m0 x + m4 y) + m8 z) +
// m12; f = ((c / w) * 0.5 + 0.5) * W with an IEEE divide). The file is also
// compiled with --fmad=false so nothing else is contracted.
#include <cstdint>

#include "pc_internal.h"

namespace pcr {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ void raise_error(Scratch s, uint32_t code, uint32_t info) {
    if (atomicCAS(&s.counters[C_ERROR], 0u, code) == 0u) s.counters[C_ERRINFO] = info;
}

// ---- k_clear -----------------------------------------------------------------

__global__ void k_clear(ViewTable vt, uint32_t view_base, Scratch s) {
    const uint32_t v = blockIdx.y;
    if (blockIdx.x == 0 && v == 0) {
        if (threadIdx.x < C_COUNT && threadIdx.x != C_ERROR && threadIdx.x != C_ERRINFO)
            s.counters[threadIdx.x] = 0u;
        for (uint32_t i = threadIdx.x; i < vt.n * S_COUNT; i += blockDim.x)
            s.stats[(uint64_t)view_base * S_COUNT + i] = 0ull;
    }
    if (v >= vt.n) return;
    const ViewParams& vp = vt.v[v];
    const uint64_t npix = (uint64_t)vp.width * vp.height;
    // 16-byte stores; vis is 16-byte aligned (checked on the host)
    ulonglong2* p2 = reinterpret_cast<ulonglong2*>(vp.vis);
    const uint64_t n2 = npix / 2;
    const ulonglong2 ones = make_ulonglong2(~0ull, ~0ull);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
         i += (uint64_t)gridDim.x * blockDim.x)
        p2[i] = ones;
    if ((npix & 1) && blockIdx.x == 0 && threadIdx.x == 0) vp.vis[npix - 1] = ~0ull;
}

// ---- k_cull: Sec. 3.2 culling and Sec. 3.3 precision ----------------------------

// Row r of the clip transform at a position: ((m[r] x + m[r+4] y) + m[r+8] z) + m[r+12].
__device__ __forceinline__ float clip_row(const float* m, int r, float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[r], x), __fmul_rn(m[r + 4], y)),
                               __fmul_rn(m[r + 8], z)),
                     m[r + 12]);
}

// Unfloored pixel coordinate from a clip coordinate: ((c / w) * 0.5 + 0.5) * W.
__device__ __forceinline__ float to_pixel(float c, float w, float W) {
    return __fmul_rn(__fadd_rn(__fmul_rn(__fdiv_rn(c, w), 0.5f), 0.5f), W);
}

// Sec. 3.3: smallest k whose cells are below the threshold, from the extent
// of the 8 projected box corners; 3 when a corner is not in front of the eye.
__device__ int select_k(const pc_batch& b, const ViewParams& v, float T) {
    const uint32_t fk = (v.flags & PC_VIEW_K_MASK) >> 4;
    if (fk >= 1) return (int)fk;
    float hi[3];
    for (int a = 0; a < 3; ++a) hi[a] = __fadd_rn(b.min[a], b.size[a]);
    float fmin0 = 0.f, fmax0 = 0.f, fmin1 = 0.f, fmax1 = 0.f;
    const float W = (float)v.width, H = (float)v.height;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        float x = (c & 1) ? hi[0] : b.min[0];
        float y = (c & 2) ? hi[1] : b.min[1];
        float z = (c & 4) ? hi[2] : b.min[2];
        float cw = clip_row(v.m, 3, x, y, z);
        if (!(cw > 0.0f)) return 3;
        float f0 = to_pixel(clip_row(v.m, 0, x, y, z), cw, W);
        float f1 = to_pixel(clip_row(v.m, 1, x, y, z), cw, H);
        if (c == 0 || f0 < fmin0) fmin0 = f0;
        if (c == 0 || f0 > fmax0) fmax0 = f0;
        if (c == 0 || f1 < fmin1) fmin1 = f1;
        if (c == 0 || f1 > fmax1) fmax1 = f1;
    }
    const float ex = __fsub_rn(fmax0, fmin0), ey = __fsub_rn(fmax1, fmin1);
    if (ex < T && ey < T) return 1;
    const float T2 = __fmul_rn(T, 1024.0f);
    if (ex < T2 && ey < T2) return 2;
    return 3;
}

// Conservative culling: the batch is dropped only if, for one clip plane, a
// rigorous bound on the binary32 rounding of every decoded point's clip
// coordinates (6u times the magnitude of the terms, u = 2^-24; decoded points
// lie in [min, fl(min + size)]) proves that every point is rejected. Evaluated
// in binary64.
__device__ __forceinline__ double row_max(const double r[4], const double lo[3], const double hi[3]) {
    double s = r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s = __dadd_rn(s, fmax(__dmul_rn(r[a], lo[a]), __dmul_rn(r[a], hi[a])));
    return s;
}
__device__ __forceinline__ double row_min(const double r[4], const double lo[3], const double hi[3]) {
    double s = r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s = __dadd_rn(s, fmin(__dmul_rn(r[a], lo[a]), __dmul_rn(r[a], hi[a])));
    return s;
}
__device__ __forceinline__ double row_mag(const double r[4], const double lo[3], const double hi[3]) {
    double s = fabs(r[3]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        s = __dadd_rn(s, __dmul_rn(fabs(r[a]), fmax(fabs(lo[a]), fabs(hi[a]))));
    return s;
}

__device__ bool cull_batch(const pc_batch& b, const ViewParams& v) {
    const double g = 6.0 * 0x1.0p-24;
    const double e1 = 1.0 + 0x1.0p-10;
    double lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)b.min[a];
        hi[a] = (double)__fadd_rn(b.min[a], b.size[a]);
    }
    const float* m = v.m;
    const double X[4] = {m[0], m[4], m[8], m[12]};
    const double Y[4] = {m[1], m[5], m[9], m[13]};
    const double Wr[4] = {m[3], m[7], m[11], m[15]};
    const double bx = row_mag(X, lo, hi), by = row_mag(Y, lo, hi), bw = row_mag(Wr, lo, hi);
    if (!isfinite(bx) || !isfinite(by) || !isfinite(bw)) return false;
    if (__dadd_rn(row_max(Wr, lo, hi), __dmul_rn(g, bw)) <= 0.0) return true;
    double sp[4], sm[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        sp[a] = __dadd_rn(X[a], __dmul_rn(e1, Wr[a]));
        sm[a] = __dsub_rn(X[a], __dmul_rn(e1, Wr[a]));
    }
    const double mx = __dmul_rn(g, __dadd_rn(bx, __dmul_rn(e1, bw)));
    if (__dadd_rn(row_max(sp, lo, hi), mx) < 0.0) return true;
    if (__dsub_rn(row_min(sm, lo, hi), mx) > 0.0) return true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        sp[a] = __dadd_rn(Y[a], __dmul_rn(e1, Wr[a]));
        sm[a] = __dsub_rn(Y[a], __dmul_rn(e1, Wr[a]));
    }
    const double my = __dmul_rn(g, __dadd_rn(by, __dmul_rn(e1, bw)));
    if (__dadd_rn(row_max(sp, lo, hi), my) < 0.0) return true;
    if (__dsub_rn(row_min(sm, lo, hi), my) > 0.0) return true;
    return false;
}

constexpr int kCullThreads = 128;

__global__ void __launch_bounds__(kCullThreads) k_cull(CloudView c, ViewTable vt, uint32_t view_base,
                                                     Scratch s) {
    __shared__ unsigned long long sh_stats[kMaxViewsPerLaunch * S_COUNT];
    __shared__ unsigned long long sh_words;
    for (uint32_t i = threadIdx.x; i < vt.n * S_COUNT; i += blockDim.x) sh_stats[i] = 0ull;
    if (threadIdx.x == 0) sh_words = 0ull;
    __syncthreads();

    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t mask = 0, nseg = 0, count = 0;
    uint64_t kcodes = 0;
    if (b < c.n_batches) {
        const pc_batch bt = c.batches[b];
        count = bt.count;
        if ((uint64_t)bt.first + bt.count > c.n_points) {
            raise_error(s, E_BATCH_RANGE, b);
            count = 0;
        }
        for (uint32_t v = 0; v < vt.n && count; ++v) {
            const ViewParams& vp = vt.v[v];
            if ((vp.flags & PC_VIEW_CULL) && cull_batch(bt, vp)) continue;
            const int k = select_k(bt, vp, vt.threshold_px);
            mask |= 1u << v;
            kcodes |= (uint64_t)k << (2 * v);
            atomicAdd(&sh_stats[v * S_COUNT + S_BATCHES], 1ull);
            atomicAdd(&sh_stats[v * S_COUNT + S_BK1 + (k - 1)], 1ull);
            atomicAdd(&sh_stats[v * S_COUNT + S_PK1 + (k - 1)], (unsigned long long)count);
        }
        if (mask) {
            nseg = (count + kSegmentPoints - 1) / kSegmentPoints;
            uint32_t kl = 0;
            for (uint32_t v = 0; v < vt.n; ++v) kl = max(kl, (uint32_t)((kcodes >> (2 * v)) & 3u));
            atomicAdd(&sh_words, (unsigned long long)kl * count);
        }
    }
    // warp-aggregated append of nseg entries
    const uint32_t lane = threadIdx.x & 31;
    uint32_t incl = nseg;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= (uint32_t)d) incl += t;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(&s.counters[C_ENTRIES], total);
    base = __shfl_sync(FULL, base, 31);
    uint64_t pos = (uint64_t)base + incl - nseg;
    for (uint32_t g = 0; g < nseg; ++g, ++pos) {
        if (pos >= s.capacity) {
            raise_error(s, E_ENTRY_RANGE, (uint32_t)pos);
            break;
        }
        DrawEntry e;
        e.kcodes = kcodes;
        e.view_mask = mask;
        e.batch = b;
        e.seg_first = g * kSegmentPoints;
        e.seg_count = min(kSegmentPoints, count - g * kSegmentPoints);
        s.entries[pos] = e;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < vt.n * S_COUNT; i += blockDim.x) {
        unsigned long long x = sh_stats[i];
        if (i % S_COUNT == S_WORDS) x = sh_words;   // the whole launch group's word loads
        if (x) atomicAdd(&s.stats[(uint64_t)view_base * S_COUNT + i], x);
    }
}

// ---- k_raster -------------------------------------------------------------------

// float(u) for u < 2^23, exactly: the bits of 2^23 + u minus 2^23.
__device__ __forceinline__ float small_u2f(uint32_t u) {
    return __fsub_rn(__uint_as_float(0x4B000000u | u), 8388608.0f);
}

// Coordinates of one point at precision k from its words (Sec. 3.3).
template <int K>
__device__ __forceinline__ void decode_q(uint32_t a, uint32_t b, uint32_t c, uint32_t& qx,
                                         uint32_t& qy, uint32_t& qz) {
    if (K == 1) {
        qx = a & 1023u;
        qy = (a >> 10) & 1023u;
        qz = (a >> 20) & 1023u;
    } else if (K == 2) {
        qx = ((a & 1023u) << 10) | (b & 1023u);
        qy = (((a >> 10) & 1023u) << 10) | ((b >> 10) & 1023u);
        qz = (((a >> 20) & 1023u) << 10) | ((b >> 20) & 1023u);
    } else {
        qx = ((a & 1023u) << 20) | ((b & 1023u) << 10) | (c & 1023u);
        qy = (((a >> 10) & 1023u) << 20) | (((b >> 10) & 1023u) << 10) | ((c >> 10) & 1023u);
        qz = (((a >> 20) & 1023u) << 20) | (((b >> 20) & 1023u) << 10) | ((c >> 20) & 1023u);
    }
}

template <int K>
__device__ __forceinline__ float q2f(uint32_t q) {
    if (K <= 2) return small_u2f(q);   // q < 2^20: exact
    return __uint2float_rn(q);         // q < 2^30: rounded to nearest, as (float)q
}

struct Decoder {
    float mn[3], cell[3];
};

__device__ __forceinline__ Decoder make_decoder(const pc_batch& b, int k) {
    Decoder d;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.mn[a] = b.min[a];
        d.cell[a] = ldexpf(b.size[a], -10 * k);   // exact power-of-two scaling
    }
    return d;
}

// Listing 1 for one decoded point and one view: project, test, early depth,
// atomicMin of (bits(w) << 32 | idx).
__device__ __forceinline__ void raster_point(float x, float y, float z, uint32_t idx,
                                             const ViewParams& v, bool early) {
    const float* m = v.m;
    const float cx = clip_row(m, 0, x, y, z);
    const float cy = clip_row(m, 1, x, y, z);
    const float cw = clip_row(m, 3, x, y, z);
    if (!(cw > 0.0f)) return;
    // ((c / w) * 0.5 + 0.5) * W: c/w * 0.5 is exact (or below 2^-126, where the
    // sum rounds to 0.5 either way), so one fused multiply-add gives the same
    // value as the separate multiply and add.
    const float fx = __fmul_rn(__fmaf_rn(__fdiv_rn(cx, cw), 0.5f, 0.5f), (float)v.width);
    const float fy = __fmul_rn(__fmaf_rn(__fdiv_rn(cy, cw), 0.5f, 0.5f), (float)v.height);
    // floor and range test in one: for 0 <= f < 2^23, 2^23 + f rounded down is
    // 2^23 + floor(f); every other f (negative, >= 2^23, inf, NaN) maps to an
    // integer outside [0, 2^23) after subtracting the bits of 2^23.
    const int px = __float_as_int(__fadd_rd(fx, 8388608.0f)) - 0x4B000000;
    const int py = __float_as_int(__fadd_rd(fy, 8388608.0f)) - 0x4B000000;
    if ((uint32_t)px >= v.width || (uint32_t)py >= v.height) return;
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(cw) << 32) | (unsigned long long)idx;
    unsigned long long* addr =
        reinterpret_cast<unsigned long long*>(v.vis) + ((size_t)py * v.width + (uint32_t)px);
    if (early) {
        // a stale read is larger than or equal to the current value, so it
        // can only cause an unnecessary atomic, never a missed one
        if (key < *addr) atomicMin(addr, key);
    } else {
        atomicMin(addr, key);
    }
}

__device__ __forceinline__ uint4 ld_stream(const uint32_t* p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t pick(const uint4& q, int j) {
    return j == 0 ? q.x : j == 1 ? q.y : j == 2 ? q.z : q.w;
}

// Process the aligned groups of 4 points of [p0, p1) for the views of mask at
// precision KL words loaded; each view decodes with its own k <= KL.
template <int KL>
__device__ __forceinline__ void raster_segment(const CloudView& c, const ViewTable& vt,
                                               const pc_batch& bt, uint64_t p0, uint64_t p1,
                                               uint32_t mask, uint64_t kcodes, uint32_t lane) {
    const uint64_t a0 = p0 & ~3ull;
    for (uint64_t g = a0 + 4ull * lane; g < p1; g += 128ull) {
        uint4 q1 = ld_stream(c.w1 + g);
        uint4 q2 = make_uint4(0, 0, 0, 0), q3 = make_uint4(0, 0, 0, 0);
        if (KL >= 2) q2 = ld_stream(c.w2 + g);
        if (KL >= 3) q3 = ld_stream(c.w3 + g);
        uint32_t mm = mask;
        while (mm) {
            const uint32_t v = __ffs(mm) - 1;
            mm &= mm - 1;
            const ViewParams& vp = vt.v[v];
            const int k = (int)((kcodes >> (2 * v)) & 3u);
            const Decoder d = make_decoder(bt, k);
            const bool early = !(vp.flags & PC_VIEW_NO_EARLY_DEPTH);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t i = g + j;
                if (i < p0 || i >= p1) continue;
                uint32_t qx, qy, qz;
                float fx, fy, fz;
                const uint32_t a = pick(q1, j), b = pick(q2, j), cc = pick(q3, j);
                if (k == 1) {
                    decode_q<1>(a, b, cc, qx, qy, qz);
                    fx = q2f<1>(qx); fy = q2f<1>(qy); fz = q2f<1>(qz);
                } else if (k == 2) {
                    decode_q<2>(a, b, cc, qx, qy, qz);
                    fx = q2f<2>(qx); fy = q2f<2>(qy); fz = q2f<2>(qz);
                } else {
                    decode_q<3>(a, b, cc, qx, qy, qz);
                    fx = q2f<3>(qx); fy = q2f<3>(qy); fz = q2f<3>(qz);
                }
                const float x = __fadd_rn(d.mn[0], __fmul_rn(fx, d.cell[0]));
                const float y = __fadd_rn(d.mn[1], __fmul_rn(fy, d.cell[1]));
                const float z = __fadd_rn(d.mn[2], __fmul_rn(fz, d.cell[2]));
                raster_point(x, y, z, (uint32_t)i, vp, early);
            }
        }
    }
}

// Single view at precision K: the common case, with everything warp-uniform.
template <int K>
__device__ __forceinline__ void raster_segment_1view(const CloudView& c, const ViewParams& vp,
                                                     const pc_batch& bt, uint64_t p0,
                                                     uint64_t p1, uint32_t lane) {
    const Decoder d = make_decoder(bt, K);
    const bool early = !(vp.flags & PC_VIEW_NO_EARLY_DEPTH);
    const uint64_t a0 = p0 & ~3ull;
    for (uint64_t g = a0 + 4ull * lane; g < p1; g += 128ull) {
        uint4 q1 = ld_stream(c.w1 + g);
        uint4 q2 = make_uint4(0, 0, 0, 0), q3 = make_uint4(0, 0, 0, 0);
        if (K >= 2) q2 = ld_stream(c.w2 + g);
        if (K >= 3) q3 = ld_stream(c.w3 + g);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t i = g + j;
            if (i < p0 || i >= p1) continue;
            uint32_t qx, qy, qz;
            decode_q<K>(pick(q1, j), pick(q2, j), pick(q3, j), qx, qy, qz);
            const float x = __fadd_rn(d.mn[0], __fmul_rn(q2f<K>(qx), d.cell[0]));
            const float y = __fadd_rn(d.mn[1], __fmul_rn(q2f<K>(qy), d.cell[1]));
            const float z = __fadd_rn(d.mn[2], __fmul_rn(q2f<K>(qz), d.cell[2]));
            raster_point(x, y, z, (uint32_t)i, vp, early);
        }
    }
}

constexpr int kRasterThreads = 256;

__global__ void __launch_bounds__(kRasterThreads) k_raster(CloudView c, ViewTable vt, Scratch s) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_entries = s.counters[C_ENTRIES];
    for (;;) {
        uint32_t e_idx = 0;
        if (lane == 0) e_idx = atomicAdd(&s.counters[C_GRAB], 1u);
        e_idx = __shfl_sync(FULL, e_idx, 0);
        if (e_idx >= n_entries || e_idx >= s.capacity) break;
        const DrawEntry e = s.entries[e_idx];
        if (e.batch >= c.n_batches) {
            if (lane == 0) raise_error(s, E_BATCH_RANGE, e.batch);
            continue;
        }
        const pc_batch bt = c.batches[e.batch];
        const uint64_t p0 = (uint64_t)bt.first + e.seg_first;
        const uint64_t p1 = p0 + e.seg_count;
        uint32_t kl = 0;
        for (uint32_t mm = e.view_mask; mm; mm &= mm - 1) {
            const uint32_t v = __ffs(mm) - 1;
            kl = max(kl, (uint32_t)((e.kcodes >> (2 * v)) & 3u));
        }
        if (e.view_mask == 1u) {
            const ViewParams& vp = vt.v[0];
            if (kl == 1) raster_segment_1view<1>(c, vp, bt, p0, p1, lane);
            else if (kl == 2) raster_segment_1view<2>(c, vp, bt, p0, p1, lane);
            else raster_segment_1view<3>(c, vp, bt, p0, p1, lane);
        } else {
            if (kl == 1) raster_segment<1>(c, vt, bt, p0, p1, e.view_mask, e.kcodes, lane);
            else if (kl == 2) raster_segment<2>(c, vt, bt, p0, p1, e.view_mask, e.kcodes, lane);
            else raster_segment<3>(c, vt, bt, p0, p1, e.view_mask, e.kcodes, lane);
        }
    }
}

// ---- k_resolve ---------------------------------------------------------------------

__global__ void k_resolve(CloudView c, ViewTable vt, Scratch s) {
    const uint32_t v = blockIdx.y;
    if (v >= vt.n) return;
    const ViewParams& vp = vt.v[v];
    if (!vp.rgba) return;
    const uint64_t npix = (uint64_t)vp.width * vp.height;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = vp.vis[p];
        uint32_t out = 0u;
        if (key != ~0ull) {
            const uint32_t idx = (uint32_t)key;
            if (idx < c.n_points) out = c.color[idx];
            else raise_error(s, E_INDEX_RANGE, idx);
        }
        vp.rgba[p] = out;
    }
}

int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

}  // namespace

cudaError_t launch_clear(const ViewTable& vt, uint32_t view_base, Scratch s, cudaStream_t st) {
    uint64_t maxpix = 0;
    for (uint32_t v = 0; v < vt.n; ++v)
        maxpix = max(maxpix, (uint64_t)vt.v[v].width * vt.v[v].height);
    const int threads = 256;
    uint64_t blocks = (maxpix / 2 + threads - 1) / threads;
    blocks = blocks < 1 ? 1 : (blocks > (uint64_t)num_sms() * 8 ? (uint64_t)num_sms() * 8 : blocks);
    dim3 grid((unsigned)blocks, vt.n ? vt.n : 1);
    k_clear<<<grid, threads, 0, st>>>(vt, view_base, s);
    return cudaGetLastError();
}

cudaError_t launch_cull(const CloudView& c, const ViewTable& vt, uint32_t view_base, Scratch s,
                        cudaStream_t st) {
    const unsigned blocks = (c.n_batches + kCullThreads - 1) / kCullThreads;
    if (blocks == 0) return cudaSuccess;
    k_cull<<<blocks, kCullThreads, 0, st>>>(c, vt, view_base, s);
    return cudaGetLastError();
}

int raster_occupancy(int threads_per_block) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_raster, threads_per_block, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_raster(const CloudView& c, const ViewTable& vt, Scratch s, RasterShape shape,
                          cudaStream_t st) {
    int threads = shape.threads_per_block > 0 ? shape.threads_per_block : kRasterThreads;
    if (threads > kRasterThreads) threads = kRasterThreads;
    int blocks = shape.blocks > 0 ? shape.blocks : num_sms() * raster_occupancy(threads);
    k_raster<<<blocks, threads, 0, st>>>(c, vt, s);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const CloudView& c, const ViewTable& vt, Scratch s, cudaStream_t st) {
    uint64_t maxpix = 0;
    for (uint32_t v = 0; v < vt.n; ++v)
        maxpix = max(maxpix, (uint64_t)vt.v[v].width * vt.v[v].height);
    const int threads = 256;
    uint64_t blocks = (maxpix + threads - 1) / threads;
    blocks = blocks < 1 ? 1 : (blocks > (uint64_t)num_sms() * 8 ? (uint64_t)num_sms() * 8 : blocks);
    dim3 grid((unsigned)blocks, vt.n ? vt.n : 1);
    k_resolve<<<grid, threads, 0, st>>>(c, vt, s);
    return cudaGetLastError();
}

}  // namespace pcr

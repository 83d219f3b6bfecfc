// raster.cu — sm_103a kernels of the point rasterizer.
//
//   k_clear     visibility buffers <- all ones (and shading sums <- 0); scratch
//               counters <- 0
//   k_lod_pass  LOD clouds: per node and view, frustum, projected extent and
//               (foveated) threshold (Sec. 3.5, 3.7)
//   k_cull      per batch and view: conservative frustum culling (Sec. 3.2) and
//               the precision k from the projected batch extent (Sec. 3.3);
//               surviving batches are appended, in segments, to a draw list
//   k_raster    persistent warps take draw-list segments, load the k coordinate
//               words of 4 consecutive points with one 16-byte load per word
//               (Sec. 3.4), decode, project (Listing 1), do the non-atomic
//               early-depth test and atomicMin the 64-bit key; one pass serves
//               every view of the launch (Sec. 3.7)
//   k_shade     high-quality shading (Sec. 3.6): the colour pass over the same
//               draw list, summing the colours of the points within 1% of their
//               pixel's closest depth
//   k_resolve   visibility key -> colour of the winning point (Sec. 3.3), the
//               average of the sums (Sec. 3.6), depth-aware dilation (Sec. 3.7)
//
// Bit-exactness: every float operation that decides a key or a pixel is an
// explicit round-to-nearest intrinsic in the same order as the CPU oracle's
// definition (decode x = min + float(X) * cell; c = ((m0 x + m4 y) + m8 z) +
// m12; f = ((c / w) * 0.5 + 0.5) * W with an IEEE divide), or a packed f32x2
// instruction that rounds each half the same way. The file is also compiled
// with --fmad=false so nothing else is contracted.
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
    const unsigned long long empty = empty_key(vp.flags);
    const ulonglong2 ones = make_ulonglong2(empty, empty);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
         i += (uint64_t)gridDim.x * blockDim.x)
        p2[i] = ones;
    if ((npix & 1) && blockIdx.x == 0 && threadIdx.x == 0) vp.vis[npix - 1] = empty;
    if (vp.accum) {
        // high-quality shading sums <- 0; each view's region is a whole number
        // of 16-byte words
        ulonglong2* a2 = reinterpret_cast<ulonglong2*>(vp.accum);
        const uint64_t na = (hqs_clear_words(vp.flags, npix) + 1) / 2;
        const ulonglong2 zero = make_ulonglong2(0ull, 0ull);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na;
             i += (uint64_t)gridDim.x * blockDim.x)
            a2[i] = zero;
    }
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

// Spread of the 8 projected box corners' unfloored pixel coordinates, with
// the same binary32 operations as a point; false when a corner has w <= 0.
__device__ bool corner_box(const pc_batch& b, const ViewParams& v, float& fmin0, float& fmax0,
                           float& fmin1, float& fmax1) {
    float hi[3];
    for (int a = 0; a < 3; ++a) hi[a] = __fadd_rn(b.min[a], b.size[a]);
    fmin0 = fmax0 = fmin1 = fmax1 = 0.f;
    const float W = (float)v.width, H = (float)v.height;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        float x = (c & 1) ? hi[0] : b.min[0];
        float y = (c & 2) ? hi[1] : b.min[1];
        float z = (c & 4) ? hi[2] : b.min[2];
        float cw = clip_row(v.m, 3, x, y, z);
        if (!(cw > 0.0f)) return false;
        float f0 = to_pixel(clip_row(v.m, 0, x, y, z), cw, W);
        float f1 = to_pixel(clip_row(v.m, 1, x, y, z), cw, H);
        if (c == 0 || f0 < fmin0) fmin0 = f0;
        if (c == 0 || f0 > fmax0) fmax0 = f0;
        if (c == 0 || f1 < fmin1) fmin1 = f1;
        if (c == 0 || f1 > fmax1) fmax1 = f1;
    }
    return true;
}

__device__ bool corner_extent(const pc_batch& b, const ViewParams& v, float& ex, float& ey) {
    float fmin0, fmax0, fmin1, fmax1;
    if (!corner_box(b, v, fmin0, fmax0, fmin1, fmax1)) return false;
    ex = __fsub_rn(fmax0, fmin0);
    ey = __fsub_rn(fmax1, fmin1);
    return true;
}

// Sec. 3.7 rings of a screen position: 0 within a third of the half-diagonal
// from the view centre, 1 within two thirds, else 2 (binary32, fixed order).
__device__ __forceinline__ int ring_of(float x, float y, uint32_t width, uint32_t height) {
    const float hw = __fmul_rn((float)width, 0.5f), hh = __fmul_rn((float)height, 0.5f);
    const float dx = __fsub_rn(x, hw), dy = __fsub_rn(y, hh);
    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    const float r2 = __fadd_rn(__fmul_rn(hw, hw), __fmul_rn(hh, hh));
    const float d9 = __fmul_rn(9.0f, d2);
    if (d9 < r2) return 0;
    if (d9 < __fmul_rn(4.0f, r2)) return 1;
    return 2;
}

// Sec. 3.3: smallest k whose cells are below the threshold, from the extent
// of the 8 projected box corners; 3 when a corner is not in front of the eye.
__device__ int select_k(const pc_batch& b, const ViewParams& v, float T) {
    const uint32_t fk = (v.flags & PC_VIEW_K_MASK) >> 4;
    if (fk >= 1) return (int)fk;
    float ex, ey;
    if (!corner_extent(b, v, ex, ey)) return 3;
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

__device__ bool cull_batch_exact(const pc_batch& b, const ViewParams& v) {
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

// The same five tests in binary32 first. Each test value t approximates the
// exact value R of its expression within about 10 * 2^-24 of the magnitude M
// of its terms, and the binary64 value within about 10 * 2^-53 M, so when
// |t| > 2^-16 M both have the sign of R and the decision equals the binary64
// one. Inside that band, or when a magnitude is not finite or below 2^-90
// (where products could lose bits to underflow), the binary64 code decides.
// Returns 1 culled, 0 not culled, -1 undecided.
__device__ __forceinline__ float row_max32(const float r[4], const float lo[3], const float hi[3]) {
    float s = r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s = __fadd_rn(s, fmaxf(__fmul_rn(r[a], lo[a]), __fmul_rn(r[a], hi[a])));
    return s;
}
__device__ __forceinline__ float row_min32(const float r[4], const float lo[3], const float hi[3]) {
    float s = r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s = __fadd_rn(s, fminf(__fmul_rn(r[a], lo[a]), __fmul_rn(r[a], hi[a])));
    return s;
}
__device__ __forceinline__ float row_mag32(const float r[4], const float lo[3], const float hi[3]) {
    float s = fabsf(r[3]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        s = __fadd_rn(s, __fmul_rn(fabsf(r[a]), fmaxf(fabsf(lo[a]), fabsf(hi[a]))));
    return s;
}

__device__ __forceinline__ int cull_batch_fast(const pc_batch& b, const ViewParams& v) {
    const float g = 6.0f * 0x1.0p-24f;
    const float e1 = 1.0f + 0x1.0p-10f;
    const float band = 0x1.0p-16f;
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = b.min[a];
        hi[a] = __fadd_rn(b.min[a], b.size[a]);
    }
    const float* m = v.m;
    const float X[4] = {m[0], m[4], m[8], m[12]};
    const float Y[4] = {m[1], m[5], m[9], m[13]};
    const float Wr[4] = {m[3], m[7], m[11], m[15]};
    const float bx = row_mag32(X, lo, hi), by = row_mag32(Y, lo, hi), bw = row_mag32(Wr, lo, hi);
    const float mag_x = __fadd_rn(bx, __fmul_rn(e1, bw)), mag_y = __fadd_rn(by, __fmul_rn(e1, bw));
    if (!(bw <= 0x1.0p100f) || !(mag_x <= 0x1.0p100f) || !(mag_y <= 0x1.0p100f)) return -1;
    if (!(bw >= 0x1.0p-90f) || !(mag_x >= 0x1.0p-90f) || !(mag_y >= 0x1.0p-90f)) return -1;
    // each test: culled when t < 0 (t <= 0 for the w plane), decided when |t| > band M
    bool undecided = false, culled = false;
    auto test = [&](float t, float mag) {
        const float lim = __fmul_rn(band, mag);
        if (t < -lim) culled = true;
        else if (!(t > lim)) undecided = true;
    };
    test(__fadd_rn(row_max32(Wr, lo, hi), __fmul_rn(g, bw)), bw);
    float sp[4], sm[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        sp[a] = __fadd_rn(X[a], __fmul_rn(e1, Wr[a]));
        sm[a] = __fsub_rn(X[a], __fmul_rn(e1, Wr[a]));
    }
    const float mx = __fmul_rn(g, mag_x);
    test(__fadd_rn(row_max32(sp, lo, hi), mx), mag_x);
    test(-__fsub_rn(row_min32(sm, lo, hi), mx), mag_x);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        sp[a] = __fadd_rn(Y[a], __fmul_rn(e1, Wr[a]));
        sm[a] = __fsub_rn(Y[a], __fmul_rn(e1, Wr[a]));
    }
    const float my = __fmul_rn(g, mag_y);
    test(__fadd_rn(row_max32(sp, lo, hi), my), mag_y);
    test(-__fsub_rn(row_min32(sm, lo, hi), my), mag_y);
    // a test decided as culling settles it; otherwise every test must be decided
    if (culled) return 1;
    return undecided ? -1 : 0;
}

__device__ __forceinline__ bool cull_batch(const pc_batch& b, const ViewParams& v) {
    const int r = cull_batch_fast(b, v);
    return r < 0 ? cull_batch_exact(b, v) : r == 1;
}

// Certificate of the raster kernel's fast path for one batch and view. True
// only if, for every point the batch can decode to (all lie in
// [min, fl(min + size)]), (1) the binary32 clip w lies in [2^-99, 2^99], so the
// point is in front of the eye and the reciprocal estimate stays normal,
// (2) c / w lies in [-1, 1 - 2^-20] on both axes, so the definition's floor
// pixel is inside the view, and (3) every size is at most 2^100, so that the
// decode constants 2^23 cell and 2^13 cell are exact. False is always safe: the
// batch then takes the general path with per-point tests.
//
// Bounds in binary32: each row's exact range over the box, widened by 32u times
// the magnitude of its terms (u = 2^-24). That covers the point's own rounding
// (at most 6u of the magnitude, as for culling) plus the rounding of these
// bounds (about 6u more), and 2^-120 covers underflow. The quotient bounds take
// the interval endpoints (w > 0) and must clear the limits by 2^-12, far more
// than the binary32 rounding of the bound itself.
__device__ bool batch_fast(const pc_batch& b, const ViewParams& v) {
    if (v.flags & PC_VIEW_NO_EARLY_DEPTH) return false;
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(b.size[a] <= 0x1.0p100f)) return false;   // also NaN and infinities
        lo[a] = b.min[a];
        hi[a] = __fadd_rn(b.min[a], b.size[a]);
    }
    const float* m = v.m;
    const float X[4] = {m[0], m[4], m[8], m[12]};
    const float Y[4] = {m[1], m[5], m[9], m[13]};
    const float Wr[4] = {m[3], m[7], m[11], m[15]};
    const float g = 32.0f * 0x1.0p-24f, tiny = 0x1.0p-120f;
    const float mw = __fadd_rn(__fmul_rn(g, row_mag32(Wr, lo, hi)), tiny);
    const float wl = __fsub_rn(row_min32(Wr, lo, hi), mw);
    const float wh = __fadd_rn(row_max32(Wr, lo, hi), mw);
    if (!(wl >= 0x1.0p-99f) || !(wh <= 0x1.0p99f)) return false;
    const float lim_lo = -1.0f + 0x1.0p-12f, lim_hi = 1.0f - 0x1.0p-12f;
    const float* rows[2] = {X, Y};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float mr = __fadd_rn(__fmul_rn(g, row_mag32(rows[r], lo, hi)), tiny);
        const float cl = __fsub_rn(row_min32(rows[r], lo, hi), mr);
        const float ch = __fadd_rn(row_max32(rows[r], lo, hi), mr);
        const float qmin = cl >= 0.0f ? __fdiv_rn(cl, wh) : __fdiv_rn(cl, wl);
        const float qmax = ch >= 0.0f ? __fdiv_rn(ch, wl) : __fdiv_rn(ch, wh);
        if (!(qmin >= lim_lo) || !(qmax <= lim_hi)) return false;
    }
    return true;
}

constexpr int kCullThreads = 128;

// Sum of a 64-bit value over the 32 lanes of a warp (butterfly on 32-bit
// halves with the carry).
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const uint32_t ol = __shfl_xor_sync(FULL, lo, d), oh = __shfl_xor_sync(FULL, hi, d);
        const uint32_t nl = lo + ol;
        hi = hi + oh + (nl < lo ? 1u : 0u);
        lo = nl;
    }
    return ((unsigned long long)hi << 32) | lo;
}

// Sec. 3.5: a node passes a view when it is in the frustum and, unless it is
// the root, its projected extent reaches the view's threshold (a corner with
// w <= 0 counts as large). lod_sel[n] gets one bit per view of the launch.
__global__ void __launch_bounds__(kCullThreads) k_lod_pass(CloudView c, ViewTable vt, Scratch s) {
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= c.n_batches) return;
    const pc_batch bt = c.batches[n];
    uint32_t mask = 0;
    for (uint32_t v = 0; v < vt.n; ++v) {
        const ViewParams& vp = vt.v[v];
        if (cull_batch(bt, vp)) continue;
        if (n > 0) {
            float fmin0, fmax0, fmin1, fmax1;
            if (corner_box(bt, vp, fmin0, fmax0, fmin1, fmax1)) {
                const float ex = __fsub_rn(fmax0, fmin0), ey = __fsub_rn(fmax1, fmin1);
                const float e = (ex != ex || ey != ey) ? __fadd_rn(ex, ey) : fmaxf(ex, ey);
                float t = vp.lod_px;
                if (vp.lod_px_periphery > 0.0f) {
                    const float cx = __fmul_rn(__fadd_rn(fmin0, fmax0), 0.5f);
                    const float cy = __fmul_rn(__fadd_rn(fmin1, fmax1), 0.5f);
                    const int r = ring_of(cx, cy, vp.width, vp.height);
                    if (r == 1) t = __fmul_rn(__fadd_rn(vp.lod_px, vp.lod_px_periphery), 0.5f);
                    if (r == 2) t = vp.lod_px_periphery;
                }
                if (e < t) continue;
            }
        }
        mask |= 1u << v;
    }
    s.lod_sel[n] = mask;
}

__global__ void __launch_bounds__(kCullThreads) k_cull(CloudView c, ViewTable vt, uint32_t view_base,
                                                     Scratch s) {
    __shared__ unsigned long long sh_stats[kMaxViewsPerLaunch * S_COUNT];
    __shared__ unsigned long long sh_words;
    for (uint32_t i = threadIdx.x; i < vt.n * S_COUNT; i += blockDim.x) sh_stats[i] = 0ull;
    if (threadIdx.x == 0) sh_words = 0ull;
    __syncthreads();

    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t mask = 0, fmask = 0, nseg = 0, count = 0;
    uint64_t kcodes = 0;
    if (b < c.n_batches) {
        const pc_batch bt = c.batches[b];
        count = bt.count;
        if ((uint64_t)bt.first + bt.count > c.n_points) {
            raise_error(s, E_BATCH_RANGE, b);
            count = 0;
        }
        uint32_t lod_mask = ~0u;
        if (c.is_lod) {
            // drawn when this node and every ancestor passed (parents come
            // first in breadth-first order; the root is its own parent)
            lod_mask = s.lod_sel[b];
            uint32_t node = b;
            for (int depth = 0; depth < 64 && lod_mask; ++depth) {
                const uint32_t par = c.parent[node];
                if (par == node || par >= c.n_batches) break;
                lod_mask &= s.lod_sel[par];
                node = par;
            }
        }
        for (uint32_t v = 0; v < vt.n && count; ++v) {
            const ViewParams& vp = vt.v[v];
            if (c.is_lod) {
                if (!((lod_mask >> v) & 1u)) continue;
            } else if ((vp.flags & PC_VIEW_CULL) && cull_batch(bt, vp)) {
                continue;
            }
            const int k = select_k(bt, vp, vt.threshold_px);
            mask |= 1u << v;
            kcodes |= (uint64_t)k << (2 * v);
            if (k <= 2 && batch_fast(bt, vp)) fmask |= 1u << v;
        }
        if (mask) nseg = (count + vt.seg_points - 1) / vt.seg_points;
    }
    const uint32_t lane = threadIdx.x & 31;
    // statistics, summed over the warp first: one shared-memory addition per
    // warp and counter (64-bit shared atomics contend badly lane by lane)
    uint32_t kl = 0;
    for (uint32_t v = 0; v < vt.n; ++v) {
        const bool drawn = (mask >> v) & 1u;
        if (!__any_sync(FULL, drawn)) continue;
        const uint32_t k = (uint32_t)((kcodes >> (2 * v)) & 3u);
        if (drawn) kl = max(kl, k);
        uint32_t nb = 0;
#pragma unroll
        for (uint32_t kk = 1; kk <= 3; ++kk) {
            const bool sel = drawn && k == kk;
            const uint32_t n = __popc(__ballot_sync(FULL, sel));
            const unsigned long long pts = warp_sum_u64(sel ? count : 0u);
            nb += n;
            if (lane == 0 && n) {
                atomicAdd(&sh_stats[v * S_COUNT + S_BK1 + (kk - 1)], (unsigned long long)n);
                atomicAdd(&sh_stats[v * S_COUNT + S_PK1 + (kk - 1)], pts);
            }
        }
        if (lane == 0) atomicAdd(&sh_stats[v * S_COUNT + S_BATCHES], (unsigned long long)nb);
    }
    {
        const unsigned long long words = warp_sum_u64((unsigned long long)kl * (mask ? count : 0u));
        if (lane == 0 && words) atomicAdd(&sh_words, words);
    }
    // warp-aggregated append of nseg entries
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
        e.fast_mask = fmask;
        e.pad = 0;
        e.batch = b;
        e.seg_first = g * vt.seg_points;
        e.seg_count = min(vt.seg_points, count - g * vt.seg_points);
        s.entries[pos] = e;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < vt.n * S_COUNT; i += blockDim.x) {
        unsigned long long x = sh_stats[i];
        if (i % S_COUNT == S_WORDS) x = sh_words;   // the whole launch group's word loads
        if (x && i % S_COUNT <= S_WORDS) atomicAdd(&s.stats[(uint64_t)view_base * S_COUNT + i], x);
    }
}

// Hardware reciprocal approximation; used only for w in [2^-100, 2^100], where
// flushing subnormals cannot matter.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed binary32 pairs (sm_100 f32x2 instructions), used where two independent
// operations of the same kind sit side by side. Each half is rounded exactly as
// the scalar instruction would round it. A packed multiply never feeds a packed
// add: ptxas contracts that pair into a packed fused multiply-add, which changes
// the bits. Every add after a packed multiply is a scalar __fadd_rn.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f2_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2_t f2_fma_rn(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ f2_t f2_fma_rd(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// ---- k_raster -------------------------------------------------------------------
//
// Every lane takes an aligned group of 4 consecutive points (one 16-byte load
// per coordinate word, Sec. 3.4): it decodes and projects all four, then issues
// the early-depth reads back to back, then compares and updates. All
// arithmetic that decides a key or a pixel uses round-to-nearest intrinsics that
// are never contracted (__fmul_rn, __fadd_rn), or packed f32x2 instructions that
// no packed multiply feeds, in the oracle's order.

// Per-view constants.
struct ViewConst {
    float mx[4], my[4], mw[4];  // clip rows x, y, w: (m[r], m[r+4], m[r+8], m[r+12])
    float W, H;
    uint32_t width, height;
    unsigned long long* vis;
    bool early;
};

__device__ __forceinline__ ViewConst make_view_const(const ViewParams& v) {
    ViewConst c;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c.mx[j] = v.m[4 * j + 0];
        c.my[j] = v.m[4 * j + 1];
        c.mw[j] = v.m[4 * j + 3];
    }
    c.W = (float)v.width;
    c.H = (float)v.height;
    c.width = v.width;
    c.height = v.height;
    c.vis = reinterpret_cast<unsigned long long*>(v.vis);
    c.early = !(v.flags & PC_VIEW_NO_EARLY_DEPTH);
    return c;
}

// The clip coordinates of one point (Listing 1), each row as
// ((m[r] x + m[r+4] y) + m[r+8] z) + m[r+12]. The x and y rows' products of
// one coordinate form a packed pair ((m0 x, m1 x), ...), as do the w row's
// first two; the sums are scalar adds, except the last one of the x and y rows,
// whose operands are sums.
__device__ __forceinline__ void clip_xyw(const ViewConst& vc, float x, float y, float z, float& cx,
                                         float& cy, float& cw) {
    float a0, a1, b0, b1, c0, c1, w0, w1;
    f2_unpack(f2_mul(f2_pack(vc.mx[0], vc.my[0]), f2_pack(x, x)), a0, a1);
    f2_unpack(f2_mul(f2_pack(vc.mx[1], vc.my[1]), f2_pack(y, y)), b0, b1);
    f2_unpack(f2_mul(f2_pack(vc.mx[2], vc.my[2]), f2_pack(z, z)), c0, c1);
    f2_unpack(f2_mul(f2_pack(vc.mw[0], vc.mw[1]), f2_pack(x, y)), w0, w1);
    const float sx = __fadd_rn(__fadd_rn(a0, b0), c0);
    const float sy = __fadd_rn(__fadd_rn(a1, b1), c1);
    f2_unpack(f2_add(f2_pack(sx, sy), f2_pack(vc.mx[3], vc.my[3])), cx, cy);
    cw = __fadd_rn(__fadd_rn(__fadd_rn(w0, w1), __fmul_rn(vc.mw[2], z)), vc.mw[3]);
}

// Per-batch decode constants at precision k.
struct DecConst {
    float mn[3], cell[3];
};

__device__ __forceinline__ DecConst make_dec_const(const pc_batch& b, int k) {
    DecConst d;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.mn[a] = b.min[a];
        d.cell[a] = ldexpf(b.size[a], -10 * k);   // exact power-of-two scaling
    }
    return d;
}

// Integer coordinates of one point at precision k from its words (Sec. 3.3):
// the first k words concatenated from the most significant part down.
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

// float(q): exact for q < 2^23 through the bits of 2^23 + q minus 2^23;
// rounded to nearest for the 30-bit values of k = 3, as (float)q.
template <int K>
__device__ __forceinline__ float q_to_float(uint32_t q) {
    if (K <= 2) return __fsub_rn(__uint_as_float(0x4B000000u | q), 8388608.0f);
    return __uint2float_rn(q);
}

// Decoded position (Sec. 3.3): x = min + float(X) * cell per axis, binary32.
// float(X) and the products of x and y are formed as one packed pair each.
template <int K>
__device__ __forceinline__ void decode_point(const DecConst& d, uint32_t a, uint32_t b, uint32_t c,
                                             float& x, float& y, float& z) {
    uint32_t qx, qy, qz;
    decode_q<K>(a, b, c, qx, qy, qz);
    f2_t fxy;
    if (K <= 2)
        fxy = f2_sub(f2_pack(__uint_as_float(0x4B000000u | qx), __uint_as_float(0x4B000000u | qy)),
                     f2_pack(8388608.0f, 8388608.0f));
    else
        fxy = f2_pack(__uint2float_rn(qx), __uint2float_rn(qy));
    float sx, sy;
    f2_unpack(f2_mul(fxy, f2_pack(d.cell[0], d.cell[1])), sx, sy);
    x = __fadd_rn(d.mn[0], sx);
    y = __fadd_rn(d.mn[1], sy);
    z = __fadd_rn(d.mn[2], __fmul_rn(q_to_float<K>(qz), d.cell[2]));
}

// Floor bits of the pixel coordinate of one axis: the bits of 2^23 + f rounded
// down, f = ((c / w) * 0.5 + 0.5) * W. For 0 <= f < 2^23 they are
// 2^23 + floor(f); every other f (negative, >= 2^23, inf, NaN) lands outside
// [2^23, 2^24) and fails the range test. The map from f is monotonic.
//
// Exact path, the definition through the IEEE divide. (c/w) * 0.5 is exact,
// or below 2^-126 where the sum rounds to 0.5 either way, so the fused
// multiply-add equals the separate multiply and add.
__device__ __forceinline__ uint32_t exact_floor_bits(float c, float w, float W) {
    const float f = __fmul_rn(__fmaf_rn(__fdiv_rn(c, w), 0.5f, 0.5f), W);
    return __float_as_uint(__fadd_rd(f, 8388608.0f));
}

// Certified fast path. q' = c * r with r the reciprocal of w refined by one
// Newton step (relative error below 2^-40 + 2^-24) is within |q'| 2^-22 of the
// IEEE quotient. With eta = 2^-21, u- = fl(q' * 0.5 + (0.5 - eta)) and
// u+ = fl(q' * 0.5 + (0.5 + eta)) bracket the definition's fl(q * 0.5 + 0.5)
// with room for the roundings of both sides whenever |q'| <= 1.01, so
// fl_down(u- * W + 2^23) <= floor bits <= fl_down(u+ * W + 2^23); when the two
// ends agree they are the floor bits. Points with |q'| > 1.01 lie outside the
// viewport either way. The x and y axes run as packed pairs.

// Floor bits of both axes of one point by the certified fast path; false when
// the two ends of the bracket differ or w is outside [2^-100, 2^100] (then the
// exact path decides). Any w may be passed: nothing here can fault.
__device__ __forceinline__ bool pixel_bits_fast(float cx, float cy, float cw, float W, float H,
                                                uint32_t& bx, uint32_t& by) {
    float r = rcp_approx(cw);
    r = __fmaf_rn(r, __fmaf_rn(-cw, r, 1.0f), r);
    const f2_t half = f2_pack(0.5f, 0.5f);
    const f2_t magic = f2_pack(8388608.0f, 8388608.0f);
    const f2_t wh = f2_pack(W, H);
    const f2_t q = f2_mul(f2_pack(cx, cy), f2_pack(r, r));
    const f2_t ulo = f2_fma_rn(q, half, f2_pack(0.5f - 0x1.0p-21f, 0.5f - 0x1.0p-21f));
    const f2_t uhi = f2_fma_rn(q, half, f2_pack(0.5f + 0x1.0p-21f, 0.5f + 0x1.0p-21f));
    const f2_t blo = f2_fma_rd(ulo, wh, magic);
    const f2_t bhi = f2_fma_rd(uhi, wh, magic);
    bx = (uint32_t)blo;
    by = (uint32_t)(blo >> 32);
    return (blo == bhi) & (cw >= 0x1.0p-100f) & (cw <= 0x1.0p100f);
}

// Listing 1 for the four points of a group: project, test, then the
// early-depth reads of all four, then atomicMin of (bits(w) << 32 | index)
// where the point may be closer. The early-depth read takes only the depth
// half of the pixel's key, and a point goes on to the atomic when its depth
// bits are not above it: a tie in depth issues an atomic that atomicMin then
// settles by index. A stale read is larger than or equal to the current value,
// so it can only cause an unnecessary atomic, never a missed one. After an
// atomic, the next point of the group on the same pixel needs one only if it
// is strictly closer (its index is larger). PARTIAL groups carry a validity
// mask. Returns the number of atomicMin issued.
template <bool PARTIAL>
__device__ __forceinline__ uint32_t raster_quad(const ViewConst& vc, const float (&x)[4],
                                                const float (&y)[4], const float (&z)[4],
                                                uint32_t idx0, uint32_t valid) {
    uint32_t w[4], pix[4], bx[4], by[4];
    float cx[4], cy[4], cw[4];
    bool live[4];
    uint32_t slow = 0;   // live points whose bracket did not settle the pixel
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        clip_xyw(vc, x[j], y[j], z[j], cx[j], cy[j], cw[j]);
        live[j] = cw[j] > 0.0f;
        if (PARTIAL) live[j] = live[j] && ((valid >> j) & 1u);
        const bool ok = pixel_bits_fast(cx[j], cy[j], cw[j], vc.W, vc.H, bx[j], by[j]);
        slow |= (uint32_t)(live[j] && !ok) << j;
    }
    if (slow) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((slow >> j) & 1u) {
                bx[j] = exact_floor_bits(cx[j], cw[j], vc.W);
                by[j] = exact_floor_bits(cy[j], cw[j], vc.H);
            }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t px = bx[j] - 0x4B000000u, py = by[j] - 0x4B000000u;
        live[j] = live[j] && px < vc.width && py < vc.height;
        w[j] = __float_as_uint(cw[j]);
        pix[j] = py * vc.width + px;
    }
    // depth halves of the pixels' keys (0xFFFFFFFF: no read, always try)
    const uint32_t* vis_hi = reinterpret_cast<const uint32_t*>(vc.vis) + 1;
    // a point on the pixel of the group's previous point reuses that read
    uint32_t lim[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool same = j > 0 && live[j - 1] && pix[j] == pix[j - 1];
        lim[j] = (live[j] && vc.early && !same) ? vis_hi[2ull * pix[j]] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (live[j - 1] && pix[j] == pix[j - 1]) lim[j] = lim[j - 1];
    uint32_t need = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) need |= (uint32_t)(live[j] && w[j] <= lim[j]) << j;
    if (!need) return 0;   // the common case: every point is behind its pixel's depth
    uint32_t n_atom = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (live[j] && w[j] <= lim[j]) {
            atomicMin(vc.vis + pix[j], ((unsigned long long)w[j] << 32) | (idx0 + j));
            ++n_atom;
            // w > 0 here, so w - 1 does not wrap
            if (j < 3 && pix[j + 1] == pix[j]) lim[j + 1] = min(lim[j + 1], w[j] - 1u);
        }
    }
    return n_atom;
}

template <bool STREAM>
__device__ __forceinline__ uint4 ld_words(const uint32_t* p) {
    uint4 r;
    if (STREAM)
        asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                     : "l"(p));
    else
        asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                     : "l"(p));
    return r;
}

// Points [p0, p1) of one batch for one view at precision K. The loop over
// groups of 4 is warp-uniform; STREAM loads bypass L1 (single view), the
// multi-view kernel keeps the words in cache for the next view.
// One lane's group of 4 points at g: load, decode, raster.
template <int K, bool STREAM, bool PARTIAL>
__device__ __forceinline__ uint32_t raster_group(const CloudView& c, const ViewConst& vc,
                                                 const DecConst& d, uint32_t g, uint32_t valid) {
    const uint4 q1 = ld_words<STREAM>(c.w1 + g);
    uint4 q2 = make_uint4(0, 0, 0, 0), q3 = make_uint4(0, 0, 0, 0);
    if (K >= 2) q2 = ld_words<STREAM>(c.w2 + g);
    if (K >= 3) q3 = ld_words<STREAM>(c.w3 + g);
    float x[4], y[4], z[4];
    decode_point<K>(d, q1.x, q2.x, q3.x, x[0], y[0], z[0]);
    decode_point<K>(d, q1.y, q2.y, q3.y, x[1], y[1], z[1]);
    decode_point<K>(d, q1.z, q2.z, q3.z, x[2], y[2], z[2]);
    decode_point<K>(d, q1.w, q2.w, q3.w, x[3], y[3], z[3]);
    return raster_quad<PARTIAL>(vc, x, y, z, g, valid);
}

// Points [p0, p1) of one batch for one view at precision K, 128 points per
// warp step. Steps that lie wholly inside the range (all of them but the last
// for batches that start on a multiple of 128, as batches of 10,240 do) need
// no bounds checks; the first step of an unaligned range and the last step
// carry a validity mask. STREAM loads bypass L1 (single view), the multi-view
// kernel keeps the words in cache for the next view.
// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned start and size).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p), "r"(bytes) : "memory");
}

template <int K, bool STREAM>
__device__ __forceinline__ uint32_t segment(const CloudView& c, const ViewConst& vc,
                                            const DecConst& d, uint32_t p0, uint32_t p1,
                                            uint32_t lane) {
    uint32_t n_atom = 0;
    uint32_t base = p0 & ~3u;
    if (lane == 0 && p1 > base) {
        // the segment's words into L2, so that steps after the first hit L2
        const uint32_t bytes = ((p1 - base) * 4u + 15u) & ~15u;
        prefetch_l2(c.w1 + base, bytes);
        if (K >= 2) prefetch_l2(c.w2 + base, bytes);
        if (K >= 3) prefetch_l2(c.w3 + base, bytes);
    }
    if (base != p0 && base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j >= p0 && g + j < p1) << j;
            n_atom += raster_group<K, STREAM, true>(c, vc, d, g, valid);
        }
        base += 128u;
    }
    for (; base + 128u <= p1; base += 128u)
        n_atom += raster_group<K, STREAM, false>(c, vc, d, base + 4u * lane, 0xFu);
    if (base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j < p1) << j;
            n_atom += raster_group<K, STREAM, true>(c, vc, d, g, valid);
        }
    }
    return n_atom;
}

// ---- k_raster fast path: batches certified by batch_fast ----------------------
//
// For a certified batch every point is in front of the eye with w in
// [2^-99, 2^99] and its floor pixel lies inside the view, so the per-point
// tests of the general path (w > 0, reciprocal range, pixel range) are known to
// pass and are left out. The arithmetic is the definition's, in its order:
//  - decode: fl(X * cell) as one fused multiply-add fma(F, cell, -2^23 cell) on
//    the binary32 number F = 2^23 + X, whose exact value F cell - 2^23 cell is
//    X cell (X < 2^23 at k <= 2; the constants are exact since the certificate
//    bounds the sizes). At k = 1 the y field is read in place: the bits
//    (w & 0xFFC00) | bits(2^13) are the number 2^13 + Y, with constant
//    -2^13 cell.
//  - clip rows: each product as fma(m, x, +0), which differs from fl(m x) only
//    in the sign of a zero product. A zero's sign cannot change a nonzero sum,
//    and a zero sum gives the same pixel (c / w = +-0) or no point (w = +-0 is
//    not > 0), so the pixel and the key are those of the definition. Products
//    formed this way can feed packed adds: ptxas does not fold an fma into the
//    add that follows it.
//  - pixel: the certified bracket of pixel_bits_fast without the Newton step.
//    rcp.approx is specified to 1 ulp, so q' = fl(c r) is within 3u |q| of c/w
//    (u = 2^-24) and within 4u |q| of the IEEE quotient; the bracket needs a
//    margin of about 5u for |q| <= 1.01 and has 2^-21 = 8u. When the two ends
//    disagree, the point takes the IEEE-divide path.

// Per-view constants of the fast path, as packed pairs of the x and y rows.
struct FastView {
    f2_t m01, m45, m89, m1213;   // (m0, m1), (m4, m5), (m8, m9), (m12, m13)
    f2_t m37;                    // the w row's first two coefficients (m3, m7)
    float m11, m15;
    f2_t wh;                     // (W, H)
    uint32_t width;
    uint32_t npix;               // width * height
    uint32_t pixbias;            // -(2^23 bits) (width + 1): pixel = by width + bx + pixbias
    unsigned long long* vis;
};

__device__ __forceinline__ f2_t f2_at(const float* p) {
    return *reinterpret_cast<const f2_t*>(p);   // two adjacent floats, 8-byte aligned
}

__device__ __forceinline__ FastView make_fast_view(const ViewParams& v) {
    FastView f;
    f.m01 = f2_at(v.m + 0);
    f.m45 = f2_at(v.m + 4);
    f.m89 = f2_at(v.m + 8);
    f.m1213 = f2_at(v.m + 12);
    f.m37 = f2_pack(v.m[3], v.m[7]);
    f.m11 = v.m[11];
    f.m15 = v.m[15];
    f.wh = f2_pack((float)v.width, (float)v.height);
    f.width = v.width;
    f.npix = v.width * v.height;
    f.pixbias = 0u - 0x4B000000u * (v.width + 1u);
    f.vis = reinterpret_cast<unsigned long long*>(v.vis);
    return f;
}

// Per-batch decode constants of the fast path at precision K: x and y as a
// packed pair, z alone; x = min + fma(F, cell, nb).
struct FastDec {
    f2_t mn, cell, nb;
    float mnz, cellz, nbz;
};

template <int K>
__device__ __forceinline__ FastDec make_fast_dec(const pc_batch& b) {
    FastDec d;
    const float cx = ldexpf(b.size[0], -10 * K), cy = ldexpf(b.size[1], -10 * K);
    const float cz = ldexpf(b.size[2], -10 * K);
    d.mn = f2_pack(b.min[0], b.min[1]);
    d.cell = f2_pack(cx, cy);
    d.nb = f2_pack(-ldexpf(cx, 23), -ldexpf(cy, K == 1 ? 13 : 23));
    d.mnz = b.min[2];
    d.cellz = cz;
    d.nbz = -ldexpf(cz, 23);
    return d;
}

// Decoded position of one point of a certified batch: (x, y) as a packed
// pair, and z.
template <int K>
__device__ __forceinline__ void fast_decode(const FastDec& d, uint32_t a, uint32_t b, f2_t& xy,
                                            float& z) {
    uint32_t fx, fy, fz;
    if (K == 1) {
        fx = (a & 0x3FFu) | 0x4B000000u;
        fy = (a & 0xFFC00u) | 0x46000000u;
        fz = ((a >> 20) & 0x3FFu) | 0x4B000000u;
    } else {
        uint32_t qx, qy, qz;
        decode_q<2>(a, b, 0u, qx, qy, qz);
        fx = qx | 0x4B000000u;
        fy = qy | 0x4B000000u;
        fz = qz | 0x4B000000u;
    }
    xy = f2_add(d.mn, f2_fma_rn(f2_pack(__uint_as_float(fx), __uint_as_float(fy)), d.cell, d.nb));
    z = __fadd_rn(d.mnz, __fmaf_rn(__uint_as_float(fz), d.cellz, d.nbz));
}

// Clip coordinates of a decoded point: (cx, cy) as a packed pair, and cw.
__device__ __forceinline__ void fast_project(const FastView& fv, f2_t xy, float z, f2_t& cxy,
                                             float& cw) {
    float x, y;
    f2_unpack(xy, x, y);
    const f2_t zero = f2_pack(0.0f, 0.0f);
    const f2_t px = f2_fma_rn(fv.m01, f2_pack(x, x), zero);
    const f2_t py = f2_fma_rn(fv.m45, f2_pack(y, y), zero);
    const f2_t pz = f2_fma_rn(fv.m89, f2_pack(z, z), zero);
    cxy = f2_add(f2_add(f2_add(px, py), pz), fv.m1213);
    float w0, w1;
    f2_unpack(f2_fma_rn(fv.m37, xy, zero), w0, w1);
    cw = __fadd_rn(__fadd_rn(__fadd_rn(w0, w1), __fmul_rn(fv.m11, z)), fv.m15);
}

// Clip coordinates of one point of a certified batch from its words.
template <int K>
__device__ __forceinline__ void fast_clip(const FastView& fv, const FastDec& d, uint32_t a,
                                          uint32_t b, f2_t& cxy, float& cw) {
    f2_t xy;
    float z;
    fast_decode<K>(d, a, b, xy, z);
    fast_project(fv, xy, z, cxy, cw);
}

// Floor bits of a point of a certified batch by the bracket (no Newton step);
// false when the two ends differ and the IEEE-divide path must decide.
__device__ __forceinline__ bool pixel_bracket(const FastView& fv, f2_t cxy, float cw,
                                              uint32_t& bx, uint32_t& by) {
    const float r = rcp_approx(cw);
    const f2_t q = f2_mul(cxy, f2_pack(r, r));
    const f2_t half = f2_pack(0.5f, 0.5f);
    const f2_t blo = f2_fma_rd(f2_fma_rn(q, half, f2_pack(0.5f - 0x1.0p-21f, 0.5f - 0x1.0p-21f)),
                               fv.wh, f2_pack(8388608.0f, 8388608.0f));
    const f2_t bhi = f2_fma_rd(f2_fma_rn(q, half, f2_pack(0.5f + 0x1.0p-21f, 0.5f + 0x1.0p-21f)),
                               fv.wh, f2_pack(8388608.0f, 8388608.0f));
    bx = (uint32_t)blo;
    by = (uint32_t)(blo >> 32);
    return blo == bhi;
}

// A lane's group of 4 decoded points of a certified batch in one view:
// projection, pixel, early-depth reads and atomics.
__device__ __forceinline__ uint32_t raster_decoded(const FastView& fv, const f2_t (&xy)[4],
                                                   const float (&z)[4], uint32_t g) {
    f2_t cxy[4];
    float cw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) fast_project(fv, xy[j], z[j], cxy[j], cw[j]);
    uint32_t bx[4], by[4];
    bool slow = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) slow |= !pixel_bracket(fv, cxy[j], cw[j], bx[j], by[j]);
    if (slow) {
        // a bracket did not settle: the definition for all four (rare)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float cx, cy;
            f2_unpack(cxy[j], cx, cy);
            bx[j] = exact_floor_bits(cx, cw[j], __uint_as_float((uint32_t)fv.wh));
            by[j] = exact_floor_bits(cy, cw[j], __uint_as_float((uint32_t)(fv.wh >> 32)));
        }
    }
    uint32_t pix[4], w[4], lim[4];
    const uint32_t* vis_hi = reinterpret_cast<const uint32_t*>(fv.vis) + 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        // the certificate puts every pixel inside the view, so the clamp changes
        // nothing; it only keeps every access inside the buffer
        pix[j] = min(by[j] * fv.width + bx[j] + fv.pixbias, fv.npix - 1u);
        w[j] = __float_as_uint(cw[j]);
        lim[j] = vis_hi[2ull * pix[j]];
    }
    bool need = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) need |= w[j] <= lim[j];
    if (!need) return 0;
    uint32_t n_atom = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (w[j] <= lim[j]) {
            atomicMin(fv.vis + pix[j], ((unsigned long long)w[j] << 32) | (g + j));
            ++n_atom;
            if (j < 3 && pix[j + 1] == pix[j]) lim[j + 1] = min(lim[j + 1], w[j] - 1u);
        }
    }
    return n_atom;
}

// Decode of a lane's group of 4 points from its words (k <= 2).
template <int K>
__device__ __forceinline__ void decode_group(const FastDec& d, const uint4& q1, const uint4& q2,
                                             f2_t (&xy)[4], float (&z)[4]) {
    fast_decode<K>(d, q1.x, q2.x, xy[0], z[0]);
    fast_decode<K>(d, q1.y, q2.y, xy[1], z[1]);
    fast_decode<K>(d, q1.z, q2.z, xy[2], z[2]);
    fast_decode<K>(d, q1.w, q2.w, xy[3], z[3]);
}

// One lane's group of 4 points of a certified batch, its words given.
template <int K>
__device__ __forceinline__ uint32_t raster_group_fast(const FastView& fv, const FastDec& d,
                                                      const uint4& q1, const uint4& q2,
                                                      uint32_t g) {
    f2_t xy[4];
    float z[4];
    decode_group<K>(d, q1, q2, xy, z);
    return raster_decoded(fv, xy, z, g);
}

// Points [p0, p1) of a certified batch at precision K (1 or 2): whole groups
// of 4 take the fast path, the groups of a ragged first or last step the
// general one. A lane loads the words of its next step while it projects the
// current one, so the load's latency hides behind that step's arithmetic. The
// depth reads are not moved ahead: a read issued before the previous step's
// atomics would miss their updates, and the extra atomics cost more than the
// latency saved.
template <int K, bool STREAM>
__device__ __forceinline__ uint32_t segment_fast(const CloudView& c, const ViewConst& vc,
                                                 const FastView& fv, const pc_batch& bt,
                                                 uint32_t p0, uint32_t p1, uint32_t lane) {
    uint32_t n_atom = 0;
    uint32_t base = p0 & ~3u;
    if (lane == 0 && p1 > base) {
        const uint32_t bytes = ((p1 - base) * 4u + 15u) & ~15u;
        prefetch_l2(c.w1 + base, bytes);
        if (K >= 2) prefetch_l2(c.w2 + base, bytes);
    }
    if (base != p0 && base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j >= p0 && g + j < p1) << j;
            n_atom += raster_group<K, STREAM, true>(c, vc, make_dec_const(bt, K), g, valid);
        }
        base += 128u;
    }
    if (base + 128u <= p1) {
        // whole steps: the next step's words are loaded while the current one
        // is projected; the last step is peeled so that the loop carries no
        // bounds test, and two steps are unrolled
        const FastDec d = make_fast_dec<K>(bt);
        const uint32_t nsteps = (p1 - base) >> 7;
        uint32_t g = base + 4u * lane;
        const uint32_t* a1 = c.w1 + g;
        const uint32_t* a2 = K >= 2 ? c.w2 + g : nullptr;
        uint4 n1 = ld_words<STREAM>(a1);
        uint4 n2 = make_uint4(0, 0, 0, 0);
        if (K >= 2) n2 = ld_words<STREAM>(a2);
#pragma unroll 2
        for (uint32_t st = 1; st < nsteps; ++st) {
            const uint4 q1 = n1, q2 = n2;
            a1 += 128;
            n1 = ld_words<STREAM>(a1);
            if (K >= 2) {
                a2 += 128;
                n2 = ld_words<STREAM>(a2);
            }
            n_atom += raster_group_fast<K>(fv, d, q1, q2, g);
            g += 128u;
        }
        n_atom += raster_group_fast<K>(fv, d, n1, n2, g);
        base += nsteps << 7;
    }
    if (base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j < p1) << j;
            n_atom += raster_group<K, STREAM, true>(c, vc, make_dec_const(bt, K), g, valid);
        }
    }
    return n_atom;
}

// Points [p0, p1) of a certified batch at precision K for every view in vmask
// (each certified for the batch, each at precision K): the words of a step are
// loaded and decoded once, then projected into each view (Sec. 3.7). The
// decoded positions are the same for every view, since they depend on the
// batch and k only. Atomics per view go to the block's counters.
template <int K>
__device__ __forceinline__ void segment_fast_views(const CloudView& c, const ViewTable& vt,
                                                   uint32_t vmask, const pc_batch& bt,
                                                   uint32_t p0, uint32_t p1, uint32_t lane,
                                                   uint32_t* sh_atom) {
    uint32_t base = p0 & ~3u;
    if (lane == 0 && p1 > base) {
        const uint32_t bytes = ((p1 - base) * 4u + 15u) & ~15u;
        prefetch_l2(c.w1 + base, bytes);
        if (K >= 2) prefetch_l2(c.w2 + base, bytes);
    }
    // the ragged first and last steps view by view on the general path
    auto partial = [&](uint32_t g, uint32_t valid) {
        for (uint32_t mm = vmask; mm; mm &= mm - 1) {
            const uint32_t v = __ffs(mm) - 1;
            const uint32_t n = raster_group<K, false, true>(c, make_view_const(vt.v[v]),
                                                           make_dec_const(bt, K), g, valid);
            if (n) atomicAdd(&sh_atom[v], n);
        }
    };
    if (base != p0 && base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j >= p0 && g + j < p1) << j;
            partial(g, valid);
        }
        base += 128u;
    }
    if (base + 128u <= p1) {
        const FastDec d = make_fast_dec<K>(bt);
        uint4 n1 = ld_words<true>(c.w1 + base + 4u * lane);
        uint4 n2 = make_uint4(0, 0, 0, 0);
        if (K >= 2) n2 = ld_words<true>(c.w2 + base + 4u * lane);
        for (; base + 128u <= p1; base += 128u) {
            const uint32_t g = base + 4u * lane;
            const uint4 q1 = n1, q2 = n2;
            if (base + 256u <= p1) {
                n1 = ld_words<true>(c.w1 + g + 128u);
                if (K >= 2) n2 = ld_words<true>(c.w2 + g + 128u);
            }
            f2_t xy[4];
            float z[4];
            decode_group<K>(d, q1, q2, xy, z);
            for (uint32_t mm = vmask; mm; mm &= mm - 1) {
                const uint32_t v = __ffs(mm) - 1;
                const uint32_t n = raster_decoded(make_fast_view(vt.v[v]), xy, z, g);
                if (n) atomicAdd(&sh_atom[v], n);
            }
        }
    }
    if (base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j < p1) << j;
            partial(g, valid);
        }
    }
}

// Points [p0, p1) of a certified batch at precision K for views 0 and 1 of a
// two-view launch (vmask: bit v set when view v is certified at K): one decode
// per step as in segment_fast_views, then each view with its constants read at
// fixed parameter offsets, as in the one-view kernel (a view index that is
// only known at run time makes them loads).
template <int K>
__device__ __forceinline__ void segment_fast_pair(const CloudView& c, const ViewTable& vt,
                                                  uint32_t vmask, const pc_batch& bt,
                                                  uint32_t p0, uint32_t p1, uint32_t lane,
                                                  uint32_t& na0, uint32_t& na1) {
    uint32_t base = p0 & ~3u;
    if (lane == 0 && p1 > base) {
        const uint32_t bytes = ((p1 - base) * 4u + 15u) & ~15u;
        prefetch_l2(c.w1 + base, bytes);
        if (K >= 2) prefetch_l2(c.w2 + base, bytes);
    }
    // the ragged first and last steps view by view on the general path
    auto partial = [&](uint32_t g, uint32_t valid) {
        if (vmask & 1u)
            na0 += raster_group<K, false, true>(c, make_view_const(vt.v[0]), make_dec_const(bt, K),
                                                g, valid);
        if (vmask & 2u)
            na1 += raster_group<K, false, true>(c, make_view_const(vt.v[1]), make_dec_const(bt, K),
                                                g, valid);
    };
    if (base != p0 && base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j >= p0 && g + j < p1) << j;
            partial(g, valid);
        }
        base += 128u;
    }
    if (base + 128u <= p1) {
        const FastDec d = make_fast_dec<K>(bt);
        const uint32_t nsteps = (p1 - base) >> 7;
        uint32_t g = base + 4u * lane;
        const uint32_t* a1 = c.w1 + g;
        const uint32_t* a2 = K >= 2 ? c.w2 + g : nullptr;
        uint4 n1 = ld_words<true>(a1);
        uint4 n2 = make_uint4(0, 0, 0, 0);
        if (K >= 2) n2 = ld_words<true>(a2);
        auto step = [&](const uint4& q1, const uint4& q2) {
            f2_t xy[4];
            float z[4];
            decode_group<K>(d, q1, q2, xy, z);
            if (vmask & 1u) na0 += raster_decoded(make_fast_view(vt.v[0]), xy, z, g);
            if (vmask & 2u) na1 += raster_decoded(make_fast_view(vt.v[1]), xy, z, g);
        };
        for (uint32_t st = 1; st < nsteps; ++st) {
            const uint4 q1 = n1, q2 = n2;
            a1 += 128;
            n1 = ld_words<true>(a1);
            if (K >= 2) {
                a2 += 128;
                n2 = ld_words<true>(a2);
            }
            step(q1, q2);
            g += 128u;
        }
        step(n1, n2);
        base += nsteps << 7;
    }
    if (base < p1) {
        const uint32_t g = base + 4u * lane;
        if (g < p1) {
            uint32_t valid = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) valid |= (uint32_t)(g + j < p1) << j;
            partial(g, valid);
        }
    }
}

constexpr int kRasterThreads = 256;

__device__ __forceinline__ bool next_entry(const Scratch& s, uint32_t n_entries, uint32_t lane,
                                           DrawEntry& e) {
    uint32_t e_idx = 0;
    if (lane == 0) e_idx = atomicAdd(&s.counters[C_GRAB], 1u);
    e_idx = __shfl_sync(FULL, e_idx, 0);
    if (e_idx >= n_entries || e_idx >= s.capacity) return false;
    e = s.entries[e_idx];
    return true;
}

// One segment for one view at its precision k; certified batches (fast) at
// k <= 2 take the fast path.
template <bool STREAM>
__device__ __forceinline__ uint32_t segment_k(const CloudView& c, const ViewConst& vc,
                                              const FastView& fv, const pc_batch& bt, int k,
                                              bool fast, uint32_t p0, uint32_t p1,
                                              uint32_t lane) {
    if (fast && k == 1) return segment_fast<1, STREAM>(c, vc, fv, bt, p0, p1, lane);
    if (fast && k == 2) return segment_fast<2, STREAM>(c, vc, fv, bt, p0, p1, lane);
    const DecConst d = make_dec_const(bt, k);
    if (k == 1) return segment<1, STREAM>(c, vc, d, p0, p1, lane);
    if (k == 2) return segment<2, STREAM>(c, vc, d, p0, p1, lane);
    return segment<3, STREAM>(c, vc, d, p0, p1, lane);
}

__device__ __forceinline__ void flush_atomics(const Scratch& s, uint32_t view, uint32_t n_atom,
                                              uint32_t lane) {
    const uint32_t t = __reduce_add_sync(FULL, n_atom);
    if (lane == 0 && t)
        atomicAdd(&s.stats[(uint64_t)view * S_COUNT + S_ATOMICS], (unsigned long long)t);
}

// One view per launch: persistent warps take draw-list segments. Five blocks
// of 256 threads per SM (48 registers): the depth reads' latency is hidden by
// other warps, and more warps hide more of it.
__global__ void __launch_bounds__(kRasterThreads, 5) k_raster1(CloudView c, ViewTable vt,
                                                           uint32_t view_base, Scratch s) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_entries = s.counters[C_ENTRIES];
    const ViewConst vc = make_view_const(vt.v[0]);
    const FastView fv = make_fast_view(vt.v[0]);
    uint32_t n_atom = 0;
    DrawEntry e;
    while (next_entry(s, n_entries, lane, e)) {
        if (e.batch >= c.n_batches) {
            if (lane == 0) raise_error(s, E_BATCH_RANGE, e.batch);
            continue;
        }
        const pc_batch bt = c.batches[e.batch];
        const uint32_t p0 = bt.first + e.seg_first;
        n_atom += segment_k<true>(c, vc, fv, bt, (int)(e.kcodes & 3u), e.fast_mask & 1u, p0,
                                  p0 + e.seg_count, lane);
    }
    flush_atomics(s, view_base, n_atom, lane);
}

// Two views per launch (a stereo pair, Sec. 3.7): as k_rasterN, with both
// views' constants at fixed parameter offsets. Four blocks of 256 threads per
// SM (64 registers).
__global__ void __launch_bounds__(kRasterThreads, 4) k_raster2(CloudView c, ViewTable vt,
                                                           uint32_t view_base, Scratch s) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_entries = s.counters[C_ENTRIES];
    uint32_t na0 = 0, na1 = 0;
    DrawEntry e;
    while (next_entry(s, n_entries, lane, e)) {
        if (e.batch >= c.n_batches) {
            if (lane == 0) raise_error(s, E_BATCH_RANGE, e.batch);
            continue;
        }
        const pc_batch bt = c.batches[e.batch];
        const uint32_t p0 = bt.first + e.seg_first, p1 = p0 + e.seg_count;
        // certified views at k = 1 and at k = 2 share one decode each
        uint32_t fast1 = 0, fast2 = 0;
#pragma unroll
        for (uint32_t v = 0; v < 2; ++v) {
            if (!(((e.view_mask & e.fast_mask) >> v) & 1u)) continue;
            const uint32_t k = (e.kcodes >> (2 * v)) & 3u;
            if (k == 1) fast1 |= 1u << v;
            if (k == 2) fast2 |= 1u << v;
        }
        if (fast1) segment_fast_pair<1>(c, vt, fast1, bt, p0, p1, lane, na0, na1);
        if (fast2) segment_fast_pair<2>(c, vt, fast2, bt, p0, p1, lane, na0, na1);
        const uint32_t rest = e.view_mask & ~(fast1 | fast2);
        if (rest & 1u)
            na0 += segment_k<false>(c, make_view_const(vt.v[0]), make_fast_view(vt.v[0]), bt,
                                    (int)(e.kcodes & 3u), false, p0, p1, lane);
        if (rest & 2u)
            na1 += segment_k<false>(c, make_view_const(vt.v[1]), make_fast_view(vt.v[1]), bt,
                                    (int)((e.kcodes >> 2) & 3u), false, p0, p1, lane);
    }
    flush_atomics(s, view_base, na0, lane);
    flush_atomics(s, view_base + 1, na1, lane);
}

// Several views per launch (Sec. 3.7): the views certified for a segment's
// batch at one precision share its word loads and its decode (one walk of the
// segment); the others walk it once each, finding the words in cache. Every
// view keeps its own culling and precision, so each image is the one-view
// image bit for bit.
__global__ void __launch_bounds__(kRasterThreads, 4) k_rasterN(CloudView c, ViewTable vt,
                                                           uint32_t view_base, Scratch s) {
    __shared__ uint32_t sh_atom[kMaxViewsPerLaunch];
    for (uint32_t i = threadIdx.x; i < kMaxViewsPerLaunch; i += blockDim.x) sh_atom[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_entries = s.counters[C_ENTRIES];
    DrawEntry e;
    while (next_entry(s, n_entries, lane, e)) {
        if (e.batch >= c.n_batches) {
            if (lane == 0) raise_error(s, E_BATCH_RANGE, e.batch);
            continue;
        }
        const pc_batch bt = c.batches[e.batch];
        const uint32_t p0 = bt.first + e.seg_first;
        // certified views at k = 1 and at k = 2 share one decode each
        uint32_t fast1 = 0, fast2 = 0;
        for (uint32_t mm = e.view_mask & e.fast_mask; mm; mm &= mm - 1) {
            const uint32_t v = __ffs(mm) - 1;
            const uint32_t k = (uint32_t)((e.kcodes >> (2 * v)) & 3u);
            if (k == 1) fast1 |= 1u << v;
            if (k == 2) fast2 |= 1u << v;
        }
        if (fast1) segment_fast_views<1>(c, vt, fast1, bt, p0, p0 + e.seg_count, lane, sh_atom);
        if (fast2) segment_fast_views<2>(c, vt, fast2, bt, p0, p0 + e.seg_count, lane, sh_atom);
        for (uint32_t mm = e.view_mask & ~(fast1 | fast2); mm; mm &= mm - 1) {
            const uint32_t v = __ffs(mm) - 1;
            const ViewConst vc = make_view_const(vt.v[v]);
            const FastView fv = make_fast_view(vt.v[v]);
            const uint32_t n = segment_k<false>(c, vc, fv, bt, (int)((e.kcodes >> (2 * v)) & 3u),
                                                false, p0, p0 + e.seg_count, lane);
            const uint32_t t = __reduce_add_sync(FULL, n);
            if (lane == 0 && t) atomicAdd(&sh_atom[v], t);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < vt.n; i += blockDim.x)
        if (sh_atom[i])
            atomicAdd(&s.stats[(uint64_t)(view_base + i) * S_COUNT + S_ATOMICS],
                      (unsigned long long)sh_atom[i]);
}

// ---- k_shade: Sec. 3.6 high-quality shading, colour pass ---------------------------
//
// Walks the same draw list as the depth pass (same segments, same precision per
// view), so every point it projects was drawn by the depth pass and its pixel
// holds the closest depth w_min. A point adds its colour to the pixel's sums
// when w <= fl(w_min * 1.01f). Consecutive points of a group that land on the
// same pixel are summed in registers first; integer sums do not depend on the
// order of the additions, so the result is exact.
//
// Sum layouts (see hqs_region_words):
//   two-word  [R | G << 32, B | n << 32] per pixel: two reductions per addition,
//             no returned value; exact while n <= 16,843,009 (255 n < 2^32), which
//             the resolve checks: a carry out of the B field needs a larger n,
//             and n itself cannot wrap (a point is counted once).
//   packed    R | G << 18 | B << 36 | n << 54 per pixel: one atomicAdd per
//             addition, exact while n <= 1023 (255 n < 2^18). The addition that
//             takes n past 1023 sees the exact old value (the fields hold every
//             earlier addition) and sets the pixel's overflow bit; the thread
//             that sets it zeroes the pixel's two-word sums, and a second pass
//             sums every point of the marked pixels there, which the resolve
//             uses for them. The check of a returned value waits until the
//             lane's next addition, so that the lane does not stall on it.

constexpr uint32_t kHqsMaxCount = 16843009u;   // largest n with 255 n < 2^32
constexpr uint32_t kHqsPackedMax = 1023u;      // largest n with 255 n < 2^18 and n < 2^10

enum class ShadeMode { kTwoWord, kPacked, kFallback };

// Where one view's sums live.
struct ShadeBuf {
    unsigned long long* sums;      // two-word sums, or packed words
    unsigned long long* flags;     // packed: overflow bits
    unsigned long long* fallback;  // packed: two-word sums of the marked pixels
    unsigned long long* fallback_pixels;   // statistics word
};

// A packed addition whose returned value is still to be checked.
struct PendingAdd {
    unsigned long long old;
    uint32_t n, pix;
};

__device__ __forceinline__ void check_packed(const ShadeBuf& sb, PendingAdd& p) {
    if (p.n && (uint32_t)(p.old >> 54) + p.n > kHqsPackedMax) {
        const unsigned long long bit = 1ull << (p.pix & 63u);
        if (!(atomicOr(sb.flags + (p.pix >> 6), bit) & bit)) {
            sb.fallback[2ull * p.pix] = 0ull;
            sb.fallback[2ull * p.pix + 1] = 0ull;
            atomicAdd(sb.fallback_pixels, 1ull);
        }
    }
    p.n = 0;
}

template <ShadeMode MODE>
__device__ __forceinline__ void hqs_add(const ShadeBuf& sb, PendingAdd& pend, uint32_t pix,
                                        uint32_t r, uint32_t g, uint32_t b, uint32_t n) {
    if (MODE == ShadeMode::kPacked) {
        const unsigned long long add = (unsigned long long)r | ((unsigned long long)g << 18) |
                                       ((unsigned long long)b << 36) |
                                       ((unsigned long long)n << 54);
        const unsigned long long old = atomicAdd(sb.sums + pix, add);
        check_packed(sb, pend);
        pend.old = old;
        pend.n = n;
        pend.pix = pix;
    } else {
        unsigned long long* a = MODE == ShadeMode::kTwoWord ? sb.sums : sb.fallback;
        atomicAdd(a + 2ull * pix, (unsigned long long)r | ((unsigned long long)g << 32));
        atomicAdd(a + 2ull * pix + 1, (unsigned long long)b | ((unsigned long long)n << 32));
    }
}

// Predicated 32-bit load: 0 when p is false, and then no access is made.
__device__ __forceinline__ uint32_t ld_u32_if(bool p, const uint32_t* a) {
    uint32_t v = 0;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.u32 %0, [%1];\n\t}"
        : "+r"(v)
        : "l"(a), "r"((uint32_t)p));
    return v;
}

// Predicated 64-bit reduction: no access when p is false.
__device__ __forceinline__ void red_add_if(bool p, unsigned long long* a, unsigned long long v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.global.add.u64 [%0], %1;\n\t}"
                 :
                 : "l"(a), "l"(v), "r"((uint32_t)p)
                 : "memory");
}

// 32 bytes from a 32-byte aligned address on the read-only path: one sector.
__device__ __forceinline__ void ld_words8(const uint32_t* p, uint4& a, uint4& b) {
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}

// Compile-time flag of a 4-point group of the colour pass: all four points lie
// inside the segment (no per-point range tests).
template <bool B>
struct IntTag {
    static constexpr bool value = B;
};
// Running sums of one lane: the pixel of its current run of points, that
// pixel's depth limit fl(w_min * 1.01f) and (second pass) its fallback flag.
struct ShadeRun {
    uint32_t pix;
    float limit;
    bool flagged;
    uint32_t r, g, b, n;
};

template <ShadeMode MODE>
__device__ __forceinline__ void shade_flush(ShadeRun& run, const ShadeBuf& sb, PendingAdd& pend) {
    if (run.n) hqs_add<MODE>(sb, pend, run.pix, run.r, run.g, run.b, run.n);
    run.r = run.g = run.b = run.n = 0;
}

// Points [p0, p1) of one batch for one shaded view at precision K. Each lane
// walks its own contiguous share of the segment, so that consecutive points
// (Morton order makes them neighbours) extend one run: the visibility buffer is
// read only where a run starts, and one addition per run reaches the sums. The
// colour words are loaded with the coordinate words (nearly every point of a
// dense view falls within its pixel's window). At k <= 2 a lane takes 8 points
// per step with 32-byte loads, each of which fills one sector (the cloud's
// arrays are 32-byte aligned and padded past the last 8-point step); otherwise
// 4 points per step with 16-byte loads.
// FAST: a certified batch (batch_fast) at k <= 2, projected as in the depth
// pass's fast path; every point is then in front of the eye and inside the view.
template <int K, ShadeMode MODE, bool FAST>
__device__ __forceinline__ uint32_t shade_segment(const CloudView& c, const ViewConst& vc,
                                                  const FastView& fv, const ShadeBuf& sb,
                                                  const DecConst& d, const FastDec& df,
                                                  uint32_t p0, uint32_t p1, uint32_t lane) {
    const uint32_t base = p0 & ~3u;
    const uint32_t groups = (p1 - base + 3u) >> 2;
    const uint32_t per = (groups + 31u) >> 5;
    const uint32_t q0 = min(lane * per, groups), q1 = min(q0 + per, groups);
    const uint32_t* vis_hi = reinterpret_cast<const uint32_t*>(vc.vis) + 1;
    ShadeRun run;
    run.pix = 0xFFFFFFFFu;
    run.limit = 0.0f;
    run.flagged = false;
    run.r = run.g = run.b = run.n = 0;
    PendingAdd pend;
    pend.old = 0ull;
    pend.n = 0;
    pend.pix = 0;
    uint32_t n_blend = 0;
    // one group of 4 points; interior (an IntTag): all four lie inside [p0, p1)
    auto group = [&](auto interior, uint32_t g, const uint4& q1w, const uint4& q2w,
                     const uint4& q3w, const uint4& col) {
        constexpr bool INTERIOR = decltype(interior)::value;
        uint32_t pix[4], w[4], bx[4], by[4];
        bool live[4];
        if (FAST) {
            const uint32_t wa[4] = {q1w.x, q1w.y, q1w.z, q1w.w};
            const uint32_t wb[4] = {q2w.x, q2w.y, q2w.z, q2w.w};
            f2_t cxy[4];
            float cw[4];
            bool slow = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                fast_clip<K>(fv, df, wa[j], wb[j], cxy[j], cw[j]);
                slow |= !pixel_bracket(fv, cxy[j], cw[j], bx[j], by[j]);
            }
            if (slow) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float cx, cy;
                    f2_unpack(cxy[j], cx, cy);
                    bx[j] = exact_floor_bits(cx, cw[j], vc.W);
                    by[j] = exact_floor_bits(cy, cw[j], vc.H);
                }
            }
            // points g + lo .. g + hi - 1 of the group lie in [p0, p1)
            const uint32_t lo = p0 > g ? p0 - g : 0u, hi = p1 - g;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // inside the view by the certificate; the index is clamped all the same
                pix[j] = min(by[j] * fv.width + bx[j] + fv.pixbias, fv.npix - 1u);
                live[j] = INTERIOR || ((uint32_t)j >= lo && (uint32_t)j < hi);
                w[j] = __float_as_uint(cw[j]);
            }
        } else {
            float x[4], y[4], z[4];
            decode_point<K>(d, q1w.x, q2w.x, q3w.x, x[0], y[0], z[0]);
            decode_point<K>(d, q1w.y, q2w.y, q3w.y, x[1], y[1], z[1]);
            decode_point<K>(d, q1w.z, q2w.z, q3w.z, x[2], y[2], z[2]);
            decode_point<K>(d, q1w.w, q2w.w, q3w.w, x[3], y[3], z[3]);
            float cx[4], cy[4], cw[4];
            uint32_t slow = 0;   // live points whose bracket did not settle the pixel
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                clip_xyw(vc, x[j], y[j], z[j], cx[j], cy[j], cw[j]);
                live[j] = cw[j] > 0.0f && g + j >= p0 && g + j < p1;
                const bool ok = pixel_bits_fast(cx[j], cy[j], cw[j], vc.W, vc.H, bx[j], by[j]);
                slow |= (uint32_t)(live[j] && !ok) << j;
            }
            if (slow) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((slow >> j) & 1u) {
                        bx[j] = exact_floor_bits(cx[j], cw[j], vc.W);
                        by[j] = exact_floor_bits(cy[j], cw[j], vc.H);
                    }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t px = bx[j] - 0x4B000000u, py = by[j] - 0x4B000000u;
                live[j] = live[j] && px < vc.width && py < vc.height;
                w[j] = __float_as_uint(cw[j]);
                pix[j] = py * vc.width + px;
            }
        }
        if (MODE == ShadeMode::kTwoWord) {
            // Straight-line form of the run walk below, with no branch at run
            // starts: a point that starts a run flushes the lane's sums (two
            // predicated reductions, skipped when the run blended nothing) and
            // takes its pixel's limit; every point adds its colour when it passes.
            const uint32_t cc[4] = {col.x, col.y, col.z, col.w};
            bool st[4];
            uint32_t wm[4];
            uint32_t prev = run.pix;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                st[j] = live[j] && pix[j] != prev;
                prev = live[j] ? pix[j] : prev;
                wm[j] = ld_u32_if(st[j], vis_hi + 2ull * pix[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool f = st[j] && run.n != 0u;
                unsigned long long* a = sb.sums + 2ull * run.pix;
                red_add_if(f, a, (unsigned long long)run.r | ((unsigned long long)run.g << 32));
                red_add_if(f, a + 1, (unsigned long long)run.b | ((unsigned long long)run.n << 32));
                run.pix = st[j] ? pix[j] : run.pix;
                run.limit = st[j] ? __fmul_rn(__uint_as_float(wm[j]), 1.01f) : run.limit;
                run.r = st[j] ? 0u : run.r;
                run.g = st[j] ? 0u : run.g;
                run.b = st[j] ? 0u : run.b;
                run.n = st[j] ? 0u : run.n;
                const bool t = live[j] && __uint_as_float(w[j]) <= run.limit;
                if (t) {
                    run.r += cc[j] & 255u;
                    run.g += __byte_perm(cc[j], 0u, 0x4441);
                    run.b += __byte_perm(cc[j], 0u, 0x4442);
                    run.n += 1;
                    ++n_blend;
                }
            }
            return;
        }
        // reads for the points that start a run, issued together
        uint32_t wmin[4];
        bool flag[4];
        uint32_t last = run.pix;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool start = live[j] && pix[j] != last;
            if (live[j]) last = pix[j];
            wmin[j] = start ? vis_hi[2ull * pix[j]] : 0u;
            if (MODE == ShadeMode::kFallback)
                flag[j] = start && ((sb.flags[pix[j] >> 6] >> (pix[j] & 63u)) & 1ull);
        }
        const uint32_t cc[4] = {col.x, col.y, col.z, col.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!live[j]) continue;
            if (pix[j] != run.pix) {
                shade_flush<MODE>(run, sb, pend);
                run.pix = pix[j];
                run.limit = __fmul_rn(__uint_as_float(wmin[j]), 1.01f);
                if (MODE == ShadeMode::kFallback) run.flagged = flag[j];
            }
            bool t = __uint_as_float(w[j]) <= run.limit;
            if (MODE == ShadeMode::kFallback) t = t && run.flagged;
            if (t) {
                run.r += cc[j] & 255u;
                run.g += (cc[j] >> 8) & 255u;
                run.b += (cc[j] >> 16) & 255u;
                run.n += 1;
                ++n_blend;
            }
        }
    };
    if (K <= 2 && ((reinterpret_cast<uintptr_t>(c.w1) | reinterpret_cast<uintptr_t>(c.color) |
                    (K >= 2 ? reinterpret_cast<uintptr_t>(c.w2) : 0)) & 31u) == 0) {
        // 8 points per lane and step: each 32-byte load fills one sector
        const uint32_t base8 = p0 & ~7u;
        const uint32_t groups8 = (p1 - base8 + 7u) >> 3;
        const uint32_t per8 = (groups8 + 31u) >> 5;
        const uint32_t r0 = min(lane * per8, groups8), r1 = min(r0 + per8, groups8);
        const uint4 zero = make_uint4(0, 0, 0, 0);
        for (uint32_t q = r0; q < r1; ++q) {
            const uint32_t g = base8 + 8u * q;
            uint4 a0, a1, b0 = zero, b1 = zero, c0, c1;
            ld_words8(c.w1 + g, a0, a1);
            if (K >= 2) ld_words8(c.w2 + g, b0, b1);
            ld_words8(c.color + g, c0, c1);
            if (g >= p0 && g + 8u <= p1) {   // both groups inside the segment
                group(IntTag<true>{}, g, a0, b0, zero, c0);
                group(IntTag<true>{}, g + 4u, a1, b1, zero, c1);
            } else {
                group(IntTag<false>{}, g, a0, b0, zero, c0);
                if (g + 4u < p1) group(IntTag<false>{}, g + 4u, a1, b1, zero, c1);
            }
        }
    } else {
        for (uint32_t q = q0; q < q1; ++q) {
            const uint32_t g = base + 4u * q;
            const uint4 q1w = ld_words<false>(c.w1 + g);
            uint4 q2w = make_uint4(0, 0, 0, 0), q3w = make_uint4(0, 0, 0, 0);
            if (K >= 2) q2w = ld_words<false>(c.w2 + g);
            if (K >= 3) q3w = ld_words<false>(c.w3 + g);
            const uint4 col = ld_words<false>(c.color + g);
            group(IntTag<false>{}, g, q1w, q2w, q3w, col);
        }
    }
    shade_flush<MODE>(run, sb, pend);
    if (MODE == ShadeMode::kPacked) check_packed(sb, pend);
    return MODE == ShadeMode::kFallback ? 0u : n_blend;
}

template <ShadeMode MODE>
__device__ __forceinline__ uint32_t shade_segment_k(const CloudView& c, const ViewConst& vc,
                                                    const FastView& fv, const ShadeBuf& sb,
                                                    const pc_batch& bt, int k, bool fast,
                                                    uint32_t p0, uint32_t p1, uint32_t lane) {
    const DecConst d = make_dec_const(bt, k);
    if (fast && k == 1)
        return shade_segment<1, MODE, true>(c, vc, fv, sb, d, make_fast_dec<1>(bt), p0, p1, lane);
    if (fast && k == 2)
        return shade_segment<2, MODE, true>(c, vc, fv, sb, d, make_fast_dec<2>(bt), p0, p1, lane);
    const FastDec none{};
    if (k == 1) return shade_segment<1, MODE, false>(c, vc, fv, sb, d, none, p0, p1, lane);
    if (k == 2) return shade_segment<2, MODE, false>(c, vc, fv, sb, d, none, p0, p1, lane);
    return shade_segment<3, MODE, false>(c, vc, fv, sb, d, none, p0, p1, lane);
}

// Persistent warps take draw-list segments (a counter of their own); each
// segment is walked once per shaded view that did not cull its batch.
// LAYOUTS: the sum layouts of the launch's shaded views (1 two-word, 2 packed,
// 3 both), so that a launch of one layout carries only its own code; 0 is the
// second pass for packed views, which returns at once unless one of its views
// flagged a pixel. ONE: a launch of one view (index 0), whose parameters the
// compiler then reads as constant operands instead of loading them per use.
// Four blocks of 256 threads per SM (64 registers): the kernel waits on loads
// and on the visibility reads at run starts, and more warps hide more of it.
template <int LAYOUTS, bool ONE>
__global__ void __launch_bounds__(256, 4) k_shade(CloudView c, ViewTable vt, uint32_t view_base, Scratch s,
                        uint32_t shade_mask) {
    constexpr bool FALLBACK = LAYOUTS == 0;
    __shared__ uint32_t sh_blend[kMaxViewsPerLaunch];
    if (FALLBACK) {
        uint32_t fb = 0;
        for (uint32_t mm = shade_mask; mm; mm &= mm - 1) {
            const uint32_t v = __ffs(mm) - 1;
            if (s.stats[(uint64_t)(view_base + v) * S_COUNT + S_FALLBACK]) fb |= 1u << v;
        }
        if (!fb) return;
        shade_mask = fb;
    }
    for (uint32_t i = threadIdx.x; i < kMaxViewsPerLaunch; i += blockDim.x) sh_blend[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_entries = s.counters[C_ENTRIES];
    unsigned int* grab = &s.counters[FALLBACK ? C_GRAB_FALLBACK : C_GRAB_SHADE];
    for (;;) {
        uint32_t e_idx = 0;
        if (lane == 0) e_idx = atomicAdd(grab, 1u);
        e_idx = __shfl_sync(FULL, e_idx, 0);
        if (e_idx >= n_entries || e_idx >= s.capacity) break;
        const DrawEntry e = s.entries[e_idx];
        if (e.batch >= c.n_batches) {
            if (lane == 0) raise_error(s, E_BATCH_RANGE, e.batch);
            continue;
        }
        const pc_batch bt = c.batches[e.batch];
        const uint32_t p0 = bt.first + e.seg_first;
        for (uint32_t mm = e.view_mask & shade_mask; mm; mm &= mm - 1) {
            // one view: its index is a constant, so its parameters are operands
            const uint32_t v = ONE ? 0u : __ffs(mm) - 1;
            const ViewConst vc = make_view_const(vt.v[v]);
            const FastView fv = make_fast_view(vt.v[v]);
            const int k = (int)((e.kcodes >> (2 * v)) & 3u);
            const bool fast = (e.fast_mask >> v) & 1u;
            const ViewParams& vp = vt.v[v];
            const uint64_t npix = (uint64_t)vp.width * vp.height;
            ShadeBuf sb;
            sb.sums = vp.accum;
            sb.flags = vp.accum + npix;
            sb.fallback = vp.accum + hqs_fallback_offset(npix);
            sb.fallback_pixels = &s.stats[(uint64_t)(view_base + v) * S_COUNT + S_FALLBACK];
            uint32_t n;
            if (FALLBACK)
                n = shade_segment_k<ShadeMode::kFallback>(c, vc, fv, sb, bt, k, fast, p0,
                                                          p0 + e.seg_count, lane);
            else if (LAYOUTS == 2 || (LAYOUTS == 3 && (vp.flags & PC_VIEW_HQS_PACKED)))
                n = shade_segment_k<ShadeMode::kPacked>(c, vc, fv, sb, bt, k, fast, p0,
                                                        p0 + e.seg_count, lane);
            else
                n = shade_segment_k<ShadeMode::kTwoWord>(c, vc, fv, sb, bt, k, fast, p0,
                                                         p0 + e.seg_count, lane);
            const uint32_t t = __reduce_add_sync(FULL, n);
            if (lane == 0 && t) atomicAdd(&sh_blend[v], t);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < vt.n; i += blockDim.x)
        if (sh_blend[i])
            atomicAdd(&s.stats[(uint64_t)(view_base + i) * S_COUNT + S_BLENDED],
                      (unsigned long long)sh_blend[i]);
}

// ---- k_resolve ---------------------------------------------------------------------

__global__ void k_resolve(CloudView c, ViewTable vt, Scratch s) {
    const uint32_t v = blockIdx.y;
    if (v >= vt.n) return;
    const ViewParams& vp = vt.v[v];
    if (!vp.rgba) return;
    const uint64_t npix = (uint64_t)vp.width * vp.height;
    const bool dilate = (vp.flags & PC_VIEW_DILATE) != 0;
    const uint32_t mode = vp.accum ? hqs_mode(vp.flags) : 0u;
    const unsigned long long empty = empty_key(vp.flags);
    if (!dilate && !mode) {
        // plain resolve, 4 pixels per thread: two 16-byte key loads, four
        // independent colour gathers, one 16-byte store (vis and rgba are
        // 16-byte aligned); the last npix % 4 pixels one by one
        const uint64_t n4 = npix / 4;
        const ulonglong2* vis2 = reinterpret_cast<const ulonglong2*>(vp.vis);
        uint4* out4 = reinterpret_cast<uint4*>(vp.rgba);
        for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
             q += (uint64_t)gridDim.x * blockDim.x) {
            const ulonglong2 a = vis2[2 * q], b = vis2[2 * q + 1];
            const unsigned long long key[4] = {a.x, a.y, b.x, b.y};
            uint32_t col[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                col[j] = 0u;
                if (key[j] != empty) {
                    const uint32_t idx = (uint32_t)key[j];
                    if (idx < c.n_points) col[j] = __ldg(c.color + idx);
                    else raise_error(s, E_INDEX_RANGE, idx);
                }
            }
            out4[q] = make_uint4(col[0], col[1], col[2], col[3]);
        }
        for (uint64_t p = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
             p += (uint64_t)gridDim.x * blockDim.x) {
            const unsigned long long key = vp.vis[p];
            uint32_t out = 0u;
            if (key != empty) {
                const uint32_t idx = (uint32_t)key;
                if (idx < c.n_points) out = c.color[idx];
                else raise_error(s, E_INDEX_RANGE, idx);
            }
            vp.rgba[p] = out;
        }
        return;
    }
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long key = vp.vis[p];
        uint64_t at = p;   // the pixel whose sums a shaded view shows
        if (dilate) {
            // Sec. 3.7: the closest point within (2r+1)^2 pixels, r by ring
            const int px = (int)(p % vp.width), py = (int)(p / vp.width);
            const int r = 1 + ring_of(__fadd_rn((float)px, 0.5f), __fadd_rn((float)py, 0.5f),
                                      vp.width, vp.height);
            const int x0 = max(px - r, 0), x1 = min(px + r, (int)vp.width - 1);
            const int y0 = max(py - r, 0), y1 = min(py + r, (int)vp.height - 1);
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x) {
                    const uint64_t q = (uint64_t)y * vp.width + x;
                    const unsigned long long k = vp.vis[q];
                    if (k < key) {
                        key = k;
                        at = q;
                    }
                }
        }
        uint32_t out = 0u;
        if (mode && key != empty) {
            // Sec. 3.6: per-channel average of the sums, rounded down
            uint32_t r, g, b, n;
            const ulonglong2* two = reinterpret_cast<const ulonglong2*>(vp.accum);   // two-word sums
            bool use_two = mode == 1;
            if (mode == 2) {
                use_two = (vp.accum[npix + (at >> 6)] >> (at & 63)) & 1ull;
                two = reinterpret_cast<const ulonglong2*>(vp.accum + hqs_fallback_offset(npix));
                const unsigned long long a = vp.accum[at];
                r = (uint32_t)(a & 0x3FFFFu);
                g = (uint32_t)((a >> 18) & 0x3FFFFu);
                b = (uint32_t)((a >> 36) & 0x3FFFFu);
                n = (uint32_t)(a >> 54);
            }
            if (use_two) {
                const ulonglong2 t = two[at];
                r = (uint32_t)t.x;
                g = (uint32_t)(t.x >> 32);
                b = (uint32_t)t.y;
                n = (uint32_t)(t.y >> 32);
                if (n > kHqsMaxCount) raise_error(s, E_HQS_OVERFLOW, (uint32_t)at);
            }
            if (n) out = (r / n) | ((g / n) << 8) | ((b / n) << 16) | 0xFF000000u;
        } else if (key != empty) {
            const uint32_t idx = (uint32_t)key;
            if (idx < c.n_points) out = c.color[idx];
            else raise_error(s, E_INDEX_RANGE, idx);
        }
        vp.rgba[p] = out;
    }
}

// ---- k_merge_min: element-wise minimum of two visibility buffers ------------------
//
// Shards of one frame (disjoint batch ranges, Sec. 3.2) merge exactly: the
// minimum over (depth bits << 32 | index) keys is associative and commutative.
// 16-byte loads and stores (both buffers 16-byte aligned); the odd last key alone.
__global__ void k_merge_min(unsigned long long* dst, const unsigned long long* src, uint64_t n) {
    ulonglong2* d2 = reinterpret_cast<ulonglong2*>(dst);
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(src);
    const uint64_t n2 = n / 2;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const ulonglong2 a = d2[i], b = s2[i];
        d2[i] = make_ulonglong2(a.x < b.x ? a.x : b.x, a.y < b.y ? a.y : b.y);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
        dst[n - 1] = dst[n - 1] < src[n - 1] ? dst[n - 1] : src[n - 1];
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

cudaError_t launch_lod_pass(const CloudView& c, const ViewTable& vt, Scratch s, cudaStream_t st) {
    const unsigned blocks = (c.n_batches + kCullThreads - 1) / kCullThreads;
    if (blocks == 0) return cudaSuccess;
    k_lod_pass<<<blocks, kCullThreads, 0, st>>>(c, vt, s);
    return cudaGetLastError();
}

cudaError_t launch_cull(const CloudView& c, const ViewTable& vt, uint32_t view_base, Scratch s,
                        cudaStream_t st) {
    const unsigned blocks = (c.n_batches + kCullThreads - 1) / kCullThreads;
    if (blocks == 0) return cudaSuccess;
    k_cull<<<blocks, kCullThreads, 0, st>>>(c, vt, view_base, s);
    return cudaGetLastError();
}

int raster_occupancy(int threads_per_block, uint32_t nviews) {
    int nb = 0;
    cudaError_t e =
        nviews > 2    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rasterN, threads_per_block, 0)
        : nviews == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_raster2, threads_per_block, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_raster1, threads_per_block, 0);
    if (e != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_raster(const CloudView& c, const ViewTable& vt, uint32_t view_base, Scratch s,
                          RasterShape shape, cudaStream_t st) {
    int threads = shape.threads_per_block > 0 ? shape.threads_per_block : kRasterThreads;
    threads = threads > kRasterThreads ? kRasterThreads : (threads < 32 ? 32 : threads & ~31);
    int blocks = shape.blocks > 0 ? shape.blocks : num_sms() * raster_occupancy(threads, vt.n);
    if (vt.n > 2) k_rasterN<<<blocks, threads, 0, st>>>(c, vt, view_base, s);
    else if (vt.n == 2) k_raster2<<<blocks, threads, 0, st>>>(c, vt, view_base, s);
    else k_raster1<<<blocks, threads, 0, st>>>(c, vt, view_base, s);
    return cudaGetLastError();
}

template <int LAYOUTS>
static cudaError_t launch_shade_kernel(const CloudView& c, const ViewTable& vt, uint32_t view_base,
                                       Scratch s, int threads, uint32_t mask, cudaStream_t st) {
    int nb = 0;
    if constexpr (LAYOUTS != 3) {   // one view: the kernel with its index fixed
        if (vt.n == 1) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<LAYOUTS, true>, threads, 0);
            const int blocks = num_sms() * (nb > 0 ? nb : 1);
            k_shade<LAYOUTS, true><<<blocks, threads, 0, st>>>(c, vt, view_base, s, mask);
            return cudaGetLastError();
        }
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<LAYOUTS, false>, threads, 0);
    const int blocks = num_sms() * (nb > 0 ? nb : 1);
    k_shade<LAYOUTS, false><<<blocks, threads, 0, st>>>(c, vt, view_base, s, mask);
    return cudaGetLastError();
}

cudaError_t launch_shade(const CloudView& c, const ViewTable& vt, uint32_t view_base, Scratch s,
                         RasterShape shape, cudaStream_t st, int* launched) {
    uint32_t mask = 0, packed = 0;
    for (uint32_t v = 0; v < vt.n; ++v) {
        if (!vt.v[v].accum || !hqs_mode(vt.v[v].flags)) continue;
        mask |= 1u << v;
        if (vt.v[v].flags & PC_VIEW_HQS_PACKED) packed |= 1u << v;
    }
    *launched = 0;
    if (!mask) return cudaSuccess;
    int threads = shape.threads_per_block > 0 ? shape.threads_per_block : kRasterThreads;
    threads = threads > kRasterThreads ? kRasterThreads : (threads < 32 ? 32 : threads & ~31);
    const int layouts = (mask != packed ? 1 : 0) | (packed ? 2 : 0);
    cudaError_t e = layouts == 1 ? launch_shade_kernel<1>(c, vt, view_base, s, threads, mask, st)
                  : layouts == 2 ? launch_shade_kernel<2>(c, vt, view_base, s, threads, mask, st)
                                 : launch_shade_kernel<3>(c, vt, view_base, s, threads, mask, st);
    *launched = 1;
    if (e != cudaSuccess || !packed) return e;
    e = launch_shade_kernel<0>(c, vt, view_base, s, threads, packed, st);
    *launched = 2;
    return e;
}

cudaError_t launch_merge_min(uint64_t* dst, const uint64_t* src, uint64_t n, cudaStream_t st) {
    const int threads = 256;
    uint64_t blocks = (n / 2 + threads - 1) / threads;
    blocks = blocks < 1 ? 1 : (blocks > (uint64_t)num_sms() * 8 ? (uint64_t)num_sms() * 8 : blocks);
    k_merge_min<<<(unsigned)blocks, threads, 0, st>>>(reinterpret_cast<unsigned long long*>(dst),
                                                      reinterpret_cast<const unsigned long long*>(src),
                                                      n);
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

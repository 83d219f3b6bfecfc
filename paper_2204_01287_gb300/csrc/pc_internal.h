// pc_internal.h — types shared by the host side (api.cpp, encoder.cpp,
// serve.cpp) and the CUDA kernels (raster.cu) of libpcr.so.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pc.h"

namespace pcr {

constexpr uint32_t kMaxViewsPerLaunch = 32;   // views in one raster launch
constexpr uint32_t kMaxViewsPerRender = 256;  // views in one pc_render call
constexpr uint32_t kSegmentPoints = 2048;     // default points one warp takes per grab
constexpr uint32_t kMinSegmentPoints = 512;   // smallest grab the draw list is sized for
constexpr uint32_t kMaxDim = 16384;           // width and height limit

// Counter slots in Scratch::counters.
enum : uint32_t {
    C_ENTRIES = 0,   // draw-list entries written by the cull pass
    C_GRAB = 1,      // entries taken by raster warps
    C_ERROR = 2,     // device error flag (nonzero = error code)
    C_ERRINFO = 3,   // first offending value
    C_GRAB_SHADE = 4,  // entries taken by high-quality shading warps
    C_GRAB_FALLBACK = 5,  // ... by the second pass of packed shading
    C_COUNT = 8
};

// Per-view statistics slots in Scratch::stats (uint64 each).
enum : uint32_t {
    S_BATCHES = 0,   // batches that passed culling
    S_BK1 = 1,       // ... with k = 1, 2, 3
    S_PK1 = 4,       // their points with k = 1, 2, 3
    S_WORDS = 7,     // coordinate words loaded for this view's launch group
    S_ATOMICS = 9,   // points that passed the early-depth test and issued atomicMin
    S_BLENDED = 10,  // high-quality shading: points summed into their pixel
    S_FALLBACK = 11, // packed shading: pixels that overflowed into the two-word sums
    S_COUNT = 16
};

// Device error codes raised by kernels.
enum : uint32_t {
    E_NONE = 0,
    E_ENTRY_RANGE = 1,     // draw-list overflow
    E_BATCH_RANGE = 2,     // batch outside the point buffers
    E_INDEX_RANGE = 3,     // visibility key with an index outside the cloud
    E_HQS_OVERFLOW = 4,    // a pixel's colour sums exceeded their field width
};

// One view as the kernels see it (passed by value in a ViewTable).
struct ViewParams {
    float m[16];          // world -> clip, column-major
    uint32_t width, height;
    uint32_t flags;       // PC_VIEW_*
    float lod_px;
    float lod_px_periphery;
    uint32_t pad;
    uint64_t* vis;        // device, width*height
    uint32_t* rgba;       // device, width*height, may be null
    unsigned long long* accum;  // high-quality shading sums (library scratch), else null
};

#ifdef __CUDACC__
#define PCR_HD __host__ __device__
#else
#define PCR_HD
#endif

// High-quality shading sum buffer of one view (64-bit words), by layout:
//   two-word: [R | G << 32, B | n << 32] per pixel (2 npix words, all cleared);
//   packed:   P[npix] (R | G << 18 | B << 36 | n << 54), then F, a bit per pixel
//             marking the pixels that overflowed (both cleared), then, from an even
//             offset, two-word sums per pixel for those pixels, zeroed by the thread
//             that sets the pixel's bit.
// hqs_mode: 0 none, 1 two-word, 2 packed.
PCR_HD inline uint32_t hqs_mode(uint32_t flags) {
    return (flags & PC_VIEW_HQS_PACKED) ? 2u : (flags & PC_VIEW_HQS) ? 1u : 0u;
}
PCR_HD inline uint64_t hqs_flag_words(uint64_t npix) { return (npix + 63) / 64; }
PCR_HD inline uint64_t hqs_fallback_offset(uint64_t npix) {
    return (npix + hqs_flag_words(npix) + 1) & ~1ull;
}
// Words the clear pass zeroes.
PCR_HD inline uint64_t hqs_clear_words(uint32_t flags, uint64_t npix) {
    const uint32_t m = hqs_mode(flags);
    return m == 1 ? 2 * npix : m == 2 ? npix + hqs_flag_words(npix) : 0;
}
// Words of the view's region (a whole number of 16-byte words).
PCR_HD inline uint64_t hqs_region_words(uint32_t flags, uint64_t npix) {
    const uint32_t m = hqs_mode(flags);
    return m == 1 ? 2 * npix : m == 2 ? hqs_fallback_offset(npix) + 2 * npix : 0;
}

// Up to kMaxViewsPerLaunch views; lives in the kernel parameter space so that
// launches need no host->device copy and can be captured in CUDA graphs.
struct ViewTable {
    uint32_t n;
    float threshold_px;   // precision threshold T
    uint32_t seg_points;  // points per draw-list segment (multiple of 128)
    uint32_t pad;
    ViewParams v[kMaxViewsPerLaunch];
};
static_assert(sizeof(ViewTable) < 4000, "ViewTable must fit the kernel parameter space");

// A resident cloud as the kernels see it.
struct CloudView {
    const pc_batch* batches;
    const uint32_t* w1;
    const uint32_t* w2;
    const uint32_t* w3;
    const uint32_t* color;
    uint64_t n_points;
    uint32_t n_batches;
    uint32_t is_lod;
    const uint32_t* parent;     // LOD: parent node of each batch (root: itself)
    const uint32_t* level;      // LOD: depth of each node
};

// One unit of raster work: a segment of at most kSegmentPoints points of a
// batch, with the views that did not cull the batch and their precisions.
struct DrawEntry {
    uint64_t kcodes;      // 2 bits per view: k in 1..3
    uint32_t view_mask;   // bit v: view v renders this batch
    uint32_t batch;
    uint32_t seg_first;   // first point of the segment, relative to the batch
    uint32_t seg_count;
    uint32_t fast_mask;   // bit v: the batch is certified for view v's fast path
                          // (every point in front of the eye, inside the viewport,
                          // and decodable with one fused multiply-add per axis)
    uint32_t pad;
};
static_assert(sizeof(DrawEntry) == 32, "draw-list entries are 32 bytes");

// Per-stream scratch memory (device).
struct Scratch {
    DrawEntry* entries;
    uint64_t capacity;    // entries
    uint32_t* counters;   // C_COUNT
    unsigned long long* stats;  // kMaxViewsPerRender * S_COUNT
    uint32_t* lod_sel;    // LOD: per node, bit v = node passes view v of the launch
};

// Launch-shape knobs for the raster kernel.
struct RasterShape {
    int threads_per_block;
    int blocks;            // total persistent blocks
};

// ---- kernel launchers (raster.cu) ----------------------------------------

cudaError_t launch_clear(const ViewTable& vt, uint32_t view_base, Scratch s,
                         cudaStream_t st);
cudaError_t launch_cull(const CloudView& c, const ViewTable& vt, uint32_t view_base,
                        Scratch s, cudaStream_t st);
// LOD clouds: per node, the views whose frustum and size tests it passes.
cudaError_t launch_lod_pass(const CloudView& c, const ViewTable& vt, Scratch s, cudaStream_t st);
cudaError_t launch_raster(const CloudView& c, const ViewTable& vt, uint32_t view_base,
                          Scratch s, RasterShape shape, cudaStream_t st);
// High-quality shading colour pass (Sec. 3.6) over the draw list of the
// launch, for the views with a sum buffer, and the fallback pass of packed
// views; after launch_raster. *launched: kernels launched.
cudaError_t launch_shade(const CloudView& c, const ViewTable& vt, uint32_t view_base, Scratch s,
                         RasterShape shape, cudaStream_t st, int* launched);
cudaError_t launch_resolve(const CloudView& c, const ViewTable& vt, Scratch s,
                           cudaStream_t st);
// dst[i] = min(dst[i], src[i]) over n keys (both 16-byte aligned).
cudaError_t launch_merge_min(uint64_t* dst, const uint64_t* src, uint64_t n, cudaStream_t st);

// The key of a pixel no point reached: all ones, or, for views with
// PC_VIEW_SIGNED_EMPTY, the largest signed 64-bit value. Every point's key is
// below 2^63 (w is a positive finite binary32), so either sorts last.
PCR_HD inline unsigned long long empty_key(uint32_t flags) {
    return (flags & PC_VIEW_SIGNED_EMPTY) ? 0x7FFFFFFFFFFFFFFFull : ~0ull;
}
// Blocks per SM the raster kernel of a launch of nviews views can keep
// resident at a block size.
int raster_occupancy(int threads_per_block, uint32_t nviews);

// ---- host encoder (encoder.cpp) -------------------------------------------

pc_status encode_host(const float* xyz, const uint32_t* rgba, uint64_t n,
                      uint32_t batch_size, unsigned threads, bool keep_order, pc_batch* batches,
                      uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color,
                      uint32_t* perm);

unsigned hw_threads();
// True when all 3n coordinates are finite (no NaN or infinity), checked with
// `threads` threads.
bool coords_finite(const float* xyz, uint64_t n, unsigned threads);

}  // namespace pcr

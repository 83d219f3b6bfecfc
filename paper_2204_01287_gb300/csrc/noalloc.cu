// noalloc.cu — pc_render_noalloc: one view of an encoded cloud that lives in
// caller-provided device buffers, rendered without allocating any memory.
//
// The render path needs scratch memory beyond its inputs and outputs (the
// draw list of surviving batches, counters, statistics). pc_render takes it
// from per-stream buffers that the library allocates; this entry point takes
// it from a file-scope __device__ array instead, so that callers which may not
// allocate device memory can still render.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "pc_internal.h"

namespace pcr {
namespace {

// Draw-list entries the static scratch holds. A cloud cut into segments of s
// points needs at most nbatches + n_points / s + 1 entries; s is the smallest
// multiple of 128 from kSegmentPoints up that fits, and at most 2^20.
constexpr uint32_t kNoAllocEntries = 1u << 17;
constexpr uint32_t kNoAllocMaxSegment = 1u << 20;

struct NoAllocLayout {
    DrawEntry entries[kNoAllocEntries];
    uint32_t counters[C_COUNT];
    unsigned long long stats[S_COUNT];
};
// counters and stats are cleared by one memset, so stats must follow counters
// with no gap
static_assert(offsetof(NoAllocLayout, stats) ==
                  offsetof(NoAllocLayout, counters) + sizeof(uint32_t) * C_COUNT,
              "stats directly follows counters");

// About 4 MB per device, held by every GPU that loads the library until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocLayout)];

// Points per draw-list segment for a cloud, or 0 when no segment size up to
// 2^20 fits the static draw list.
uint32_t noalloc_segment(uint64_t nbatches, uint64_t n_points) {
    if (nbatches + 1 >= kNoAllocEntries) return 0;
    const uint64_t room = kNoAllocEntries - nbatches - 1;   // entries left for splits
    uint64_t seg = (n_points + room - 1) / room;             // n_points / seg <= room
    seg = (seg + 127) & ~127ull;
    if (seg < kSegmentPoints) seg = kSegmentPoints;
    return seg <= kNoAllocMaxSegment ? (uint32_t)seg : 0u;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the static scratch on the current device. The host-side
// name of the array is only a stand-in, so the address is looked up once per
// device (with that device current) and cached.
pc_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return PC_ENOTSUP;
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PC_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PC_OK;
}

}  // namespace
}  // namespace pcr

using namespace pcr;

extern "C" pc_status pc_render_noalloc(const pc_batch* batches, uint64_t nbatches,
                                       const uint32_t* w1, const uint32_t* w2,
                                       const uint32_t* w3, const uint32_t* color,
                                       uint64_t n_points, const pc_view* view,
                                       uint64_t* vis, uint32_t* rgba, float precision_px,
                                       uint32_t* device_error, void* stream) {
    if (!view || !vis || (nbatches && !batches)) return PC_EINVAL;
    if (n_points && (!w1 || !w2 || !w3 || !color)) return PC_EINVAL;
    if (n_points >= 0xFFFFFFFFull || !(precision_px > 0.0f)) return PC_EINVAL;
    const uint32_t seg = noalloc_segment(nbatches, n_points);
    if (seg == 0) return PC_EINVAL;
    if (view->width == 0 || view->height == 0 || view->width > kMaxDim || view->height > kMaxDim)
        return PC_EINVAL;
    if (hqs_mode(view->flags)) return PC_ENOTSUP;   // the sum buffer would need memory
    const uintptr_t align = (uintptr_t)vis | (uintptr_t)rgba | (uintptr_t)w1 | (uintptr_t)w2 |
                            (uintptr_t)w3 | (uintptr_t)color | (uintptr_t)batches;
    if (align & 15) return PC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PC_ECUDA;
    void* base = nullptr;
    pc_status rc = scratch_address(dev, &base);
    if (rc != PC_OK) return rc;
    NoAllocLayout* L = static_cast<NoAllocLayout*>(base);
    cudaStream_t st = (cudaStream_t)stream;

    Scratch s;
    s.entries = L->entries;
    s.capacity = kNoAllocEntries;
    s.counters = L->counters;
    s.stats = L->stats;
    s.lod_sel = nullptr;
    // the array keeps the previous call's contents: counters and statistics
    // (including the error flag) start from zero every call
    if (cudaMemsetAsync(L->counters, 0, sizeof L->counters + sizeof L->stats, st) != cudaSuccess)
        return PC_ECUDA;

    CloudView c;
    std::memset(&c, 0, sizeof c);
    c.batches = batches;
    c.w1 = w1;
    c.w2 = w2;
    c.w3 = w3;
    c.color = color;
    c.n_points = n_points;
    c.n_batches = (uint32_t)nbatches;

    ViewTable vt;
    std::memset(&vt, 0, sizeof vt);
    vt.n = 1;
    vt.threshold_px = precision_px;
    vt.seg_points = seg;
    std::memcpy(vt.v[0].m, view->view_proj, sizeof vt.v[0].m);
    vt.v[0].width = view->width;
    vt.v[0].height = view->height;
    vt.v[0].flags = view->flags;
    vt.v[0].lod_px = view->lod_px;
    vt.v[0].lod_px_periphery = view->lod_px_periphery;
    vt.v[0].vis = vis;
    vt.v[0].rgba = rgba;

    RasterShape shape;
    shape.threads_per_block = 256;
    shape.blocks = 0;   // one resident wave
    if (launch_clear(vt, 0, s, st) != cudaSuccess) return PC_ECUDA;
    if (nbatches && launch_cull(c, vt, 0, s, st) != cudaSuccess) return PC_ECUDA;
    if (nbatches && launch_raster(c, vt, 0, s, shape, st) != cudaSuccess) return PC_ECUDA;
    if (launch_resolve(c, vt, s, st) != cudaSuccess) return PC_ECUDA;
    // the device error flag and its value, for the caller to read once the
    // stream has reached this point (a copy into caller memory, no allocation)
    if (device_error && cudaMemcpyAsync(device_error, L->counters + C_ERROR, 2 * sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PC_ECUDA;
    return PC_OK;
}

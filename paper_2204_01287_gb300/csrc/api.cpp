// api.cpp — the C ABI of libpcr.so (include/pc.h): contexts, resident clouds,
// per-stream scratch, frame orchestration and event timing. The serving loop
// is in serve.cpp, the LOD builder in lod.cpp.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pc_api_internal.h"

using namespace pcr;

namespace pcr {

void Ctx::fail_msg(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> g(err_mu);
    last_error = buf;
}

pc_status Ctx::cuda_fail(cudaError_t e, const char* what) {
    fail_msg("%s: %s", what, cudaGetErrorString(e));
    return PC_ECUDA;
}

double Ctx::now_ms() const {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now() - t0).count();
}

void Cloud::free_device() {
    cudaFree(batches);
    cudaFree(w1);
    cudaFree(w2);
    cudaFree(w3);
    cudaFree(color);
    cudaFree(parent);
    cudaFree(level);
    batches = nullptr;
    w1 = w2 = w3 = color = nullptr;
    parent = level = nullptr;
}

CloudView Cloud::view() const {
    CloudView c;
    c.batches = batches;
    c.w1 = w1;
    c.w2 = w2;
    c.w3 = w3;
    c.color = color;
    c.n_points = n_points;
    c.n_batches = (uint32_t)n_batches;
    c.is_lod = is_lod;
    c.parent = parent;
    c.level = level;
    return c;
}

Slot::~Slot() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(scratch.entries);
    cudaFree(scratch.counters);
    cudaFree(scratch.stats);
    cudaFree(scratch.lod_sel);
    cudaFree(hqs_accum);
    cudaFree(host_vis);
    cudaFree(host_rgba);
}

pc_status Ctx::ensure_capacity(Slot& s, uint64_t entries, uint64_t nodes) {
    // each buffer on its own, so a failed allocation is retried by the next call
    if (!s.scratch.counters) {
        cudaError_t e = cudaMalloc(&s.scratch.counters, sizeof(uint32_t) * C_COUNT);
        if (e != cudaSuccess) {
            s.scratch.counters = nullptr;
            return cuda_fail(e, "scratch counters");
        }
        cudaMemsetAsync(s.scratch.counters, 0, sizeof(uint32_t) * C_COUNT, s.stream);
    }
    if (!s.scratch.stats) {
        const size_t bytes = sizeof(unsigned long long) * kMaxViewsPerRender * S_COUNT;
        cudaError_t e = cudaMalloc(&s.scratch.stats, bytes);
        if (e != cudaSuccess) {
            s.scratch.stats = nullptr;
            return cuda_fail(e, "scratch stats");
        }
        cudaMemsetAsync(s.scratch.stats, 0, bytes, s.stream);
    }
    if (entries > s.scratch.capacity) {
        cudaStreamSynchronize(s.stream);
        cudaFree(s.scratch.entries);
        s.scratch.entries = nullptr;
        s.scratch.capacity = 0;
        cudaError_t e = cudaMalloc(&s.scratch.entries, sizeof(DrawEntry) * entries);
        if (e != cudaSuccess) return cuda_fail(e, "draw list");
        s.scratch.capacity = entries;
    }
    if (nodes > s.lod_capacity) {
        cudaStreamSynchronize(s.stream);
        cudaFree(s.scratch.lod_sel);
        s.scratch.lod_sel = nullptr;
        s.lod_capacity = 0;
        cudaError_t e = cudaMalloc(&s.scratch.lod_sel, nodes * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail(e, "lod selection");
        s.lod_capacity = nodes;
    }
    return PC_OK;
}

static uint64_t view_hqs_words(const pc_view& v) {
    return hqs_region_words(v.flags, (uint64_t)v.width * v.height);
}

// The shading sum buffer holds the regions of every view of the largest
// launch group of a render call.
pc_status Ctx::ensure_hqs(Slot& s, const pc_view* views, uint32_t nviews, uint32_t maxv) {
    uint64_t need = 0;
    for (uint32_t base = 0; base < nviews; base += maxv) {
        uint64_t group = 0;
        for (uint32_t j = base; j < std::min(nviews, base + maxv); ++j)
            group += view_hqs_words(views[j]);
        need = std::max(need, group);
    }
    if (need <= s.hqs_capacity) return PC_OK;
    cudaStreamSynchronize(s.stream);
    cudaFree(s.hqs_accum);
    s.hqs_accum = nullptr;
    s.hqs_capacity = 0;
    cudaError_t e = cudaMalloc(&s.hqs_accum, need * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "shading sum buffer");
    s.hqs_capacity = need;
    return PC_OK;
}

Slot* Ctx::slot_for(cudaStream_t st) {
    std::lock_guard<std::mutex> g(mu);
    auto it = slots.find(st);
    if (it != slots.end()) return it->second.get();
    auto s = std::make_unique<Slot>();
    s->stream = st;
    Slot* p = s.get();
    slots[st] = std::move(s);
    return p;
}

std::shared_ptr<Cloud> Ctx::find_cloud(pc_cloud h) {
    std::lock_guard<std::mutex> g(mu);
    auto it = clouds.find(h);
    return it == clouds.end() ? nullptr : it->second;
}

Tune Ctx::tune_for(const Cloud& cl, uint32_t nviews) const {
    std::lock_guard<std::mutex> g(tune_mu);
    return cl.tune[std::min<uint32_t>(nviews, kMaxViewsPerLaunch)];
}

void Ctx::set_tune(Cloud& cl, uint32_t nviews, const Tune& t) {
    std::lock_guard<std::mutex> g(tune_mu);
    cl.tune[std::min<uint32_t>(nviews, kMaxViewsPerLaunch)] = t;
}

// The cloud's tuned launch shape (pc_config fields override it); untuned: 256
// threads and as many resident blocks as the kernel allows.
RasterShape Ctx::shape_for(const Cloud& cl, uint32_t nviews) {
    const Tune t = tune_for(cl, nviews);
    RasterShape r;
    r.threads_per_block = cfg.threads_per_block ? (int)cfg.threads_per_block
                          : t.threads_per_block ? t.threads_per_block : 256;
    int per_sm = cfg.blocks_per_sm ? (int)cfg.blocks_per_sm
                 : t.blocks_per_sm ? t.blocks_per_sm
                                   : raster_occupancy(r.threads_per_block, nviews);
    r.blocks = num_sms * per_sm;
    return r;
}

// Points per draw-list segment: the tuned size, made smaller (down to
// kMinSegmentPoints, in multiples of 128) when the cloud is too small to give
// every resident raster warp about four segments. LOD frames draw a small part
// of their cloud, so they take the smallest size.
uint32_t Ctx::seg_points_for(uint32_t nviews, const Cloud& cl, const RasterShape& shape) const {
    const Tune t = tune_for(cl, nviews);
    const uint32_t seg = t.seg_points ? t.seg_points : kSegmentPoints;
    if (cl.is_lod) return kMinSegmentPoints;
    const uint64_t warps = std::max<uint64_t>(1, (uint64_t)shape.blocks * shape.threads_per_block / 32);
    const uint64_t fit = (cl.n_points / (4 * warps)) & ~127ull;
    return (uint32_t)std::max<uint64_t>(kMinSegmentPoints, std::min<uint64_t>(seg, fit));
}

// Views per launch for a cloud: pc_set_views_per_launch's value when one is
// set, else the autotuner's choice for this cloud, else the configured maximum.
uint32_t Ctx::views_per_launch(const Cloud& cl) const {
    const uint32_t f = forced_vpl.load(), t = cl.tuned_vpl.load();
    uint32_t v = f ? f : t ? t : cfg.max_views_per_launch;
    return std::max<uint32_t>(1, std::min<uint32_t>(v, kMaxViewsPerLaunch));
}

// The kernels of one frame: per launch group, clear / cull / raster / resolve.
pc_status Ctx::launch_frame(const Cloud& cl, const pc_view* views, uint32_t nviews,
                            const pc_framebuffer* fbs, cudaStream_t st, Slot* slot,
                            uint32_t maxv, bool timing, const FrameOpts& fo) {
    CloudView cv = cl.view();
    if (fo.first || fo.count < cl.n_batches) {
        // a shard: the kernels see only the batches of the range (their point
        // indices stay those of the whole cloud)
        cv.batches += fo.first;
        cv.n_batches = (uint32_t)std::min<uint64_t>(fo.count, cl.n_batches - fo.first);
    }
    for (uint32_t base = 0; base < nviews; base += maxv) {
        uint64_t accum_off = 0;
        bool shade = false;
        ViewTable vt;
        std::memset(&vt, 0, sizeof vt);
        vt.n = std::min(maxv, nviews - base);
        vt.threshold_px = cfg.precision_px;
        const RasterShape shape = shape_for(cl, vt.n);
        vt.seg_points = seg_points_for(vt.n, cl, shape);
        for (uint32_t j = 0; j < vt.n; ++j) {
            const pc_view& pv = views[base + j];
            ViewParams& p = vt.v[j];
            std::memcpy(p.m, pv.view_proj, sizeof p.m);
            p.width = pv.width;
            p.height = pv.height;
            p.flags = pv.flags;
            p.lod_px = pv.lod_px;
            p.lod_px_periphery = pv.lod_px_periphery;
            p.vis = fbs[base + j].vis;
            p.rgba = fbs[base + j].rgba;
            if (hqs_mode(pv.flags)) {
                if (accum_off + view_hqs_words(pv) > slot->hqs_capacity) {
                    fail_msg("view %u: shading sum buffer too small for its launch group",
                             base + j);
                    return PC_EINVAL;
                }
                p.accum = slot->hqs_accum + accum_off;
                accum_off += view_hqs_words(pv);
                shade = true;
            }
        }
        FrameEvents* fe = nullptr;
        if (timing) {
            std::lock_guard<std::mutex> g(mu);
            frame_events.emplace_back();
            fe = &frame_events.back();
            for (auto& ev : fe->ev) cudaEventCreate(&ev);
            cudaEventRecord(fe->ev[0], st);
        }
        cudaError_t e = cudaSuccess;
        if (fo.resolve_only) {
            if (fe) for (int i = 1; i < 5; ++i) cudaEventRecord(fe->ev[i], st);
            e = launch_resolve(cv, vt, slot->scratch, st);
            if (e != cudaSuccess) return cuda_fail(e, "resolve launch");
            if (fe) cudaEventRecord(fe->ev[5], st);
            launches += 1;
            continue;
        }
        e = launch_clear(vt, base, slot->scratch, st);
        if (e != cudaSuccess) return cuda_fail(e, "clear launch");
        if (fe) cudaEventRecord(fe->ev[1], st);
        if (cl.is_lod) {
            e = launch_lod_pass(cv, vt, slot->scratch, st);
            if (e != cudaSuccess) return cuda_fail(e, "LOD selection launch");
            launches += 1;
        }
        e = launch_cull(cv, vt, base, slot->scratch, st);
        if (e != cudaSuccess) return cuda_fail(e, "cull launch");
        if (fe) cudaEventRecord(fe->ev[2], st);
        e = launch_raster(cv, vt, base, slot->scratch, shape, st);
        if (e != cudaSuccess) return cuda_fail(e, "raster launch");
        if (fe) cudaEventRecord(fe->ev[3], st);
        if (shade) {
            int nk = 0;
            e = launch_shade(cv, vt, base, slot->scratch, shape, st, &nk);
            if (e != cudaSuccess) return cuda_fail(e, "shading launch");
            launches += nk;
        }
        if (fe) cudaEventRecord(fe->ev[4], st);
        e = launch_resolve(cv, vt, slot->scratch, st);
        if (e != cudaSuccess) return cuda_fail(e, "resolve launch");
        if (fe) cudaEventRecord(fe->ev[5], st);
        launches += 4;
        raster_launches += 1;
    }
    return PC_OK;
}

// Render nviews views with per-view framebuffers on one stream. With
// PC_CFG_GRAPHS (and no per-pass timing) the frame's kernels are captured into
// a CUDA graph that is updated in place and replayed; a frame with the same
// launch layout reuses the instantiated graph.
pc_status Ctx::render(const Cloud& cl, const pc_view* views, uint32_t nviews,
                      const pc_framebuffer* fbs, cudaStream_t st, Slot* slot,
                      const FrameOpts& fo) {
    if (!views || !fbs || nviews == 0 || nviews > kMaxViewsPerRender) {
        fail_msg("pc_render: need 1..%u views and framebuffers", kMaxViewsPerRender);
        return PC_EINVAL;
    }
    const bool shard = fo.first != 0 || fo.count < cl.n_batches || fo.resolve_only;
    if (shard) {
        if (fo.first > cl.n_batches || (fo.count != ~0ull && fo.first + fo.count > cl.n_batches)) {
            fail_msg("batch range %llu + %llu outside the cloud's %llu batches",
                     (unsigned long long)fo.first, (unsigned long long)fo.count,
                     (unsigned long long)cl.n_batches);
            return PC_EINVAL;
        }
        if (cl.is_lod) {
            fail_msg("batch ranges and separate resolves need a plain cloud (not LOD)");
            return PC_ENOTSUP;
        }
        for (uint32_t v = 0; v < nviews; ++v)
            if (hqs_mode(views[v].flags)) {
                fail_msg("view %u: high-quality shading needs the whole frame in one call", v);
                return PC_ENOTSUP;
            }
    }
    for (uint32_t v = 0; v < nviews; ++v) {
        const pc_view& pv = views[v];
        if (pv.width == 0 || pv.height == 0 || pv.width > kMaxDim || pv.height > kMaxDim) {
            fail_msg("view %u: size %ux%u outside 1..%u", v, pv.width, pv.height, kMaxDim);
            return PC_EINVAL;
        }
        if (!fbs[v].vis || ((uintptr_t)fbs[v].vis & 15) || ((uintptr_t)fbs[v].rgba & 15)) {
            fail_msg("view %u: framebuffer missing or not 16-byte aligned", v);
            return PC_EINVAL;
        }
    }
    // PC_VIEW_HQS_PACKED is a preference: with more than 256 points of the
    // cloud per pixel of a view, many pixels pass 1023 points and the packed
    // sums' second pass costs more than two-word sums; both are exact, so the
    // image is the same
    std::vector<pc_view> eff;
    for (uint32_t v = 0; v < nviews; ++v) {
        const uint64_t npix = (uint64_t)views[v].width * views[v].height;
        if ((views[v].flags & PC_VIEW_HQS_PACKED) && cl.n_points > 256ull * npix) {
            if (eff.empty()) eff.assign(views, views + nviews);
            eff[v].flags = (eff[v].flags & ~PC_VIEW_HQS_PACKED) | PC_VIEW_HQS;
        }
    }
    if (!eff.empty()) views = eff.data();
    if (!slot) slot = slot_for(st);
    std::lock_guard<std::mutex> sg(slot->mu);
    const uint32_t maxv = views_per_launch(cl);   // one value for the whole call
    pc_status rc = ensure_capacity(*slot, cl.n_entries, cl.is_lod ? cl.n_batches : 0);
    if (rc == PC_OK) rc = ensure_hqs(*slot, views, nviews, maxv);
    if (rc != PC_OK) return rc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    const bool timing = timing_on.load();
    const bool graph = (cfg.flags & PC_CFG_GRAPHS) && !timing &&
                       cs == cudaStreamCaptureStatusNone && st != nullptr;
    if (graph) {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    }
    rc = launch_frame(cl, views, nviews, fbs, st, slot, maxv, timing, fo);
    if (graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc != PC_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        uint64_t shaded = 0;   // the views with a colour pass change the launch layout
        for (uint32_t v = 0; v < nviews; ++v) shaded |= (uint64_t)(hqs_mode(views[v].flags) != 0);
        const uint64_t key = ((uint64_t)nviews << 8) | maxv | ((uint64_t)cl.is_lod << 40) |
                             (shaded << 41) | ((uint64_t)fo.resolve_only << 42);
        cudaGraphExec_t& exec = slot->graphs[key];
        if (exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(exec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
        }
        if (!exec) e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            exec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    }
    if (rc != PC_OK) return rc;
    if (!fo.resolve_only) {
        slot->last_nviews = nviews;
        slot->last_total_batches = std::min<uint64_t>(fo.count, cl.n_batches - fo.first);
    }
    return PC_OK;
}

pc_status Ctx::check_device_error(Slot& s) {
    uint32_t c[C_COUNT];
    cudaError_t e = cudaMemcpyAsync(c, s.scratch.counters, sizeof c, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading device counters");
    if (c[C_ERROR] != E_NONE) {
        fail_msg("device error %u (value %u)", c[C_ERROR], c[C_ERRINFO]);
        uint32_t zero[2] = {0, 0};
        cudaMemcpyAsync(s.scratch.counters + C_ERROR, zero, sizeof zero, cudaMemcpyHostToDevice,
                        s.stream);
        cudaStreamSynchronize(s.stream);
        return PC_EDEVICE;
    }
    return PC_OK;
}

}  // namespace pcr

// ==== C ABI ================================================================

extern "C" {

void pc_config_default(pc_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->batch_size = 10240;
    cfg->precision_px = 512.0f;
    cfg->encoder_threads = 0;
    cfg->flags = 0;
    cfg->serve_pool_bytes = 2ull << 30;
    cfg->serve_streams = 4;
    cfg->max_views_per_launch = kMaxViewsPerLaunch;
}

const char* pc_strerror(pc_status s) {
    switch (s) {
        case PC_OK: return "ok";
        case PC_EINVAL: return "invalid argument";
        case PC_ENOMEM: return "out of memory";
        case PC_ENOTFOUND: return "no such cloud or ticket";
        case PC_EBUSY: return "admission refused";
        case PC_ETIMEDOUT: return "timed out";
        case PC_ECUDA: return "CUDA error";
        case PC_ENOTSUP: return "not supported";
        case PC_EDEVICE: return "device error flag raised";
        default: return "unknown status";
    }
}

pc_status pc_create(pc_ctx** out, int device, const pc_config* cfg) {
    if (!out) return PC_EINVAL;
    *out = nullptr;
    pc_config c;
    pc_config_default(&c);
    if (cfg) c = *cfg;
    if (c.batch_size == 0 || c.batch_size % 4 != 0) return PC_EINVAL;
    if (!(c.precision_px > 0.0f)) return PC_EINVAL;
    if (c.max_views_per_launch == 0 || c.max_views_per_launch > kMaxViewsPerLaunch)
        c.max_views_per_launch = kMaxViewsPerLaunch;
    if (c.serve_streams == 0) c.serve_streams = 1;
    if (c.serve_streams > 16) c.serve_streams = 16;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PC_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return PC_ECUDA;
    Ctx* ctx = nullptr;
    try {
        ctx = new Ctx();
    } catch (...) {
        return PC_ENOMEM;
    }
    ctx->device = device;
    ctx->cfg = c;
    ctx->t0 = std::chrono::steady_clock::now();
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (ctx->num_sms <= 0) ctx->num_sms = 1;
    ctx->timing_on = (c.flags & PC_CFG_TIMING) != 0;
    *out = reinterpret_cast<pc_ctx*>(ctx);
    return PC_OK;
}

void pc_destroy(pc_ctx* h) {
    if (!h) return;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    cudaSetDevice(ctx->device);
    serve_shutdown(*ctx);
    cudaDeviceSynchronize();
    for (auto& fe : ctx->frame_events)
        for (auto& ev : fe.ev) cudaEventDestroy(ev);
    ctx->clouds.clear();
    ctx->slots.clear();
    delete ctx;
}

const char* pc_last_error(pc_ctx* h) {
    if (!h) return "";
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->err_copy = ctx->last_error;
    return ctx->err_copy.c_str();
}

pc_status pc_encode(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
                    uint32_t threads, uint32_t flags, pc_batch* batches, uint32_t* w1,
                    uint32_t* w2, uint32_t* w3, uint32_t* color, uint32_t* perm) {
    if (n && (!xyz || !batches || !w1 || !w2 || !w3 || !color)) return PC_EINVAL;
    try {
        return encode_host(xyz, rgba, n, batch_size, threads, (flags & PC_ENCODE_KEEP_ORDER) != 0,
                           batches, w1, w2, w3, color, perm);
    } catch (...) {
        return PC_ENOMEM;
    }
}

}  // extern "C"

namespace pcr {

pc_cloud Ctx::register_cloud(const std::shared_ptr<Cloud>& cl) {
    std::lock_guard<std::mutex> g(mu);
    pc_cloud handle = ++next_handle;
    clouds[handle] = cl;
    return handle;
}

// Copy an encoded cloud to library-owned device memory (no handle yet).
pc_status upload_encoded_internal(Ctx& c, const pc_batch* batches, uint64_t nbatches,
                                  const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                                  const uint32_t* color, uint64_t n,
                                  std::shared_ptr<Cloud>& out) {
    Ctx* ctx = &c;
    if (n >= 0xFFFFFFFFull || nbatches >= 0xFFFFFFFFull) {
        ctx->fail_msg("cloud too large: %llu points", (unsigned long long)n);
        return PC_EINVAL;
    }
    if ((n && (!w1 || !w2 || !w3 || !color)) || (nbatches && !batches)) return PC_EINVAL;
    uint64_t entries = 0;
    for (uint64_t b = 0; b < nbatches; ++b) {
        if ((uint64_t)batches[b].first + batches[b].count > n) {
            ctx->fail_msg("batch %llu outside the point buffers", (unsigned long long)b);
            return PC_EINVAL;
        }
        entries += (batches[b].count + kMinSegmentPoints - 1) / kMinSegmentPoints;
    }
    cudaSetDevice(ctx->device);
    auto cl = std::make_shared<Cloud>();
    cl->n_points = n;
    cl->n_batches = nbatches;
    cl->n_entries = std::max<uint64_t>(entries, 1);
    const uint64_t npad = ((n + 3) & ~3ull) + 4;   // 16-byte groups never run past the end
    const size_t wb = npad * sizeof(uint32_t);
    cudaError_t e = cudaSuccess;
    uint32_t** bufs[4] = {&cl->w1, &cl->w2, &cl->w3, &cl->color};
    const uint32_t* src[4] = {w1, w2, w3, color};
    e = cudaMalloc(&cl->batches, std::max<uint64_t>(1, nbatches) * sizeof(pc_batch));
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(bufs[i], wb);
    if (e != cudaSuccess) {
        cl->free_device();
        ctx->fail_msg("cloud allocation (%llu points): %s", (unsigned long long)n,
                      cudaGetErrorString(e));
        return PC_ENOMEM;
    }
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
        e = cudaMemset(*bufs[i], 0, wb);
        if (e == cudaSuccess && n) e = cudaMemcpy(*bufs[i], src[i], n * sizeof(uint32_t),
                                                  cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && nbatches)
        e = cudaMemcpy(cl->batches, batches, nbatches * sizeof(pc_batch), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cl->free_device();
        return ctx->cuda_fail(e, "cloud upload");
    }
    cl->device_bytes = 4 * wb + nbatches * sizeof(pc_batch);
    out = cl;
    return PC_OK;
}

}  // namespace pcr

extern "C" {



pc_status pc_upload_encoded(pc_ctx* h, const pc_batch* batches, uint64_t nbatches,
                            const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                            const uint32_t* color, uint64_t n, pc_cloud* out) {
    if (!h || !out) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    *out = 0;
    std::shared_ptr<Cloud> cl;
    pc_status rc = upload_encoded_internal(*ctx, batches, nbatches, w1, w2, w3, color, n, cl);
    if (rc != PC_OK) return rc;
    *out = ctx->register_cloud(cl);
    return PC_OK;
}

pc_status pc_upload_cloud(pc_ctx* h, const float* xyz, const uint32_t* rgba, uint64_t n,
                          pc_cloud* out) {
    if (!h || !out || (n && !xyz)) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    *out = 0;
    if (n >= 0xFFFFFFFFull) {
        ctx->fail_msg("cloud too large: %llu points", (unsigned long long)n);
        return PC_EINVAL;
    }
    const uint32_t bs = ctx->cfg.batch_size;
    const uint64_t nb = (n + bs - 1) / bs;
    std::vector<pc_batch> batches;
    std::vector<uint32_t> w1, w2, w3, color;
    try {
        batches.resize(nb);
        w1.resize(n);
        w2.resize(n);
        w3.resize(n);
        color.resize(n);
    } catch (...) {
        ctx->fail_msg("host memory for encoding %llu points", (unsigned long long)n);
        return PC_ENOMEM;
    }
    const uint32_t eflags = (ctx->cfg.flags & PC_CFG_KEEP_ORDER) ? PC_ENCODE_KEEP_ORDER : 0u;
    pc_status rc = pc_encode(xyz, rgba, n, bs, ctx->cfg.encoder_threads, eflags, batches.data(),
                             w1.data(), w2.data(), w3.data(), color.data(), nullptr);
    if (rc != PC_OK) {
        ctx->fail_msg("encoder failed: %s", pc_strerror(rc));
        return rc;
    }
    return pc_upload_encoded(h, batches.data(), nb, w1.data(), w2.data(), w3.data(),
                             color.data(), n, out);
}

pc_status pc_cloud_get_info(pc_ctx* h, pc_cloud cloud, pc_cloud_info* info) {
    if (!h || !info) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    auto cl = ctx->find_cloud(cloud);
    if (!cl) return PC_ENOTFOUND;
    info->n_points = cl->n_points;
    info->n_batches = cl->n_batches;
    info->device_bytes = cl->device_bytes;
    info->is_lod = cl->is_lod;
    info->lod_levels = cl->lod_levels;
    return PC_OK;
}

pc_status pc_cloud_download(pc_ctx* h, pc_cloud cloud, pc_batch* batches, uint32_t* w1,
                            uint32_t* w2, uint32_t* w3, uint32_t* color) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    auto cl = ctx->find_cloud(cloud);
    if (!cl) return PC_ENOTFOUND;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaSuccess;
    const size_t wb = cl->n_points * sizeof(uint32_t);
    if (batches && cl->n_batches)
        e = cudaMemcpy(batches, cl->batches, cl->n_batches * sizeof(pc_batch), cudaMemcpyDeviceToHost);
    uint32_t* dst[4] = {w1, w2, w3, color};
    const uint32_t* srcs[4] = {cl->w1, cl->w2, cl->w3, cl->color};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        if (dst[i] && wb) e = cudaMemcpy(dst[i], srcs[i], wb, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PC_OK : ctx->cuda_fail(e, "cloud download");
}

pc_status pc_release_cloud(pc_ctx* h, pc_cloud cloud) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    std::shared_ptr<Cloud> cl;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->clouds.find(cloud);
        if (it == ctx->clouds.end()) return PC_ENOTFOUND;
        cl = it->second;
        ctx->clouds.erase(it);
    }
    cudaSetDevice(ctx->device);
    cl.reset();   // frees the device buffers unless a queued request still holds them
    return PC_OK;
}

pc_status pc_render(pc_ctx* h, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                    const pc_framebuffer* fbs, void* stream) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    auto cl = ctx->find_cloud(cloud);
    if (!cl) {
        ctx->fail_msg("pc_render: unknown cloud %llu", (unsigned long long)cloud);
        return PC_ENOTFOUND;
    }
    cudaSetDevice(ctx->device);
    return ctx->render(*cl, views, nviews, fbs, (cudaStream_t)stream, nullptr);
}

pc_status pc_render_range(pc_ctx* h, pc_cloud cloud, uint64_t first_batch, uint64_t batch_count,
                          const pc_view* views, uint32_t nviews, const pc_framebuffer* fbs,
                          void* stream) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    auto cl = ctx->find_cloud(cloud);
    if (!cl) {
        ctx->fail_msg("pc_render_range: unknown cloud %llu", (unsigned long long)cloud);
        return PC_ENOTFOUND;
    }
    if (batch_count == 0 || first_batch + batch_count > cl->n_batches ||
        first_batch + batch_count < first_batch) {
        ctx->fail_msg("pc_render_range: batches %llu + %llu outside 0..%llu",
                      (unsigned long long)first_batch, (unsigned long long)batch_count,
                      (unsigned long long)cl->n_batches);
        return PC_EINVAL;
    }
    cudaSetDevice(ctx->device);
    FrameOpts fo;
    fo.first = first_batch;
    fo.count = batch_count;
    return ctx->render(*cl, views, nviews, fbs, (cudaStream_t)stream, nullptr, fo);
}

pc_status pc_resolve(pc_ctx* h, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                     const pc_framebuffer* fbs, void* stream) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    auto cl = ctx->find_cloud(cloud);
    if (!cl) {
        ctx->fail_msg("pc_resolve: unknown cloud %llu", (unsigned long long)cloud);
        return PC_ENOTFOUND;
    }
    if (fbs)
        for (uint32_t v = 0; v < nviews && views; ++v)
            if (!fbs[v].rgba) {
                ctx->fail_msg("pc_resolve: view %u has no rgba buffer", v);
                return PC_EINVAL;
            }
    cudaSetDevice(ctx->device);
    FrameOpts fo;
    fo.resolve_only = true;
    return ctx->render(*cl, views, nviews, fbs, (cudaStream_t)stream, nullptr, fo);
}

pc_status pc_merge_min(uint64_t* dst, const uint64_t* src, uint64_t n, void* stream) {
    if (n == 0) return PC_OK;
    if (!dst || !src || ((uintptr_t)dst & 15) || ((uintptr_t)src & 15)) return PC_EINVAL;
    return launch_merge_min(dst, src, n, (cudaStream_t)stream) == cudaSuccess ? PC_OK
                                                                               : PC_ECUDA;
}

pc_status pc_render_host(pc_ctx* h, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                         uint32_t* const* host_rgba, void* stream) {
    if (!h || !views || !host_rgba || nviews == 0 || nviews > kMaxViewsPerRender) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    auto cl = ctx->find_cloud(cloud);
    if (!cl) return PC_ENOTFOUND;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Slot* slot = ctx->slot_for(st);
    uint64_t total = 0;
    std::vector<uint64_t> off(nviews);
    for (uint32_t v = 0; v < nviews; ++v) {
        if (!host_rgba[v] || views[v].width == 0 || views[v].height == 0 ||
            views[v].width > kMaxDim || views[v].height > kMaxDim)
            return PC_EINVAL;
        off[v] = total;
        total += ((uint64_t)views[v].width * views[v].height + 1) & ~1ull;
    }
    {
        std::lock_guard<std::mutex> sg(slot->mu);
        if (total > slot->host_pixels) {
            cudaStreamSynchronize(st);
            cudaFree(slot->host_vis);
            cudaFree(slot->host_rgba);
            slot->host_vis = nullptr;
            slot->host_rgba = nullptr;
            slot->host_pixels = 0;
            cudaError_t e = cudaMalloc(&slot->host_vis, total * sizeof(uint64_t));
            if (e == cudaSuccess) e = cudaMalloc(&slot->host_rgba, total * sizeof(uint32_t));
            if (e != cudaSuccess) return ctx->cuda_fail(e, "framebuffers for pc_render_host");
            slot->host_pixels = total;
        }
    }
    std::vector<pc_framebuffer> fbs(nviews);
    for (uint32_t v = 0; v < nviews; ++v) {
        fbs[v].vis = slot->host_vis + off[v];
        fbs[v].rgba = slot->host_rgba + off[v];
    }
    pc_status rc = ctx->render(*cl, views, nviews, fbs.data(), st, slot);
    if (rc != PC_OK) return rc;
    for (uint32_t v = 0; v < nviews; ++v) {
        cudaError_t e = cudaMemcpyAsync(host_rgba[v], fbs[v].rgba,
                                        (size_t)views[v].width * views[v].height * sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return ctx->cuda_fail(e, "image download");
    }
    return ctx->check_device_error(*slot);
}

pc_status pc_get_view_stats(pc_ctx* h, void* stream, uint32_t view, pc_view_stats* out) {
    if (!h || !out || view >= kMaxViewsPerRender) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    cudaSetDevice(ctx->device);
    Slot* slot = ctx->slot_for((cudaStream_t)stream);
    if (!slot->scratch.stats) return PC_ENOTFOUND;
    unsigned long long st[S_COUNT];
    cudaError_t e = cudaMemcpyAsync(st, slot->scratch.stats + (uint64_t)view * S_COUNT, sizeof st,
                                    cudaMemcpyDeviceToHost, slot->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(slot->stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "reading stats");
    std::memset(out, 0, sizeof *out);
    uint64_t nb_total = 0;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        nb_total = slot->last_total_batches;
    }
    out->batches_total = nb_total;
    out->batches_rendered = st[S_BATCHES];
    for (int k = 1; k <= 3; ++k) {
        out->batches_k[k] = st[S_BK1 + k - 1];
        out->points_k[k] = st[S_PK1 + k - 1];
        out->points_processed += out->points_k[k];
    }
    out->words_loaded_bytes = 4ull * st[S_WORDS];
    out->points_atomic = st[S_ATOMICS];
    out->points_blended = st[S_BLENDED];
    out->hqs_fallback_pixels = st[S_FALLBACK];
    return ctx->check_device_error(*slot);
}

pc_status pc_timing_begin(pc_ctx* h) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> g(ctx->mu);
    for (auto& fe : ctx->frame_events)
        for (auto& ev : fe.ev) cudaEventDestroy(ev);
    ctx->frame_events.clear();
    ctx->launches = 0;
    ctx->raster_launches = 0;
    ctx->timing_on = true;
    return PC_OK;
}

pc_status pc_timing_end(pc_ctx* h, pc_timing* out) {
    if (!h || !out) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> g(ctx->mu);
    std::memset(out, 0, sizeof *out);
    for (auto& fe : ctx->frame_events) {
        if (cudaEventSynchronize(fe.ev[5]) != cudaSuccess) return PC_ECUDA;
        float t[5];
        for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&t[i], fe.ev[i], fe.ev[i + 1]);
        out->ms_clear += t[0];
        out->ms_cull += t[1];
        out->ms_raster += t[2];
        out->ms_shade += t[3];
        out->ms_resolve += t[4];
        out->frames += 1;
    }
    out->launches = (uint32_t)ctx->launches;
    out->raster_launches = ctx->raster_launches;
    for (auto& fe : ctx->frame_events)
        for (auto& ev : fe.ev) cudaEventDestroy(ev);
    ctx->frame_events.clear();
    ctx->timing_on = (ctx->cfg.flags & PC_CFG_TIMING) != 0;
    return PC_OK;
}

}  // extern "C"

// autotune.cpp — pc_autotune: picks, for one cloud, the raster launch shape
// (threads per block, resident blocks per SM, points per warp grab) and the
// views per multi-view launch by timing candidates with CUDA events on the
// caller's stream. Every candidate renders the same bits; only the time
// differs. The choices are kept with the cloud: a 10M-point cloud and a
// 2B-point cloud on one context want different shapes and views per launch.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pc_api_internal.h"

using namespace pcr;

namespace {

// Median time of `reps` renders of views[0..n) with the current tuning.
pc_status time_render(Ctx& ctx, const Cloud& cl, const pc_view* views, uint32_t n,
                      const pc_framebuffer* fbs, cudaStream_t st, Slot* slot, int reps,
                      double& ms) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<float> t;
    pc_status rc = ctx.render(cl, views, n, fbs, st, slot);   // warm-up
    for (int r = 0; r < reps && rc == PC_OK; ++r) {
        cudaEventRecord(a, st);
        rc = ctx.render(cl, views, n, fbs, st, slot);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = PC_ECUDA;
        float x = 0;
        cudaEventElapsedTime(&x, a, b);
        t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != PC_OK) return rc;
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return PC_OK;
}

}  // namespace

extern "C" pc_status pc_autotune(pc_ctx* h, pc_cloud cloud, const pc_view* views,
                                 uint32_t nviews, void* stream, pc_tune_result* out) {
    if (!h || !views || !out || nviews == 0 || nviews > kMaxViewsPerRender) return PC_EINVAL;
    Ctx& ctx = *reinterpret_cast<Ctx*>(h);
    auto cl = ctx.find_cloud(cloud);
    if (!cl) return PC_ENOTFOUND;
    cudaSetDevice(ctx.device);
    cudaStream_t st = (cudaStream_t)stream;
    Slot* slot = ctx.slot_for(st);
    // library-owned framebuffers for the candidates
    uint64_t total = 0;
    std::vector<uint64_t> off(nviews);
    for (uint32_t v = 0; v < nviews; ++v) {
        if (views[v].width == 0 || views[v].height == 0 || views[v].width > kMaxDim ||
            views[v].height > kMaxDim)
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
            if (e != cudaSuccess) return ctx.cuda_fail(e, "autotune framebuffers");
            slot->host_pixels = total;
        }
    }
    std::vector<pc_framebuffer> fbs(nviews);
    for (uint32_t v = 0; v < nviews; ++v) {
        fbs[v].vis = slot->host_vis + off[v];
        fbs[v].rgba = slot->host_rgba + off[v];
    }
    const bool timing = ctx.timing_on;
    ctx.timing_on = false;
    // candidates run with the context's override cleared and this cloud's
    // views per launch set; both are restored or replaced at the end
    const uint32_t saved_forced = ctx.forced_vpl.exchange(0);
    const uint32_t saved_vpl = cl->tuned_vpl.load();
    std::memset(out, 0, sizeof *out);

    // 1. single-view launch shape on views[0]
    const Tune saved = ctx.tune_for(*cl, 1);
    Tune best = saved;
    double best_ms = 1e30;
    uint32_t cand = 0;
    pc_status rc = PC_OK;
    cl->tuned_vpl = 1;
    for (int tpb : {128, 256}) {
        const int occ = raster_occupancy(tpb, 1);
        for (int bps = std::max(1, occ / 2); bps <= occ && rc == PC_OK; ++bps) {
            for (uint32_t seg : {1024u, 2048u, 4096u}) {
                Tune t;
                t.threads_per_block = tpb;
                t.blocks_per_sm = bps;
                t.seg_points = seg;
                ctx.set_tune(*cl, 1, t);
                double ms = 0;
                rc = time_render(ctx, *cl, views, 1, fbs.data(), st, slot, 3, ms);
                if (rc != PC_OK) break;
                ++cand;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
        }
    }
    bool shape_chosen = false;
    if (rc == PC_OK) {
        shape_chosen = true;
        for (uint32_t v = 1; v <= kMaxViewsPerLaunch; ++v) {
            Tune t = best;
            if (v > 1) t.blocks_per_sm = 0;   // multi-view kernel: its own occupancy
            ctx.set_tune(*cl, v, t);
        }
        out->threads_per_block = (uint32_t)best.threads_per_block;
        out->blocks_per_sm = (uint32_t)best.blocks_per_sm;
        out->points_per_warp = best.seg_points;
        out->ms_per_view_single = best_ms;
        out->ms_per_view = best_ms;
        out->views_per_launch = 1;
    }
    // 2. views per launch over all views
    if (rc == PC_OK && nviews > 1) {
        double single_ms = 0;
        cl->tuned_vpl = 1;
        rc = time_render(ctx, *cl, views, nviews, fbs.data(), st, slot, 3, single_ms);
        ++cand;
        out->ms_per_view_single = single_ms / nviews;
        double best_view = single_ms / nviews;
        uint32_t best_vpl = 1;
        for (uint32_t vpl : {2u, 4u, 8u, 16u, 32u}) {
            if (rc != PC_OK || vpl > std::min<uint32_t>(nviews, ctx.cfg.max_views_per_launch)) break;
            cl->tuned_vpl = vpl;
            double ms = 0;
            rc = time_render(ctx, *cl, views, nviews, fbs.data(), st, slot, 3, ms);
            ++cand;
            if (rc == PC_OK && ms / nviews < best_view) {
                best_view = ms / nviews;
                best_vpl = vpl;
            }
        }
        if (rc == PC_OK) {
            cl->tuned_vpl = best_vpl;
            out->views_per_launch = best_vpl;
            out->ms_per_view = best_view;
        }
    } else {
        cl->tuned_vpl = saved_vpl;
    }
    if (rc != PC_OK) {   // keep the previous choices that were not replaced
        cl->tuned_vpl = saved_vpl;
        if (!shape_chosen) ctx.set_tune(*cl, 1, saved);
    }
    ctx.forced_vpl = saved_forced;
    out->candidates = cand;
    ctx.timing_on = timing;
    return rc != PC_OK ? rc : ctx.check_device_error(*slot);
}

extern "C" pc_status pc_set_views_per_launch(pc_ctx* h, uint32_t views_per_launch) {
    if (!h || views_per_launch > kMaxViewsPerLaunch) return PC_EINVAL;
    Ctx& ctx = *reinterpret_cast<Ctx*>(h);
    ctx.forced_vpl = views_per_launch;
    return PC_OK;
}

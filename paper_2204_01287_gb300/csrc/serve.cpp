// serve.cpp — serving loop behind pc_submit / pc_poll (continuous batching).
//
// Requests (1..32 views of a resident cloud) enter a FIFO queue. A scheduler
// thread admits a request once the device framebuffer pool has room for its
// visibility buffers and images and a launch slot is free, groups admitted
// requests of the same cloud into one multi-view launch (up to
// max_views_per_launch views), and runs up to serve_streams groups at once on
// their own CUDA streams. Requests that arrive while groups are on the GPU join
// the next group that starts, so work of several requests overlaps on the
// device. Each group copies its images to pinned host memory on a second
// stream of its lane, which waits for the group's render only: the lane takes
// its next group as soon as the render is done, so the next render overlaps
// the image copies. Host callbacks signal the end of a render and of a group's
// copies; pc_poll waits on a condition variable with a bounded timeout. Every
// wait in this file is bounded or woken by a state change; nothing waits on the
// device without a limit.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>

#include "arena.h"
#include "pc_api_internal.h"

namespace pcr {

namespace serve_detail {

constexpr uint32_t kMaxViewsPerRequest = 32;
constexpr int32_t kMaxPollMs = 60000;   // the longest single wait of pc_poll

enum ReqState { R_QUEUED = 0, R_RUNNING = 1, R_DONE = 2 };

struct Request {
    pc_ticket id = 0;
    std::shared_ptr<Cloud> cloud;
    std::vector<pc_view> views;
    std::vector<uint64_t> dev_off;    // per view: vis at dev_off, rgba after it
    std::vector<pc_framebuffer> user_fb;   // caller-owned framebuffers (else empty)
    std::vector<uint32_t*> host;      // per view pinned image
    std::vector<uint32_t> widths, heights;
    uint64_t dev_bytes = 0, dev_base = 0;
    uint64_t host_bytes = 0, host_base = 0;
    bool has_dev = false, has_host = false;
    double t_submit = 0, t_start = 0, t_done = 0;
    pc_status status = PC_OK;
    int state = R_QUEUED;
};

struct Lane {
    cudaStream_t stream = nullptr;        // renders
    cudaStream_t copy_stream = nullptr;   // image copies and completion
    cudaEvent_t rendered = nullptr;       // end of the latest render
    bool busy = false;                    // a render is in flight
    bool finished = false;                // its end was signalled (host callback)
    std::deque<std::vector<Request*>> groups;   // groups not yet complete, oldest first
    uint32_t completed = 0;               // completion callbacks not yet retired
};

}  // namespace serve_detail

using namespace serve_detail;

struct ServeState {
    Ctx* ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<pc_ticket, std::unique_ptr<Request>> reqs;
    uint8_t* dev_base = nullptr;
    Arena dev;
    uint8_t* host_base = nullptr;
    Arena host;
    std::vector<std::unique_ptr<Lane>> lanes;
    std::thread th;
    bool stop = false;
    pc_ticket next = 0;
};

namespace {

struct LaneSignal {
    ServeState* s;
    Lane* lane;
    bool copies;   // false: end of a render, true: end of a group's copies
};

void CUDART_CB lane_signal(void* p) {
    // runs on a CUDA callback thread: no CUDA calls here
    auto* sig = static_cast<LaneSignal*>(p);
    {
        std::lock_guard<std::mutex> g(sig->s->mu);
        if (sig->copies)
            ++sig->lane->completed;
        else
            sig->lane->finished = true;
    }
    sig->s->cv_work.notify_all();
    delete sig;
}

void release_device(ServeState& s, Request& r) {
    if (r.has_dev) {
        s.dev.release(r.dev_base, r.dev_bytes);
        r.has_dev = false;
    }
}

// Launch one group on a lane that the caller reserved (busy = true) under s.mu.
// Called WITHOUT s.mu: CUDA calls here may synchronize the device (a growing
// scratch buffer is freed), which waits for other lanes' host callbacks, and
// those take s.mu.
void launch_group(ServeState& s, Lane& lane, std::vector<Request*>& group) {
    Ctx& ctx = *s.ctx;
    std::vector<pc_view> views;
    std::vector<pc_framebuffer> fbs;
    for (Request* r : group) {
        for (size_t v = 0; v < r->views.size(); ++v) {
            views.push_back(r->views[v]);
            const uint64_t npix = (uint64_t)r->views[v].width * r->views[v].height;
            pc_framebuffer fb;
            if (!r->user_fb.empty()) {
                fb = r->user_fb[v];
            } else {
                fb.vis = reinterpret_cast<uint64_t*>(s.dev_base + r->dev_off[v]);
                fb.rgba = reinterpret_cast<uint32_t*>(s.dev_base + r->dev_off[v] + round_up(npix * 8));
            }
            fbs.push_back(fb);
        }
    }
    Slot* slot = ctx.slot_for(lane.stream);
    pc_status rc = ctx.render(*group[0]->cloud, views.data(), (uint32_t)views.size(), fbs.data(),
                              lane.stream, slot);
    // the copies wait for this render only, on the lane's copy stream
    cudaError_t e = cudaEventRecord(lane.rendered, lane.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(lane.copy_stream, lane.rendered, 0);
    if (e != cudaSuccess && rc == PC_OK) rc = ctx.cuda_fail(e, "serving stream order");
    size_t k = 0;
    for (Request* r : group) {
        for (size_t v = 0; v < r->views.size(); ++v, ++k) {
            if (rc != PC_OK) break;
            if (!r->user_fb.empty()) continue;   // the images stay in the caller's framebuffers
            const uint64_t npix = (uint64_t)r->views[v].width * r->views[v].height;
            e = cudaMemcpyAsync(r->host[v], fbs[k].rgba, npix * 4, cudaMemcpyDeviceToHost,
                                lane.copy_stream);
            if (e != cudaSuccess) rc = ctx.cuda_fail(e, "serving image copy");
        }
        if (rc != PC_OK) r->status = rc;
    }
    auto* rendered = new LaneSignal{&s, &lane, false};
    auto* copied = new LaneSignal{&s, &lane, true};
    const bool ok_render = cudaLaunchHostFunc(lane.stream, lane_signal, rendered) == cudaSuccess;
    const bool ok_copies = cudaLaunchHostFunc(lane.copy_stream, lane_signal, copied) == cudaSuccess;
    if (!ok_render) delete rendered;
    if (!ok_copies) delete copied;
    if (!ok_render || !ok_copies) {
        // a callback that cannot be queued is signalled here: the lane is
        // retired on the next pass and the statuses show the failure (a queued
        // callback of the other kind still arrives and finds nothing to do)
        std::lock_guard<std::mutex> g(s.mu);
        if (!ok_render) lane.finished = true;
        if (!ok_copies) ++lane.completed;
        for (Request* r : group)
            if (r->status == PC_OK) r->status = PC_ECUDA;
    }
}

// Retire the lane's completed groups (oldest first) and free its render slot
// once its render has ended (called with s.mu held).
void retire(ServeState& s, Lane& lane) {
    if (lane.busy && lane.finished) {
        lane.busy = false;
        lane.finished = false;
    }
    if (!lane.completed) return;
    const double t = s.ctx->now_ms();
    while (lane.completed && !lane.groups.empty()) {
        for (Request* r : lane.groups.front()) {
            release_device(s, *r);
            r->t_done = t;
            r->state = R_DONE;
        }
        lane.groups.pop_front();
        --lane.completed;
    }
    lane.completed = 0;
    s.cv_done.notify_all();
}

// Pick the next group from the queue (called with s.mu held): the oldest
// request that fits the pool decides the cloud, and that cloud's views per
// launch the group's size; later requests of the same cloud join while views
// and memory allow. A request that has waited more
// than 200 ms blocks everything behind it, so large requests cannot starve.
bool next_group(ServeState& s, std::vector<Request*>& group) {
    group.clear();
    uint32_t maxv = kMaxViewsPerLaunch;   // set by the group's cloud
    uint32_t nviews = 0;
    const double now = s.ctx->now_ms();
    for (auto it = s.queue.begin(); it != s.queue.end();) {
        Request* r = *it;
        const bool aged = now - r->t_submit > 200.0;
        if (!group.empty() && (r->cloud != group[0]->cloud || nviews + r->views.size() > maxv)) {
            if (aged) break;
            ++it;
            continue;
        }
        if (r->user_fb.empty()) {
            uint64_t off = 0;
            if (!s.dev.alloc(r->dev_bytes, off)) {
                if (aged) break;
                ++it;
                continue;
            }
            r->dev_base = off;
            r->has_dev = true;
            uint64_t o = off;
            for (size_t v = 0; v < r->views.size(); ++v) {
                r->dev_off[v] = o;
                const uint64_t npix = (uint64_t)r->views[v].width * r->views[v].height;
                o += round_up(npix * 8) + round_up(npix * 4);
            }
        }
        if (group.empty()) maxv = s.ctx->views_per_launch(*r->cloud);
        group.push_back(r);
        nviews += (uint32_t)r->views.size();
        it = s.queue.erase(it);
        if (nviews >= maxv) break;
    }
    return !group.empty();
}

void scheduler(ServeState* sp) {
    ServeState& s = *sp;
    cudaSetDevice(s.ctx->device);
    std::unique_lock<std::mutex> lk(s.mu);
    while (!s.stop) {
        for (auto& l : s.lanes) retire(s, *l);
        bool launched = false;
        for (auto& l : s.lanes) {
            if (l->busy) continue;
            std::vector<Request*> group;
            if (!next_group(s, group)) break;
            const double t = s.ctx->now_ms();
            for (Request* r : group) {
                r->t_start = t;
                r->state = R_RUNNING;
            }
            l->groups.push_back(group);
            l->busy = true;
            l->finished = false;
            lk.unlock();
            launch_group(s, *l, group);
            lk.lock();
            launched = true;
        }
        if (launched) continue;
        // sleep until a submission, a finished group or shutdown; the timeout
        // only bounds the wait, progress is driven by notifications
        s.cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace

void serve_shutdown(Ctx& ctx) {
    ServeState* s = ctx.serve;
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto& l : s->lanes) {
        for (cudaStream_t st : {l->stream, l->copy_stream}) {
            if (!st) continue;
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        if (l->rendered) cudaEventDestroy(l->rendered);
    }
    cudaFree(s->dev_base);
    cudaFreeHost(s->host_base);
    delete s;
    ctx.serve = nullptr;
}

static pc_status serve_start(Ctx& ctx) {
    if (ctx.serve) return PC_OK;
    auto* s = new ServeState();
    s->ctx = &ctx;
    const uint64_t dev_bytes = ctx.cfg.serve_pool_bytes ? ctx.cfg.serve_pool_bytes : (2ull << 30);
    const uint64_t host_bytes = dev_bytes / 3 + kAlign;
    cudaError_t e = cudaMalloc(&s->dev_base, dev_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_base, host_bytes);
    if (e != cudaSuccess) {
        cudaFree(s->dev_base);
        delete s;
        ctx.fail_msg("serving pools (%llu bytes): %s", (unsigned long long)dev_bytes,
                     cudaGetErrorString(e));
        return PC_ENOMEM;
    }
    s->dev.init(dev_bytes);
    s->host.init(host_bytes);
    for (uint32_t i = 0; i < ctx.cfg.serve_streams && e == cudaSuccess; ++i) {
        auto l = std::make_unique<Lane>();
        e = cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l->rendered, cudaEventDisableTiming);
        s->lanes.push_back(std::move(l));
    }
    if (e != cudaSuccess) {
        for (auto& l : s->lanes) {
            if (l->stream) cudaStreamDestroy(l->stream);
            if (l->copy_stream) cudaStreamDestroy(l->copy_stream);
            if (l->rendered) cudaEventDestroy(l->rendered);
        }
        cudaFree(s->dev_base);
        cudaFreeHost(s->host_base);
        delete s;
        ctx.fail_msg("serving streams: %s", cudaGetErrorString(e));
        return PC_ECUDA;
    }
    ctx.serve = s;
    s->th = std::thread(scheduler, s);
    return PC_OK;
}

}  // namespace pcr

using namespace pcr;

extern "C" {

pc_status pc_submit(pc_ctx* h, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                    const pc_framebuffer* fbs, pc_ticket* out) {
    if (!h || !views || !out || nviews == 0 || nviews > kMaxViewsPerRequest) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    *out = 0;
    auto cl = ctx->find_cloud(cloud);
    if (!cl) return PC_ENOTFOUND;
    cudaSetDevice(ctx->device);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!ctx->serve) {
            pc_status rc = serve_start(*ctx);
            if (rc != PC_OK) return rc;
        }
    }
    ServeState& s = *ctx->serve.load();
    auto r = std::make_unique<Request>();
    r->cloud = cl;
    r->views.assign(views, views + nviews);
    r->dev_off.resize(nviews);
    r->host.resize(nviews);
    for (uint32_t v = 0; v < nviews; ++v) {
        const pc_view& pv = views[v];
        if (pv.width == 0 || pv.height == 0 || pv.width > kMaxDim || pv.height > kMaxDim) {
            ctx->fail_msg("view %u: size %ux%u outside 1..%u", v, pv.width, pv.height, kMaxDim);
            return PC_EINVAL;
        }
        if (fbs && (!fbs[v].vis || ((uintptr_t)fbs[v].vis & 15) || ((uintptr_t)fbs[v].rgba & 15))) {
            ctx->fail_msg("view %u: framebuffer missing or not 16-byte aligned", v);
            return PC_EINVAL;
        }
        const uint64_t npix = (uint64_t)pv.width * pv.height;
        r->widths.push_back(pv.width);
        r->heights.push_back(pv.height);
        if (fbs) continue;
        r->dev_bytes += round_up(npix * 8) + round_up(npix * 4);
        r->host_bytes += round_up(npix * 4);
    }
    if (fbs) r->user_fb.assign(fbs, fbs + nviews);
    std::lock_guard<std::mutex> g(s.mu);
    if (fbs) {
        r->id = ++s.next;
        r->t_submit = ctx->now_ms();
        *out = r->id;
        s.queue.push_back(r.get());
        s.reqs[r->id] = std::move(r);
        s.cv_work.notify_all();
        return PC_OK;
    }
    if (r->dev_bytes > s.dev.size || r->host_bytes > s.host.size) {
        ctx->fail_msg("request needs %llu device bytes, pool holds %llu",
                      (unsigned long long)r->dev_bytes, (unsigned long long)s.dev.size);
        return PC_EBUSY;
    }
    uint64_t hoff = 0;
    if (!s.host.alloc(r->host_bytes, hoff)) {
        ctx->fail_msg("pinned image memory exhausted: release finished tickets");
        return PC_EBUSY;
    }
    r->host_base = hoff;
    r->has_host = true;
    uint64_t o = hoff;
    for (uint32_t v = 0; v < nviews; ++v) {
        r->host[v] = reinterpret_cast<uint32_t*>(s.host_base + o);
        o += round_up((uint64_t)views[v].width * views[v].height * 4);
    }
    r->id = ++s.next;
    r->t_submit = ctx->now_ms();
    *out = r->id;
    s.queue.push_back(r.get());
    s.reqs[r->id] = std::move(r);
    s.cv_work.notify_all();
    return PC_OK;
}

pc_status pc_poll(pc_ctx* h, pc_ticket ticket, int32_t timeout_ms, pc_result* out) {
    if (!h || !out) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    ServeState* sp = ctx->serve.load();
    if (!sp) return PC_ENOTFOUND;
    ServeState& s = *sp;
    if (timeout_ms < 0) {
        ctx->fail_msg("pc_poll: timeout %d ms is negative (0..%d)", timeout_ms, kMaxPollMs);
        return PC_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return PC_ENOTFOUND;
    Request* r = it->second.get();
    auto done = [&] { return r->state == R_DONE; };
    // one bounded wait: a request whose stream never finishes (held by a
    // callback, a hung kernel) costs the caller at most kMaxPollMs
    if (!done())
        s.cv_done.wait_for(lk, std::chrono::milliseconds(std::min(timeout_ms, kMaxPollMs)), done);
    if (!done()) return PC_ETIMEDOUT;
    std::memset(out, 0, sizeof *out);
    out->status = r->status;
    out->nviews = (uint32_t)r->views.size();
    out->rgba = r->user_fb.empty() ? r->host.data() : nullptr;
    out->widths = r->widths.data();
    out->heights = r->heights.data();
    out->t_submit_ms = r->t_submit;
    out->t_start_ms = r->t_start;
    out->t_done_ms = r->t_done;
    return PC_OK;
}

pc_status pc_release_ticket(pc_ctx* h, pc_ticket ticket) {
    if (!h) return PC_EINVAL;
    Ctx* ctx = reinterpret_cast<Ctx*>(h);
    ServeState* sp = ctx->serve.load();
    if (!sp) return PC_ENOTFOUND;
    ServeState& s = *sp;
    std::unique_ptr<Request> gone;
    {
        std::lock_guard<std::mutex> g(s.mu);
        auto it = s.reqs.find(ticket);
        if (it == s.reqs.end()) return PC_ENOTFOUND;
        Request* r = it->second.get();
        if (r->state != R_DONE) return PC_EBUSY;
        if (r->has_host) s.host.release(r->host_base, r->host_bytes);
        gone = std::move(it->second);
        s.reqs.erase(it);
    }
    // destroyed without s.mu: dropping the last holder of a released cloud
    // frees its device memory, which synchronizes the device
    gone.reset();
    return PC_OK;
}

}  // extern "C"

// pc_api_internal.h — host-side state of a context (api.cpp, serve.cpp).
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pc_internal.h"

namespace pcr {

// Launch parameters pc_autotune chose for a cloud, by views per launch.
struct Tune {
    int threads_per_block = 0;
    int blocks_per_sm = 0;
    uint32_t seg_points = 0;
};

// A resident cloud: device buffers owned by the library.
struct Cloud {
    pc_batch* batches = nullptr;
    uint32_t* w1 = nullptr;
    uint32_t* w2 = nullptr;
    uint32_t* w3 = nullptr;
    uint32_t* color = nullptr;
    uint32_t* parent = nullptr;   // LOD clouds
    uint32_t* level = nullptr;
    uint64_t n_points = 0;
    uint64_t n_batches = 0;
    uint64_t n_entries = 0;       // draw-list entries a frame can need
    uint64_t device_bytes = 0;
    uint32_t is_lod = 0;
    uint32_t lod_levels = 0;
    std::atomic<uint32_t> tuned_vpl{0};   // views per launch pc_autotune chose for this
                                          // cloud (0: none yet)
    Tune tune[kMaxViewsPerLaunch + 1];    // its launch shapes (Ctx::tune_mu guards them)
    void free_device();
    CloudView view() const;
    // Device memory goes with the last holder (a queued serving request may
    // still hold the cloud after pc_release_cloud); cudaFree waits for the
    // device work that uses it.
    ~Cloud() { free_device(); }
};

// Scratch and library-owned framebuffers of one stream.
struct Slot {
    cudaStream_t stream = nullptr;
    std::mutex mu;
    Scratch scratch{};
    uint64_t lod_capacity = 0;      // nodes the LOD selection buffer holds
    unsigned long long* hqs_accum = nullptr;   // high-quality shading sums of a launch group
    uint64_t hqs_capacity = 0;      // 64-bit words hqs_accum holds
    uint64_t* host_vis = nullptr;     // pc_render_host framebuffers
    uint32_t* host_rgba = nullptr;
    uint64_t host_pixels = 0;
    uint32_t last_nviews = 0;
    uint64_t last_total_batches = 0;
    std::map<uint64_t, cudaGraphExec_t> graphs;   // replayable frames by launch layout
    ~Slot();
};

struct FrameEvents {
    cudaEvent_t ev[6];   // start, after clear, cull, raster, shade (colour pass), resolve
};

// What one render call draws: batches [first, first + count) of the cloud (a
// shard, Sec. 3.2's batches being independent), or, with resolve_only, only
// the resolve of visibility buffers that earlier calls filled.
struct FrameOpts {
    uint64_t first = 0;
    uint64_t count = ~0ull;
    bool resolve_only = false;
};

struct ServeState;   // serve.cpp

struct Ctx {
    int device = 0;
    int num_sms = 1;
    pc_config cfg{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;                          // clouds, slots, timing records
    std::map<pc_cloud, std::shared_ptr<Cloud>> clouds;
    std::map<cudaStream_t, std::unique_ptr<Slot>> slots;
    pc_cloud next_handle = 0;
    std::mutex err_mu;
    std::string last_error, err_copy;
    std::atomic<bool> timing_on{false};   // read once per pc_render call
    std::deque<FrameEvents> frame_events;
    std::atomic<uint64_t> launches{0};
    std::atomic<uint64_t> raster_launches{0};
    mutable std::mutex tune_mu;             // guards the clouds' tune[]: pc_autotune
                                            // writes it while serving threads launch
    std::atomic<uint32_t> forced_vpl{0};   // pc_set_views_per_launch (0: per cloud)
    std::atomic<ServeState*> serve{nullptr};   // set once, by the first pc_submit

    void fail_msg(const char* fmt, ...);
    pc_status cuda_fail(cudaError_t e, const char* what);
    double now_ms() const;
    Slot* slot_for(cudaStream_t st);
    std::shared_ptr<Cloud> find_cloud(pc_cloud h);
    pc_status ensure_capacity(Slot& s, uint64_t entries, uint64_t nodes);
    pc_status ensure_hqs(Slot& s, const pc_view* views, uint32_t nviews, uint32_t maxv);
    RasterShape shape_for(const Cloud& cl, uint32_t nviews);
    uint32_t seg_points_for(uint32_t nviews, const Cloud& cl, const RasterShape& shape) const;
    uint32_t views_per_launch(const Cloud& cl) const;
    Tune tune_for(const Cloud& cl, uint32_t nviews) const;
    void set_tune(Cloud& cl, uint32_t nviews, const Tune& t);
    pc_status launch_frame(const Cloud& cl, const pc_view* views, uint32_t nviews,
                           const pc_framebuffer* fbs, cudaStream_t st, Slot* slot, uint32_t maxv,
                           bool timing, const FrameOpts& fo);
    pc_status render(const Cloud& cl, const pc_view* views, uint32_t nviews,
                     const pc_framebuffer* fbs, cudaStream_t st, Slot* slot,
                     const FrameOpts& fo = FrameOpts());
    pc_status check_device_error(Slot& s);
    pc_cloud register_cloud(const std::shared_ptr<Cloud>& cl);
};

pc_status upload_encoded_internal(Ctx& ctx, const pc_batch* batches, uint64_t nbatches,
                                  const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                                  const uint32_t* color, uint64_t n,
                                  std::shared_ptr<Cloud>& out);

pc_status lod_encode_host(const float* xyz, const uint32_t* rgba, uint64_t n,
                          uint32_t max_levels, uint32_t M, uint32_t seed, unsigned threads,
                          std::vector<pc_batch>& nodes, std::vector<uint32_t>& parent,
                          std::vector<uint32_t>& level, uint32_t* perm, uint32_t* w1,
                          uint32_t* w2, uint32_t* w3, uint32_t* color);

// serve.cpp
void serve_shutdown(Ctx& ctx);

}  // namespace pcr

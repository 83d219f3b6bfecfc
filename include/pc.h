/* pc.h — C ABI of the GB300 point-cloud rasterizer (libpcr.so).
 *
 * One-pixel point rasterization of large coloured point clouds after Schuetz,
 * Kerbl and Wimmer, "Software Rasterization of 2 Billion Points in Real Time"
 * (2022): points are Morton-sorted and cut into batches (Sec. 3.1), each batch
 * stores its coordinates as three 10-bit-per-axis words relative to its box
 * (Eq. 1, Listing 2), and every frame culls batches (Sec. 3.2), picks 10, 20
 * or 30 bits per batch from its projected size (Sec. 3.3), writes
 * (depth bits << 32 | point index) into a 64-bit visibility buffer with
 * atomicMin (Listing 1) and resolves the winners' colours (Sec. 3.3).
 *
 * Conventions
 *  - Every entry point returns a pc_status (PC_OK = 0, errors < 0); no C++
 *    exception crosses this boundary. pc_last_error() gives the message of the
 *    last failure on a context.
 *  - Sizes are 64-bit. A cloud holds at most 2^32 - 1 points (the point index
 *    is the low 32 bits of a visibility-buffer key).
 *  - "host" pointers are ordinary CPU memory (pinned or pageable); "device"
 *    pointers are CUDA global memory on the context's device (for example the
 *    data_ptr() of a torch CUDA tensor). Streams are cudaStream_t values passed
 *    as void*; NULL is the legacy default stream.
 *  - Device work never traps and never waits without a bound: anomalies set a
 *    device error flag that the next synchronizing call reports as PC_EDEVICE.
 *  - Matrices are 4x4 float, column-major: clip = M * (x, y, z, 1), element
 *    (row r, column c) at view_proj[r + 4c]; w_clip > 0 in front of the camera.
 *  - Pixel (px, py) of a width x height view is element py * width + px, row 0
 *    at the bottom (ndc y = -1).
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pc_status;
#define PC_OK         0
#define PC_EINVAL    -1   /* bad argument (null pointer, size out of range) */
#define PC_ENOMEM    -2   /* host or device allocation failed */
#define PC_ENOTFOUND -3   /* unknown cloud handle or ticket */
#define PC_EBUSY     -4   /* admission refused: no view slot or framebuffer memory */
#define PC_ETIMEDOUT -5   /* pc_poll: the request did not finish in time */
#define PC_ECUDA     -6   /* a CUDA runtime call failed */
#define PC_ENOTSUP   -7   /* operation not supported for this cloud or device */
#define PC_EDEVICE   -8   /* a kernel raised its error flag (see pc_last_error) */

typedef struct pc_ctx pc_ctx;
typedef uint64_t pc_cloud;    /* 0 is never a valid handle */
typedef uint64_t pc_ticket;   /* 0 is never a valid ticket */

/* ---- configuration ------------------------------------------------------ */

#define PC_CFG_TIMING 1u      /* record per-pass CUDA events in pc_render */
#define PC_CFG_GRAPHS 2u      /* replay each frame's kernels as a captured CUDA graph
                                 (updated in place when the views change) */
#define PC_CFG_KEEP_ORDER 4u  /* pc_upload_cloud: batches of consecutive input points,
                                 no Morton sort (the unsorted baseline of Sec. 4.2) */

#define PC_ENCODE_KEEP_ORDER 1u   /* pc_encode flag: skip the Morton sort */

typedef struct {
    uint32_t batch_size;          /* points per batch, multiple of 4 (default 10240, Sec. 3.1) */
    float    precision_px;        /* T: k = 1 if the projected batch extent < T px,
                                     2 if < 1024 T, else 3 (default 512 = 0.5 px per cell
                                     of 1024; the paper's 500 is selectable, Sec. 3.3) */
    uint32_t encoder_threads;     /* host encoder threads, 0 = all cores */
    uint32_t flags;               /* PC_CFG_* */
    uint64_t serve_pool_bytes;    /* device memory for library-owned serving framebuffers
                                     (default 2 GiB) */
    uint32_t serve_streams;       /* CUDA streams of the serving loop (default 4) */
    uint32_t max_views_per_launch;/* views rendered by one raster launch, 1..32 (default 32) */
    uint32_t threads_per_block;   /* raster launch shape; 0 = autotuned */
    uint32_t blocks_per_sm;       /* raster launch shape; 0 = autotuned */
    uint32_t reserved[4];
} pc_config;

/* Fill cfg with the defaults listed above. */
void pc_config_default(pc_config* cfg);

/* ---- data layout (Sec. 3.1, Fig. "batches", Listing 2) ------------------- */

/* One batch: binary32 box (min corner, size = max - min), index of the first
 * point in the encoded buffers and number of points. 32 bytes. */
typedef struct {
    float    min[3];
    float    size[3];
    uint32_t first;
    uint32_t count;
} pc_batch;

/* ---- contexts ------------------------------------------------------------ */

/* Create a context on CUDA device `device` (cfg may be NULL for defaults).
 * Allocates the context's scratch memory. *out receives the context. */
pc_status pc_create(pc_ctx** out, int device, const pc_config* cfg);

/* Release every cloud, ticket and buffer of the context (waits for its work). */
void pc_destroy(pc_ctx* ctx);

/* Static text for a status code. */
const char* pc_strerror(pc_status s);

/* Message of the last failure on ctx (empty string if none). Owned by ctx. */
const char* pc_last_error(pc_ctx* ctx);

/* ---- encoding and upload (Sec. 3.1, Eq. 1, Listing 2) -------------------- */

/* Host encoder, alone (no GPU needed). Sorts the n points of xyz (host, n*3
 * floats, x y z per point) by 63-bit Morton code over the cloud's box (21 bits
 * per axis, binary64, ties keep input order; skipped with PC_ENCODE_KEEP_ORDER
 * in flags), cuts them into batches of
 * batch_size consecutive points, computes each batch's binary32 box and writes
 * Eq. 1's 30-bit coordinates split into three words per point. Outputs (host,
 * caller-allocated): batches[ceil(n / batch_size)], w1/w2/w3/color[n] in sorted
 * order, perm[n] (sorted position -> input index; may be NULL). rgba may be NULL
 * (colour 0). threads = 0 uses all cores. PC_EINVAL if n >= 2^32, batch_size
 * is 0 or not a multiple of 4, or a coordinate is a NaN or an infinity (Eq. 1
 * needs finite boxes). */
pc_status pc_encode(const float* xyz, const uint32_t* rgba, uint64_t n,
                    uint32_t batch_size, uint32_t threads, uint32_t flags, pc_batch* batches,
                    uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color,
                    uint32_t* perm);

/* Encode host points (as pc_encode, batch size and PC_CFG_KEEP_ORDER from the
 * context's config) and
 * upload the cloud to device memory owned by the library. Synchronous. xyz and
 * rgba are read only during the call. *out receives a cloud handle. */
pc_status pc_upload_cloud(pc_ctx* ctx, const float* xyz, const uint32_t* rgba,
                          uint64_t n, pc_cloud* out);

/* Upload an already encoded cloud (host buffers in the pc_encode layout; the
 * library copies them). Every batch must satisfy first + count <= n. */
pc_status pc_upload_encoded(pc_ctx* ctx, const pc_batch* batches, uint64_t nbatches,
                            const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                            const uint32_t* color, uint64_t n, pc_cloud* out);

typedef struct {
    uint64_t n_points;
    uint64_t n_batches;
    uint64_t device_bytes;   /* device memory held by the cloud */
    uint32_t is_lod;         /* 1 for a cloud made by pc_build_lod */
    uint32_t lod_levels;
} pc_cloud_info;

pc_status pc_cloud_get_info(pc_ctx* ctx, pc_cloud cloud, pc_cloud_info* info);

/* Copy a cloud's device buffers back to host arrays sized as in pc_encode
 * (any pointer may be NULL to skip it). Synchronous. */
pc_status pc_cloud_download(pc_ctx* ctx, pc_cloud cloud, pc_batch* batches,
                            uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color);

/* Free a cloud's device memory (waits for work that uses it). */
pc_status pc_release_cloud(pc_ctx* ctx, pc_cloud cloud);

/* ---- level of detail (Sec. 3.5) ------------------------------------------ */

typedef struct {
    uint32_t max_levels;      /* octree depth limit (default 12) */
    uint32_t max_node_points; /* points per node (default 10240) */
    uint32_t seed;            /* subsampling seed */
    uint32_t reserved;
} pc_lod_opts;

/* Build a layered octree (Sec. 3.5) from a resident cloud: the points are
 * decoded at full precision (k = 3); the root is the cloud's cubic box; a node
 * with more than max_node_points points (depth below max_levels - 1) keeps the
 * max_node_points of smallest priority SplitMix64(seed * 2^32 + index), a
 * uniform subset, and hands the rest to its octant children (additive: each
 * point lives in one node). Each node is a batch on its cube, quantized with
 * Eq. 1 against it. Rendering a LOD cloud draws a node when it is in the
 * frustum, its projected extent is >= the view's lod_px (the root needs only
 * the frustum) and its parent is drawn. *out receives a new cloud; src stays.
 * The host holds copies of the cloud and the tree while it builds (up to 56
 * bytes per point); PC_ENOMEM when they do not fit. */
pc_status pc_build_lod(pc_ctx* ctx, pc_cloud src, const pc_lod_opts* opts, pc_cloud* out);

/* Host LOD builder alone (no GPU needed): the tree pc_build_lod uploads, from
 * host positions xyz (n*3 floats) and colours (may be NULL). Outputs (host,
 * caller-allocated): up to max_nodes nodes (pc_batch on the node's cube,
 * breadth-first order), parent[] (root: 0) and level[] per node, and per LOD
 * point perm (input index), w1/w2/w3 (Eq. 1 against the node cube) and color,
 * n entries each (every input point lands in exactly one node). *n_nodes gets
 * the node count; PC_ENOMEM when it exceeds max_nodes (n always suffices).
 * PC_EINVAL if a coordinate is a NaN or an infinity. */
pc_status pc_lod_encode(const float* xyz, const uint32_t* rgba, uint64_t n,
                        const pc_lod_opts* opts, uint32_t threads, uint64_t max_nodes,
                        pc_batch* nodes, uint32_t* parent, uint32_t* level, uint64_t* n_nodes,
                        uint32_t* perm, uint32_t* w1, uint32_t* w2, uint32_t* w3,
                        uint32_t* color);

/* ---- rendering (Sec. 3.2-3.3, Sec. 3.7) ---------------------------------- */

#define PC_VIEW_CULL           1u          /* batch frustum culling (Sec. 3.2) */
#define PC_VIEW_NO_EARLY_DEPTH 2u          /* skip the non-atomic depth pre-test */
#define PC_VIEW_FORCE_K(k)     (((uint32_t)(k) & 3u) << 4)  /* 1..3: fixed precision */
#define PC_VIEW_K_MASK         0x30u
#define PC_VIEW_DILATE         0x40u       /* depth-aware dilation in the resolve (Sec. 3.7):
                                              each pixel shows the closest point within 3x3,
                                              5x5 or 7x7 pixels by its ring (see lod_px_periphery) */
#define PC_VIEW_HQS            0x80u       /* high-quality shading (Sec. 3.6): after the depth pass
                                              a colour pass sums R, G, B and a count per pixel over
                                              the points with w <= fl(w_min * 1.01f), two 64-bit
                                              atomic adds per point into 32-bit sums, and the
                                              resolve writes the per-channel average (rounded
                                              down) with alpha 255. Exact up to 16,843,009 points
                                              per pixel; beyond, the resolve raises the device
                                              error flag (PC_EDEVICE) */
#define PC_VIEW_SIGNED_EMPTY   0x200u      /* pixels no point reached hold 2^63 - 1 instead of
                                              2^64 - 1, so that a signed 64-bit minimum (MPI or
                                              torch.distributed MIN on int64) merges shards
                                              exactly: every point's key is below 2^63 */
#define PC_VIEW_HQS_PACKED     0x100u      /* the same with one 64-bit atomic add per point into
                                              18-bit sums and a 10-bit count; a pixel that gets
                                              more than 1023 points is summed again by a second
                                              pass with two atomics per point, so the image is
                                              exact in every case (the second pass returns at
                                              once when no pixel overflowed). Set alone or with
                                              PC_VIEW_HQS; takes precedence, except for a cloud
                                              of more than 256 points per pixel of the view,
                                              where two-word sums are used (faster there; the
                                              image is the same) */

typedef struct {
    float    view_proj[16];   /* world -> clip, column-major; finite (a NaN or an infinity
                                 gives an unspecified image, never a write outside the
                                 framebuffers: every pixel index is bounds-checked) */
    uint32_t width, height;   /* 1..16384 */
    uint32_t flags;           /* PC_VIEW_* */
    float    lod_px;          /* LOD clouds: node threshold in px (Sec. 3.5); 0 = all nodes */
    float    lod_px_periphery;/* > 0: foveated thresholds (Sec. 3.7) by the ring of the node's
                                 projected centre: lod_px within a third of the half-diagonal
                                 from the view centre, the mean of both within two thirds,
                                 lod_px_periphery beyond; 0: lod_px everywhere */
    uint32_t reserved[3];
} pc_view;

/* Caller-owned device framebuffer of one view: vis[width*height] (uint64 keys)
 * and rgba[width*height] (R | G<<8 | B<<16 | A<<24, 0 where no point landed).
 * rgba may be NULL to skip the resolve. Both 16-byte aligned. Views with
 * PC_VIEW_HQS or PC_VIEW_HQS_PACKED also use a per-pixel sum buffer (16 or
 * 32 bytes per pixel) that the library owns, one per stream, sized to the
 * largest launch group of views seen. */
typedef struct {
    uint64_t* vis;
    uint32_t* rgba;
} pc_framebuffer;

/* Render nviews (1..256) views of a cloud, stream-ordered and asynchronous:
 * per view, clear vis to all ones, cull and choose precision per batch, raster
 * every point of the surviving batches into vis with atomicMin on
 * (bits(w_clip) << 32 | index), then resolve rgba. Views are rendered by
 * multi-view launches of up to max_views_per_launch views that read each
 * batch's coordinate words once (Sec. 3.7). The result is bit-identical to
 * rendering each view alone. Calls sharing a context may use different
 * streams; each stream gets its own scratch. */
pc_status pc_render(pc_ctx* ctx, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                    const pc_framebuffer* fbs, void* stream);

/* Allocation-free variant of the render path (this entry point has no
 * counterpart in the paper; it exists for callers of this library that must not
 * allocate device memory: code that runs while another thread captures a CUDA
 * graph in global mode, where cudaMalloc is refused; plug-ins whose host
 * application owns every device allocation through its own allocator; render
 * loops that fix their memory at start-up). It renders one view of an encoded
 * cloud held in caller-owned device buffers (the pc_encode layout: batches,
 * w1/w2/w3/color with room for a multiple of 4 words, all 16-byte aligned) into
 * caller-owned vis and rgba (rgba may be NULL), stream-ordered and
 * asynchronous, with precision threshold precision_px (512 is the default of
 * pc_config). It allocates nothing: its scratch (draw list, counters) is a
 * static device array of about 4 MB that every GPU loading the library holds
 * until the process exits, so a cloud may have at most
 * 131,072 - n_points / 2^20 - 1 batches; larger ones get PC_EINVAL, as do
 * missing buffers and any buffer (batches included) that is not 16-byte
 * aligned, all refused on the host before anything is launched; views with
 * high-quality shading get PC_ENOTSUP (their sum buffer would need memory).
 * device_error (host memory, two words, may be NULL): the call ends by copying
 * the kernels' error flag and its value there, stream-ordered; once the stream
 * has reached that point, a nonzero first word means the image is not valid
 * (a batch outside the point buffers, batches that overlap so that the draw
 * list overflows). Pinned memory keeps the copy asynchronous; pageable memory
 * makes the call wait for the stream and cannot be used during a capture.
 * The first call on a device looks up that
 * array's device address (a runtime call, no allocation) and keeps it for the
 * life of the process; make that first call before any stream capture, and do
 * not reset the device (cudaDeviceReset) after it. All calls share the array and reset its
 * counters, so calls that overlap on the GPU (different streams, or different
 * host threads without ordering) race and corrupt each other's results. */
pc_status pc_render_noalloc(const pc_batch* batches, uint64_t nbatches,
                            const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                            const uint32_t* color, uint64_t n_points, const pc_view* view,
                            uint64_t* vis, uint32_t* rgba, float precision_px,
                            uint32_t* device_error, void* stream);

/* Render one shard of a frame: as pc_render, but only batches
 * [first_batch, first_batch + batch_count) of the cloud (Sec. 3.2: batches are
 * drawn independently). Frames split into disjoint ranges merge exactly by the
 * element-wise minimum of their visibility buffers (pc_merge_min, or a MIN
 * reduction across GPUs with PC_VIEW_SIGNED_EMPTY), after which pc_resolve
 * writes the image; rgba may be NULL here to skip each shard's own resolve.
 * Plain clouds only (PC_ENOTSUP for LOD clouds and high-quality shading);
 * PC_EINVAL for an empty range or one outside the cloud. */
pc_status pc_render_range(pc_ctx* ctx, pc_cloud cloud, uint64_t first_batch,
                          uint64_t batch_count, const pc_view* views, uint32_t nviews,
                          const pc_framebuffer* fbs, void* stream);

/* Resolve visibility buffers that were filled earlier (shards merged by
 * pc_merge_min or by a reduction across GPUs) into their rgba images (required
 * here), stream-ordered: the colour of each pixel's key, 0 where the pixel holds
 * the empty key of its view's flags; PC_VIEW_DILATE applies. */
pc_status pc_resolve(pc_ctx* ctx, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                     const pc_framebuffer* fbs, void* stream);

/* dst[i] = min(dst[i], src[i]) for n visibility keys (device, 16-byte aligned,
 * unsigned compare), stream-ordered: merges two shards of one frame rendered
 * with the same empty key. PC_EINVAL for null or misaligned buffers. */
pc_status pc_merge_min(uint64_t* dst, const uint64_t* src, uint64_t n, void* stream);

/* End-to-end variant: renders into library-owned device framebuffers and
 * copies each view's RGBA image into host_rgba[v] (host, width*height
 * uint32). Returns when the host images are complete. */
pc_status pc_render_host(pc_ctx* ctx, pc_cloud cloud, const pc_view* views,
                         uint32_t nviews, uint32_t* const* host_rgba, void* stream);

/* Per-view counters of the last pc_render on `stream` of this context
 * (synchronizes that stream). Mirrors Table 2's processed nodes and points. */
typedef struct {
    uint64_t batches_total;
    uint64_t batches_rendered;     /* passed culling (and LOD selection) */
    uint64_t batches_k[4];         /* rendered batches per precision k (index 1..3) */
    uint64_t points_k[4];          /* their points */
    uint64_t points_processed;     /* sum of points_k */
    uint64_t words_loaded_bytes;   /* coordinate bytes the raster launch loaded for this view */
    uint64_t points_atomic;        /* points that issued atomicMin (Table 2 "rendered points") */
    uint64_t points_blended;       /* high-quality shading: points summed into a pixel */
    uint64_t hqs_fallback_pixels;  /* PC_VIEW_HQS_PACKED: pixels summed by the second pass */
} pc_view_stats;

pc_status pc_get_view_stats(pc_ctx* ctx, void* stream, uint32_t view, pc_view_stats* out);

/* ---- autotuner ------------------------------------------------------------- */

typedef struct {
    uint32_t threads_per_block;   /* raster block size chosen */
    uint32_t blocks_per_sm;       /* resident raster blocks per SM chosen */
    uint32_t points_per_warp;     /* points a raster warp takes per grab (points per
                                     thread = points_per_warp / 32) */
    uint32_t views_per_launch;    /* views rendered by one launch (multi-view) */
    double   ms_per_view;         /* best time per view measured */
    double   ms_per_view_single;  /* time per view at one view per launch, same shape */
    uint32_t candidates;          /* configurations timed */
    uint32_t reserved;
} pc_tune_result;

/* Time candidate raster launch shapes (threads per block, blocks per SM,
 * points per warp grab) on views[0], then candidate views per launch on all
 * nviews views, all on `stream` with library-owned framebuffers, and keep the
 * fastest for later pc_render and serving launches of this cloud (a small
 * cloud gains from many views per launch, a large one may not): the launch
 * shape (fields set in pc_config override it) and the views per launch
 * (unless pc_set_views_per_launch has set one for the context). Results are identical for every candidate; only
 * the time differs. Synchronous. Renders and serving groups that other threads
 * launch on this context meanwhile stay correct but take the candidate being
 * timed, and their time skews the measurement: tune on an idle context. */
pc_status pc_autotune(pc_ctx* ctx, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                      void* stream, pc_tune_result* out);

/* Set the views rendered by one launch (1..32) for later pc_render calls and
 * serving groups of every cloud on this context, in place of the autotuner's
 * per-cloud choices; 1 gives one view per launch, 0 goes back to the per-cloud
 * choices (the configured maximum for clouds never tuned). */
pc_status pc_set_views_per_launch(pc_ctx* ctx, uint32_t views_per_launch);

/* ---- timing (per-pass CUDA events) --------------------------------------- */

typedef struct {
    uint32_t frames;            /* pc_render calls recorded */
    uint32_t launches;          /* kernels launched by those calls */
    double   ms_clear, ms_cull, ms_raster, ms_shade, ms_resolve;  /* summed over frames;
                                   ms_shade: the colour pass of high-quality shading */
    uint64_t raster_launches;
} pc_timing;

/* Start recording per-pass events for pc_render on this context (needs
 * PC_CFG_TIMING or enables it), discarding earlier records. */
pc_status pc_timing_begin(pc_ctx* ctx);
/* Synchronize the recorded events and sum them. */
pc_status pc_timing_end(pc_ctx* ctx, pc_timing* out);

/* ---- serving loop ---------------------------------------------------------- */

typedef struct {
    pc_status status;         /* PC_OK or the failure of this request */
    uint32_t  nviews;
    uint32_t* const* rgba;    /* host images, one per view, owned by the context
                                 until pc_release_ticket; NULL for requests with
                                 caller-owned framebuffers */
    const uint32_t* widths;
    const uint32_t* heights;
    double    t_submit_ms, t_start_ms, t_done_ms;   /* steady clock, ms since ctx creation */
} pc_result;

/* Queue a request: nviews (1..32) views of a resident cloud. Requests that
 * arrive while others run join the next launch group of the same cloud.
 * fbs == NULL: the library owns the framebuffers (admitted when
 * serve_pool_bytes has room and a view slot is free) and returns host RGBA
 * images through pc_poll; PC_EBUSY when the request can never fit the pool
 * or the pinned image memory is full.
 * fbs != NULL: nviews caller-owned device framebuffers (as for pc_render,
 * 16-byte aligned, vis required); nothing is admitted or copied to the host,
 * the images are in fbs once pc_poll reports the request done, and the caller
 * must not use them before. */
pc_status pc_submit(pc_ctx* ctx, pc_cloud cloud, const pc_view* views, uint32_t nviews,
                    const pc_framebuffer* fbs, pc_ticket* out);

/* Wait up to timeout_ms for a request: 0 = just test; values above 60000 wait
 * 60000 ms, so a call never blocks longer than a minute, even when the
 * request's stream never finishes; a negative timeout is PC_EINVAL.
 * PC_ETIMEDOUT if it has not finished; on PC_OK *out describes the result. */
pc_status pc_poll(pc_ctx* ctx, pc_ticket ticket, int32_t timeout_ms, pc_result* out);

/* Free a finished request's host images. */
pc_status pc_release_ticket(pc_ctx* ctx, pc_ticket ticket);

#ifdef __cplusplus
}
#endif
#endif /* PC_H */

/* pcr_oracle.h — plain, slow CPU oracle for one-pixel point rasterization of
 * batched, adaptively quantized point clouds (Schuetz, Kerbl, Wimmer,
 * "Software Rasterization of 2 Billion Points in Real Time", 2022).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline
 * leg of the benchmark use it to check the GPU library; the library never
 * calls it and shares no code with it.
 *
 * Compiled with -ffp-contract=off: every float operation below is one IEEE
 * binary32 (or binary64 where stated) operation rounded to nearest, in the
 * order written.
 */
#ifndef PCR_ORACLE_H
#define PCR_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* One batch (Sec. 3.1): bounding box (min corner and size, binary32), index of
 * its first point in the encoded buffers and its number of points. */
typedef struct {
    float min[3];
    float size[3];
    uint32_t first;
    uint32_t count;
} or_batch;

/* One camera view. m is the 4x4 world-to-clip matrix, column-major
 * (clip = m * (x,y,z,1), element (row r, column c) at m[r + 4c]). */
typedef struct {
    float m[16];
    uint32_t width, height;
    int cull;            /* 1: batch frustum culling (Sec. 3.2) */
    int force_k;         /* 0: adaptive precision (Sec. 3.3); 1..3: forced */
    float threshold_px;  /* k = 1 if extent < T, 2 if extent < 1024 T, else 3 */
} or_view;

typedef struct {
    uint64_t batches_rendered;   /* batches that passed culling */
    uint64_t points_processed;   /* points of those batches */
    uint64_t batches_k[4];       /* rendered batches per precision k */
    uint64_t points_k[4];
    uint64_t points_accepted;    /* points that landed inside the viewport */
} or_stats;

#define OR_EMPTY 0xFFFFFFFFFFFFFFFFull

/* Eq. 1: 30-bit fixed-point coordinate relative to the batch box. */
uint32_t or_quantize30(float v, float box_min, float box_size);

/* Listing 2 and Sec. 3.3: split three 30-bit coordinates into the low (bits
 * 20-29), medium (10-19) and high (0-9) precision words, each packing
 * x | y << 10 | z << 20. */
void or_split_words(uint32_t X30, uint32_t Y30, uint32_t Z30, uint32_t w[3]);

/* Sec. 3.3: the k-word (10k-bit) integer coordinates of a point: the first k
 * words concatenated from the most significant part down. out[a] < 2^(10k). */
void or_decode_words(uint32_t w1, uint32_t w2, uint32_t w3, int k, uint32_t out[3]);

/* Sec. 3.1: 63-bit Morton code (21 bits per axis, x in the lowest bit of each
 * triple) of p over the cloud box (cmin, csize), computed in binary64. */
uint64_t or_morton_code(const float p[3], const double cmin[3], const double csize[3]);

/* Number of batches for n points and batch_size points per batch. */
uint64_t or_num_batches(uint64_t n, uint32_t batch_size);

/* Sec. 3.1 and 3.3: Morton-sort the cloud (stable: ties keep input order),
 * cut it into batches of batch_size consecutive points, compute each batch's
 * binary32 box and write the three coordinate words and the colour of every
 * point in sorted order. perm[j] = input index of sorted point j. */
int or_encode(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
              uint32_t* perm, or_batch* batches, uint32_t* w1, uint32_t* w2,
              uint32_t* w3, uint32_t* color);

/* The same without the Morton sort: batches of consecutive input points
 * (the unsorted baseline of Sec. 4.2). */
int or_encode_in_order(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
                       or_batch* batches, uint32_t* w1, uint32_t* w2, uint32_t* w3,
                       uint32_t* color);

/* Listing 1: project one world position. Returns 1 and writes the pixel id
 * (py * width + px) and the 64-bit key (bits of w_clip << 32 | idx) when the
 * point lands in the viewport, else 0. When fxy is not NULL it receives the
 * unfloored pixel coordinates. */
int or_project_position(const float p[3], const or_view* v, uint32_t idx,
                        uint32_t* pixel, uint64_t* key, float fxy[2]);

/* Decode point idx of batch b at precision k (Sec. 3.3) and project it. */
int or_project_point(const or_batch* b, int k, uint32_t w1, uint32_t w2, uint32_t w3,
                     uint32_t idx, const or_view* v, uint32_t* pixel, uint64_t* key);

/* The position a point decodes to at precision k (Sec. 3.3). */
void or_decode_position(const or_batch* b, int k, uint32_t w1, uint32_t w2,
                        uint32_t w3, float p[3]);

/* Sec. 3.3: precision of a batch in a view, from its projected extent. */
int or_select_k(const or_batch* b, const or_view* v);

/* Decoded positions of every point of an encoded cloud at precision k. */
void or_decode_cloud(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                     const uint32_t* w2, const uint32_t* w3, int k, float* xyz);

/* Sec. 3.2: 1 if no point of the batch can land in the viewport. */
int or_cull(const or_batch* b, const or_view* v);

/* Sec. 3.2-3.3 geometry pass: vis[W*H] <- min key per pixel. vis is cleared
 * first. order (may be NULL) lists the batch indices in processing order. */
void or_render(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
               const uint32_t* w2, const uint32_t* w3, const or_view* v,
               const uint64_t* order, uint64_t* vis, or_stats* st);

/* The same on `threads` threads, each with a private visibility buffer that
 * is merged by element-wise minimum. */
void or_render_threaded(const or_batch* batches, uint64_t nbatches,
                        const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                        const or_view* v, int threads, uint64_t* vis, or_stats* st);

/* Unquantized image: every float position projected directly, key index = i. */
void or_render_positions(const float* xyz, uint64_t n, const or_view* v, uint64_t* vis);

/* Brute force: for every pixel, search every point of every batch for the
 * smallest key that lands on that pixel (no culling). O(pixels * points). */
void or_brute_force(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                    const uint32_t* w2, const uint32_t* w3, const or_view* v,
                    uint64_t* vis);

/* ---- Sec. 3.5 level of detail ------------------------------------------- */

/* Projected extent of a batch box in a view: max over x and y of the spread
 * of the 8 corners' unfloored pixel coordinates (the same binary32 operations
 * as a point). Returns 0 and leaves *extent unset when a corner has w <= 0. */
int or_projected_extent(const or_batch* b, const or_view* v, float* extent);

/* SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014). */
uint64_t or_splitmix64(uint64_t z);

/* Number of LOD nodes or_lod_build would create (first pass), or -1. */
int64_t or_lod_count_nodes(const float* xyz, uint64_t n, uint32_t max_levels,
                           uint32_t max_node_points, uint32_t seed);

/* Sec. 3.5 layered octree, additive: the root is the cubic box of the cloud;
 * a node with more than max_node_points points (and depth below max_levels-1)
 * keeps the max_node_points points of smallest priority SplitMix64(seed*2^32 +
 * index) (a uniform subset; ties by index) and hands the rest to its 8 octant
 * children; other nodes keep all their points. Nodes are numbered breadth
 * first, children in octant order (bit 0 = x upper half, bit 1 = y, bit 2 = z).
 * Each node is one batch on its cubic box (min = cube corner, size = cube side
 * on all axes) whose points (in input order) are quantized with Eq. 1 against
 * that box. perm[j] = input index of LOD point j. Returns the number of nodes. */
int64_t or_lod_build(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t max_levels,
                     uint32_t max_node_points, uint32_t seed, or_batch* nodes,
                     uint32_t* parent, uint32_t* level, uint32_t* perm, uint32_t* w1,
                     uint32_t* w2, uint32_t* w3, uint32_t* color);

/* Sec. 3.7 rings of a screen position (x, y) in pixels: 0 within a third of
 * the half-diagonal from the view centre, 1 within two thirds, else 2;
 * binary32: d2 = dx*dx + dy*dy, R2 = (W/2)^2 + (H/2)^2, ring 0 iff 9 d2 < R2,
 * ring 1 iff 9 d2 < 4 R2. */
int or_ring(float x, float y, uint32_t width, uint32_t height);

/* Sec. 3.5 node selection: node n is drawn when it is in the frustum (the
 * culling test of Sec. 3.2), its projected extent is at least its threshold
 * (any corner with w <= 0 counts as large; the root needs only the frustum
 * test), and its parent is drawn. The threshold is lod_px, or with
 * lod_px_periphery > 0 (Sec. 3.7 foveation) lod_px in ring 0,
 * (lod_px + lod_px_periphery) * 0.5 in ring 1 and lod_px_periphery in ring 2,
 * the ring of the centre of the node's projected corner box. sel[n] = 1 for
 * drawn nodes. Nodes must be in breadth-first order (parents first). */
void or_lod_select(const or_batch* nodes, const uint32_t* parent, uint64_t nnodes,
                   const or_view* v, float lod_px, float lod_px_periphery, uint8_t* sel);

/* Geometry pass over the drawn nodes of a LOD cloud. */
void or_lod_render(const or_batch* nodes, const uint32_t* parent, uint64_t nnodes,
                   const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                   const or_view* v, float lod_px, float lod_px_periphery, uint64_t* vis,
                   or_stats* st);

/* Sec. 3.7 depth-aware dilation: every pixel shows the colour of the smallest
 * key (the closest point) within a (2r+1) x (2r+1) window, r = 1, 2, 3 in
 * rings 0, 1, 2 of the pixel centre (px + 0.5, py + 0.5); 0 where the window
 * is empty. */
void or_resolve_dilated(const uint64_t* vis, uint32_t width, uint32_t height,
                        const uint32_t* color, uint32_t* out);

/* Sec. 3.6 high-quality shading: after the geometry pass (vis), every point
 * that lands on pixel p (same batches, culling, precision and projection as
 * or_render) with w <= fl(w_min * 1.01), w_min the depth of vis[p], adds its
 * R, G, B to the pixel's sums and 1 to its count; out[p] = (floor(sumR/n),
 * floor(sumG/n), floor(sumB/n), 255), 0 where no point landed. */
void or_render_hqs(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                   const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                   const or_view* v, const uint64_t* vis, uint32_t* out);

/* The same on `threads` threads, each summing a range of batches; the integer
 * sums of the threads are added before the average. */
void or_render_hqs_threaded(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                            const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                            const or_view* v, const uint64_t* vis, int threads, uint32_t* out);

/* or_render_hqs for a LOD cloud: the points of the nodes that or_lod_select
 * keeps, each node at its own precision. */
void or_lod_render_hqs(const or_batch* nodes, const uint32_t* parent, uint64_t nnodes,
                       const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                       const uint32_t* color, const or_view* v, float lod_px,
                       float lod_px_periphery, const uint64_t* vis, uint32_t* out);

/* Depth-aware dilation (Sec. 3.7) of a high-quality shading image: out[p] is
 * hqs[q] of the pixel q holding the smallest key within the window of
 * or_resolve_dilated around p, 0 where the window is empty. */
void or_hqs_resolve_dilated(const uint64_t* vis, uint32_t width, uint32_t height,
                            const uint32_t* hqs, uint32_t* out);

/* Check an encoding of n points against Sec. 3.1, Eq. 1 and Listing 2, in
 * O(n) on `threads` threads: perm must be a permutation that sorts the Morton
 * codes (over the cloud box) with ties in input order, batches must be the
 * consecutive runs of batch_size sorted points with their binary32 boxes,
 * and w1/w2/w3/color the split Eq. 1 coordinates and colours. The encoding
 * is unique, so one that passes equals or_encode's. Returns 0, or the first
 * failure found: 1 batch count/header, 2 not a permutation, 3 order, 4 box,
 * 5 words, 6 colour, with its index (sorted position or batch) in *where;
 * -2 when out of memory. */
int or_verify_encoding(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
                       const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                       const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                       const uint32_t* perm, int threads, uint64_t* where);

/* Check a LOD tree of n input points against Sec. 3.5 as or_lod_build builds
 * it, in O(n * depth) on `threads` threads: the root cube (the points' corner
 * and largest extent), breadth-first numbering with each child the cube of
 * its octant (children in octant order), every point routed down the octants
 * of all its ancestors, the split rule (a node keeps max_node_points points
 * and has children exactly when it held more and is above the last level),
 * every own point of a node before every point below it in (SplitMix64
 * priority, index) order, input order within a node, a permutation, and Eq. 1
 * against the node cube with Listing 2 and the colours. The tree is unique, so
 * one that passes is or_lod_build's. Returns 0, or the first failure found:
 * 1 header/root, 2 structure, 3 permutation/order, 4 octant, 5 split or
 * priority rule, 6 words, 7 colour, with its node or point in *where; -2 when
 * out of memory. */
int or_verify_lod(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t max_levels,
                  uint32_t max_node_points, uint32_t seed, const or_batch* nodes,
                  const uint32_t* parent, const uint32_t* level, uint64_t nnodes,
                  const uint32_t* perm, const uint32_t* w1, const uint32_t* w2,
                  const uint32_t* w3, const uint32_t* color, int threads, uint64_t* where);

/* Sec. 3.3 visibility buffer: out[p] = colour of the winning point, 0 where
 * no point landed. */
void or_resolve(const uint64_t* vis, uint64_t npixels, const uint32_t* color,
                uint32_t* out);

#ifdef __cplusplus
}
#endif
#endif

/* pcr_oracle.c — plain, slow CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Restates, step by step and without any blocking, fusion or reordering, what
 * the rasterizer of Schuetz, Kerbl and Wimmer (2022) computes:
 *   Sec. 3.1   Morton order, batches of consecutive points, batch boxes;
 *   Eq. 1      30-bit coordinates relative to the batch box;
 *   Listing 2  three 10-bit-per-axis coordinate words;
 *   Sec. 3.3   precision k chosen from the projected batch extent;
 *   Sec. 3.2   batch frustum culling;
 *   Listing 1  projection, 64-bit (depth bits << 32 | index) key, minimum;
 *   Sec. 3.3   visibility buffer resolved to colours.
 * Where the paper leaves the arithmetic open the readings are:
 *   decode     x = min + float(Xk) * (size * 2^-10k), binary32;
 *   project    c = ((m0 x + m4 y) + m8 z) + m12 per row, binary32, no FMA;
 *   pixel      f = ((c / w) * 0.5 + 0.5) * W with an IEEE divide, accepted iff
 *              w > 0 and 0 <= f < W, px = floor(f); row 0 at the bottom;
 *   ties       the smaller key wins, so equal depths go to the smaller index;
 *   precision  k = 1 if the extent of the 8 projected box corners is below
 *              T = 512 px (0.5 px per cell of 1024), 2 if below 1024 T, else 3,
 *              and 3 whenever a corner has w <= 0;
 *   culling    conservative: a batch is dropped only when a rigorous rounding
 *              bound proves every decoded point is rejected by one clip plane.
 * Parity pins live in tests/test_oracle_*.py.
 */
#include "pcr_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---- Eq. 1 and Listing 2 ------------------------------------------------- */

uint32_t or_quantize30(float v, float box_min, float box_size) {
    /* Eq. 1, evaluated in binary64 from the binary32 inputs; a zero-size box
     * maps every point to 0; the result is clamped to 2^30 - 1 as printed. */
    if (!(box_size > 0.0f)) return 0;
    double t = floor(1073741824.0 * ((double)v - (double)box_min) / (double)box_size);
    if (t < 0.0) t = 0.0;
    if (t > 1073741823.0) t = 1073741823.0;
    return (uint32_t)t;
}

void or_split_words(uint32_t X30, uint32_t Y30, uint32_t Z30, uint32_t w[3]) {
    /* word 0 = low precision = bits 20..29, word 1 = medium = bits 10..19,
     * word 2 = high = bits 0..9; each packs x | y << 10 | z << 20 */
    for (int j = 0; j < 3; ++j) {
        int shift = 20 - 10 * j;
        uint32_t xs = (X30 >> shift) & 1023u;
        uint32_t ys = (Y30 >> shift) & 1023u;
        uint32_t zs = (Z30 >> shift) & 1023u;
        w[j] = xs | (ys << 10) | (zs << 20);
    }
}

void or_decode_words(uint32_t w1, uint32_t w2, uint32_t w3, int k, uint32_t out[3]) {
    uint32_t words[3] = {w1, w2, w3};
    for (int a = 0; a < 3; ++a) {
        uint32_t v = 0;
        for (int j = 0; j < k; ++j) v = (v << 10) | ((words[j] >> (10 * a)) & 1023u);
        out[a] = v;
    }
}

/* ---- Sec. 3.1: Morton order and batches ---------------------------------- */

uint64_t or_morton_code(const float p[3], const double cmin[3], const double csize[3]) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        double t = 0.0;
        if (csize[a] > 0.0) t = floor(2097152.0 * ((double)p[a] - cmin[a]) / csize[a]);
        if (t < 0.0) t = 0.0;
        if (t > 2097151.0) t = 2097151.0;
        q[a] = (uint32_t)t;
    }
    uint64_t code = 0;
    for (int bit = 0; bit < 21; ++bit)
        for (int a = 0; a < 3; ++a)
            code |= (uint64_t)((q[a] >> bit) & 1u) << (3 * bit + a);
    return code;
}

uint64_t or_num_batches(uint64_t n, uint32_t batch_size) {
    return batch_size ? (n + batch_size - 1) / batch_size : 0;
}

typedef struct { uint64_t code; uint32_t idx; } keyed;

static int keyed_cmp(const void* a, const void* b) {
    const keyed* x = (const keyed*)a;
    const keyed* y = (const keyed*)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

int or_encode(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
              uint32_t* perm, or_batch* batches, uint32_t* w1, uint32_t* w2,
              uint32_t* w3, uint32_t* color) {
    if (batch_size == 0 || n > 0xFFFFFFFFull) return -1;
    if (n == 0) return 0;
    /* cloud box */
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = xyz[a];
    for (uint64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float v = xyz[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double cmin[3], csize[3];
    for (int a = 0; a < 3; ++a) {
        cmin[a] = (double)lo[a];
        csize[a] = (double)hi[a] - (double)lo[a];
    }
    /* stable sort by Morton code */
    keyed* ks = (keyed*)malloc(sizeof(keyed) * n);
    if (!ks) return -2;
    for (uint64_t i = 0; i < n; ++i) {
        ks[i].code = or_morton_code(&xyz[3 * i], cmin, csize);
        ks[i].idx = (uint32_t)i;
    }
    qsort(ks, n, sizeof(keyed), keyed_cmp);
    for (uint64_t j = 0; j < n; ++j) perm[j] = ks[j].idx;
    free(ks);
    /* batches of consecutive sorted points */
    uint64_t nb = or_num_batches(n, batch_size);
    for (uint64_t b = 0; b < nb; ++b) {
        uint64_t first = b * batch_size;
        uint64_t end = first + batch_size < n ? first + batch_size : n;
        float bmin[3], bmax[3];
        for (int a = 0; a < 3; ++a) bmin[a] = bmax[a] = xyz[3 * (uint64_t)perm[first] + a];
        for (uint64_t j = first; j < end; ++j)
            for (int a = 0; a < 3; ++a) {
                float v = xyz[3 * (uint64_t)perm[j] + a];
                if (v < bmin[a]) bmin[a] = v;
                if (v > bmax[a]) bmax[a] = v;
            }
        or_batch* B = &batches[b];
        for (int a = 0; a < 3; ++a) {
            B->min[a] = bmin[a];
            B->size[a] = bmax[a] - bmin[a];   /* binary32 subtraction */
        }
        B->first = (uint32_t)first;
        B->count = (uint32_t)(end - first);
        for (uint64_t j = first; j < end; ++j) {
            const float* p = &xyz[3 * (uint64_t)perm[j]];
            uint32_t X = or_quantize30(p[0], B->min[0], B->size[0]);
            uint32_t Y = or_quantize30(p[1], B->min[1], B->size[1]);
            uint32_t Z = or_quantize30(p[2], B->min[2], B->size[2]);
            uint32_t w[3];
            or_split_words(X, Y, Z, w);
            w1[j] = w[0];
            w2[j] = w[1];
            w3[j] = w[2];
            color[j] = rgba[perm[j]];
        }
    }
    return (int)(nb > 0x7FFFFFFF ? 0x7FFFFFFF : nb);
}

int or_encode_in_order(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
                       or_batch* batches, uint32_t* w1, uint32_t* w2, uint32_t* w3,
                       uint32_t* color) {
    if (batch_size == 0 || n > 0xFFFFFFFFull) return -1;
    uint64_t nb = or_num_batches(n, batch_size);
    for (uint64_t b = 0; b < nb; ++b) {
        uint64_t first = b * batch_size;
        uint64_t end = first + batch_size < n ? first + batch_size : n;
        float bmin[3], bmax[3];
        for (int a = 0; a < 3; ++a) bmin[a] = bmax[a] = xyz[3 * first + a];
        for (uint64_t j = first; j < end; ++j)
            for (int a = 0; a < 3; ++a) {
                float v = xyz[3 * j + a];
                if (v < bmin[a]) bmin[a] = v;
                if (v > bmax[a]) bmax[a] = v;
            }
        or_batch* B = &batches[b];
        for (int a = 0; a < 3; ++a) {
            B->min[a] = bmin[a];
            B->size[a] = bmax[a] - bmin[a];
        }
        B->first = (uint32_t)first;
        B->count = (uint32_t)(end - first);
        for (uint64_t j = first; j < end; ++j) {
            const float* p = &xyz[3 * j];
            uint32_t w[3];
            or_split_words(or_quantize30(p[0], B->min[0], B->size[0]),
                           or_quantize30(p[1], B->min[1], B->size[1]),
                           or_quantize30(p[2], B->min[2], B->size[2]), w);
            w1[j] = w[0];
            w2[j] = w[1];
            w3[j] = w[2];
            color[j] = rgba[j];
        }
    }
    return (int)(nb > 0x7FFFFFFF ? 0x7FFFFFFF : nb);
}

/* ---- Sec. 3.3 decode and Listing 1 projection ---------------------------- */

void or_decode_position(const or_batch* b, int k, uint32_t w1, uint32_t w2,
                        uint32_t w3, float p[3]) {
    uint32_t q[3];
    or_decode_words(w1, w2, w3, k, q);
    for (int a = 0; a < 3; ++a) {
        float cell = ldexpf(b->size[a], -10 * k);   /* exact power-of-two scaling */
        float fq = (float)q[a];                     /* exact for k <= 2, rounded for k = 3 */
        float off = fq * cell;
        p[a] = b->min[a] + off;
    }
}

void or_decode_cloud(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                     const uint32_t* w2, const uint32_t* w3, int k, float* xyz) {
    for (uint64_t b = 0; b < nbatches; ++b)
        for (uint32_t j = 0; j < batches[b].count; ++j) {
            uint64_t i = (uint64_t)batches[b].first + j;
            or_decode_position(&batches[b], k, w1[i], w2[i], w3[i], &xyz[3 * i]);
        }
}

int or_project_position(const float p[3], const or_view* v, uint32_t idx,
                        uint32_t* pixel, uint64_t* key, float fxy[2]) {
    const float* m = v->m;
    float x = p[0], y = p[1], z = p[2];
    float cx = ((m[0] * x + m[4] * y) + m[8] * z) + m[12];
    float cy = ((m[1] * x + m[5] * y) + m[9] * z) + m[13];
    float cw = ((m[3] * x + m[7] * y) + m[11] * z) + m[15];
    if (!(cw > 0.0f)) return 0;
    float ndx = cx / cw;
    float ndy = cy / cw;
    float fx = (ndx * 0.5f + 0.5f) * (float)v->width;
    float fy = (ndy * 0.5f + 0.5f) * (float)v->height;
    if (fxy) { fxy[0] = fx; fxy[1] = fy; }
    if (!(fx >= 0.0f && fx < (float)v->width)) return 0;
    if (!(fy >= 0.0f && fy < (float)v->height)) return 0;
    uint32_t px = (uint32_t)floorf(fx);
    uint32_t py = (uint32_t)floorf(fy);
    uint32_t bits;
    memcpy(&bits, &cw, 4);
    *pixel = py * v->width + px;
    *key = ((uint64_t)bits << 32) | (uint64_t)idx;
    return 1;
}

int or_project_point(const or_batch* b, int k, uint32_t w1, uint32_t w2, uint32_t w3,
                     uint32_t idx, const or_view* v, uint32_t* pixel, uint64_t* key) {
    float p[3];
    or_decode_position(b, k, w1, w2, w3, p);
    return or_project_position(p, v, idx, pixel, key, NULL);
}

/* ---- Sec. 3.3: precision from the projected extent ----------------------- */

int or_select_k(const or_batch* b, const or_view* v) {
    if (v->force_k >= 1 && v->force_k <= 3) return v->force_k;
    float fmin[2] = {0, 0}, fmax[2] = {0, 0};
    for (int c = 0; c < 8; ++c) {
        float p[3];
        for (int a = 0; a < 3; ++a)
            p[a] = ((c >> a) & 1) ? b->min[a] + b->size[a] : b->min[a];
        const float* m = v->m;
        float cw = ((m[3] * p[0] + m[7] * p[1]) + m[11] * p[2]) + m[15];
        if (!(cw > 0.0f)) return 3;
        float f[2];
        uint32_t pix;
        uint64_t key;
        or_project_position(p, v, 0, &pix, &key, f);
        for (int a = 0; a < 2; ++a) {
            if (c == 0 || f[a] < fmin[a]) fmin[a] = f[a];
            if (c == 0 || f[a] > fmax[a]) fmax[a] = f[a];
        }
    }
    float ex = fmax[0] - fmin[0];
    float ey = fmax[1] - fmin[1];
    float T = v->threshold_px;
    if (ex < T && ey < T) return 1;
    float T2 = T * 1024.0f;
    if (ex < T2 && ey < T2) return 2;
    return 3;
}

/* ---- Sec. 3.2: conservative batch frustum culling ------------------------ */

/* Every decoded position lies in [min, fl(min + size)] per axis (rounding is
 * monotonic and float(Xk) * cell <= size). For one matrix row r, the binary32
 * value c computed by or_project_position differs from the exact r.(x,y,z,1)
 * by at most gamma_4 * (|r0 x| + |r1 y| + |r2 z| + |r3|), gamma_4 = 4u/(1-4u),
 * u = 2^-24 (dot-product error bound, Higham, Accuracy and Stability of
 * Numerical Algorithms, 2nd ed., Sec. 3.1). The bound below uses 6u, which
 * also covers the binary64 rounding of this test itself. */

static double row_max(const double r[4], const double lo[3], const double hi[3]) {
    double s = r[3];
    for (int a = 0; a < 3; ++a) s += fmax(r[a] * lo[a], r[a] * hi[a]);
    return s;
}

static double row_min(const double r[4], const double lo[3], const double hi[3]) {
    double s = r[3];
    for (int a = 0; a < 3; ++a) s += fmin(r[a] * lo[a], r[a] * hi[a]);
    return s;
}

static double row_mag(const double r[4], const double lo[3], const double hi[3]) {
    double s = fabs(r[3]);
    for (int a = 0; a < 3; ++a) s += fabs(r[a]) * fmax(fabs(lo[a]), fabs(hi[a]));
    return s;
}

int or_cull(const or_batch* b, const or_view* v) {
    const double g = 6.0 * 0x1.0p-24;    /* rounding bound factor */
    const double e1 = 1.0 + 0x1.0p-10;   /* clip-plane margin 1 + 2^-10 */
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)b->min[a];
        hi[a] = (double)(float)(b->min[a] + b->size[a]);
    }
    const float* m = v->m;
    double X[4] = {m[0], m[4], m[8], m[12]};
    double Y[4] = {m[1], m[5], m[9], m[13]};
    double Wr[4] = {m[3], m[7], m[11], m[15]};
    double bx = row_mag(X, lo, hi), by = row_mag(Y, lo, hi), bw = row_mag(Wr, lo, hi);
    if (!isfinite(bx) || !isfinite(by) || !isfinite(bw)) return 0;
    /* every point has w <= 0 */
    if (row_max(Wr, lo, hi) + g * bw <= 0.0) return 1;
    double sp[4], sm[4];
    /* x: left of -w and right of +w, each with margin 1 + 2^-10 */
    for (int a = 0; a < 4; ++a) { sp[a] = X[a] + e1 * Wr[a]; sm[a] = X[a] - e1 * Wr[a]; }
    double mx = g * (bx + e1 * bw);
    if (row_max(sp, lo, hi) + mx < 0.0) return 1;
    if (row_min(sm, lo, hi) - mx > 0.0) return 1;
    for (int a = 0; a < 4; ++a) { sp[a] = Y[a] + e1 * Wr[a]; sm[a] = Y[a] - e1 * Wr[a]; }
    double my = g * (by + e1 * bw);
    if (row_max(sp, lo, hi) + my < 0.0) return 1;
    if (row_min(sm, lo, hi) - my > 0.0) return 1;
    return 0;
}

/* ---- geometry pass (Listing 1 over all batches) -------------------------- */

static void render_range(const or_batch* batches, uint64_t lo, uint64_t hi,
                         const uint64_t* order, const uint32_t* w1, const uint32_t* w2,
                         const uint32_t* w3, const or_view* v, uint64_t* vis,
                         or_stats* st) {
    for (uint64_t t = lo; t < hi; ++t) {
        const or_batch* b = &batches[order ? order[t] : t];
        if (v->cull && or_cull(b, v)) continue;
        int k = or_select_k(b, v);
        if (st) {
            st->batches_rendered += 1;
            st->points_processed += b->count;
            st->batches_k[k] += 1;
            st->points_k[k] += b->count;
        }
        for (uint32_t j = 0; j < b->count; ++j) {
            uint32_t i = b->first + j;
            uint32_t pix;
            uint64_t key;
            if (!or_project_point(b, k, w1[i], w2[i], w3[i], i, v, &pix, &key)) continue;
            if (st) st->points_accepted += 1;
            if (key < vis[pix]) vis[pix] = key;
        }
    }
}

void or_render(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
               const uint32_t* w2, const uint32_t* w3, const or_view* v,
               const uint64_t* order, uint64_t* vis, or_stats* st) {
    uint64_t npix = (uint64_t)v->width * v->height;
    for (uint64_t p = 0; p < npix; ++p) vis[p] = OR_EMPTY;
    if (st) memset(st, 0, sizeof(*st));
    render_range(batches, 0, nbatches, order, w1, w2, w3, v, vis, st);
}

typedef struct {
    const or_batch* batches;
    uint64_t lo, hi;
    const uint32_t *w1, *w2, *w3;
    const or_view* v;
    uint64_t* vis;
    or_stats st;
} render_job;

static void* render_thread(void* a) {
    render_job* j = (render_job*)a;
    uint64_t npix = (uint64_t)j->v->width * j->v->height;
    for (uint64_t p = 0; p < npix; ++p) j->vis[p] = OR_EMPTY;
    render_range(j->batches, j->lo, j->hi, NULL, j->w1, j->w2, j->w3, j->v, j->vis, &j->st);
    return NULL;
}

void or_render_threaded(const or_batch* batches, uint64_t nbatches,
                        const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                        const or_view* v, int threads, uint64_t* vis, or_stats* st) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    uint64_t npix = (uint64_t)v->width * v->height;
    render_job* jobs = (render_job*)calloc((size_t)threads, sizeof(render_job));
    pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    int* ok = (int*)calloc((size_t)threads, sizeof(int));
    for (int t = 0; t < threads; ++t) {
        render_job* j = &jobs[t];
        j->batches = batches;
        j->lo = nbatches * (uint64_t)t / (uint64_t)threads;
        j->hi = nbatches * (uint64_t)(t + 1) / (uint64_t)threads;
        j->w1 = w1; j->w2 = w2; j->w3 = w3; j->v = v;
        j->vis = t == 0 ? vis : (uint64_t*)malloc(sizeof(uint64_t) * (npix ? npix : 1));
        ok[t] = pthread_create(&tid[t], NULL, render_thread, j) == 0;
        if (!ok[t]) render_thread(j);
    }
    if (st) memset(st, 0, sizeof(*st));
    for (int t = 0; t < threads; ++t) {
        if (ok[t]) pthread_join(tid[t], NULL);
        if (t > 0) {
            for (uint64_t p = 0; p < npix; ++p)
                if (jobs[t].vis[p] < vis[p]) vis[p] = jobs[t].vis[p];
            free(jobs[t].vis);
        }
        if (st) {
            st->batches_rendered += jobs[t].st.batches_rendered;
            st->points_processed += jobs[t].st.points_processed;
            st->points_accepted += jobs[t].st.points_accepted;
            for (int k = 0; k < 4; ++k) {
                st->batches_k[k] += jobs[t].st.batches_k[k];
                st->points_k[k] += jobs[t].st.points_k[k];
            }
        }
    }
    free(jobs);
    free(tid);
    free(ok);
}

void or_render_positions(const float* xyz, uint64_t n, const or_view* v, uint64_t* vis) {
    uint64_t npix = (uint64_t)v->width * v->height;
    for (uint64_t p = 0; p < npix; ++p) vis[p] = OR_EMPTY;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t pix;
        uint64_t key;
        if (or_project_position(&xyz[3 * i], v, (uint32_t)i, &pix, &key, NULL) &&
            key < vis[pix])
            vis[pix] = key;
    }
}

void or_brute_force(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                    const uint32_t* w2, const uint32_t* w3, const or_view* v,
                    uint64_t* vis) {
    uint64_t npix = (uint64_t)v->width * v->height;
    for (uint64_t p = 0; p < npix; ++p) {
        uint64_t best = OR_EMPTY;
        for (uint64_t b = 0; b < nbatches; ++b) {
            int k = or_select_k(&batches[b], v);
            for (uint32_t j = 0; j < batches[b].count; ++j) {
                uint32_t i = batches[b].first + j;
                uint32_t pix;
                uint64_t key;
                if (or_project_point(&batches[b], k, w1[i], w2[i], w3[i], i, v, &pix, &key) &&
                    pix == p && key < best)
                    best = key;
            }
        }
        vis[p] = best;
    }
}

void or_resolve(const uint64_t* vis, uint64_t npixels, const uint32_t* color,
                uint32_t* out) {
    for (uint64_t p = 0; p < npixels; ++p)
        out[p] = vis[p] == OR_EMPTY ? 0u : color[(uint32_t)(vis[p] & 0xFFFFFFFFull)];
}

/* ---- Sec. 3.5 level of detail --------------------------------------------- */

static int projected_box(const or_batch* b, const or_view* v, float fmin[2], float fmax[2]);

int or_projected_extent(const or_batch* b, const or_view* v, float* extent) {
    float fmin[2], fmax[2];
    if (!projected_box(b, v, fmin, fmax)) return 0;
    float ex = fmax[0] - fmin[0];
    float ey = fmax[1] - fmin[1];
    if (ex != ex || ey != ey) *extent = ex + ey;   /* NaN: never below a threshold */
    else *extent = ex > ey ? ex : ey;
    return 1;
}

/* the 8 corners' unfloored pixel coordinates: min and max per axis */
static int projected_box(const or_batch* b, const or_view* v, float fmin[2], float fmax[2]) {
    for (int c = 0; c < 8; ++c) {
        float p[3];
        for (int a = 0; a < 3; ++a)
            p[a] = ((c >> a) & 1) ? b->min[a] + b->size[a] : b->min[a];
        const float* m = v->m;
        float cw = ((m[3] * p[0] + m[7] * p[1]) + m[11] * p[2]) + m[15];
        if (!(cw > 0.0f)) return 0;
        float f[2];
        uint32_t pix;
        uint64_t key;
        or_project_position(p, v, 0, &pix, &key, f);
        for (int a = 0; a < 2; ++a) {
            if (c == 0 || f[a] < fmin[a]) fmin[a] = f[a];
            if (c == 0 || f[a] > fmax[a]) fmax[a] = f[a];
        }
    }
    return 1;
}

int or_ring(float x, float y, uint32_t width, uint32_t height) {
    float hw = (float)width * 0.5f, hh = (float)height * 0.5f;
    float dx = x - hw, dy = y - hh;
    float d2 = dx * dx + dy * dy;
    float r2 = hw * hw + hh * hh;
    if (9.0f * d2 < r2) return 0;
    if (9.0f * d2 < 4.0f * r2) return 1;
    return 2;
}

uint64_t or_splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    float lo[3];
    float size;
    uint32_t level;
    uint32_t parent;
    uint32_t* idx;      /* input indices of the node's points and its subtree */
    uint64_t n;
} lod_work;

typedef struct { uint64_t pri; uint32_t idx; } lod_pri;

static int lod_pri_cmp(const void* a, const void* b) {
    const lod_pri* x = (const lod_pri*)a;
    const lod_pri* y = (const lod_pri*)b;
    if (x->pri != y->pri) return x->pri < y->pri ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int u32_cmp(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y);
}

/* Builds the tree breadth first. When out_nodes is NULL only counts nodes. */
static int64_t lod_build_impl(const float* xyz, const uint32_t* rgba, uint64_t n,
                              uint32_t max_levels, uint32_t max_node_points, uint32_t seed,
                              or_batch* nodes, uint32_t* parent, uint32_t* level, uint32_t* perm,
                              uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color) {
    if (n == 0 || max_levels == 0 || max_node_points == 0) return 0;
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = xyz[a];
    for (uint64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (xyz[3 * i + a] < lo[a]) lo[a] = xyz[3 * i + a];
            if (xyz[3 * i + a] > hi[a]) hi[a] = xyz[3 * i + a];
        }
    float side = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float e = hi[a] - lo[a];
        if (e > side) side = e;
    }
    /* breadth-first queue of work items */
    uint64_t cap = 1024, head = 0, tail = 0;
    lod_work* q = (lod_work*)malloc(sizeof(lod_work) * cap);
    uint32_t* all = (uint32_t*)malloc(sizeof(uint32_t) * n);
    for (uint64_t i = 0; i < n; ++i) all[i] = (uint32_t)i;
    q[tail].lo[0] = lo[0]; q[tail].lo[1] = lo[1]; q[tail].lo[2] = lo[2];
    q[tail].size = side; q[tail].level = 0; q[tail].parent = 0;
    q[tail].idx = all; q[tail].n = n;
    ++tail;
    uint64_t out_pts = 0;
    int64_t id = 0;
    while (head < tail) {
        lod_work w = q[head++];
        uint64_t keep = w.n;
        uint32_t* kept = w.idx;            /* the node's own points, input order */
        uint32_t* rest = NULL;
        uint64_t nrest = 0;
        if (w.n > max_node_points && w.level + 1 < max_levels) {
            lod_pri* pr = (lod_pri*)malloc(sizeof(lod_pri) * w.n);
            for (uint64_t j = 0; j < w.n; ++j) {
                pr[j].idx = w.idx[j];
                pr[j].pri = or_splitmix64(((uint64_t)seed << 32) + w.idx[j]);
            }
            qsort(pr, w.n, sizeof(lod_pri), lod_pri_cmp);
            keep = max_node_points;
            kept = (uint32_t*)malloc(sizeof(uint32_t) * keep);
            rest = (uint32_t*)malloc(sizeof(uint32_t) * (w.n - keep));
            for (uint64_t j = 0; j < keep; ++j) kept[j] = pr[j].idx;
            for (uint64_t j = keep; j < w.n; ++j) rest[nrest++] = pr[j].idx;
            free(pr);
            qsort(kept, keep, sizeof(uint32_t), u32_cmp);   /* input order */
            qsort(rest, nrest, sizeof(uint32_t), u32_cmp);
        }
        if (nodes) {
            or_batch* B = &nodes[id];
            for (int a = 0; a < 3; ++a) { B->min[a] = w.lo[a]; B->size[a] = w.size; }
            B->first = (uint32_t)out_pts;
            B->count = (uint32_t)keep;
            parent[id] = w.parent;
            level[id] = w.level;
            for (uint64_t j = 0; j < keep; ++j) {
                const float* p = &xyz[3 * (uint64_t)kept[j]];
                uint32_t X = or_quantize30(p[0], B->min[0], B->size[0]);
                uint32_t Y = or_quantize30(p[1], B->min[1], B->size[1]);
                uint32_t Z = or_quantize30(p[2], B->min[2], B->size[2]);
                uint32_t ws[3];
                or_split_words(X, Y, Z, ws);
                perm[out_pts + j] = kept[j];
                w1[out_pts + j] = ws[0];
                w2[out_pts + j] = ws[1];
                w3[out_pts + j] = ws[2];
                color[out_pts + j] = rgba ? rgba[kept[j]] : 0u;
            }
        }
        out_pts += keep;
        if (nrest) {
            /* octant of each remaining point against the cube's midpoints */
            float half = w.size * 0.5f;
            float mid[3];
            for (int a = 0; a < 3; ++a) mid[a] = w.lo[a] + half;
            for (int o = 0; o < 8; ++o) {
                uint64_t cnt = 0;
                for (uint64_t j = 0; j < nrest; ++j) {
                    const float* p = &xyz[3 * (uint64_t)rest[j]];
                    int oct = (p[0] >= mid[0]) | ((p[1] >= mid[1]) << 1) | ((p[2] >= mid[2]) << 2);
                    if (oct == o) ++cnt;
                }
                if (!cnt) continue;
                uint32_t* ci = (uint32_t*)malloc(sizeof(uint32_t) * cnt);
                uint64_t k = 0;
                for (uint64_t j = 0; j < nrest; ++j) {
                    const float* p = &xyz[3 * (uint64_t)rest[j]];
                    int oct = (p[0] >= mid[0]) | ((p[1] >= mid[1]) << 1) | ((p[2] >= mid[2]) << 2);
                    if (oct == o) ci[k++] = rest[j];
                }
                if (tail == cap) {
                    cap *= 2;
                    q = (lod_work*)realloc(q, sizeof(lod_work) * cap);
                }
                lod_work* c = &q[tail++];
                for (int a = 0; a < 3; ++a) c->lo[a] = ((o >> a) & 1) ? mid[a] : w.lo[a];
                c->size = half;
                c->level = w.level + 1;
                c->parent = (uint32_t)id;
                c->idx = ci;
                c->n = cnt;
            }
            free(rest);
        }
        if (kept != w.idx) free(kept);
        free(w.idx);
        ++id;
    }
    free(q);
    return id;
}

int64_t or_lod_count_nodes(const float* xyz, uint64_t n, uint32_t max_levels,
                           uint32_t max_node_points, uint32_t seed) {
    return lod_build_impl(xyz, NULL, n, max_levels, max_node_points, seed, NULL, NULL, NULL,
                          NULL, NULL, NULL, NULL, NULL);
}

int64_t or_lod_build(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t max_levels,
                     uint32_t max_node_points, uint32_t seed, or_batch* nodes,
                     uint32_t* parent, uint32_t* level, uint32_t* perm, uint32_t* w1,
                     uint32_t* w2, uint32_t* w3, uint32_t* color) {
    return lod_build_impl(xyz, rgba, n, max_levels, max_node_points, seed, nodes, parent, level,
                          perm, w1, w2, w3, color);
}

void or_lod_select(const or_batch* nodes, const uint32_t* parent, uint64_t nnodes,
                   const or_view* v, float lod_px, float lod_px_periphery, uint8_t* sel) {
    for (uint64_t i = 0; i < nnodes; ++i) {
        int ok = !or_cull(&nodes[i], v);
        if (ok && i > 0) {
            float e;
            if (or_projected_extent(&nodes[i], v, &e)) {
                float t = lod_px;
                if (lod_px_periphery > 0.0f) {
                    float fmin[2], fmax[2];
                    projected_box(&nodes[i], v, fmin, fmax);
                    float cx = (fmin[0] + fmax[0]) * 0.5f;
                    float cy = (fmin[1] + fmax[1]) * 0.5f;
                    int ring = or_ring(cx, cy, v->width, v->height);
                    if (ring == 1) t = (lod_px + lod_px_periphery) * 0.5f;
                    if (ring == 2) t = lod_px_periphery;
                }
                ok = !(e < t);
            }
        }
        if (ok && i > 0) ok = sel[parent[i]];
        sel[i] = (uint8_t)ok;
    }
}

void or_lod_render(const or_batch* nodes, const uint32_t* parent, uint64_t nnodes,
                   const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                   const or_view* v, float lod_px, float lod_px_periphery, uint64_t* vis,
                   or_stats* st) {
    uint64_t npix = (uint64_t)v->width * v->height;
    for (uint64_t p = 0; p < npix; ++p) vis[p] = OR_EMPTY;
    if (st) memset(st, 0, sizeof(*st));
    uint8_t* sel = (uint8_t*)malloc(nnodes ? nnodes : 1);
    or_lod_select(nodes, parent, nnodes, v, lod_px, lod_px_periphery, sel);
    for (uint64_t i = 0; i < nnodes; ++i) {
        if (!sel[i]) continue;
        const or_batch* b = &nodes[i];
        int k = or_select_k(b, v);
        if (st) {
            st->batches_rendered += 1;
            st->points_processed += b->count;
            st->batches_k[k] += 1;
            st->points_k[k] += b->count;
        }
        for (uint32_t j = 0; j < b->count; ++j) {
            uint32_t idx = b->first + j;
            uint32_t pix;
            uint64_t key;
            if (!or_project_point(b, k, w1[idx], w2[idx], w3[idx], idx, v, &pix, &key)) continue;
            if (st) st->points_accepted += 1;
            if (key < vis[pix]) vis[pix] = key;
        }
    }
    free(sel);
}

void or_resolve_dilated(const uint64_t* vis, uint32_t width, uint32_t height,
                        const uint32_t* color, uint32_t* out) {
    for (uint32_t py = 0; py < height; ++py)
        for (uint32_t px = 0; px < width; ++px) {
            int r = 1 + or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);
            uint64_t best = OR_EMPTY;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int x = (int)px + dx, y = (int)py + dy;
                    if (x < 0 || y < 0 || x >= (int)width || y >= (int)height) continue;
                    uint64_t k = vis[(uint64_t)y * width + (uint64_t)x];
                    if (k < best) best = k;
                }
            out[(uint64_t)py * width + px] =
                best == OR_EMPTY ? 0u : color[(uint32_t)(best & 0xFFFFFFFFull)];
        }
}

/* Sec. 3.6, colour pass for one point: it contributes to its pixel when its
 * depth is within 1% of the closest depth there, w <= fl(w_min * 1.01). */
static void hqs_point(const or_batch* b, int k, uint32_t idx, const uint32_t* w1,
                      const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                      const or_view* v, const uint64_t* vis, uint64_t* sum) {
    uint32_t pix;
    uint64_t key;
    if (!or_project_point(b, k, w1[idx], w2[idx], w3[idx], idx, v, &pix, &key)) return;
    uint32_t wbits = (uint32_t)(vis[pix] >> 32), kbits = (uint32_t)(key >> 32);
    float wmin, w;
    memcpy(&wmin, &wbits, 4);
    memcpy(&w, &kbits, 4);
    float limit = wmin * 1.01f;
    if (!(w <= limit)) return;
    uint32_t c = color[idx];
    sum[4 * (uint64_t)pix + 0] += c & 255u;
    sum[4 * (uint64_t)pix + 1] += (c >> 8) & 255u;
    sum[4 * (uint64_t)pix + 2] += (c >> 16) & 255u;
    sum[4 * (uint64_t)pix + 3] += 1;
}

/* Sec. 3.6 resolve: the average of the sums, each channel rounded down. */
static void hqs_average(const uint64_t* sum, uint64_t npix, uint32_t* out) {
    for (uint64_t p = 0; p < npix; ++p) {
        uint64_t n = sum[4 * p + 3];
        out[p] = n == 0 ? 0u
                        : (uint32_t)(sum[4 * p + 0] / n) | ((uint32_t)(sum[4 * p + 1] / n) << 8) |
                              ((uint32_t)(sum[4 * p + 2] / n) << 16) | (255u << 24);
    }
}

void or_render_hqs(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                   const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                   const or_view* v, const uint64_t* vis, uint32_t* out) {
    uint64_t npix = (uint64_t)v->width * v->height;
    uint64_t* sum = (uint64_t*)calloc(npix ? 4 * npix : 1, sizeof(uint64_t));
    for (uint64_t b = 0; b < nbatches; ++b) {
        const or_batch* B = &batches[b];
        if (v->cull && or_cull(B, v)) continue;
        int k = or_select_k(B, v);
        for (uint32_t j = 0; j < B->count; ++j)
            hqs_point(B, k, B->first + j, w1, w2, w3, color, v, vis, sum);
    }
    hqs_average(sum, npix, out);
    free(sum);
}

typedef struct {
    const or_batch* batches;
    uint64_t lo, hi;
    const uint32_t *w1, *w2, *w3, *color;
    const or_view* v;
    const uint64_t* vis;
    uint64_t* sum;
} hqs_job;

static void* hqs_thread(void* a) {
    hqs_job* j = (hqs_job*)a;
    for (uint64_t b = j->lo; b < j->hi; ++b) {
        const or_batch* B = &j->batches[b];
        if (j->v->cull && or_cull(B, j->v)) continue;
        int k = or_select_k(B, j->v);
        for (uint32_t i = 0; i < B->count; ++i)
            hqs_point(B, k, B->first + i, j->w1, j->w2, j->w3, j->color, j->v, j->vis, j->sum);
    }
    return NULL;
}

void or_render_hqs_threaded(const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                            const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                            const or_view* v, const uint64_t* vis, int threads, uint32_t* out) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    uint64_t npix = (uint64_t)v->width * v->height;
    hqs_job* jobs = (hqs_job*)calloc((size_t)threads, sizeof(hqs_job));
    pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    int* ok = (int*)calloc((size_t)threads, sizeof(int));
    for (int t = 0; t < threads; ++t) {
        hqs_job* j = &jobs[t];
        j->batches = batches;
        j->lo = nbatches * (uint64_t)t / (uint64_t)threads;
        j->hi = nbatches * (uint64_t)(t + 1) / (uint64_t)threads;
        j->w1 = w1; j->w2 = w2; j->w3 = w3; j->color = color; j->v = v; j->vis = vis;
        j->sum = (uint64_t*)calloc(npix ? 4 * npix : 1, sizeof(uint64_t));
        ok[t] = pthread_create(&tid[t], NULL, hqs_thread, j) == 0;
        if (!ok[t]) hqs_thread(j);
    }
    /* integer sums: adding the threads' partial sums gives the same totals */
    for (int t = 0; t < threads; ++t) {
        if (ok[t]) pthread_join(tid[t], NULL);
        if (t > 0) {
            for (uint64_t q = 0; q < 4 * npix; ++q) jobs[0].sum[q] += jobs[t].sum[q];
            free(jobs[t].sum);
        }
    }
    hqs_average(jobs[0].sum, npix, out);
    free(jobs[0].sum);
    free(jobs);
    free(tid);
    free(ok);
}

void or_lod_render_hqs(const or_batch* nodes, const uint32_t* parent, uint64_t nnodes,
                       const uint32_t* w1, const uint32_t* w2, const uint32_t* w3,
                       const uint32_t* color, const or_view* v, float lod_px,
                       float lod_px_periphery, const uint64_t* vis, uint32_t* out) {
    uint64_t npix = (uint64_t)v->width * v->height;
    uint64_t* sum = (uint64_t*)calloc(npix ? 4 * npix : 1, sizeof(uint64_t));
    uint8_t* sel = (uint8_t*)malloc(nnodes ? nnodes : 1);
    or_lod_select(nodes, parent, nnodes, v, lod_px, lod_px_periphery, sel);
    for (uint64_t i = 0; i < nnodes; ++i) {
        if (!sel[i]) continue;
        const or_batch* B = &nodes[i];
        int k = or_select_k(B, v);
        for (uint32_t j = 0; j < B->count; ++j)
            hqs_point(B, k, B->first + j, w1, w2, w3, color, v, vis, sum);
    }
    hqs_average(sum, npix, out);
    free(sel);
    free(sum);
}

void or_hqs_resolve_dilated(const uint64_t* vis, uint32_t width, uint32_t height,
                            const uint32_t* hqs, uint32_t* out) {
    for (uint32_t py = 0; py < height; ++py)
        for (uint32_t px = 0; px < width; ++px) {
            int r = 1 + or_ring((float)px + 0.5f, (float)py + 0.5f, width, height);
            uint64_t best = OR_EMPTY, at = 0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int x = (int)px + dx, y = (int)py + dy;
                    if (x < 0 || y < 0 || x >= (int)width || y >= (int)height) continue;
                    uint64_t q = (uint64_t)y * width + (uint64_t)x;
                    if (vis[q] < best) {
                        best = vis[q];
                        at = q;
                    }
                }
            out[(uint64_t)py * width + px] = best == OR_EMPTY ? 0u : hqs[at];
        }
}

/* ---- Sec. 3.1 at full size: checking an encoding against the definition ---- */

typedef struct {
    const float* xyz;
    const uint32_t* rgba;
    uint64_t n;
    uint32_t batch_size;
    const or_batch* batches;
    uint64_t nbatches;
    const uint32_t *w1, *w2, *w3, *color, *perm;
    double cmin[3], csize[3];
    uint64_t lo, hi;         /* range of sorted positions (pass 1) or batches (pass 2) */
    float bmin[3], bmax[3];  /* pass 0: box of xyz[lo, hi) */
    int code;
    uint64_t where;
} verify_job;

static void* verify_box(void* a) {
    verify_job* j = (verify_job*)a;
    for (int c = 0; c < 3; ++c) j->bmin[c] = j->bmax[c] = j->xyz[3 * j->lo + c];
    for (uint64_t i = j->lo; i < j->hi; ++i)
        for (int c = 0; c < 3; ++c) {
            float v = j->xyz[3 * i + c];
            if (v < j->bmin[c]) j->bmin[c] = v;
            if (v > j->bmax[c]) j->bmax[c] = v;
        }
    return NULL;
}

/* pass 1: perm sorts the Morton codes stably. Its entries are below n, and
 * strictly increasing (code, index) pairs make them distinct, so it is a
 * permutation. */
static void* verify_order(void* a) {
    verify_job* j = (verify_job*)a;
    uint64_t prev_code = 0;
    uint32_t prev_idx = 0;
    if (j->lo > 0) {
        prev_idx = j->perm[j->lo - 1];
        if ((uint64_t)prev_idx < j->n) prev_code = or_morton_code(&j->xyz[3 * (uint64_t)prev_idx], j->cmin, j->csize);
    }
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        uint32_t idx = j->perm[i];
        if ((uint64_t)idx >= j->n) { j->code = 2; j->where = i; return NULL; }
        uint64_t code = or_morton_code(&j->xyz[3 * (uint64_t)idx], j->cmin, j->csize);
        if (i > 0 && !(prev_code < code || (prev_code == code && prev_idx < idx))) {
            j->code = 3; j->where = i; return NULL;
        }
        prev_code = code;
        prev_idx = idx;
    }
    return NULL;
}

/* pass 2: batch headers, boxes, Eq. 1 words (Listing 2) and colours */
static void* verify_batches(void* a) {
    verify_job* j = (verify_job*)a;
    for (uint64_t b = j->lo; b < j->hi; ++b) {
        const or_batch* B = &j->batches[b];
        uint64_t first = b * j->batch_size;
        uint64_t end = first + j->batch_size < j->n ? first + j->batch_size : j->n;
        if (B->first != first || B->count != end - first) { j->code = 1; j->where = b; return NULL; }
        float bmin[3], bmax[3];
        for (int c = 0; c < 3; ++c) bmin[c] = bmax[c] = j->xyz[3 * (uint64_t)j->perm[first] + c];
        for (uint64_t i = first; i < end; ++i)
            for (int c = 0; c < 3; ++c) {
                float v = j->xyz[3 * (uint64_t)j->perm[i] + c];
                if (v < bmin[c]) bmin[c] = v;
                if (v > bmax[c]) bmax[c] = v;
            }
        for (int c = 0; c < 3; ++c) {
            float size = bmax[c] - bmin[c];
            if (memcmp(&B->min[c], &bmin[c], 4) != 0 || memcmp(&B->size[c], &size, 4) != 0) {
                j->code = 4; j->where = b; return NULL;
            }
        }
        for (uint64_t i = first; i < end; ++i) {
            const float* p = &j->xyz[3 * (uint64_t)j->perm[i]];
            uint32_t w[3];
            or_split_words(or_quantize30(p[0], B->min[0], B->size[0]),
                           or_quantize30(p[1], B->min[1], B->size[1]),
                           or_quantize30(p[2], B->min[2], B->size[2]), w);
            if (w[0] != j->w1[i] || w[1] != j->w2[i] || w[2] != j->w3[i]) {
                j->code = 5; j->where = i; return NULL;
            }
            uint32_t col = j->rgba ? j->rgba[j->perm[i]] : 0u;
            if (col != j->color[i]) { j->code = 6; j->where = i; return NULL; }
        }
    }
    return NULL;
}

static void run_jobs(verify_job* jobs, int threads, void* (*fn)(void*)) {
    pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    int* ok = (int*)calloc((size_t)threads, sizeof(int));
    for (int t = 0; t < threads; ++t) {
        ok[t] = pthread_create(&tid[t], NULL, fn, &jobs[t]) == 0;
        if (!ok[t]) fn(&jobs[t]);
    }
    for (int t = 0; t < threads; ++t)
        if (ok[t]) pthread_join(tid[t], NULL);
    free(tid);
    free(ok);
}

int or_verify_encoding(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t batch_size,
                       const or_batch* batches, uint64_t nbatches, const uint32_t* w1,
                       const uint32_t* w2, const uint32_t* w3, const uint32_t* color,
                       const uint32_t* perm, int threads, uint64_t* where) {
    *where = 0;
    if (batch_size == 0 || n > 0xFFFFFFFFull || nbatches != or_num_batches(n, batch_size)) return 1;
    if (n == 0) return 0;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    verify_job* jobs = (verify_job*)calloc((size_t)threads, sizeof(verify_job));
    if (!jobs) return -2;
    for (int t = 0; t < threads; ++t) {
        verify_job* j = &jobs[t];
        j->xyz = xyz; j->rgba = rgba; j->n = n; j->batch_size = batch_size;
        j->batches = batches; j->nbatches = nbatches;
        j->w1 = w1; j->w2 = w2; j->w3 = w3; j->color = color; j->perm = perm;
        j->lo = n * (uint64_t)t / (uint64_t)threads;
        j->hi = n * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    /* the cloud box, as the encoder takes it */
    run_jobs(jobs, threads, verify_box);
    float lo[3], hi[3];
    int have = 0;
    for (int t = 0; t < threads; ++t) {
        if (jobs[t].hi <= jobs[t].lo) continue;
        for (int c = 0; c < 3; ++c) {
            if (!have || jobs[t].bmin[c] < lo[c]) lo[c] = jobs[t].bmin[c];
            if (!have || jobs[t].bmax[c] > hi[c]) hi[c] = jobs[t].bmax[c];
        }
        have = 1;
    }
    for (int t = 0; t < threads; ++t)
        for (int c = 0; c < 3; ++c) {
            jobs[t].cmin[c] = (double)lo[c];
            jobs[t].csize[c] = (double)hi[c] - (double)lo[c];
        }
    int code = 0;
    run_jobs(jobs, threads, verify_order);
    for (int t = 0; t < threads && !code; ++t)
        if (jobs[t].code) { code = jobs[t].code; *where = jobs[t].where; }
    if (!code) {
        for (int t = 0; t < threads; ++t) {
            jobs[t].lo = nbatches * (uint64_t)t / (uint64_t)threads;
            jobs[t].hi = nbatches * (uint64_t)(t + 1) / (uint64_t)threads;
        }
        run_jobs(jobs, threads, verify_batches);
        for (int t = 0; t < threads && !code; ++t)
            if (jobs[t].code) { code = jobs[t].code; *where = jobs[t].where; }
    }
    free(jobs);
    return code;
}

/* ---- Sec. 3.5 at full size: checking a LOD tree against the definition ---- */

typedef struct { uint64_t pri; uint32_t idx; } pri_key;

static int pri_less(pri_key a, pri_key b) {
    return a.pri < b.pri || (a.pri == b.pri && a.idx < b.idx);
}

typedef struct {
    const float* xyz;
    const uint32_t* rgba;
    uint64_t n;
    uint32_t seed;
    const or_batch* nodes;
    const uint32_t* parent;
    uint64_t nnodes;
    const uint32_t *perm, *w1, *w2, *w3, *color;
    const int* oct;          /* octant of each node in its parent (root: -1) */
    uint64_t* seen;          /* bitmap of perm values */
    pri_key *own_min, *own_max;
    uint64_t lo, hi;         /* node range */
    int code;
    uint64_t where;
} lod_verify_job;

static int octant_of(const float* p, const or_batch* node) {
    float half = node->size[0] * 0.5f;
    int o = 0;
    for (int a = 0; a < 3; ++a) o |= (p[a] >= node->min[a] + half) << a;
    return o;
}

static void* lod_verify_nodes(void* arg) {
    lod_verify_job* j = (lod_verify_job*)arg;
    for (uint64_t b = j->lo; b < j->hi; ++b) {
        const or_batch* B = &j->nodes[b];
        uint32_t prev = 0;
        for (uint64_t i = B->first; i < (uint64_t)B->first + B->count; ++i) {
            uint32_t idx = j->perm[i];
            /* a permutation, and input order within the node */
            if ((uint64_t)idx >= j->n || (i > B->first && idx <= prev)) { j->code = 3; j->where = i; return NULL; }
            uint64_t bit = 1ull << (idx & 63);
            if (__atomic_fetch_or(&j->seen[idx >> 6], bit, __ATOMIC_RELAXED) & bit) {
                j->code = 3; j->where = i; return NULL;
            }
            prev = idx;
            /* routed down the octants of every ancestor */
            const float* p = &j->xyz[3 * (uint64_t)idx];
            for (uint64_t c = b; c != 0; c = j->parent[c])
                if (octant_of(p, &j->nodes[j->parent[c]]) != j->oct[c]) { j->code = 4; j->where = i; return NULL; }
            /* priorities */
            pri_key k = {or_splitmix64(((uint64_t)j->seed << 32) + idx), idx};
            if (i == B->first || pri_less(k, j->own_min[b])) j->own_min[b] = k;
            if (i == B->first || pri_less(j->own_max[b], k)) j->own_max[b] = k;
            /* Eq. 1 against the node cube, Listing 2, colour */
            uint32_t w[3];
            or_split_words(or_quantize30(p[0], B->min[0], B->size[0]),
                           or_quantize30(p[1], B->min[1], B->size[1]),
                           or_quantize30(p[2], B->min[2], B->size[2]), w);
            if (w[0] != j->w1[i] || w[1] != j->w2[i] || w[2] != j->w3[i]) { j->code = 6; j->where = i; return NULL; }
            if ((j->rgba ? j->rgba[idx] : 0u) != j->color[i]) { j->code = 7; j->where = i; return NULL; }
        }
    }
    return NULL;
}

int or_verify_lod(const float* xyz, const uint32_t* rgba, uint64_t n, uint32_t max_levels,
                  uint32_t max_node_points, uint32_t seed, const or_batch* nodes,
                  const uint32_t* parent, const uint32_t* level, uint64_t nnodes,
                  const uint32_t* perm, const uint32_t* w1, const uint32_t* w2,
                  const uint32_t* w3, const uint32_t* color, int threads, uint64_t* where) {
    *where = 0;
    if (n == 0) return nnodes == 0 ? 0 : 1;
    if (nnodes == 0 || n > 0xFFFFFFFFull || max_levels == 0 || max_node_points == 0) return 1;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    /* the root: the cloud's corner and largest extent (the encoder's box, threaded) */
    verify_job* bj = (verify_job*)calloc((size_t)threads, sizeof(verify_job));
    if (!bj) return -2;
    for (int t = 0; t < threads; ++t) {
        bj[t].xyz = xyz;
        bj[t].lo = n * (uint64_t)t / (uint64_t)threads;
        bj[t].hi = n * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    run_jobs(bj, threads, verify_box);
    float lo[3], hi[3];
    int have = 0;
    for (int t = 0; t < threads; ++t) {
        if (bj[t].hi <= bj[t].lo) continue;
        for (int c = 0; c < 3; ++c) {
            if (!have || bj[t].bmin[c] < lo[c]) lo[c] = bj[t].bmin[c];
            if (!have || bj[t].bmax[c] > hi[c]) hi[c] = bj[t].bmax[c];
        }
        have = 1;
    }
    free(bj);
    float side = 0.0f;
    for (int c = 0; c < 3; ++c) {
        float e = hi[c] - lo[c];
        if (e > side) side = e;
    }
    for (int c = 0; c < 3; ++c)
        if (memcmp(&nodes[0].min[c], &lo[c], 4) != 0 || memcmp(&nodes[0].size[c], &side, 4) != 0) return 1;
    if (parent[0] != 0 || level[0] != 0) return 2;
    /* headers, breadth-first structure, child cubes in octant order */
    int* oct = (int*)malloc(sizeof(int) * nnodes);
    uint8_t* has_child = (uint8_t*)calloc(nnodes, 1);
    int code = 0;
    uint64_t total = 0;
    oct[0] = -1;
    for (uint64_t b = 0; b < nnodes && !code; ++b) {
        if (nodes[b].first != total || nodes[b].count == 0) { code = 1; *where = b; break; }
        total += nodes[b].count;
        if (b == 0) continue;
        uint32_t p = parent[b];
        if (p >= b || (b > 1 && p < parent[b - 1]) || level[b] != level[p] + 1 || level[b] >= max_levels) {
            code = 2; *where = b; break;
        }
        has_child[p] = 1;
        float half = nodes[p].size[0] * 0.5f;
        int o = 0;
        for (int c = 0; c < 3; ++c) {
            float mid = nodes[p].min[c] + half;
            if (memcmp(&nodes[b].min[c], &mid, 4) == 0) o |= 1 << c;
            else if (memcmp(&nodes[b].min[c], &nodes[p].min[c], 4) != 0) { code = 2; *where = b; }
            if (memcmp(&nodes[b].size[c], &half, 4) != 0) { code = 2; *where = b; }
        }
        oct[b] = o;
        if (b > 1 && parent[b - 1] == p && oct[b - 1] >= o) { code = 2; *where = b; }
    }
    if (!code && total != n) { code = 1; *where = nnodes; }
    /* the split rule: a node splits, keeping max_node_points points, exactly when
     * it holds more than that and is above the last level */
    for (uint64_t b = 0; b < nnodes && !code; ++b) {
        int last = level[b] + 1 >= max_levels;
        if (has_child[b] ? (nodes[b].count != max_node_points || last)
                         : (nodes[b].count > max_node_points && !last)) { code = 5; *where = b; }
    }
    pri_key* own_min = (pri_key*)malloc(sizeof(pri_key) * nnodes);
    pri_key* own_max = (pri_key*)malloc(sizeof(pri_key) * nnodes);
    uint64_t* seen = (uint64_t*)calloc((size_t)((n + 63) / 64), sizeof(uint64_t));
    if (!code) {
        lod_verify_job* jobs = (lod_verify_job*)calloc((size_t)threads, sizeof(lod_verify_job));
        pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
        int* ok = (int*)calloc((size_t)threads, sizeof(int));
        for (int t = 0; t < threads; ++t) {
            lod_verify_job* j = &jobs[t];
            j->xyz = xyz; j->rgba = rgba; j->n = n; j->seed = seed;
            j->nodes = nodes; j->parent = parent; j->nnodes = nnodes;
            j->perm = perm; j->w1 = w1; j->w2 = w2; j->w3 = w3; j->color = color;
            j->oct = oct; j->seen = seen; j->own_min = own_min; j->own_max = own_max;
            j->lo = nnodes * (uint64_t)t / (uint64_t)threads;
            j->hi = nnodes * (uint64_t)(t + 1) / (uint64_t)threads;
            ok[t] = pthread_create(&tid[t], NULL, lod_verify_nodes, j) == 0;
            if (!ok[t]) lod_verify_nodes(j);
        }
        for (int t = 0; t < threads; ++t) {
            if (ok[t]) pthread_join(tid[t], NULL);
            if (!code && jobs[t].code) { code = jobs[t].code; *where = jobs[t].where; }
        }
        free(jobs);
        free(tid);
        free(ok);
    }
    /* priorities: a node's own points all come before every point below it */
    if (!code) {
        pri_key* sub = (pri_key*)malloc(sizeof(pri_key) * nnodes);    /* min over the subtree */
        pri_key* below = (pri_key*)malloc(sizeof(pri_key) * nnodes);  /* min over the descendants */
        uint8_t* any = (uint8_t*)calloc(nnodes, 1);
        for (uint64_t b = 0; b < nnodes; ++b) sub[b] = own_min[b];
        for (uint64_t b = nnodes - 1; b >= 1; --b) {
            uint32_t p = parent[b];
            if (pri_less(sub[b], sub[p])) sub[p] = sub[b];
            if (!any[p] || pri_less(sub[b], below[p])) below[p] = sub[b];
            any[p] = 1;
        }
        for (uint64_t b = 0; b < nnodes && !code; ++b)
            if (any[b] && !pri_less(own_max[b], below[b])) { code = 5; *where = b; }
        free(sub);
        free(below);
        free(any);
    }
    free(seen);
    free(own_min);
    free(own_max);
    free(oct);
    free(has_child);
    return code;
}

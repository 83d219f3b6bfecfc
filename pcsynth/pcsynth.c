/* pcsynth.c — seeded synthetic point clouds and camera matrices (inputs only).
 *
 * See pcsynth.h. Nothing in this file sorts, batches, quantizes or projects
 * points the way the rasterizer does; it only produces raw positions, colours
 * and camera matrices.
 */
#include "pcsynth.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- counter-based random numbers (SplitMix64 output function) ---------- */

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t index) {
    return mix64(mix64(seed * 0xD1342543DE82EF95ull + stream) ^ index);
}

static inline double u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }

double pcs_uniform(uint64_t seed, uint64_t stream, uint64_t index) {
    return u01(rnd(seed, stream, index));
}

enum {
    S_X = 1, S_Y, S_Z, S_RGBA, S_JIT, S_CNOISE, S_KIND, S_BLD, S_FACE,
    S_FU, S_FV, S_BPARAM, S_PATH, S_VIEW
};

/* ---- thread fan-out ------------------------------------------------------ */

typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } range_job;

static void* range_thread(void* a) {
    range_job* j = (range_job*)a;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_range(range_fn fn, void* ctx, uint64_t n, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > n / 4096 + 1) threads = (int)(n / 4096 + 1);
    if (threads == 1) { fn(ctx, 0, n); return; }
    pthread_t tid[256];
    int ok[256];
    range_job job[256];
    for (int t = 0; t < threads; ++t) {
        job[t].fn = fn; job[t].ctx = ctx;
        job[t].lo = n * (uint64_t)t / (uint64_t)threads;
        job[t].hi = n * (uint64_t)(t + 1) / (uint64_t)threads;
        ok[t] = pthread_create(&tid[t], NULL, range_thread, &job[t]) == 0;
        if (!ok[t]) fn(ctx, job[t].lo, job[t].hi);  /* no thread: run inline */
    }
    for (int t = 0; t < threads; ++t) if (ok[t]) pthread_join(tid[t], NULL);
}

/* ---- unit cube ------------------------------------------------------------ */

typedef struct { uint64_t seed, first; float* xyz; uint32_t* rgba; } cube_ctx;

static void cube_range(void* c, uint64_t lo, uint64_t hi) {
    cube_ctx* k = (cube_ctx*)c;
    for (uint64_t j = lo; j < hi; ++j) {
        uint64_t i = k->first + j;
        /* 24 random bits per axis give a float in [0,1) exactly */
        k->xyz[3 * j + 0] = (float)(rnd(k->seed, S_X, i) >> 40) * 0x1.0p-24f;
        k->xyz[3 * j + 1] = (float)(rnd(k->seed, S_Y, i) >> 40) * 0x1.0p-24f;
        k->xyz[3 * j + 2] = (float)(rnd(k->seed, S_Z, i) >> 40) * 0x1.0p-24f;
        k->rgba[j] = (uint32_t)(rnd(k->seed, S_RGBA, i) >> 32);
    }
}

void pcs_unit_cube(uint64_t seed, uint64_t first, uint64_t n, float* xyz,
                   uint32_t* rgba, int threads) {
    cube_ctx c = {seed, first, xyz, rgba};
    parallel_range(cube_range, &c, n, threads);
}

/* ---- terrain: fractal value noise over a square area --------------------- */

void pcs_terrain_defaults(pcs_terrain_params* p, double extent_m) {
    memset(p, 0, sizeof(*p));
    p->extent_m = extent_m;
    p->wavelength_m = 2000.0;
    p->amplitude_m = 300.0;
    p->persistence = 0.5;
    p->lacunarity = 2.0;
    p->octaves = 6;
    p->jitter_m = 0.01;
    p->buildings_frac = 0.0;
    p->n_buildings = 0;
}

static inline double lattice(uint64_t seed, uint32_t octave, int64_t ix, int64_t iy) {
    uint64_t h = mix64(seed ^ mix64((uint64_t)octave * 0x632BE59BD9B4E019ull +
                                    (uint64_t)ix * 0x9E3779B97F4A7C15ull +
                                    (uint64_t)iy * 0xC2B2AE3D27D4EB4Full));
    return u01(h) * 2.0 - 1.0;
}

static inline double fade(double t) { return t * t * (3.0 - 2.0 * t); }

static double value_noise(uint64_t seed, uint32_t octave, double x, double y) {
    double fx = floor(x), fy = floor(y);
    int64_t ix = (int64_t)fx, iy = (int64_t)fy;
    double tx = fade(x - fx), ty = fade(y - fy);
    double a = lattice(seed, octave, ix, iy), b = lattice(seed, octave, ix + 1, iy);
    double c = lattice(seed, octave, ix, iy + 1), d = lattice(seed, octave, ix + 1, iy + 1);
    double ab = a + (b - a) * tx, cd = c + (d - c) * tx;
    return ab + (cd - ab) * ty;
}

double pcs_terrain_height(uint64_t seed, const pcs_terrain_params* p, double x,
                          double y) {
    double h = 0.0, amp = p->amplitude_m, freq = 1.0 / p->wavelength_m;
    for (uint32_t o = 0; o < p->octaves; ++o) {
        h += amp * value_noise(seed, o, x * freq, y * freq);
        amp *= p->persistence;
        freq *= p->lacunarity;
    }
    return h;
}

static inline uint32_t pack_rgba(double r, double g, double b) {
    int ir = (int)r, ig = (int)g, ib = (int)b;
    ir = ir < 0 ? 0 : ir > 255 ? 255 : ir;
    ig = ig < 0 ? 0 : ig > 255 ? 255 : ig;
    ib = ib < 0 ? 0 : ib > 255 ? 255 : ib;
    return (uint32_t)ir | ((uint32_t)ig << 8) | ((uint32_t)ib << 16) | (255u << 24);
}

static uint32_t terrain_color(uint64_t seed, const pcs_terrain_params* p,
                              double h, uint64_t i) {
    double t = (h + p->amplitude_m) / (2.0 * p->amplitude_m);
    t = t < 0 ? 0 : t > 1 ? 1 : t;
    double r, g, b;
    if (t < 0.35) { double s = t / 0.35; r = 50 + 60 * s; g = 100 + 45 * s; b = 35 + 25 * s; }
    else if (t < 0.7) { double s = (t - 0.35) / 0.35; r = 110 + 40 * s; g = 145 - 35 * s; b = 60 + 20 * s; }
    else { double s = (t - 0.7) / 0.3; r = 150 + 90 * s; g = 110 + 130 * s; b = 80 + 160 * s; }
    double n = (u01(rnd(seed, S_CNOISE, i)) - 0.5) * 24.0;
    return pack_rgba(r + n, g + n, b + n);
}

/* building j: centre, footprint, height and base level */
typedef struct { double cx, cy, wx, wy, hz, z0; uint32_t tint; } building;

static void make_building(uint64_t seed, const pcs_terrain_params* p, uint32_t j,
                          building* bd) {
    double e = p->extent_m;
    bd->cx = (u01(rnd(seed, S_BPARAM, 8ull * j + 0)) - 0.5) * e * 0.98;
    bd->cy = (u01(rnd(seed, S_BPARAM, 8ull * j + 1)) - 0.5) * e * 0.98;
    bd->wx = 10.0 + 50.0 * u01(rnd(seed, S_BPARAM, 8ull * j + 2));
    bd->wy = 10.0 + 50.0 * u01(rnd(seed, S_BPARAM, 8ull * j + 3));
    bd->hz = 5.0 + 75.0 * u01(rnd(seed, S_BPARAM, 8ull * j + 4));
    bd->z0 = pcs_terrain_height(seed, p, bd->cx, bd->cy) - 2.0;
    bd->tint = (uint32_t)(rnd(seed, S_BPARAM, 8ull * j + 5) >> 40);
}

typedef struct {
    uint64_t seed, first;
    const pcs_terrain_params* p;
    float* xyz;
    uint32_t* rgba;
    building* bld;
} terrain_ctx;

static void terrain_range(void* c, uint64_t lo, uint64_t hi) {
    terrain_ctx* k = (terrain_ctx*)c;
    const pcs_terrain_params* p = k->p;
    double e = p->extent_m;
    for (uint64_t j = lo; j < hi; ++j) {
        uint64_t i = k->first + j;
        double x, y, z;
        uint32_t col;
        int on_building = p->n_buildings > 0 && p->buildings_frac > 0 &&
                          u01(rnd(k->seed, S_KIND, i)) < p->buildings_frac;
        if (on_building) {
            const building* bd = &k->bld[rnd(k->seed, S_BLD, i) % p->n_buildings];
            double top = bd->wx * bd->wy, wall_x = bd->wx * bd->hz, wall_y = bd->wy * bd->hz;
            double pick = u01(rnd(k->seed, S_FACE, i)) * (top + 2 * wall_x + 2 * wall_y);
            double fu = u01(rnd(k->seed, S_FU, i)), fv = u01(rnd(k->seed, S_FV, i));
            double x0 = bd->cx - 0.5 * bd->wx, y0 = bd->cy - 0.5 * bd->wy;
            if (pick < top) { x = x0 + fu * bd->wx; y = y0 + fv * bd->wy; z = bd->z0 + bd->hz; }
            else if (pick < top + wall_x) { x = x0 + fu * bd->wx; y = y0; z = bd->z0 + fv * bd->hz; }
            else if (pick < top + 2 * wall_x) { x = x0 + fu * bd->wx; y = y0 + bd->wy; z = bd->z0 + fv * bd->hz; }
            else if (pick < top + 2 * wall_x + wall_y) { x = x0; y = y0 + fu * bd->wy; z = bd->z0 + fv * bd->hz; }
            else { x = x0 + bd->wx; y = y0 + fu * bd->wy; z = bd->z0 + fv * bd->hz; }
            uint32_t t = bd->tint;
            double n = (u01(rnd(k->seed, S_CNOISE, i)) - 0.5) * 20.0;
            col = pack_rgba(150 + (double)(t & 63) - 32 + n, 150 + (double)((t >> 6) & 63) - 32 + n,
                            160 + (double)((t >> 12) & 63) - 32 + n);
        } else {
            x = (u01(rnd(k->seed, S_X, i)) - 0.5) * e;
            y = (u01(rnd(k->seed, S_Y, i)) - 0.5) * e;
            double h = pcs_terrain_height(k->seed, p, x, y);
            z = h + (u01(rnd(k->seed, S_JIT, i)) * 2.0 - 1.0) * p->jitter_m;
            col = terrain_color(k->seed, p, h, i);
        }
        k->xyz[3 * j + 0] = (float)x;
        k->xyz[3 * j + 1] = (float)y;
        k->xyz[3 * j + 2] = (float)z;
        k->rgba[j] = col;
    }
}

void pcs_terrain(uint64_t seed, const pcs_terrain_params* p, uint64_t first,
                 uint64_t n, float* xyz, uint32_t* rgba, int threads) {
    terrain_ctx c = {seed, first, p, xyz, rgba, NULL};
    if (p->n_buildings > 0 && p->buildings_frac > 0) {
        c.bld = (building*)malloc(sizeof(building) * p->n_buildings);
        if (!c.bld) return;
        for (uint32_t j = 0; j < p->n_buildings; ++j) make_building(seed, p, j, &c.bld[j]);
    }
    parallel_range(terrain_range, &c, n, threads);
    free(c.bld);
}

/* ---- scan-ordered terrain --------------------------------------------------- */

typedef struct {
    uint64_t seed, first, total, per_line;
    const pcs_terrain_params* p;
    double sx, sy, dmax;
    float* xyz;
    uint32_t* rgba;
} scan_ctx;

static void scan_range(void* c, uint64_t lo, uint64_t hi) {
    scan_ctx* k = (scan_ctx*)c;
    const uint64_t lines = (k->total + k->per_line - 1) / k->per_line;
    for (uint64_t j = lo; j < hi; ++j) {
        uint64_t i = k->first + j;
        uint64_t line = i / k->per_line, r = i % k->per_line;
        double yaw = 2.0 * M_PI * ((double)line + 0.5 * u01(rnd(k->seed, S_X, i))) / (double)lines;
        double t = ((double)r + u01(rnd(k->seed, S_Y, i))) / (double)k->per_line;
        double d = 5.0 + (k->dmax - 5.0) * t;
        double x = k->sx + d * cos(yaw), y = k->sy + d * sin(yaw);
        double h = pcs_terrain_height(k->seed, k->p, x, y);
        double z = h + (u01(rnd(k->seed, S_JIT, i)) * 2.0 - 1.0) * k->p->jitter_m;
        k->xyz[3 * j + 0] = (float)x;
        k->xyz[3 * j + 1] = (float)y;
        k->xyz[3 * j + 2] = (float)z;
        k->rgba[j] = terrain_color(k->seed, k->p, h, i);
    }
}

void pcs_terrain_scan(uint64_t seed, const pcs_terrain_params* p, double sx, double sy,
                      double max_dist_m, uint64_t total, uint64_t points_per_line,
                      uint64_t first, uint64_t n, float* xyz, uint32_t* rgba, int threads) {
    if (points_per_line == 0) points_per_line = 1;
    scan_ctx c = {seed, first, total, points_per_line, p, sx, sy, max_dist_m, xyz, rgba};
    parallel_range(scan_range, &c, n, threads);
}

/* ---- cameras -------------------------------------------------------------- */

static void normalize3(double v[3]) {
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (l > 0) { v[0] /= l; v[1] /= l; v[2] /= l; }
}

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void pcs_look_at_perspective(const double eye[3], const double target[3],
                             const double up[3], double fovy_deg, double aspect,
                             double zn, double zf, float out[16]) {
    double f[3] = {target[0] - eye[0], target[1] - eye[1], target[2] - eye[2]};
    normalize3(f);
    double s[3], u[3];
    cross3(f, up, s);
    normalize3(s);
    cross3(s, f, u);
    /* view matrix rows: s, u, -f with translation */
    double V[16] = {0};
    V[0] = s[0]; V[4] = s[1]; V[8] = s[2];  V[12] = -(s[0] * eye[0] + s[1] * eye[1] + s[2] * eye[2]);
    V[1] = u[0]; V[5] = u[1]; V[9] = u[2];  V[13] = -(u[0] * eye[0] + u[1] * eye[1] + u[2] * eye[2]);
    V[2] = -f[0]; V[6] = -f[1]; V[10] = -f[2]; V[14] = (f[0] * eye[0] + f[1] * eye[1] + f[2] * eye[2]);
    V[15] = 1.0;
    double t = 1.0 / tan(fovy_deg * M_PI / 360.0);
    double P[16] = {0};
    P[0] = t / aspect;
    P[5] = t;
    P[10] = (zf + zn) / (zn - zf);
    P[14] = 2.0 * zf * zn / (zn - zf);
    P[11] = -1.0;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0;
            for (int k = 0; k < 4; ++k) acc += P[r + 4 * k] * V[k + 4 * c];
            out[r + 4 * c] = (float)acc;
        }
}

static void path_point(uint64_t seed, const pcs_terrain_params* p, double t,
                       double o[2]) {
    double e = p->extent_m;
    double ph = 2 * M_PI * u01(rnd(seed, S_PATH, 0));
    double rot = 2 * M_PI * u01(rnd(seed, S_PATH, 1));
    double rx = 0.33 * e, ry = 0.22 * e;
    double a = 2 * M_PI * t + ph;
    /* a closed loop with a wobble, rotated by a seeded angle */
    double x = rx * cos(a) + 0.05 * e * cos(3 * a + ph);
    double y = ry * sin(a) + 0.05 * e * sin(2 * a);
    o[0] = x * cos(rot) - y * sin(rot);
    o[1] = x * sin(rot) + y * cos(rot);
}

void pcs_flythrough(uint64_t seed, const pcs_terrain_params* p, uint32_t frame,
                    uint32_t nframes, uint32_t width, uint32_t height,
                    float out[16], double eye_out[3]) {
    double t = nframes ? (double)frame / (double)nframes : 0.0;
    double e2[2], l2[2];
    path_point(seed, p, t, e2);
    path_point(seed, p, t + 0.03, l2);
    double ph2 = 2 * M_PI * u01(rnd(seed, S_PATH, 2));
    double alt = 275.0 + 225.0 * sin(4 * M_PI * t + ph2);   /* 50..500 m */
    double eye[3] = {e2[0], e2[1], pcs_terrain_height(seed, p, e2[0], e2[1]) + alt};
    double tgt[3] = {l2[0], l2[1], pcs_terrain_height(seed, p, l2[0], l2[1])};
    double up[3] = {0, 0, 1};
    pcs_look_at_perspective(eye, tgt, up, 60.0, (double)width / (double)height,
                            1.0, 4.0 * p->extent_m, out);
    if (eye_out) { eye_out[0] = eye[0]; eye_out[1] = eye[1]; eye_out[2] = eye[2]; }
}

void pcs_overview(const pcs_terrain_params* p, uint32_t width, uint32_t height,
                  float out[16]) {
    double e = p->extent_m;
    double eye[3] = {0.0, -0.95 * e, 0.62 * e};
    double tgt[3] = {0.0, -0.02 * e, 0.0};
    double up[3] = {0, 0, 1};
    pcs_look_at_perspective(eye, tgt, up, 55.0, (double)width / (double)height,
                            0.01 * e, 4.0 * e, out);
}

void pcs_stereo(const pcs_terrain_params* p, uint32_t width, uint32_t height,
                double ipd_m, int eye_index, float out[16]) {
    double e = p->extent_m;
    double eye[3] = {0.0, -0.8 * e, 0.45 * e};
    double tgt[3] = {0.0, -0.05 * e, 0.0};
    double f[3] = {tgt[0] - eye[0], tgt[1] - eye[1], tgt[2] - eye[2]};
    double up[3] = {0, 0, 1}, s[3];
    normalize3(f);
    cross3(f, up, s);
    normalize3(s);
    double off = (eye_index ? 0.5 : -0.5) * ipd_m;
    double ey[3] = {eye[0] + off * s[0], eye[1] + off * s[1], eye[2] + off * s[2]};
    double tg[3] = {tgt[0] + off * s[0], tgt[1] + off * s[1], tgt[2] + off * s[2]};
    pcs_look_at_perspective(ey, tg, up, 90.0, (double)width / (double)height,
                            0.01 * e, 4.0 * e, out);
}

void pcs_random_view(uint64_t seed, const pcs_terrain_params* p, uint64_t index,
                     uint32_t width, uint32_t height, float out[16]) {
    double e = p->extent_m;
    double ex = (u01(rnd(seed, S_VIEW, 6 * index + 0)) - 0.5) * e;
    double ey = (u01(rnd(seed, S_VIEW, 6 * index + 1)) - 0.5) * e;
    double alt = 50.0 + 2950.0 * u01(rnd(seed, S_VIEW, 6 * index + 2));
    double tx = (u01(rnd(seed, S_VIEW, 6 * index + 3)) - 0.5) * e;
    double ty = (u01(rnd(seed, S_VIEW, 6 * index + 4)) - 0.5) * e;
    double fov = 45.0 + 45.0 * u01(rnd(seed, S_VIEW, 6 * index + 5));
    double eye[3] = {ex, ey, pcs_terrain_height(seed, p, ex, ey) + alt};
    double tgt[3] = {tx, ty, pcs_terrain_height(seed, p, tx, ty)};
    if (fabs(tgt[0] - eye[0]) + fabs(tgt[1] - eye[1]) < 1.0) tgt[0] += 10.0;
    double up[3] = {0, 0, 1};
    pcs_look_at_perspective(eye, tgt, up, fov, (double)width / (double)height,
                            1.0, 4.0 * e, out);
}

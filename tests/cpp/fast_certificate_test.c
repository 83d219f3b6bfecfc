/* Adversarial check of the fast-path certificate that the cull pass computes
 * for each batch and view (batch_fast in the raster kernels).
 *
 * A certified batch skips the per-point tests of the general path, so the
 * certificate must be sound: every point the batch can decode to must be in
 * front of the eye with a binary32 clip w in [2^-99, 2^99] (the reciprocal
 * estimate stays normal), and its floor pixel must lie inside the view. This
 * program restates the certificate's binary32 steps and checks, for every
 * certified (box, view) pair, the eight corners at k = 1 and k = 2 and random
 * points in between with the oracle's own decode and projection
 * (or_project_point): each must be accepted, with w in range.
 *
 * The cases are adversarial: boxes placed at controlled distances (2^-28 to
 * 2^-4 in normalized device units) inside and outside each edge of the view,
 * boxes close to the eye plane, tiny and huge boxes, matrices scaled over
 * 2^-60 .. 2^60, and widths from 1 to 16384 pixels.
 *
 * argv[1] == "narrow": the certificate without its margins (no rounding
 * bound, limits at exactly -1 and 1); that version must fail somewhere, which
 * shows the cases reach the edges the margins protect.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pcr_oracle.h"

static int narrow = 0;

static float row_max32(const float r[4], const float lo[3], const float hi[3]) {
    float s = r[3];
    for (int a = 0; a < 3; ++a) s = s + fmaxf(r[a] * lo[a], r[a] * hi[a]);
    return s;
}
static float row_min32(const float r[4], const float lo[3], const float hi[3]) {
    float s = r[3];
    for (int a = 0; a < 3; ++a) s = s + fminf(r[a] * lo[a], r[a] * hi[a]);
    return s;
}
static float row_mag32(const float r[4], const float lo[3], const float hi[3]) {
    float s = fabsf(r[3]);
    for (int a = 0; a < 3; ++a) s = s + fabsf(r[a]) * fmaxf(fabsf(lo[a]), fabsf(hi[a]));
    return s;
}

/* The certificate: 1 when the batch may take the fast path. */
static int certified(const or_batch* b, const float* m) {
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (!(b->size[a] <= 0x1p100f)) return 0;
        lo[a] = b->min[a];
        hi[a] = b->min[a] + b->size[a];
    }
    const float X[4] = {m[0], m[4], m[8], m[12]}, Y[4] = {m[1], m[5], m[9], m[13]};
    const float Wr[4] = {m[3], m[7], m[11], m[15]};
    const float g = narrow ? 0.0f : 32.0f * 0x1p-24f, tiny = narrow ? 0.0f : 0x1p-120f;
    const float mw = g * row_mag32(Wr, lo, hi) + tiny;
    const float wl = row_min32(Wr, lo, hi) - mw, wh = row_max32(Wr, lo, hi) + mw;
    if (!(wl >= 0x1p-99f) || !(wh <= 0x1p99f)) return 0;
    const float lim_lo = narrow ? -1.0f : -1.0f + 0x1p-12f;
    const float lim_hi = narrow ? nextafterf(1.0f, 0.0f) : 1.0f - 0x1p-12f;
    const float* rows[2] = {X, Y};
    for (int r = 0; r < 2; ++r) {
        const float mr = g * row_mag32(rows[r], lo, hi) + tiny;
        const float cl = row_min32(rows[r], lo, hi) - mr, ch = row_max32(rows[r], lo, hi) + mr;
        const float qmin = cl >= 0.0f ? cl / wh : cl / wl;
        const float qmax = ch >= 0.0f ? ch / wl : ch / wh;
        if (!(qmin >= lim_lo) || !(qmax <= lim_hi)) return 0;
    }
    return 1;
}

/* SplitMix64 stream for the test's own random inputs */
static uint64_t rng_state = 0x2545F4914F6CDD1Dull;
static uint64_t next_u64(void) {
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uniform(void) { return (double)(next_u64() >> 11) * 0x1p-53; }

/* column-major perspective * look-at, in binary64 then rounded to binary32 */
static void camera(const double eye[3], const double at[3], double fovy, double aspect, float* m) {
    double f[3], s[3], u[3], up[3] = {0, 0, 1};
    double n = 0;
    for (int a = 0; a < 3; ++a) {
        f[a] = at[a] - eye[a];
        n += f[a] * f[a];
    }
    n = sqrt(n);
    for (int a = 0; a < 3; ++a) f[a] /= n;
    if (fabs(f[2]) > 0.99) {
        up[0] = 1;
        up[2] = 0;
    }
    s[0] = f[1] * up[2] - f[2] * up[1];
    s[1] = f[2] * up[0] - f[0] * up[2];
    s[2] = f[0] * up[1] - f[1] * up[0];
    n = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int a = 0; a < 3; ++a) s[a] /= n;
    u[0] = s[1] * f[2] - s[2] * f[1];
    u[1] = s[2] * f[0] - s[0] * f[2];
    u[2] = s[0] * f[1] - s[1] * f[0];
    const double t = 1.0 / tan(fovy * 0.5), zn = 0.1, zf = 1e5;
    double V[16] = {0}, P[16] = {0}, M[16];
    for (int a = 0; a < 3; ++a) {
        V[4 * a + 0] = s[a];
        V[4 * a + 1] = u[a];
        V[4 * a + 2] = -f[a];
    }
    V[12] = -(s[0] * eye[0] + s[1] * eye[1] + s[2] * eye[2]);
    V[13] = -(u[0] * eye[0] + u[1] * eye[1] + u[2] * eye[2]);
    V[14] = f[0] * eye[0] + f[1] * eye[1] + f[2] * eye[2];
    V[15] = 1;
    P[0] = t / aspect;
    P[5] = t;
    P[10] = (zf + zn) / (zn - zf);
    P[11] = -1;
    P[14] = 2 * zf * zn / (zn - zf);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0;
            for (int k = 0; k < 4; ++k) acc += P[r + 4 * k] * V[k + 4 * c];
            M[r + 4 * c] = acc;
        }
    for (int i = 0; i < 16; ++i) m[i] = (float)M[i];
}

/* world point at normalized device coordinates (qx, qy) and view depth d */
static void unproject(const double eye[3], const double at[3], double fovy, double aspect,
                      double qx, double qy, double d, double p[3]) {
    double f[3], s[3], u[3], up[3] = {0, 0, 1}, n = 0;
    for (int a = 0; a < 3; ++a) {
        f[a] = at[a] - eye[a];
        n += f[a] * f[a];
    }
    n = sqrt(n);
    for (int a = 0; a < 3; ++a) f[a] /= n;
    if (fabs(f[2]) > 0.99) {
        up[0] = 1;
        up[2] = 0;
    }
    s[0] = f[1] * up[2] - f[2] * up[1];
    s[1] = f[2] * up[0] - f[0] * up[2];
    s[2] = f[0] * up[1] - f[1] * up[0];
    n = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int a = 0; a < 3; ++a) s[a] /= n;
    u[0] = s[1] * f[2] - s[2] * f[1];
    u[1] = s[2] * f[0] - s[0] * f[2];
    u[2] = s[0] * f[1] - s[1] * f[0];
    const double t = tan(fovy * 0.5);
    for (int a = 0; a < 3; ++a)
        p[a] = eye[a] + d * (f[a] + qx * t * aspect * s[a] + qy * t * u[a]);
}

static long checked, certified_n, failures, decode_failures;

/* The fast path's decode: the quantized coordinate is placed in the low
 * mantissa bits of 2^23 (2^13 for the in-place y field of a one-word point),
 * and one fused multiply-add with -2^23 cell (-2^13 cell) gives the rounded
 * product q cell, which is then added to the box minimum. It must give the
 * bits of the definition's min + q cell. */
static void fast_decode(const or_batch* b, int k, const uint32_t q[3], float p[3]) {
    for (int a = 0; a < 3; ++a) {
        const float cell = ldexpf(b->size[a], -10 * k);
        uint32_t bits;
        int e = 23;
        if (k == 1 && a == 1) {
            bits = (q[a] << 10) | 0x46000000u;
            e = 13;
        } else {
            bits = q[a] | 0x4B000000u;
        }
        float f;
        memcpy(&f, &bits, 4);
        p[a] = b->min[a] + fmaf(f, cell, -ldexpf(cell, e));
    }
}

/* every corner at k = 1 and 2, and random points, through the oracle */
static void check_batch(const or_batch* b, const or_view* v) {
    ++checked;
    if (!certified(b, v->m)) return;
    ++certified_n;
    for (int k = 1; k <= 2; ++k) {
        const uint32_t top = k == 1 ? 1023u << 20 : 0xFFFFFu << 10;
        for (int c = 0; c < 8 + 24; ++c) {
            uint32_t q[3];
            for (int a = 0; a < 3; ++a)
                q[a] = c < 8 ? (((c >> a) & 1) ? top : 0u) : (uint32_t)(next_u64() & 0x3FFFFFFFu) & top;
            uint32_t w[3], pix;
            uint64_t key;
            or_split_words(q[0], q[1], q[2], w);
            {
                uint32_t dq[3];
                float pd[3], pf[3];
                or_decode_words(w[0], w[1], w[2], k, dq);
                or_decode_position(b, k, w[0], w[1], w[2], pd);
                fast_decode(b, k, dq, pf);
                if (memcmp(pd, pf, sizeof pd) != 0 && decode_failures++ < 10)
                    printf("FAIL decode k=%d q (%u %u %u)\n", k, dq[0], dq[1], dq[2]);
            }
            const int in = or_project_point(b, k, w[0], w[1], w[2], 0, v, &pix, &key);
            uint32_t wb = (uint32_t)(key >> 32);
            float cw;
            memcpy(&cw, &wb, 4);
            if (!in || !(cw >= 0x1p-99f && cw <= 0x1p99f)) {
                if (failures++ < 10)
                    printf("FAIL box min (%a %a %a) size (%a %a %a) k=%d corner %d in=%d w=%a\n",
                           b->min[0], b->min[1], b->min[2], b->size[0], b->size[1], b->size[2], k,
                           c, in, cw);
            }
        }
    }
}

int main(int argc, char** argv) {
    if (argc > 1 && strcmp(argv[1], "narrow") == 0) narrow = 1;
    const uint32_t widths[] = {1, 64, 1000, 1920, 16384};
    for (int it = 0; it < 20000; ++it) {
        or_view v;
        memset(&v, 0, sizeof v);
        v.width = widths[next_u64() % 5];
        v.height = widths[next_u64() % 5];
        const double aspect = (double)v.width / v.height;
        const double fovy = (20.0 + 80.0 * uniform()) * 3.14159265358979323846 / 180.0;
        const double R = exp2(-10.0 + 30.0 * uniform());   /* scene scale */
        double eye[3], at[3];
        for (int a = 0; a < 3; ++a) {
            eye[a] = R * (2.0 * uniform() - 1.0);
            at[a] = eye[a] + R * (2.0 * uniform() - 1.0);
        }
        camera(eye, at, fovy, aspect, v.m);
        /* a matrix scaled by a power of two gives the same pixels */
        const float sc = ldexpf(1.0f, (int)(next_u64() % 121) - 60);
        for (int i = 0; i < 16; ++i) v.m[i] *= sc;
        for (int j = 0; j < 8; ++j) {
            /* a box corner near an edge (or anywhere), at a view depth from near the
             * eye plane to far away */
            const double d = R * exp2(-12.0 + 16.0 * uniform());
            double qx = 2.0 * uniform() - 1.0, qy = 2.0 * uniform() - 1.0;
            const double off = exp2(-28.0 + 24.0 * uniform()) * ((next_u64() & 1) ? 1 : -1);
            switch (next_u64() % 5) {
                case 0: qx = 1.0 + off; break;
                case 1: qx = -1.0 + off; break;
                case 2: qy = 1.0 + off; break;
                case 3: qy = -1.0 + off; break;
                default: break;
            }
            double p[3];
            unproject(eye, at, fovy, aspect, qx, qy, d, p);
            or_batch b;
            memset(&b, 0, sizeof b);
            const double ext = d * exp2(-30.0 + 26.0 * uniform());
            for (int a = 0; a < 3; ++a) {
                const double sz = ext * uniform();
                /* the corner at p is the box's max or min corner along each axis */
                const double mn = (next_u64() & 1) ? p[a] - sz : p[a];
                b.min[a] = (float)mn;
                b.size[a] = (float)sz;
            }
            b.count = 1;
            check_batch(&b, &v);
        }
    }
    printf("checked %ld, certified %ld (%.1f%%), failures %ld\n", checked, certified_n,
           100.0 * (double)certified_n / (double)checked, failures);
    if (decode_failures) printf("decode failures %ld\n", decode_failures);
    if (failures || decode_failures) return 1;
    if (certified_n < checked / 10) {
        printf("FAIL too few certified\n");
        return 1;
    }
    printf("fast certificate ok\n");
    return 0;
}

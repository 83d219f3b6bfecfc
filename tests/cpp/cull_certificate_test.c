/* Adversarial check of the culling kernel's binary32 fast test against the
 * oracle's conservative binary64 test of Sec. 3.2 (or_cull): a batch is culled
 * only when a rounding bound proves every decoded point outside one clip
 * plane.
 *
 * The kernel evaluates each plane test of the binary64 definition in binary32,
 * with the same terms (rounding bound 6u times the row magnitude, plane margin
 * 1 + 2^-10). It decides a plane only when its binary32 value t is farther
 * than 2^-16 times the row magnitude from 0 (the binary32 evaluation of each
 * of these few-term sums is off by far less); otherwise, or when a magnitude
 * leaves [2^-90, 2^100], it falls back to the binary64 test. The function below
 * restates those binary32 steps; this program checks, on boxes placed at
 * controlled distances from each clip plane and under matrices scaled over
 * 2^-60 .. 2^60, that every decided result equals or_cull.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pcr_oracle.h"

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

static int undecided, culled;
static void plane(float t, float mag) {
    const float lim = 0x1p-16f * mag;
    if (t < -lim) culled = 1;
    else if (!(t > lim)) undecided = 1;
}

/* 1: culled, 0: kept, -1: left to the binary64 test */
static int fast_cull(const or_batch* b, const float* m) {
    const float g = 6.0f * 0x1p-24f, e1 = 1.0f + 0x1p-10f;
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = b->min[a];
        hi[a] = b->min[a] + b->size[a];
    }
    const float X[4] = {m[0], m[4], m[8], m[12]}, Y[4] = {m[1], m[5], m[9], m[13]};
    const float Wr[4] = {m[3], m[7], m[11], m[15]};
    const float bx = row_mag32(X, lo, hi), by = row_mag32(Y, lo, hi), bw = row_mag32(Wr, lo, hi);
    const float mag_x = bx + e1 * bw, mag_y = by + e1 * bw;
    if (!(bw <= 0x1p100f) || !(mag_x <= 0x1p100f) || !(mag_y <= 0x1p100f)) return -1;
    if (!(bw >= 0x1p-90f) || !(mag_x >= 0x1p-90f) || !(mag_y >= 0x1p-90f)) return -1;
    undecided = culled = 0;
    plane(row_max32(Wr, lo, hi) + g * bw, bw);
    float sp[4], sm[4];
    for (int a = 0; a < 4; ++a) { sp[a] = X[a] + e1 * Wr[a]; sm[a] = X[a] - e1 * Wr[a]; }
    const float mx = g * mag_x;
    plane(row_max32(sp, lo, hi) + mx, mag_x);
    plane(-(row_min32(sm, lo, hi) - mx), mag_x);
    for (int a = 0; a < 4; ++a) { sp[a] = Y[a] + e1 * Wr[a]; sm[a] = Y[a] - e1 * Wr[a]; }
    const float my = g * mag_y;
    plane(row_max32(sp, lo, hi) + my, mag_y);
    plane(-(row_min32(sm, lo, hi) - my), mag_y);
    if (culled) return 1;
    return undecided ? -1 : 0;
}

static uint64_t rng_state = 0x2545F4914F6CDD1Dull;
static uint64_t next_u64(void) {
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uniform(void) { return (double)(next_u64() >> 11) * 0x1p-53; }

/* a perspective camera at a random eye looking at a random target */
static void camera(float m[16], double scale) {
    double eye[3], tgt[3], f[3], s[3], u[3], up[3] = {0, 0, 1};
    for (int a = 0; a < 3; ++a) {
        eye[a] = (uniform() - 0.5) * 2000.0;
        tgt[a] = eye[a] + (uniform() - 0.5) * 200.0;
    }
    double n = 0;
    for (int a = 0; a < 3; ++a) { f[a] = tgt[a] - eye[a]; n += f[a] * f[a]; }
    n = sqrt(n);
    for (int a = 0; a < 3; ++a) f[a] /= n;
    s[0] = f[1] * up[2] - f[2] * up[1]; s[1] = f[2] * up[0] - f[0] * up[2]; s[2] = f[0] * up[1] - f[1] * up[0];
    n = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (n < 1e-6) { s[0] = 1; s[1] = 0; s[2] = 0; n = 1; }
    for (int a = 0; a < 3; ++a) s[a] /= n;
    u[0] = s[1] * f[2] - s[2] * f[1]; u[1] = s[2] * f[0] - s[0] * f[2]; u[2] = s[0] * f[1] - s[1] * f[0];
    const double fy = 1.0 / tan((20.0 + 80.0 * uniform()) * 3.14159265358979323846 / 360.0);
    const double fx = fy / (0.5 + 2.0 * uniform());
    const double zn = 0.1 + uniform(), zf = 1000.0 + 1e5 * uniform();
    double r[4][4] = {{0}};
    /* rows: x = fx * (s . (p - eye)), y = fy * (u . (p - eye)), z, w = f . (p - eye) */
    for (int a = 0; a < 3; ++a) {
        r[0][a] = fx * s[a];
        r[1][a] = fy * u[a];
        r[2][a] = f[a] * (zf + zn) / (zf - zn);
        r[3][a] = f[a];
    }
    r[0][3] = -fx * (s[0] * eye[0] + s[1] * eye[1] + s[2] * eye[2]);
    r[1][3] = -fy * (u[0] * eye[0] + u[1] * eye[1] + u[2] * eye[2]);
    r[2][3] = -(f[0] * eye[0] + f[1] * eye[1] + f[2] * eye[2]) * (zf + zn) / (zf - zn) - 2 * zf * zn / (zf - zn);
    r[3][3] = -(f[0] * eye[0] + f[1] * eye[1] + f[2] * eye[2]);
    for (int row = 0; row < 4; ++row)
        for (int col = 0; col < 4; ++col) m[row + 4 * col] = (float)(r[row][col] * scale);
}

/* one plane test of the definition for a box, in binary64: its row (plane 0
 * is w > 0, 1/2 are x >= -w / x <= w, 3/4 the same for y, each with the margin
 * 1 + 2^-10 and signed so that the plane culls when the test value is < 0),
 * the row's largest value over the box, and the magnitude that scales the
 * rounding bound and the fast test's band */
static void plane_row(const float* m, int p, double r[4]) {
    const double e1 = 1.0 + 0x1p-10;
    for (int a = 0; a < 4; ++a) {
        const double x = m[0 + 4 * a], y = m[1 + 4 * a], w = m[3 + 4 * a];
        r[a] = p == 0 ? w : p == 1 ? x + e1 * w : p == 2 ? -(x - e1 * w) : p == 3 ? y + e1 * w : -(y - e1 * w);
    }
}
static double row_max64(const double r[4], const double lo[3], const double hi[3]) {
    double s = r[3];
    for (int a = 0; a < 3; ++a) s += fmax(r[a] * lo[a], r[a] * hi[a]);
    return s;
}
static double row_mag64(const float* m, int row, const double lo[3], const double hi[3]) {
    double s = fabs((double)m[row + 12]);
    for (int a = 0; a < 3; ++a) s += fabs((double)m[row + 4 * a]) * fmax(fabs(lo[a]), fabs(hi[a]));
    return s;
}
static double plane_mag(const float* m, int p, const double lo[3], const double hi[3]) {
    const double bw = row_mag64(m, 3, lo, hi);
    if (p == 0) return bw;
    return row_mag64(m, p <= 2 ? 0 : 1, lo, hi) + (1.0 + 0x1p-10) * bw;
}
/* the definition's decision value: culled when < 0 (<= 0 for the w plane) */
static double decision(const float* m, int p, const double lo[3], const double hi[3]) {
    double r[4];
    plane_row(m, p, r);
    return row_max64(r, lo, hi) + 6.0 * 0x1p-24 * plane_mag(m, p, lo, hi);
}

int main(void) {
    long checked = 0, decided = 0, failures = 0, culled_total = 0;
    /* distances from the plane, relative to the plane's magnitude; the fast
     * test's band is 2^-16 */
    const double offs[] = {0.0, 0x1p-40, -0x1p-40, 0x1p-30, -0x1p-30, 0x1p-24, -0x1p-24,
                           0x1p-20, -0x1p-20, 0x1p-17, -0x1p-17, 0x1.1p-16, -0x1.1p-16,
                           0x1.ep-17, -0x1.ep-17, 0x1p-15, -0x1p-15, 0x1p-12, -0x1p-12,
                           0x1p-10, -0x1p-10, 0x1p-5, -0x1p-5, 0.5, -0.5};
    const int noffs = (int)(sizeof offs / sizeof offs[0]);
    for (int cam = 0; cam < 4000; ++cam) {
        float m[16];
        const double scale = exp2(-60.0 + 120.0 * uniform());
        camera(m, cam % 4 == 0 ? 1.0 : scale);
        for (int it = 0; it < 400; ++it) {
            /* a random box in front of or around the eye */
            double c[3], h[3];
            const double ext = exp2(-8.0 + 20.0 * uniform());
            for (int a = 0; a < 3; ++a) {
                c[a] = (uniform() - 0.5) * 4000.0;
                h[a] = ext * uniform();
            }
            /* slide it along its largest-effect axis so that one plane's
             * decision value sits at a chosen distance from 0 */
            const int p = (int)(next_u64() % 5);
            const double off = offs[next_u64() % (uint64_t)noffs];
            double lo[3], hi[3], r[4];
            for (int a = 0; a < 3; ++a) { lo[a] = c[a] - h[a]; hi[a] = c[a] + h[a]; }
            plane_row(m, p, r);
            int ax = 0;
            for (int a = 1; a < 3; ++a)
                if (fabs(r[a]) > fabs(r[ax])) ax = a;
            for (int pass = 0; pass < 3 && r[ax] != 0.0; ++pass) {
                const double shift = (off * plane_mag(m, p, lo, hi) - decision(m, p, lo, hi)) / r[ax];
                lo[ax] += shift;
                hi[ax] += shift;
            }
            or_batch b;
            memset(&b, 0, sizeof b);
            for (int a = 0; a < 3; ++a) {
                b.min[a] = (float)lo[a];
                b.size[a] = (float)(hi[a] - lo[a]);
            }
            or_view v;
            memset(&v, 0, sizeof v);
            memcpy(v.m, m, sizeof v.m);
            v.width = v.height = 64;
            v.cull = 1;
            ++checked;
            const int fast = fast_cull(&b, m);
            if (fast < 0) continue;
            ++decided;
            const int ref = or_cull(&b, &v);
            culled_total += ref;
            if (fast != ref && failures++ < 10)
                printf("FAIL cam %d it %d plane %d off %a: fast %d, definition %d\n", cam, it, p, off, fast, ref);
        }
    }
    printf("checked %ld, decided %ld (%.2f%%), culled %ld, failures %ld\n", checked, decided,
           100.0 * (double)decided / (double)checked, culled_total, failures);
    if (failures) return 1;
    if (decided < checked / 2 || culled_total < decided / 20) {
        printf("FAIL too few decided or culled cases\n");
        return 1;
    }
    printf("cull certificate ok\n");
    return 0;
}

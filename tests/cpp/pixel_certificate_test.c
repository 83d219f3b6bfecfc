/* Adversarial check of the raster kernel's certified fast pixel stage.
 *
 * The definition (the oracle's reading of Listing 1's pixel): f =
 * fl(fl(fl(c / w) * 0.5 + 0.5) * W) with an IEEE divide, then the floor bits
 * fl_down(f + 2^23), which fall in [2^23, 2^23 + W) exactly for accepted
 * points.
 *
 * The kernel's fast stage never divides: r is an approximate reciprocal of w
 * (a hardware estimate), refined by one Newton step r' = fma(r, fma(-w, r, 1),
 * r) in the general path and used as it is in the fast path of certified
 * batches; q' = fl(c * r'); with eta = 2^-21 it forms u- = fma(q', 0.5, 0.5 - eta)
 * and u+ = fma(q', 0.5, 0.5 + eta) and the bracket fl_down(u- * W + 2^23),
 * fl_down(u+ * W + 2^23) (fused, rounded down). When both ends agree and
 * 2^-100 <= w <= 2^100 it takes them as the floor bits; otherwise it falls back
 * to the definition.
 *
 * With the Newton step this program takes r as ANY float within a relative
 * distance 2^-20 of 1/w (far looser than the estimate's documented accuracy of
 * 1 ulp); without it, any float up to 2 ulps from 1/w. Either is flushed to
 * zero below the smallest normal as the estimate does, and it checks on random and on
 * pixel-edge inputs that a certified bracket always gives the same
 * accept/reject decision as the definition, and the same bits when accepted.
 *
 * The fused roundings are computed exactly, without relying on the C library's
 * fmaf: a*b is exact in binary64, and
 *  - round-down: RD_float(RD_double(a*b + c)) = RD_float(a*b + c), since every
 *    float is a double;
 *  - round-to-nearest: the binary64 sum rounded to odd (toward zero, lowest bit
 *    set when inexact), then rounded to the nearest float, is the correctly
 *    rounded result (round-to-odd with at least 2 extra bits; Boldo and
 *    Melquiond, "Emulation of FMA and correctly rounded sums: proved algorithms
 *    using rounding to odd", IEEE Trans. Computers 57(4), 2008).
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

static uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

static float fma_rd(float a, float b, float c) {
    volatile double p = (double)a * (double)b;   /* exact */
    fesetround(FE_DOWNWARD);
    volatile double s = p + (double)c;
    volatile float r = (float)s;
    fesetround(FE_TONEAREST);
    return r;
}

static float fma_rn(float a, float b, float c) {
    volatile double p = (double)a * (double)b;   /* exact */
    feclearexcept(FE_INEXACT);
    fesetround(FE_TOWARDZERO);
    volatile double s = p + (double)c;
    fesetround(FE_TONEAREST);
    if (fetestexcept(FE_INEXACT)) {              /* round to odd */
        uint64_t u;
        double d = s;
        memcpy(&u, &d, 8);
        u |= 1u;
        memcpy(&d, &u, 8);
        s = d;
    }
    volatile float r = (float)s;
    return r;
}

/* the definition, with separate round-to-nearest operations */
static uint32_t exact_floor_bits(float c, float w, float W) {
    volatile float q = c / w;
    volatile float h = q * 0.5f;
    volatile float t = h + 0.5f;
    volatile float f = t * W;
    fesetround(FE_DOWNWARD);
    volatile float s = f + 8388608.0f;
    fesetround(FE_TONEAREST);
    return fbits(s);
}

/* newton: refine r by one Newton step first (the general path); without it
 * (the fast path of certified batches) r is used as it is. eta: the margin. */
static int newton = 1;
static float eta = 0x1p-21f;

static int fast_floor_bits(float c, float w, float W, float r, uint32_t* out) {
    float r2 = r;
    if (newton) {
        const float e = fma_rn(-w, r, 1.0f);
        r2 = fma_rn(r, e, r);
    }
    volatile float q = c * r2;
    const float ulo = fma_rn(q, 0.5f, 0.5f - eta);
    const float uhi = fma_rn(q, 0.5f, 0.5f + eta);
    const uint32_t blo = fbits(fma_rd(ulo, W, 8388608.0f));
    const uint32_t bhi = fbits(fma_rd(uhi, W, 8388608.0f));
    *out = blo;
    return blo == bhi && w >= 0x1p-100f && w <= 0x1p100f;
}

static int inside(uint32_t b, float W) {   /* the kernel's range test */
    return b - 0x4B000000u < (uint32_t)W;
}

/* SplitMix64 stream for the test's own random inputs */
static uint64_t rng_state = 0x853c49e6748fea9bull;
static uint64_t next_u64(void) {
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uniform(void) { return (double)(next_u64() >> 11) * 0x1p-53; }

static long checked, certified, failures;

static void one(float c, float w, float W, float r) {
    uint32_t fast;
    ++checked;
    if (!fast_floor_bits(c, w, W, r, &fast)) return;
    ++certified;
    const uint32_t ex = exact_floor_bits(c, w, W);
    const int ok = inside(fast, W) ? (fast == ex) : !inside(ex, W);
    if (!ok && failures++ < 10)
        printf("FAIL c=%a w=%a W=%g r=%a fast=%08x exact=%08x\n", c, w, W, r, fast, ex);
}

/* the estimate flushes results below the smallest normal to zero (ftz) */
static float ftz(float r) { return fabsf(r) < 0x1p-126f ? copysignf(0.0f, r) : r; }

static void with_reciprocals(float c, float w, float W) {
    const float r0 = 1.0f / w;
    if (newton) {
        /* any float within a relative 2^-20 of 1/w */
        const double d[] = {0.0, 0x1p-20, -0x1p-20, 0x1p-23, -0x1p-23};
        for (int i = 0; i < 5; ++i) one(c, w, W, ftz((float)((double)r0 * (1.0 + d[i]))));
        one(c, w, W, ftz((float)((double)r0 * (1.0 + (2.0 * uniform() - 1.0) * 0x1p-20))));
    } else {
        /* no Newton step: the estimate is specified to 1 ulp; this takes every
         * float up to 2 ulps from the correctly rounded reciprocal, and random
         * ones within a relative 2^-23 of it */
        one(c, w, W, ftz(r0));
        one(c, w, W, ftz(nextafterf(nextafterf(r0, INFINITY), INFINITY)));
        one(c, w, W, ftz(nextafterf(nextafterf(r0, 0.0f), 0.0f)));
        one(c, w, W, ftz((float)((double)r0 * (1.0 + (2.0 * uniform() - 1.0) * 0x1p-23))));
    }
    one(c, w, W, ftz(nextafterf(r0, INFINITY)));
    one(c, w, W, ftz(nextafterf(r0, 0.0f)));
}

int main(int argc, char** argv) {
    /* the rounding helpers against hand-checked cases */
    if (fma_rd(1.0f, 1.0f, 0x1p-30f) != 1.0f || fma_rd(-1.0f, 1.0f, -0x1p-30f) != -1.0f - 0x1p-23f ||
        fma_rn(1.0f, 1.0f, 0x1p-24f) != 1.0f || fma_rn(1.0f, 1.0f, 0x1p-24f + 0x1p-40f) != 1.0f + 0x1p-23f ||
        fma_rn(1.0f + 0x1p-23f, 1.0f, 0x1p-24f) != 1.0f + 0x1p-22f) {
        printf("FAIL rounding helpers\n");
        return 1;
    }
    /* argv[1]: "newton" (default), "plain" (no Newton step), or "plain-narrow"
     * (no Newton step and a margin of 2^-23, which must fail) */
    if (argc > 1 && strcmp(argv[1], "plain") == 0) newton = 0;
    if (argc > 1 && strcmp(argv[1], "plain-narrow") == 0) {
        newton = 0;
        eta = 0x1p-23f;
    }
    const float Ws[] = {1.0f, 64.0f, 1000.0f, 1080.0f, 1920.0f, 2016.0f, 2240.0f, 3840.0f, 16384.0f};
    for (int wi = 0; wi < 9; ++wi) {
        const float W = Ws[wi];
        for (int it = 0; it < 24000; ++it) {
            /* depth: log-uniform over [2^-40, 2^40]; now and then over the whole
             * normal range, and at the limits of the fast range */
            float w = (float)exp2(-40.0 + 80.0 * uniform());
            if (it % 13 == 0) w = (float)exp2(-126.0 + 253.0 * uniform());
            if (it % 97 == 0) w = (it & 1) ? 0x1p-100f : 0x1p100f;
            if (it % 89 == 0) w = (it & 1) ? nextafterf(0x1p-100f, 0.0f) : nextafterf(0x1p100f, INFINITY);
            /* a pixel coordinate near a column edge k, or anywhere in [-2W, 3W] */
            double f;
            if (it & 1) {
                const double k = floor(uniform() * (W + 1.0));
                const double eps[] = {0.0, 0x1p-30, -0x1p-30, 0x1p-22, -0x1p-22, 0x1p-12, -0x1p-12};
                f = k + eps[next_u64() % 7] * (k > 1.0 ? k : 1.0);
            } else {
                f = -2.0 * W + 5.0 * W * uniform();
            }
            const double q = (f / W - 0.5) * 2.0;
            float c = (float)(q * (double)w);
            with_reciprocals(c, w, W);
            /* the neighbouring floats of c cross the edge from both sides */
            with_reciprocals(nextafterf(c, INFINITY), w, W);
            with_reciprocals(nextafterf(c, -INFINITY), w, W);
        }
    }
    printf("checked %ld, certified %ld (%.2f%%), failures %ld\n", checked, certified,
           100.0 * (double)certified / (double)checked, failures);
    if (failures) return 1;
    if (certified < checked / 2) {
        printf("FAIL too few certified\n");
        return 1;
    }
    printf("pixel certificate ok\n");
    return 0;
}

/*
 * Seeded synthetic inputs for the LATCH extraction and Hamming matching workloads:
 * grey images, keypoints, triplet tables, random descriptor galleries with planted
 * near-duplicates, and Poisson request arrivals.
 *
 * This module holds none of the descriptor or matching arithmetic.  It is the one
 * piece of code that both the CPU oracle's tests and the CUDA library's tests and
 * benchmarks use, so that both sides see the same bytes.
 *
 * Random numbers: splitmix64 seeds a xoshiro256** state (Blackman & Vigna);
 * bounded integers use Lemire's multiply-and-reject method; uniform doubles take
 * the top 53 bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* Uniform integer in [0, n), n >= 1 (Lemire 2019). */
static uint32_t rng_below(rng_t *r, uint32_t n) {
    uint32_t x = (uint32_t)(rng_next(r) >> 32);
    uint64_t m = (uint64_t)x * (uint64_t)n;
    uint32_t l = (uint32_t)m;
    if (l < n) {
        uint32_t t = (uint32_t)(-n) % n;
        while (l < t) {
            x = (uint32_t)(rng_next(r) >> 32);
            m = (uint64_t)x * (uint64_t)n;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* Uniform integer in [lo, hi] inclusive. */
static int32_t rng_int(rng_t *r, int32_t lo, int32_t hi) {
    return lo + (int32_t)rng_below(r, (uint32_t)(hi - lo + 1));
}

/* Uniform double in [0, 1). */
static double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

uint64_t synth_seed(int config, int index, int kind) {
    return 0x160903986ULL ^ ((uint64_t)(uint32_t)config << 32) ^ ((uint64_t)(uint32_t)index << 8) ^
           (uint64_t)(uint32_t)kind;
}

static inline int reflect101(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

static inline uint8_t round_clamp_u8(double v) {
    double r = round(v); /* half away from zero */
    if (r < 0.0) r = 0.0;
    if (r > 255.0) r = 255.0;
    return (uint8_t)r;
}

/*
 * Grey image: uniform 8-bit noise, separable Gaussian blur (sigma 1.5, radius 5,
 * normalised FP64 taps, reflect-101 border, rounded half away from zero and
 * clamped), then `n_ellipses` filled ellipses of random intensity drawn on top.
 * Pixel (x, y) is filled when the point (x, y) lies inside the ellipse.
 * Bytes of each row beyond `width` (pitch padding) are set to zero.
 * Returns 0, or -1 if the temporary buffer could not be allocated.
 */
int synth_image(uint64_t seed, int width, int height, int64_t pitch, uint8_t *out, int n_ellipses) {
    rng_t r;
    rng_seed(&r, seed);
    const int W = width, H = height;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)W * (size_t)H);
    uint8_t *noise = (uint8_t *)malloc((size_t)W * (size_t)H);
    if (!tmp || !noise) {
        free(tmp);
        free(noise);
        return -1;
    }
    for (size_t i = 0; i < (size_t)W * (size_t)H; ++i) noise[i] = (uint8_t)(rng_next(&r) >> 56);

    const int R = 5;
    const double sigma = 1.5;
    double taps[11], sum = 0.0;
    for (int k = -R; k <= R; ++k) {
        taps[k + R] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        sum += taps[k + R];
    }
    for (int k = 0; k < 2 * R + 1; ++k) taps[k] /= sum;

    /* horizontal pass (the same sum in the same tap order inside and near the border) */
    for (int y = 0; y < H; ++y) {
        const uint8_t *nr = noise + (size_t)y * W;
        double *tr = tmp + (size_t)y * W;
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            if (x >= R && x < W - R) {
                for (int k = -R; k <= R; ++k) acc += taps[k + R] * nr[x + k];
            } else {
                for (int k = -R; k <= R; ++k) acc += taps[k + R] * nr[reflect101(x + k, W)];
            }
            tr[x] = acc;
        }
    }
    /* vertical pass, row by row so that the inner loop runs along x */
    double *acc = (double *)malloc(sizeof(double) * (size_t)W);
    if (!acc) {
        free(tmp);
        free(noise);
        return -1;
    }
    for (int y = 0; y < H; ++y) {
        uint8_t *row = out + (size_t)y * (size_t)pitch;
        for (int x = 0; x < W; ++x) acc[x] = 0.0;
        for (int k = -R; k <= R; ++k) {
            const double *src = tmp + (size_t)reflect101(y + k, H) * W;
            const double t = taps[k + R];
            for (int x = 0; x < W; ++x) acc[x] += t * src[x];
        }
        for (int x = 0; x < W; ++x) row[x] = round_clamp_u8(acc[x]);
        for (int64_t x = W; x < pitch; ++x) row[x] = 0;
    }
    free(acc);
    free(tmp);
    free(noise);

    const double mind = (double)(W < H ? W : H);
    for (int e = 0; e < n_ellipses; ++e) {
        double cx = rng_unit(&r) * W;
        double cy = rng_unit(&r) * H;
        double ra = (0.01 + 0.09 * rng_unit(&r)) * mind;
        double rb = (0.01 + 0.09 * rng_unit(&r)) * mind;
        double ang = rng_unit(&r) * M_PI;
        uint8_t val = (uint8_t)rng_int(&r, 0, 255);
        double c = cos(ang), s = sin(ang);
        double ext = ra > rb ? ra : rb;
        int x0 = (int)floor(cx - ext), x1 = (int)ceil(cx + ext);
        int y0 = (int)floor(cy - ext), y1 = (int)ceil(cy + ext);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (y1 > H - 1) y1 = H - 1;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                double dx = x - cx, dy = y - cy;
                double u = (dx * c + dy * s) / ra;
                double v = (-dx * s + dy * c) / rb;
                if (u * u + v * v <= 1.0) out[(size_t)y * (size_t)pitch + x] = val;
            }
    }
    return 0;
}

/*
 * Keypoints: n records of 4 int32 (x, y, angle_bin, scale_idx).  x is uniform in
 * [border, W-1-border], y in [border, H-1-border]; angle_bin uniform in 0..31 when
 * `oriented`, else 0; scale_idx uniform in 0..nscales-1.  Draw order per keypoint:
 * x, y, then angle (if oriented), then scale (if nscales > 1).
 */
void synth_keypoints(uint64_t seed, int width, int height, int n, int border, int oriented, int nscales,
                     int32_t *out) {
    rng_t r;
    rng_seed(&r, seed);
    for (int i = 0; i < n; ++i) {
        out[4 * i + 0] = rng_int(&r, border, width - 1 - border);
        out[4 * i + 1] = rng_int(&r, border, height - 1 - border);
        out[4 * i + 2] = oriented ? rng_int(&r, 0, 31) : 0;
        out[4 * i + 3] = nscales > 1 ? rng_int(&r, 0, nscales - 1) : 0;
    }
}

/* Triplet table: `count` records of 6 bytes (ax, ay, c1x, c1y, c2x, c2y), each
 * uniform in [lo, hi], drawn in that order. */
void synth_triplets(uint64_t seed, int count, int lo, int hi, uint8_t *out) {
    rng_t r;
    rng_seed(&r, seed);
    for (int i = 0; i < 6 * count; ++i) out[i] = (uint8_t)rng_int(&r, lo, hi);
}

/* i.i.d. uniform bytes (every bit Bernoulli 1/2). */
void synth_bytes(uint64_t seed, int64_t nbytes, uint8_t *out) {
    rng_t r;
    rng_seed(&r, seed);
    int64_t i = 0;
    for (; i + 8 <= nbytes; i += 8) {
        uint64_t v = rng_next(&r);
        memcpy(out + i, &v, 8);
    }
    if (i < nbytes) {
        uint64_t v = rng_next(&r);
        memcpy(out + i, &v, (size_t)(nbytes - i));
    }
}

/*
 * Plant one near-duplicate of every query in the gallery: query i overwrites a
 * distinct gallery slot (chosen without replacement) with a copy of itself in
 * which h_i distinct bits are flipped, h_i uniform in [hmin, hmax].  Descriptors
 * are `desc_bytes` long.  Returns 0, or -1 on a bad argument / allocation failure.
 */
int synth_plant(uint64_t seed, const uint8_t *queries, int nq, uint8_t *gallery, int64_t ng, int desc_bytes,
                int hmin, int hmax, int32_t *slot_out, int32_t *h_out) {
    if (nq > ng || desc_bytes <= 0 || desc_bytes > 4096) return -1;
    rng_t r;
    rng_seed(&r, seed);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
    int nbits = 8 * desc_bytes;
    int32_t *bits = (int32_t *)malloc(sizeof(int32_t) * (size_t)nbits);
    if (!perm || !bits) {
        free(perm);
        free(bits);
        return -1;
    }
    for (int64_t i = 0; i < ng; ++i) perm[i] = (int32_t)i;
    for (int q = 0; q < nq; ++q) {
        /* partial Fisher-Yates over the gallery slots */
        int64_t j = q + (int64_t)rng_below(&r, (uint32_t)(ng - q));
        int32_t t = perm[q];
        perm[q] = perm[j];
        perm[j] = t;
        int32_t slot = perm[q];
        int h = rng_int(&r, hmin, hmax);
        for (int b = 0; b < nbits; ++b) bits[b] = b;
        uint8_t *dst = gallery + (int64_t)slot * desc_bytes;
        memcpy(dst, queries + (int64_t)q * desc_bytes, (size_t)desc_bytes);
        for (int k = 0; k < h; ++k) {
            int m = k + (int)rng_below(&r, (uint32_t)(nbits - k));
            int32_t tb = bits[k];
            bits[k] = bits[m];
            bits[m] = tb;
            dst[bits[k] >> 3] ^= (uint8_t)(1u << (bits[k] & 7));
        }
        slot_out[q] = slot;
        h_out[q] = h;
    }
    free(perm);
    free(bits);
    return 0;
}

/*
 * Poisson request stream of rate `rate` per second over `duration` seconds.
 * For each request: arrival time (s), a size class in [0, n_sizes), a keypoint
 * count uniform in [kmin, kmax] and a gallery id in [0, n_galleries).
 * Writes at most `cap` requests and returns how many were generated.
 */
int synth_arrivals(uint64_t seed, double rate, double duration, int n_sizes, int kmin, int kmax, int n_galleries,
                   int cap, double *t_out, int32_t *size_out, int32_t *kps_out, int32_t *gal_out) {
    rng_t r;
    rng_seed(&r, seed);
    double t = 0.0;
    int n = 0;
    while (n < cap) {
        t += -log(1.0 - rng_unit(&r)) / rate;
        if (t >= duration) break;
        t_out[n] = t;
        size_out[n] = rng_int(&r, 0, n_sizes - 1);
        kps_out[n] = rng_int(&r, kmin, kmax);
        gal_out[n] = rng_int(&r, 0, n_galleries - 1);
        ++n;
    }
    return n;
}

/*
 * CPU oracle for the LATCH descriptor (Sec. 3.1, Eq. 1), its oriented and scaled
 * window sampling (Sec. 3.2, "Memory optimization") and brute-force Hamming
 * matching (Sec. 4, "Descriptor matching on the GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or constant
 * generator with the CUDA library; the two sides build their sample-offset tables
 * independently from the same written reading.
 *
 * Everything is plain, single-threaded and unblocked, in the order the method is
 * defined, so that a reader can check it against the paper line by line:
 *   1. sample the upright 48x48 window at the keypoint's angle bin and scale;
 *   2. for each of the 512 triplets compute the two squared Frobenius distances
 *      between 7x7 patches (Eq. 1) and set the bit when the first is larger;
 *   3. pack the bits least-significant first;
 *   4. match by computing every Hamming distance and taking the two smallest.
 *
 * Readings where the paper is silent (all parity is pinned by the tests):
 *   - angle bin b in 0..31 means theta = 2*pi*b/32; b is taken modulo 32;
 *   - window coordinates a = u - 24, e = v - 24 for u, v in 0..47;
 *   - sample offset dx = rha(s*(cos*a - sin*e)), dy = rha(s*(sin*a + cos*e)),
 *     evaluated in FP64 in exactly that order without contraction, rha = round
 *     half away from zero; cos/sin from libm for the 7 in-quadrant bins, exact
 *     quarter turns;
 *   - samples outside the image read as 0; intensities are the raw 8-bit values;
 *   - Eq. 1 is strict: equal distances give bit 0;
 *   - bit t is bit (t mod 8) of byte t/8;
 *   - matching: lowest distance, ties to the lowest train index; the second match
 *     is the best over the other train indices; accepted iff 1000*d1 < r*d2 with
 *     r = rha(1000*ratio); an absent second match has distance 65535.
 *
 * Weighted patches (Sec. 3.2, "Weighing pixels in LATCH patches": 8x8 patches
 * whose pixels each carry a weight; zero weights on the last row and column give
 * the 7x7 result): pixel (i, j), i, j = 0..7, of the patch centred at (cx, cy) is
 * window pixel (cx - 3 + j, cy - 3 + i) with weight w[8 i + j], a non-negative
 * integer (0..255); the distance is the weighted sum of squared differences, so
 * every triplet coordinate must lie in [3, 43].
 *
 * Keypoint detection (Sec. 3.2: keypoints come from the FAST detector, and the
 * window is read at the keypoint's orientation).  The paper uses a library FAST
 * and states no parameters; readings:
 *   - FAST-9 segment test (Rosten and Drummond): the 16 pixels of the radius-3
 *     Bresenham circle, in circular order; p is a corner at threshold t when 9
 *     contiguous circle pixels are all brighter than I(p) + t or all darker than
 *     I(p) - t;
 *   - score: the largest t' >= t at which p is still a corner (0: not a corner);
 *   - non-maximum suppression: a corner is kept when its score is strictly larger
 *     than the score of each of its 8 neighbours;
 *   - detection region: pixels at least 16 from every border;
 *   - orientation: intensity centroid over the disc x^2 + y^2 <= 15^2 around p,
 *     m10 = sum x I, m01 = sum y I (x right, y down, the frame of the window
 *     rotation above), theta = atan2(m01, m10), angle bin = rha(theta * 16 / pi)
 *     mod 32, in FP64; keypoints are reported in raster order.
 *
 * Multi-scale pyramid (Sec. 6: CLATCH extracted at multiple scales).  Reading: the
 * levels are the scale table's entries s >= 1; level s is the base image sampled at
 * spacing s, I_s(x, y) = I(rha(s x), rha(s y)) for x < floor(W / s), y < floor(H / s)
 * (the nearest-pixel rule of the scaled window); keypoints are detected on every
 * level, a level keypoint (x, y) becomes the base keypoint (rha(s x), rha(s y)) with
 * the level's orientation bin and the level's scale index; levels follow one another
 * in table order.
 * Dense per-pixel LATCH (Sec. 6: dense pixel matching as an alternative to
 * PatchMatch).  Reading: every pixel is a keypoint at angle bin 0 and scale 1,
 * descriptors in raster order; pixel p of image A is matched against the pixels of
 * image B within a Chebyshev radius R of p (inside B), in raster order of B, by the
 * top-two and ratio rule above (train index = raster index in B).
 * Parity pins: every function here is pinned by tests (closed forms, invariants,
 * brute force against full sorting, hand-made images); none is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WIN 48
#define HALF 24
#define NBITS 512
#define PATCH_R 3

/* Sample-offset table for one angle bin and scale (Sec. 3.2, "Memory optimization":
 * the rotated window is loaded as an upright square).  dx/dy are indexed v*48+u. */
void oracle_offsets(double scale, int bin, int32_t *dx, int32_t *dy) {
    int b = ((bin % 32) + 32) % 32;
    int quarter = b / 8, r = b % 8;
    double c = 1.0, s = 0.0;
    if (r != 0) {
        c = cos((double)r * M_PI / 16.0);
        s = sin((double)r * M_PI / 16.0);
    }
    for (int k = 0; k < quarter; ++k) { /* rotate the direction by +90 degrees */
        double t = c;
        c = -s;
        s = t;
    }
    for (int v = 0; v < WIN; ++v)
        for (int u = 0; u < WIN; ++u) {
            double a = (double)(u - HALF), e = (double)(v - HALF);
            double fx = scale * (c * a - s * e);
            double fy = scale * (s * a + c * e);
            dx[v * WIN + u] = (int32_t)round(fx);
            dy[v * WIN + u] = (int32_t)round(fy);
        }
}

/* Squared Frobenius distance between two 7x7 patches of the window (Eq. 1). */
static int64_t patch_ssd(const int32_t *win, int px, int py, int qx, int qy) {
    int64_t acc = 0;
    for (int i = -PATCH_R; i <= PATCH_R; ++i)
        for (int j = -PATCH_R; j <= PATCH_R; ++j) {
            int64_t d = (int64_t)win[(py + i) * WIN + (px + j)] - (int64_t)win[(qy + i) * WIN + (qx + j)];
            acc += d * d;
        }
    return acc;
}

/* Fill the upright window of one keypoint: window pixel (u, v) is the image pixel at
 * the keypoint plus the table offset, or 0 outside the image. */
static void sample_window(const uint8_t *img, int width, int height, int64_t pitch, int32_t x0, int32_t y0,
                          const int32_t *dx, const int32_t *dy, int32_t *win) {
    for (int i = 0; i < WIN * WIN; ++i) {
        int64_t x = (int64_t)x0 + dx[i], y = (int64_t)y0 + dy[i];
        win[i] = (x >= 0 && x < width && y >= 0 && y < height) ? img[y * pitch + x] : 0;
    }
}

/* The two squared distances of Eq. 1 for every triplet of one keypoint:
 * d1[t] = ||P_A - P_1||^2_F, d2[t] = ||P_A - P_2||^2_F.  Returns -1 on a bad scale. */
int oracle_distances(const uint8_t *img, int width, int height, int64_t pitch, int32_t kx, int32_t ky, int32_t kbin,
                     int32_t kscale, const uint8_t *triplets, const double *scales, int nscales, int64_t *d1,
                     int64_t *d2) {
    int32_t dx[WIN * WIN], dy[WIN * WIN], win[WIN * WIN];
    if (kscale < 0 || kscale >= nscales) return -1;
    oracle_offsets(scales[kscale], kbin, dx, dy);
    sample_window(img, width, height, pitch, kx, ky, dx, dy, win);
    for (int t = 0; t < NBITS; ++t) {
        const uint8_t *tr = triplets + 6 * t;
        d1[t] = patch_ssd(win, tr[0], tr[1], tr[2], tr[3]);
        d2[t] = patch_ssd(win, tr[0], tr[1], tr[4], tr[5]);
    }
    return 0;
}

/*
 * LATCH descriptors for n keypoints (Sec. 3.1 Eq. 1; Sec. 3.2).
 * img: width x height bytes with row pitch `pitch`.  Keypoint k is
 * (kx[k], ky[k], kbin[k], kscale[k]) with kscale an index into `scales`.
 * triplets: 512 records (ax, ay, c1x, c1y, c2x, c2y), each coordinate in [3, 44].
 * out: n x 64 bytes.  Returns 0, or -1 on an invalid scale index or triplet.
 */
int oracle_extract(const uint8_t *img, int width, int height, int64_t pitch, const int32_t *kx, const int32_t *ky,
                   const int32_t *kbin, const int32_t *kscale, int n, const uint8_t *triplets, const double *scales,
                   int nscales, uint8_t *out) {
    int32_t dx[WIN * WIN], dy[WIN * WIN], win[WIN * WIN];
    for (int t = 0; t < 6 * NBITS; ++t)
        if (triplets[t] < PATCH_R || triplets[t] > WIN - 1 - PATCH_R) return -1;
    for (int k = 0; k < n; ++k) {
        if (kscale[k] < 0 || kscale[k] >= nscales) return -1;
        oracle_offsets(scales[kscale[k]], kbin[k], dx, dy);
        sample_window(img, width, height, pitch, kx[k], ky[k], dx, dy, win);
        uint8_t *d = out + (int64_t)k * (NBITS / 8);
        memset(d, 0, NBITS / 8);
        for (int t = 0; t < NBITS; ++t) {
            const uint8_t *tr = triplets + 6 * t;
            int64_t d1 = patch_ssd(win, tr[0], tr[1], tr[2], tr[3]); /* ||P_A - P_1||^2 */
            int64_t d2 = patch_ssd(win, tr[0], tr[1], tr[4], tr[5]); /* ||P_A - P_2||^2 */
            if (d1 > d2) d[t >> 3] |= (uint8_t)(1u << (t & 7));
        }
    }
    return 0;
}

/* Weighted squared distance between two 8x8 patches of the window (Sec. 3.2,
 * weighted patches): sum over i, j = 0..7 of w[8 i + j] times the squared
 * difference of window pixels (px - 3 + j, py - 3 + i) and (qx - 3 + j, qy - 3 + i). */
static int64_t patch_wssd(const int32_t *win, int px, int py, int qx, int qy, const uint8_t *w) {
    int64_t acc = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            const int64_t d = (int64_t)win[(py - PATCH_R + i) * WIN + (px - PATCH_R + j)] -
                              (int64_t)win[(qy - PATCH_R + i) * WIN + (qx - PATCH_R + j)];
            acc += (int64_t)w[8 * i + j] * d * d;
        }
    return acc;
}

/*
 * LATCH descriptors with weighted 8x8 patches (Sec. 3.1 Eq. 1 with each squared
 * Frobenius distance weighted pixel by pixel, Sec. 3.2).  As oracle_extract, with
 * `weights` the 64 patch weights (row-major 8x8) and triplet coordinates in [3, 43].
 * Returns 0, or -1 on an invalid scale index or triplet.
 */
int oracle_extract_weighted(const uint8_t *img, int width, int height, int64_t pitch, const int32_t *kx,
                            const int32_t *ky, const int32_t *kbin, const int32_t *kscale, int n,
                            const uint8_t *triplets, const double *scales, int nscales, const uint8_t *weights,
                            uint8_t *out) {
    int32_t dx[WIN * WIN], dy[WIN * WIN], win[WIN * WIN];
    for (int t = 0; t < 6 * NBITS; ++t)
        if (triplets[t] < PATCH_R || triplets[t] > WIN - 2 - PATCH_R) return -1;
    for (int k = 0; k < n; ++k) {
        if (kscale[k] < 0 || kscale[k] >= nscales) return -1;
        oracle_offsets(scales[kscale[k]], kbin[k], dx, dy);
        sample_window(img, width, height, pitch, kx[k], ky[k], dx, dy, win);
        uint8_t *d = out + (int64_t)k * (NBITS / 8);
        memset(d, 0, NBITS / 8);
        for (int t = 0; t < NBITS; ++t) {
            const uint8_t *tr = triplets + 6 * t;
            const int64_t d1 = patch_wssd(win, tr[0], tr[1], tr[2], tr[3], weights);
            const int64_t d2 = patch_wssd(win, tr[0], tr[1], tr[4], tr[5], weights);
            if (d1 > d2) d[t >> 3] |= (uint8_t)(1u << (t & 7));
        }
    }
    return 0;
}

/* Hamming distance between two descriptors of `nbytes` bytes: number of differing bits. */
int oracle_hamming(const uint8_t *a, const uint8_t *b, int nbytes) {
    int d = 0;
    for (int i = 0; i < nbytes; ++i) {
        unsigned x = (unsigned)(a[i] ^ b[i]);
        while (x) {
            d += (int)(x & 1u);
            x >>= 1;
        }
    }
    return d;
}

/*
 * Brute-force top-k (k = 1 or 2) Hamming matching with the ratio test (Sec. 4).
 * For every query: all nt distances, the smallest (lowest index on ties), the
 * smallest over the remaining indices, then the ratio rule.  Outputs per query:
 * idx1, idx2 (-1 when absent), d1, d2 (65535 when absent) and accepted (0/1).
 * Returns 0, or -1 on bad arguments.
 */
int oracle_match(const uint8_t *q, int nq, const uint8_t *t, int nt, int k, float ratio, int32_t *idx1,
                 int32_t *idx2, int32_t *d1, int32_t *d2, uint8_t *accepted) {
    if (k != 1 && k != 2) return -1;
    if (!(ratio >= 0.0f && ratio <= 1.0f)) return -1;
    const int64_t r = (int64_t)round((double)ratio * 1000.0);
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
    if (!dist) return -1;
    for (int i = 0; i < nq; ++i) {
        for (int j = 0; j < nt; ++j) dist[j] = oracle_hamming(q + (int64_t)i * 64, t + (int64_t)j * 64, 64);
        int b1 = -1, b2 = -1;
        for (int j = 0; j < nt; ++j)
            if (b1 < 0 || dist[j] < dist[b1]) b1 = j;
        if (k == 2)
            for (int j = 0; j < nt; ++j)
                if (j != b1 && (b2 < 0 || dist[j] < dist[b2])) b2 = j;
        idx1[i] = b1;
        idx2[i] = b2;
        d1[i] = b1 >= 0 ? dist[b1] : 65535;
        d2[i] = b2 >= 0 ? dist[b2] : 65535;
        if (b1 < 0)
            accepted[i] = 0;
        else if (k == 1)
            accepted[i] = 1;
        else
            accepted[i] = (uint8_t)(1000 * (int64_t)d1[i] < r * (int64_t)d2[i]);
    }
    free(dist);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Keypoint detection: FAST-9 corners with non-maximum suppression, oriented by
 * the intensity centroid (Sec. 3.2).  Plain loops, one pixel at a time.
 * ------------------------------------------------------------------------- */

#define FAST_ARC 9
#define CENTROID_R 15
#define DETECT_BORDER 16

/* The radius-3 Bresenham circle in circular order (x right, y down), from the pixel
 * straight above the centre, clockwise. */
static const int kCircle[16][2] = {{0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0},  {3, 1},  {2, 2},  {1, 3},
                                   {0, 3},  {-1, 3}, {-2, 2}, {-3, 1}, {-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}};

/* Segment test: 9 contiguous circle pixels (circularly) all > I(p) + t, or all
 * < I(p) - t.  (x, y) must be at least 3 pixels from every border. */
static int fast_is_corner(const uint8_t *img, int64_t pitch, int x, int y, int t) {
    const int ip = img[(int64_t)y * pitch + x];
    for (int start = 0; start < 16; ++start) {
        int bright = 1, dark = 1;
        for (int k = 0; k < FAST_ARC; ++k) {
            const int *c = kCircle[(start + k) % 16];
            const int q = img[(int64_t)(y + c[1]) * pitch + (x + c[0])];
            if (!(q > ip + t)) bright = 0;
            if (!(q < ip - t)) dark = 0;
        }
        if (bright || dark) return 1;
    }
    return 0;
}

/* FAST score of pixel (x, y) at threshold t: 0 when it is not a corner at t, else
 * the largest t' >= t at which it is still a corner (found by trying t' = t, t+1,
 * ... in turn). */
int oracle_fast_score(const uint8_t *img, int width, int height, int64_t pitch, int x, int y, int t) {
    if (x < 3 || y < 3 || x >= width - 3 || y >= height - 3) return 0;
    if (!fast_is_corner(img, pitch, x, y, t)) return 0;
    int s = t;
    while (s < 255 && fast_is_corner(img, pitch, x, y, s + 1)) ++s;
    return s;
}

/* Angle bin of the intensity centroid of the radius-15 disc around (x, y), which
 * must be at least 15 pixels from every border. */
int oracle_orientation_bin(const uint8_t *img, int64_t pitch, int x, int y) {
    int64_t m10 = 0, m01 = 0;
    for (int dy = -CENTROID_R; dy <= CENTROID_R; ++dy)
        for (int dx = -CENTROID_R; dx <= CENTROID_R; ++dx)
            if (dx * dx + dy * dy <= CENTROID_R * CENTROID_R) {
                const int64_t v = img[(int64_t)(y + dy) * pitch + (x + dx)];
                m10 += dx * v;
                m01 += dy * v;
            }
    const double theta = atan2((double)m01, (double)m10);
    const int b = (int)round(theta * 16.0 / M_PI);
    return ((b % 32) + 32) % 32;
}

/*
 * Oriented FAST keypoints of an image at threshold t (1 <= t <= 254), in raster
 * order: every pixel of the detection region whose score is non-zero and strictly
 * larger than each of its 8 neighbours' scores, with its orientation bin.  Writes
 * at most `cap` keypoints to xs, ys, bins and returns the number found (which may
 * exceed cap), or -1 on bad arguments.
 */
int oracle_detect(const uint8_t *img, int width, int height, int64_t pitch, int t, int cap, int32_t *xs,
                  int32_t *ys, int32_t *bins) {
    if (t < 1 || t > 254 || width < 1 || height < 1 || cap < 0) return -1;
    int *score = (int *)calloc((size_t)width * (size_t)height, sizeof(int));
    if (!score) return -1;
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x) score[(int64_t)y * width + x] = oracle_fast_score(img, width, height, pitch, x, y, t);
    int n = 0;
    for (int y = DETECT_BORDER; y <= height - 1 - DETECT_BORDER; ++y)
        for (int x = DETECT_BORDER; x <= width - 1 - DETECT_BORDER; ++x) {
            const int s = score[(int64_t)y * width + x];
            if (s == 0) continue;
            int keep = 1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    if ((dx || dy) && !(s > score[(int64_t)(y + dy) * width + (x + dx)])) keep = 0;
            if (!keep) continue;
            if (n < cap) {
                xs[n] = x;
                ys[n] = y;
                bins[n] = oracle_orientation_bin(img, pitch, x, y);
            }
            ++n;
        }
    free(score);
    return n;
}

/* ---------------------------------------------------------------------------
 * Multi-scale pyramid (Sec. 6).
 * ------------------------------------------------------------------------- */

/* Level image of scale s >= 1: out[y * out_pitch + x] = I(rha(s x), rha(s y)) for
 * x < floor(W / s), y < floor(H / s).  Writes the level's size to *lw, *lh. */
void oracle_pyramid_level(const uint8_t *img, int width, int height, int64_t pitch, double s, uint8_t *out,
                          int64_t out_pitch, int *lw, int *lh) {
    const int w = (int)floor((double)width / s), h = (int)floor((double)height / s);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const int64_t sx = (int64_t)round(s * (double)x), sy = (int64_t)round(s * (double)y);
            out[(int64_t)y * out_pitch + x] = img[sy * pitch + sx];
        }
    *lw = w;
    *lh = h;
}

/*
 * Oriented FAST keypoints of every pyramid level (scales[0 .. n) each >= 1), level
 * after level, each level in raster order of its own image, mapped to the base
 * image: (rha(s x), rha(s y)), the level's bin, scale index = the level.  Writes at
 * most `cap` keypoints and returns the number found, or -1 on bad arguments.
 */
int oracle_detect_pyramid(const uint8_t *img, int width, int height, int64_t pitch, int t, const double *scales,
                          int n, int cap, int32_t *xs, int32_t *ys, int32_t *bins, int32_t *levels) {
    if (n < 1 || cap < 0) return -1;
    int total = 0;
    for (int l = 0; l < n; ++l) {
        const double s = scales[l];
        if (!(s >= 1.0)) return -1;
        const int w = (int)floor((double)width / s), h = (int)floor((double)height / s);
        if (w < 1 || h < 1) continue;
        const int64_t lp = w;
        uint8_t *lev = (uint8_t *)malloc((size_t)w * (size_t)h);
        int32_t *lx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)w * (size_t)h / 4 + 1));
        int32_t *ly = (int32_t *)malloc(sizeof(int32_t) * ((size_t)w * (size_t)h / 4 + 1));
        int32_t *lb = (int32_t *)malloc(sizeof(int32_t) * ((size_t)w * (size_t)h / 4 + 1));
        if (!lev || !lx || !ly || !lb) {
            free(lev), free(lx), free(ly), free(lb);
            return -1;
        }
        int lw = 0, lh = 0;
        oracle_pyramid_level(img, width, height, pitch, s, lev, lp, &lw, &lh);
        /* strict suppression keeps at most one pixel of every 2x2 block */
        const int m = oracle_detect(lev, lw, lh, lp, t, w * h / 4 + 1, lx, ly, lb);
        if (m < 0) {
            free(lev), free(lx), free(ly), free(lb);
            return -1;
        }
        for (int i = 0; i < m; ++i, ++total)
            if (total < cap) {
                xs[total] = (int32_t)round(s * (double)lx[i]);
                ys[total] = (int32_t)round(s * (double)ly[i]);
                bins[total] = lb[i];
                levels[total] = l;
            }
        free(lev), free(lx), free(ly), free(lb);
    }
    return total;
}

/* ---------------------------------------------------------------------------
 * Dense per-pixel LATCH and matching (Sec. 6: CLATCH for dense pixel matching,
 * as an alternative to PatchMatch).  Readings: every pixel (x, y) of the image is
 * a keypoint at angle bin 0 and scale 1, so its window pixel (u, v) is image pixel
 * (x + u - 24, y + v - 24) (0 outside the image); descriptors are stored in raster
 * order, row y * width + x.  Pixel p of image A is matched against the pixels q of
 * image B (same size) with |q.x - p.x| <= R and |q.y - p.y| <= R that lie inside
 * B, taken in raster order of B, with the top-two rule and ratio test of
 * oracle_match (train index = raster index y * width + x of q in B).
 * ------------------------------------------------------------------------- */

/* Descriptors of every pixel: out receives width * height * 64 bytes.  Returns 0, or
 * -1 on an invalid triplet. */
int oracle_dense_extract(const uint8_t *img, int width, int height, int64_t pitch, const uint8_t *triplets,
                         uint8_t *out) {
    int32_t dx[WIN * WIN], dy[WIN * WIN], win[WIN * WIN];
    for (int t = 0; t < 6 * NBITS; ++t)
        if (triplets[t] < PATCH_R || triplets[t] > WIN - 1 - PATCH_R) return -1;
    oracle_offsets(1.0, 0, dx, dy);
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x) {
            sample_window(img, width, height, pitch, x, y, dx, dy, win);
            uint8_t *d = out + ((int64_t)y * width + x) * (NBITS / 8);
            memset(d, 0, NBITS / 8);
            for (int t = 0; t < NBITS; ++t) {
                const uint8_t *tr = triplets + 6 * t;
                int64_t d1 = patch_ssd(win, tr[0], tr[1], tr[2], tr[3]); /* ||P_A - P_1||^2 */
                int64_t d2 = patch_ssd(win, tr[0], tr[1], tr[4], tr[5]); /* ||P_A - P_2||^2 */
                if (d1 > d2) d[t >> 3] |= (uint8_t)(1u << (t & 7));
            }
        }
    return 0;
}

/* Windowed matching of two dense descriptor fields of width x height pixels: for
 * every pixel of A, the candidates of B within `radius` (Chebyshev) in raster order,
 * every distance, the smallest (lowest raster index on ties), the smallest over the
 * other candidates, then the ratio rule of oracle_match.  Outputs per pixel of A as
 * oracle_match.  Returns 0, or -1 on bad arguments. */
int oracle_dense_match(const uint8_t *da, const uint8_t *db, int width, int height, int radius, int k, float ratio,
                       int32_t *idx1, int32_t *idx2, int32_t *d1, int32_t *d2, uint8_t *accepted) {
    if (k != 1 && k != 2) return -1;
    if (!(ratio >= 0.0f && ratio <= 1.0f)) return -1;
    if (radius < 0 || width < 0 || height < 0) return -1;
    const int64_t r = (int64_t)round((double)ratio * 1000.0);
    const int64_t side = 2 * (int64_t)radius + 1;
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(side * side));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(side * side));
    if (!cand || !dist) {
        free(cand), free(dist);
        return -1;
    }
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x) {
            const int64_t p = (int64_t)y * width + x;
            int nc = 0;
            for (int qy = y - radius; qy <= y + radius; ++qy)
                for (int qx = x - radius; qx <= x + radius; ++qx) {
                    if (qx < 0 || qx >= width || qy < 0 || qy >= height) continue;
                    cand[nc] = qy * width + qx;
                    dist[nc] = oracle_hamming(da + p * 64, db + (int64_t)cand[nc] * 64, 64);
                    ++nc;
                }
            int b1 = -1, b2 = -1;
            for (int j = 0; j < nc; ++j)
                if (b1 < 0 || dist[j] < dist[b1]) b1 = j;
            if (k == 2)
                for (int j = 0; j < nc; ++j)
                    if (j != b1 && (b2 < 0 || dist[j] < dist[b2])) b2 = j;
            idx1[p] = b1 >= 0 ? cand[b1] : -1;
            idx2[p] = b2 >= 0 ? cand[b2] : -1;
            d1[p] = b1 >= 0 ? dist[b1] : 65535;
            d2[p] = b2 >= 0 ? dist[b2] : 65535;
            if (b1 < 0)
                accepted[p] = 0;
            else if (k == 1)
                accepted[p] = 1;
            else
                accepted[p] = (uint8_t)(1000 * (int64_t)d1[p] < r * (int64_t)d2[p]);
        }
    free(cand);
    free(dist);
    return 0;
}

// Dense per-pixel LATCH and windowed matching (Sec. 6: CLATCH for dense pixel
// matching, as an alternative to PatchMatch).
//
// Every pixel is an upright keypoint at scale 1, so a triplet (a, c1, c2) gives, at
// all pixels p at once,
//   D1(p) - D2(p) = sum over the 7x7 box of (A - C1)^2 - (A - C2)^2
//                 = box7[ (C2 - C1)(2A - C1 - C2) ](p),
// with A = I(p + a - 24 + d), C1, C2 likewise (Eq. 1; one product image per triplet,
// then a separable 7x7 box sum; all exact in int32, |box| <= 49 * 255 * 510).
//
// dense_extract_kernel: one block per 32x32-pixel tile; the image region under the
// tile and every window (79 x 79 bytes, 0 outside the image) is staged once in shared
// memory.  Per round two triplets t and t + 256:
//   phase A (304 threads, 2 x 38 rows x 4 segments): a thread forms the product image
//            along 14 pixels of one row (each patch's 14 bytes from five aligned
//            words) and writes 8 horizontal 7-sums;
//   phase B (256 threads, 2 x 32 columns x 4 segments): a thread adds 7 of them
//            vertically for 8 pixels of one column, and bit t of those pixels is
//            box > 0 (D1 > D2, strict).
// The horizontal sums are double-buffered, so one barrier separates the rounds;
// each phase-B thread gathers 32 consecutive bits per pixel in registers and
// writes the descriptor word once.
//
// dense_match_kernel: one block per 16x16 pixels of image A; the descriptors of B
// under the tile and its radius-R halo are staged in shared memory (16-byte chunks
// swizzled so that a warp's neighbouring descriptors hit different banks); each
// thread keeps its pixel's descriptor in registers and visits the (2R + 1)^2
// candidates in raster order of B (those inside B), computing XOR + population
// count (popc.cuh) and keeping the two best with strict comparisons, which is the
// lowest-raster-index tie rule.
#include <cstdint>

#include "internal.h"
#include "popc.cuh"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kTile = 32;                       // output pixels per tile side
constexpr int kRegion = kTile + kWin - 1;       // 79: staged image rows / columns
constexpr int kRegionPitch = 84;                // bytes per staged row (21 words: odd)
constexpr int kHRows = kTile + 2 * kPatchR;     // 38: rows of horizontal sums
constexpr int kHPitch = 36;                     // words per row of horizontal sums
constexpr int kSegs = 4;                        // 8-pixel segments per row / column
constexpr int kAThreads = kHRows * kSegs;       // 152 per triplet
constexpr int kBThreads = kTile * kSegs;        // 128 per triplet
constexpr int kDenseThreads = 320;
constexpr int kHalfBits = kBits / 2;            // triplets t and t + 256 share a round

struct DenseTriplets {
    latch_triplet t[kBits];
};

struct DenseSmem {
    uint8_t img[kRegion * kRegionPitch];
    uint8_t pad[16];                            // the last row's word loads may read past it
    uint16_t off[3][kBits];                     // staged-region offset of each patch's top-left pixel
    alignas(16) int32_t h[2][2][kHRows][kHPitch];  // [round parity][triplet slot][row][column]
};

__global__ void __launch_bounds__(kDenseThreads) dense_extract_kernel(const uint8_t* __restrict__ img, int width,
                                                                      int height, int64_t pitch,
                                                                      const __grid_constant__ DenseTriplets tr,
                                                                      uint32_t* __restrict__ out) {
    __shared__ __align__(16) DenseSmem S;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    griddep_wait();
    griddep_launch_dependents();
    // stage the region [x0 - 24, x0 + 55) x [y0 - 24, y0 + 55); samples outside read 0
    for (int i = tid; i < kRegion * kRegion; i += kDenseThreads) {
        const int rr = i / kRegion, cc = i - rr * kRegion;
        const int gy = y0 - kHalf + rr, gx = x0 - kHalf + cc;
        uint8_t v = 0;
        if (gx >= 0 && gx < width && gy >= 0 && gy < height) v = img[static_cast<int64_t>(gy) * pitch + gx];
        S.img[rr * kRegionPitch + cc] = v;
    }
    // patch at window point (x, y) of the pixel at tile offset (fx, fy): staged pixel
    // (fx + x - 3 + dx, fy + y - 3 + dy) for dx, dy in 0..6 -- the thread's base plus off
    for (int t = tid; t < kBits; t += kDenseThreads) {
        const uint8_t* c = &tr.t[t].ax;
        for (int p = 0; p < 3; ++p)
            S.off[p][t] = static_cast<uint16_t>((c[2 * p + 1] - kPatchR) * kRegionPitch + (c[2 * p] - kPatchR));
    }
    __syncthreads();

    // phase A role: slot ja, segment sa (pixels 8 sa .. 8 sa + 7), row ra of the
    // horizontal sums (image row y0 + ra - 3)
    const int ja = tid / kAThreads, la = tid - ja * kAThreads;
    const int sa = la / kHRows, ra = la - sa * kHRows;
    const uint8_t* abase = S.img + ra * kRegionPitch + kTile / kSegs * sa;
    // phase B role: slot jb, segment sb (rows 8 sb .. 8 sb + 7), column cb
    const int jb = tid / kBThreads, lb = tid - jb * kBThreads;
    const int sb = lb / kTile, cb = lb - sb * kTile;
    uint32_t bits[8] = {0, 0, 0, 0, 0, 0, 0, 0};

    // the 14 bytes at p as four words (byte i in byte i % 4 of word i / 4): five
    // aligned word loads and funnel shifts instead of 14 byte loads
    auto load14 = [](const uint8_t* p, uint32_t (&y)[4]) {
        const uintptr_t addr = reinterpret_cast<uintptr_t>(p);
        const uint32_t* w = reinterpret_cast<const uint32_t*>(addr & ~static_cast<uintptr_t>(3));
        const uint32_t sh = static_cast<uint32_t>(addr & 3u) * 8u;
        uint32_t x[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) x[q] = w[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) y[q] = __funnelshift_r(x[q], x[q + 1], sh);
    };
    auto byte_of = [](const uint32_t (&y)[4], int i) {
        return static_cast<int>(__byte_perm(y[i >> 2], 0u, 0x4440u | static_cast<uint32_t>(i & 3)));
    };
    auto phase_a = [&](int k) {
        const int t = ja * kHalfBits + k;
        uint32_t ya[4], y1[4], y2[4];
        load14(abase + S.off[0][t], ya);
        load14(abase + S.off[1][t], y1);
        load14(abase + S.off[2][t], y2);
        int f[14];
#pragma unroll
        for (int i = 0; i < 14; ++i) {
            const int a = byte_of(ya, i), c1 = byte_of(y1, i), c2 = byte_of(y2, i);
            f[i] = (c2 - c1) * (2 * a - c1 - c2);
        }
        int h[8];
        h[0] = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6];
#pragma unroll
        for (int j = 1; j < 8; ++j) h[j] = h[j - 1] + f[j + 6] - f[j - 1];
        int4* dst = reinterpret_cast<int4*>(&S.h[k & 1][ja][ra][kTile / kSegs * sa]);
        dst[0] = make_int4(h[0], h[1], h[2], h[3]);
        dst[1] = make_int4(h[4], h[5], h[6], h[7]);
    };

    if (tid < 2 * kAThreads) phase_a(0);
    __syncthreads();
    for (int k = 0; k < kHalfBits; ++k) {
        if (tid < 2 * kBThreads) {
            const int32_t* hc = &S.h[k & 1][jb][kTile / kSegs * sb][cb];
            int hv[14];
#pragma unroll
            for (int i = 0; i < 14; ++i) hv[i] = hc[i * kHPitch];
            int v = hv[0] + hv[1] + hv[2] + hv[3] + hv[4] + hv[5] + hv[6];
            const uint32_t b = static_cast<uint32_t>(k & 31);
            bits[0] |= static_cast<uint32_t>(v > 0) << b;
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                v += hv[j + 6] - hv[j - 1];
                bits[j] |= static_cast<uint32_t>(v > 0) << b;
            }
            if (b == 31) {
                // descriptor word (jb * 256 + k) / 32 of the segment's 8 pixels
                const int w = jb * (kHalfBits / 32) + (k >> 5);
                const int x = x0 + cb;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int y = y0 + kTile / kSegs * sb + j;
                    if (x < width && y < height) out[(static_cast<int64_t>(y) * width + x) * kDescWords + w] = bits[j];
                    bits[j] = 0;
                }
            }
        }
        if (k + 1 < kHalfBits && tid < 2 * kAThreads) phase_a(k + 1);
        __syncthreads();
    }
}

constexpr int kMTile = 16;          // pixels of A per tile side
constexpr int kMatchThreads = kMTile * kMTile;

// 16-byte chunk q of staged descriptor `cell`: chunks rotate with the cell so that
// the 8 neighbouring descriptors read by a quarter warp fill all 32 banks.
__device__ __forceinline__ int chunk_slot(int cell, int q) { return cell * 4 + ((q ^ (cell >> 1)) & 3); }

__global__ void __launch_bounds__(kMatchThreads) dense_match_kernel(const uint4* __restrict__ da,
                                                                    const uint4* __restrict__ db, int width,
                                                                    int height, int radius, int k, int r_milli,
                                                                    latch_match* __restrict__ out) {
    extern __shared__ uint4 s_desc[];
    const int side = kMTile + 2 * radius;
    const int x0 = blockIdx.x * kMTile, y0 = blockIdx.y * kMTile;
    griddep_wait();
    griddep_launch_dependents();
    for (int i = threadIdx.x; i < side * side * 4; i += kMatchThreads) {
        const int cell = i >> 2, q = i & 3;
        const int ry = cell / side, rx = cell - ry * side;
        const int gy = y0 - radius + ry, gx = x0 - radius + rx;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gx >= 0 && gx < width && gy >= 0 && gy < height) v = db[(static_cast<int64_t>(gy) * width + gx) * 4 + q];
        s_desc[chunk_slot(cell, q)] = v;
    }
    const int tx = threadIdx.x % kMTile, ty = threadIdx.x / kMTile;
    const int px = x0 + tx, py = y0 + ty;
    const bool live = px < width && py < height;
    uint32_t a[16];
    if (live) {
        const uint4* src = da + (static_cast<int64_t>(py) * width + px) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = src[q];
            a[4 * q] = v.x, a[4 * q + 1] = v.y, a[4 * q + 2] = v.z, a[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int w = 0; w < 16; ++w) a[w] = 0;
    }
    __syncthreads();
    if (!live) return;
    int d1 = 0x7fffffff, d2 = 0x7fffffff, i1 = -1, i2 = -1;
    const int ylo = py - radius < 0 ? 0 : py - radius, yhi = py + radius >= height ? height - 1 : py + radius;
    const int xlo = px - radius < 0 ? 0 : px - radius, xhi = px + radius >= width ? width - 1 : px + radius;
    for (int qy = ylo; qy <= yhi; ++qy) {
        const int rowcell = (qy - y0 + radius) * side - x0 + radius;
        for (int qx = xlo; qx <= xhi; ++qx) {
            const int cell = rowcell + qx;
            uint32_t x[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = s_desc[chunk_slot(cell, q)];
                x[4 * q] = v.x ^ a[4 * q], x[4 * q + 1] = v.y ^ a[4 * q + 1];
                x[4 * q + 2] = v.z ^ a[4 * q + 2], x[4 * q + 3] = v.w ^ a[4 * q + 3];
            }
            const int d = popc16(x);
            const int idx = qy * width + qx;
            if (d < d1) {
                d2 = d1, i2 = i1;
                d1 = d, i1 = idx;
            } else if (d < d2) {
                d2 = d, i2 = idx;
            }
        }
    }
    latch_match m;
    m.idx1 = i1;
    m.dist1 = static_cast<uint16_t>(d1);
    const bool has2 = k == 2 && i2 >= 0;
    m.idx2 = has2 ? i2 : -1;
    m.dist2 = has2 ? static_cast<uint16_t>(d2) : 0xffff;
    if (k == 1)
        m.accepted = 1;
    else
        m.accepted = (1000ll * m.dist1 < static_cast<long long>(r_milli) * m.dist2) ? 1 : 0;
    m.pad[0] = m.pad[1] = m.pad[2] = 0;
    out[static_cast<int64_t>(py) * width + px] = m;
}

}  // namespace

static size_t dense_match_smem_bytes(int radius) {
    const size_t side = static_cast<size_t>(kMTile + 2 * radius);
    return side * side * kDescBytes;
}

cudaError_t launch_dense_extract(const latch_context* ctx, const latch_image* img, uint8_t* d_out,
                                 cudaStream_t stream) {
    DenseTriplets tr;
    for (int t = 0; t < kBits; ++t) tr.t[t] = ctx->h_trip[t];
    const dim3 grid(static_cast<unsigned>((img->width + kTile - 1) / kTile),
                    static_cast<unsigned>((img->height + kTile - 1) / kTile));
    return launch_chained(dense_extract_kernel, grid, dim3(kDenseThreads), 0, stream, img->data, img->width,
                          img->height, img->pitch, tr, reinterpret_cast<uint32_t*>(d_out));
}

static cudaError_t set_dense_match_attributes() {
    return cudaFuncSetAttribute(dense_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(dense_match_smem_bytes(kDenseMaxRadius)));
}

cudaError_t launch_dense_match(const uint8_t* d_a, const uint8_t* d_b, int32_t width, int32_t height, int32_t radius,
                               int32_t k, int32_t r_milli, latch_match* d_out, cudaStream_t stream) {
    static unsigned long long attr_done = 0;
    const cudaError_t e = once_per_device(&attr_done, set_dense_match_attributes);
    if (e != cudaSuccess) return e;
    const dim3 grid(static_cast<unsigned>((width + kMTile - 1) / kMTile),
                    static_cast<unsigned>((height + kMTile - 1) / kMTile));
    return launch_chained(dense_match_kernel, grid, dim3(kMatchThreads), dense_match_smem_bytes(radius), stream,
                          reinterpret_cast<const uint4*>(d_a), reinterpret_cast<const uint4*>(d_b), width, height,
                          radius, k, r_milli, d_out);
}

}  // namespace latch

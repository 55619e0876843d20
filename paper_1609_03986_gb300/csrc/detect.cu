// Oriented FAST keypoints on the GPU (Sec. 3.2: keypoints come from the FAST
// detector, and their orientation sets the angle at which the LATCH window is read).
//
// Readings (the paper names the detector only): FAST-9 segment test on the
// radius-3 Bresenham circle, a corner's score is the largest threshold at which it
// is still a corner, a corner is kept when its score is strictly larger than each
// of its 8 neighbours', only pixels at least 16 from every border are detected, and
// the orientation is the intensity centroid of the radius-15 disc quantised to the
// 32 angle bins (round half away from zero of theta * 16 / pi, FP64).
//
// Pyramid (Sec. 6, CLATCH at multiple scales; reading: level s is the base image
// sampled at spacing s, I_s(x, y) = I(rha(s x), rha(s y)), x < floor(W / s), the
// nearest-pixel rule of the scaled window): pyramid_level_kernel writes the levels
// with s != 1, and one launch of each kernel below covers every level; a level
// keypoint (x, y) is written as the base keypoint (rha(s x), rha(s y)) with the
// level's scale index, levels one after another.
//
// Three chained kernels per image (all levels):
//   detect_cells_kernel   one block per 32x32 cell: the cell plus a 16-pixel halo
//                         (64 x 64 bytes) is staged in shared memory; scores of the
//                         cell and a 1-pixel apron; suppression; the cell's survivors
//                         in raster order, each oriented by one warp; the cell's
//                         count and its survivors (2 bytes each) go to scratch;
//   detect_scan_kernel    one block: exclusive scan of the cell counts, total count;
//   detect_expand_kernel  one warp per cell: keypoint records at the cell's offset
//                         (cells row by row, raster order inside a cell), the first
//                         max_kps of them.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kCellD = 32;          // detection cell (the extraction's cell size)
constexpr int kHaloD = 16;          // staged halo: the centroid disc (15) + 1
constexpr int kTileD = kCellD + 2 * kHaloD;  // 64
constexpr int kApron = kCellD + 2;           // scores of the cell and a 1-pixel apron
constexpr int kDetThreads = 256;
constexpr int kDiscR = 15;
constexpr int kMaxPerCell = kCellD * kCellD / 4;  // strict 3x3 suppression keeps at most one pixel per 2x2
constexpr double kPi = 3.141592653589793;

// Circle offsets in circular order (x right, y down), clockwise from the top.
__constant__ int8_t c_circle[16][2] = {{0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0},  {3, 1},  {2, 2},  {1, 3},
                                       {0, 3},  {-1, 3}, {-2, 2}, {-3, 1}, {-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}};

// FAST score of the pixel at tile position (tx, ty): the best arc of 9 over both
// polarities, max over arcs of min over the arc of (I_k - I_p) (bright) or of
// (I_p - I_k) (dark), minus 1; 0 when below t.
__device__ __forceinline__ int fast_score(const uint8_t (*tile)[kTileD], int tx, int ty, int t) {
    const int p = tile[ty][tx];
    // quick rejection: a run of 9 covers two neighbouring compass points (0, 4, 8, 12)
    const int n0 = tile[ty - 3][tx], n4 = tile[ty][tx + 3], n8 = tile[ty + 3][tx], n12 = tile[ty][tx - 3];
    const int hi = p + t, lo = p - t;
    const bool b0 = n0 > hi, b4 = n4 > hi, b8 = n8 > hi, b12 = n12 > hi;
    const bool d0 = n0 < lo, d4 = n4 < lo, d8 = n8 < lo, d12 = n12 < lo;
    const bool bright = (b0 && b4) || (b4 && b8) || (b8 && b12) || (b12 && b0);
    const bool dark = (d0 && d4) || (d4 && d8) || (d8 && d12) || (d12 && d0);
    if (!bright && !dark) return 0;
    int d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) d[k] = static_cast<int>(tile[ty + c_circle[k][1]][tx + c_circle[k][0]]) - p;
    // windowed min / max of 9 consecutive (circularly) from windows of 2, 4, 8
    int mn2[16], mx2[16], mn4[16], mx4[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        mn2[k] = min(d[k], d[(k + 1) & 15]);
        mx2[k] = max(d[k], d[(k + 1) & 15]);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        mn4[k] = min(mn2[k], mn2[(k + 2) & 15]);
        mx4[k] = max(mx2[k], mx2[(k + 2) & 15]);
    }
    int best_b = -1000, best_d = -1000;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int mn9 = min(min(mn4[k], mn4[(k + 4) & 15]), d[(k + 8) & 15]);
        const int mx9 = max(max(mx4[k], mx4[(k + 4) & 15]), d[(k + 8) & 15]);
        best_b = max(best_b, mn9);
        best_d = max(best_d, -mx9);
    }
    const int s = max(best_b, best_d) - 1;
    return s >= t ? s : 0;
}

struct DetectLevel {
    const uint8_t* img;  // the level image (the base image for scale 1)
    int64_t pitch;
    int32_t width, height;
    int32_t gx, gy;      // cells per row / column
    int32_t cell0;       // the level's first cell in the launch's cell numbering
    int32_t scale_idx;   // written into the level's keypoints
    double scale;        // base coordinate = rha(scale * level coordinate)
};

struct DetectParams {
    DetectLevel lv[kMaxDetectLevels];
    int32_t nlev;
    int32_t ncells;      // cells of all levels
    int32_t t;           // FAST threshold
    int32_t max_kps;
};

// Level of global cell `cell` (largest l with lv[l].cell0 <= cell).
__device__ __forceinline__ int level_of_cell(const DetectParams& prm, int cell) {
    int l = 0;
    for (int i = 1; i < prm.nlev; ++i)
        if (prm.lv[i].cell0 <= cell) l = i;
    return l;
}

__global__ void __launch_bounds__(kDetThreads) detect_cells_kernel(const DetectParams prm, int32_t* __restrict__ counts,
                                                                   uint16_t* __restrict__ slots) {
    __shared__ __align__(16) uint8_t tile[kTileD][kTileD];
    __shared__ uint8_t sc[kApron][kApron];
    __shared__ uint16_t keep[kMaxPerCell];
    __shared__ int warp_tot[kDetThreads / 32];
    griddep_wait();
    griddep_launch_dependents();
    const int cell = blockIdx.x;
    const DetectLevel& L = prm.lv[level_of_cell(prm, cell)];
    const int lc = cell - L.cell0;
    const int cx = lc % L.gx, cy = lc / L.gx;
    const int x0 = cx * kCellD, y0 = cy * kCellD;
    const int W = L.width, H = L.height;
    // the detection region [16, W-17] x [16, H-17] meets this cell?
    const int rx0 = max(x0, kHaloD), rx1 = min(x0 + kCellD - 1, W - 1 - kHaloD);
    const int ry0 = max(y0, kHaloD), ry1 = min(y0 + kCellD - 1, H - 1 - kHaloD);
    if (rx0 > rx1 || ry0 > ry1) {
        if (threadIdx.x == 0) counts[cell] = 0;
        return;
    }
    // ---- stage rows y0-16 .. y0+47, columns x0-16 .. x0+47 (zero outside the image) ----
    {
        const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
        const int gy = y0 - kHaloD + r, gx = x0 - kHaloD + 16 * q;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const uint8_t* src = L.img + static_cast<int64_t>(gy) * L.pitch + gx;
            if (gx + 16 <= W) {
                v = *reinterpret_cast<const uint4*>(src);
            } else {  // the image's last bytes of the row: no read past the width
                union {
                    uint4 v;
                    uint8_t b[16];
                } u;
#pragma unroll
                for (int i = 0; i < 16; ++i) u.b[i] = gx + i < W ? src[i] : 0;
                v = u.v;
            }
        }
        *reinterpret_cast<uint4*>(&tile[r][16 * q]) = v;
    }
    __syncthreads();
    // ---- scores of pixels x0-1 .. x0+32, y0-1 .. y0+32 (0 where the circle leaves the image) ----
    for (int i = threadIdx.x; i < kApron * kApron; i += kDetThreads) {
        const int ay = i / kApron, ax = i % kApron;
        const int gx = x0 - 1 + ax, gy = y0 - 1 + ay;
        int s = 0;
        if (gx >= 3 && gy >= 3 && gx < W - 3 && gy < H - 3) s = fast_score(tile, ax + kHaloD - 1, ay + kHaloD - 1, prm.t);
        sc[ay][ax] = static_cast<uint8_t>(s);
    }
    __syncthreads();
    // ---- suppression: thread = 4 consecutive pixels of one cell row (raster order) ----
    const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = c0 + j;
        const int gx = x0 + c, gy = y0 + r;
        const int s = sc[r + 1][c + 1];
        bool k = s > 0 && gx >= rx0 && gx <= rx1 && gy >= ry0 && gy <= ry1;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx)
                if (dx || dy) k = k && s > sc[r + 1 + dy][c + 1 + dx];
        mask |= static_cast<uint32_t>(k) << j;
    }
    // exclusive scan of the per-thread counts (thread order = raster order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kDetThreads / 32; ++w) {
        base += w < warp ? warp_tot[w] : 0;
        total += warp_tot[w];
    }
    int pos = base + incl - cnt;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (mask & (1u << j)) keep[pos++] = static_cast<uint16_t>((r << 5) | (c0 + j));
    __syncthreads();
    // ---- orientation: one warp per survivor; lane l covers dx = l - 15 of every disc row ----
    const int dxl = lane - kDiscR;
    for (int i = warp; i < total; i += kDetThreads / 32) {
        const int rr = keep[i] >> 5, cc = keep[i] & 31;
        const int tx = cc + kHaloD, ty = rr + kHaloD;
        int m10 = 0, m01 = 0;
        if (lane <= 2 * kDiscR) {
#pragma unroll
            for (int dy = -kDiscR; dy <= kDiscR; ++dy)
                if (dxl * dxl + dy * dy <= kDiscR * kDiscR) {
                    const int v = tile[ty + dy][tx + dxl];
                    m10 += dxl * v;
                    m01 += dy * v;
                }
        }
        m10 = __reduce_add_sync(0xffffffffu, m10);
        m01 = __reduce_add_sync(0xffffffffu, m01);
        if (lane == 0) {
            const double theta = atan2(static_cast<double>(m01), static_cast<double>(m10));
            const int b = static_cast<int>(round(theta * 16.0 / kPi));
            const int bin = ((b % 32) + 32) % 32;
            slots[static_cast<int64_t>(cell) * kMaxPerCell + i] = static_cast<uint16_t>((bin << 10) | keep[i]);
        }
    }
    if (threadIdx.x == 0) counts[cell] = total;
}

// Exclusive scan of the cell counts in place (offsets), total -> *d_count.
__global__ void __launch_bounds__(1024) detect_scan_kernel(int32_t* __restrict__ counts, int32_t ncells,
                                                           int32_t* __restrict__ d_count) {
    __shared__ int part[32];
    griddep_wait();
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int c0 = 0; c0 < ncells; c0 += 8 * 1024) {
        const int c = c0 + 8 * threadIdx.x;
        int v[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = c + q < ncells ? counts[c + q] : 0;
            sum += v[q];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        __syncthreads();
        if (lane == 31) part[warp] = incl;
        __syncthreads();
        int run = carry + incl - sum, tile_total = 0;
        for (int w = 0; w < 32; ++w) {
            run += w < warp ? part[w] : 0;
            tile_total += part[w];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (c + q < ncells) {
                counts[c + q] = run;
                run += v[q];
            }
        carry += tile_total;
    }
    if (threadIdx.x == 0) *d_count = carry;
}

// One warp per cell: its survivors become keypoint records at the cell's offset.
// `counts` holds the offsets now; the cell's count is the next offset minus its own.
__global__ void __launch_bounds__(256) detect_expand_kernel(const DetectParams prm, const int32_t* __restrict__ offsets,
                                                            const int32_t* __restrict__ d_count,
                                                            const uint16_t* __restrict__ slots,
                                                            latch_keypoint* __restrict__ out) {
    griddep_wait();
    griddep_launch_dependents();
    const int ncells = prm.ncells;
    const int cell = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= ncells) return;
    const DetectLevel& L = prm.lv[level_of_cell(prm, cell)];
    const int o = offsets[cell];
    const int n = (cell + 1 < ncells ? offsets[cell + 1] : *d_count) - o;
    const int lc = cell - L.cell0;
    const int x0 = (lc % L.gx) * kCellD, y0 = (lc / L.gx) * kCellD;
    for (int i = lane; i < n && o + i < prm.max_kps; i += 32) {
        const uint32_t v = slots[static_cast<int64_t>(cell) * kMaxPerCell + i];
        const int32_t lx = x0 + static_cast<int32_t>(v & 31u), ly = y0 + static_cast<int32_t>((v >> 5) & 31u);
        latch_keypoint k;
        if (L.scale == 1.0) {
            k.x = lx;
            k.y = ly;
        } else {  // FP64 product, rounded half away from zero (non-negative here)
            k.x = static_cast<int32_t>(round(L.scale * static_cast<double>(lx)));
            k.y = static_cast<int32_t>(round(L.scale * static_cast<double>(ly)));
        }
        k.angle_bin = static_cast<uint8_t>(v >> 10);
        k.scale_idx = static_cast<uint8_t>(L.scale_idx);
        k.reserved = 0;
        out[o + i] = k;
    }
}

// Level images of the levels with scale != 1: one thread per 16 output bytes of a
// row, rows of all levels in one grid (row r of the launch is level `lev`'s row
// r - row0[lev]).  out(x, y) = base(rha(s x), rha(s y)).
struct ResampleParams {
    const uint8_t* base;
    int64_t base_pitch;
    uint8_t* out[kMaxDetectLevels];
    int64_t pitch[kMaxDetectLevels];
    int32_t width[kMaxDetectLevels];
    int32_t row0[kMaxDetectLevels + 1];  // first launch row of each level; row0[n] = rows of all levels
    double scale[kMaxDetectLevels];
    int32_t n;
    int32_t chunks;  // 16-byte chunks per launch row: those of the widest level
};

__global__ void __launch_bounds__(256) pyramid_level_kernel(const ResampleParams prm) {
    griddep_wait();
    griddep_launch_dependents();
    const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t chunks_per_row = prm.chunks;
    const int64_t row = gid / chunks_per_row;
    if (row >= prm.row0[prm.n]) return;
    int l = 0;
    while (l + 1 < prm.n && prm.row0[l + 1] <= row) ++l;
    const int y = static_cast<int>(row - prm.row0[l]);
    const int x0 = static_cast<int>(gid % chunks_per_row) * 16;
    const int w = prm.width[l];
    if (x0 >= w) return;
    const double s = prm.scale[l];
    const uint8_t* src = prm.base + static_cast<int64_t>(round(s * static_cast<double>(y))) * prm.base_pitch;
    union {
        uint4 v;
        uint8_t b[16];
    } u;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        u.b[i] = x0 + i < w ? src[static_cast<int64_t>(round(s * static_cast<double>(x0 + i)))] : 0;
    *reinterpret_cast<uint4*>(prm.out[l] + static_cast<int64_t>(y) * prm.pitch[l] + x0) = u.v;
}

}  // namespace

// Size of pyramid level s of a W x H image (the same expression as the reading).
static void level_size(int32_t w, int32_t h, double s, int32_t* lw, int32_t* lh) {
    *lw = static_cast<int32_t>(std::floor(static_cast<double>(w) / s));
    *lh = static_cast<int32_t>(std::floor(static_cast<double>(h) / s));
}

static int64_t level_pitch(int32_t lw) { return (static_cast<int64_t>(lw) + 15) / 16 * 16; }

static int64_t cells_of(int32_t w, int32_t h) {
    return static_cast<int64_t>((w + kCellD - 1) / kCellD) * ((h + kCellD - 1) / kCellD);
}

size_t detect_scratch_bytes(const latch_image* img, const double* scales, int nlev) {
    int64_t ncells = 0;
    size_t level_bytes = 0;
    for (int l = 0; l < nlev; ++l) {
        int32_t lw, lh;
        level_size(img->width, img->height, scales[l], &lw, &lh);
        if (lw < 1 || lh < 1) continue;
        ncells += cells_of(lw, lh);
        if (scales[l] != 1.0) level_bytes += (static_cast<size_t>(lh) * level_pitch(lw) + 255) / 256 * 256;
    }
    return (static_cast<size_t>(ncells) * 4 + 255) / 256 * 256 +
           (static_cast<size_t>(ncells) * kMaxPerCell * sizeof(uint16_t) + 255) / 256 * 256 + level_bytes + 256;
}

cudaError_t launch_detect(const latch_image* img, const double* scales, const int32_t* scale_idx, int nlev,
                          int32_t threshold, int32_t max_kps, latch_keypoint* d_kps, int32_t* d_count, void* scratch,
                          cudaStream_t stream) {
    DetectParams prm;
    ResampleParams rs;
    rs.base = img->data;
    rs.base_pitch = img->pitch;
    rs.n = 0;
    rs.row0[0] = 0;
    rs.chunks = 1;
    prm.nlev = 0;
    prm.t = threshold;
    prm.max_kps = max_kps;
    int64_t ncells = 0;
    for (int l = 0; l < nlev; ++l) {
        int32_t lw, lh;
        level_size(img->width, img->height, scales[l], &lw, &lh);
        if (lw < 1 || lh < 1) continue;
        DetectLevel& L = prm.lv[prm.nlev++];
        L.width = lw;
        L.height = lh;
        L.gx = (lw + kCellD - 1) / kCellD;
        L.gy = (lh + kCellD - 1) / kCellD;
        L.cell0 = static_cast<int32_t>(ncells);
        L.scale_idx = scale_idx[l];
        L.scale = scales[l];
        L.img = img->data;
        L.pitch = img->pitch;
        ncells += cells_of(lw, lh);
    }
    prm.ncells = static_cast<int32_t>(ncells);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    int32_t* counts = reinterpret_cast<int32_t*>(base);
    size_t off = (static_cast<size_t>(ncells) * 4 + 255) / 256 * 256;
    uint16_t* slots = reinterpret_cast<uint16_t*>(base + off);
    off += (static_cast<size_t>(ncells) * kMaxPerCell * sizeof(uint16_t) + 255) / 256 * 256;
    for (int l = 0; l < prm.nlev; ++l) {
        DetectLevel& L = prm.lv[l];
        if (L.scale == 1.0) continue;
        const int k = rs.n++;
        L.img = base + off;
        L.pitch = level_pitch(L.width);
        rs.out[k] = base + off;
        rs.pitch[k] = L.pitch;
        rs.width[k] = L.width;
        rs.scale[k] = L.scale;
        rs.row0[k + 1] = rs.row0[k] + L.height;
        rs.chunks = std::max<int32_t>(rs.chunks, (L.width + 15) / 16);
        off += (static_cast<size_t>(L.height) * L.pitch + 255) / 256 * 256;
    }
    cudaError_t e = cudaSuccess;
    if (rs.n > 0) {
        const int64_t threads = static_cast<int64_t>(rs.row0[rs.n]) * rs.chunks;
        e = launch_chained(pyramid_level_kernel, dim3(static_cast<unsigned>((threads + 255) / 256)), dim3(256), 0,
                           stream, rs);
    }
    if (e != cudaSuccess) return e;
    if (ncells == 0) return cudaMemsetAsync(d_count, 0, sizeof(int32_t), stream);
    e = launch_chained(detect_cells_kernel, dim3(static_cast<unsigned>(ncells)), dim3(kDetThreads), 0, stream, prm,
                       counts, slots);
    if (e == cudaSuccess)
        e = launch_chained(detect_scan_kernel, dim3(1), dim3(1024), 0, stream, counts, static_cast<int32_t>(ncells),
                           d_count);
    if (e == cudaSuccess)
        e = launch_chained(detect_expand_kernel, dim3(static_cast<unsigned>((ncells + 7) / 8)), dim3(256), 0, stream,
                           prm, static_cast<const int32_t*>(counts), static_cast<const int32_t*>(d_count),
                           static_cast<const uint16_t*>(slots), d_kps);
    return e;
}

}  // namespace latch

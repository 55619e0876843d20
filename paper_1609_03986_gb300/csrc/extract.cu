// LATCH descriptor extraction (Sec. 3.1 Eq. 1; Sec. 3.2).
//
// 1. sort_count_kernel + sort_scatter_kernel (1024 keypoints per block): counting
//    sort of the keypoints into 32x32-pixel image cells; the launch's record array
//    receives one 16-byte record per keypoint (position, output row, offset table,
//    image), cell by cell.  The
//    cell grid reaches 128 px beyond every border; keypoints further out have
//    windows wholly outside the image (the window reaches at most `reach` <= 78
//    px), whose samples all read 0, so their descriptor is all zeros and is written
//    here directly.  Keypoints with a scale index outside the scale table also get
//    zeros and raise the context's device flag.
// 2. extract_lanes_kernel (one block of 28 warps per SM): the records are taken 32
//    at a time ("batches", in sort order), one keypoint per lane.  A batch's work
//    is 64 chunks of 8 triplets; the chunks of all batches are split into G equal
//    contiguous ranges, range b for block b, so a batch may be shared by two
//    blocks (each builds its windows and evaluates its own chunks).  The block
//    is a two-stage pipeline over double-buffered windows:
//      - 12 builder warps build the 32 windows of batch i: for each run of
//        keypoints in one image cell, the tile under the cell plus a `reach`
//        halo is staged into shared memory by one TMA 2-D load (samples outside
//        the image arrive as 0, the border reading; two tile slots, the next
//        run's tile requested while the current one is read), and every window
//        pixel is read from it through the per-(scale, bin) offset table
//        (nearest pixel; offsets pre-multiplied into tile offsets), in units of
//        half a window spread over the builder warps, each warp loading the
//        table words of its next unit while it gathers the current one.  Window
//        j sits at word 577 j: with an odd stride, the 32 lanes reading the same
//        word of their windows hit 32 different banks;
//      - 16 evaluator warps evaluate Eq. 1 on batch i - 1, warp w on chunks 4w ..
//        4w+3, all 32 lanes on the same triplet at a time (the triplet table is
//        staged in shared memory: one broadcast load per triplet): a 7-pixel
//        patch row is two or three words, aligned by a funnel shift; D1 - D2 =
//        (sum C1^2 - sum C2^2) - 2 (sum A.C1 - sum A.C2) over the 7 rows with
//        __dp4a, all exact in 32-bit integers.  Each warp writes its bytes of
//        every lane's descriptor (bit t = bit t % 8 of byte t / 8) and, when
//        the caller also wants the tensor matcher's input, its 16 bytes of the
//        expanded row (4-bit value t = E2M1 -1.0 or +1.0 for bit t set or clear).
//    The stages hand the window buffers over through mbarriers (full: 384
//    builder arrivals, empty: 16 evaluator arrivals); every wait is bounded.
#include <cuda.h>

#include <cstdint>
#include <cstring>

#include "internal.h"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kCell = 32;
constexpr int kMargin = 128;            // cell grid reaches this far beyond each border
constexpr int kBuildWarps = 12;         // window builders (4, 8, 16 measured slower)
constexpr int kComputeWarps = 16;       // Eq. 1 evaluators (4 chunks each per batch)
constexpr int kBuildThreads = 32 * kBuildWarps;
constexpr int kComputeThreads = 32 * kComputeWarps;
constexpr int kThreads = kBuildThreads + kComputeThreads;  // 896
constexpr int kRowWords = 12;           // 48 bytes per window row
constexpr int kWinWords = kWinPix / 4;  // 576 words per window
constexpr int kLaneWords = kWinWords + 1;          // window stride: odd, so a warp's same-offset loads hit 32 banks
constexpr int kBatch = 32;              // keypoints per batch, one per lane
constexpr int kChunks = kBits / 8;      // chunks of 8 triplets per batch
constexpr int kSortThreads = 256;
constexpr int kSortKps = 1024;          // keypoints per sorting block (4 per thread)

struct CellGrid {
    int gx, gy;  // cells in x / y (including the margins)
    int width, height;
};

// Cell of a keypoint: >= 0, -1 (window wholly outside: zero descriptor), -2 (bad scale).
__device__ __forceinline__ int cell_of(const latch_keypoint& kp, int nscales, const CellGrid& g) {
    if (kp.scale_idx >= nscales) return -2;
    const int64_t x = static_cast<int64_t>(kp.x) + kMargin, y = static_cast<int64_t>(kp.y) + kMargin;
    if (x < 0 || y < 0 || x >= static_cast<int64_t>(g.width) + 2 * kMargin ||
        y >= static_cast<int64_t>(g.height) + 2 * kMargin)
        return -1;
    return static_cast<int>(y / kCell) * g.gx + static_cast<int>(x / kCell);
}

struct TileGeom {
    int tw, th;      // staged tile (bytes per row, rows)
    int mx, my;      // tile origin relative to the cell origin (negative)
};

// Per-launch description of a batch of images (kernel parameters).
template <int NI>
struct ExtractParams {
    CUtensorMap map[NI];  // one TMA map per image
    CellGrid grid[NI];
    int32_t kp0[NI];      // first keypoint of image i in the concatenated keypoint array
    int32_t n[NI];        // keypoints of image i
    int32_t cell0[NI];    // first entry of image i in the global cell-count scratch
    int32_t blk0[NI];     // first sorting block of image i (ceil(n / kSortKps) blocks each)
    int32_t count;        // images in this launch
    int32_t nscales;
    TileGeom tg;
    const int32_t* n_dev;  // single-image launches: the keypoint count on the device (n[0] is its bound), or NULL
};

// Keypoints of image `img` in this launch.
template <int NI>
__device__ __forceinline__ int keypoints_of(const ExtractParams<NI>& prm, int img) {
    const int n = prm.n[img];
    if (!prm.n_dev) return n;
    const int d = *prm.n_dev;
    return d < n ? (d > 0 ? d : 0) : n;
}

// Sorted keypoint record: x, y, output row (the keypoint's index), table (scale *
// 32 + bin) | launch-local image << 16.
__device__ __forceinline__ int4 kp_record(const latch_keypoint& kp, int row, int img) {
    return make_int4(kp.x, kp.y, row, (kp.scale_idx * kBins + (kp.angle_bin & (kBins - 1))) | (img << 16));
}

// Image of sorting block `blk` (largest i with blk0[i] <= blk).
template <int NI>
__device__ __forceinline__ int image_of_block(const ExtractParams<NI>& prm, int blk) {
    int lo = 0, hi = prm.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prm.blk0[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Sorting, pass 1 (kSortKps keypoints of one image per block): the cell of every
// keypoint; a keypoint with a cell takes its rank in the cell from an atomic on the
// cell's count (order of arrival), one without gets its zero descriptor here.  The
// last block of an image to finish turns the image's counts into exclusive starts.
// Scratch zeroed by the host: img_tot / img_done, the cell counts.
template <int NI>
__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(
    const __grid_constant__ ExtractParams<NI> prm, const latch_keypoint* __restrict__ kps, int* __restrict__ cells,
    int* __restrict__ rank, int* __restrict__ img_tot, int* __restrict__ img_done, uint4* __restrict__ out,
    uint4* __restrict__ exp_out, uint32_t* __restrict__ flags) {
    __shared__ int s_part[kSortThreads / 32];
    __shared__ int s_flag;
    griddep_wait();
    griddep_launch_dependents();
    const int img = image_of_block(prm, blockIdx.x);
    const CellGrid g = prm.grid[img];
    const int n = keypoints_of(prm, img), kp0 = prm.kp0[img];
    int* cnt = cells + prm.cell0[img];
    const int i0 = (blockIdx.x - prm.blk0[img]) * kSortKps + threadIdx.x;
    // all loads first, then the atomics
    latch_keypoint kp[kSortKps / kSortThreads];
#pragma unroll
    for (int q = 0; q < kSortKps / kSortThreads; ++q)
        if (i0 + q * kSortThreads < n) kp[q] = kps[kp0 + i0 + q * kSortThreads];
    int valid = 0;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < kSortKps / kSortThreads; ++q) {
        const int i = i0 + q * kSortThreads;
        const int c = i < n ? cell_of(kp[q], prm.nscales, g) : -3;
        if (c >= 0) {
            rank[kp0 + i] = atomicAdd(&cnt[c], 1);
            ++valid;
        } else if (c > -3) {
            const uint4 z = make_uint4(0, 0, 0, 0);
            uint4* d = out + static_cast<size_t>(kp0 + i) * 4;
            d[0] = z;
            d[1] = z;
            d[2] = z;
            d[3] = z;
            if (exp_out) {  // the expanded row of the zero descriptor: every value +1.0
                uint4* x = exp_out + static_cast<size_t>(kp0 + i) * (kExpRowBytes / 16);
                const uint4 one = expand_word_e2m1(0u);
                for (int u = 0; u < kExpRowBytes / 16; ++u) x[u] = one;
            }
            bad |= (c == -2);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    valid = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(valid));
    if (lane == 0) s_part[warp] = valid;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagBadScale);
    if (threadIdx.x == 0) {
        int v = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) v += s_part[w];
        atomicAdd(&img_tot[img], v);
        // release: the block's count increments (ordered before this by the barrier
        // above) and its total, before its arrival
        __threadfence();
        const int nblk = (prm.n[img] + kSortKps - 1) / kSortKps;  // every launched block of the image arrives
        s_flag = atomicAdd(&img_done[img], 1) == nblk - 1;
    }
    __syncthreads();
    if (!s_flag) return;
    // ---- last block of the image: exclusive starts of its cells, in place, in
    // tiles of 8 cells per thread (eight independent loads in flight) ----
    __threadfence();
    const int ncell = g.gx * g.gy;
    int carry = 0;
    for (int tb = 0; tb < ncell; tb += 8 * kSortThreads) {
        const int c0 = tb + 8 * threadIdx.x;
        int v[8];
        int sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = c0 + q < ncell ? __ldcg(&cnt[c0 + q]) : 0;
            sum += v[q];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        __syncthreads();  // s_part free (its previous readers are done)
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        int run = carry + incl - sum, tile_total = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const int x = s_part[w];
            if (w < warp) run += x;
            tile_total += x;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (c0 + q < ncell) {
                cnt[c0 + q] = run;
                run += v[q];
            }
        carry += tile_total;
    }
}

// Sorting, pass 2 (same blocks): each keypoint with a cell writes its record at
// image base + cell start + rank; the records of all images are contiguous, image
// by image (base = the totals of the earlier images).  Block 0 sets counters[0] =
// the launch's number of records.
template <int NI>
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(
    const __grid_constant__ ExtractParams<NI> prm, const latch_keypoint* __restrict__ kps,
    const int* __restrict__ cells, const int* __restrict__ rank, const int* __restrict__ img_tot,
    int* __restrict__ counters, int4* __restrict__ recs) {
    __shared__ int s_base;
    griddep_wait();
    griddep_launch_dependents();
    const int img = image_of_block(prm, blockIdx.x);
    const CellGrid g = prm.grid[img];
    const int n = keypoints_of(prm, img), kp0 = prm.kp0[img];
    const int* start = cells + prm.cell0[img];
    const int i0 = (blockIdx.x - prm.blk0[img]) * kSortKps + threadIdx.x;
    latch_keypoint kp[kSortKps / kSortThreads];
#pragma unroll
    for (int q = 0; q < kSortKps / kSortThreads; ++q)
        if (i0 + q * kSortThreads < n) kp[q] = kps[kp0 + i0 + q * kSortThreads];
    if (threadIdx.x < 32) {  // at most 64 images
        const int lane = threadIdx.x;
        const int a = lane < prm.count ? img_tot[lane] : 0;
        const int b = lane + 32 < prm.count ? img_tot[lane + 32] : 0;
        const int before = (lane < img ? a : 0) + (lane + 32 < img ? b : 0);
        const int base = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(before));
        const int total = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(a + b));
        if (lane == 0) {
            s_base = base;
            if (blockIdx.x == 0) counters[0] = total;
        }
    }
    __syncthreads();
    const int base = s_base;
#pragma unroll
    for (int q = 0; q < kSortKps / kSortThreads; ++q) {
        const int i = i0 + q * kSortThreads;
        const int c = i < n ? cell_of(kp[q], prm.nscales, g) : -3;
        if (c >= 0) recs[base + start[c] + rank[kp0 + i]] = kp_record(kp[q], kp0 + i, img);
    }
}

// Tile key of a record: launch-local image, cell row and column (the record's
// keypoint has a cell, so x + kMargin and y + kMargin are >= 0).
__device__ __forceinline__ int tile_key(const int4& r) {
    return ((r.w >> 16) << 22) | (((r.y + kMargin) / kCell) << 11) | ((r.x + kMargin) / kCell);
}

// Window words of every triplet's three patches (top-left word of the 7x7 patch
// in a 48x48 window of 12-word rows) and their byte shifts: x = A | C1 << 16,
// y = C2 | shift A << 16 | shift C1 << 18 | shift C2 << 20.
struct LaneTriplets {
    uint2 e[kBits];
};

// One patch row: the 7 bytes at byte `sh` of word p[0] onwards, as two words whose
// last byte is junk (the third word is read only when the bytes reach into it).
__device__ __forceinline__ void patch_row(const uint32_t* p, uint32_t sh, uint32_t& lo, uint32_t& hi) {
    const uint32_t w0 = p[0], w1 = p[1];
    const uint32_t w2 = sh >= 2 ? p[2] : 0u;
    lo = __funnelshift_r(w0, w1, 8 * sh);
    hi = __funnelshift_r(w1, w2, 8 * sh);
}

// Bit i of the result: Eq. 1 for triplet 8 c + i of the window at `wl` (`trip`:
// the LaneTriplets entries, in shared memory: one broadcast load per triplet).
__device__ __forceinline__ uint32_t eval_chunk(const uint2* trip, const uint32_t* wl, int c) {
    uint32_t byte = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint2 e = trip[8 * c + i];
        const uint32_t* pa = wl + (e.x & 0xffffu);
        const uint32_t* p1 = wl + (e.x >> 16);
        const uint32_t* p2 = wl + (e.y & 0xffffu);
        const uint32_t sa = (e.y >> 16) & 3u, s1 = (e.y >> 18) & 3u, s2 = (e.y >> 20) & 3u;
        uint32_t sa1 = 0, sa2 = 0, s11 = 0, s22 = 0;
#pragma unroll
        for (int rr = 0; rr < 2 * kPatchR + 1; ++rr) {
            uint32_t a0, a1, c0, c1, d0, d1;
            patch_row(pa + rr * kRowWords, sa, a0, a1);
            patch_row(p1 + rr * kRowWords, s1, c0, c1);
            patch_row(p2 + rr * kRowWords, s2, d0, d1);
            c1 &= 0x00ffffffu;  // pixel 8 of the run is not in the patch (A's is multiplied by 0)
            d1 &= 0x00ffffffu;
            sa1 = __dp4a(a0, c0, sa1);
            sa1 = __dp4a(a1, c1, sa1);
            sa2 = __dp4a(a0, d0, sa2);
            sa2 = __dp4a(a1, d1, sa2);
            s11 = __dp4a(c0, c0, s11);
            s11 = __dp4a(c1, c1, s11);
            s22 = __dp4a(d0, d0, s22);
            s22 = __dp4a(d1, d1, s22);
        }
        // D1 - D2 = sum C1^2 - sum C2^2 - 2 (sum A.C1 - sum A.C2)
        const int diff =
            (static_cast<int>(s11) - static_cast<int>(s22)) - 2 * (static_cast<int>(sa1) - static_cast<int>(sa2));
        byte |= (diff > 0 ? 1u : 0u) << i;
    }
    return byte;
}

// Weights of the 8x8 patch pixels (row-major), a kernel parameter: with the pixel
// loops unrolled, every weight is a constant-bank operand of its multiply-add.
struct PatchWeights {
    int32_t w[64];
};

// One 8-pixel patch row: the 8 bytes at byte `sh` of word p[0] onwards, as two words.
__device__ __forceinline__ void patch_row8(const uint32_t* p, uint32_t sh, uint32_t& lo, uint32_t& hi) {
    const uint32_t w0 = p[0], w1 = p[1];
    const uint32_t w2 = sh != 0 ? p[2] : 0u;
    lo = __funnelshift_r(w0, w1, 8 * sh);
    hi = __funnelshift_r(w1, w2, 8 * sh);
}

// Eq. 1 with weighted 8x8 patches (Sec. 3.2, weighing pixels in LATCH patches) for
// triplets 8 c .. 8 c + 7: D1 - D2 = sum w (C1 - C2)(C1 + C2 - 2 A), exact in int32
// (|w (C1 - C2)(C1 + C2 - 2 A)| <= 255 * 255^2 per pixel, 64 pixels).
__device__ __forceinline__ uint32_t eval_chunk_weighted(const uint2* trip, const uint32_t* wl, int c,
                                                        const PatchWeights& pw) {
    uint32_t byte = 0;
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const uint2 e = trip[8 * c + i];
        const uint32_t* pa = wl + (e.x & 0xffffu);
        const uint32_t* p1 = wl + (e.x >> 16);
        const uint32_t* p2 = wl + (e.y & 0xffffu);
        const uint32_t sa = (e.y >> 16) & 3u, s1 = (e.y >> 18) & 3u, s2 = (e.y >> 20) & 3u;
        int acc = 0;
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            uint32_t a[2], c1[2], c2[2];
            patch_row8(pa + rr * kRowWords, sa, a[0], a[1]);
            patch_row8(p1 + rr * kRowWords, s1, c1[0], c1[1]);
            patch_row8(p2 + rr * kRowWords, s2, c2[0], c2[1]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int av = static_cast<int>((a[j >> 2] >> (8 * (j & 3))) & 0xffu);
                const int cv = static_cast<int>((c1[j >> 2] >> (8 * (j & 3))) & 0xffu);
                const int dv = static_cast<int>((c2[j >> 2] >> (8 * (j & 3))) & 0xffu);
                acc += pw.w[rr * 8 + j] * ((cv - dv) * (cv + dv - 2 * av));
            }
        }
        byte |= (acc > 0 ? 1u : 0u) << i;
    }
    return byte;
}

struct LanesSmem {  // static part
    uint2 trip[kBits];                // LaneTriplets
    int4 rec[2][kBatch];              // builders: the batch's records
    int32_t row[2][kBatch];           // output row of each lane's keypoint
    uint64_t tile_bar[2], full[2], empty[2];
    uint32_t runs[2];
    int abort;
};

// Block b takes chunks [b U / G, (b+1) U / G) of the U = 64 * ceil(V / 32) chunks
// of the launch's V records (cell-sorted), batch by batch.  Warps 0-11 build the
// windows of batch i into buffer i % 2 while warps 12-27 evaluate batch i - 1.
template <int NI, bool kWeighted>
__global__ void __launch_bounds__(kThreads, 1) extract_lanes_kernel(
    const __grid_constant__ ExtractParams<NI> prm, const __grid_constant__ LaneTriplets tt,
    const __grid_constant__ PatchWeights pw,
    const int4* __restrict__ recs, const int* __restrict__ counters, const int16_t* __restrict__ toff,
    uint8_t* __restrict__ out, uint8_t* __restrict__ exp_out, uint32_t* __restrict__ flags) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ LanesSmem S;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const TileGeom tg = prm.tg;
    const int tile_bytes = (tg.tw * tg.th + 127) / 128 * 128;
    uint32_t* s_win0 = reinterpret_cast<uint32_t*>(smem);  // [2][32][kLaneWords]
    uint8_t* s_tile0 = smem + 2 * static_cast<size_t>(kBatch) * kLaneWords * 4;  // [2][tile_bytes]
    griddep_wait();
    griddep_launch_dependents();
    const int nrec = counters[0];
    if (nrec <= 0) return;
    const int64_t units = static_cast<int64_t>((nrec + kBatch - 1) / kBatch) * kChunks;
    const int64_t u0 = static_cast<int64_t>(blockIdx.x) * units / gridDim.x;
    const int64_t u1 = static_cast<int64_t>(blockIdx.x + 1) * units / gridDim.x;
    if (u0 >= u1) return;
    const int bfirst = static_cast<int>(u0 / kChunks), blast = static_cast<int>((u1 - 1) / kChunks);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &S.abort;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&S.tile_bar[s], 1);
            mbar_init(&S.full[s], kBuildThreads);
            mbar_init(&S.empty[s], kComputeWarps);
        }
        S.abort = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < kBatch && kBatch * bfirst + lane < nrec) S.rec[0][lane] = recs[kBatch * bfirst + lane];
    for (int t = threadIdx.x; t < kBits; t += kThreads) S.trip[t] = tt.e[t];
    __syncthreads();  // the last block-wide barrier: the two roles meet only at mbarriers from here on

    if (warp < kBuildWarps) {
        // ================= builders (named barrier 1) =================
        const int tb = threadIdx.x;
        auto issue_tile = [&](int slot, int key) {  // thread 0; the slot is free
            const int img = key >> 22;
            const int tx = (key & 2047) * kCell - kMargin + tg.mx;
            const int ty = ((key >> 11) & 2047) * kCell - kMargin + tg.my;
            mbar_arrive_expect_tx(&S.tile_bar[slot], static_cast<uint32_t>(tg.tw * tg.th));
            tma_load_2d(s_tile0 + slot * tile_bytes, &prm.map[img], tx, ty, &S.tile_bar[slot]);
        };
        int g = 0, issued = 1;  // runs started / tiles requested (run r uses slot r % 2)
        if (tb == 0) issue_tile(0, tile_key(S.rec[0][0]));
        bool ok = true;
        for (int bt = bfirst; bt <= blast && ok; ++bt) {
            const int i = bt - bfirst, buf = i & 1;
            const int4* rec = S.rec[buf];
            const int nk = nrec - kBatch * bt < kBatch ? nrec - kBatch * bt : kBatch;
            uint32_t* win = s_win0 + buf * (kBatch * kLaneWords);
            // the next batch's first record (for its first tile) and all its records
            int4 next_first = make_int4(0, 0, 0, 0);
            if (bt < blast) {
                if (tb == 0) next_first = recs[kBatch * (bt + 1)];
                if (warp == kBuildWarps - 1 && kBatch * (bt + 1) + lane < nrec)
                    cp_async_16(&S.rec[buf ^ 1][lane], recs + kBatch * (bt + 1) + lane);
            }
            if (warp == 0) {  // runs of keypoints in one cell
                const int key = lane < nk ? tile_key(rec[lane]) : -1;
                const int prev = __shfl_up_sync(0xffffffffu, key, 1);
                const uint32_t starts = __ballot_sync(0xffffffffu, lane < nk && (lane == 0 || key != prev));
                if (lane == 0) S.runs[buf] = starts;
            }
            // window buffer `buf` is free once the evaluators are done with batch i - 2
            if (i >= 2) ok = mbar_wait(&S.empty[buf], ((i >> 1) - 1) & 1, abort);
            if (ok && tb < nk) S.row[buf][tb] = rec[tb].z;
            ok = bar_and<1, kBuildThreads>(ok);
            if (!ok) break;
            // Each run of keypoints in one cell is built as units of half a window
            // (288 words, 9 per lane) spread over the builder warps: unit u of a run is
            // keypoint j0 + u / 2, half u % 2, and warp w takes units w, w + 12, ..., so
            // the keypoints of a run are gathered in parallel.  A warp loads the
            // offset-table words of its next unit (in this run or a later one of the
            // batch) into B while it gathers the current unit from A.
            constexpr int kHalves = 2;
            constexpr int kUnitWords = kWinWords / kHalves;     // 288
            constexpr int kLaneUnitWords = kUnitWords / 32;     // 9
            // this warp's unit after unit u of run [j0, j1) (later runs: `rest`), as
            // keypoint << 1 | half, or -1
            auto next_unit = [&](int j0, int j1, int u, uint32_t rest) -> int {
                if (u + kBuildWarps < (j1 - j0) * kHalves) {
                    const int v = u + kBuildWarps;
                    return ((j0 + v / kHalves) << 1) | (v % kHalves);
                }
                while (rest) {
                    const int a0 = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const int a1 = rest ? __ffs(rest) - 1 : nk;
                    if (warp < (a1 - a0) * kHalves) return ((a0 + warp / kHalves) << 1) | (warp % kHalves);
                }
                return -1;
            };
            auto load_unit = [&](int code, uint2 (&e)[kLaneUnitWords]) {
                if (code < 0) return;
                const uint2* tab = reinterpret_cast<const uint2*>(toff + static_cast<size_t>(rec[code >> 1].w & 0xffff) * kWinPix) +
                                   (code & 1) * kUnitWords + lane;
#pragma unroll
                for (int q = 0; q < kLaneUnitWords; ++q) e[q] = __ldg(tab + 32 * q);
            };
            uint32_t rem = S.runs[buf];
            uint2 A[kLaneUnitWords], B[kLaneUnitWords];
            load_unit(next_unit(0, 0, -kBuildWarps, rem), A);
            while (rem) {
                const int j0 = __ffs(rem) - 1;
                rem &= rem - 1;
                const int j1 = rem ? __ffs(rem) - 1 : nk;
                const int slot = g & 1;
                const int key = tile_key(rec[j0]);
                // request the following run's tile into the other slot (its last
                // reader, run g - 1, finished at the barrier that ended it)
                if (tb == 0) {
                    const int nkey = rem ? tile_key(rec[__ffs(rem) - 1]) : bt < blast ? tile_key(next_first) : -1;
                    if (nkey >= 0) {
                        issue_tile(slot ^ 1, nkey);
                        ++issued;
                    }
                }
                const bool tok = mbar_wait(&S.tile_bar[slot], (g >> 1) & 1, abort);
                if (tok) {
                    const uint8_t* tile = s_tile0 + slot * tile_bytes;
                    const int ox = (key & 2047) * kCell - kMargin + tg.mx;
                    const int oy = ((key >> 11) & 2047) * kCell - kMargin + tg.my;
                    for (int u = warp; u < (j1 - j0) * kHalves; u += kBuildWarps) {
                        load_unit(next_unit(j0, j1, u, rem), B);  // lands during this unit's gathers
                        const int j = j0 + u / kHalves, half = u % kHalves;
                        const int4 r = rec[j];
                        const uint8_t* t = tile + (r.y - oy) * tg.tw + (r.x - ox);
                        uint32_t* w = win + j * kLaneWords + half * kUnitWords + lane;
#pragma unroll
                        for (int q = 0; q < kLaneUnitWords; ++q) {
                            const uint32_t b0 = t[static_cast<int16_t>(A[q].x & 0xffffu)];
                            const uint32_t b1 = t[static_cast<int16_t>(A[q].x >> 16)];
                            const uint32_t b2 = t[static_cast<int16_t>(A[q].y & 0xffffu)];
                            const uint32_t b3 = t[static_cast<int16_t>(A[q].y >> 16)];
                            w[32 * q] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
                        }
#pragma unroll
                        for (int q = 0; q < kLaneUnitWords; ++q) A[q] = B[q];
                    }
                }
                if (j1 == nk && warp == kBuildWarps - 1) cp_async_wait_all();
                ok = bar_and<1, kBuildThreads>(tok);  // the run's tile slot is free after it
                if (!ok) break;
                ++g;
            }
            // batch i's windows are complete (the barrier above ordered all builders' stores)
            if (ok) mbar_arrive(&S.full[buf]);
        }
        if (!ok) {  // let the copies in flight land before the block's memory is released
            if (tb == 0) {
                atomicOr(flags, kFlagTimeout);
                const uint64_t t0 = globaltimer();
                for (int r = g; r < issued; ++r)
                    while (!mbar_try_wait(&S.tile_bar[r & 1], (r >> 1) & 1) && globaltimer() - t0 < 200000000ull) {
                    }
            }
            if (warp == kBuildWarps - 1) cp_async_wait_all();
        }
        return;
    }

    // ================= evaluators (named barrier 2) =================
    const int cw = warp - kBuildWarps;
    const int ct = cw * 32 + lane;  // 0 .. kComputeThreads - 1
    for (int bt = bfirst; bt <= blast; ++bt) {
        const int i = bt - bfirst, buf = i & 1;
        const int nk = nrec - kBatch * bt < kBatch ? nrec - kBatch * bt : kBatch;
        const int64_t bu = static_cast<int64_t>(bt) * kChunks;  // the batch's first chunk
        const int ca = static_cast<int>((u0 > bu ? u0 : bu) - bu);
        const int cb = static_cast<int>((u1 < bu + kChunks ? u1 : bu + kChunks) - bu);
        // the evaluator warps agree on the outcome of the wait, so that all of them
        // reach the barriers below or none does
        const bool got = mbar_wait(&S.full[buf], (i >> 1) & 1, abort);
        if (!bar_and<2, kComputeThreads>(got)) {
            if (!got && lane == 0) atomicOr(flags, kFlagTimeout);
            return;
        }
        // ---- Eq. 1: this warp's chunks [wa, wb), lane = keypoint ----
        const int n = cb - ca;
        const int wa = ca + cw * n / kComputeWarps, wb = ca + (cw + 1) * n / kComputeWarps;
        uint32_t* wbuf = s_win0 + buf * (kBatch * kLaneWords);
        const uint32_t* wl = wbuf + lane * kLaneWords;
        uint32_t v = 0;  // byte c - wa: chunk c
#pragma unroll 1
        for (int c = wa; c < wb; ++c) {
            if constexpr (kWeighted)
                v |= eval_chunk_weighted(S.trip, wl, c, pw) << (8 * (c - wa));
            else
                v |= eval_chunk(S.trip, wl, c) << (8 * (c - wa));
        }
        if (n == kChunks) {
            // ---- the whole batch is this block's: warp cw holds bytes [4 cw, 4 cw + 4)
            // of every lane's descriptor.  Once every warp is done with the windows,
            // the words are staged in the buffer's head (transposed: word cw of lane r at
            // [cw][r]) and whole rows leave as 16-byte stores: 4 threads per 64-byte
            // descriptor, 16 per 256-byte expanded row ----
            bar_sync<2, kComputeThreads>();
            wbuf[cw * kBatch + lane] = v;
            bar_sync<2, kComputeThreads>();
            if (ct < 4 * nk) {
                const int r = ct >> 2, q = ct & 3;
                const uint4 d = make_uint4(wbuf[(4 * q) * kBatch + r], wbuf[(4 * q + 1) * kBatch + r],
                                           wbuf[(4 * q + 2) * kBatch + r], wbuf[(4 * q + 3) * kBatch + r]);
                reinterpret_cast<uint4*>(out + static_cast<size_t>(S.row[buf][r]) * kDescBytes)[q] = d;
            }
            if (exp_out && ct < 16 * nk) {
                const int r = ct >> 4, w = ct & 15;
                reinterpret_cast<uint4*>(exp_out + static_cast<size_t>(S.row[buf][r]) * kExpRowBytes)[w] =
                    expand_word_e2m1(wbuf[w * kBatch + r]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[buf]);  // the windows and rows are free again
            continue;
        }
        // ---- a batch shared with the neighbouring block: this block's bytes [ca, cb)
        // only, descriptor bytes [wa, wb) and expanded bytes [8 wa, 8 wb) per warp ----
        const int32_t row = S.row[buf][lane];
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[buf]);  // the windows and rows are free again
        if (wb == wa || lane >= nk) continue;
        uint8_t* d = out + static_cast<size_t>(row) * kDescBytes;
        for (int c = wa; c < wb; ++c) {
            const uint32_t byte = (v >> (8 * (c - wa))) & 0xffu;
            d[c] = static_cast<uint8_t>(byte);
            if (exp_out)
                reinterpret_cast<uint32_t*>(exp_out + static_cast<size_t>(row) * kExpRowBytes)[c] =
                    expand_byte_e2m1(byte);
        }
    }
}

}  // namespace

// Host-side precomputation for the extraction kernel ------------------------------

static TileGeom tile_geom(int reach) {
    TileGeom t;
    const int rx = (reach + 15) / 16 * 16;  // x margin rounded to the 16-byte TMA granule
    t.tw = kCell + 2 * rx;
    // an odd number of 16-byte granules per row: rows then start in 8 different bank
    // groups (an even number gives 2 or 4), so the gathers along a rotated window
    // row collide less
    if ((t.tw / 16) % 2 == 0) t.tw += 16;
    t.th = kCell + 2 * reach;
    t.mx = -rx;
    t.my = -reach;
    return t;
}

int extract_tile_pitch(int reach) { return tile_geom(reach).tw; }

// Per triplet: the window word holding the first pixel of each patch's top row and
// the pixel's byte in it (LaneTriplets layout).
void build_triplet_offsets(const latch_triplet* trip, uint32_t* out /* 2 per triplet */) {
    for (int t = 0; t < kBits; ++t) {
        const uint8_t* c = &trip[t].ax;
        uint32_t word[3], shift[3];
        for (int p = 0; p < 3; ++p) {
            const int x0 = c[2 * p] - kPatchR, y0 = c[2 * p + 1] - kPatchR;
            word[p] = static_cast<uint32_t>(y0 * kRowWords + (x0 >> 2));
            shift[p] = static_cast<uint32_t>(x0 & 3);
        }
        out[2 * t] = word[0] | (word[1] << 16);
        out[2 * t + 1] = word[2] | (shift[0] << 16) | (shift[1] << 18) | (shift[2] << 20);
    }
}

static CellGrid cell_grid(const latch_image* img) {
    CellGrid g;
    g.width = img->width;
    g.height = img->height;
    g.gx = (img->width + 2 * kMargin + kCell - 1) / kCell;
    g.gy = (img->height + 2 * kMargin + kCell - 1) / kCell;
    return g;
}

// Two buffers of 32 windows, then two tiles (128 bytes of alignment slack).  At the
// largest reach 221 KB (+5 KB static): one block per SM.
static size_t extract_smem_bytes(const TileGeom& tg) {
    return 128 + 2 * static_cast<size_t>(kBatch) * kLaneWords * 4 + 2 * ((static_cast<size_t>(tg.tw) * tg.th + 127) / 128 * 128);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn extract_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Scratch of one launch over images [i0, i1): sorted keypoint records, ranks, then
// the region the host zeroes: counters, image totals, image arrival counters, cell
// counts.
struct ChunkLayout {
    size_t recs, rank, zero, counters, img_tot, img_done, cells, total;
    int64_t ncell, nkp;
};

static ChunkLayout chunk_layout(const latch_image* imgs, const int64_t* n, int i0, int i1) {
    ChunkLayout l;
    l.ncell = 0;
    l.nkp = 0;
    for (int i = i0; i < i1; ++i) {
        const CellGrid g = cell_grid(&imgs[i]);
        l.ncell += static_cast<int64_t>(g.gx) * g.gy;
        l.nkp += n[i];
    }
    l.recs = 0;  // int4, 16-byte aligned
    l.rank = l.recs + static_cast<size_t>(l.nkp) * sizeof(int4);
    l.zero = (l.rank + static_cast<size_t>(l.nkp) * sizeof(int) + 255) / 256 * 256;
    l.counters = l.zero;
    l.img_tot = l.counters + 16;
    l.img_done = l.img_tot + 64 * sizeof(int);
    l.cells = l.img_done + 64 * sizeof(int);
    l.total = (l.cells + static_cast<size_t>(l.ncell) * sizeof(int) + 255) / 256 * 256;
    return l;
}

static constexpr int kBatchImages = 64;  // images per launch in the batched form

size_t extract_batch_scratch_bytes(const latch_image* imgs, const int64_t* n, int count) {
    size_t total = 0;
    for (int i0 = 0; i0 < count; i0 += kBatchImages) {
        const int i1 = i0 + kBatchImages < count ? i0 + kBatchImages : count;
        total += chunk_layout(imgs, n, i0, i1).total;
    }
    return total;
}

size_t extract_scratch_bytes(const latch_image* img, int64_t n) { return extract_batch_scratch_bytes(img, &n, 1); }

template <int NI, bool kWeighted>
static cudaError_t set_extract_attributes() {
    cudaError_t e = cudaFuncSetAttribute(extract_lanes_kernel<NI, kWeighted>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(extract_smem_bytes(tile_geom(kMaxReach + 1))));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(extract_lanes_kernel<NI, kWeighted>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
    return e;
}

template <int NI>
static cudaError_t launch_chunk(const latch_context* ctx, const latch_image* imgs, const int64_t* kp0,
                                const int64_t* n, int i0, int i1, const latch_keypoint* d_kps, uint8_t* d_out,
                                uint8_t* exp_out, uint8_t* scratch, cudaStream_t stream,
                                uint32_t* flags, const int32_t* n_dev) {
    static unsigned long long attr_done[2] = {0, 0};
    const TileGeom tg = tile_geom(ctx->reach);
    cudaError_t e = ctx->weighted ? once_per_device(&attr_done[1], set_extract_attributes<NI, true>)
                                  : once_per_device(&attr_done[0], set_extract_attributes<NI, false>);
    if (e != cudaSuccess) return e;
    EncodeTiledFn enc = extract_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const ChunkLayout l = chunk_layout(imgs, n, i0, i1);
    int4* recs = reinterpret_cast<int4*>(scratch + l.recs);
    int* rank = reinterpret_cast<int*>(scratch + l.rank);
    int* counters = reinterpret_cast<int*>(scratch + l.counters);
    int* img_tot = reinterpret_cast<int*>(scratch + l.img_tot);
    int* img_done = reinterpret_cast<int*>(scratch + l.img_done);
    int* cells = reinterpret_cast<int*>(scratch + l.cells);

    ExtractParams<NI>* prm = new ExtractParams<NI>;
    prm->count = i1 - i0;
    prm->nscales = ctx->nscales;
    prm->tg = tg;
    prm->n_dev = n_dev;
    int64_t cell0 = 0;
    int blocks = 0;
    for (int i = i0; i < i1; ++i) {
        const int j = i - i0;
        const CellGrid g = cell_grid(&imgs[i]);
        prm->grid[j] = g;
        prm->kp0[j] = static_cast<int32_t>(kp0[i]);
        prm->n[j] = static_cast<int32_t>(n[i]);
        prm->cell0[j] = static_cast<int32_t>(cell0);
        prm->blk0[j] = blocks;
        cell0 += static_cast<int64_t>(g.gx) * g.gy;
        blocks += static_cast<int>((n[i] + kSortKps - 1) / kSortKps);
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(imgs[i].width), static_cast<cuuint64_t>(imgs[i].height)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(imgs[i].pitch)};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(tg.tw), static_cast<cuuint32_t>(tg.th)};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&prm->map[j], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(imgs[i].data), dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            delete prm;
            return cudaErrorInvalidValue;
        }
    }
    e = cudaMemsetAsync(scratch + l.zero, 0, l.total - l.zero, stream);
    if (e == cudaSuccess)
        e = launch_chained(sort_count_kernel<NI>, dim3(blocks), dim3(kSortThreads), 0, stream, *prm, d_kps, cells,
                           rank, img_tot, img_done, reinterpret_cast<uint4*>(d_out),
                           reinterpret_cast<uint4*>(exp_out), flags);
    if (e == cudaSuccess)
        e = launch_chained(sort_scatter_kernel<NI>, dim3(blocks), dim3(kSortThreads), 0, stream, *prm, d_kps,
                           static_cast<const int*>(cells), static_cast<const int*>(rank),
                           static_cast<const int*>(img_tot), counters, recs);
    LaneTriplets* tt = e == cudaSuccess ? new LaneTriplets : nullptr;
    if (tt) {
        static_assert(sizeof(LaneTriplets) == sizeof(ctx->h_trip_offsets), "triplet table layout");
        memcpy(tt, ctx->h_trip_offsets, sizeof(LaneTriplets));
        // the chunks are split evenly over the blocks, at least item_kps keypoints' worth each
        const int64_t want = (l.nkp + ctx->item_kps - 1) / ctx->item_kps;
        const int64_t grid = want < ctx->sm_count ? want : ctx->sm_count;
        PatchWeights pw;
        for (int i = 0; i < 64; ++i) pw.w[i] = ctx->patch_weights[i];
        e = launch_chained(ctx->weighted ? extract_lanes_kernel<NI, true> : extract_lanes_kernel<NI, false>,
                           dim3(static_cast<unsigned>(grid)), dim3(kThreads), extract_smem_bytes(tg), stream, *prm, *tt,
                           pw, static_cast<const int4*>(recs), static_cast<const int*>(counters), ctx->d_tile_offsets,
                           d_out, exp_out, flags);
        delete tt;
    }
    delete prm;
    return e;
}

cudaError_t launch_extract_batch(const latch_context* ctx, const latch_image* imgs, const int64_t* kp0,
                                 const int64_t* n, int count, const latch_keypoint* d_kps, uint8_t* d_out,
                                 void* scratch, cudaStream_t stream, uint8_t* exp_out, uint32_t* flags) {
    uint8_t* base = static_cast<uint8_t*>(scratch);
    if (!flags) flags = ctx->d_flags;
    for (int i0 = 0; i0 < count; i0 += kBatchImages) {
        const int i1 = i0 + kBatchImages < count ? i0 + kBatchImages : count;
        int64_t nk = 0;
        for (int i = i0; i < i1; ++i) nk += n[i];
        if (nk > 0) {
            // the kernel parameters hold one tensor map per image: the smallest
            // instance that fits keeps the launch's parameter block small
            const int ni = i1 - i0;
            const cudaError_t e =
                ni == 1    ? launch_chunk<1>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, base, stream, flags, nullptr)
                : ni <= 4  ? launch_chunk<4>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, base, stream, flags, nullptr)
                : ni <= 16 ? launch_chunk<16>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, base, stream, flags, nullptr)
                           : launch_chunk<kBatchImages>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, base,
                                                        stream, flags, nullptr);
            if (e != cudaSuccess) return e;
        }
        base += chunk_layout(imgs, n, i0, i1).total;
    }
    return cudaSuccess;
}

cudaError_t launch_extract(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps, int32_t n,
                           uint8_t* d_out, void* scratch, cudaStream_t stream) {
    const int64_t kp0 = 0, nn = n;
    return launch_extract_batch(ctx, img, &kp0, &nn, 1, d_kps, d_out, scratch, stream, nullptr);
}

cudaError_t launch_extract_dev_count(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps,
                                     int32_t max_n, const int32_t* d_n, uint8_t* d_out, void* scratch,
                                     cudaStream_t stream) {
    if (max_n <= 0) return cudaSuccess;
    const int64_t kp0 = 0, nn = max_n;
    return launch_chunk<1>(ctx, img, &kp0, &nn, 0, 1, d_kps, d_out, nullptr, static_cast<uint8_t*>(scratch),
                           stream, ctx->d_flags, d_n);
}

}  // namespace latch

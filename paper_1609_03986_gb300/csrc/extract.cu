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
// 2. extract_cells_kernel (8 warps per block, four blocks per SM): block b takes
//    the b-th of G equal shares of the records.  The image tile under a cell plus a
//    `reach` halo is staged into shared memory by one TMA 2-D load (samples outside
//    the image arrive as 0, the border reading) whenever the next keypoint lies in
//    another cell.  For each keypoint in turn, the block
//      - samples the 48x48 window through the per-(scale, bin) offset table
//        (nearest pixel; offsets pre-multiplied into tile offsets) and stores it
//        as 4 byte-shifted copies, so that the 8 bytes holding any 7-pixel patch
//        row are two aligned 32-bit words;
//      - evaluates Eq. 1 for 32 triplets per warp at a time, one triplet per lane:
//        D1 - D2 = (sum C1^2 - sum C2^2) - 2 (sum A.C1 - sum A.C2) over the 7 rows,
//        with __dp4a on 4 pixels at a time, all exact in 32-bit integers;
//      - packs the 32 bits of each warp-group with __ballot_sync (bit t = bit
//        t % 32 of word t / 32, i.e. bit t % 8 of byte t / 8) and writes the
//        64-byte descriptor as four 128-bit stores (the last warp, which builds no
//        window, does this); when the caller also wants the tensor matcher's
//        input, it writes the expanded row (byte t = E4M3 1.0 or 0 for bit t) and
//        the descriptor's popcount as well, so no separate pass over the
//        descriptors is needed.
//    Windows are double-buffered so one __syncthreads per keypoint suffices.
#include <cuda.h>

#include <cmath>
#include <cstdint>

#include "internal.h"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kCell = 32;
constexpr int kMargin = 128;            // cell grid reaches this far beyond each border
constexpr int kThreads = 256;           // 8 warps
constexpr int kRowWords = 12;           // 48 bytes per window row
constexpr int kCopyWords = kWin * kRowWords + 4;   // one byte-shifted copy (+4: bank offset; 16-byte multiple)
constexpr int kWinWords = 4 * kCopyWords;          // 4 copies
constexpr int kSortThreads = 256;
constexpr int kSortKps = 1024;          // keypoints per sorting block (4 per thread)
constexpr int kRing = 64;               // keypoint records in flight per block (1 KB: four blocks still fit an SM)

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
};

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
    uint4* __restrict__ exp_out, int32_t* __restrict__ pop_out, uint32_t* __restrict__ flags) {
    __shared__ int s_part[kSortThreads / 32];
    __shared__ int s_flag;
    griddep_wait();
    griddep_launch_dependents();
    const int img = image_of_block(prm, blockIdx.x);
    const CellGrid g = prm.grid[img];
    const int n = prm.n[img], kp0 = prm.kp0[img];
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
            if (exp_out) {
                uint4* x = exp_out + static_cast<size_t>(kp0 + i) * 32;
                for (int u = 0; u < 32; ++u) x[u] = z;
                pop_out[kp0 + i] = 0;
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
        const int nblk = (n + kSortKps - 1) / kSortKps;
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
    const int n = prm.n[img], kp0 = prm.kp0[img];
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

// Offset-table entries 16*bseg .. 16*bseg+19 of window row `by` of table `tab`
// (scale * 32 + bin): two 16-byte and one 8-byte load.
__device__ __forceinline__ void load_table_segment(const int16_t* __restrict__ toff, int tab, int by, int bseg,
                                                   int32_t (&tw)[10]) {
    const int16_t* t = toff + static_cast<size_t>(tab) * kWinPix + by * kWin + 16 * bseg;
    const int4 ta = reinterpret_cast<const int4*>(t)[0];
    const int4 tb = reinterpret_cast<const int4*>(t)[1];
    const int2 tc = reinterpret_cast<const int2*>(t)[4];
    tw[0] = ta.x; tw[1] = ta.y; tw[2] = ta.z; tw[3] = ta.w;
    tw[4] = tb.x; tw[5] = tb.y; tw[6] = tb.z; tw[7] = tb.w;
    tw[8] = tc.x; tw[9] = tc.y;
}

// Tile key of a record: launch-local image, cell row and column (the record's
// keypoint has a cell, so x + kMargin and y + kMargin are >= 0).
__device__ __forceinline__ int tile_key(const int4& r) {
    return ((r.w >> 16) << 22) | (((r.y + kMargin) / kCell) << 11) | ((r.x + kMargin) / kCell);
}

// Block b extracts the records [b V / G, (b+1) V / G) of the launch's V records
// (cell-sorted), one keypoint per step.  Records reach shared memory through a
// ring filled 32 keypoints ahead by asynchronous copies; the tile under the next
// keypoint's cell is requested, when the cell changes, right after the barrier of
// the last keypoint that reads the current tile, so it lands during that
// keypoint's triplets.
template <int NI>
__global__ void __launch_bounds__(kThreads, 4) extract_cells_kernel(
    const __grid_constant__ ExtractParams<NI> prm, const int4* __restrict__ recs, const int* __restrict__ counters,
    const int16_t* __restrict__ toff, const uint2* __restrict__ trip_off, uint4* __restrict__ out,
    uint4* __restrict__ exp_out, int32_t* __restrict__ pop_out, uint32_t* __restrict__ flags) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ int4 s_rec[kRing];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint32_t* s_win = reinterpret_cast<uint32_t*>(smem);                  // [2][kWinWords]
    uint8_t* s_bits = reinterpret_cast<uint8_t*>(s_win + 2 * kWinWords);  // [2][512] one byte per bit
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_bits + 2 * kBits);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_bar + 1);
    uint8_t* s_tile = reinterpret_cast<uint8_t*>(s_bar + 2);
    s_tile = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_tile) + 127) & ~uintptr_t(127));
    const TileGeom tg = prm.tg;
    griddep_wait();
    griddep_launch_dependents();
    const int nrec = counters[0];
    const int j0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * nrec / gridDim.x);
    const int m = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * nrec / gridDim.x) - j0;
    if (m <= 0) return;
    const int4* brec = recs + j0;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kLastWarp = kThreads / 32 - 1;
    if (threadIdx.x == 0) {
        mbar_init(s_bar, 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    for (int t = threadIdx.x; t < m && t < kRing - 32; t += kThreads) s_rec[t] = brec[t];
    // this thread's window-build job (threads 0..143): row by, 16-pixel segment bseg
    const int by = threadIdx.x / 3, bseg = threadIdx.x % 3;
    // this lane's two triplets (slots 64*warp + lane and +32 of the bank-conflict
    // minimising order): patch word offsets and the triplet's bit position
    const uint2 to0 = trip_off[64 * warp + lane];
    const uint2 to1 = trip_off[64 * warp + 32 + lane];
    __syncthreads();

    int cur_key = -1, ox = 0, oy = 0;
    uint32_t tile_par = 0;
    auto issue_tile = [&](const int4& r) {  // thread 0
        const int key = tile_key(r);
        const int img = key >> 22;
        const int tx = (key & 2047) * kCell - kMargin + tg.mx, ty = ((key >> 11) & 2047) * kCell - kMargin + tg.my;
        mbar_arrive_expect_tx(s_bar, static_cast<uint32_t>(tg.tw * tg.th));
        tma_load_2d(s_tile, &prm.map[img], tx, ty, s_bar);
    };
    if (threadIdx.x == 0) issue_tile(s_rec[0]);

    // offset-table entries 0..19 of this thread's row segment for the first keypoint
    // (32-byte aligned: 96*by + 32*bseg bytes); later ones are prefetched one keypoint
    // ahead, during the previous keypoint's triplets, into the other register set
    // (the two sets swap roles every keypoint)
    int32_t ta[10], tb[10];
    if (threadIdx.x < 144) load_table_segment(toff, s_rec[0].w & 0xffff, by, bseg, ta);

    // One step: build the window of keypoint k from `tw` (prefetching k+1's entries
    // into `tn`), then, after the barrier, pack keypoint k-1 and evaluate keypoint k's
    // triplets.  Returns true after the last step.
    auto step = [&](int k, int32_t (&tw)[10], int32_t (&tn)[10]) -> bool {
        const int buf = k & 1;
        bool ok = true;
        if (k < m) {
            const int4 r = s_rec[k % kRing];
            const int key = tile_key(r);
            if (key != cur_key) {  // block-uniform: a new tile was requested for this keypoint
                if (threadIdx.x < 144) ok = mbar_wait(s_bar, tile_par, s_abort);
                tile_par ^= 1;
                cur_key = key;
                ox = (key & 2047) * kCell - kMargin + tg.mx;
                oy = ((key >> 11) & 2047) * kCell - kMargin + tg.my;
            }
            if (threadIdx.x < 144 && ok) {
                // ---- sample the window of keypoint k into 4 byte-shifted copies; this
                // thread: row by, pixels 16*bseg .. 16*bseg+18 ----
                const int base = (r.y - oy) * tg.tw + (r.x - ox);
                uint32_t p[5] = {0, 0, 0, 0, 0};
#pragma unroll
                for (int u = 0; u < 19; ++u) {
                    if (16 * bseg + u < kWin) {
                        const int16_t o = static_cast<int16_t>((tw[u >> 1] >> (16 * (u & 1))) & 0xffff);
                        p[u >> 2] |= static_cast<uint32_t>(s_tile[base + o]) << (8 * (u & 3));
                    }
                }
                uint4* w = reinterpret_cast<uint4*>(s_win + buf * kWinWords + by * kRowWords + 4 * bseg);
                w[0] = make_uint4(p[0], p[1], p[2], p[3]);
                w[kCopyWords / 4] = make_uint4(__funnelshift_r(p[0], p[1], 8), __funnelshift_r(p[1], p[2], 8),
                                               __funnelshift_r(p[2], p[3], 8), __funnelshift_r(p[3], p[4], 8));
                w[2 * kCopyWords / 4] =
                    make_uint4(__funnelshift_r(p[0], p[1], 16), __funnelshift_r(p[1], p[2], 16),
                               __funnelshift_r(p[2], p[3], 16), __funnelshift_r(p[3], p[4], 16));
                w[3 * kCopyWords / 4] =
                    make_uint4(__funnelshift_r(p[0], p[1], 24), __funnelshift_r(p[1], p[2], 24),
                               __funnelshift_r(p[2], p[3], 24), __funnelshift_r(p[3], p[4], 24));
                if (k + 1 < m) load_table_segment(toff, s_rec[(k + 1) % kRing].w & 0xffff, by, bseg, tn);
            }
        }
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicOr(flags, kFlagTimeout);
                const uint64_t t0 = globaltimer();  // let the copy land before the block exits
                while (!mbar_try_wait(s_bar, tile_par ^ 1) && globaltimer() - t0 < 200000000ull) {
                }
            }
            if (warp == kLastWarp) cp_async_wait_all();
            return true;
        }
        // the tile is free once keypoint k's window is built: request the next cell's
        if (threadIdx.x == 0 && k + 1 < m && tile_key(s_rec[(k + 1) % kRing]) != cur_key)
            issue_tile(s_rec[(k + 1) % kRing]);
        if (warp == kLastWarp) {
            if (k > 0) {
                // ---- pack and store the descriptor of keypoint k-1 (all its bits were
                // written before the barrier above; this warp builds no window): word w
                // collects bits 32w..32w+31 ----
                const uint8_t* b = s_bits + ((k - 1) & 1) * kBits;
                uint32_t mine = 0;  // lane w < 16 keeps word w
#pragma unroll
                for (int w = 0; w < kDescWords; ++w) {
                    const uint32_t word = __ballot_sync(0xffffffffu, b[32 * w + lane] != 0);
                    if (lane == w) mine = word;
                }
                const int src = (4 * lane) & 31;
                const uint32_t x = __shfl_sync(0xffffffffu, mine, src);
                const uint32_t y = __shfl_sync(0xffffffffu, mine, src + 1);
                const uint32_t z = __shfl_sync(0xffffffffu, mine, src + 2);
                const uint32_t v = __shfl_sync(0xffffffffu, mine, src + 3);
                const size_t row = static_cast<size_t>(s_rec[(k - 1) % kRing].z);
                if (lane < 4) out[row * 4 + lane] = make_uint4(x, y, z, v);
                if (exp_out) {
                    // bytes 16*lane .. 16*lane+15 are 0 or 1: times 0x38 gives E4M3 0 / 1.0
                    const uint4 e = reinterpret_cast<const uint4*>(b)[lane];
                    exp_out[row * 32 + lane] = make_uint4(e.x * 0x38u, e.y * 0x38u, e.z * 0x38u, e.w * 0x38u);
                    const int pc = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(__popc(mine)));
                    if (lane == 0) pop_out[row] = pc;
                }
            }
            // ---- record ring: at steps k = 32i the records k+32 .. k+63 are requested
            // (their slots held k-32 .. k-1, all consumed, the last by the pack above);
            // at step k+16 this warp waits for them, so the barrier of step k+17
            // publishes them before step k+31 first reads one
            if ((k & 31) == 0) {
                const int t = k + kRing - 32 + lane;
                if (t < m) cp_async_16(&s_rec[t % kRing], brec + t);
            } else if ((k & 31) == 16) {
                cp_async_wait_all();
            }
        }
        if (k == m) {
            if (warp == kLastWarp) cp_async_wait_all();
            return true;
        }
        // ---- Eq. 1 for this lane's two triplets ----
        const uint32_t* wb = s_win + buf * kWinWords;
        uint8_t* bits = s_bits + buf * kBits;
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
            const uint2 to = gi == 0 ? to0 : to1;
            const uint32_t* pa = wb + (to.x & 0xffffu);
            const uint32_t* p1 = wb + (to.x >> 16);
            const uint32_t* p2 = wb + (to.y & 0xffffu);
            uint32_t sa1 = 0, sa2 = 0, s11 = 0, s22 = 0;
#pragma unroll
            for (int i = 0; i < 2 * kPatchR + 1; ++i) {
                const uint32_t a0 = pa[i * kRowWords], a1 = pa[i * kRowWords + 1];
                const uint32_t c0 = p1[i * kRowWords], c1 = p1[i * kRowWords + 1] & 0x00ffffffu;
                const uint32_t e0 = p2[i * kRowWords], e1 = p2[i * kRowWords + 1] & 0x00ffffffu;
                sa1 = __dp4a(a0, c0, sa1);
                sa1 = __dp4a(a1, c1, sa1);
                sa2 = __dp4a(a0, e0, sa2);
                sa2 = __dp4a(a1, e1, sa2);
                s11 = __dp4a(c0, c0, s11);
                s11 = __dp4a(c1, c1, s11);
                s22 = __dp4a(e0, e0, s22);
                s22 = __dp4a(e1, e1, s22);
            }
            // D1 - D2 = sum C1^2 - sum C2^2 - 2 (sum A.C1 - sum A.C2)
            const int diff = (static_cast<int>(s11) - static_cast<int>(s22)) -
                             2 * (static_cast<int>(sa1) - static_cast<int>(sa2));
            bits[to.y >> 16] = diff > 0 ? 1 : 0;
        }
        return false;
    };
    for (int k = 0;; k += 2) {
        if (step(k, ta, tb)) break;
        if (step(k + 1, tb, ta)) break;
    }
}

}  // namespace

// Host-side precomputation for the cell kernel ------------------------------------

static TileGeom tile_geom(int reach) {
    TileGeom t;
    const int rx = (reach + 15) / 16 * 16;  // x margin rounded to the 16-byte TMA granule
    t.tw = kCell + 2 * rx;
    t.th = kCell + 2 * reach;
    t.mx = -rx;
    t.my = -reach;
    return t;
}

int extract_tile_pitch(int reach) { return tile_geom(reach).tw; }

// Word offset of the top-left 8-byte run of the patch centred at (cx, cy) in the
// 4-copy window layout.
static uint32_t patch_word(int cx, int cy) {
    const int x0 = cx - kPatchR, y0 = cy - kPatchR;
    return static_cast<uint32_t>((x0 & 3) * kCopyWords + y0 * kRowWords + (x0 >> 2));
}

// Order in which the lanes evaluate the triplets.  32 lanes of a warp read the
// same row of their patches with one shared-memory instruction; lanes whose words
// fall in the same bank serialise.  A short deterministic annealing over swaps
// between the 16 groups of 32 minimises the sum over groups and patch roles of the
// squared bank occupancies.  Bits go back to their triplet positions through
// shared memory, so the descriptor does not depend on the order.
static void plan_triplet_order(const latch_triplet* trip, int* order) {
    int bank[kBits][3];
    for (int t = 0; t < kBits; ++t) {
        const uint8_t* c = &trip[t].ax;
        for (int p = 0; p < 3; ++p) bank[t][p] = static_cast<int>(patch_word(c[2 * p], c[2 * p + 1]) & 31);
    }
    constexpr int kGroups = kBits / 32;
    int cnt[kGroups][3][32] = {};
    for (int i = 0; i < kBits; ++i) {
        order[i] = i;
        for (int p = 0; p < 3; ++p) ++cnt[i / 32][p][bank[i][p]];
    }
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto next = [&st]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return st;
    };
    const int iters = 400000;
    for (int it = 0; it < iters; ++it) {
        const int s1 = static_cast<int>(next() % kBits), s2 = static_cast<int>(next() % kBits);
        const int g1 = s1 / 32, g2 = s2 / 32;
        if (g1 == g2) continue;
        const int t1 = order[s1], t2 = order[s2];
        // change of sum(count^2) when t1 moves g1 -> g2 and t2 moves g2 -> g1
        int delta = 0;
        for (int p = 0; p < 3; ++p) {
            const int b1 = bank[t1][p], b2 = bank[t2][p];
            if (b1 == b2) continue;
            delta += 2 * (cnt[g1][p][b2] - cnt[g1][p][b1] + 1);  // g1 loses b1, gains b2
            delta += 2 * (cnt[g2][p][b1] - cnt[g2][p][b2] + 1);  // g2 loses b2, gains b1
        }
        const double temp = 3.0 * (1.0 - static_cast<double>(it) / iters) + 1e-3;
        const double u = static_cast<double>(next() >> 11) * 0x1.0p-53;
        if (delta <= 0 || u < std::exp(-delta / temp)) {
            for (int p = 0; p < 3; ++p) {
                --cnt[g1][p][bank[t1][p]];
                ++cnt[g1][p][bank[t2][p]];
                --cnt[g2][p][bank[t2][p]];
                ++cnt[g2][p][bank[t1][p]];
            }
            order[s1] = t2;
            order[s2] = t1;
        }
    }
}

// Per lane slot: the three patches' word offsets and the triplet's bit position.
void build_triplet_offsets(const latch_triplet* trip, uint32_t* out /* 2 per triplet */) {
    int order[kBits];
    plan_triplet_order(trip, order);
    for (int slot = 0; slot < kBits; ++slot) {
        const int t = order[slot];
        const uint8_t* c = &trip[t].ax;
        out[2 * slot] = patch_word(c[0], c[1]) | (patch_word(c[2], c[3]) << 16);
        out[2 * slot + 1] = patch_word(c[4], c[5]) | (static_cast<uint32_t>(t) << 16);
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

static size_t extract_smem_bytes(const TileGeom& tg) {
    return 128 + static_cast<size_t>(2 * kWinWords) * 4 + 2 * kBits + 16 + 128 + static_cast<size_t>(tg.tw) * tg.th;
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

template <int NI>
static cudaError_t launch_chunk(const latch_context* ctx, const latch_image* imgs, const int64_t* kp0,
                                const int64_t* n, int i0, int i1, const latch_keypoint* d_kps, uint8_t* d_out,
                                uint8_t* exp_out, int32_t* pop_out, uint8_t* scratch, cudaStream_t stream) {
    static bool attr = false;
    const TileGeom tg = tile_geom(ctx->reach);
    cudaError_t e;
    if (!attr) {
        e = cudaFuncSetAttribute(extract_cells_kernel<NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(extract_smem_bytes(tile_geom(kMaxReach + 1))));
        if (e == cudaSuccess)  // four 57 KB blocks per SM
            e = cudaFuncSetAttribute(extract_cells_kernel<NI>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        attr = true;
    }
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
                           reinterpret_cast<uint4*>(exp_out), pop_out, ctx->d_flags);
    if (e == cudaSuccess)
        e = launch_chained(sort_scatter_kernel<NI>, dim3(blocks), dim3(kSortThreads), 0, stream, *prm, d_kps,
                           static_cast<const int*>(cells), static_cast<const int*>(rank),
                           static_cast<const int*>(img_tot), counters, recs);
    if (e == cudaSuccess) {
        // the records are split evenly over the blocks, at least item_kps keypoints each
        const int64_t want = (l.nkp + ctx->item_kps - 1) / ctx->item_kps;
        const int64_t grid = want < 4 * ctx->sm_count ? want : 4 * ctx->sm_count;
        e = launch_chained(extract_cells_kernel<NI>, dim3(static_cast<unsigned>(grid)), dim3(kThreads),
                           extract_smem_bytes(tg), stream, *prm, static_cast<const int4*>(recs),
                           static_cast<const int*>(counters), ctx->d_tile_offsets,
                           reinterpret_cast<const uint2*>(ctx->d_trip_offsets), reinterpret_cast<uint4*>(d_out),
                           reinterpret_cast<uint4*>(exp_out), pop_out, ctx->d_flags);
    }
    delete prm;
    return e;
}

cudaError_t launch_extract_batch(const latch_context* ctx, const latch_image* imgs, const int64_t* kp0,
                                 const int64_t* n, int count, const latch_keypoint* d_kps, uint8_t* d_out,
                                 void* scratch, cudaStream_t stream, uint8_t* exp_out, int32_t* pop_out) {
    uint8_t* base = static_cast<uint8_t*>(scratch);
    for (int i0 = 0; i0 < count; i0 += kBatchImages) {
        const int i1 = i0 + kBatchImages < count ? i0 + kBatchImages : count;
        int64_t nk = 0;
        for (int i = i0; i < i1; ++i) nk += n[i];
        if (nk > 0) {
            // the kernel parameters hold one tensor map per image: the smallest
            // instance that fits keeps the launch's parameter block small
            const int ni = i1 - i0;
            const cudaError_t e =
                ni == 1    ? launch_chunk<1>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, pop_out, base, stream)
                : ni <= 4  ? launch_chunk<4>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, pop_out, base, stream)
                : ni <= 16 ? launch_chunk<16>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, pop_out, base, stream)
                           : launch_chunk<kBatchImages>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, exp_out, pop_out,
                                                        base, stream);
            if (e != cudaSuccess) return e;
        }
        base += chunk_layout(imgs, n, i0, i1).total;
    }
    return cudaSuccess;
}

cudaError_t launch_extract(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps, int32_t n,
                           uint8_t* d_out, void* scratch, cudaStream_t stream) {
    const int64_t kp0 = 0, nn = n;
    return launch_extract_batch(ctx, img, &kp0, &nn, 1, d_kps, d_out, scratch, stream, nullptr, nullptr);
}

}  // namespace latch

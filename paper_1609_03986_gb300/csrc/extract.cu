// LATCH descriptor extraction (Sec. 3.1 Eq. 1; Sec. 3.2).
//
// 1. bucket_kernel (one block): counting sort of the keypoints into 32x32-pixel
//    image cells.  The cell grid reaches 128 px beyond every border; keypoints
//    further out have windows wholly outside the image (the window reaches at most
//    `reach` <= 78 px), whose samples all read 0, so their descriptor is all zeros
//    and is written here directly.  Keypoints with a scale index outside the scale
//    table also get zeros and raise the context's device flag.
// 2. extract_cells_kernel (one block per cell, 8 warps): the image tile under the
//    cell plus a `reach` halo is staged into shared memory by one TMA 2-D load
//    (samples outside the image arrive as 0, the border reading).  For each
//    keypoint of the cell in turn, the block
//      - samples the 48x48 window through the per-(scale, bin) offset table
//        (nearest pixel; offsets pre-multiplied into tile offsets) and stores it
//        as 4 byte-shifted copies, so that the 8 bytes holding any 7-pixel patch
//        row are two aligned 32-bit words;
//      - evaluates Eq. 1 for 32 triplets per warp at a time, one triplet per lane:
//        D1 - D2 = (sum C1^2 - sum C2^2) - 2 (sum A.C1 - sum A.C2) over the 7 rows,
//        with __dp4a on 4 pixels at a time, all exact in 32-bit integers;
//      - packs the 32 bits of each warp-group with __ballot_sync (bit t = bit
//        t % 32 of word t / 32, i.e. bit t % 8 of byte t / 8) and writes the
//        64-byte descriptor as four 128-bit stores.
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
constexpr int kBucketThreads = 1024;
constexpr int kMaxSmemCells = 12288;
constexpr int kMaxItemKps = 32;         // largest work item (keypoints per block visit)

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
    int32_t count;        // images in this launch
    int32_t nscales;
    int32_t item_kps;     // keypoints per work item (1 .. kMaxItemKps; tuned)
    TileGeom tg;
};

// One block per image: counting sort of its keypoints into cells, then its work
// items (chunks of at most item_kps keypoints of one cell) are appended to the
// launch's global item list.  counters[0] = number of items (zeroed by the host).
template <int NI>
__global__ void __launch_bounds__(kBucketThreads) bucket_kernel(const __grid_constant__ ExtractParams<NI> prm,
                                                                const latch_keypoint* __restrict__ kps,
                                                                int* __restrict__ gcount, int4* __restrict__ items,
                                                                int* __restrict__ counters, int* __restrict__ perm,
                                                                uint4* __restrict__ out, uint32_t* __restrict__ flags) {
    extern __shared__ int s_cnt[];
    __shared__ int s_part[kBucketThreads / 32];
    __shared__ int s_ipart[kBucketThreads / 32];
    __shared__ int s_item_base;
    const int img = blockIdx.x;
    const CellGrid g = prm.grid[img];
    const int n = prm.n[img], kp0 = prm.kp0[img];
    const int ncell = g.gx * g.gy;
    const bool in_smem = ncell <= kMaxSmemCells;
    int* cnt = in_smem ? s_cnt : gcount + prm.cell0[img];  // the global counts were zeroed by the host
    if (in_smem)
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    bool bad = false;
    // the cells of the first 16 * 1024 keypoints stay in registers for the second
    // pass; 8 independent keypoint loads are in flight per thread
    constexpr int kCached = 16;
    int cached[kCached];
    auto count_cells = [&](int* cc, int i0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = i0 + j * blockDim.x;
            cc[j] = i < n ? cell_of(kps[kp0 + i], prm.nscales, g) : -3;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = i0 + j * blockDim.x;
            if (cc[j] >= 0) {
                atomicAdd(&cnt[cc[j]], 1);
            } else if (cc[j] > -3) {
                const uint4 z = make_uint4(0, 0, 0, 0);
                uint4* d = out + static_cast<size_t>(kp0 + i) * 4;
                d[0] = z;
                d[1] = z;
                d[2] = z;
                d[3] = z;
                bad |= (cc[j] == -2);
            }
        }
    };
    count_cells(cached, threadIdx.x);
    count_cells(cached + 8, threadIdx.x + 8 * blockDim.x);
    for (int i0 = threadIdx.x + kCached * blockDim.x; i0 < n; i0 += 8 * blockDim.x) {
        int cc[8];
        count_cells(cc, i0);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagBadScale);
    // exclusive scans of the counts and of the work items: each thread sums a
    // contiguous run of cells
    const int per = (ncell + blockDim.x - 1) / blockDim.x;
    const int c0 = threadIdx.x * per, c1 = min(c0 + per, ncell);
    int sum = 0, isum = 0;
    for (int c = c0; c < c1; ++c) {
        const int k = cnt[c];
        sum += k;
        isum += (k + prm.item_kps - 1) / prm.item_kps;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = sum, iincl = isum;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        const int w = __shfl_up_sync(0xffffffffu, iincl, o);
        if (lane >= o) {
            incl += v;
            iincl += w;
        }
    }
    if (lane == 31) {
        s_part[warp] = incl;
        s_ipart[warp] = iincl;
    }
    __syncthreads();
    if (warp == 0) {
        int v = lane < kBucketThreads / 32 ? s_part[lane] : 0;
        int vi = lane < kBucketThreads / 32 ? s_ipart[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int w = __shfl_up_sync(0xffffffffu, v, o);
            const int wi = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) {
                v += w;
                vi += wi;
            }
        }
        if (lane < kBucketThreads / 32) {
            s_part[lane] = v;
            s_ipart[lane] = vi;
        }
        if (lane == kBucketThreads / 32 - 1) s_item_base = atomicAdd(&counters[0], vi);
    }
    __syncthreads();
    int run = kp0 + incl - sum + (warp > 0 ? s_part[warp - 1] : 0);
    int irun = s_item_base + iincl - isum + (warp > 0 ? s_ipart[warp - 1] : 0);
    for (int c = c0; c < c1; ++c) {
        const int k = cnt[c];
        for (int j = 0; j < k; j += prm.item_kps)
            items[irun++] = make_int4(img, c, run + j, run + min(j + prm.item_kps, k));
        cnt[c] = run;  // becomes the insertion cursor (a position in perm)
        run += k;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kCached; ++j)
        if (cached[j] >= 0) perm[atomicAdd(&cnt[cached[j]], 1)] = kp0 + threadIdx.x + j * blockDim.x;
    for (int i0 = threadIdx.x + kCached * blockDim.x; i0 < n; i0 += 8 * blockDim.x) {
        int cc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = i0 + j * blockDim.x;
            cc[j] = i < n ? cell_of(kps[kp0 + i], prm.nscales, g) : -3;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (cc[j] >= 0) perm[atomicAdd(&cnt[cc[j]], 1)] = kp0 + i0 + j * blockDim.x;
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

// Persistent: blocks take work items from the launch's queue (counters[1]).
template <int NI>
__global__ void __launch_bounds__(kThreads) extract_cells_kernel(
    const __grid_constant__ ExtractParams<NI> prm, const latch_keypoint* __restrict__ kps,
    const int* __restrict__ perm, const int4* __restrict__ items, int* __restrict__ counters,
    const int16_t* __restrict__ toff, const uint2* __restrict__ trip_off, uint4* __restrict__ out,
    uint32_t* __restrict__ flags) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_item;
    __shared__ int4 s_kp[kMaxItemKps];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint32_t* s_win = reinterpret_cast<uint32_t*>(smem);                  // [2][kWinWords]
    uint8_t* s_bits = reinterpret_cast<uint8_t*>(s_win + 2 * kWinWords);  // [2][512] one byte per bit
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_bits + 2 * kBits);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_bar + 1);
    uint8_t* s_tile = reinterpret_cast<uint8_t*>(s_bar + 2);
    s_tile = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_tile) + 127) & ~uintptr_t(127));
    const TileGeom tg = prm.tg;
    const int n_items = counters[0];

    if (threadIdx.x == 0) {
        mbar_init(s_bar, 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this thread's window-build job (threads 0..143): row by, 16-pixel segment bseg
    const int by = threadIdx.x / 3, bseg = threadIdx.x % 3;
    // this lane's two triplets (slots 64*warp + lane and +32 of the bank-conflict
    // minimising order): patch word offsets and the triplet's bit position
    const uint2 to0 = trip_off[64 * warp + lane];
    const uint2 to1 = trip_off[64 * warp + 32 + lane];

    for (uint32_t phase = 0;; phase ^= 1) {
        if (threadIdx.x == 0) s_item = atomicAdd(&counters[1], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 item = items[it];
        const int img = item.x, cell = item.y, k0 = item.z, k1 = item.w;
        const CellGrid g = prm.grid[img];
        const int cx = cell % g.gx, cy = cell / g.gx;
        const int ox = cx * kCell - kMargin + tg.mx;  // tile origin in image coordinates
        const int oy = cy * kCell - kMargin + tg.my;
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(s_bar, static_cast<uint32_t>(tg.tw * tg.th));
            tma_load_2d(s_tile, &prm.map[img], ox, oy, s_bar);
        }
        // the item's keypoints, while the tile is in flight: (x, y, table, output row)
        if (threadIdx.x < k1 - k0) {
            const int pi = perm[k0 + threadIdx.x];
            const latch_keypoint kp = kps[pi];
            s_kp[threadIdx.x] = make_int4(kp.x, kp.y, kp.scale_idx * kBins + (kp.angle_bin & (kBins - 1)), pi);
        }
        const bool ok = mbar_wait(s_bar, phase, s_abort);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicOr(flags, kFlagTimeout);
                const uint64_t t0 = globaltimer();  // let the copy land before the block exits
                while (!mbar_try_wait(s_bar, phase) && globaltimer() - t0 < 200000000ull) {
                }
            }
            return;
        }

        // offset-table entries 0..19 of this thread's row segment for the item's first
        // keypoint (32-byte aligned: 96*by + 32*bseg bytes); later ones are prefetched
        // one keypoint ahead, during the previous keypoint's triplets
        int32_t tw[10], tn[10];
        if (threadIdx.x < 144) load_table_segment(toff, s_kp[0].z, by, bseg, tw);

        for (int k = k0; k <= k1; ++k) {
            const int buf = k & 1;
            if (k < k1 && threadIdx.x < 144) {
                // ---- sample the window of keypoint k into 4 byte-shifted copies; this
                // thread: row by, pixels 16*bseg .. 16*bseg+18 ----
                const int4 kp = s_kp[k - k0];
                const int base = (kp.y - oy) * tg.tw + (kp.x - ox);
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
                if (k + 1 < k1) load_table_segment(toff, s_kp[k + 1 - k0].z, by, bseg, tn);
            }
            __syncthreads();
            if (k > k0 && warp == 0) {
                // ---- pack and store the descriptor of keypoint k-1 (all its bits were
                // written before the barrier above): word w collects bits 32w..32w+31 ----
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
                if (lane < 4) out[static_cast<size_t>(s_kp[k - 1 - k0].w) * 4 + lane] = make_uint4(x, y, z, v);
            }
            if (k == k1) break;
#pragma unroll
            for (int j = 0; j < 10; ++j) tw[j] = tn[j];
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
        }
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

// Upper bound on the work items of n keypoints for any item size >= 1.
static int64_t max_items(int64_t n, const CellGrid&) { return n; }

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

// Scratch of one launch over images [i0, i1): counters, cell counts, perm, items.
struct ChunkLayout {
    size_t counters, cells, perm, items, total;
    int64_t ncell, nkp, nitem;
};

static ChunkLayout chunk_layout(const latch_image* imgs, const int64_t* n, int i0, int i1) {
    ChunkLayout l;
    l.ncell = 0;
    l.nkp = 0;
    l.nitem = 0;
    for (int i = i0; i < i1; ++i) {
        const CellGrid g = cell_grid(&imgs[i]);
        l.ncell += static_cast<int64_t>(g.gx) * g.gy;
        l.nkp += n[i];
        l.nitem += max_items(n[i], g);
    }
    l.items = 0;  // int4, 16-byte aligned
    l.counters = l.items + static_cast<size_t>(l.nitem) * sizeof(int4);
    l.cells = l.counters + 16;
    l.perm = l.cells + static_cast<size_t>(l.ncell) * sizeof(int);
    l.total = (l.perm + static_cast<size_t>(l.nkp) * sizeof(int) + 255) / 256 * 256;
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
                                uint8_t* scratch, cudaStream_t stream) {
    static bool attr = false;
    const TileGeom tg = tile_geom(ctx->reach);
    cudaError_t e;
    if (!attr) {
        e = cudaFuncSetAttribute(bucket_kernel<NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sizeof(int) * kMaxSmemCells));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(extract_cells_kernel<NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(extract_smem_bytes(tile_geom(kMaxReach + 1))));
        if (e == cudaSuccess)  // four 56 KB blocks per SM
            e = cudaFuncSetAttribute(extract_cells_kernel<NI>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    EncodeTiledFn enc = extract_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const ChunkLayout l = chunk_layout(imgs, n, i0, i1);
    int4* items = reinterpret_cast<int4*>(scratch + l.items);
    int* counters = reinterpret_cast<int*>(scratch + l.counters);
    int* cells = reinterpret_cast<int*>(scratch + l.cells);
    int* perm = reinterpret_cast<int*>(scratch + l.perm);

    ExtractParams<NI>* prm = new ExtractParams<NI>;
    prm->count = i1 - i0;
    prm->nscales = ctx->nscales;
    prm->item_kps = ctx->item_kps;
    prm->tg = tg;
    bool global_cells = false;
    int64_t cell0 = 0;
    size_t bucket_smem = 0;
    for (int i = i0; i < i1; ++i) {
        const int j = i - i0;
        const CellGrid g = cell_grid(&imgs[i]);
        const int64_t ncell = static_cast<int64_t>(g.gx) * g.gy;
        prm->grid[j] = g;
        prm->kp0[j] = static_cast<int32_t>(kp0[i]);
        prm->n[j] = static_cast<int32_t>(n[i]);
        prm->cell0[j] = static_cast<int32_t>(cell0);
        cell0 += ncell;
        if (ncell > kMaxSmemCells)
            global_cells = true;
        else if (sizeof(int) * ncell > bucket_smem)
            bucket_smem = sizeof(int) * ncell;
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
    e = cudaMemsetAsync(counters, 0, 16, stream);
    if (e == cudaSuccess && global_cells) e = cudaMemsetAsync(cells, 0, sizeof(int) * l.ncell, stream);
    if (e == cudaSuccess) {
        bucket_kernel<NI><<<i1 - i0, kBucketThreads, bucket_smem, stream>>>(
            *prm, d_kps, cells, items, counters, perm, reinterpret_cast<uint4*>(d_out), ctx->d_flags);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t grid = l.nitem < 4 * ctx->sm_count ? l.nitem : 4 * ctx->sm_count;
        extract_cells_kernel<NI><<<static_cast<unsigned>(grid), kThreads, extract_smem_bytes(tg), stream>>>(
            *prm, d_kps, perm, items, counters, ctx->d_tile_offsets,
            reinterpret_cast<const uint2*>(ctx->d_trip_offsets), reinterpret_cast<uint4*>(d_out), ctx->d_flags);
        note_launches(1);
        e = cudaGetLastError();
    }
    delete prm;
    return e;
}

cudaError_t launch_extract_batch(const latch_context* ctx, const latch_image* imgs, const int64_t* kp0,
                                 const int64_t* n, int count, const latch_keypoint* d_kps, uint8_t* d_out,
                                 void* scratch, cudaStream_t stream) {
    uint8_t* base = static_cast<uint8_t*>(scratch);
    for (int i0 = 0; i0 < count; i0 += kBatchImages) {
        const int i1 = i0 + kBatchImages < count ? i0 + kBatchImages : count;
        int64_t nk = 0;
        for (int i = i0; i < i1; ++i) nk += n[i];
        if (nk > 0) {
            const cudaError_t e =
                (i1 - i0 == 1) ? launch_chunk<1>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, base, stream)
                               : launch_chunk<kBatchImages>(ctx, imgs, kp0, n, i0, i1, d_kps, d_out, base, stream);
            if (e != cudaSuccess) return e;
        }
        base += chunk_layout(imgs, n, i0, i1).total;
    }
    return cudaSuccess;
}

cudaError_t launch_extract(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps, int32_t n,
                           uint8_t* d_out, void* scratch, cudaStream_t stream) {
    const int64_t kp0 = 0, nn = n;
    return launch_extract_batch(ctx, img, &kp0, &nn, 1, d_kps, d_out, scratch, stream);
}

}  // namespace latch

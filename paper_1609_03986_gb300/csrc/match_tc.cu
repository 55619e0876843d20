// Brute-force Hamming matching on the 5th-generation tensor cores (Sec. 4's
// all-pairs distance computation, done as a dense contraction).
//
// Every descriptor bit b is expanded to the 4-bit E2M1 float 1 - 2 b (+1 or -1, two
// per byte), so the dot product of two expanded descriptors is (bits that agree) -
// (bits that differ) = 512 - 2 Hamming(q, t): one contraction gives the distance,
// with no popcount term.  The block-scaled fp4 MMA (kind::mxf4, every scale factor
// 2^0) issues twice the products per clock of the 8-bit kind; the products are +-1
// and the sums at most 512 in magnitude, so fp32 accumulation is exact.
//
// One launch serves a batch of matching problems (query set x train set pairs; a
// single hamming_match call is a batch of one).  All descriptors live in one
// expanded buffer (two TMA tensor maps over it: 128-row query boxes, 240-row train
// boxes).  The units (problem, 128-query tile, 240-train tile) of all problems are
// linearised and split into one contiguous range per block (one block per SM,
// persistent):
//   warp 0     TMA producer: the query tile (128 rows x 256 B, 32 KB) stays resident
//              while consecutive units share it; train chunks (240 rows x 128 B, half
//              of K) go through a 6-stage ring, 128-byte swizzle;
//   warps 1-2  MMA issuers (even / odd units): per unit 8 tcgen05.mma (M=128,
//              N=240, K=64) into one of two TMEM accumulators (columns 0 and 256; the
//              constant scale factors in 496-511); warp 2 also allocates TMEM;
//   warp 3     idle;
//   warps 4-23 epilogue (one query row and 48 columns per thread): three reducing
//              TMEM loads (tcgen05.ld.red .max) bring the 48 values and the largest
//              of each 16, and the accumulator is released at once.  A group of 16
//              whose largest value is below the row's bound costs nothing more: the
//              bound is the smallest second-best distance any of the row's five
//              column groups holds (shared memory), and a column displaces one of its
//              own group's keys only with a larger value (later columns have larger
//              train indices).  The others take the top-two update (a tournament over
//              64 v - column, unique values that break ties to the lower index).  When
//              the block leaves a query tile the row's two (distance << 32 | index)
//              keys go to a partial record.  In a launch of at most
//              kFusedUnitsPerBlock units per block the last block to leave a tile (a
//              per-tile arrival counter) combines the records of its rows and writes
//              their matches (ties to the lowest train index, ratio test).
// The unit width is a compile-time choice (LATCH_TC_COLS): 160 gives three
// accumulators in rotation (columns 0, 160, 320) and 32 columns per epilogue thread.
// match_merge_kernel does the same combination as a separate pass; it serves longer
// launches and the batches in which some problem has queries but an empty train set
// (no unit, so no block visits its tiles).  All mbarrier waits are bounded (sm103.h); on a timeout
// the block raises the device flag, drains its copies and MMAs, frees TMEM.
#include <cuda.h>

#include <cmath>
#include <new>

#include "match_common.cuh"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kRowsA = 128;             // rows per MMA (M) = queries per tile
constexpr int kRowsQ = kRowsA;
#ifndef LATCH_TC_COLS
#define LATCH_TC_COLS 240
#endif
constexpr int kColsB = LATCH_TC_COLS;   // train rows per unit (N): 240 (two accumulators) or 160 (three)
constexpr int kRowsP = kRowsQ;          // partial records per tile slot: one per query row
constexpr int kKBytes = kExpRowBytes;   // expanded descriptor: 512 x 4-bit
constexpr int kChunk = 128;             // K bytes per swizzle atom / TMA box
constexpr int kChunks = kKBytes / kChunk;
constexpr int kMmaKBytes = 32;          // K bytes per MMA: 64 E2M1 values
constexpr int kStages = kColsB > 192 ? 6 : 8;  // train chunks in flight (three / four units)
constexpr int kTileBytes = kRowsA * kChunk;   // 16 KB: a query chunk of 128 rows x 128 B (one TMA box)
constexpr int kStageBytes = kColsB * kChunk;  // a train chunk of kColsB rows x 128 B (one TMA box)
constexpr int kAccs = kColsB > 160 ? 2 : 3;    // TMEM accumulators in rotation (unit i uses i % kAccs)
constexpr int kAccStride = kColsB > 160 ? 256 : kColsB;  // accumulator a at TMEM columns [a kAccStride, +kColsB)
constexpr int kEpiWarps = 20;           // epilogue: 4 lane quarters x 5 column groups
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 128 + kEpiThreads;         // producer, two MMA issuers, an idle warp, then the epilogue
constexpr int kColGroups = kEpiWarps / 4;
constexpr int kColsPerThread = kColsB / kColGroups;  // accumulator columns one epilogue thread scans
constexpr int kLdCols = 16;                          // columns per tcgen05.ld
constexpr int kLds = kColsPerThread / kLdCols;       // loads per unit and thread
constexpr int kTmemCols = 512;
constexpr uint32_t kSfaCol = (kAccs - 1) * kAccStride + kColsB;  // scale factors of A: 4 columns (128 rows)
constexpr uint32_t kSfbCol = kSfaCol + 8;  // scale factors of B: 4 columns per 128 rows
constexpr uint32_t kScaleOne = 0x7F7F7F7Fu;  // four UE8M0 scale factors 2^0 (columns 480-511 all hold it)
constexpr uint32_t kIdesc = idesc_mxf4_e2m1(kRowsA, kColsB);
constexpr int32_t kNoBound = 1024;      // a distance bound above every distance (512 bits)
constexpr int64_t kFusedUnitsPerBlock = 64;  // longer launches combine the tiles' records in a separate pass
constexpr int64_t kWholeTilesPerBlock = 8;   // batches with this many query tiles per block share whole tiles
static_assert(kSfaCol % 8 == 0 && kSfbCol + 4 * ((kColsB + 127) / 128) <= kTmemCols, "TMEM columns overlap");
static_assert(kColsPerThread == kLds * kLdCols && kColsB == kColGroups * kColsPerThread, "epilogue column split");
static_assert(kColsB % 16 == 0 && kColsB <= 256 && kColsPerThread < 64 && kAccStride % 32 == 0, "unit shape");

// max(a, b, c) in one instruction.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Barrier of the epilogue threads (named barrier 1).
__device__ __forceinline__ void group_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

struct Smem {
    // offsets in the 1024-aligned dynamic buffer
    static constexpr int a = 0;                                        // [kChunks] boxes of 16 KB
    static constexpr int b = a + kChunks * kTileBytes;                 // [kStages] chunks of 20 KB
    static constexpr int part = b + kStages * kStageBytes;             // uint64 [kEpiThreads][2]
    static constexpr int bound = part + kEpiThreads * 16;              // int32 [kRowsQ]
    static constexpr int bars = bound + kRowsQ * 4;                    // uint64 barriers
    static constexpr int nbars = 2 * kStages + 2 + 2 * kAccs + 2;
    static constexpr int misc = bars + nbars * 8;                      // tmem base, abort flag, last-arrival flag
    static constexpr int total = misc + 16;
};
constexpr int kSmemBytes = Smem::total + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory per block");

// Walks the units of block c: for every problem in turn, the block's share of that
// problem's U units, [start(c'), start(c' + 1)) with start(x) = floor(x U / G) and
// c' = (c - unit0) mod G (the rotation continues each problem where the previous
// one ended, so problems smaller than G still spread over all blocks), without
// dividing inside a share.  All blocks thus work on the same problem at a time and
// share its train set in L2.  last_of_tile(): the next unit of the walk is in
// another query tile.  A block's record of tile g in problem p sits in slot
// g + c' + p (G - 1): within a problem a later share never touches an earlier
// tile, and the problems' slot ranges follow one another.
// A block's share of one problem: the first unit (m, n), the share index and the
// number of units; p == count when there is none left.
struct Share {
    int32_t p, m, n, cs;
    int64_t left;
};

// The first problem from p on in which block c has a non-empty share.  Out of line:
// it divides, and runs only where a share starts.
template <class B>
__device__ __noinline__ Share next_share(const B& b, int p, int64_t c) {
    for (; p < b.count; ++p) {
        const MatchProblem& P = b.p[p];
        const int64_t U = static_cast<int64_t>(P.mt) * P.ntl;
        if (U == 0) continue;
        if (b.whole_tiles) {
            // tiles [start(c'), start(c' + 1)) of the problem's mt, c' rotated by the
            // problem's first tile index
            const int64_t rot = P.g0 % b.grid;
            const int64_t cp = c >= rot ? c - rot : c - rot + b.grid;
            const int64_t t0 = split_start(cp, P.mt, b.grid), t1 = split_start(cp + 1, P.mt, b.grid);
            if (t1 > t0)
                return Share{p, static_cast<int32_t>(t0), 0, static_cast<int32_t>(cp), (t1 - t0) * P.ntl};
            continue;
        }
        const int64_t rot = P.unit0 % b.grid;
        const int64_t cp = c >= rot ? c - rot : c - rot + b.grid;
        const int64_t s0 = split_start(cp, U, b.grid), s1 = split_start(cp + 1, U, b.grid);
        if (s1 > s0) {
            const int32_t m = static_cast<int32_t>(s0 / P.ntl);
            return Share{p, m, static_cast<int32_t>(s0 - static_cast<int64_t>(m) * P.ntl), static_cast<int32_t>(cp),
                         s1 - s0};
        }
    }
    return Share{b.count, 0, 0, 0, 0};
}

// The fields of the current problem that the walk needs every unit are kept in
// registers (reading the problem table, a kernel parameter, with a run-time index
// costs hundreds of cycles per unit on the MMA warp's path).
struct UnitIter {
    int p;          // current problem (count once the walk is over)
    int count;      // problems in the batch
    int32_t m, n;   // query tile, train tile of the current unit
    int32_t cs;     // c': the block's share index in problem p
    int32_t ntl;    // train tiles of problem p
    int32_t g0;     // global index of problem p's first query tile
    int32_t t_row0; // first train row of problem p
    int32_t nt;     // train rows of problem p
    int64_t left;   // units left in the share, the current one included
    template <class B>
    __device__ __forceinline__ void take(const B& b, int from, int64_t c) {
        const Share s = next_share(b, from, c);
        p = s.p;
        m = s.m;
        n = s.n;
        cs = s.cs;
        left = s.left;
        if (p < count) {
            const MatchProblem& P = b.p[p];
            ntl = P.ntl;
            g0 = P.g0;
            t_row0 = P.t_row0;
            nt = P.nt;
        }
    }
    template <class B>
    __device__ __forceinline__ void init(const B& b, int64_t c) {
        count = b.count;
        take(b, 0, c);
    }
    template <class B>
    __device__ __forceinline__ bool done(const B&) const { return p >= count; }
    template <class B>
    __device__ __forceinline__ int64_t g(const B&) const { return g0 + m; }
    template <class B>
    __device__ __forceinline__ int64_t slot(const B& b) const {
        return g0 + m + cs + static_cast<int64_t>(p) * (b.grid - 1);
    }
    template <class B>
    __device__ __forceinline__ bool last_of_tile(const B&) const { return left == 1 || n + 1 == ntl; }
    template <class B>
    __device__ __forceinline__ void next(const B& b, int64_t c) {
        if (--left == 0) {
            take(b, p + 1, c);
            return;
        }
        if (++n == ntl) {
            n = 0;
            ++m;
        }
    }
};

// The block's walk as runs: a run is the consecutive units of one query tile (a run
// ends where its tile or its share ends, so consecutive runs are different tiles).
// The MMA issuers step through runs and count units inside them, which keeps the
// iterator off their per-unit path.
struct RunIter {
    UnitIter u;     // at the run's first unit
    int32_t len;    // units in the run
    template <class B>
    __device__ __forceinline__ void init(const B& b, int64_t c) {
        u.init(b, c);
        set(b);
    }
    template <class B>
    __device__ __forceinline__ void set(const B& b) {
        const int64_t rest = static_cast<int64_t>(u.ntl - u.n);
        len = u.done(b) ? 0 : static_cast<int32_t>(u.left < rest ? u.left : rest);
    }
    template <class B>
    __device__ __forceinline__ bool done(const B& b) const { return u.done(b); }
    template <class B>
    __device__ __forceinline__ void next(const B& b, int64_t c) {
        if (len == u.left) {
            u.take(b, u.p + 1, c);  // the share ends with this run
        } else {
            u.left -= len;          // the run ends with its tile
            ++u.m;
            u.n = 0;
        }
        set(b);
    }
};

// Calls f(c') for the share index of every block that holds a record of query tile
// m of problem P, and returns how many there are.  With U >= G every share is
// non-empty and the owners are the contiguous range from the share of the tile's
// first unit to that of its last; with U < G every non-empty share holds one unit,
// so the owners are those of the tile's ntl units.
template <class B, class F>
__device__ __forceinline__ int64_t for_each_owner(const B& b, const MatchProblem& P, int64_t m, F&& f) {
    if (b.whole_tiles) {
        f(split_owner(m, P.mt, b.grid));
        return 1;
    }
    const int64_t U = static_cast<int64_t>(P.mt) * P.ntl;
    const int64_t u0 = m * P.ntl;
    if (U >= b.grid) {
        const int64_t clo = split_owner(u0, U, b.grid), chi = split_owner(u0 + P.ntl - 1, U, b.grid);
        for (int64_t cs = clo; cs <= chi; ++cs) f(cs);
        return chi - clo + 1;
    }
    for (int64_t u = u0; u < u0 + P.ntl; ++u) f(split_owner(u, U, b.grid));
    return P.ntl;
}

// Number of blocks that hold a record of query tile m of problem P.
template <class B>
__device__ __forceinline__ int64_t tile_owner_count(const B& b, const MatchProblem& P, int64_t m) {
    if (b.whole_tiles) return 1;
    const int64_t U = static_cast<int64_t>(P.mt) * P.ntl;
    if (U < b.grid) return P.ntl;
    const int64_t u0 = m * P.ntl;
    return split_owner(u0 + P.ntl - 1, U, b.grid) - split_owner(u0, U, b.grid) + 1;
}

// Combines the partial records of row r of query tile m (global index g) of problem
// p over the blocks that own the tile's units.
template <class B>
__device__ __forceinline__ void combine_row(const B& b, int p, int64_t m, int64_t g, int r,
                                            const uint64_t* partials, uint64_t& k1, uint64_t& k2) {
    for_each_owner(b, b.p[p], m, [&](int64_t cs) {
        const uint64_t* rec = partials + ((g + cs + static_cast<int64_t>(p) * (b.grid - 1)) * kRowsP + r) * 2;
        top2_insert_u64(__ldcg(rec), k1, k2);
        top2_insert_u64(__ldcg(rec + 1), k1, k2);
    });
}

// The output record of a query from its two best keys (Sec. 4 ratio test).
__device__ __forceinline__ latch_match final_match(uint64_t k1, uint64_t k2, int k, int r_milli) {
    latch_match mres;
    mres.idx1 = k1 == kNoKey ? -1 : static_cast<int32_t>(k1 & 0xffffffffu);
    mres.dist1 = k1 == kNoKey ? 0xffff : static_cast<uint16_t>(k1 >> 32);
    const bool has2 = k == 2 && k2 != kNoKey;
    mres.idx2 = has2 ? static_cast<int32_t>(k2 & 0xffffffffu) : -1;
    mres.dist2 = has2 ? static_cast<uint16_t>(k2 >> 32) : 0xffff;
    if (k1 == kNoKey)
        mres.accepted = 0;
    else if (k == 1)
        mres.accepted = 1;
    else
        mres.accepted = (1000ll * mres.dist1 < static_cast<long long>(r_milli) * mres.dist2) ? 1 : 0;
    mres.pad[0] = mres.pad[1] = mres.pad[2] = 0;
    return mres;
}

// tile_cnt: per-query-tile arrival counters, zero at launch and zero again after a
// complete launch; NULL = leave the combination to match_merge_kernel.
template <int NP>
__global__ void __launch_bounds__(kThreads, 1) match_tc_kernel(const __grid_constant__ CUtensorMap tmq,
                                                              const __grid_constant__ CUtensorMap tmt,
                                                              const __grid_constant__ MatchBatchT<NP> batch,
                                                              uint64_t* __restrict__ partials,
                                                              int32_t* __restrict__ tile_cnt,
                                                              latch_match* __restrict__ out,
                                                              uint32_t* __restrict__ flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem + Smem::a;
    uint8_t* sB = smem + Smem::b;
    uint64_t* sPart = reinterpret_cast<uint64_t*>(smem + Smem::part);
    int32_t* sBound = reinterpret_cast<int32_t*>(smem + Smem::bound);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Smem::bars);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* a_full = bars + 2 * kStages;
    uint64_t* a_empty = a_full + 1;
    uint64_t* acc_full = a_full + 2;               // [kAccs]
    uint64_t* acc_empty = acc_full + kAccs;        // [kAccs]
    uint64_t* mma_done = acc_empty + kAccs;        // [2]: one per MMA warp
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Smem::misc);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + Smem::misc + 4);
    volatile int* last_arrival = reinterpret_cast<volatile int*>(smem + Smem::misc + 8);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t c = blockIdx.x;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 2);  // both MMA warps commit once per query tile
        for (int i = 0; i < kAccs; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kEpiThreads / 32);
        }
        mbar_init(&mma_done[0], 1);
        mbar_init(&mma_done[1], 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(&tmq);
        prefetch_tmap(&tmt);
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, kTmemCols);
        tc_fence_before();
    }
    for (int r = threadIdx.x; r < kRowsQ; r += kThreads) sBound[r] = kNoBound;
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 4 && warp < 8) {
        // block scale factors 2^0 in columns kSfaCol..511 of all 128 lanes (warp w may
        // address lane quarter w % 4)
        const uint32_t base = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
#pragma unroll
        for (uint32_t col = kSfaCol; col < kTmemCols; col += 8) tmem_st_32x32b_x8_same(base + col, kScaleOne);
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // everything above touched only this block's shared memory and TMEM
    griddep_wait();
    griddep_launch_dependents();

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            UnitIter it;
            it.init(batch, c);
            int stage = 0;
            uint32_t ring = 0, a_par = 0;
            // bit s: stage s has a copy issued / the parity of its latest fill (bit masks
            // rather than arrays, which a run-time index would put in local memory)
            uint32_t filled = 0, fill_par = 0;
            int64_t prev_g = -1;
            for (; !it.done(batch); it.next(batch, c)) {
                const MatchProblem& P = batch.p[it.p];
                const int64_t m = it.m, n = it.n;
                const int64_t g = it.g(batch);
                if (g != prev_g) {
                    if (prev_g >= 0) {
                        if (!mbar_wait(a_empty, a_par, abort)) break;
                        a_par ^= 1;
                    }
                    mbar_arrive_expect_tx(a_full, kChunks * kTileBytes);
                    for (int kc = 0; kc < kChunks; ++kc)
                        tma_load_2d(sA + kc * kTileBytes, &tmq, kc * kChunk, static_cast<int32_t>(P.q_row0 + m * kRowsQ),
                                    a_full);
                    prev_g = g;
                }
                bool ok = true;
                for (int kc = 0; kc < kChunks; ++kc) {
                    if (!mbar_wait(&empty[stage], ring ^ 1, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], kStageBytes);
                    tma_load_2d(sB + stage * kStageBytes, &tmt, kc * kChunk, static_cast<int32_t>(it.t_row0 + n * kColsB),
                                &full[stage]);
                    filled |= 1u << stage;
                    fill_par = (fill_par & ~(1u << stage)) | (ring << stage);
                    if (++stage == kStages) {
                        stage = 0;
                        ring ^= 1;
                    }
                }
                if (!ok) break;
            }
            if (*abort) {
                // let copies still in flight land before the block exits (bounded)
                const uint64_t t0 = globaltimer();
                for (int s = 0; s < kStages; ++s)
                    while (((filled >> s) & 1u) && !mbar_try_wait(&full[s], (fill_par >> s) & 1u) &&
                           globaltimer() - t0 < 200000000ull) {
                    }
                if (prev_g >= 0)  // the last A load completes the a_full phase of parity a_par
                    while (!mbar_try_wait(a_full, a_par) && globaltimer() - t0 < 200000000ull) {
                    }
            }
        }
    } else if (warp == 1 || warp == 2) {
        // ---------------- MMA issuers: warp 1 issues the even units, warp 2 the odd ones
        // (a thread's tcgen05.mma waits until the tensor pipe takes it, so a single
        // issuer leaves the pipe idle while it waits on barriers between units; with two,
        // one issuer's waits overlap the other's MMAs).  Unit i uses accumulator i % 3
        // and stages 2 i, 2 i + 1 of the ring; both issuers walk every unit, wait for
        // every query tile and commit a_empty (count 2) at every tile's end. ----------------
        if (lane == 0) {
            const int mine = warp - 1;
            RunIter run;
            run.init(batch, c);
            uint32_t a_par = 0;
            // shared-memory descriptors of the first query box and train chunk; the others
            // differ only in the start-address field (bits 0-13: address / 16), so each MMA
            // adds a constant to them
            const uint64_t a_desc0 = umma_desc_sw128(smem_u32(sA));
            const uint64_t b_desc0 = umma_desc_sw128(smem_u32(sB));
            const uint32_t sfa = tmem + kSfaCol, sfb = tmem + kSfbCol;
            int i = 0;  // the run's first unit in the block's walk
            bool ok = true;
            for (; ok && !run.done(batch); run.next(batch, c)) {
                if (!mbar_wait(a_full, a_par, abort)) break;  // every run is a new query tile
                a_par ^= 1;
                const int end = i + run.len;
                for (int j = i + ((i & 1) ^ mine); ok && j < end; j += 2) {
                    const int acc = j % kAccs;
                    if (!mbar_wait(&acc_empty[acc], static_cast<uint32_t>((j / kAccs) & 1) ^ 1u, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + static_cast<uint32_t>(acc * kAccStride);
                    // unit j reads ring positions 2 j and 2 j + 1; its first MMA overwrites D
#pragma unroll
                    for (int kc = 0; kc < kChunks; ++kc) {
                        const int pos = kChunks * j + kc;
                        const int stage = pos % kStages;
                        if (!mbar_wait(&full[stage], static_cast<uint32_t>(pos / kStages) & 1u, abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t bd = b_desc0 + static_cast<uint64_t>((stage * kStageBytes) >> 4);
                        const uint64_t ad = a_desc0 + static_cast<uint64_t>((kc * kTileBytes) >> 4);
#pragma unroll
                        for (int ks = 0; ks < kChunk / kMmaKBytes; ++ks)
                            mma_mxf4(d, ad + static_cast<uint64_t>((ks * kMmaKBytes) >> 4),
                                     bd + static_cast<uint64_t>((ks * kMmaKBytes) >> 4), kIdesc, sfa, sfb,
                                     (kc | ks) != 0);
                        mma_commit(&empty[stage]);
                    }
                    if (ok) mma_commit(&acc_full[acc]);
                }
                i = end;
                if (ok) mma_commit(a_empty);
            }
            // every issued MMA has finished before TMEM is released
            mma_commit(&mma_done[mine]);
            const uint64_t t0 = globaltimer();
            while (!mbar_try_wait(&mma_done[mine], 0) && globaltimer() - t0 < 200000000ull) {
            }
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: kEpiWarps warps; thread = one query row x one
        // group of kColsPerThread accumulator columns.  The walk goes by runs (the
        // consecutive units of one query tile), so the per-unit path touches only
        // counters in registers; the problem table is read where a run ends. ----------------
        const int et = threadIdx.x - 128;  // 0 .. kEpiThreads-1 = cg * kRowsQ + row_in_tile
        const int quarter = warp & 3;      // TMEM lane quarter this warp may access
        const int cg = (warp - 4) >> 2;    // column group [cg * kColsPerThread, +kColsPerThread)
        const int col0 = cg * kColsPerThread;
        const int row_in_tile = quarter * 32 + lane;
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(col0);
        const float kNegInf = __int_as_float(0xff800000);
        RunIter run;
        run.init(batch, c);
        int acc = 0;           // accumulator of the next unit (unit i uses i % kAccs)
        uint32_t acc_par = 0;  // bit a: the phase parity of accumulator a
        bool aborted = false;  // warp-uniform
        for (; !run.done(batch); run.next(batch, c)) {
            const UnitIter& u = run.u;  // the run's first unit
            uint64_t k1 = kNoKey, k2 = kNoKey;
            // 2 + the value (512 - 2 distance) of the thread's second-best key: the
            // thread's later columns have larger train indices, so one displaces a key
            // of the thread only with a larger value (values are even integers)
            float vown2 = kNegInf;
            // the thread's columns in the problem's last train tile that lie inside the
            // train set (the rest are rows of zeros or of the next problem)
            const int32_t n_last = u.ntl - 1;
            const int32_t lim_last = u.nt - n_last * kColsB - col0;
            // the top-two update from 16 of the thread's columns (group h: columns
            // 16 h .. 16 h + 15) of train tile n.  w = 64 v - j orders the columns by
            // value, then by lower index, and is unique (|v| <= 512, j < 64: exact in
            // fp32); the best two of the 16 by a tournament: (max, min) of each pair,
            // then three rounds of (a1, a2) + (b1, b2) -> (max, second max)
            auto update = [&](const float (&e)[kColsPerThread], int h, int32_t n, float vmin) {
                float t1[kLdCols / 2], t2[kLdCols / 2];
#pragma unroll
                for (int q = 0; q < kLdCols / 2; ++q) {
                    const int j = h * kLdCols + 2 * q;
                    const float wa = fmaf(e[j], 64.0f, -static_cast<float>(j));
                    const float wb = fmaf(e[j + 1], 64.0f, -static_cast<float>(j + 1));
                    t1[q] = fmaxf(wa, wb);
                    t2[q] = fminf(wa, wb);
                }
#pragma unroll
                for (int w = kLdCols / 4; w >= 1; w >>= 1)
#pragma unroll
                    for (int q = 0; q < w; ++q) {
                        const float lo = fminf(t1[q], t1[q + w]);
                        t1[q] = fmaxf(t1[q], t1[q + w]);
                        t2[q] = fmaxf(lo, fmaxf(t2[q], t2[q + w]));
                    }
                const float m1 = t1[0], m2 = t2[0];
                // the two best -> (distance << 32 | index) keys (-inf marks masked
                // columns); the second only where it can still enter (v >= vmin: w >=
                // 64 vmin - 63) or the thread holds fewer than two keys, so that its own
                // second-best stays defined
                const bool want2 = m2 >= fmaf(vmin, 64.0f, -63.0f) || k2 == kNoKey;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const float mv = b == 0 ? m1 : m2;
                    if (mv != kNegInf && (b == 0 || want2)) {
                        const int32_t w = static_cast<int32_t>(mv);
                        const int32_t j = (-w) & 63;
                        const int32_t d = 256 - ((w + j) >> 7);  // v = (w + j) / 64, d = (512 - v) / 2
                        const uint32_t idx = static_cast<uint32_t>(n) * kColsB + static_cast<uint32_t>(col0 + j);
                        top2_insert_u64((static_cast<uint64_t>(d) << 32) | idx, k1, k2);
                    }
                }
                // the row's bound: the smallest second-best distance of its column groups
                if (k2 != kNoKey) {
                    const int32_t d2 = static_cast<int32_t>(k2 >> 32);
                    vown2 = static_cast<float>(514 - 2 * d2);
                    atomicMin(&sBound[row_in_tile], d2);
                }
            };
            const int32_t n_end = u.n + run.len;
            for (int32_t n = u.n; n < n_end; ++n) {
                // after a failed wait a warp keeps walking the units without work, so that
                // every warp reaches the barriers at the ends of query tiles
                if (!aborted) aborted = !__all_sync(0xffffffffu, mbar_wait(&acc_full[acc], (acc_par >> acc) & 1u, abort));
                if (!aborted) {
                    acc_par ^= 1u << acc;
                    tc_fence_after();
                    // the thread's columns (512 - 2 Hamming, exact integers) and the largest
                    // of each half in one round trip; the accumulator is free again as soon
                    // as they are in registers
                    const uint32_t base = lane_base + static_cast<uint32_t>(acc * kAccStride);
                    uint32_t v[kLds][kLdCols];
                    float mx[kLds];
#pragma unroll
                    for (int h = 0; h < kLds; ++h)
                        tmem_ld_red_max_32x32b_x16(base + static_cast<uint32_t>(h * kLdCols), v[h], mx[h]);
                    // some column group of the row holds two keys at distance <= bound, so a
                    // column enters the row's final top two only at a distance <= bound
                    // (equal: when its index is lower than a key's of another group), i.e.
                    // with a value >= 512 - 2 bound, and only above the thread's second best
                    const float vmin = fmaxf(
                        static_cast<float>(512 - 2 * *static_cast<volatile int32_t*>(&sBound[row_in_tile])), vown2);
                    tmem_ld_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[acc]);
                    float e[kColsPerThread];
#pragma unroll
                    for (int h = 0; h < kLds; ++h)
#pragma unroll
                        for (int j = 0; j < kLdCols; ++j) e[h * kLdCols + j] = __uint_as_float(v[h][j]);
                    if (n == n_last && lim_last < kColsPerThread) {
#pragma unroll
                        for (int h = 0; h < kLds; ++h) {
                            mx[h] = kNegInf;
#pragma unroll
                            for (int j = h * kLdCols; j < (h + 1) * kLdCols; ++j) {
                                if (j >= lim_last) e[j] = kNegInf;
                                mx[h] = fmaxf(mx[h], e[j]);
                            }
                        }
                    }
                    // only a group of 16 that reaches the row's bound takes the top-two update
#pragma unroll
                    for (int h = 0; h < kLds; ++h)
                        if (__any_sync(0xffffffffu, mx[h] >= vmin)) update(e, h, n, vmin);
                }
                if (++acc == kAccs) acc = 0;
            }
            // the run ends where the block leaves its query tile: the column groups of
            // each row meet in shared memory; group 0 writes the row's partial record
            // (slot g + c')
            const MatchProblem& P = batch.p[u.p];
            const int64_t m = u.m;
            const int64_t g = u.g(batch);
            sPart[2 * et] = k1;
            sPart[2 * et + 1] = k2;
            group_sync();  // every thread is past the run's last bound read
            if (cg == 0) {
                sBound[row_in_tile] = kNoBound;
#pragma unroll
                for (int q = 1; q < kColGroups; ++q) {
                    top2_insert_u64(sPart[2 * (q * kRowsQ + row_in_tile)], k1, k2);
                    top2_insert_u64(sPart[2 * (q * kRowsQ + row_in_tile) + 1], k1, k2);
                }
                if (batch.whole_tiles) {
                    // the block owns the whole tile: the row's two keys are final
                    const int64_t row = m * kRowsQ + row_in_tile;
                    if (row < P.nq) out[P.out0 + row] = final_match(k1, k2, P.k, P.r_milli);
                } else {
                    uint64_t* rec = partials + (u.slot(batch) * kRowsP + row_in_tile) * 2;
                    rec[0] = k1;
                    rec[1] = k2;
                    if (tile_cnt) __threadfence();  // the records are published before the arrival below
                }
            }
            group_sync();  // the shared records are free for the next run
            if (tile_cnt && !batch.whole_tiles) {
                // the last owner of the tile to arrive combines the records
                if (et == 0) {
                    const bool last = atomicAdd(&tile_cnt[g], 1) == tile_owner_count(batch, P, m) - 1;
                    if (last) tile_cnt[g] = 0;  // no other block touches it again: leave it zero
                    *last_arrival = last;
                }
                group_sync();
                if (*last_arrival && cg == 0) {
                    __threadfence();
                    const int64_t row = m * kRowsQ + row_in_tile;
                    uint64_t f1 = kNoKey, f2 = kNoKey;
                    combine_row(batch, u.p, m, g, row_in_tile, partials, f1, f2);
                    if (row < P.nq) out[P.out0 + row] = final_match(f1, f2, P.k, P.r_milli);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicOr(flags, kFlagTimeout);
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Combine the partial records of every query row; write one latch_match per query.
template <int NP>
__global__ void match_merge_kernel(const __grid_constant__ MatchBatchT<NP> batch,
                                   const uint64_t* __restrict__ partials, latch_match* __restrict__ out) {
    griddep_wait();
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= batch.queries) return;
    int lo = 0, hi = batch.count - 1;  // problem: largest p with out0 <= q
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (batch.p[mid].out0 <= q) lo = mid; else hi = mid - 1;
    }
    const MatchProblem& P = batch.p[lo];
    const int64_t ql = q - P.out0;
    uint64_t k1 = kNoKey, k2 = kNoKey;
    if (P.ntl > 0) {
        const int64_t m = ql / kRowsQ;
        combine_row(batch, lo, m, P.g0 + m, static_cast<int>(ql % kRowsQ), partials, k1, k2);
    }
    out[q] = final_match(k1, k2, P.k, P.r_milli);
}

// Bits -> E2M1 +-1 values (bit t of a descriptor -> 4-bit value t, kExpRowBytes per
// row); one thread per 32-bit descriptor word.
__global__ void expand_kernel(const uint32_t* __restrict__ in, int64_t nwords, uint4* __restrict__ out) {
    griddep_wait();
    griddep_launch_dependents();
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < nwords) out[i] = expand_word_e2m1(in[i]);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kKBytes), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kKBytes)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kChunk), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

cudaError_t launch_expand(const uint8_t* desc, int64_t n, uint8_t* out, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t nwords = n * 16;
    const int threads = 256;
    const int64_t grid = (nwords + threads - 1) / threads;
    return launch_chained(expand_kernel, dim3(static_cast<unsigned>(grid)), dim3(threads), 0, stream,
                          reinterpret_cast<const uint32_t*>(desc), nwords, reinterpret_cast<uint4*>(out));
}

// Fills tiles, unit offsets, query-tile prefixes and the block split.  problems[i]
// must have q_row0, t_row0, nq, nt and out0 set.
void plan_match_batch(MatchBatch* b, int count, int64_t max_grid) {
    b->count = count;
    int64_t units = 0, g = 0, queries = 0;
    for (int i = 0; i < count; ++i) {
        MatchProblem& P = b->p[i];
        P.mt = (P.nq + kRowsQ - 1) / kRowsQ;
        P.ntl = P.nq > 0 ? (P.nt + kColsB - 1) / kColsB : 0;
        P.unit0 = units;
        P.g0 = static_cast<int32_t>(g);
        units += static_cast<int64_t>(P.mt) * P.ntl;
        g += P.mt;
        queries = P.out0 + P.nq > queries ? P.out0 + P.nq : queries;
    }
    b->units = units;
    b->tiles = static_cast<int32_t>(g);
    b->queries = queries;
    b->grid = units < max_grid ? units : max_grid;
    // whole query tiles per share when there are enough of them to balance the
    // blocks (the block that walks a whole tile writes its matches directly, and a
    // tile's walk pays its start-up -- the first units' top-two updates -- once);
    // not when some problem has queries but no train rows (its tiles have no unit)
    bool whole = g >= kWholeTilesPerBlock * b->grid;
    for (int i = 0; i < count; ++i)
        if (b->p[i].nq > 0 && b->p[i].ntl == 0) whole = false;
    b->whole_tiles = whole ? 1 : 0;
}

// Slots g + c' + p (G - 1) (UnitIter): tiles + count (G - 1) of them.
static size_t partial_record_bytes(const MatchBatch& b) {
    return static_cast<size_t>(b.tiles + static_cast<int64_t>(b.count) * b.grid + 1) * kRowsP * 16;
}

size_t match_tc_partial_bytes(const MatchBatch& b) { return partial_record_bytes(b); }

size_t match_tc_counter_bytes(int64_t tiles) { return align_up(static_cast<size_t>(tiles) * 4, 256); }

// A launch over `problems` problems with `queries` query rows in total has at most
// queries / 128 + problems query tiles and at most `sms` blocks.
size_t match_tc_partial_bound(int64_t queries, int64_t problems, int64_t sms) {
    const int64_t tiles = queries / kRowsQ + problems;
    return static_cast<size_t>(tiles + problems * sms + 1) * kRowsP * 16 + match_tc_counter_bytes(tiles) + 512;
}

size_t match_tc_batch_scratch_bytes(int64_t rows, const MatchBatch& b, int64_t counter_tiles) {
    const size_t exp_bytes = align_up(static_cast<size_t>(rows) * kKBytes, 1024);
    return exp_bytes + match_tc_counter_bytes(counter_tiles) + match_tc_partial_bytes(b) + 256;
}

// The batched layout's arrival counters: [expanded rows][counters][partials].
int32_t* match_tc_batch_counters(void* scratch, int64_t rows) {
    const size_t exp_bytes = align_up(static_cast<size_t>(rows) * kKBytes, 1024);
    return reinterpret_cast<int32_t*>(static_cast<uint8_t*>(scratch) + exp_bytes);
}

// Copies the header and the first b.count problems into the table of capacity NP.
template <int NP>
static void shrink(const MatchBatch& b, MatchBatchT<NP>* o) {
    o->count = b.count;
    o->tiles = b.tiles;
    o->whole_tiles = b.whole_tiles;
    o->units = b.units;
    o->grid = b.grid;
    o->queries = b.queries;
    for (int i = 0; i < b.count; ++i) o->p[i] = b.p[i];
}

template <int NP>
static cudaError_t set_match_attributes() {
    return cudaFuncSetAttribute(match_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

template <int NP>
static cudaError_t launch_match_np(const MatchBatch& full, const CUtensorMap& mapq, const CUtensorMap& mapt,
                                   uint64_t* partials, int32_t* tile_cnt, latch_match* out, uint32_t* flags,
                                   cudaStream_t stream) {
    static unsigned long long attr_done = 0;
    {
        const cudaError_t e = once_per_device(&attr_done, set_match_attributes<NP>);
        if (e != cudaSuccess) return e;
    }
    MatchBatchT<NP>* b = new (std::nothrow) MatchBatchT<NP>;
    if (!b) return cudaErrorMemoryAllocation;
    shrink(full, b);
    cudaError_t e = cudaSuccess;
    if (b->units > 0)
        e = launch_chained(match_tc_kernel<NP>, dim3(static_cast<unsigned>(b->grid)), dim3(kThreads), kSmemBytes,
                           stream, mapq, mapt, *b, partials, tile_cnt, out, flags);
    if (e == cudaSuccess && !tile_cnt && !b->whole_tiles && b->queries > 0) {
        const int threads = 256;
        const int64_t grid = (b->queries + threads - 1) / threads;
        e = launch_chained(match_merge_kernel<NP>, dim3(static_cast<unsigned>(grid)), dim3(threads), 0, stream, *b,
                           partials, out);
    }
    delete b;
    return e;
}

cudaError_t launch_match_tc_rows(const MatchBatch& b, const uint8_t* exp, int64_t rows, uint64_t* partials, int32_t* tile_cnt, latch_match* out, uint32_t* flags,
                                 cudaStream_t stream) {
    if (b.queries == 0) return cudaSuccess;
    CUtensorMap mapq, mapt;
    if (b.units > 0 && !(make_map(&mapq, exp, rows, kRowsA) && make_map(&mapt, exp, rows, kColsB)))
        return cudaErrorInvalidValue;
    // a short launch (at most kFusedUnitsPerBlock units per block) combines each query
    // tile's records itself, which saves the merge launch; a long one leaves them to
    // match_merge_kernel, because the combine at a tile's end (a fence and an atomic
    // round trip per block) holds the epilogue while the MMAs can run only an
    // accumulator's worth ahead.  Neither when some problem has queries but no train
    // rows (its tiles have no unit, so no block visits them).
    bool fused = b.units > 0 && tile_cnt != nullptr && b.units <= kFusedUnitsPerBlock * b.grid;
    for (int i = 0; i < b.count; ++i)
        if (b.p[i].nq > 0 && b.p[i].ntl == 0) fused = false;
    if (!fused) tile_cnt = nullptr;
    if (b.count <= 1) return launch_match_np<1>(b, mapq, mapt, partials, tile_cnt, out, flags, stream);
    if (b.count <= 16) return launch_match_np<16>(b, mapq, mapt, partials, tile_cnt, out, flags, stream);
    return launch_match_np<kMaxProblems>(b, mapq, mapt, partials, tile_cnt, out, flags, stream);
}

// Scratch: expanded rows (rows x kExpRowBytes), arrival counters, partial records.
// The expanded rows must already be filled (launch_expand).
cudaError_t launch_match_tc_batch(const MatchBatch& b, int64_t rows, int64_t counter_tiles, void* scratch,
                                  latch_match* out, uint32_t* flags, cudaStream_t stream) {
    uint8_t* base = static_cast<uint8_t*>(scratch);
    const size_t exp_bytes = align_up(static_cast<size_t>(rows) * kKBytes, 1024);
    const size_t cnt_bytes = match_tc_counter_bytes(counter_tiles);
    return launch_match_tc_rows(b, base, rows, reinterpret_cast<uint64_t*>(base + exp_bytes + cnt_bytes),
                                reinterpret_cast<int32_t*>(base + exp_bytes), out, flags, stream);
}

static void single_problem(MatchBatch* b, int32_t nq, int32_t nt, int64_t sms, int32_t k = 2, int32_t r = 800) {
    b->p[0].k = k;
    b->p[0].r_milli = r;
    b->p[0].q_row0 = 0;
    b->p[0].t_row0 = nq;
    b->p[0].nq = nq;
    b->p[0].nt = nt;
    b->p[0].out0 = 0;
    plan_match_batch(b, 1, sms);
}

size_t match_tc_scratch_bytes_sms(int64_t sms, int64_t nq, int64_t nt) {
    MatchBatch* b = new MatchBatch;
    single_problem(b, static_cast<int32_t>(nq), static_cast<int32_t>(nt), sms);
    const size_t r = match_tc_batch_scratch_bytes(nq + nt, *b, b->tiles);
    delete b;
    return r;
}

size_t match_tc_scratch_bytes(const latch_context* ctx, int64_t nq, int64_t nt) {
    return match_tc_scratch_bytes_sms(ctx->sm_count, nq, nt);
}

cudaError_t launch_match_tc(const latch_context* ctx, const uint8_t* q, int32_t nq, const uint8_t* t, int32_t nt,
                            int32_t k, int32_t r_milli, latch_match* out, void* scratch, cudaStream_t stream) {
    MatchBatch* b = new MatchBatch;
    single_problem(b, nq, nt, ctx->sm_count, k, r_milli);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    cudaError_t e = cudaSuccess;
    if (b->units > 0) {
        // the arrival counters are cleared ahead of the kernels, off their dependency chain
        e = cudaMemsetAsync(match_tc_batch_counters(scratch, nq + nt), 0, match_tc_counter_bytes(b->tiles), stream);
        if (e == cudaSuccess) e = launch_expand(q, nq, base, stream);
        if (e == cudaSuccess) e = launch_expand(t, nt, base + static_cast<size_t>(nq) * kKBytes, stream);
    }
    if (e == cudaSuccess) e = launch_match_tc_batch(*b, nq + nt, b->tiles, scratch, out, ctx->d_flags, stream);
    delete b;
    return e;
}

}  // namespace latch

// ---------------------------------------------------------------------------
// Allocation-free variant of the tensor-core matcher.
//
// Some callers may not allocate device memory at all: a library embedded in a host
// application that owns every byte of HBM through its own pool (so a cudaMalloc
// from us could fail, or steal memory the application has budgeted), or a
// latency-bound pipeline where cudaMalloc/cudaFree would synchronise the device and
// stall the application's other streams.  hamming_match_noalloc serves them: its
// scratch (expanded operands, per-block partial results, status word)
// lives in the fixed array below, which the CUDA module reserves on every device
// that loads this library for as long as the process lives.
// ---------------------------------------------------------------------------

namespace latch {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr size_t kStaticFlagBytes = 256;  // status word: zero at load, raised by the kernels, cleared when read

}  // namespace latch

static __device__ __align__(256) uint8_t g_match_static_scratch[latch::kStaticScratchBytes];

#include <mutex>

namespace latch {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_match_static_scratch on `dev` (which must be current).  The
// symbol's host-side name is only a stand-in, so its address is looked up once per
// device and cached.
latch_status static_scratch(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, LATCH_EUNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_match_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(nullptr, LATCH_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return LATCH_OK;
}

}  // namespace
}  // namespace latch

extern "C" latch_status hamming_match_noalloc(const uint8_t* d_query, int32_t nq, const uint8_t* d_train,
                                              int32_t nt, int32_t k, float ratio, latch_match* d_out,
                                              latch_stream_t stream) {
    using namespace latch;
    if (nq < 0 || nt < 0) return fail(nullptr, LATCH_EINVAL, "negative size");
    if (k != 1 && k != 2) return fail(nullptr, LATCH_EINVAL, "k = %d must be 1 or 2", k);
    if (!(ratio >= 0.0f && ratio <= 1.0f)) return fail(nullptr, LATCH_EINVAL, "ratio %g not in [0, 1]", ratio);
    if (nq > 0 && (!d_query || !d_out)) return fail(nullptr, LATCH_EINVAL, "NULL query or output");
    if (nq > 0 && nt > 0 && !d_train) return fail(nullptr, LATCH_EINVAL, "NULL train");
    if ((reinterpret_cast<uintptr_t>(d_query) | reinterpret_cast<uintptr_t>(d_train) |
         reinterpret_cast<uintptr_t>(d_out)) & 15)
        return fail(nullptr, LATCH_EINVAL, "descriptor and output pointers must be 16-byte aligned");
    if (nq == 0) return LATCH_OK;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "device query: %s", cudaGetErrorString(e));
    const size_t need = match_tc_scratch_bytes_sms(sms, nq, nt) + kStaticFlagBytes;
    if (need > kStaticScratchBytes)
        return fail(nullptr, LATCH_EINVAL,
                    "nq = %d, nt = %d needs %zu bytes of scratch; the static scratch holds %zu (about 60,000 "
                    "descriptors in total)",
                    nq, nt, need, kStaticScratchBytes);
    void* base = nullptr;
    latch_status st = static_scratch(dev, &base);
    if (st != LATCH_OK) return st;
    uint8_t* bytes = static_cast<uint8_t*>(base);
    uint32_t* flags = reinterpret_cast<uint32_t*>(bytes);  // sticky until hamming_match_noalloc_status reads it
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // launch_match_tc reads only the SM count and the status-word pointer of its context
    latch_context shim;
    shim.device = dev;
    shim.sm_count = sms;
    shim.d_flags = flags;
    const int32_t r_milli = static_cast<int32_t>(std::round(static_cast<double>(ratio) * 1000.0));
    e = launch_match_tc(&shim, d_query, nq, d_train, nt, k, r_milli, d_out, bytes + kStaticFlagBytes, cs);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "tensor match launch: %s", cudaGetErrorString(e));
    return LATCH_OK;
}

extern "C" latch_status hamming_match_noalloc_status(void) {
    using namespace latch;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    void* base = nullptr;
    latch_status st = static_scratch(dev, &base);
    if (st != LATCH_OK) return st;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "earlier work failed: %s", cudaGetErrorString(e));
    uint32_t word = 0;
    e = cudaMemcpy(&word, base, sizeof(word), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && word) e = cudaMemset(base, 0, sizeof(word));
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "status word: %s", cudaGetErrorString(e));
    if (word & kFlagTimeout)
        return fail(nullptr, LATCH_ETIMEOUT, "a device-side wait of hamming_match_noalloc gave up (word 0x%x)", word);
    if (word) return fail(nullptr, LATCH_EDEVICE, "hamming_match_noalloc status word 0x%x", word);
    return LATCH_OK;
}

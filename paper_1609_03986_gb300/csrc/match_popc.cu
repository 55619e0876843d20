// Brute-force Hamming matching on the CUDA cores (Sec. 4): XOR + population count.
//
// The grid is (query blocks) x (train slices).  Each thread owns two query
// descriptors (32 words in registers); a block streams its slice of the train set
// through shared memory in double-buffered tiles (cp.async) and every thread computes
// the exact Hamming distance of its queries to every train descriptor of the slice.
// Half of the 16 XOR words of a pair are folded by a carry-save adder tree into words
// of weight 1, 2, 4 and 8 (4 population counts for 8), the other half are counted
// directly, which balances the logic pipe against the population-count pipe.  Keys are
// (distance << 21 | index in the slice), unique within a slice, so min / second-min
// is the top-2 with ties to the lowest index.  With one slice the block writes the
// matches; otherwise it writes its two best (distance << 32 | train index) keys per
// query and match_popc_merge_kernel combines the slices.
#include <cstdint>

#include "internal.h"
#include "popc.cuh"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kTile = 256;                          // train descriptors per shared-memory tile (16 KB)
constexpr int kSliceBits = 21;                      // slice-local index bits of a key
constexpr uint32_t kNone32 = 0xffffffffu;
constexpr uint64_t kNone64 = ~0ull;

__device__ __forceinline__ void top2_insert32(uint32_t key, uint32_t& m1, uint32_t& m2) {
    const uint32_t hi = max(key, m1);
    m1 = min(key, m1);
    m2 = min(hi, m2);
}

__device__ __forceinline__ void top2_insert64(uint64_t key, uint64_t& m1, uint64_t& m2) {
    const uint64_t hi = key > m1 ? key : m1;
    m1 = key < m1 ? key : m1;
    m2 = hi < m2 ? hi : m2;
}

__device__ __forceinline__ void write_match(latch_match* out, uint64_t m1, uint64_t m2, int k, int r_milli) {
    latch_match m;
    m.idx1 = m1 == kNone64 ? -1 : static_cast<int32_t>(m1 & 0xffffffffu);
    m.dist1 = m1 == kNone64 ? 0xffff : static_cast<uint16_t>(m1 >> 32);
    const bool has2 = (k == 2) && m2 != kNone64;
    m.idx2 = has2 ? static_cast<int32_t>(m2 & 0xffffffffu) : -1;
    m.dist2 = has2 ? static_cast<uint16_t>(m2 >> 32) : 0xffff;
    if (m1 == kNone64)
        m.accepted = 0;
    else if (k == 1)
        m.accepted = 1;
    else
        m.accepted = (1000ll * m.dist1 < static_cast<long long>(r_milli) * m.dist2) ? 1 : 0;
    m.pad[0] = m.pad[1] = m.pad[2] = 0;
    *out = m;
}

// slice-local 32-bit key -> (distance << 32 | train index)
__device__ __forceinline__ uint64_t widen(uint32_t key, int64_t slice0) {
    if (key == kNone32) return kNone64;
    return (static_cast<uint64_t>(key >> kSliceBits) << 32) |
           static_cast<uint64_t>(slice0 + (key & ((1u << kSliceBits) - 1)));
}

// Tile `ti` of the slice [t0, t1) into shared buffer `buf` (16-byte asynchronous
// copies, committed as one group per thread).
template <int kThreads>
__device__ __forceinline__ void load_tile(uint4* buf, const uint4* __restrict__ t, int64_t t0, int64_t t1, int ti) {
    const int64_t first = t0 + static_cast<int64_t>(ti) * kTile;
    const int cnt = static_cast<int>(t1 - first < kTile ? t1 - first : kTile);
    for (int i = threadIdx.x; i < cnt * 4; i += kThreads) cp_async_16(&buf[i], &t[first * 4 + i]);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// kThreads threads x kQPerThread queries per block; two train descriptors per step,
// so each thread has 2 kQPerThread independent adder trees in flight.
template <int kThreads, int kQPerThread>
__global__ void __launch_bounds__(kThreads) match_popc_kernel(const uint4* __restrict__ q, int nq,
                                                              const uint4* __restrict__ t, int nt, int k,
                                                              int r_milli, int slices, latch_match* __restrict__ out,
                                                              uint4* __restrict__ partial) {
    constexpr int kQPerBlock = kThreads * kQPerThread;
    __shared__ uint4 s_t[2][kTile * 4];
    const int s = blockIdx.y;
    const int64_t t0 = static_cast<int64_t>(s) * nt / slices, t1 = static_cast<int64_t>(s + 1) * nt / slices;
    uint32_t qw[kQPerThread][16];
#pragma unroll
    for (int a = 0; a < kQPerThread; ++a) {
        const int qi = blockIdx.x * kQPerBlock + a * kThreads + threadIdx.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint4 v = qi < nq ? q[static_cast<size_t>(qi) * 4 + j] : make_uint4(0, 0, 0, 0);
            qw[a][4 * j + 0] = v.x;
            qw[a][4 * j + 1] = v.y;
            qw[a][4 * j + 2] = v.z;
            qw[a][4 * j + 3] = v.w;
        }
    }
    uint32_t m1[kQPerThread], m2[kQPerThread];
#pragma unroll
    for (int a = 0; a < kQPerThread; ++a) m1[a] = m2[a] = kNone32;
    const int tiles = static_cast<int>((t1 - t0 + kTile - 1) / kTile);
    if (tiles > 0) load_tile<kThreads>(s_t[0], t, t0, t1, 0);
    for (int ti = 0; ti < tiles; ++ti) {
        const int buf = ti & 1;
        // the next tile streams in while this one is scanned
        if (ti + 1 < tiles) load_tile<kThreads>(s_t[buf ^ 1], t, t0, t1, ti + 1);
        if (ti + 1 < tiles)
            asm volatile("cp.async.wait_group 1;" ::: "memory");  // tile ti's group is complete
        else
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const int64_t first = static_cast<int64_t>(ti) * kTile;  // slice-local index of the tile's first row
        const int cnt = static_cast<int>(t1 - t0 - first < kTile ? t1 - t0 - first : kTile);
        for (int j = 0; j < cnt; j += 2) {
            // rows j and j + 1 (at an odd end the first row stands in for the missing
            // second and its repeated key is not inserted)
            const int j2 = j + 1 < cnt ? j + 1 : j;
            uint32_t tw[2][16];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint4 v = s_t[buf][j * 4 + w], u = s_t[buf][j2 * 4 + w];
                tw[0][4 * w + 0] = v.x;
                tw[0][4 * w + 1] = v.y;
                tw[0][4 * w + 2] = v.z;
                tw[0][4 * w + 3] = v.w;
                tw[1][4 * w + 0] = u.x;
                tw[1][4 * w + 1] = u.y;
                tw[1][4 * w + 2] = u.z;
                tw[1][4 * w + 3] = u.w;
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t idx = static_cast<uint32_t>(first + (r == 0 ? j : j2));
#pragma unroll
                for (int a = 0; a < kQPerThread; ++a) {
                    uint32_t x[16];
#pragma unroll
                    for (int w = 0; w < 16; ++w) x[w] = qw[a][w] ^ tw[r][w];
                    const uint32_t key = (static_cast<uint32_t>(popc16(x)) << kSliceBits) | idx;
                    if (r == 0 || j2 != j) top2_insert32(key, m1[a], m2[a]);
                }
            }
        }
        __syncthreads();  // the buffer is refilled two tiles later
    }
#pragma unroll
    for (int a = 0; a < kQPerThread; ++a) {
        const int qi = blockIdx.x * kQPerBlock + a * kThreads + threadIdx.x;
        if (qi >= nq) continue;
        const uint64_t w1 = widen(m1[a], t0), w2 = widen(m2[a], t0);
        if (slices == 1) {
            write_match(out + qi, w1, w2, k, r_milli);
        } else {
            uint64_t* p = reinterpret_cast<uint64_t*>(partial + static_cast<size_t>(qi) * slices + s);
            p[0] = w1;
            p[1] = w2;
        }
    }
}

// Combines the slices' two best keys of every query.
__global__ void match_popc_merge_kernel(const uint4* __restrict__ partial, int nq, int slices, int k, int r_milli,
                                        latch_match* __restrict__ out) {
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    uint64_t m1 = kNone64, m2 = kNone64;
    const uint64_t* p = reinterpret_cast<const uint64_t*>(partial + static_cast<size_t>(qi) * slices);
    for (int s = 0; s < slices; ++s) {
        top2_insert64(p[2 * s], m1, m2);
        top2_insert64(p[2 * s + 1], m1, m2);
    }
    write_match(out + qi, m1, m2, k, r_milli);
}

// Block shape: 512 queries per block (256 threads x 2) where that still gives two
// blocks per SM, else 128 (128 threads x 1) for more blocks on small shapes.
int popc_queries_per_block(const latch_context* ctx, int64_t nq, int64_t nt) {
    const int64_t max_slices = nt > 0 ? (nt + kTile - 1) / kTile : 1;
    return ((nq + 511) / 512) * max_slices >= 2 * static_cast<int64_t>(ctx->sm_count) ? 512 : 128;
}

// Train slices: enough blocks for about six per SM, slices of at least one tile, and
// every slice below 2^21 rows (the key's index field).
int popc_slices(const latch_context* ctx, int64_t nq, int64_t nt) {
    if (nt <= 0) return 1;
    const int64_t qpb = popc_queries_per_block(ctx, nq, nt);
    const int64_t qblocks = (nq + qpb - 1) / qpb;
    const int64_t want = (6 * static_cast<int64_t>(ctx->sm_count) + qblocks - 1) / qblocks;
    const int64_t most = (nt + kTile - 1) / kTile;
    const int64_t least = (nt + (int64_t(1) << kSliceBits) - 1) >> kSliceBits;
    int64_t s = want < most ? want : most;
    if (s < least) s = least;
    if (s < 1) s = 1;
    return static_cast<int>(s);
}

}  // namespace

size_t match_popc_scratch_bytes(const latch_context* ctx, int64_t nq, int64_t nt) {
    const int s = popc_slices(ctx, nq, nt);
    return s > 1 ? static_cast<size_t>(nq) * s * 16 : 0;
}

cudaError_t launch_match_popc(const latch_context* ctx, const uint8_t* q, int32_t nq, const uint8_t* t, int32_t nt,
                              int32_t k, int32_t r_milli, latch_match* out, void* scratch, cudaStream_t stream) {
    const int slices = popc_slices(ctx, nq, nt);
    const int qpb = popc_queries_per_block(ctx, nq, nt);
    const dim3 grid(static_cast<unsigned>((nq + qpb - 1) / qpb), static_cast<unsigned>(slices));
    uint4* partial = static_cast<uint4*>(scratch);
    const uint4* qv = reinterpret_cast<const uint4*>(q);
    const uint4* tv = reinterpret_cast<const uint4*>(t);
    if (qpb == 512)
        match_popc_kernel<256, 2><<<grid, 256, 0, stream>>>(qv, nq, tv, nt, k, r_milli, slices, out, partial);
    else
        match_popc_kernel<128, 1><<<grid, 128, 0, stream>>>(qv, nq, tv, nt, k, r_milli, slices, out, partial);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && slices > 1) {
        match_popc_merge_kernel<<<(nq + 255) / 256, 256, 0, stream>>>(partial, nq, slices, k, r_milli, out);
        note_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace latch

// Brute-force Hamming matching on the CUDA cores (Sec. 4): XOR + population count.
//
// Each thread owns one query descriptor (16 words in registers); the block streams
// the train set through shared memory in tiles and every thread computes the exact
// Hamming distance to every train descriptor, keeping its two smallest keys
// (distance << 32 | index).  Keys are unique, so min/second-min over them is the
// top-2 with ties resolved to the lowest train index.
#include <cstdint>

#include "internal.h"

namespace latch {

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 256;  // train descriptors per shared-memory tile (16 KB)

__device__ __forceinline__ void top2_insert(uint64_t key, uint64_t& m1, uint64_t& m2) {
    const uint64_t hi = key > m1 ? key : m1;
    m1 = key < m1 ? key : m1;
    m2 = hi < m2 ? hi : m2;
}

__device__ __forceinline__ void write_match(latch_match* out, uint64_t m1, uint64_t m2, int k, int r_milli) {
    const uint64_t kNone = ~0ull;
    latch_match m;
    m.idx1 = m1 == kNone ? -1 : static_cast<int32_t>(m1 & 0xffffffffu);
    m.dist1 = m1 == kNone ? 0xffff : static_cast<uint16_t>(m1 >> 32);
    const bool has2 = (k == 2) && m2 != kNone;
    m.idx2 = has2 ? static_cast<int32_t>(m2 & 0xffffffffu) : -1;
    m.dist2 = has2 ? static_cast<uint16_t>(m2 >> 32) : 0xffff;
    if (m1 == kNone)
        m.accepted = 0;
    else if (k == 1)
        m.accepted = 1;
    else
        m.accepted = (1000ll * m.dist1 < static_cast<long long>(r_milli) * m.dist2) ? 1 : 0;
    m.pad[0] = m.pad[1] = m.pad[2] = 0;
    *out = m;
}

__global__ void __launch_bounds__(kThreads) match_popc_kernel(const uint4* __restrict__ q, int nq,
                                                              const uint4* __restrict__ t, int nt, int k,
                                                              int r_milli, latch_match* __restrict__ out) {
    __shared__ uint4 s_t[kTile * 4];
    const int qi = blockIdx.x * kThreads + threadIdx.x;
    uint32_t qw[16];
    if (qi < nq) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint4 v = q[static_cast<size_t>(qi) * 4 + j];
            qw[4 * j + 0] = v.x;
            qw[4 * j + 1] = v.y;
            qw[4 * j + 2] = v.z;
            qw[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) qw[j] = 0;
    }
    uint64_t m1 = ~0ull, m2 = ~0ull;
    for (int base = 0; base < nt; base += kTile) {
        const int cnt = nt - base < kTile ? nt - base : kTile;
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * 4; i += kThreads) s_t[i] = t[static_cast<size_t>(base) * 4 + i];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            int d = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint4 v = s_t[j * 4 + w];
                d += __popc(qw[4 * w + 0] ^ v.x) + __popc(qw[4 * w + 1] ^ v.y) + __popc(qw[4 * w + 2] ^ v.z) +
                     __popc(qw[4 * w + 3] ^ v.w);
            }
            top2_insert((static_cast<uint64_t>(d) << 32) | static_cast<uint32_t>(base + j), m1, m2);
        }
    }
    if (qi < nq) write_match(out + qi, m1, m2, k, r_milli);
}

}  // namespace

size_t match_popc_scratch_bytes(const latch_context*, int64_t, int64_t) { return 0; }

cudaError_t launch_match_popc(const latch_context*, const uint8_t* q, int32_t nq, const uint8_t* t, int32_t nt,
                              int32_t k, int32_t r_milli, latch_match* out, void*, cudaStream_t stream) {
    const int grid = (nq + kThreads - 1) / kThreads;
    match_popc_kernel<<<grid, kThreads, 0, stream>>>(reinterpret_cast<const uint4*>(q), nq,
                                                     reinterpret_cast<const uint4*>(t), nt, k, r_milli, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace latch

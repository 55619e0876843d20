// Brute-force Hamming matching on the 5th-generation tensor cores (Sec. 4's
// all-pairs distance computation, done as a dense contraction).
//
// With every descriptor bit expanded to an 8-bit float that is exactly 0 or 1
// (E4M3 0x00 / 0x38), the dot product of two expanded descriptors counts their
// common 1-bits, and Hamming(q, t) = popc(q) + popc(t) - 2 * dot(q, t).  Products
// are 0/1 and sums are at most 512, so fp32 accumulation is exact.
//
// Per block (one per SM, persistent over a contiguous range of (query tile, train
// tile) units; see match_common.cuh):
//   warp 0     TMA producer: a 256-query tile (two 128-row A operands, 128 KB,
//              resident while the block stays on that query tile) and 128-row x
//              128-byte train chunks into a 4-stage ring (16 KB each), 128-byte
//              swizzle;
//   warp 1     MMA issuer: for each 256 x 128 unit, 2 x 16 tcgen05.mma (M=128,
//              N=128, K=32) into one of two double-buffered TMEM accumulators;
//   warp 2     TMEM allocator (all 512 columns);
//   warps 4-7  epilogue: tcgen05.ld of the fp32 dot products, key =
//              ((popc(t) - 2*dot + 512) << 8 | column) formed exactly in fp32 by
//              one FMA, running min / second-min with FMNMX, then the two best of
//              the tile are merged into the row's (distance << 32 | index) keys.
// All mbarrier waits are bounded (sm103.h); on a timeout the block raises the
// context's device flag, drains and frees TMEM.
#include <cuda.h>

#include <cmath>

#include "match_common.cuh"
#include "sm103.h"

namespace latch {

namespace {

using namespace sm103;

constexpr int kRowsA = 128;             // rows per MMA (M)
constexpr int kSubA = 2;                // A operands per query tile
constexpr int kRowsQ = kRowsA * kSubA;  // queries per tile: 256
constexpr int kColsB = 128;             // train rows per unit (N)
constexpr int kKBytes = 512;            // expanded descriptor: 512 x 8-bit
constexpr int kChunk = 128;             // K bytes per swizzle atom / TMA box
constexpr int kChunks = kKBytes / kChunk;
constexpr int kStages = 4;
constexpr int kTileBytes = kRowsA * kChunk;  // 16 KB
constexpr int kThreads = 256;
constexpr int kTmemCols = 512;
constexpr uint32_t kIdesc = idesc_e4m3_f32(kRowsA, kColsB);

// AND of `v` over the 128 epilogue threads (named barrier 1).
__device__ __forceinline__ bool group_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v))
        : "memory");
    return r != 0;
}

struct Smem {
    // offsets in the 1024-aligned dynamic buffer
    static constexpr int a = 0;                                        // [kSubA][kChunks] tiles
    static constexpr int b = a + kSubA * kChunks * kTileBytes;         // [kStages] tiles
    static constexpr int cvec = b + kStages * kTileBytes;              // float [2][kColsB]
    static constexpr int bars = cvec + 2 * kColsB * 4;                 // uint64 barriers
    static constexpr int nbars = 2 * kStages + 2 + 4 + 1;
    static constexpr int misc = bars + nbars * 8;                      // tmem base, abort flag
    static constexpr int total = misc + 16;
};
constexpr int kSmemBytes = Smem::total + 1024;

__global__ void __launch_bounds__(kThreads, 1) match_tc_kernel(const __grid_constant__ CUtensorMap tm_q,
                                                              const __grid_constant__ CUtensorMap tm_t,
                                                              const int32_t* __restrict__ pop_q,
                                                              const int32_t* __restrict__ pop_t, int nq, int nt,
                                                              WorkSplit split, uint64_t* __restrict__ partials,
                                                              uint32_t* __restrict__ flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem + Smem::a;
    uint8_t* sB = smem + Smem::b;
    float* sC = reinterpret_cast<float*>(smem + Smem::cvec);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Smem::bars);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* a_full = bars + 2 * kStages;
    uint64_t* a_empty = a_full + 1;
    uint64_t* acc_full = a_full + 2;
    uint64_t* acc_empty = a_full + 4;
    uint64_t* mma_done = a_full + 6;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Smem::misc);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + Smem::misc + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t c = blockIdx.x;
    const int64_t u0 = split_start(c, split.units, split.grid);
    const int64_t u1 = split_start(c + 1, split.units, split.grid);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4);
        }
        mbar_init(mma_done, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(&tm_q);
        prefetch_tmap(&tm_t);
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, kTmemCols);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t ring = 0, a_par = 0;
            uint32_t fill_par[kStages];
            bool filled[kStages];
            for (int s = 0; s < kStages; ++s) filled[s] = false, fill_par[s] = 0;
            int64_t prev_m = -1;
            for (int64_t u = u0; u < u1; ++u) {
                const int64_t m = u / split.nt, n = u % split.nt;
                if (m != prev_m) {
                    if (prev_m >= 0) {
                        if (!mbar_wait(a_empty, a_par, abort)) break;
                        a_par ^= 1;
                    }
                    mbar_arrive_expect_tx(a_full, kSubA * kChunks * kTileBytes);
                    for (int a = 0; a < kSubA; ++a)
                        for (int kc = 0; kc < kChunks; ++kc)
                            tma_load_2d(sA + (a * kChunks + kc) * kTileBytes, &tm_q, kc * kChunk,
                                        static_cast<int32_t>(m * kRowsQ + a * kRowsA), a_full);
                    prev_m = m;
                }
                bool ok = true;
                for (int kc = 0; kc < kChunks; ++kc) {
                    if (!mbar_wait(&empty[stage], ring ^ 1, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], kTileBytes);
                    tma_load_2d(sB + stage * kTileBytes, &tm_t, kc * kChunk, static_cast<int32_t>(n * kColsB),
                                &full[stage]);
                    filled[stage] = true;
                    fill_par[stage] = ring;
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
                    while (filled[s] && !mbar_try_wait(&full[s], fill_par[s]) && globaltimer() - t0 < 200000000ull) {
                    }
                if (prev_m >= 0)  // the last A load completes the a_full phase of parity a_par
                    while (!mbar_try_wait(a_full, a_par) && globaltimer() - t0 < 200000000ull) {
                    }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t ring = 0, a_par = 0;
            uint32_t acc_par[2] = {0, 0};
            int64_t prev_m = -1;
            int i = 0;
            for (int64_t u = u0; u < u1 && !*abort; ++u, ++i) {
                const int64_t m = u / split.nt;
                const int buf = i & 1;
                if (m != prev_m) {
                    if (!mbar_wait(a_full, a_par, abort)) break;
                    a_par ^= 1;
                    prev_m = m;
                }
                if (!mbar_wait(&acc_empty[buf], acc_par[buf] ^ 1, abort)) break;
                acc_par[buf] ^= 1;
                tc_fence_after();
                bool ok = true;
                for (int kc = 0; kc < kChunks; ++kc) {
                    if (!mbar_wait(&full[stage], ring, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t b_addr = smem_u32(sB + stage * kTileBytes);
#pragma unroll
                    for (int a = 0; a < kSubA; ++a) {
                        const uint32_t a_addr = smem_u32(sA + (a * kChunks + kc) * kTileBytes);
                        const uint32_t d = tmem + static_cast<uint32_t>((a * 2 + buf) * kColsB);
#pragma unroll
                        for (int ks = 0; ks < kChunk / 32; ++ks)
                            mma_f8f6f4(d, umma_desc_sw128(a_addr + ks * 32), umma_desc_sw128(b_addr + ks * 32), kIdesc,
                                       (kc | ks) != 0);
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == kStages) {
                        stage = 0;
                        ring ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&acc_full[buf]);
                const int64_t next_m = (u + 1 < u1) ? (u + 1) / split.nt : -1;
                if (next_m != m) mma_commit(a_empty);
            }
            // every issued MMA has finished before TMEM is released
            mma_commit(mma_done);
            const uint64_t t0 = globaltimer();
            while (!mbar_try_wait(mma_done, 0) && globaltimer() - t0 < 200000000ull) {
            }
        }
    } else if (warp >= 4) {
        // ---------------- epilogue ----------------
        const int et = threadIdx.x - 128;  // 0..127: TMEM lane / column index
        const int quarter = warp & 3;
        uint32_t acc_par[2] = {0, 0};
        uint64_t k1[kSubA], k2[kSubA];
        int32_t pq[kSubA];
        int64_t prev_m = -1;
        int i = 0;
        for (int64_t u = u0; u < u1; ++u, ++i) {
            const int64_t m = u / split.nt, n = u % split.nt;
            const int buf = i & 1;
            if (m != prev_m) {
#pragma unroll
                for (int a = 0; a < kSubA; ++a) {
                    const int64_t row = m * kRowsQ + a * kRowsA + quarter * 32 + lane;
                    pq[a] = row < nq ? pop_q[row] : 0;
                    k1[a] = k2[a] = kNoKey;
                }
                prev_m = m;
            }
            {
                const int64_t col = n * kColsB + et;
                sC[buf * kColsB + et] =
                    col < nt ? static_cast<float>((pop_t[col] + 512) * 256 + et) : __int_as_float(0x7f800000);
            }
            // one vote of the 128 epilogue threads: also publishes sC; exits are group-uniform
            if (!group_all(mbar_wait(&acc_full[buf], acc_par[buf], abort))) break;
            acc_par[buf] ^= 1;
            tc_fence_after();
            const float* cv = sC + buf * kColsB;
#pragma unroll
            for (int a = 0; a < kSubA; ++a) {
                float m1 = __int_as_float(0x7f800000), m2 = m1;
                const uint32_t base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                                      static_cast<uint32_t>((a * 2 + buf) * kColsB);
#pragma unroll 1
                for (int ch = 0; ch < kColsB / 32; ++ch) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(base + ch * 32, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 cc = *reinterpret_cast<const float4*>(cv + ch * 32 + j);
                        const float e0 = fmaf(__uint_as_float(v[j + 0]), -512.0f, cc.x);
                        const float e1 = fmaf(__uint_as_float(v[j + 1]), -512.0f, cc.y);
                        const float e2 = fmaf(__uint_as_float(v[j + 2]), -512.0f, cc.z);
                        const float e3 = fmaf(__uint_as_float(v[j + 3]), -512.0f, cc.w);
                        float h;
                        h = fmaxf(m1, e0); m1 = fminf(m1, e0); m2 = fminf(m2, h);
                        h = fmaxf(m1, e1); m1 = fminf(m1, e1); m2 = fminf(m2, h);
                        h = fmaxf(m1, e2); m1 = fminf(m1, e2); m2 = fminf(m2, h);
                        h = fmaxf(m1, e3); m1 = fminf(m1, e3); m2 = fminf(m2, h);
                    }
                }
                // the tile's two best (exact integers below 2^19) -> global keys
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const float mk = b == 0 ? m1 : m2;
                    if (mk < 1.0e30f) {
                        const uint32_t kk = static_cast<uint32_t>(mk);
                        const int32_t d = pq[a] + static_cast<int32_t>(kk >> 8) - 512;
                        const uint64_t idx = static_cast<uint64_t>(n * kColsB + (kk & 255u));
                        top2_insert_u64((static_cast<uint64_t>(d) << 32) | idx, k1[a], k2[a]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            const int64_t next_m = (u + 1 < u1) ? (u + 1) / split.nt : -1;
            if (next_m != m) {
#pragma unroll
                for (int a = 0; a < kSubA; ++a) {
                    uint64_t* p = partial_ptr(partials, split, m, c, a * kRowsA + quarter * 32 + lane);
                    p[0] = k1[a];
                    p[1] = k2[a];
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

// Bits -> E4M3 0/1 bytes (bit t of a descriptor -> byte t) and per-descriptor popcount.
__global__ void expand_kernel(const uint32_t* __restrict__ in, int64_t nwords, uint4* __restrict__ out,
                              int32_t* __restrict__ pop) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint32_t w = i < nwords ? in[i] : 0u;
    uint32_t o[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t nib = (w >> (4 * b)) & 15u;
        o[b] = ((nib * 0x00204081u) & 0x01010101u) * 0x38u;  // E4M3 1.0 = 0x38
    }
    if (i < nwords) {
        out[2 * i] = make_uint4(o[0], o[1], o[2], o[3]);
        out[2 * i + 1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
    int p = __popc(w);
    p += __shfl_xor_sync(0xffffffffu, p, 8);
    p += __shfl_xor_sync(0xffffffffu, p, 4);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    if ((i & 15) == 0 && i < nwords) pop[i >> 4] = p;
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

bool make_map(CUtensorMap* map, const void* base, int64_t rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kKBytes), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kKBytes)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kChunk), static_cast<cuuint32_t>(kRowsA)};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcLayout {
    size_t exp_q, exp_t, pop_q, pop_t, part, total;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

TcLayout tc_layout(const WorkSplit& s, int64_t nq, int64_t nt) {
    TcLayout l;
    l.exp_q = 0;
    l.exp_t = align_up(l.exp_q + static_cast<size_t>(nq) * kKBytes, 1024);
    l.pop_q = align_up(l.exp_t + static_cast<size_t>(nt) * kKBytes, 1024);
    l.pop_t = align_up(l.pop_q + static_cast<size_t>(nq) * 4, 256);
    l.part = align_up(l.pop_t + static_cast<size_t>(nt) * 4, 256);
    l.total = align_up(l.part + static_cast<size_t>(s.mt * s.slots * s.rows) * 16, 256);
    return l;
}

cudaError_t launch_expand(const uint8_t* desc, int64_t n, uint8_t* out, int32_t* pop, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t nwords = n * 16;
    const int threads = 256;
    const int64_t grid = (nwords + threads - 1) / threads;
    expand_kernel<<<static_cast<unsigned>(grid), threads, 0, stream>>>(reinterpret_cast<const uint32_t*>(desc), nwords,
                                                                      reinterpret_cast<uint4*>(out), pop);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

size_t match_tc_scratch_bytes(const latch_context* ctx, int64_t nq, int64_t nt) {
    const WorkSplit s = make_split(nq, nt, kRowsQ, kColsB, ctx->sm_count);
    return tc_layout(s, nq, nt).total;
}

cudaError_t launch_match_tc(const latch_context* ctx, const uint8_t* q, int32_t nq, const uint8_t* t, int32_t nt,
                            int32_t k, int32_t r_milli, latch_match* out, void* scratch, cudaStream_t stream) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(match_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const WorkSplit s = make_split(nq, nt, kRowsQ, kColsB, ctx->sm_count);
    const TcLayout l = tc_layout(s, nq, nt);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    uint64_t* partials = reinterpret_cast<uint64_t*>(base + l.part);
    if (s.units > 0) {
        int32_t* pq = reinterpret_cast<int32_t*>(base + l.pop_q);
        int32_t* pt = reinterpret_cast<int32_t*>(base + l.pop_t);
        cudaError_t e = launch_expand(q, nq, base + l.exp_q, pq, stream);
        if (e == cudaSuccess) e = launch_expand(t, nt, base + l.exp_t, pt, stream);
        if (e != cudaSuccess) return e;
        CUtensorMap mq, mt;
        if (!make_map(&mq, base + l.exp_q, nq) || !make_map(&mt, base + l.exp_t, nt)) return cudaErrorInvalidValue;
        match_tc_kernel<<<static_cast<unsigned>(s.grid), kThreads, kSmemBytes, stream>>>(mq, mt, pq, pt, nq, nt, s,
                                                                                          partials, ctx->d_flags);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_match_merge(partials, s, nq, k, r_milli, out, stream);
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
// scratch (expanded operands, popcounts, per-block partial results, status word)
// lives in the fixed array below, which the CUDA module reserves on every device
// that loads this library for as long as the process lives.
// ---------------------------------------------------------------------------

namespace latch {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr size_t kStaticFlagBytes = 256;                  // status word, cleared every call

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
    const WorkSplit s = make_split(nq, nt, kRowsQ, kColsB, sms);
    const size_t need = tc_layout(s, nq, nt).total + kStaticFlagBytes;
    if (need > kStaticScratchBytes)
        return fail(nullptr, LATCH_EINVAL,
                    "nq = %d, nt = %d needs %zu bytes of scratch; the static scratch holds %zu (about 30,000 "
                    "descriptors in total)",
                    nq, nt, need, kStaticScratchBytes);
    void* base = nullptr;
    latch_status st = static_scratch(dev, &base);
    if (st != LATCH_OK) return st;
    uint8_t* bytes = static_cast<uint8_t*>(base);
    uint32_t* flags = reinterpret_cast<uint32_t*>(bytes);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(flags, 0, sizeof(uint32_t), cs);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "clear status word: %s", cudaGetErrorString(e));
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

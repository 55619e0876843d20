// Final step of matching: combine the per-block top-2 partial keys of every query
// and apply the ratio test (Sec. 4; readings in latch.h).
#include "match_common.cuh"

namespace latch {

namespace {

__global__ void match_merge_kernel(const uint64_t* __restrict__ partials, WorkSplit s, int nq, int k, int r_milli,
                                   latch_match* __restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    uint64_t k1 = kNoKey, k2 = kNoKey;
    if (s.units > 0) {
        const int64_t m = q / s.rows;
        const int r = q % s.rows;
        const int64_t lo = split_owner(m * s.nt, s.units, s.grid);
        const int64_t hi = split_owner((m + 1) * s.nt - 1, s.units, s.grid);
        for (int64_t c = lo; c <= hi; ++c) {
            const uint64_t* p = partials + ((m * s.slots + (c - lo)) * s.rows + r) * 2;
            top2_insert_u64(p[0], k1, k2);
            top2_insert_u64(p[1], k1, k2);
        }
    }
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
    out[q] = mres;
}

}  // namespace

cudaError_t launch_match_merge(const uint64_t* partials, const WorkSplit& s, int32_t nq, int32_t k, int32_t r_milli,
                               latch_match* out, cudaStream_t stream) {
    const int threads = 256;
    const int grid = (nq + threads - 1) / threads;
    match_merge_kernel<<<grid, threads, 0, stream>>>(partials, s, nq, k, r_milli, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace latch

// Work split and top-2 merge shared by the matching kernels.
//
// The (query tile, train tile) grid of a matching call is linearised query-tile
// major, u = m * NT + n, and split into G contiguous ranges, range c = [start(c),
// start(c+1)) with start(c) = floor(c * U / G).  Every block writes, for each query
// tile it touched, the two smallest keys of each query row over its train tiles
// ("partials", slot = c - first block of that query tile).  The merge kernel
// combines the slots of a query row.  Keys are (distance << 32) | train index, so
// the minimum of unique keys is the nearest train descriptor with ties resolved to
// the lowest index (Sec. 4 matching; tie and ratio readings as in latch.h).
#pragma once

#include <stdint.h>

#include "internal.h"

namespace latch {

constexpr uint64_t kNoKey = ~0ull;

struct WorkSplit {
    int64_t mt;     // query tiles
    int64_t nt;     // train tiles
    int64_t units;  // mt * nt
    int64_t grid;   // blocks
    int64_t slots;  // max blocks touching one query tile
    int rows;       // query rows per tile
};

__host__ __device__ __forceinline__ int64_t split_start(int64_t c, int64_t units, int64_t grid) {
    return (c * units) / grid;
}

// Block owning unit u.
__host__ __device__ __forceinline__ int64_t split_owner(int64_t u, int64_t units, int64_t grid) {
    int64_t c = (u * grid) / units;
    while (c + 1 < grid && split_start(c + 1, units, grid) <= u) ++c;
    while (c > 0 && split_start(c, units, grid) > u) --c;
    return c;
}

inline WorkSplit make_split(int64_t nq, int64_t nt, int rows, int cols, int64_t max_grid) {
    WorkSplit s;
    s.rows = rows;
    s.mt = (nq + rows - 1) / rows;
    s.nt = (nt + cols - 1) / cols;
    s.units = s.mt * s.nt;
    s.grid = s.units < max_grid ? s.units : max_grid;
    s.slots = 0;
    for (int64_t m = 0; m < s.mt && s.units > 0; ++m) {
        const int64_t lo = split_owner(m * s.nt, s.units, s.grid);
        const int64_t hi = split_owner((m + 1) * s.nt - 1, s.units, s.grid);
        if (hi - lo + 1 > s.slots) s.slots = hi - lo + 1;
    }
    return s;
}

__device__ __forceinline__ void top2_insert_u64(uint64_t key, uint64_t& k1, uint64_t& k2) {
    const uint64_t hi = key > k1 ? key : k1;
    k1 = key < k1 ? key : k1;
    k2 = hi < k2 ? hi : k2;
}

// Partial record of (block c, query tile m, row r).
__device__ __forceinline__ uint64_t* partial_ptr(uint64_t* partials, const WorkSplit& s, int64_t m, int64_t c,
                                                 int r) {
    const int64_t lo = split_owner(m * s.nt, s.units, s.grid);
    return partials + ((m * s.slots + (c - lo)) * s.rows + r) * 2;
}

cudaError_t launch_match_merge(const uint64_t* partials, const WorkSplit& s, int32_t nq, int32_t k, int32_t r_milli,
                               latch_match* out, cudaStream_t stream);

}  // namespace latch

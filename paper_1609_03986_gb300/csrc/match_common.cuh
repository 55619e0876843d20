// Work split shared by the matching kernels.
//
// A matching launch serves a batch of problems (a query set against a train set).
// The units of problem p -- (query tile m, train tile n), m-major -- are numbered
// from p.unit0.  Each problem's units are split into G contiguous shares, share c' =
// [start(c'), start(c'+1)) with start(c') = floor(c' * U / G) (c' rotated per
// problem); a batch with enough query tiles splits whole tiles the same way
// (whole_tiles).  With unit shares, every block writes, for each query tile it
// touches, the two smallest keys of each query row over its train tiles ("partial
// records", slot = tile index + share index), and the merge combines the records of
// a row; with whole tiles the tile's only block writes the matches.  Keys are (distance << 32) | train
// index, so the minimum of unique keys is the nearest train descriptor with ties
// resolved to the lowest index (Sec. 4 matching; tie and ratio readings in latch.h).
#pragma once

#include <stdint.h>

#include "internal.h"

namespace latch {

constexpr uint64_t kNoKey = ~0ull;
constexpr int kMaxProblems = 512;  // problems per launch (kernel-parameter space)

struct MatchProblem {
    int64_t unit0;   // first global unit
    int32_t q_row0;  // first row of the query set in the expanded buffer
    int32_t t_row0;  // first row of the train set
    int32_t nq, nt;
    int32_t mt, ntl;  // query tiles, train tiles
    int32_t g0;       // global index of the problem's first query tile
    int32_t out0;     // first output record
    int32_t k;        // 1 or 2
    int32_t r_milli;  // ratio test threshold, rha(1000 * ratio)
};

// A launch's problem table, passed as a kernel parameter; NP is the capacity (the
// launcher picks the smallest instance that holds the batch, so a single problem
// costs ~100 bytes of parameters rather than the full table).
template <int NP>
struct MatchBatchT {
    int32_t count;
    int32_t tiles;        // query tiles over all problems (sum of mt)
    int32_t whole_tiles;  // 1: shares are whole query tiles (one owner per tile)
    int64_t units, grid, queries;
    MatchProblem p[NP];
};
using MatchBatch = MatchBatchT<kMaxProblems>;

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

__device__ __forceinline__ void top2_insert_u64(uint64_t key, uint64_t& k1, uint64_t& k2) {
    const uint64_t hi = key > k1 ? key : k1;
    k1 = key < k1 ? key : k1;
    k2 = hi < k2 ? hi : k2;
}

void plan_match_batch(MatchBatch* b, int count, int64_t max_grid);
// Scratch of the batched layout [expanded rows][arrival counters for
// counter_tiles query tiles][partial records]; counter_tiles >= b.tiles.
size_t match_tc_batch_scratch_bytes(int64_t rows, const MatchBatch& b, int64_t counter_tiles);
int32_t* match_tc_batch_counters(void* scratch, int64_t rows);
size_t match_tc_partial_bytes(const MatchBatch& b);
size_t match_tc_counter_bytes(int64_t tiles);
// Upper bound of match_tc_partial_bytes + match_tc_counter_bytes (each rounded up
// to 256 bytes) for any launch over `problems` problems, `queries` query rows.
size_t match_tc_partial_bound(int64_t queries, int64_t problems, int64_t sms);
// The batched layout: the expanded rows of every problem's query and
// train sets must be filled already, and the arrival counters zero (a complete
// launch leaves them zero, so consecutive launches need one clearing).
cudaError_t launch_match_tc_batch(const MatchBatch& b, int64_t rows, int64_t counter_tiles, void* scratch,
                                  latch_match* out, uint32_t* flags, cudaStream_t stream);
// Same with explicit buffers: `exp` holds `rows` expanded rows, `partials`
// match_tc_partial_bytes(b) of scratch, `tile_cnt` b.tiles zero counters (NULL:
// combine the records in a separate pass).
cudaError_t launch_match_tc_rows(const MatchBatch& b, const uint8_t* exp, int64_t rows, uint64_t* partials,
                                 int32_t* tile_cnt, latch_match* out, uint32_t* flags, cudaStream_t stream);
cudaError_t launch_expand(const uint8_t* desc, int64_t n, uint8_t* out, cudaStream_t stream);
size_t match_tc_scratch_bytes_sms(int64_t sms, int64_t nq, int64_t nt);

}  // namespace latch

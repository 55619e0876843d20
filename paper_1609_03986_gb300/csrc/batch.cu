// Batched extract-then-match (the structure-from-motion shape of Sec. 4-5: many
// images, each matched against its neighbours).  Enqueues, on one stream:
//   1. one bucket launch and one persistent extraction launch per 64 images; the
//      extraction also writes every descriptor's +-1 E2M1 row for the tensor
//      matcher (each image's set once, although it serves as query and as train
//      in several pairs),
//   2. one persistent tensor-core matching launch per 512 pairs, whose blocks share
//      the (pair, query tile, train tile) units of all pairs: whole query tiles per
//      block in a large batch (each block writes its tiles' matches), otherwise
//      units, with each query tile's partial results combined in the launch (short
//      launches) or by a merge pass.
// Nothing is allocated once latch_reserve_batch has sized the scratch, and nothing
// synchronises, so the whole sequence can be captured into a CUDA graph.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "match_common.cuh"

namespace latch {

namespace {

struct BatchPlan {
    std::vector<int64_t> kp0, n, out0;
    int64_t total_kp = 0, total_out = 0;
    int64_t max_tiles = 0;  // query tiles of the largest matching launch
    size_t ext_bytes = 0, match_bytes = 0;
};

latch_status plan_batch(latch_context* ctx, const latch_batch_desc* b, BatchPlan* plan) {
    if (!b) return fail(ctx, LATCH_EINVAL, "NULL batch");
    if (b->n_images < 0 || b->n_pairs < 0) return fail(ctx, LATCH_EINVAL, "negative image or pair count");
    if (b->n_images > 0 && (!b->h_images || !b->h_n_kps)) return fail(ctx, LATCH_EINVAL, "NULL image arrays");
    if (b->n_pairs > 0 && !b->h_pairs) return fail(ctx, LATCH_EINVAL, "NULL pair array");
    if (b->k != 1 && b->k != 2) return fail(ctx, LATCH_EINVAL, "k = %d must be 1 or 2", b->k);
    if (!(b->ratio >= 0.0f && b->ratio <= 1.0f)) return fail(ctx, LATCH_EINVAL, "ratio %g not in [0, 1]", b->ratio);
    plan->kp0.resize(b->n_images);
    plan->n.resize(b->n_images);
    for (int i = 0; i < b->n_images; ++i) {
        const latch_image& im = b->h_images[i];
        if (im.width < 1 || im.height < 1 || im.width > 32768 || im.height > 32768 || im.pitch < im.width ||
            im.pitch % 16 != 0 || !im.data || (reinterpret_cast<uintptr_t>(im.data) & 15))
            return fail(ctx, LATCH_EINVAL, "image %d: bad size, pitch or alignment", i);
        if (b->h_n_kps[i] < 0) return fail(ctx, LATCH_EINVAL, "image %d: negative keypoint count", i);
        plan->kp0[i] = plan->total_kp;
        plan->n[i] = b->h_n_kps[i];
        plan->total_kp += b->h_n_kps[i];
    }
    if (plan->total_kp > INT32_MAX / 2) return fail(ctx, LATCH_EINVAL, "too many keypoints in one batch");
    if (plan->total_kp > 0 && (!b->d_kps || !b->d_desc)) return fail(ctx, LATCH_EINVAL, "NULL keypoints or output");
    if ((reinterpret_cast<uintptr_t>(b->d_desc) | reinterpret_cast<uintptr_t>(b->d_matches)) & 15)
        return fail(ctx, LATCH_EINVAL, "descriptor and match outputs must be 16-byte aligned");
    plan->out0.resize(b->n_pairs);
    for (int p = 0; p < b->n_pairs; ++p) {
        const int qi = b->h_pairs[2 * p], ti = b->h_pairs[2 * p + 1];
        if (qi < 0 || qi >= b->n_images || ti < 0 || ti >= b->n_images)
            return fail(ctx, LATCH_EINVAL, "pair %d refers to image %d / %d of %d", p, qi, ti, b->n_images);
        plan->out0[p] = plan->total_out;
        plan->total_out += plan->n[qi];
    }
    if (plan->total_out > 0 && !b->d_matches) return fail(ctx, LATCH_EINVAL, "NULL match output");
    plan->ext_bytes = (extract_batch_scratch_bytes(b->h_images, plan->n.data(), b->n_images) + 1023) / 1024 * 1024;
    // matching scratch: the largest chunk of pairs
    MatchBatch* mb = new (std::nothrow) MatchBatch;
    if (!mb) return fail(ctx, LATCH_ENOMEM, "host allocation failed");
    size_t mbytes = 0;
    // the arrival counters are sized for every launch first (they precede the records)
    for (int p0 = 0; p0 < b->n_pairs; p0 += kMaxProblems) {
        const int p1 = p0 + kMaxProblems < b->n_pairs ? p0 + kMaxProblems : b->n_pairs;
        int64_t tiles = 0;
        for (int p = p0; p < p1; ++p) tiles += (plan->n[b->h_pairs[2 * p]] + 127) / 128;
        if (tiles > plan->max_tiles) plan->max_tiles = tiles;
    }
    for (int p0 = 0; p0 < b->n_pairs; p0 += kMaxProblems) {
        const int p1 = p0 + kMaxProblems < b->n_pairs ? p0 + kMaxProblems : b->n_pairs;
        for (int p = p0; p < p1; ++p) {
            MatchProblem& P = mb->p[p - p0];
            const int qi = b->h_pairs[2 * p], ti = b->h_pairs[2 * p + 1];
            P.q_row0 = static_cast<int32_t>(plan->kp0[qi]);
            P.t_row0 = static_cast<int32_t>(plan->kp0[ti]);
            P.nq = static_cast<int32_t>(plan->n[qi]);
            P.nt = static_cast<int32_t>(plan->n[ti]);
            P.out0 = static_cast<int32_t>(plan->out0[p] - plan->out0[p0]);
            P.k = b->k;
            P.r_milli = 0;
        }
        plan_match_batch(mb, p1 - p0, ctx->sm_count);
        const size_t need = match_tc_batch_scratch_bytes(plan->total_kp, *mb, plan->max_tiles);
        if (need > mbytes) mbytes = need;
    }
    delete mb;
    plan->match_bytes = mbytes;
    return LATCH_OK;
}

}  // namespace

}  // namespace latch

using namespace latch;

extern "C" latch_status latch_reserve_batch(latch_context* ctx, const latch_batch_desc* b) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    BatchPlan plan;
    latch_status st = plan_batch(ctx, b, &plan);
    if (st != LATCH_OK) return st;
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    void* p = nullptr;
    return scratch_reserve(ctx, 3, plan.ext_bytes + plan.match_bytes, &p);
}

extern "C" latch_status latch_batch_run(latch_context* ctx, const latch_batch_desc* b, latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    BatchPlan plan;
    latch_status st = plan_batch(ctx, b, &plan);
    if (st != LATCH_OK) return st;
    if (!ctx->has_trip) return fail(ctx, LATCH_EINVAL, "no triplet table: call latch_set_triplets");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    void* scratch = nullptr;
    st = scratch_reserve(ctx, 3, plan.ext_bytes + plan.match_bytes, &scratch);
    if (st != LATCH_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    cudaEvent_t* ev = (ctx->trace_ev && ctx->trace_n < ctx->trace_cap) ? ctx->trace_ev + 3 * ctx->trace_n++ : nullptr;
    // the extraction also writes the matcher's expanded rows when there is
    // matching to do
    const bool matching = b->n_pairs > 0 && plan.total_out > 0;
    uint8_t* mbase = base + plan.ext_bytes;
    if (ev) cudaEventRecord(ev[0], s);
    if (matching) {
        // cleared before the extraction, so that nothing sits between the extraction
        // and the matching launch; each complete matching launch leaves them zero
        st = cuda_check(ctx,
                        cudaMemsetAsync(match_tc_batch_counters(mbase, plan.total_kp), 0,
                                        match_tc_counter_bytes(plan.max_tiles), s),
                        "clearing the arrival counters");
        if (st != LATCH_OK) return st;
    }
    if (plan.total_kp > 0) {
        st = cuda_check(ctx,
                        launch_extract_batch(ctx, b->h_images, plan.kp0.data(), plan.n.data(), b->n_images, b->d_kps,
                                             b->d_desc, base, s, matching ? mbase : nullptr),
                        "batched extraction launch");
        if (st != LATCH_OK) return st;
    }
    if (ev) cudaEventRecord(ev[1], s);
    if (!matching) {
        if (ev) cudaEventRecord(ev[2], s);
        return LATCH_OK;
    }
    const int32_t r_milli = static_cast<int32_t>(std::round(static_cast<double>(b->ratio) * 1000.0));
    MatchBatch* mb = new (std::nothrow) MatchBatch;
    if (!mb) return fail(ctx, LATCH_ENOMEM, "host allocation failed");
    for (int p0 = 0; p0 < b->n_pairs && st == LATCH_OK; p0 += kMaxProblems) {
        const int p1 = p0 + kMaxProblems < b->n_pairs ? p0 + kMaxProblems : b->n_pairs;
        for (int p = p0; p < p1; ++p) {
            MatchProblem& P = mb->p[p - p0];
            const int qi = b->h_pairs[2 * p], ti = b->h_pairs[2 * p + 1];
            P.q_row0 = static_cast<int32_t>(plan.kp0[qi]);
            P.t_row0 = static_cast<int32_t>(plan.kp0[ti]);
            P.nq = static_cast<int32_t>(plan.n[qi]);
            P.nt = static_cast<int32_t>(plan.n[ti]);
            P.out0 = static_cast<int32_t>(plan.out0[p] - plan.out0[p0]);
            P.k = b->k;
            P.r_milli = r_milli;
        }
        plan_match_batch(mb, p1 - p0, ctx->sm_count);
        st = cuda_check(ctx,
                        launch_match_tc_batch(*mb, plan.total_kp, plan.max_tiles, mbase, b->d_matches + plan.out0[p0],
                                              ctx->d_flags, s),
                        "batched match launch");
    }
    delete mb;
    if (ev) cudaEventRecord(ev[2], s);
    return st;
}

// Autotuner: picks, by measurement on this device, (1) the fewest keypoints an
// extraction block takes (which sets the grid on small inputs) and (2) the pair count
// from which LATCH_PATH_AUTO matches on
// the tensor cores instead of the CUDA cores.  It runs on synthetic device data
// shaped like the caller's workload (image size, keypoints, query and train counts),
// times every candidate with CUDA events (median of 3 after a warm-up), and stores
// the winners in the context.  latch_get_tuning / latch_set_tuning read and restore
// them, so a caller can cache them per device.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace latch {
namespace {

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Smooth-ish synthetic image: a hashed value per 4x4 block plus fine noise.
__global__ void tune_image_kernel(uint8_t* img, int w, int h, int64_t pitch, uint32_t seed) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<int64_t>(h) * pitch) return;
    const int y = static_cast<int>(i / pitch), x = static_cast<int>(i % pitch);
    const uint32_t coarse = hash32(seed ^ (static_cast<uint32_t>(y >> 2) * 0x9E3779B1u) ^ static_cast<uint32_t>(x >> 2));
    const uint32_t fine = hash32(seed * 3u + static_cast<uint32_t>(i));
    img[i] = x < w ? static_cast<uint8_t>((coarse & 0xff) / 2 + (fine & 0x3f)) : 0;
}

__global__ void tune_keypoints_kernel(latch_keypoint* kps, int n, int w, int h, int nscales, uint32_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t a = hash32(seed ^ (2u * i)), b = hash32(seed ^ (2u * i + 1));
    latch_keypoint k;
    k.x = w > 64 ? 32 + static_cast<int32_t>(a % static_cast<uint32_t>(w - 64)) : static_cast<int32_t>(a % w);
    k.y = h > 64 ? 32 + static_cast<int32_t>(b % static_cast<uint32_t>(h - 64)) : static_cast<int32_t>(b % h);
    k.angle_bin = static_cast<uint8_t>((a >> 24) & 31);
    k.scale_idx = static_cast<uint8_t>((b >> 24) % static_cast<uint32_t>(nscales));
    k.reserved = 0;
    kps[i] = k;
}

__global__ void tune_bits_kernel(uint32_t* d, int64_t nwords, uint32_t seed) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < nwords) d[i] = hash32(seed ^ static_cast<uint32_t>(i) ^ static_cast<uint32_t>(i >> 32));
}

template <class F>
float median_ms(F&& run, cudaStream_t s) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    run();  // warm-up
    std::vector<float> t;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(a, s);
        run();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t.begin(), t.end());
    return t[1];
}

}  // namespace
}  // namespace latch

using namespace latch;

extern "C" {

latch_status latch_get_tuning(const latch_context* ctx, latch_tuning* out) {
    if (!ctx || !out) return LATCH_EINVAL;
    out->item_kps = ctx->item_kps;
    out->tensor_min_pairs = ctx->tensor_min_pairs;
    return LATCH_OK;
}

latch_status latch_set_tuning(latch_context* ctx, const latch_tuning* t) {
    if (!ctx || !t) return fail(ctx, LATCH_EINVAL, "NULL argument");
    if (t->item_kps < 1 || t->item_kps > 32 || t->tensor_min_pairs < 0)
        return fail(ctx, LATCH_EINVAL, "item_kps must be in [1, 32], tensor_min_pairs >= 0");
    ctx->item_kps = t->item_kps;
    ctx->tensor_min_pairs = t->tensor_min_pairs;
    return LATCH_OK;
}

latch_status latch_autotune(latch_context* ctx, const latch_tune_shape* shape, latch_tuning* out) {
    if (!ctx || !shape) return fail(ctx, LATCH_EINVAL, "NULL argument");
    const latch_tune_shape& sh = *shape;
    if (sh.width < 1 || sh.height < 1 || sh.width > 32768 || sh.height > 32768 || sh.n_keypoints < 0 ||
        sh.n_query < 0 || sh.n_train < 0)
        return fail(ctx, LATCH_EINVAL, "bad tuning shape");
    if (!ctx->has_trip) return fail(ctx, LATCH_EINVAL, "no triplet table: call latch_set_triplets first");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = nullptr;
    LATCH_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    latch_status st = LATCH_OK;
    // ---- extraction: fewest keypoints per block ----
    if (sh.n_keypoints > 0) {
        const int64_t pitch = (static_cast<int64_t>(sh.width) + 15) / 16 * 16;
        uint8_t *img = nullptr, *out_desc = nullptr;
        latch_keypoint* kps = nullptr;
        cudaError_t e = cudaMalloc(&img, static_cast<size_t>(sh.height) * pitch);
        if (e == cudaSuccess) e = cudaMalloc(&kps, static_cast<size_t>(sh.n_keypoints) * sizeof(latch_keypoint));
        if (e == cudaSuccess) e = cudaMalloc(&out_desc, static_cast<size_t>(sh.n_keypoints) * 64);
        if (e == cudaSuccess) {
            const int64_t total = static_cast<int64_t>(sh.height) * pitch;
            tune_image_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(img, sh.width, sh.height,
                                                                                        pitch, 1234u);
            tune_keypoints_kernel<<<(sh.n_keypoints + 255) / 256, 256, 0, s>>>(kps, sh.n_keypoints, sh.width,
                                                                               sh.height, ctx->nscales, 99u);
            note_launches(2);
            e = cudaGetLastError();
        }
        const latch_image im{img, sh.width, sh.height, pitch};
        const int32_t saved = ctx->item_kps;
        int32_t best = saved;
        float best_ms = 1e30f;
        for (const int cand : {4, 8, 16, 32}) {
            if (e != cudaSuccess || st != LATCH_OK) break;
            ctx->item_kps = cand;
            const float ms = median_ms(
                [&] { st = latch_extract(ctx, &im, kps, sh.n_keypoints, nullptr, out_desc, s); }, s);
            if (st == LATCH_OK && ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        ctx->item_kps = best;
        if (img) cudaFree(img);
        if (kps) cudaFree(kps);
        if (out_desc) cudaFree(out_desc);
        if (e != cudaSuccess && st == LATCH_OK) st = cuda_check(ctx, e, "autotune extraction");
    }
    // ---- matching: crossover of the CUDA-core and tensor-core paths ----
    if (st == LATCH_OK && sh.n_query > 0 && sh.n_train > 0) {
        const int64_t nq = sh.n_query, nt = sh.n_train;
        uint8_t *q = nullptr, *t = nullptr;
        latch_match* m = nullptr;
        cudaError_t e = cudaMalloc(&q, static_cast<size_t>(nq) * 64);
        if (e == cudaSuccess) e = cudaMalloc(&t, static_cast<size_t>(nt) * 64);
        if (e == cudaSuccess) e = cudaMalloc(&m, static_cast<size_t>(nq) * sizeof(latch_match));
        if (e == cudaSuccess) {
            tune_bits_kernel<<<static_cast<unsigned>((nq * 16 + 255) / 256), 256, 0, s>>>(
                reinterpret_cast<uint32_t*>(q), nq * 16, 7u);
            tune_bits_kernel<<<static_cast<unsigned>((nt * 16 + 255) / 256), 256, 0, s>>>(
                reinterpret_cast<uint32_t*>(t), nt * 16, 11u);
            note_launches(2);
            e = cudaGetLastError();
        }
        // ladder of train-set sizes (the query set fixed): the smallest size at
        // which the tensor path wins sets the pair threshold
        int64_t threshold = -1;
        for (int64_t ntr = std::min<int64_t>(nt, 64); e == cudaSuccess && st == LATCH_OK; ntr *= 4) {
            if (ntr > nt) ntr = nt;
            float ms[2] = {0.f, 0.f};
            const int paths[2] = {LATCH_PATH_POPC, LATCH_PATH_TENSOR};
            for (int k = 0; k < 2 && st == LATCH_OK; ++k)
                ms[k] = median_ms(
                    [&] {
                        st = hamming_match(ctx, q, static_cast<int32_t>(nq), t, static_cast<int32_t>(ntr), 2, 0.8f, m,
                                           paths[k], s);
                    },
                    s);
            if (st == LATCH_OK && ms[1] <= ms[0]) {
                threshold = nq * ntr;
                break;
            }
            if (ntr == nt) break;
        }
        if (st == LATCH_OK) ctx->tensor_min_pairs = threshold >= 0 ? threshold : nq * nt * 4;
        if (q) cudaFree(q);
        if (t) cudaFree(t);
        if (m) cudaFree(m);
        if (e != cudaSuccess && st == LATCH_OK) st = cuda_check(ctx, e, "autotune matching");
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (st == LATCH_OK && out) latch_get_tuning(ctx, out);
    return st;
}

}  // extern "C"

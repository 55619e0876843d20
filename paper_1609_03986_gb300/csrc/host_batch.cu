// latch_batch_run_host: the batched extract-then-match with host-resident inputs and
// outputs (upload, the batch of Sec. 4-5, download).  Two device staging sets owned
// by the context alternate between calls; uploads run on the context's upload
// stream, ordered with the batch and the (small) downloads on the caller's stream
// by events, so the upload of call i+1 overlaps the kernels of call i.
#include <vector>

#include "internal.h"

namespace latch {
namespace {

int64_t device_pitch(int32_t width) { return (static_cast<int64_t>(width) + 15) / 16 * 16; }

// Grows `sc` to `bytes`.  The set's previous use must be finished (the caller
// synchronises its out_done event first).
cudaError_t grow(Scratch* sc, size_t bytes) {
    if (sc->bytes >= bytes) return cudaSuccess;
    if (sc->ptr) cudaFree(sc->ptr);
    sc->ptr = nullptr;
    sc->bytes = 0;
    const size_t want = bytes + bytes / 4;
    const cudaError_t e = cudaMalloc(&sc->ptr, want);
    if (e == cudaSuccess) sc->bytes = want;
    return e;
}

latch_status ensure_streams(latch_context* ctx) {
    if (!ctx->up_stream) LATCH_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
    for (HostStaging& h : ctx->staging)
        for (cudaEvent_t* e : {&h.in_ready, &h.out_done})
            if (!*e) LATCH_CUDA_TRY(ctx, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return LATCH_OK;
}

}  // namespace
}  // namespace latch

using namespace latch;

extern "C" latch_status latch_batch_run_host(latch_context* ctx, const latch_host_batch_desc* hb,
                                             latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (!hb) return fail(ctx, LATCH_EINVAL, "NULL batch");
    if (hb->n_images < 0 || hb->n_pairs < 0) return fail(ctx, LATCH_EINVAL, "negative image or pair count");
    if (hb->n_images > 0 && (!hb->h_images || !hb->h_n_kps)) return fail(ctx, LATCH_EINVAL, "NULL image arrays");
    int64_t total_kp = 0, total_out = 0, img_bytes = 0;
    for (int i = 0; i < hb->n_images; ++i) {
        const latch_image& im = hb->h_images[i];
        if (im.width < 1 || im.height < 1 || im.width > 32768 || im.height > 32768 || im.pitch < im.width ||
            !im.data)
            return fail(ctx, LATCH_EINVAL, "image %d: bad size, pitch or data", i);
        if (hb->h_n_kps[i] < 0) return fail(ctx, LATCH_EINVAL, "image %d: negative keypoint count", i);
        total_kp += hb->h_n_kps[i];
        img_bytes += (static_cast<int64_t>(im.height) * device_pitch(im.width) + 255) / 256 * 256;
    }
    if (hb->n_pairs > 0 && !hb->h_pairs) return fail(ctx, LATCH_EINVAL, "NULL pair array");
    for (int p = 0; p < hb->n_pairs; ++p) {
        const int qi = hb->h_pairs[2 * p];
        if (qi < 0 || qi >= hb->n_images) return fail(ctx, LATCH_EINVAL, "pair %d refers to image %d", p, qi);
        total_out += hb->h_n_kps[qi];
    }
    if (total_kp > 0 && !hb->h_kps) return fail(ctx, LATCH_EINVAL, "NULL host keypoints");
    if (total_out > 0 && !hb->h_matches) return fail(ctx, LATCH_EINVAL, "NULL host match output");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    latch_status st = ensure_streams(ctx);
    if (st != LATCH_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HostStaging& h = ctx->staging[ctx->host_calls & 1];

    // ---- staging buffers (a set that must grow first waits for its previous use) ----
    const size_t need_img = static_cast<size_t>(img_bytes), need_kps = static_cast<size_t>(total_kp) * 12,
                 need_desc = static_cast<size_t>(total_kp) * 64, need_m = static_cast<size_t>(total_out) * 16;
    if (h.img.bytes < need_img || h.kps.bytes < need_kps || h.desc.bytes < need_desc || h.matches.bytes < need_m) {
        LATCH_CUDA_TRY(ctx, cudaEventSynchronize(h.out_done));
        LATCH_CUDA_TRY(ctx, grow(&h.img, need_img));
        LATCH_CUDA_TRY(ctx, grow(&h.kps, need_kps));
        LATCH_CUDA_TRY(ctx, grow(&h.desc, need_desc));
        LATCH_CUDA_TRY(ctx, grow(&h.matches, need_m));
    }

    // ---- uploads, once the set's previous use (batch and downloads) is over ----
    LATCH_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->up_stream, h.out_done, 0));
    std::vector<latch_image> dimg(hb->n_images);
    uint8_t* ip = static_cast<uint8_t*>(h.img.ptr);
    for (int i = 0; i < hb->n_images; ++i) {
        const latch_image& im = hb->h_images[i];
        const int64_t dp = device_pitch(im.width);
        dimg[i] = latch_image{ip, im.width, im.height, dp};
        LATCH_CUDA_TRY(ctx, cudaMemcpy2DAsync(ip, static_cast<size_t>(dp), im.data, static_cast<size_t>(im.pitch),
                                              static_cast<size_t>(im.width), static_cast<size_t>(im.height),
                                              cudaMemcpyHostToDevice, ctx->up_stream));
        ip += (static_cast<int64_t>(im.height) * dp + 255) / 256 * 256;
    }
    if (total_kp > 0)
        LATCH_CUDA_TRY(ctx, cudaMemcpyAsync(h.kps.ptr, hb->h_kps, need_kps, cudaMemcpyHostToDevice, ctx->up_stream));
    LATCH_CUDA_TRY(ctx, cudaEventRecord(h.in_ready, ctx->up_stream));

    // ---- the batch on the caller's stream ----
    LATCH_CUDA_TRY(ctx, cudaStreamWaitEvent(s, h.in_ready, 0));
    latch_batch_desc b;
    b.n_images = hb->n_images;
    b.h_images = dimg.data();
    b.h_n_kps = hb->h_n_kps;
    b.d_kps = static_cast<const latch_keypoint*>(h.kps.ptr);
    b.d_desc = static_cast<uint8_t*>(h.desc.ptr);
    b.n_pairs = hb->n_pairs;
    b.h_pairs = hb->h_pairs;
    b.k = hb->k;
    b.ratio = hb->ratio;
    b.d_matches = static_cast<latch_match*>(h.matches.ptr);
    st = latch_batch_run(ctx, &b, stream);
    if (st != LATCH_OK) return st;

    // ---- downloads on the caller's stream; then the set is free again ----
    if (total_out > 0)
        LATCH_CUDA_TRY(ctx, cudaMemcpyAsync(hb->h_matches, h.matches.ptr, need_m, cudaMemcpyDeviceToHost, s));
    if (hb->h_desc && total_kp > 0)
        LATCH_CUDA_TRY(ctx, cudaMemcpyAsync(hb->h_desc, h.desc.ptr, need_desc, cudaMemcpyDeviceToHost, s));
    LATCH_CUDA_TRY(ctx, cudaEventRecord(h.out_done, s));
    ++ctx->host_calls;
    return LATCH_OK;
}

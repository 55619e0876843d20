// Context management and the C-ABI entry points of include/latch.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"
#include "sm103.h"

namespace latch {

// Failure-detection self-test: waits, with the kernels' bounded-wait routine, on an
// mbarrier that nothing ever arrives at; when the limit runs out the block raises
// the context's timeout flag and returns, exactly as a stalled pipeline would.
__global__ void selftest_wait_kernel(uint64_t limit_ns, uint32_t* flags) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        sm103::mbar_init(&bar, 1);
        abort_flag = 0;
        sm103::fence_mbar_init();
    }
    __syncthreads();
    const bool ok = sm103::mbar_wait(&bar, 0, &abort_flag, limit_ns);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(flags, kFlagTimeout);
}

static char g_create_err[256] = "";
static std::atomic<uint64_t> g_launches{0};

void note_launches(int count) { g_launches.fetch_add(static_cast<uint64_t>(count), std::memory_order_relaxed); }

cudaError_t once_per_device(unsigned long long* done, cudaError_t (*set)()) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (__atomic_load_n(done, __ATOMIC_ACQUIRE) & bit)) return cudaSuccess;
    e = set();  // idempotent: two threads racing here both set the same attributes
    if (e == cudaSuccess && bit) __atomic_fetch_or(done, bit, __ATOMIC_RELEASE);
    return e;
}

latch_status fail(latch_context* ctx, latch_status st, const char* fmt, ...) {
    char* dst = ctx ? ctx->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

latch_status cuda_check(latch_context* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LATCH_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, LATCH_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(ctx, LATCH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

latch_status scratch_reserve(latch_context* ctx, int slot, size_t bytes, void** out) {
    Scratch& s = ctx->scratch[slot];
    if (bytes > s.bytes) {
        if (s.ptr) {
            cudaError_t e = cudaFree(s.ptr);
            s.ptr = nullptr;
            s.bytes = 0;
            if (e != cudaSuccess) return cuda_check(ctx, e, "cudaFree(scratch)");
        }
        size_t want = bytes + bytes / 4 + 256;  // room to grow a little
        cudaError_t e = cudaMalloc(&s.ptr, want);
        if (e != cudaSuccess) {
            s.ptr = nullptr;
            return cuda_check(ctx, e, "cudaMalloc(scratch)");
        }
        s.bytes = want;
    }
    *out = s.ptr;
    return LATCH_OK;
}

static latch_status upload_scales(latch_context* ctx, const double* scales, int n) {
    const size_t entries = static_cast<size_t>(n) * kBins * kWinPix;
    int8_t* host = static_cast<int8_t*>(malloc(entries * 2));
    int16_t* toff = static_cast<int16_t*>(malloc((entries + 16) * sizeof(int16_t)));
    if (!host || !toff) {
        free(host);
        free(toff);
        return fail(ctx, LATCH_ENOMEM, "host allocation of offset tables failed");
    }
    build_offset_tables(scales, n, host);
    const int reach = max_reach(scales, n);
    const int pitch = extract_tile_pitch(reach);
    for (size_t i = 0; i < entries; ++i) toff[i] = static_cast<int16_t>(host[2 * i + 1] * pitch + host[2 * i]);
    for (size_t i = entries; i < entries + 16; ++i) toff[i] = 0;
    free(host);
    int16_t* dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, (entries + 16) * sizeof(int16_t));
    if (e == cudaSuccess) e = cudaMemcpy(dev, toff, (entries + 16) * sizeof(int16_t), cudaMemcpyHostToDevice);
    free(toff);
    if (e != cudaSuccess) {
        if (dev) cudaFree(dev);
        return cuda_check(ctx, e, "upload offset tables");
    }
    for (latch::HostStaging& h : ctx->staging) {
        for (latch::Scratch* sc : {&h.img, &h.kps, &h.desc, &h.matches})
            if (sc->ptr) cudaFree(sc->ptr);
        for (cudaEvent_t e : {h.in_ready, h.out_done})
            if (e) cudaEventDestroy(e);
    }
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->d_tile_offsets) cudaFree(ctx->d_tile_offsets);
    ctx->d_tile_offsets = dev;
    ctx->nscales = n;
    for (int i = 0; i < n; ++i) ctx->scales[i] = scales[i];
    ctx->reach = reach;
    return LATCH_OK;
}

// Matching path for AUTO: the tensor-core path once the pair count amortises its
// operand expansion and merge launches (threshold set by latch_autotune).
static int choose_match_path(const latch_context* ctx, int64_t nq, int64_t nt) {
    return nq * nt >= ctx->tensor_min_pairs ? LATCH_PATH_TENSOR : LATCH_PATH_POPC;
}

// Triplet coordinates must keep every patch inside the 48x48 window: [3, 44] for the
// 7x7 patches, [3, 43] for the weighted 8x8 ones (one more pixel right and down).
static latch_status validate_triplets(latch_context* ctx, const latch_triplet* t, bool weighted) {
    const int hi = weighted ? kWin - 2 - kPatchR : kWin - 1 - kPatchR;
    for (int i = 0; i < kBits; ++i) {
        const uint8_t* c = &t[i].ax;
        for (int j = 0; j < 6; ++j)
            if (c[j] < kPatchR || c[j] > hi)
                return fail(ctx, LATCH_EINVAL, "triplet %d coordinate %d = %d outside [3, %d]", i, j, c[j], hi);
    }
    return LATCH_OK;
}

// The table reaches the kernels as a launch parameter (copied at each launch), so
// loading one needs no device copy and orders itself with the calls that follow.
static latch_status load_triplets(latch_context* ctx, const latch_triplet* t) {
    if (ctx->has_trip && memcmp(ctx->h_trip, t, sizeof(ctx->h_trip)) == 0) return LATCH_OK;
    latch_status st = validate_triplets(ctx, t, ctx->weighted);
    if (st != LATCH_OK) return st;
    memcpy(ctx->h_trip, t, sizeof(ctx->h_trip));
    build_triplet_offsets(ctx->h_trip, ctx->h_trip_offsets);
    ctx->has_trip = true;
    return LATCH_OK;
}

}  // namespace latch

using namespace latch;

extern "C" {

uint64_t latch_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* latch_version(void) { return "latch-gb300 0.1 (sm_103a)"; }

const char* latch_last_error(const latch_context* ctx) { return ctx ? ctx->err : g_create_err; }

latch_status latch_context_create(int device, latch_context** out) {
    if (!out) return fail(nullptr, LATCH_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, LATCH_EINVAL, "device %d of %d", device, ndev);
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(nullptr, LATCH_EUNSUPPORTED, "device %d is sm_%d%d; this build targets sm_103a", device,
                    prop.major, prop.minor);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, LATCH_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    latch_context* ctx = new (std::nothrow) latch_context();
    if (!ctx) return fail(nullptr, LATCH_ENOMEM, "host allocation failed");
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    const double defaults[3] = {1.0, 1.5, 2.25};
    latch_status st = upload_scales(ctx, defaults, 3);
    if (st == LATCH_OK) st = cuda_check(ctx, cudaMalloc(&ctx->d_flags, 64), "cudaMalloc(flags)");
    if (st == LATCH_OK) st = cuda_check(ctx, cudaMemset(ctx->d_flags, 0, 64), "cudaMemset(flags)");
    if (st != LATCH_OK) {
        fail(nullptr, st, "%s", ctx->err);
        latch_context_destroy(ctx);
        return st;
    }
    *out = ctx;
    return LATCH_OK;
}

latch_status latch_trace_enable(latch_context* ctx, int32_t max_records) {
    if (!ctx || max_records < 0 || max_records > (1 << 20)) return fail(ctx, LATCH_EINVAL, "bad trace capacity");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (ctx->trace_ev) {
        cudaDeviceSynchronize();
        for (int i = 0; i < 3 * ctx->trace_cap; ++i) cudaEventDestroy(ctx->trace_ev[i]);
        delete[] ctx->trace_ev;
        ctx->trace_ev = nullptr;
        ctx->trace_cap = ctx->trace_n = 0;
    }
    if (max_records == 0) return LATCH_OK;
    ctx->trace_ev = new (std::nothrow) cudaEvent_t[3 * static_cast<size_t>(max_records)];
    if (!ctx->trace_ev) return fail(ctx, LATCH_ENOMEM, "host allocation failed");
    for (int i = 0; i < 3 * max_records; ++i) {
        const cudaError_t e = cudaEventCreate(&ctx->trace_ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->trace_ev[j]);
            delete[] ctx->trace_ev;
            ctx->trace_ev = nullptr;
            return cuda_check(ctx, e, "cudaEventCreate");
        }
    }
    ctx->trace_cap = max_records;
    ctx->trace_n = 0;
    return LATCH_OK;
}

latch_status latch_trace_collect(latch_context* ctx, float* out_ms, int32_t capacity, int32_t* n) {
    if (!ctx || !n || (capacity > 0 && !out_ms)) return fail(ctx, LATCH_EINVAL, "NULL argument");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int32_t m = ctx->trace_n < capacity ? ctx->trace_n : capacity;
    for (int i = 0; i < m; ++i) {
        cudaEvent_t* ev = ctx->trace_ev + 3 * i;
        LATCH_CUDA_TRY(ctx, cudaEventSynchronize(ev[2]));
        LATCH_CUDA_TRY(ctx, cudaEventElapsedTime(&out_ms[2 * i], ev[0], ev[1]));
        LATCH_CUDA_TRY(ctx, cudaEventElapsedTime(&out_ms[2 * i + 1], ev[1], ev[2]));
    }
    *n = m;
    ctx->trace_n = 0;
    return LATCH_OK;
}

latch_status latch_context_destroy(latch_context* ctx) {
    if (!ctx) return LATCH_OK;
    latch_trace_enable(ctx, 0);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (latch::HostStaging& h : ctx->staging) {
        for (latch::Scratch* sc : {&h.img, &h.kps, &h.desc, &h.matches})
            if (sc->ptr) cudaFree(sc->ptr);
        for (cudaEvent_t e : {h.in_ready, h.out_done})
            if (e) cudaEventDestroy(e);
    }
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->d_tile_offsets) cudaFree(ctx->d_tile_offsets);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    for (auto& s : ctx->scratch)
        if (s.ptr) cudaFree(s.ptr);
    delete ctx;
    return LATCH_OK;
}

latch_status latch_set_scales(latch_context* ctx, const double* scales, int32_t n) {
    if (!ctx || !scales) return fail(ctx, LATCH_EINVAL, "NULL argument");
    if (n < 1 || n > LATCH_MAX_SCALES) return fail(ctx, LATCH_EINVAL, "number of scales %d not in [1, 8]", n);
    for (int i = 0; i < n; ++i)
        if (!(scales[i] >= 0.25 && scales[i] <= kMaxScale))
            return fail(ctx, LATCH_EINVAL, "scale %d = %g not in [0.25, 2.25]", i, scales[i]);
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    LATCH_CUDA_TRY(ctx, cudaDeviceSynchronize());
    return upload_scales(ctx, scales, n);
}

latch_status latch_set_triplets(latch_context* ctx, const latch_triplet* h_triplets) {
    if (!ctx || !h_triplets) return fail(ctx, LATCH_EINVAL, "NULL argument");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return load_triplets(ctx, h_triplets);
}

latch_status latch_set_patch_weights(latch_context* ctx, const uint8_t* h_weights) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (!h_weights) {
        ctx->weighted = false;
        return LATCH_OK;
    }
    if (ctx->has_trip) {
        latch_status st = validate_triplets(ctx, ctx->h_trip, true);
        if (st != LATCH_OK) return st;
    }
    for (int i = 0; i < 64; ++i) ctx->patch_weights[i] = h_weights[i];
    ctx->weighted = true;
    return LATCH_OK;
}

latch_status latch_reserve(latch_context* ctx, int64_t max_keypoints, int64_t max_query, int64_t max_train) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (max_keypoints < 0 || max_query < 0 || max_train < 0) return fail(ctx, LATCH_EINVAL, "negative size");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    void* p = nullptr;
    latch_image big{nullptr, 32768, 32768, 32768};
    latch_status st = scratch_reserve(ctx, 0, extract_scratch_bytes(&big, max_keypoints), &p);
    if (st == LATCH_OK) st = scratch_reserve(ctx, 1, match_popc_scratch_bytes(ctx, max_query, max_train), &p);
    if (st == LATCH_OK) st = scratch_reserve(ctx, 2, match_tc_scratch_bytes(ctx, max_query, max_train), &p);
    return st;
}

int32_t hamming_match_path(const latch_context* ctx, int64_t nq, int64_t nt) {
    return ctx ? choose_match_path(ctx, nq, nt) : -1;
}

latch_status latch_selftest_wait_timeout(latch_context* ctx, int32_t limit_us, latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (limit_us < 1 || limit_us > 2000000) return fail(ctx, LATCH_EINVAL, "limit_us must be in [1, 2e6]");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<uint64_t>(limit_us) * 1000,
                                                                          ctx->d_flags);
    note_launches(1);
    return cuda_check(ctx, cudaGetLastError(), "self-test launch");
}

latch_status latch_check(latch_context* ctx) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    LATCH_CUDA_TRY(ctx, cudaDeviceSynchronize());
    uint32_t flags = 0;
    LATCH_CUDA_TRY(ctx, cudaMemcpy(&flags, ctx->d_flags, sizeof(flags), cudaMemcpyDeviceToHost));
    if (flags) {
        LATCH_CUDA_TRY(ctx, cudaMemset(ctx->d_flags, 0, sizeof(flags)));
        if (flags & kFlagTimeout) return fail(ctx, LATCH_ETIMEOUT, "a device-side wait timed out (flags 0x%x)", flags);
        return fail(ctx, LATCH_EDEVICE, "a keypoint had a scale index outside the scale table (flags 0x%x)", flags);
    }
    return LATCH_OK;
}

latch_status latch_extract(latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps, int32_t n,
                           const latch_triplet* h_triplets, uint8_t* d_out, latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (n < 0) return fail(ctx, LATCH_EINVAL, "n = %d < 0", n);
    if (!img) return fail(ctx, LATCH_EINVAL, "NULL image");
    if (img->width < 1 || img->height < 1 || img->width > 32768 || img->height > 32768)
        return fail(ctx, LATCH_EINVAL, "image size %dx%d outside [1, 32768]", img->width, img->height);
    if (img->pitch < img->width || img->pitch % 16 != 0)
        return fail(ctx, LATCH_EINVAL, "pitch %lld must be >= width and a multiple of 16", (long long)img->pitch);
    if (!img->data || (reinterpret_cast<uintptr_t>(img->data) & 15))
        return fail(ctx, LATCH_EINVAL, "image data must be non-NULL and 16-byte aligned");
    if (n > 0 && (!d_kps || !d_out)) return fail(ctx, LATCH_EINVAL, "NULL keypoints or output");
    if (d_out && (reinterpret_cast<uintptr_t>(d_out) & 15)) return fail(ctx, LATCH_EINVAL, "d_out not 16-byte aligned");
    if (d_kps && (reinterpret_cast<uintptr_t>(d_kps) & 3)) return fail(ctx, LATCH_EINVAL, "d_kps not 4-byte aligned");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h_triplets) {
        latch_status st = load_triplets(ctx, h_triplets);
        if (st != LATCH_OK) return st;
    }
    if (!ctx->has_trip) return fail(ctx, LATCH_EINVAL, "no triplet table: pass one or call latch_set_triplets");
    if (n == 0) return LATCH_OK;
    void* scratch = nullptr;
    latch_status st = scratch_reserve(ctx, 0, extract_scratch_bytes(img, n), &scratch);
    if (st != LATCH_OK) return st;
    return cuda_check(ctx, launch_extract(ctx, img, d_kps, n, d_out, scratch, s), "extract kernel launch");
}

static latch_status validate_image(latch_context* ctx, const latch_image* img) {
    if (!img) return fail(ctx, LATCH_EINVAL, "NULL image");
    if (img->width < 1 || img->height < 1 || img->width > 32768 || img->height > 32768)
        return fail(ctx, LATCH_EINVAL, "image size %dx%d outside [1, 32768]", img->width, img->height);
    if (img->pitch < img->width || img->pitch % 16 != 0)
        return fail(ctx, LATCH_EINVAL, "pitch %lld must be >= width and a multiple of 16", (long long)img->pitch);
    if (!img->data || (reinterpret_cast<uintptr_t>(img->data) & 15))
        return fail(ctx, LATCH_EINVAL, "image data must be non-NULL and 16-byte aligned");
    return LATCH_OK;
}

static latch_status validate_detect(latch_context* ctx, const latch_image* img, int32_t threshold, int32_t scale_idx,
                                    int32_t max_kps, const latch_keypoint* d_kps, const int32_t* d_count) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    latch_status st = validate_image(ctx, img);
    if (st != LATCH_OK) return st;
    if (threshold < 1 || threshold > 254) return fail(ctx, LATCH_EINVAL, "FAST threshold %d not in [1, 254]", threshold);
    if (scale_idx < 0 || scale_idx >= ctx->nscales)
        return fail(ctx, LATCH_EINVAL, "scale index %d outside the scale table (%d entries)", scale_idx, ctx->nscales);
    if (max_kps < 0) return fail(ctx, LATCH_EINVAL, "max_kps = %d < 0", max_kps);
    if (!d_count || (reinterpret_cast<uintptr_t>(d_count) & 3)) return fail(ctx, LATCH_EINVAL, "bad d_count");
    if (max_kps > 0 && (!d_kps || (reinterpret_cast<uintptr_t>(d_kps) & 3)))
        return fail(ctx, LATCH_EINVAL, "NULL or misaligned keypoint output");
    return LATCH_OK;
}

latch_status latch_detect(latch_context* ctx, const latch_image* img, int32_t threshold, int32_t scale_idx,
                          int32_t max_kps, latch_keypoint* d_kps, int32_t* d_count, latch_stream_t stream) {
    latch_status st = validate_detect(ctx, img, threshold, scale_idx, max_kps, d_kps, d_count);
    if (st != LATCH_OK) return st;
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const double one = 1.0;
    void* scratch = nullptr;
    st = scratch_reserve(ctx, 4, detect_scratch_bytes(img, &one, 1), &scratch);
    if (st != LATCH_OK) return st;
    return cuda_check(ctx,
                      launch_detect(img, &one, &scale_idx, 1, threshold, max_kps, d_kps, d_count, scratch,
                                    static_cast<cudaStream_t>(stream)),
                      "detection launch");
}

// Detection over the pyramid levels of the first n_levels scales (each >= 1), then
// optionally the descriptors (level l's keypoints carry scale index l).
static latch_status detect_levels(latch_context* ctx, const latch_image* img, const double* scales,
                                  const int32_t* idx, int nlev, int32_t threshold, int32_t max_kps,
                                  latch_keypoint* d_kps, int32_t* d_count, uint8_t* d_desc, cudaStream_t s) {
    void* dscratch = nullptr;
    void* escratch = nullptr;
    latch_status st = scratch_reserve(ctx, 4, detect_scratch_bytes(img, scales, nlev), &dscratch);
    if (st == LATCH_OK && d_desc) st = scratch_reserve(ctx, 0, extract_scratch_bytes(img, max_kps), &escratch);
    if (st != LATCH_OK) return st;
    st = cuda_check(ctx, launch_detect(img, scales, idx, nlev, threshold, max_kps, d_kps, d_count, dscratch, s),
                    "detection launch");
    if (st != LATCH_OK || !d_desc) return st;
    return cuda_check(ctx, launch_extract_dev_count(ctx, img, d_kps, max_kps, d_count, d_desc, escratch, s),
                      "extraction launch");
}

latch_status latch_detect_pyramid(latch_context* ctx, const latch_image* img, int32_t threshold, int32_t n_levels,
                                  int32_t max_kps, latch_keypoint* d_kps, int32_t* d_count, uint8_t* d_desc,
                                  latch_stream_t stream) {
    latch_status st = validate_detect(ctx, img, threshold, 0, max_kps, d_kps, d_count);
    if (st != LATCH_OK) return st;
    if (n_levels < 1 || n_levels > ctx->nscales)
        return fail(ctx, LATCH_EINVAL, "n_levels = %d not in [1, %d] (the scale table)", n_levels, ctx->nscales);
    int32_t idx[LATCH_MAX_SCALES];
    for (int l = 0; l < n_levels; ++l) {
        if (!(ctx->scales[l] >= 1.0))
            return fail(ctx, LATCH_EINVAL, "pyramid level %d has scale %g < 1", l, ctx->scales[l]);
        idx[l] = l;
    }
    if (d_desc && max_kps > 0 && (reinterpret_cast<uintptr_t>(d_desc) & 15))
        return fail(ctx, LATCH_EINVAL, "misaligned descriptor output");
    if (d_desc && !ctx->has_trip) return fail(ctx, LATCH_EINVAL, "no triplet table: call latch_set_triplets");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return detect_levels(ctx, img, ctx->scales, idx, n_levels, threshold, max_kps, d_kps, d_count,
                         max_kps > 0 ? d_desc : nullptr, static_cast<cudaStream_t>(stream));
}

latch_status latch_detect_extract(latch_context* ctx, const latch_image* img, int32_t threshold, int32_t scale_idx,
                                  int32_t max_kps, latch_keypoint* d_kps, int32_t* d_count, uint8_t* d_desc,
                                  latch_stream_t stream) {
    latch_status st = validate_detect(ctx, img, threshold, scale_idx, max_kps, d_kps, d_count);
    if (st != LATCH_OK) return st;
    if (max_kps > 0 && (!d_desc || (reinterpret_cast<uintptr_t>(d_desc) & 15)))
        return fail(ctx, LATCH_EINVAL, "NULL or misaligned descriptor output");
    if (!ctx->has_trip) return fail(ctx, LATCH_EINVAL, "no triplet table: call latch_set_triplets");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const double one = 1.0;
    return detect_levels(ctx, img, &one, &scale_idx, 1, threshold, max_kps, d_kps, d_count,
                         max_kps > 0 ? d_desc : nullptr, static_cast<cudaStream_t>(stream));
}

latch_status hamming_match(latch_context* ctx, const uint8_t* d_query, int32_t nq, const uint8_t* d_train,
                           int32_t nt, int32_t k, float ratio, latch_match* d_out, int32_t path,
                           latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (nq < 0 || nt < 0) return fail(ctx, LATCH_EINVAL, "negative size");
    if (k != 1 && k != 2) return fail(ctx, LATCH_EINVAL, "k = %d must be 1 or 2", k);
    if (!(ratio >= 0.0f && ratio <= 1.0f)) return fail(ctx, LATCH_EINVAL, "ratio %g not in [0, 1]", ratio);
    if (path != LATCH_PATH_AUTO && path != LATCH_PATH_POPC && path != LATCH_PATH_TENSOR)
        return fail(ctx, LATCH_EINVAL, "unknown path %d", path);
    if (nq > 0 && (!d_query || !d_out)) return fail(ctx, LATCH_EINVAL, "NULL query or output");
    if (nq > 0 && nt > 0 && !d_train) return fail(ctx, LATCH_EINVAL, "NULL train");
    if ((reinterpret_cast<uintptr_t>(d_query) | reinterpret_cast<uintptr_t>(d_train) |
         reinterpret_cast<uintptr_t>(d_out)) & 15)
        return fail(ctx, LATCH_EINVAL, "descriptor and output pointers must be 16-byte aligned");
    if (nq == 0) return LATCH_OK;
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int32_t r_milli = static_cast<int32_t>(std::round(static_cast<double>(ratio) * 1000.0));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (path == LATCH_PATH_AUTO) path = choose_match_path(ctx, nq, nt);
    void* scratch = nullptr;
    if (path == LATCH_PATH_TENSOR) {
        latch_status st = scratch_reserve(ctx, 2, match_tc_scratch_bytes(ctx, nq, nt), &scratch);
        if (st != LATCH_OK) return st;
        return cuda_check(ctx, launch_match_tc(ctx, d_query, nq, d_train, nt, k, r_milli, d_out, scratch, s),
                          "tensor match launch");
    }
    latch_status st = scratch_reserve(ctx, 1, match_popc_scratch_bytes(ctx, nq, nt), &scratch);
    if (st != LATCH_OK) return st;
    return cuda_check(ctx, launch_match_popc(ctx, d_query, nq, d_train, nt, k, r_milli, d_out, scratch, s),
                      "popc match launch");
}

latch_status latch_dense_extract(latch_context* ctx, const latch_image* img, uint8_t* d_out, latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    latch_status st = validate_image(ctx, img);
    if (st != LATCH_OK) return st;
    if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15))
        return fail(ctx, LATCH_EINVAL, "d_out must be non-NULL and 16-byte aligned");
    if (!ctx->has_trip) return fail(ctx, LATCH_EINVAL, "no triplet table: call latch_set_triplets");
    if (ctx->weighted) return fail(ctx, LATCH_EUNSUPPORTED, "dense extraction uses 7x7 patches (weights are set)");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return cuda_check(ctx, launch_dense_extract(ctx, img, d_out, static_cast<cudaStream_t>(stream)),
                      "dense extract launch");
}

latch_status latch_dense_match(latch_context* ctx, const uint8_t* d_a, const uint8_t* d_b, int32_t width,
                               int32_t height, int32_t radius, int32_t k, float ratio, latch_match* d_out,
                               latch_stream_t stream) {
    if (!ctx) return fail(ctx, LATCH_EINVAL, "NULL context");
    if (width < 1 || height < 1 || width > 32768 || height > 32768)
        return fail(ctx, LATCH_EINVAL, "field size %dx%d outside [1, 32768]", width, height);
    if (radius < 0 || radius > LATCH_DENSE_MAX_RADIUS)
        return fail(ctx, LATCH_EINVAL, "radius %d outside [0, %d]", radius, LATCH_DENSE_MAX_RADIUS);
    if (k != 1 && k != 2) return fail(ctx, LATCH_EINVAL, "k = %d must be 1 or 2", k);
    if (!(ratio >= 0.0f && ratio <= 1.0f)) return fail(ctx, LATCH_EINVAL, "ratio %g not in [0, 1]", ratio);
    if (!d_a || !d_b || !d_out) return fail(ctx, LATCH_EINVAL, "NULL descriptor field or output");
    if ((reinterpret_cast<uintptr_t>(d_a) | reinterpret_cast<uintptr_t>(d_b) | reinterpret_cast<uintptr_t>(d_out)) &
        15)
        return fail(ctx, LATCH_EINVAL, "descriptor and output pointers must be 16-byte aligned");
    LATCH_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int32_t r_milli = static_cast<int32_t>(std::round(static_cast<double>(ratio) * 1000.0));
    return cuda_check(ctx,
                      launch_dense_match(d_a, d_b, width, height, radius, k, r_milli, d_out,
                                         static_cast<cudaStream_t>(stream)),
                      "dense match launch");
}

}  // extern "C"

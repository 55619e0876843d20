// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "latch.h"

namespace latch {

constexpr int kWin = LATCH_WINDOW;          // 48
constexpr int kWinPix = kWin * kWin;        // 2304
constexpr int kHalf = kWin / 2;             // 24
constexpr int kPatchR = LATCH_PATCH / 2;    // 3
constexpr int kBits = LATCH_TRIPLETS;       // 512
constexpr int kDescBytes = LATCH_DESC_BYTES;
constexpr int kDescWords = kDescBytes / 4;  // 16
constexpr int kBins = LATCH_ANGLE_BINS;
constexpr double kMaxScale = 2.25;
constexpr int kMaxReach = 77;               // max |offset| at scale 2.25 (24*sqrt(2)*2.25 = 76.4)

// The tensor matcher's input row of one descriptor: its 512 bits as 4-bit E2M1
// floats, two per byte, bit t -> value t = 1 - 2 bit (+1.0 = 0x2 when clear, -1.0 =
// 0xA when set; value t in the low nibble of byte t / 2 when t is even).  The dot
// product of two rows is then (bits that agree) - (bits that differ) =
// 512 - 2 Hamming, so one contraction gives the distance with no popcount term.
constexpr int kExpRowBytes = 256;

#ifdef __CUDACC__
// Byte -> its 8 bits as 8 E2M1 values (nibble q = 0x2 | 8 bit q), by spreading the
// bits in three mask-and-shift steps (4-bit groups, then pairs, then single bits) to
// the sign position of their nibbles.
__device__ __forceinline__ uint32_t expand_byte_e2m1(uint32_t b) {
    uint32_t x = b & 0xffu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return (x << 3) | 0x22222222u;
}
// 32 descriptor bits (bit q = descriptor bit 32 i + q) -> their 16 expanded bytes.
__device__ __forceinline__ uint4 expand_word_e2m1(uint32_t w) {
    return make_uint4(expand_byte_e2m1(w), expand_byte_e2m1(w >> 8), expand_byte_e2m1(w >> 16),
                      expand_byte_e2m1(w >> 24));
}
#endif

// Device-side error flags (OR-ed into ctx->d_flags).
enum : uint32_t { kFlagBadScale = 1u, kFlagTimeout = 2u };

// Host-built sample-offset tables (tables.cpp).  For each scale s and angle bin b,
// kWinPix entries of (dx, dy) as int8 pairs, entry index v * 48 + u.
void build_offset_tables(const double* scales, int nscales, int8_t* out /* nscales*32*2304*2 */);
int max_reach(const double* scales, int nscales);
// Staged-tile row pitch of the extraction kernel for a given reach.
int extract_tile_pitch(int reach);
// Window words and byte shifts of every triplet's three patches (the extraction
// kernel's triplet parameter).
void build_triplet_offsets(const latch_triplet* trip, uint32_t* out /* 2 per triplet */);

struct Scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// One device staging set of latch_batch_run_host: images, keypoints, descriptors,
// matches (grow-only), and the events that order its use.
struct HostStaging {
    Scratch img, kps, desc, matches;
    cudaEvent_t in_ready = nullptr;  // uploads done (upload stream)
    cudaEvent_t out_done = nullptr;  // batch and downloads done (caller's stream): the set is free again
};

}  // namespace latch

struct latch_context {
    int device = 0;
    int sm_count = 0;
    int nscales = 0;
    double scales[LATCH_MAX_SCALES] = {};
    int reach = 0;                       // max |offset| over the scale table
    int16_t* d_tile_offsets = nullptr;   // nscales * 32 * 2304 (+16 pad) tile offsets dy * pitch + dx
    latch_triplet h_trip[LATCH_TRIPLETS] = {};
    bool has_trip = false;
    uint32_t h_trip_offsets[2 * LATCH_TRIPLETS] = {};
    bool weighted = false;               // 8x8 weighted patches (latch_set_patch_weights) instead of 7x7
    int32_t patch_weights[64] = {};
    uint32_t* d_flags = nullptr;         // device error word
    int32_t item_kps = 16;               // extraction: fewest keypoints per block (latch_autotune)
    // tracing (latch_trace_enable): per batch run, events before extraction, between
    // extraction and matching, and after matching
    cudaEvent_t* trace_ev = nullptr;
    int32_t trace_cap = 0, trace_n = 0;
    int64_t tensor_min_pairs = int64_t(1) << 22;  // matching: AUTO uses the tensor path from here
    latch::Scratch scratch[5];           // grow-only scratch regions (4: detection)
    // latch_batch_run_host: two staging sets used alternately, upload stream
    latch::HostStaging staging[2];
    cudaStream_t up_stream = nullptr;
    uint64_t host_calls = 0;
    char err[256] = {};
};

namespace latch {

// Records an error message on the context and returns `st`.
latch_status fail(latch_context* ctx, latch_status st, const char* fmt, ...);
// Maps a CUDA error to LATCH_ECUDA (recorded on ctx) or LATCH_OK.
latch_status cuda_check(latch_context* ctx, cudaError_t e, const char* what);
// Ensures scratch region `slot` holds at least `bytes` (cudaMalloc, grow-only).
latch_status scratch_reserve(latch_context* ctx, int slot, size_t bytes, void** out);

// Counts kernel launches made by the library (latch_kernel_launches()).
void note_launches(int count);

// Runs `set` (a cudaFuncSetAttribute sequence for one kernel) once per device: the
// attributes belong to the current device's context.  `done` is the kernel's mask of
// devices already set up (devices 0..63; larger indices run `set` on every call).
cudaError_t once_per_device(unsigned long long* done, cudaError_t (*set)());

// Launches `kernel` so that it may start while the previous kernel on the stream
// is still running (programmatic dependent launch).  Every kernel launched this way
// executes griddepcontrol.wait before it reads or writes global memory that earlier
// work on the stream may touch, so the stream order of the results is unchanged;
// what overlaps is the launch and the kernel's shared-memory / barrier prologue.
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                           Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launches(1);
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Kernel launchers (one per .cu file); return cudaGetLastError() of the launch.
cudaError_t launch_extract(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps, int32_t n,
                           uint8_t* d_out, void* scratch, cudaStream_t stream);
size_t extract_scratch_bytes(const latch_image* img, int64_t n);
// Images [0, count) with keypoints d_kps[kp0[i] .. kp0[i] + n[i]) -> d_out rows at the same positions.
// When exp_out is not NULL, row r of the tensor matcher's input (kExpRowBytes bytes, E2M1 +-1.0
// per bit) is written as well.
// `flags`: the device error word the kernels raise flags in (NULL: the context's).
cudaError_t launch_extract_batch(const latch_context* ctx, const latch_image* imgs, const int64_t* kp0,
                                 const int64_t* n, int count, const latch_keypoint* d_kps, uint8_t* d_out,
                                 void* scratch, cudaStream_t stream, uint8_t* exp_out, uint32_t* flags = nullptr);
size_t extract_batch_scratch_bytes(const latch_image* imgs, const int64_t* n, int count);
// One image whose keypoint count is on the device (*d_n, at most max_n keypoints in
// d_kps); scratch as extract_scratch_bytes(img, max_n).
cudaError_t launch_extract_dev_count(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps,
                                     int32_t max_n, const int32_t* d_n, uint8_t* d_out, void* scratch,
                                     cudaStream_t stream);

// Oriented FAST keypoints (detect.cu) of the pyramid levels scales[0 .. nlev) (each >= 1;
// scale 1 is the image itself), level l's keypoints given scale index scale_idx[l]:
// up to max_kps into d_kps, the number found into *d_count.
constexpr int kMaxDetectLevels = LATCH_MAX_SCALES;
cudaError_t launch_detect(const latch_image* img, const double* scales, const int32_t* scale_idx, int nlev,
                          int32_t threshold, int32_t max_kps, latch_keypoint* d_kps, int32_t* d_count, void* scratch,
                          cudaStream_t stream);
size_t detect_scratch_bytes(const latch_image* img, const double* scales, int nlev);

// Dense per-pixel descriptors and windowed matching (dense.cu).
constexpr int kDenseMaxRadius = LATCH_DENSE_MAX_RADIUS;
cudaError_t launch_dense_extract(const latch_context* ctx, const latch_image* img, uint8_t* d_out,
                                 cudaStream_t stream);
cudaError_t launch_dense_match(const uint8_t* d_a, const uint8_t* d_b, int32_t width, int32_t height, int32_t radius,
                               int32_t k, int32_t r_milli, latch_match* d_out, cudaStream_t stream);

cudaError_t launch_match_popc(const latch_context* ctx, const uint8_t* q, int32_t nq, const uint8_t* t, int32_t nt,
                              int32_t k, int32_t r_milli, latch_match* out, void* scratch, cudaStream_t stream);
size_t match_popc_scratch_bytes(const latch_context* ctx, int64_t nq, int64_t nt);

cudaError_t launch_match_tc(const latch_context* ctx, const uint8_t* q, int32_t nq, const uint8_t* t, int32_t nt,
                            int32_t k, int32_t r_milli, latch_match* out, void* scratch, cudaStream_t stream);
size_t match_tc_scratch_bytes(const latch_context* ctx, int64_t nq, int64_t nt);

}  // namespace latch

#define LATCH_CUDA_TRY(ctx, expr)                                         \
    do {                                                                  \
        cudaError_t e_ = (expr);                                          \
        if (e_ != cudaSuccess) return latch::cuda_check((ctx), e_, #expr); \
    } while (0)

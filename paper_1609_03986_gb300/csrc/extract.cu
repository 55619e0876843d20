// LATCH descriptor extraction (Sec. 3.1 Eq. 1; Sec. 3.2).
//
// One warp per keypoint: the lanes gather the oriented, scaled 48x48 window into
// shared memory through the per-(scale, bin) offset table (nearest pixel; samples
// outside the image read 0), then every lane evaluates 16 triplets
// t = 32*w + lane, w = 0..15: D1 = ||P_A - P_1||^2, D2 = ||P_A - P_2||^2 over the
// 7x7 patches in exact integer arithmetic, bit = D1 > D2.  __ballot_sync packs the
// 32 bits of word w (bit i = triplet 32*w + i, i.e. bit t is bit t%8 of byte t/8),
// and lanes 0..15 write the 16 words of the descriptor as one coalesced 64-byte row.
#include <cstdint>

#include "internal.h"

namespace latch {

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = kWarps * 32;

__global__ void __launch_bounds__(kThreads) extract_naive_kernel(
    const uint8_t* __restrict__ img, int width, int height, int64_t pitch, const latch_keypoint* __restrict__ kps,
    int n, const int8_t* __restrict__ offsets, int nscales, const uint8_t* __restrict__ trip_g,
    uint32_t* __restrict__ out, uint32_t* __restrict__ flags) {
    __shared__ uint8_t s_trip[kBits * 6];
    __shared__ uint8_t s_win[kWarps][kWinPix];
    for (int i = threadIdx.x; i < kBits * 6; i += kThreads) s_trip[i] = trip_g[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t* win = s_win[warp];
    for (int k = blockIdx.x * kWarps + warp; k < n; k += gridDim.x * kWarps) {
        const latch_keypoint kp = kps[k];
        uint32_t word = 0;
        if (kp.scale_idx < nscales) {
            const char2* tab = reinterpret_cast<const char2*>(offsets) +
                               (static_cast<size_t>(kp.scale_idx) * kBins + (kp.angle_bin & (kBins - 1))) * kWinPix;
            for (int i = lane; i < kWinPix; i += 32) {
                const char2 o = tab[i];
                const int64_t x = static_cast<int64_t>(kp.x) + o.x;
                const int64_t y = static_cast<int64_t>(kp.y) + o.y;
                win[i] = (x >= 0 && x < width && y >= 0 && y < height) ? img[y * pitch + x] : 0;
            }
            __syncwarp();
            for (int w = 0; w < kDescWords; ++w) {
                const uint8_t* t = s_trip + 6 * (32 * w + lane);
                const int ax = t[0] - kPatchR, ay = t[1] - kPatchR;
                const int c1x = t[2] - kPatchR, c1y = t[3] - kPatchR;
                const int c2x = t[4] - kPatchR, c2y = t[5] - kPatchR;
                int d1 = 0, d2 = 0;  // <= 49 * 255^2 < 2^22
                for (int i = 0; i < 2 * kPatchR + 1; ++i)
                    for (int j = 0; j < 2 * kPatchR + 1; ++j) {
                        const int a = win[(ay + i) * kWin + ax + j];
                        const int p1 = win[(c1y + i) * kWin + c1x + j];
                        const int p2 = win[(c2y + i) * kWin + c2x + j];
                        d1 += (a - p1) * (a - p1);
                        d2 += (a - p2) * (a - p2);
                    }
                const uint32_t b = __ballot_sync(0xffffffffu, d1 > d2);
                if (lane == w) word = b;
            }
            __syncwarp();
        } else if (lane == 0) {
            atomicOr(flags, kFlagBadScale);
        }
        if (lane < kDescWords) out[static_cast<size_t>(k) * kDescWords + lane] = word;
    }
}

}  // namespace

size_t extract_scratch_bytes(const latch_image*, int64_t) { return 0; }

cudaError_t launch_extract(const latch_context* ctx, const latch_image* img, const latch_keypoint* d_kps, int32_t n,
                           uint8_t* d_out, void*, cudaStream_t stream) {
    const int blocks_needed = (n + kWarps - 1) / kWarps;
    const int grid = blocks_needed < ctx->sm_count * 16 ? blocks_needed : ctx->sm_count * 16;
    extract_naive_kernel<<<grid, kThreads, 0, stream>>>(img->data, img->width, img->height, img->pitch, d_kps, n,
                                                        ctx->d_offsets, ctx->nscales, ctx->d_trip,
                                                        reinterpret_cast<uint32_t*>(d_out), ctx->d_flags);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace latch

/* A plain C client of include/latch.h: no Python, no C++, only the CUDA runtime for
 * device memory.  It extracts descriptors for a small synthetic image, matches the
 * set against itself on both paths (every query must find itself at distance 0),
 * checks an argument error, and prints "ok".  Exit status 0 on success. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "latch.h"

#define CHECK(cond, msg)                                  \
    do {                                                  \
        if (!(cond)) {                                    \
            fprintf(stderr, "FAILED: %s\n", msg);         \
            return 1;                                     \
        }                                                 \
    } while (0)

static uint32_t rng = 12345u;
static uint32_t next_u32(void) {
    rng ^= rng << 13;
    rng ^= rng >> 17;
    rng ^= rng << 5;
    return rng;
}

int main(void) {
    enum { W = 320, H = 240, N = 500 };
    latch_context *ctx = NULL;
    latch_status st = latch_context_create(0, &ctx);
    CHECK(st == LATCH_OK, "latch_context_create");

    latch_triplet trip[512];
    for (int t = 0; t < 512; ++t) {
        uint8_t *c = &trip[t].ax;
        for (int q = 0; q < 6; ++q) c[q] = (uint8_t)(3 + next_u32() % 42); /* patch centres in [3, 44] */
    }
    CHECK(latch_set_triplets(ctx, trip) == LATCH_OK, "latch_set_triplets");

    /* image: smooth gradient plus noise, pitch 320 (a multiple of 16) */
    uint8_t *h_img = (uint8_t *)malloc((size_t)W * H);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) h_img[y * W + x] = (uint8_t)((x * 3 + y * 5 + (next_u32() & 31)) & 255);
    latch_keypoint h_kps[N];
    for (int i = 0; i < N; ++i) {
        h_kps[i].x = 30 + (int32_t)(next_u32() % (W - 60));
        h_kps[i].y = 30 + (int32_t)(next_u32() % (H - 60));
        h_kps[i].angle_bin = (uint8_t)(next_u32() % 32);
        h_kps[i].scale_idx = (uint8_t)(next_u32() % 3);
        h_kps[i].reserved = 0;
    }
    uint8_t *d_img = NULL, *d_desc = NULL;
    latch_keypoint *d_kps = NULL;
    latch_match *d_m = NULL;
    CHECK(cudaMalloc((void **)&d_img, (size_t)W * H) == cudaSuccess, "cudaMalloc image");
    CHECK(cudaMalloc((void **)&d_kps, sizeof h_kps) == cudaSuccess, "cudaMalloc keypoints");
    CHECK(cudaMalloc((void **)&d_desc, (size_t)N * 64) == cudaSuccess, "cudaMalloc descriptors");
    CHECK(cudaMalloc((void **)&d_m, (size_t)N * sizeof(latch_match)) == cudaSuccess, "cudaMalloc matches");
    cudaMemcpy(d_img, h_img, (size_t)W * H, cudaMemcpyHostToDevice);
    cudaMemcpy(d_kps, h_kps, sizeof h_kps, cudaMemcpyHostToDevice);

    latch_image img = {d_img, W, H, W};
    CHECK(latch_extract(ctx, &img, d_kps, N, NULL, d_desc, NULL) == LATCH_OK, "latch_extract");
    uint8_t *h_desc = (uint8_t *)malloc((size_t)N * 64);
    cudaMemcpy(h_desc, d_desc, (size_t)N * 64, cudaMemcpyDeviceToHost);
    int nonzero = 0;
    for (int i = 0; i < N * 64; ++i) nonzero += h_desc[i] != 0;
    CHECK(nonzero > N * 16, "descriptors look empty");

    const int32_t paths[2] = {LATCH_PATH_POPC, LATCH_PATH_TENSOR};
    latch_match h_m[N];
    for (int p = 0; p < 2; ++p) {
        CHECK(hamming_match(ctx, d_desc, N, d_desc, N, 2, 0.8f, d_m, paths[p], NULL) == LATCH_OK, "hamming_match");
        cudaMemcpy(h_m, d_m, sizeof h_m, cudaMemcpyDeviceToHost);
        for (int i = 0; i < N; ++i) {
            /* a duplicate descriptor would tie at 0 and go to the lower index */
            CHECK(h_m[i].dist1 == 0, "self match distance");
            CHECK(memcmp(h_desc + 64 * (size_t)h_m[i].idx1, h_desc + 64 * (size_t)i, 64) == 0, "self match row");
            CHECK(h_m[i].idx1 <= i, "ties to the lowest index");
        }
    }
    CHECK(latch_check(ctx) == LATCH_OK, "latch_check");

    /* argument errors are status codes with a message, not crashes */
    CHECK(hamming_match(ctx, d_desc, N, d_desc, N, 3, 0.8f, d_m, LATCH_PATH_AUTO, NULL) == LATCH_EINVAL, "k = 3");
    CHECK(latch_last_error(ctx) && latch_last_error(ctx)[0], "error message");

    cudaFree(d_img);
    cudaFree(d_kps);
    cudaFree(d_desc);
    cudaFree(d_m);
    free(h_img);
    free(h_desc);
    CHECK(latch_context_destroy(ctx) == LATCH_OK, "latch_context_destroy");
    printf("ok\n");
    return 0;
}

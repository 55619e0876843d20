/*
 * latch.h -- C ABI of the GB300 LATCH library: oriented, scaled LATCH binary
 * descriptors (Parker et al., "CLATCH", arXiv 1609.03986, Sec. 3) and brute-force
 * Hamming matching with a ratio test (Sec. 4).
 *
 * Conventions for every entry point
 *  - Pointers prefixed d_ are DEVICE pointers owned by the caller; h_ are HOST
 *    pointers owned by the caller.  The library keeps no caller pointer after a
 *    call returns (asynchronous work may still read/write them until the stream
 *    reaches that point).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL means the legacy default
 *    stream) and the call returns without waiting for it.  Argument errors are
 *    detected on the host before anything is enqueued and leave outputs untouched.
 *  - Errors are returned as latch_status; nothing aborts, traps or exits.
 *    latch_last_error() gives a one-line description of the last failure on a
 *    context.  Errors that only the device can see (a keypoint scale index outside
 *    the scale table) set a device-side flag that latch_check() reports.
 *  - A context is bound to one device and is not thread-safe: use one context per
 *    host thread, or serialise calls.  Calls on one context that use its scratch
 *    memory must be ordered (same stream, or synchronised streams).
 */
#ifndef LATCH_H_
#define LATCH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LATCH_OK = 0,
    LATCH_EINVAL = 1,        /* bad argument; nothing was enqueued */
    LATCH_ENOMEM = 2,        /* device or host allocation failed */
    LATCH_ECUDA = 3,         /* a CUDA runtime/driver call failed */
    LATCH_EUNSUPPORTED = 4,  /* device or request not supported by this build */
    LATCH_EBUSY = 5,         /* queue or slots full (session API) */
    LATCH_ETIMEOUT = 6,      /* a bounded wait gave up */
    LATCH_ECANCELLED = 7,    /* request cancelled (session API) */
    LATCH_EDEVICE = 8        /* a kernel reported bad input (see latch_check) */
} latch_status;

/* Opaque library context: device, scale table, triplet table, scratch memory. */
typedef struct latch_context latch_context;

/* cudaStream_t, kept opaque so that this header needs no CUDA header. */
typedef void *latch_stream_t;

/* 8-bit grey image in DEVICE memory: pixel (x, y) is data[y * pitch + x].
 * pitch >= width and pitch % 16 == 0 (the tile loads use the tensor-memory
 * accelerator, whose row strides are multiples of 16 bytes); data 16-byte aligned.
 * 1 <= width, height <= 32768. */
typedef struct {
    const uint8_t *data;
    int32_t width;
    int32_t height;
    int64_t pitch;
} latch_image;

/* Keypoint p = (x, y, theta) of Sec. 3.2 at integer pixel position, with the
 * orientation quantised to one of 32 angle bins (theta = 2*pi*angle_bin/32, taken
 * modulo 32) and a scale given as an index into the context's scale table.
 * Any x, y is allowed: window samples outside the image read 0.  12 bytes. */
typedef struct {
    int32_t x;
    int32_t y;
    uint8_t angle_bin;
    uint8_t scale_idx;
    uint16_t reserved; /* ignored */
} latch_keypoint;

/* One LATCH triplet (Sec. 3.1): centres of the anchor patch P_A and the two
 * companion patches P_1, P_2 in window coordinates (u right, v down, 0..47).
 * Patches are 7x7, so every coordinate must lie in [3, 44]. */
typedef struct {
    uint8_t ax, ay;
    uint8_t c1x, c1y;
    uint8_t c2x, c2y;
} latch_triplet;

/* Result of matching one query (Sec. 4): the nearest train descriptor (idx1,
 * dist1; ties go to the lowest index), the nearest among the others (idx2,
 * dist2), and the ratio-test verdict.  idx = -1 and dist = 65535 when absent.
 * 16 bytes. */
typedef struct {
    int32_t idx1;
    int32_t idx2;
    uint16_t dist1;
    uint16_t dist2;
    uint8_t accepted;
    uint8_t pad[3];
} latch_match;

enum {
    LATCH_DESC_BYTES = 64,  /* 512 bits (Sec. 3.1: 512 triplets; Sec. 3.2: 64-byte vector) */
    LATCH_TRIPLETS = 512,
    LATCH_WINDOW = 48,      /* window side in pixels */
    LATCH_PATCH = 7,        /* patch side in pixels */
    LATCH_MAX_SCALES = 8,
    LATCH_ANGLE_BINS = 32,
    LATCH_DENSE_MAX_RADIUS = 16  /* largest search radius of latch_dense_match */
};

/* Matching paths (both exact). */
enum {
    LATCH_PATH_AUTO = 0,    /* chosen per shape */
    LATCH_PATH_POPC = 1,    /* XOR + population count on the CUDA cores */
    LATCH_PATH_TENSOR = 2   /* bits expanded to +-1 4-bit floats, dot products (512 - 2 Hamming) on the tensor cores */
};

/* Create a context on CUDA device `device` (makes it current on this thread).
 * Default scale table {1, 1.5, 2.25}; no triplet table until one is given.
 * Fails with LATCH_EUNSUPPORTED on a device other than compute capability 10.3. */
latch_status latch_context_create(int device, latch_context **out);

/* Release the context and all device memory it owns.  Waits for its work. */
latch_status latch_context_destroy(latch_context *ctx);

/* Replace the scale table (Sec. 6 names multi-scale extraction; the scale
 * multiplies the sample spacing of the 48x48 window).  1 <= n <= 8, each scale in
 * [0.25, 2.25] (the window then reaches at most 77 pixels from the keypoint).
 * Rebuilds the sample-offset tables: FP64, no contraction, rounded half away from
 * zero.  Synchronous. */
latch_status latch_set_scales(latch_context *ctx, const double *h_scales, int32_t n);

/* Load the 512-triplet table (Sec. 3.1: the triplets are fixed for every
 * keypoint).  Coordinates are checked to lie in [3, 44].  Synchronous.  Each
 * extraction launch carries the table in its parameters, so a call captured in a
 * CUDA graph keeps the table (and the scale table) of its capture: capture again
 * after latch_set_triplets or latch_set_scales. */
latch_status latch_set_triplets(latch_context *ctx, const latch_triplet *h_triplets);

/* Weighted patches (Sec. 3.2, "Weighing pixels in LATCH patches"): with a table of
 * 64 weights, every later extraction on this context compares 8x8 patches, pixel
 * (i, j), i, j = 0..7 (row, column), of the patch centred at (cx, cy) being window
 * pixel (cx - 3 + j, cy - 3 + i) with weight h_weights[8 i + j]:
 *   bit t = sum w (P_A - P_1)^2 > sum w (P_A - P_2)^2   (strict, exact integers).
 * Zero weights on row 7 and column 7 and ones elsewhere give exactly the 7x7
 * descriptor; a Gaussian table weighs the patch centres more.  Triplet coordinates
 * must then lie in [3, 43] (checked now against the loaded table, and on every
 * later table).  NULL returns to the plain 7x7 patches.  Synchronous; as with the
 * triplet table, a captured CUDA graph keeps the weights of its capture. */
latch_status latch_set_patch_weights(latch_context *ctx, const uint8_t *h_weights);

/* Pre-size the context's scratch memory so that later calls up to these sizes
 * allocate nothing (required before capturing calls in a CUDA graph). */
latch_status latch_reserve(latch_context *ctx, int64_t max_keypoints, int64_t max_query, int64_t max_train);

/*
 * LATCH descriptors (Sec. 3.1 Eq. 1; Sec. 3.2).  For keypoint k the 48x48 window
 * is sampled at the keypoint's angle bin and scale (nearest pixel), and bit t of
 * the 512-bit descriptor is 1 iff ||P_A - P_1||^2_F > ||P_A - P_2||^2_F for the 7x7
 * patches of triplet t (strict).  Bit t is bit (t % 8) of byte t / 8.
 *   img        image in device memory (see latch_image)
 *   d_kps      n keypoints in device memory
 *   h_triplets 512 triplets in host memory, or NULL to use the context's table;
 *              a new table is loaded as by latch_set_triplets
 *   d_out      n * 64 bytes, device memory, 16-byte aligned
 * n == 0 is a no-op.  A keypoint whose scale_idx is outside the scale table gets
 * an all-zero descriptor and raises the device flag reported by latch_check.
 */
latch_status latch_extract(latch_context *ctx, const latch_image *img, const latch_keypoint *d_kps, int32_t n,
                           const latch_triplet *h_triplets, uint8_t *d_out, latch_stream_t stream);

/*
 * Oriented keypoints (Sec. 3.2: the keypoints come from the FAST detector, and each
 * keypoint's orientation sets the angle at which its window is read).  The paper
 * names the detector only; this library reads it as:
 *   - FAST-9: the 16 pixels of the radius-3 Bresenham circle around p; p is a corner
 *     at `threshold` t when 9 contiguous of them (circularly) are all > I(p) + t or
 *     all < I(p) - t;
 *   - score: the largest t' >= t at which p is still a corner;
 *   - a corner is kept when its score is strictly larger than each of its 8
 *     neighbours' scores (equal neighbours suppress each other);
 *   - only pixels at least 16 from every border are detected;
 *   - angle_bin = round_half_away(theta * 16 / pi) mod 32 with theta = atan2(m01,
 *     m10) of the intensity centroid of the disc dx^2 + dy^2 <= 15^2 (FP64; x right,
 *     y down, the frame of the window rotation); scale_idx = `scale_idx`.
 * Keypoints are written in 32x32-pixel cell order (cells row by row from the image
 * origin, then row by row inside a cell), the first max_kps of them.
 *   img        image in device memory (see latch_image)
 *   threshold  1..254;  scale_idx: index into the scale table, given to every keypoint
 *   d_kps      device out: min(count, max_kps) keypoints
 *   d_count    device out: one int32, the number of keypoints found (may exceed max_kps)
 * Asynchronous like every call; read *d_count after synchronising the stream.
 */
latch_status latch_detect(latch_context *ctx, const latch_image *img, int32_t threshold, int32_t scale_idx,
                          int32_t max_kps, latch_keypoint *d_kps, int32_t *d_count, latch_stream_t stream);

/* latch_detect, then the descriptors of the keypoints it wrote (as latch_extract on
 * d_kps[0 .. min(count, max_kps)) with the context's triplet table), without a host
 * round trip: the extraction reads the count from d_count.  d_desc: max_kps * 64
 * bytes, 16-byte aligned; rows from min(count, max_kps) on are left untouched. */
latch_status latch_detect_extract(latch_context *ctx, const latch_image *img, int32_t threshold, int32_t scale_idx,
                                  int32_t max_kps, latch_keypoint *d_kps, int32_t *d_count, uint8_t *d_desc,
                                  latch_stream_t stream);

/* Multi-scale keypoints (Sec. 6: CLATCH extracted at multiple scales; FAST alone has
 * no scale).  Reading: pyramid level l uses the context's scale s_l = scale table
 * entry l (l < n_levels; each must be >= 1): the level image is the input sampled
 * at spacing s_l, I_l(x, y) = I(round_half_away(s_l x), round_half_away(s_l y)) for
 * x < floor(W / s_l), y < floor(H / s_l), the nearest-pixel rule of the scaled
 * window.  Keypoints are detected on every level as by latch_detect (orientation
 * from the level image), and a level keypoint (x, y) is written as
 * (round_half_away(s_l x), round_half_away(s_l y)) with scale_idx = l: its
 * descriptor then samples the input at the same spacing s_l.  Levels follow one
 * another (level 0 first), each in the cell order of its own image; the first
 * max_kps are written and *d_count receives the total.  d_desc: NULL, or max_kps * 64
 * bytes (16-byte aligned) that receive the descriptors as latch_detect_extract does,
 * with no host round trip. */
latch_status latch_detect_pyramid(latch_context *ctx, const latch_image *img, int32_t threshold, int32_t n_levels,
                                  int32_t max_kps, latch_keypoint *d_kps, int32_t *d_count, uint8_t *d_desc,
                                  latch_stream_t stream);

/*
 * Brute-force Hamming matching (Sec. 4): for every query descriptor the nearest
 * train descriptor and, for k == 2, the nearest among the others, with the ratio
 * test accepted = (1000 * dist1 < r * dist2), r = round_half_away(1000 * ratio).
 * For k == 1 a found match is always accepted.
 *   d_query  nq * 64 bytes, d_train nt * 64 bytes (device, 16-byte aligned)
 *   k        1 or 2;  ratio in [0, 1]
 *   d_out    nq latch_match records (device)
 *   path     LATCH_PATH_AUTO / _POPC / _TENSOR (all give identical results)
 * nq == 0 is a no-op; nt == 0 gives idx = -1, dist = 65535, accepted = 0.
 */
latch_status hamming_match(latch_context *ctx, const uint8_t *d_query, int32_t nq, const uint8_t *d_train,
                           int32_t nt, int32_t k, float ratio, latch_match *d_out, int32_t path,
                           latch_stream_t stream);

/*
 * Dense per-pixel LATCH (Sec. 6: CLATCH for dense pixel matching, an alternative to
 * PatchMatch).  Reading: every pixel (x, y) of `img` is a keypoint at angle bin 0
 * and scale 1 (window pixel (u, v) = image pixel (x + u - 24, y + v - 24), 0
 * outside the image) with the context's 7x7 triplet table; descriptors are written
 * in raster order, row y * width + x.
 *   d_out    width * height * 64 bytes (device, 16-byte aligned)
 * LATCH_EUNSUPPORTED when the context uses weighted 8x8 patches.
 */
latch_status latch_dense_extract(latch_context *ctx, const latch_image *img, uint8_t *d_out, latch_stream_t stream);

/*
 * Windowed matching of two dense descriptor fields of the same size (Sec. 6):
 * pixel p of A is matched against the pixels q of B with |q.x - p.x| <= radius and
 * |q.y - p.y| <= radius that lie inside B, in raster order of B, with the rule of
 * hamming_match (nearest, second nearest among the others, ties to the lowest
 * index, ratio test); idx1 / idx2 are raster indices y * width + x in B.
 *   d_a, d_b width * height * 64 bytes each (device, 16-byte aligned)
 *   radius   0 .. LATCH_DENSE_MAX_RADIUS;  k 1 or 2;  ratio in [0, 1]
 *   d_out    width * height latch_match records (device)
 * Radius 0 (or a 1-pixel image) leaves no second candidate: idx2 = -1, dist2 = 65535.
 */
latch_status latch_dense_match(latch_context *ctx, const uint8_t *d_a, const uint8_t *d_b, int32_t width,
                               int32_t height, int32_t radius, int32_t k, float ratio, latch_match *d_out,
                               latch_stream_t stream);

/* A batch of images, each matched against others (the structure-from-motion
 * pattern of Sec. 4-5: every image against its neighbours in sequence).
 * Keypoints and descriptors of all images are concatenated image by image: image i
 * owns rows [o_i, o_i + h_n_kps[i]) with o_i = sum of the earlier counts.  Matches
 * are concatenated pair by pair: pair p owns h_n_kps[query image of p] records
 * starting at the sum of the earlier pairs' query counts; train indices in a
 * record are relative to the train image. */
typedef struct {
    int32_t n_images;
    const latch_image *h_images;     /* host array [n_images] of device images */
    const int32_t *h_n_kps;          /* host array [n_images]: keypoints per image */
    const latch_keypoint *d_kps;     /* device: all keypoints, image by image */
    uint8_t *d_desc;                 /* device out: 64 bytes per keypoint, same order */
    int32_t n_pairs;
    const int32_t *h_pairs;          /* host array [2 * n_pairs]: (query image, train image) */
    int32_t k;                       /* 1 or 2 */
    float ratio;                     /* in [0, 1] */
    latch_match *d_matches;          /* device out: see above */
} latch_batch_desc;

/* Size the context's batch scratch for `batch` (same shapes later allocate
 * nothing; required before capturing latch_batch_run in a CUDA graph). */
latch_status latch_reserve_batch(latch_context *ctx, const latch_batch_desc *batch);

/* Extract every image's descriptors (as latch_extract, with the context's triplet
 * and scale tables) and match every pair (as hamming_match on the tensor-core
 * path), enqueued on `stream` as a few batched persistent launches.  Results are
 * identical to calling latch_extract and hamming_match one by one. */
latch_status latch_batch_run(latch_context *ctx, const latch_batch_desc *batch, latch_stream_t stream);

/* The batch of latch_batch_run with every buffer in host memory (pinned memory,
 * cudaHostAlloc / cudaHostRegister, makes the copies asynchronous; pageable memory
 * works but serialises them).  Layouts as in latch_batch_desc. */
typedef struct {
    int32_t n_images;
    const latch_image *h_images;     /* host array [n_images] of HOST images (any pitch >= width) */
    const int32_t *h_n_kps;          /* host array [n_images]: keypoints per image */
    const latch_keypoint *h_kps;     /* host: all keypoints, image by image */
    uint8_t *h_desc;                 /* host out, 64 bytes per keypoint; NULL: not copied back */
    int32_t n_pairs;
    const int32_t *h_pairs;          /* host array [2 * n_pairs]: (query image, train image) */
    int32_t k;                       /* 1 or 2 */
    float ratio;                     /* in [0, 1] */
    latch_match *h_matches;          /* host out */
} latch_host_batch_desc;

/* latch_batch_run from and to host memory (the end-to-end form of Sec. 4's
 * pipeline: upload, extract, match, download).  Enqueued without synchronising:
 * the inputs are copied into one of two device staging sets owned by the context
 * (alternating per call, grown on demand) on the context's upload stream, then the
 * batch and the copies of the outputs back to host memory run on `stream`, so once
 * `stream` is synchronised the host outputs are valid.  The host inputs must stay unchanged, and the outputs
 * unread, until then.  Consecutive calls overlap: the upload of call i+1 runs while
 * call i computes.  A call that must grow a staging set first waits for that set's
 * previous use.  Errors as latch_batch_run. */
latch_status latch_batch_run_host(latch_context *ctx, const latch_host_batch_desc *batch, latch_stream_t stream);

/* ---- Serving session: extract-and-match requests against resident galleries ----
 *
 * A session owns a context, an HBM budget and a host scheduler thread.  Galleries
 * (descriptor sets) are copied in once and stay on the device, pre-expanded for
 * the tensor-core matcher.  Requests are queued by latch_submit and run with
 * continuous batching: whenever one of the session's two lanes is free, the
 * requests at the head of the queue that fit the lane (count, keypoints and the
 * lane's share of the HBM budget) are admitted together and run as one batched
 * extraction and one batched match; the two lanes run concurrently on their own
 * streams.  Each result is bit-identical to latch_extract + hamming_match on that
 * request alone.  All session calls are thread-safe. */
typedef struct latch_session latch_session;

typedef struct {
    const uint8_t *h_image;          /* host image, row pitch `pitch` bytes (any pitch >= width) */
    int32_t width, height;
    int64_t pitch;
    const latch_keypoint *h_kps;     /* host keypoints */
    int32_t n;
    int32_t gallery_id;              /* from latch_gallery_add */
    int32_t k;                       /* 1 or 2 */
    float ratio;                     /* in [0, 1] */
    latch_match *h_matches;          /* host out: n records */
    uint8_t *h_desc;                 /* host out: n * 64 bytes, or NULL */
} latch_request;                     /* all host buffers must stay valid until latch_wait returns */

typedef struct {
    latch_status status;
    int32_t n;
    int32_t batch_size;              /* requests in the micro-batch this one ran in */
    double submit_s, start_s, done_s;  /* seconds on the session clock: queued, admitted, completed */
} latch_result;

typedef struct {
    int64_t submitted, completed, rejected, failed, batches, max_queue, queued, lane_bytes;
    int64_t hbm_free;    /* free device bytes measured (cudaMemGetInfo) when the session was created */
    int64_t hbm_budget;  /* device bytes the session holds: min(hbm_budget, hbm_free - 512 MiB) */
} latch_session_stats;

/* hbm_budget: device bytes the session may hold (arena of max_gallery_rows +
 * lanes x max_batch_kps expanded rows, the rest split between the lanes; each lane
 * needs at least 64 MB).  The budget is clamped to the free device memory measured
 * at creation less 512 MiB, and the session reserves all of it then, so admission
 * (latch_submit, and the scheduler filling a lane) is against memory that is really
 * free.  max_batch: requests per micro-batch (1..64); max_batch_kps: keypoints per
 * micro-batch; h_triplets: the 512-triplet table.
 * A batch's kernels report device-side failures through a per-lane error word that
 * completes its tickets: latch_wait then returns LATCH_ETIMEOUT (a bounded device
 * wait gave up; results incomplete) or LATCH_EDEVICE. */
latch_status latch_session_create(int device, size_t hbm_budget, int64_t max_gallery_rows, int32_t max_batch,
                                  int64_t max_batch_kps, const latch_triplet *h_triplets, latch_session **out);
/* As latch_session_create with `lanes` (1..8) lanes instead of 2: micro-batches that
 * run concurrently, each on its own stream with its own share of the budget. */
latch_status latch_session_create_lanes(int device, size_t hbm_budget, int64_t max_gallery_rows, int32_t max_batch,
                                        int64_t max_batch_kps, int32_t lanes, const latch_triplet *h_triplets,
                                        latch_session **out);
/* Stops the scheduler, waits for work in flight, frees everything. */
latch_status latch_session_destroy(latch_session *s);
/* Copy n packed descriptors (host) into a new resident gallery (synchronous). */
latch_status latch_gallery_add(latch_session *s, const uint8_t *h_desc, int32_t n, int32_t *gallery_id);
/* Queue a request; LATCH_ENOMEM if it can never fit a lane, LATCH_EINVAL on bad
 * arguments, an unknown gallery or a keypoint whose scale_idx is outside the scale
 * table (checked on the host, so that the micro-batch the request would share stays
 * valid).  Returns at once. */
latch_status latch_submit(latch_session *s, const latch_request *req, uint64_t *ticket);
/* Wait for a ticket (timeout_ms < 0: forever); LATCH_ETIMEOUT if still running.
 * On completion the request's host outputs are filled. */
latch_status latch_wait(latch_session *s, uint64_t ticket, int32_t timeout_ms, latch_result *out);
/* Forget a completed ticket. */
latch_status latch_release(latch_session *s, uint64_t ticket);
latch_status latch_session_get_stats(latch_session *s, latch_session_stats *out);
const char *latch_session_last_error(const latch_session *s);

/* ---- Autotuning (tile shapes and path choice, by measurement on this device) ---- */
typedef struct {
    int32_t item_kps;           /* extraction: fewest keypoints per block (sets the grid), 1..32 */
    int64_t tensor_min_pairs;   /* matching: LATCH_PATH_AUTO uses the tensor cores from nq*nt >= this */
} latch_tuning;

typedef struct {
    int32_t width, height;      /* representative image size */
    int32_t n_keypoints;        /* keypoints per image (0: skip the extraction tuning) */
    int32_t n_query, n_train;   /* representative matching shape (0: skip the matching tuning) */
} latch_tune_shape;

/* Measure the candidate extraction work-item sizes and the matching paths on
 * synthetic device data of this shape and keep the fastest in the context; results
 * do not change (all candidates compute identical outputs), only speed.  Synchronous;
 * allocates temporary device memory.  `out` (may be NULL) receives the choice. */
latch_status latch_autotune(latch_context *ctx, const latch_tune_shape *shape, latch_tuning *out);
latch_status latch_get_tuning(const latch_context *ctx, latch_tuning *out);
latch_status latch_set_tuning(latch_context *ctx, const latch_tuning *tuning);

/* The path LATCH_PATH_AUTO takes for nq x nt on this context (LATCH_PATH_POPC or
 * LATCH_PATH_TENSOR); -1 on a NULL context. */
int32_t hamming_match_path(const latch_context *ctx, int64_t nq, int64_t nt);

/*
 * hamming_match without any device allocation: same results as hamming_match on
 * the tensor-core path, for callers that must not allocate device memory (for
 * example a host application that owns all HBM through its own pool, or a
 * latency-bound pipeline in which a cudaMalloc would synchronise the device).  The
 * paper has no counterpart; this is an interface convenience.
 *   Uses the current device and no context.  Scratch lives in one 16 MiB array
 *   that the library's CUDA module reserves on every device it is loaded on until
 *   the process exits; a request whose scratch would not fit (roughly nq + nt above
 *   30,000 descriptors) returns LATCH_EINVAL and enqueues nothing.
 *   The first call on a device looks up the array's device address (once per
 *   device); make that first call before any stream capture.
 *   All calls share the one array: calls whose work overlaps on the GPU (different
 *   streams, or several host threads) race and must be serialised by the caller.
 *   Errors are described by latch_last_error(NULL); failures that only the device
 *   sees are reported by hamming_match_noalloc_status().
 */
latch_status hamming_match_noalloc(const uint8_t *d_query, int32_t nq, const uint8_t *d_train, int32_t nt, int32_t k,
                                   float ratio, latch_match *d_out, latch_stream_t stream);

/* Device-side status of hamming_match_noalloc on the current device (the paper has
 * no counterpart).  The kernels of every hamming_match_noalloc call OR their error
 * flags into one status word at the head of the fixed array, which stays set until
 * this call reads it.  Waits for all work on the current device, reads the word and
 * clears it: LATCH_OK when no call since the last read reported a problem,
 * LATCH_ETIMEOUT when a bounded device-side wait gave up (those calls' records are
 * incomplete).  Allocates nothing. */
latch_status hamming_match_noalloc_status(void);

/* Wait for all work on the context's device, then report (and clear) a
 * device-side input error (LATCH_EDEVICE) or an asynchronous CUDA error. */
latch_status latch_check(latch_context *ctx);

/* Failure-detection self-test (no counterpart in the paper): enqueue a kernel whose
 * bounded device-side wait can never be satisfied, so that after limit_us
 * microseconds (1 .. 2e6) it gives up and raises the context's timeout flag, the
 * path every pipeline wait of the library takes.  The next latch_check returns
 * LATCH_ETIMEOUT (and clears the flag); the context stays usable. */
latch_status latch_selftest_wait_timeout(latch_context *ctx, int32_t limit_us, latch_stream_t stream);

/* Tracing (no counterpart in the paper): with max_records > 0, each
 * latch_batch_run on this context records CUDA events on its stream before
 * extraction, between extraction and matching, and after matching, until
 * max_records runs are recorded (0 disables and frees the events).  Synchronous. */
latch_status latch_trace_enable(latch_context *ctx, int32_t max_records);
/* Waits for the recorded runs, writes per run [extraction ms, matching ms] into
 * out_ms (2 * capacity floats), the number of runs into *n, and starts over. */
latch_status latch_trace_collect(latch_context *ctx, float *out_ms, int32_t capacity, int32_t *n);

/* One-line description of the last error on `ctx` (or of the last failed
 * latch_context_create when ctx is NULL).  Valid until the next call. */
const char *latch_last_error(const latch_context *ctx);

/* Number of CUDA kernels the library has launched in this process (all contexts),
 * for accounting in benchmarks. */
uint64_t latch_kernel_launches(void);

/* Library version string. */
const char *latch_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LATCH_H_ */

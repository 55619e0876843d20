// Serving session: extract-and-match requests against device-resident descriptor
// sets ("galleries"), with continuous batching.
//
// Host side, one scheduler thread.  Requests wait in a FIFO.  Whenever one of the
// session's lanes (2 by default, up to 8) is free, the scheduler takes requests from the head of the
// queue for as long as they fit the lane (count, keypoints, and the lane's share of
// the HBM budget -- admission by free device memory) and enqueues them on the
// lane's stream as one micro-batch:
//   host -> device copies of every image and keypoint set,
//   one batched extraction over all the batch's images,
//   one expansion of the new descriptors into the lane's rows of the session arena,
//   one batched tensor-core match of every request against its gallery (the
//   galleries sit pre-expanded in the same arena, so one TMA map covers both),
//   device -> host copies of the matches (and descriptors if asked for),
//   a host callback that completes the batch's tickets.
// The lanes take turns, so a batch's copies and kernels overlap the other
// lanes', and requests that arrive while a batch runs are admitted into the next
// one as soon as a lane frees up.  Results are bit-identical to latch_extract +
// hamming_match on each request alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "match_common.cuh"

namespace latch {
namespace {

constexpr int kMaxLanes = 8;
constexpr int64_t kRowBytes = kExpRowBytes;  // expanded row
constexpr size_t kFreeMargin = size_t(512) << 20;  // device memory left free at session creation

struct Ticket {
    latch_request req;
    uint64_t id;
    latch_status status = LATCH_OK;
    bool done = false;
    double t_submit = 0, t_start = 0, t_done = 0;
    int32_t batch_size = 0;
    size_t bytes = 0;  // lane bytes this request needs
};

struct Gallery {
    int64_t row0;
    int32_t n;
};

struct DoneArg {
    latch_session* s;
    int lane;
};

struct Lane {
    cudaStream_t stream = nullptr;
    DoneArg done{nullptr, 0};  // argument of the lane's completion callback
    uint8_t* region = nullptr;  // lane_bytes of device memory
    uint32_t* d_flags = nullptr;  // the lane's device error word, cleared at the start of each batch
    uint32_t* h_flags = nullptr;  // pinned host copy, written at the end of each batch
    int64_t qrow0 = 0;          // first arena row of this lane's query rows
    bool busy = false;
    std::vector<Ticket*> batch;
    MatchBatch* mb = nullptr;
};

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int64_t dev_pitch(int32_t width) { return (static_cast<int64_t>(width) + 15) / 16 * 16; }

}  // namespace
}  // namespace latch

struct latch_session {
    latch_context* ctx = nullptr;
    int32_t max_batch = 0;
    int64_t max_batch_kps = 0;
    size_t lane_bytes = 0;
    size_t budget = 0;  // device bytes the session holds: min(caller's budget, free memory - margin)
    // arena: [gallery rows | lane 0 query rows | lane 1 query rows | ...] x kExpRowBytes
    uint8_t* arena = nullptr;
    int64_t arena_rows = 0;
    int64_t gallery_cap = 0;
    int64_t gallery_used = 0;
    std::vector<latch::Gallery> galleries;
    int nlanes = 0;
    latch::Lane lanes[latch::kMaxLanes];
    std::mutex mu;
    std::condition_variable cv_sched;  // scheduler: new work or a free lane
    std::condition_variable cv_done;   // waiters: a ticket completed
    std::deque<latch::Ticket*> queue;
    std::unordered_map<uint64_t, latch::Ticket*> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    latch_session_stats stats{};
    char err[256] = {};
};

namespace latch {
namespace {

double now_s(const latch_session* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

latch_status sfail(latch_session* s, latch_status st, const char* msg) {
    if (s) snprintf(s->err, sizeof(s->err), "%s", msg);
    return st;
}

// Device bytes one request needs in a lane (image, keypoints, descriptors, matches,
// its share of the extraction scratch) -- the partial records of the match are
// budgeted per batch.
size_t request_bytes(const latch_request& r) {
    const latch_image img{nullptr, r.width, r.height, dev_pitch(r.width)};
    return round_up(static_cast<size_t>(r.height) * dev_pitch(r.width), 256) +
           round_up(static_cast<size_t>(r.n) * (12 + 64 + 16), 256) + extract_scratch_bytes(&img, r.n) + 1024;
}

struct Carve {
    uint8_t* base;
    size_t used = 0, cap;
    uint8_t* take(size_t bytes) {
        uint8_t* p = base + used;
        used += round_up(bytes, 256);
        return used <= cap ? p : nullptr;
    }
};

void CUDART_CB on_batch_done(void* arg);

// Enqueue lane `li`'s batch on its stream.  Called by the scheduler without the lock.
latch_status run_batch(latch_session* s, int li, DoneArg* done) {
    Lane& L = s->lanes[li];
    cudaStream_t st = L.stream;
    const int nb = static_cast<int>(L.batch.size());
    Carve cv{L.region, 0, s->lane_bytes};
    std::vector<latch_image> imgs(nb);
    std::vector<int64_t> kp0(nb), n(nb);
    int64_t total = 0;
    for (int i = 0; i < nb; ++i) {
        n[i] = L.batch[i]->req.n;
        kp0[i] = total;
        total += n[i];
    }
    latch_keypoint* d_kps = reinterpret_cast<latch_keypoint*>(cv.take(std::max<int64_t>(total, 1) * 12));
    uint8_t* d_desc = cv.take(std::max<int64_t>(total, 1) * 64);
    latch_match* d_match = reinterpret_cast<latch_match*>(cv.take(std::max<int64_t>(total, 1) * 16));
    if (!d_kps || !d_desc || !d_match) return LATCH_ENOMEM;  // admission bug guard
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        const latch_request& r = L.batch[i]->req;
        const int64_t pitch = dev_pitch(r.width);
        uint8_t* d_img = cv.take(static_cast<size_t>(r.height) * pitch);
        if (!d_img) return LATCH_ENOMEM;  // admission bug guard
        imgs[i] = latch_image{d_img, r.width, r.height, pitch};
        e = cudaMemcpy2DAsync(d_img, pitch, r.h_image, r.pitch, r.width, r.height, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && r.n > 0)
            e = cudaMemcpyAsync(d_kps + kp0[i], r.h_kps, static_cast<size_t>(r.n) * 12, cudaMemcpyHostToDevice, st);
    }
    const size_t ext_bytes = extract_batch_scratch_bytes(imgs.data(), n.data(), nb);
    uint8_t* ext_scratch = cv.take(ext_bytes);
    // match problems: request i's query rows -> its gallery
    MatchBatch* mb = L.mb;
    for (int i = 0; i < nb; ++i) {
        const latch_request& r = L.batch[i]->req;
        MatchProblem& P = mb->p[i];
        P.q_row0 = static_cast<int32_t>(L.qrow0 + kp0[i]);
        P.t_row0 = static_cast<int32_t>(s->galleries[r.gallery_id].row0);
        P.nq = r.n;
        P.nt = s->galleries[r.gallery_id].n;
        P.out0 = static_cast<int32_t>(kp0[i]);
        P.k = r.k;
        P.r_milli = static_cast<int32_t>(std::round(static_cast<double>(r.ratio) * 1000.0));
    }
    plan_match_batch(mb, nb, s->ctx->sm_count);
    uint64_t* partials = reinterpret_cast<uint64_t*>(cv.take(match_tc_partial_bytes(*mb) + 16));
    int32_t* tile_cnt = reinterpret_cast<int32_t*>(cv.take(match_tc_counter_bytes(mb->tiles)));
    if (!ext_scratch || !partials || !tile_cnt) e = cudaErrorMemoryAllocation;  // admission bug guard
    if (e == cudaSuccess) e = cudaMemsetAsync(L.d_flags, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess && total > 0) e = cudaMemsetAsync(tile_cnt, 0, match_tc_counter_bytes(mb->tiles), st);
    // the extraction writes the queries' expanded rows into the lane's arena rows
    if (e == cudaSuccess && total > 0)
        e = launch_extract_batch(s->ctx, imgs.data(), kp0.data(), n.data(), nb, d_kps, d_desc, ext_scratch, st,
                                 s->arena + L.qrow0 * kExpRowBytes, L.d_flags);
    if (e == cudaSuccess && total > 0)
        e = launch_match_tc_rows(*mb, s->arena, s->arena_rows, partials, tile_cnt, d_match, L.d_flags, st);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        const latch_request& r = L.batch[i]->req;
        if (r.n == 0) continue;
        e = cudaMemcpyAsync(r.h_matches, d_match + kp0[i], static_cast<size_t>(r.n) * 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && r.h_desc)
            e = cudaMemcpyAsync(r.h_desc, d_desc + kp0[i] * 64, static_cast<size_t>(r.n) * 64, cudaMemcpyDeviceToHost,
                                st);
    }
    // the batch's device error word reaches the completion callback through pinned memory
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.h_flags, L.d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_batch_done, done);
    if (e == cudaErrorMemoryAllocation) return LATCH_ENOMEM;
    return e == cudaSuccess ? LATCH_OK : LATCH_ECUDA;
}

void finish_lane(latch_session* s, int li, latch_status status) {
    // caller holds the lock
    Lane& L = s->lanes[li];
    const double t = now_s(s);
    for (Ticket* tk : L.batch) {
        tk->done = true;
        tk->status = status;
        tk->t_done = t;
        if (status == LATCH_OK)
            ++s->stats.completed;
        else
            ++s->stats.failed;
    }
    L.batch.clear();
    L.busy = false;
}

// Status of a finished batch from its device error word: a device-side wait that
// gave up (the batch's results are incomplete) or bad input seen by a kernel.
latch_status batch_status(uint32_t flags) {
    if (flags & kFlagTimeout) return LATCH_ETIMEOUT;
    return flags ? LATCH_EDEVICE : LATCH_OK;
}

void CUDART_CB on_batch_done(void* arg) {
    DoneArg* d = static_cast<DoneArg*>(arg);
    latch_session* s = d->s;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const uint32_t flags = *s->lanes[d->lane].h_flags;  // copied before this callback on the lane's stream
        if (flags) snprintf(s->err, sizeof(s->err), "lane %d: device error word 0x%x", d->lane, flags);
        finish_lane(s, d->lane, batch_status(flags));
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
}

void scheduler(latch_session* s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        int li = -1;
        s->cv_sched.wait(lock, [&] {
            if (s->stop) return true;
            if (s->queue.empty()) return false;
            for (int i = 0; i < s->nlanes; ++i)
                if (!s->lanes[i].busy) {
                    li = i;
                    return true;
                }
            return false;
        });
        if (s->stop) break;
        // form a micro-batch from the head of the queue
        Lane& L = s->lanes[li];
        size_t bytes = 0;
        int64_t kps = 0;
        const double t = now_s(s);
        while (!s->queue.empty() && static_cast<int>(L.batch.size()) < s->max_batch) {
            Ticket* tk = s->queue.front();
            // per-batch partial records and arrival counters
            const size_t part = match_tc_partial_bound(kps + tk->req.n, static_cast<int64_t>(L.batch.size()) + 1,
                                                       s->ctx->sm_count) + 512;
            if (kps + tk->req.n > s->max_batch_kps || bytes + tk->bytes + part > s->lane_bytes) break;
            s->queue.pop_front();
            bytes += tk->bytes;
            kps += tk->req.n;
            tk->t_start = t;
            L.batch.push_back(tk);
        }
        for (Ticket* tk : L.batch) tk->batch_size = static_cast<int32_t>(L.batch.size());
        ++s->stats.batches;
        L.busy = true;
        lock.unlock();
        const latch_status st = run_batch(s, li, &L.done);
        lock.lock();
        if (st != LATCH_OK) {
            // nothing was left pending on the stream that refers to this batch's tickets
            cudaStreamSynchronize(L.stream);
            finish_lane(s, li, st);
            s->cv_done.notify_all();
        }
    }
}

}  // namespace
}  // namespace latch

using namespace latch;

extern "C" {

latch_status latch_session_create(int device, size_t hbm_budget, int64_t max_gallery_rows, int32_t max_batch,
                                  int64_t max_batch_kps, const latch_triplet* h_triplets, latch_session** out) {
    return latch_session_create_lanes(device, hbm_budget, max_gallery_rows, max_batch, max_batch_kps, 2, h_triplets,
                                      out);
}

latch_status latch_session_create_lanes(int device, size_t hbm_budget, int64_t max_gallery_rows, int32_t max_batch,
                                        int64_t max_batch_kps, int32_t lanes, const latch_triplet* h_triplets,
                                        latch_session** out) {
    if (!out || !h_triplets) return LATCH_EINVAL;
    *out = nullptr;
    if (lanes < 1 || lanes > kMaxLanes || max_batch < 1 || max_batch > 64 || max_batch_kps < 1 ||
        max_gallery_rows < 1 || max_gallery_rows + lanes * max_batch_kps > INT32_MAX / 2)
        return LATCH_EINVAL;
    latch_session* s = new (std::nothrow) latch_session();
    if (!s) return LATCH_ENOMEM;
    s->nlanes = lanes;
    s->t0 = std::chrono::steady_clock::now();
    latch_status st = latch_context_create(device, &s->ctx);
    if (st == LATCH_OK) st = latch_set_triplets(s->ctx, h_triplets);
    s->max_batch = max_batch;
    s->max_batch_kps = max_batch_kps;
    s->gallery_cap = max_gallery_rows;
    s->arena_rows = max_gallery_rows + lanes * max_batch_kps;
    const size_t arena_bytes = static_cast<size_t>(s->arena_rows) * kRowBytes + 4096;
    // admission by free device memory: the session never holds more than the device
    // has free when it is created, less a margin for the context's own tables and
    // scratch; every request is then admitted against this reservation
    size_t free_b = 0, total_b = 0;
    if (st == LATCH_OK && cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) st = LATCH_ECUDA;
    if (st == LATCH_OK) {
        const size_t usable = free_b > kFreeMargin ? free_b - kFreeMargin : 0;
        s->budget = hbm_budget < usable ? hbm_budget : usable;
        s->stats.hbm_free = static_cast<int64_t>(free_b);
        s->stats.hbm_budget = static_cast<int64_t>(s->budget);
    }
    if (st == LATCH_OK && (s->budget <= arena_bytes || (s->budget - arena_bytes) / lanes < (size_t(64) << 20)))
        st = LATCH_ENOMEM;  // budget (or free memory) too small for the arena plus lanes of 64 MB
    if (st == LATCH_OK) {
        s->lane_bytes = (s->budget - arena_bytes) / lanes / 256 * 256;
        if (cudaMalloc(&s->arena, arena_bytes) != cudaSuccess) st = LATCH_ENOMEM;
    }
    if (st == LATCH_OK) {
        for (int i = 0; i < lanes && st == LATCH_OK; ++i) {
            Lane& L = s->lanes[i];
            L.qrow0 = max_gallery_rows + i * max_batch_kps;
            L.done = DoneArg{s, i};
            L.mb = new (std::nothrow) MatchBatch;
            if (!L.mb || cudaMalloc(&L.region, s->lane_bytes) != cudaSuccess ||
                cudaMalloc(&L.d_flags, 256) != cudaSuccess ||
                cudaHostAlloc(&L.h_flags, sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess ||
                cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess)
                st = LATCH_ENOMEM;
            else
                *L.h_flags = 0;
        }
    }
    if (st != LATCH_OK) {
        latch_session_destroy(s);
        return st;
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return LATCH_OK;
}

latch_status latch_session_destroy(latch_session* s) {
    if (!s) return LATCH_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->ctx) cudaSetDevice(s->ctx->device);
    for (Lane& L : s->lanes) {
        if (L.stream) {
            cudaStreamSynchronize(L.stream);
            cudaStreamDestroy(L.stream);
        }
        if (L.region) cudaFree(L.region);
        if (L.d_flags) cudaFree(L.d_flags);
        if (L.h_flags) cudaFreeHost(L.h_flags);
        delete L.mb;
    }
    if (s->arena) cudaFree(s->arena);
    for (auto& kv : s->tickets) delete kv.second;
    for (Ticket* t : s->queue)
        if (!s->tickets.count(t->id)) delete t;
    if (s->ctx) latch_context_destroy(s->ctx);
    delete s;
    return LATCH_OK;
}

latch_status latch_gallery_add(latch_session* s, const uint8_t* h_desc, int32_t n, int32_t* gallery_id) {
    if (!s || !gallery_id || n < 0 || (n > 0 && !h_desc)) return sfail(s, LATCH_EINVAL, "bad gallery arguments");
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->gallery_used + n > s->gallery_cap) return sfail(s, LATCH_ENOMEM, "gallery rows exceed the session's capacity");
    LATCH_CUDA_TRY(s->ctx, cudaSetDevice(s->ctx->device));
    uint8_t* tmp = nullptr;
    if (n > 0) {
        // packed descriptors -> expanded arena rows (synchronous; galleries are added between requests)
        if (cudaMalloc(&tmp, static_cast<size_t>(n) * 64) != cudaSuccess) return sfail(s, LATCH_ENOMEM, "cudaMalloc");
        cudaError_t e = cudaMemcpy(tmp, h_desc, static_cast<size_t>(n) * 64, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_expand(tmp, n, s->arena + s->gallery_used * kExpRowBytes, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(tmp);
        if (e != cudaSuccess) return sfail(s, LATCH_ECUDA, cudaGetErrorString(e));
    }
    *gallery_id = static_cast<int32_t>(s->galleries.size());
    s->galleries.push_back(Gallery{s->gallery_used, n});
    s->gallery_used += n;
    return LATCH_OK;
}

latch_status latch_submit(latch_session* s, const latch_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return sfail(s, LATCH_EINVAL, "NULL argument");
    if (r->width < 1 || r->height < 1 || r->width > 32768 || r->height > 32768 || r->pitch < r->width || !r->h_image)
        return sfail(s, LATCH_EINVAL, "bad image");
    if (r->n < 0 || (r->n > 0 && (!r->h_kps || !r->h_matches))) return sfail(s, LATCH_EINVAL, "bad keypoints or output");
    if (r->k != 1 && r->k != 2) return sfail(s, LATCH_EINVAL, "k must be 1 or 2");
    if (!(r->ratio >= 0.0f && r->ratio <= 1.0f)) return sfail(s, LATCH_EINVAL, "ratio not in [0, 1]");
    // a keypoint with a scale index outside the scale table is refused here, so that it
    // cannot spoil the micro-batch it would share with other requests
    for (int32_t i = 0; i < r->n; ++i)
        if (r->h_kps[i].scale_idx >= s->ctx->nscales) {
            std::lock_guard<std::mutex> lock(s->mu);
            ++s->stats.rejected;
            return sfail(s, LATCH_EINVAL, "keypoint scale index outside the scale table");
        }
    Ticket* tk = new (std::nothrow) Ticket;
    if (!tk) return sfail(s, LATCH_ENOMEM, "host allocation failed");
    tk->req = *r;
    tk->bytes = request_bytes(*r);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (r->gallery_id < 0 || r->gallery_id >= static_cast<int32_t>(s->galleries.size())) {
            delete tk;
            ++s->stats.rejected;
            return sfail(s, LATCH_EINVAL, "unknown gallery");
        }
        const size_t part = match_tc_partial_bound(r->n, 1, s->ctx->sm_count) + 512;
        if (r->n > s->max_batch_kps || tk->bytes + part > s->lane_bytes) {
            delete tk;
            ++s->stats.rejected;
            return sfail(s, LATCH_ENOMEM, "request larger than a lane of this session's HBM budget");
        }
        tk->id = s->next_ticket++;
        tk->t_submit = now_s(s);
        s->tickets[tk->id] = tk;
        s->queue.push_back(tk);
        ++s->stats.submitted;
        if (static_cast<int64_t>(s->queue.size()) > s->stats.max_queue)
            s->stats.max_queue = static_cast<int64_t>(s->queue.size());
        *ticket = tk->id;
    }
    s->cv_sched.notify_all();
    return LATCH_OK;
}

latch_status latch_wait(latch_session* s, uint64_t ticket, int32_t timeout_ms, latch_result* out) {
    if (!s) return LATCH_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return sfail(s, LATCH_EINVAL, "unknown ticket");
    Ticket* tk = it->second;
    const auto pred = [tk] { return tk->done; };
    if (timeout_ms < 0)
        s->cv_done.wait(lock, pred);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred))
        return LATCH_ETIMEOUT;
    if (out) {
        out->status = tk->status;
        out->n = tk->req.n;
        out->batch_size = tk->batch_size;
        out->submit_s = tk->t_submit;
        out->start_s = tk->t_start;
        out->done_s = tk->t_done;
    }
    return tk->status;
}

latch_status latch_release(latch_session* s, uint64_t ticket) {
    if (!s) return LATCH_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return sfail(s, LATCH_EINVAL, "unknown ticket");
    if (!it->second->done) return sfail(s, LATCH_EBUSY, "ticket still in flight");
    delete it->second;
    s->tickets.erase(it);
    return LATCH_OK;
}

latch_status latch_session_get_stats(latch_session* s, latch_session_stats* out) {
    if (!s || !out) return LATCH_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->queued = static_cast<int64_t>(s->queue.size());
    out->lane_bytes = static_cast<int64_t>(s->lane_bytes);
    return LATCH_OK;
}

const char* latch_session_last_error(const latch_session* s) { return s ? s->err : ""; }

}  // extern "C"

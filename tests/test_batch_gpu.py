"""Parity of the batched extract-then-match entry point (latch_batch_run) with the
CPU oracle and with the one-call-per-image / per-pair entry points."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
import oracle_shards
from conftest import same_matches, to_dev

pytestmark = pytest.mark.gpu


def _run_batch(ctx, imgs, sizes, kps_list, pairs, k=2, ratio=0.8):
    dev_imgs = [to_dev(im) for im in imgs]
    n = [len(k_) for k_ in kps_list]
    allk = np.concatenate([P.pack_keypoints(k_) for k_ in kps_list]) if sum(n) else np.zeros((0, 12), np.uint8)
    d_kps = to_dev(allk) if sum(n) else torch.zeros((1, 12), dtype=torch.uint8, device="cuda")
    d_desc = torch.zeros((max(1, sum(n)), 64), dtype=torch.uint8, device="cuda")
    nout = sum(n[q] for q, _ in pairs)
    d_m = torch.zeros((max(1, nout), 16), dtype=torch.uint8, device="cuda")
    images = [(t, w, h, t.stride(0)) for t, (w, h) in zip(dev_imgs, sizes)]
    b = P.BatchDesc(images, n, d_kps, d_desc, pairs, k, ratio, d_m)
    P.latch_batch_run(ctx.handle, b, int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    ctx.check()
    off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    descs = [d_desc[off[i]:off[i + 1]].cpu().numpy() for i in range(len(imgs))]
    mo = b.match_offsets()
    recs = P.matches_from_bytes(d_m.cpu().numpy())
    matches = [recs[mo[p]:mo[p + 1]] for p in range(len(pairs))]
    return descs, matches


def _same(got, want):
    for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
        assert np.array_equal(got[f].astype(np.int64), np.asarray(want[f]).astype(np.int64)), f


def test_small_mixed_batch(gpu_ctx, triplets):
    """Images of different sizes and pitches, empty and tiny keypoint sets,
    keypoints near and beyond borders, self pairs and pairs with an empty side."""
    sizes = [(320, 240), (641, 480), (200, 150), (1000, 700), (48, 48), (333, 333)]
    counts = [300, 1000, 0, 2500, 7, 800]
    imgs, kps = [], []
    for i, ((w, h), c) in enumerate(zip(sizes, counts)):
        imgs.append(synth.image(synth.seed(31, i, synth.KIND_IMAGE), w, h, n_ellipses=30))
        k = synth.keypoints(synth.seed(31, i, synth.KIND_KEYPOINTS), w + 40, h + 40, c, 0, True, 3)
        k[:, 0] -= 20
        k[:, 1] -= 20
        kps.append(k)
    pairs = [(0, 1), (1, 0), (0, 0), (2, 3), (3, 2), (3, 5), (4, 4), (5, 1), (1, 3), (4, 2)]
    descs, matches = _run_batch(gpu_ctx, imgs, sizes, kps, pairs)
    wants = [oracle.extract(imgs[i], sizes[i][0], sizes[i][1], kps[i], triplets, synth.SCALES)
             for i in range(len(imgs))]
    for i in range(len(imgs)):
        assert np.array_equal(descs[i], wants[i]), i
    for p, (q, t) in enumerate(pairs):
        if counts[q] == 0:
            assert len(matches[p]) == 0
            continue
        _same(matches[p], oracle.match(wants[q], wants[t], 2, 0.8))


def test_far_outside_keypoints_match_as_zero_descriptors(gpu_ctx, triplets):
    """Keypoints so far outside their image that the window misses it get the zero
    descriptor without being sampled; in the batched matcher they still take part on
    both sides of a pair, at distance popc(other) (Eq. 1 with every SSD 0)."""
    sizes = [(320, 240), (400, 300), (256, 256)]
    imgs, kps = [], []
    for i, (w, h) in enumerate(sizes):
        imgs.append(synth.image(synth.seed(34, i, synth.KIND_IMAGE), w, h, n_ellipses=30))
        k = synth.keypoints(synth.seed(34, i, synth.KIND_KEYPOINTS), w, h, 600, 0, True, 3)
        far = np.array([[-5000, -5000], [w + 4000, 10], [20, h + 9000], [-3000, h // 2]], np.int32)
        rows = np.arange(5 + i, 600, 37)[:len(far) * 6]
        k[rows, 0] = np.tile(far[:, 0], 6)[:len(rows)]
        k[rows, 1] = np.tile(far[:, 1], 6)[:len(rows)]
        kps.append(k)
    pairs = [(0, 1), (1, 0), (2, 2), (1, 2), (2, 0)]
    descs, matches = _run_batch(gpu_ctx, imgs, sizes, kps, pairs)
    wants = [oracle.extract(imgs[i], sizes[i][0], sizes[i][1], kps[i], triplets, synth.SCALES)
             for i in range(len(imgs))]
    for i in range(len(imgs)):
        assert np.array_equal(descs[i], wants[i]), i
        assert (wants[i][np.arange(5 + i, 600, 37)[:24]] == 0).all()
    for p, (q, t) in enumerate(pairs):
        _same(matches[p], oracle.match(wants[q], wants[t], 2, 0.8))


def test_batch_equals_single_calls(gpu_ctx, triplets):
    """Same bytes as latch_extract per image and hamming_match per pair, for k = 1."""
    sizes = [(400, 300)] * 4
    imgs = [synth.image(synth.seed(32, i, synth.KIND_IMAGE), 400, 300, n_ellipses=20) for i in range(4)]
    kps = [synth.keypoints(synth.seed(32, i, synth.KIND_KEYPOINTS), 400, 300, 1500 + 97 * i, 32, True, 3)
           for i in range(4)]
    pairs = [(0, 1), (1, 2), (2, 3), (3, 0)]
    descs, matches = _run_batch(gpu_ctx, imgs, sizes, kps, pairs, k=1, ratio=0.7)
    single = [gpu_ctx.extract(to_dev(im), 400, 300, to_dev(P.pack_keypoints(k))) for im, k in zip(imgs, kps)]
    for i in range(4):
        assert np.array_equal(descs[i], single[i].cpu().numpy())
    for p, (q, t) in enumerate(pairs):
        one = P.matches_from_bytes(gpu_ctx.match(single[q], single[t], 1, 0.7, P.PATH_TENSOR).cpu().numpy())
        _same(matches[p], one)


def test_sfm_batch_full_size(gpu_ctx, triplets):
    """The full batched workload (64 images of 4000x3000, 5k-50k oriented and scaled
    keypoints each, 476 neighbour pairs) in one latch_batch_run: every descriptor of
    every image equals the oracle's, and in every pair a seeded 1% of the query rows
    (at least one) equals the oracle's matching of its own descriptors against the
    whole train image.  The oracle runs sharded over the host cores."""
    wl = synth.sfm_batch()
    w, h = wl["width"], wl["height"]
    sizes = [(w, h)] * len(wl["images"])
    descs, matches = _run_batch(gpu_ctx, wl["images"], sizes, wl["kps"], wl["pairs"])
    wants = oracle_shards.extract_many([(im, w, h, k, triplets, synth.SCALES) for im, k in zip(wl["images"], wl["kps"])],
                                       per=1024)
    for i in range(len(wl["images"])):
        assert np.array_equal(descs[i], wants[i]), i
    rng = np.random.default_rng(7)
    jobs, picks = [], []
    for p, (q, t) in enumerate(wl["pairs"]):
        nq = len(wl["kps"][q])
        rows = np.sort(rng.choice(nq, max(1, -(-nq // 100)), replace=False))
        picks.append(rows)
        jobs.append((wants[q][rows], wants[t], 2, 0.8))
    for p, want in enumerate(oracle_shards.match_many(jobs, per=16)):
        same_matches(matches[p], want, picks[p])


def test_whole_tile_shares_every_row(gpu_ctx, triplets):
    """A batch with at least 8 query tiles per block (72 pairs x 21 tiles of 128
    queries) takes whole query tiles per block, and each block writes its tiles'
    matches itself: every match row of every pair equals the oracle's (sharded over
    the host cores), ragged query and train tiles included."""
    nimg, w, h = 24, 640, 480
    imgs = [synth.image(synth.seed(36, i, synth.KIND_IMAGE), w, h, n_ellipses=60) for i in range(nimg)]
    counts = [2600 - 37 * (i % 5) for i in range(nimg)]
    kps = [synth.keypoints(synth.seed(36, i, synth.KIND_KEYPOINTS), w, h, counts[i], 32, True, 3) for i in range(nimg)]
    pairs = [(i, (i + d) % nimg) for i in range(nimg) for d in (1, 2, 3)]
    assert sum(-(-counts[q] // 128) for q, _ in pairs) >= 8 * 152
    descs, matches = _run_batch(gpu_ctx, imgs, [(w, h)] * nimg, kps, pairs)
    wants = oracle_shards.extract_many([(im, w, h, k, triplets, synth.SCALES) for im, k in zip(imgs, kps)], per=512)
    for i in range(nimg):
        assert np.array_equal(descs[i], wants[i]), i
    for p, want in enumerate(oracle_shards.match_many([(wants[q], wants[t], 2, 0.8) for q, t in pairs], per=256)):
        same_matches(matches[p], want)


def test_more_pairs_than_one_launch(gpu_ctx, triplets):
    """700 pairs: two matching launches share the scratch (partial records and the
    per-query-tile arrival counters, which each complete launch leaves zero).  The
    second launch holds a pair with an empty train set, so it combines its records
    in a separate pass; the first combines them in the matching kernel.  Every
    pair's matches equal a single hamming_match call on the same descriptors, and a
    second run of the batch gives the same bytes."""
    rng = np.random.default_rng(35)
    nimg = 30
    sizes = [(160, 120)] * nimg
    imgs = [synth.image(synth.seed(35, i, synth.KIND_IMAGE), 160, 120, n_ellipses=10) for i in range(nimg)]
    counts = [0] + [int(c) for c in rng.integers(1, 400, nimg - 1)]  # image 0 has no keypoints
    kps = [synth.keypoints(synth.seed(35, i, synth.KIND_KEYPOINTS), 160, 120, counts[i], 16, True, 3)
           if counts[i] else np.zeros((0, 4), np.int32) for i in range(nimg)]
    pairs = [(int(q), int(t)) for q, t in zip(rng.integers(1, nimg, 700), rng.integers(1, nimg, 700))]
    pairs[600] = (5, 0)  # queries against an empty train set, in the second launch
    descs, matches = _run_batch(gpu_ctx, imgs, sizes, kps, pairs)
    _, again = _run_batch(gpu_ctx, imgs, sizes, kps, pairs)
    dev = [to_dev(d) if len(d) else torch.zeros((1, 64), dtype=torch.uint8, device="cuda") for d in descs]
    for p, (q, t) in enumerate(pairs):
        _same(again[p], matches[p])
        if counts[q] == 0:
            assert len(matches[p]) == 0
            continue
        out = torch.empty((counts[q], 16), dtype=torch.uint8, device="cuda")
        P.hamming_match(gpu_ctx.handle, dev[q], counts[q], dev[t], counts[t], 2, 0.8, out, P.PATH_TENSOR,
                        int(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        _same(matches[p], P.matches_from_bytes(out.cpu().numpy()))
    assert np.all(matches[600]["idx1"] == -1) and np.all(matches[600]["dist1"] == 65535)
    q3, t3 = pairs[3]
    wq, wt = (oracle.extract(imgs[i], 160, 120, kps[i], triplets, synth.SCALES) for i in (q3, t3))
    assert np.array_equal(descs[q3], wq) and np.array_equal(descs[t3], wt)
    _same(matches[3], oracle.match(wq, wt, 2, 0.8))


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
    t.numpy()[:] = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    return t


def test_host_batch_pipelined_equals_device_batch(gpu_ctx, triplets):
    """latch_batch_run_host: three calls with different inputs enqueued back to back
    (the two staging sets alternate, uploads overlap the previous call's kernels,
    the first call grows the sets), synchronised once; each call's host outputs
    equal latch_batch_run on device copies of the same inputs."""
    sizes = [(320, 240), (641, 480), (200, 150), (1000, 700)]
    pairs = [(0, 1), (1, 0), (2, 3), (3, 2), (1, 3)]
    calls = []
    for c in range(3):
        imgs, kps = [], []
        for i, (w, h) in enumerate(sizes):
            imgs.append(synth.image(synth.seed(36, 10 * c + i, synth.KIND_IMAGE), w, h, n_ellipses=20))
            kps.append(synth.keypoints(synth.seed(36, 10 * c + i, synth.KIND_KEYPOINTS), w, h,
                                       [400, 1500, 0, 2200][i] + 37 * c, 0, True, 3))
        calls.append((imgs, kps))
    stream = torch.cuda.current_stream()
    outs = []
    for imgs, kps in calls:
        n = [len(k) for k in kps]
        h_imgs = [_pinned(im) for im in imgs]
        h_kps = _pinned(np.concatenate([P.pack_keypoints(k) for k in kps]))
        h_desc = torch.zeros(sum(n) * 64, dtype=torch.uint8, pin_memory=True)
        nout = sum(n[q] for q, _ in pairs)
        h_m = torch.zeros(nout * 16, dtype=torch.uint8, pin_memory=True)
        # host rows keep synth.image's padded pitch (the array's row stride)
        hb = P.HostBatchDesc([(t, w, h, im.shape[1]) for t, im, (w, h) in zip(h_imgs, imgs, sizes)], n, h_kps,
                             h_desc, pairs, 2, 0.8, h_m)
        P.latch_batch_run_host(gpu_ctx.handle, hb, int(stream.cuda_stream))
        outs.append((h_imgs, h_kps, h_desc, h_m, hb, n))  # inputs stay alive until the sync
    torch.cuda.synchronize()
    gpu_ctx.check()
    for (imgs, kps), (_, _, h_desc, h_m, hb, n) in zip(calls, outs):
        descs, matches = _run_batch(gpu_ctx, imgs, sizes, kps, pairs)
        off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
        got_d = h_desc.numpy().reshape(-1, 64)
        for i in range(len(imgs)):
            assert np.array_equal(got_d[off[i]:off[i + 1]], descs[i]), i
        mo = hb.match_offsets()
        recs = P.matches_from_bytes(h_m.numpy().reshape(-1, 16))
        for p in range(len(pairs)):
            _same(recs[mo[p]:mo[p + 1]], matches[p])


def test_oriented_pair_batched(gpu_ctx, oriented_pair_oracle):
    """The oriented and scaled pair as one latch_batch_run (2 x 1920x1080, 10,000
    keypoints each, 10k x 10k top-2, ratio 0.8): all 20,000 descriptors and all
    10,000 match records equal the oracle's."""
    wl, descs_o, want = oriented_pair_oracle["wl"], oriented_pair_oracle["descs"], oriented_pair_oracle["match"]
    w, h = wl["width"], wl["height"]
    descs, matches = _run_batch(gpu_ctx, wl["images"], [(w, h)] * 2, wl["kps"], [(0, 1)])
    for i in range(2):
        assert np.array_equal(descs[i], descs_o[i]), i
    same_matches(matches[0], want)


def test_graph_replay_with_new_inputs(gpu_ctx, triplets):
    """latch_batch_run captured once in a CUDA graph and replayed on new images and
    keypoints written into the same device buffers: each replay equals the oracle
    on its own inputs (nothing of the capture-time inputs is baked into the graph)."""
    sizes = [(500, 380), (500, 380), (640, 400)]
    n = [1200, 900, 1500]
    pairs = [(0, 1), (1, 2), (2, 0), (1, 1)]

    def scene(s):
        imgs = [synth.image(synth.seed(33, 10 * s + i, synth.KIND_IMAGE), w, h, pitch=640, n_ellipses=40)
                for i, (w, h) in enumerate(sizes)]
        kps = [synth.keypoints(synth.seed(33, 10 * s + i, synth.KIND_KEYPOINTS), w, h, c, 16, True, 3)
               for i, ((w, h), c) in enumerate(zip(sizes, n))]
        return imgs, kps

    d_imgs = [torch.zeros((h, 640), dtype=torch.uint8, device="cuda") for _, h in sizes]
    d_kps = torch.zeros((sum(n), 12), dtype=torch.uint8, device="cuda")
    d_desc = torch.zeros((sum(n), 64), dtype=torch.uint8, device="cuda")
    nout = sum(n[q] for q, _ in pairs)
    d_m = torch.zeros((nout, 16), dtype=torch.uint8, device="cuda")
    b = P.BatchDesc([(t, w, h, t.stride(0)) for t, (w, h) in zip(d_imgs, sizes)], n, d_kps, d_desc, pairs, 2, 0.8,
                    d_m)
    P.latch_reserve_batch(gpu_ctx.handle, b)
    stream = torch.cuda.Stream()
    off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    mo = b.match_offsets()

    def load(s):
        imgs, kps = scene(s)
        with torch.cuda.stream(stream):
            for t, im in zip(d_imgs, imgs):
                t.copy_(torch.from_numpy(im))
            d_kps.copy_(torch.from_numpy(np.concatenate([P.pack_keypoints(k) for k in kps])))
        return imgs, kps

    with torch.cuda.stream(stream):
        load(0)
        P.latch_batch_run(gpu_ctx.handle, b, int(stream.cuda_stream))  # warm: kernel attributes, tensor maps
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            P.latch_batch_run(gpu_ctx.handle, b, int(stream.cuda_stream))
    for s in (1, 2):
        imgs, kps = load(s)
        with torch.cuda.stream(stream):
            d_m.zero_()
            graph.replay()
        torch.cuda.synchronize()
        gpu_ctx.check()
        wants = oracle_shards.extract_many([(im, w, h, k, triplets, synth.SCALES)
                                            for im, (w, h), k in zip(imgs, sizes, kps)])
        descs = d_desc.cpu().numpy()
        for i in range(len(sizes)):
            assert np.array_equal(descs[off[i]:off[i + 1]], wants[i]), (s, i)
        recs = P.matches_from_bytes(d_m.cpu().numpy())
        for p, (q, t) in enumerate(pairs):
            _same(recs[mo[p]:mo[p + 1]], oracle.match(wants[q], wants[t], 2, 0.8))
    del graph

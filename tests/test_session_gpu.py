"""The serving session: requests against resident galleries, continuous batching.

Each request's matches and descriptors must be byte-identical whether it runs
alone or batched with others, and equal to latch_extract + hamming_match (whose
parity with the oracle is tested elsewhere); a sample is also checked against the
oracle directly.  Admission refuses what can never fit."""
import threading

import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
from conftest import to_dev

pytestmark = pytest.mark.gpu

SIZES = [(640, 480), (1280, 720), (333, 251), (1920, 1080), (48, 48)]


def _requests(n_req, seed=41):
    rng = np.random.default_rng(seed)
    imgs = {}
    reqs = []
    for r in range(n_req):
        si = int(rng.integers(0, len(SIZES)))
        w, h = SIZES[si]
        if si not in imgs:
            imgs[si] = synth.image(synth.seed(seed, si, synth.KIND_IMAGE), w, h, n_ellipses=40)
        n = int(rng.choice([0, 1, 7, 300, 2000, 9000]))
        kps = synth.keypoints(synth.seed(seed, 100 + r, synth.KIND_KEYPOINTS), w, h, n, 0, True, 3)
        reqs.append({"img": imgs[si], "w": w, "h": h, "kps": P.pack_keypoints(kps), "raw_kps": kps,
                     "gallery": int(rng.integers(0, 3)), "k": int(rng.choice([1, 2])),
                     "ratio": float(rng.choice([0.8, 0.6, 1.0]))})
    return reqs


@pytest.fixture(scope="module")
def served(triplets):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1609_03986_gb300 import build
    build.build()
    sess = P.Session(triplets, hbm_budget=3 << 30, max_gallery_rows=1 << 20, max_batch=16, max_batch_kps=1 << 17)
    gals = [synth.random_descriptors(synth.seed(42, g, synth.KIND_GALLERY), n) for g, n in
            enumerate((5000, 20011, 0))]
    ids = [sess.add_gallery(g) for g in gals]
    assert ids == [0, 1, 2]
    yield sess, gals
    sess.close()


def _single_call(ctx, req, gals):
    """The request through latch_extract + hamming_match."""
    n = len(req["kps"])
    if n == 0:
        return np.zeros((0, 64), np.uint8), P.matches_from_bytes(np.zeros((0, 16), np.uint8))
    d = ctx.extract(to_dev(req["img"]), req["w"], req["h"], to_dev(req["kps"]))
    g = gals[req["gallery"]]
    gt = to_dev(g) if len(g) else torch.zeros((1, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
    P.hamming_match(ctx.handle, d, n, gt, len(g), req["k"], req["ratio"], out, P.PATH_TENSOR,
                    int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return d.cpu().numpy(), P.matches_from_bytes(out.cpu().numpy())


def _same(a, b):
    for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
        assert np.array_equal(a[f], b[f]), f


def test_alone_and_in_the_mix_are_identical(served, gpu_ctx):
    sess, gals = served
    reqs = _requests(14)
    want = [_single_call(gpu_ctx, r, gals) for r in reqs]
    # alone: one request in flight at a time
    for r, (wd, wm) in zip(reqs, want):
        t = sess.submit(r["img"], r["w"], r["h"], r["kps"], r["gallery"], r["k"], r["ratio"], want_desc=True)
        res, m, d = sess.wait(t)
        assert res.batch_size == 1
        assert np.array_equal(d, wd)
        _same(m, wm)
    # in the mix: everything submitted at once, admitted into shared micro-batches
    tickets = [sess.submit(r["img"], r["w"], r["h"], r["kps"], r["gallery"], r["k"], r["ratio"], want_desc=True)
               for r in reqs]
    sizes = []
    for t, (wd, wm) in zip(tickets, want):
        res, m, d = sess.wait(t)
        sizes.append(res.batch_size)
        assert res.done_s >= res.start_s >= res.submit_s
        assert np.array_equal(d, wd)
        _same(m, wm)
    assert max(sizes) > 1, "requests submitted together should share a micro-batch"


def test_oracle_sample(served, triplets):
    sess, gals = served
    w, h = 640, 480
    img = synth.image(synth.seed(43, 0, synth.KIND_IMAGE), w, h, n_ellipses=30)
    kps = synth.keypoints(synth.seed(43, 0, synth.KIND_KEYPOINTS), w, h, 700, 16, True, 3)
    t = sess.submit(img, w, h, P.pack_keypoints(kps), 1, 2, 0.8, want_desc=True)
    res, m, d = sess.wait(t)
    want = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
    assert np.array_equal(d, want)
    _same(m, oracle.match(want, gals[1], 2, 0.8))


def test_concurrent_submitters(served, gpu_ctx):
    """Four host threads submit and wait at the same time."""
    sess, gals = served
    reqs = _requests(20, seed=44)
    want = [_single_call(gpu_ctx, r, gals) for r in reqs]
    errors = []

    def worker(idx):
        try:
            for i in idx:
                r = reqs[i]
                t = sess.submit(r["img"], r["w"], r["h"], r["kps"], r["gallery"], r["k"], r["ratio"])
                res, m, _ = sess.wait(t)
                _same(m, want[i][1])
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(list(range(j, 20, 4)),)) for j in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    st = sess.stats()
    assert st["failed"] == 0 and st["queued"] == 0


def test_admission(served):
    sess, gals = served
    img = np.zeros((64, 64), np.uint8)
    big = P.pack_keypoints(np.zeros((200000, 4), np.int32))
    with pytest.raises(P.LatchError) as e:
        sess.submit(img, 64, 64, big, 0)
    assert e.value.status == 2  # never fits a micro-batch of this session
    with pytest.raises(P.LatchError) as e:
        sess.submit(img, 64, 64, big[:10], 7)
    assert e.value.status == 1  # unknown gallery
    with pytest.raises(P.LatchError):
        sess.submit(img, 64, 64, big[:10], 0, k=3)
    assert sess.stats()["rejected"] >= 2


def test_bad_scale_is_refused_and_the_mix_stays_exact(served, gpu_ctx):
    """A request holding one keypoint with a scale index outside the scale table is
    refused at submit (LATCH_EINVAL), while requests submitted around it still
    complete with the bytes of the plain calls."""
    sess, gals = served
    reqs = _requests(6, seed=45)
    want = [_single_call(gpu_ctx, r, gals) for r in reqs]
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(sess.submit(r["img"], r["w"], r["h"], r["kps"], r["gallery"], r["k"], r["ratio"],
                                   want_desc=True))
        if i == 2:
            bad = reqs[3]["raw_kps"].copy() if len(reqs[3]["raw_kps"]) else np.array([[10, 10, 0, 0]], np.int32)
            bad[len(bad) // 2, 3] = 3  # the session's scale table has 3 entries
            with pytest.raises(P.LatchError) as e:
                sess.submit(reqs[3]["img"], reqs[3]["w"], reqs[3]["h"], P.pack_keypoints(bad), 0)
            assert e.value.status == 1
            assert "scale" in P.latch_session_last_error(sess.handle)
    for t, (wd, wm) in zip(tickets, want):
        res, m, d = sess.wait(t)
        assert res.status == 0
        assert np.array_equal(d, wd)
        _same(m, wm)
    st = sess.stats()
    assert st["failed"] == 0
    assert 0 < st["hbm_budget"] <= st["hbm_free"]


@pytest.mark.parametrize("lanes", [1, 4])
def test_lane_counts(triplets, gpu_ctx, lanes):
    """Sessions with one and with four lanes give the bytes of the plain calls for a
    burst of requests (with four lanes, several micro-batches run at once)."""
    sess = P.Session(triplets, hbm_budget=2 << 30, max_gallery_rows=1 << 18, max_batch=8, max_batch_kps=1 << 16,
                     lanes=lanes)
    try:
        gals = [synth.random_descriptors(synth.seed(46, g, synth.KIND_GALLERY), n) for g, n in
                enumerate((3000, 12007, 1))]
        assert [sess.add_gallery(g) for g in gals] == [0, 1, 2]
        reqs = _requests(16, seed=47)
        want = [_single_call(gpu_ctx, r, gals) for r in reqs]
        tickets = [sess.submit(r["img"], r["w"], r["h"], r["kps"], r["gallery"], r["k"], r["ratio"], want_desc=True)
                   for r in reqs]
        for t, (wd, wm) in zip(tickets, want):
            res, m, d = sess.wait(t)
            assert res.status == 0
            assert np.array_equal(d, wd)
            _same(m, wm)
        st = sess.stats()
        assert st["failed"] == 0 and st["completed"] == len(reqs)
    finally:
        sess.close()
    with pytest.raises(P.LatchError):
        P.latch_session_create_lanes(0, 1 << 30, 1000, 4, 1000, 9, triplets)

"""Parity of dense per-pixel LATCH and windowed matching (Sec. 6, dense pixel matching)
with the oracle through the C ABI: every pixel of ragged-size images, every match row
of ragged fields at several radii, the 640x480 field in full against the sharded
oracle and sampled match rows of it, degenerate sizes and argument errors."""
import numpy as np
import pytest
import torch

import oracle
import oracle_shards
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
from conftest import match_records, same_matches, to_dev

pytestmark = pytest.mark.gpu


def _dense(ctx, img, w, h):
    out = ctx.dense_extract(to_dev(img), w, h)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _dmatch(ctx, da, db, w, h, radius, k=2, ratio=0.8):
    out = ctx.dense_match(to_dev(da), to_dev(db), w, h, radius, k, ratio)
    torch.cuda.synchronize()
    return match_records(out)


@pytest.mark.parametrize("w,h", [(45, 38), (97, 70), (130, 33), (33, 130)])
def test_dense_extract_every_pixel(gpu_ctx, triplets, w, h):
    """Tiles that straddle every border (sizes not multiples of the 32-pixel tile)."""
    img = synth.image(synth.seed(31, w, synth.KIND_IMAGE), w, h, n_ellipses=12)
    got = _dense(gpu_ctx, img, w, h)
    want = oracle.dense_extract(img, w, h, triplets)
    assert np.array_equal(got, want)


def test_dense_extract_pitch_and_tiny(gpu_ctx, triplets):
    """A padded row pitch, a 1x1 image and an image thinner than the patch."""
    w, h = 50, 41
    img = synth.image(synth.seed(31, 1, synth.KIND_IMAGE), w, h, pitch=64, n_ellipses=8)
    assert np.array_equal(_dense(gpu_ctx, img, w, h), oracle.dense_extract(img, w, h, triplets))
    one = np.zeros((1, 16), np.uint8)
    one[0, 0] = 201
    assert np.array_equal(_dense(gpu_ctx, one, 1, 1), oracle.dense_extract(one, 1, 1, triplets))
    thin = synth.image(synth.seed(31, 2, synth.KIND_IMAGE), 3, 60, pitch=16, n_ellipses=3)
    assert np.array_equal(_dense(gpu_ctx, thin, 3, 60), oracle.dense_extract(thin, 3, 60, triplets))


def test_dense_extract_full_640x480(gpu_ctx, triplets):
    """Every pixel of a 640x480 field against the oracle's keypoint form (an upright
    scale-1 keypoint at every pixel, which the oracle's dense form equals), sharded."""
    w, h = 640, 480
    img = synth.image(synth.seed(31, 3, synth.KIND_IMAGE), w, h)
    got = _dense(gpu_ctx, img, w, h)
    ys, xs = np.mgrid[0:h, 0:w]
    kps = np.stack([xs.ravel(), ys.ravel(), np.zeros(w * h), np.zeros(w * h)], axis=1).astype(np.int32)
    want = oracle_shards.extract(img, w, h, kps, triplets, (1.0,), per=4096)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("radius", [0, 1, 4, 16])
def test_dense_match_every_row(gpu_ctx, triplets, radius):
    """Every pixel's match on ragged fields: real dense descriptors (smooth regions
    give ties) and a field drawn from a pool of 5 descriptors (ties everywhere)."""
    w, h = 37, 23
    img_a = synth.image(synth.seed(32, 0, synth.KIND_IMAGE), w, h, n_ellipses=6)
    img_b = synth.image(synth.seed(32, 1, synth.KIND_IMAGE), w, h, n_ellipses=6)
    da, db = oracle.dense_extract(img_a, w, h, triplets), oracle.dense_extract(img_b, w, h, triplets)
    for k, ratio in ((2, 0.8), (1, 0.8), (2, 1.0), (2, 0.0)):
        same_matches(_dmatch(gpu_ctx, da, db, w, h, radius, k, ratio),
                     oracle.dense_match(da, db, w, h, radius, k, ratio))
    rng = np.random.default_rng(radius)
    pool = synth.random_descriptors(synth.seed(32, 2, synth.KIND_GALLERY), 5)
    pa, pb = pool[rng.integers(0, 5, w * h)], pool[rng.integers(0, 5, w * h)]
    same_matches(_dmatch(gpu_ctx, pa, pb, w, h, radius), oracle.dense_match(pa, pb, w, h, radius))


def test_dense_match_planted_flow(gpu_ctx):
    """A(p) = B(p + f(p)) with |f| <= 8 on random descriptors: every pixel finds its
    planted source at distance 0."""
    w, h, r = 70, 45, 8
    rng = np.random.default_rng(5)
    db = synth.random_descriptors(synth.seed(32, 3, synth.KIND_GALLERY), w * h)
    ys, xs = np.mgrid[0:h, 0:w]
    q = (np.clip(ys.ravel() + rng.integers(-r, r + 1, w * h), 0, h - 1) * w +
         np.clip(xs.ravel() + rng.integers(-r, r + 1, w * h), 0, w - 1))
    got = _dmatch(gpu_ctx, db[q], db, w, h, r)
    assert np.array_equal(got["idx1"], q) and (got["dist1"] == 0).all()
    same_matches(got, oracle.dense_match(db[q], db, w, h, r))


def test_dense_match_full_640x480_sampled(gpu_ctx, triplets):
    """A 640x480 pair (the second image the first shifted by (3, -2) plus a new ellipse
    layer) at radius 8: the GPU field's match of 4,000 sampled pixels and of every
    pixel of the four border rows / columns, each against the oracle's top-two over
    that pixel's candidates in raster order."""
    w, h, r = 640, 480, 8
    base = synth.image(synth.seed(33, 0, synth.KIND_IMAGE), w + 16, h + 16)
    img_a = np.ascontiguousarray(base[8:8 + h, 8:8 + w])
    img_b = np.ascontiguousarray(base[10:10 + h, 5:5 + w])
    da, db = _dense(gpu_ctx, img_a, w, h), _dense(gpu_ctx, img_b, w, h)
    got = _dmatch(gpu_ctx, da, db, w, h, r)
    rng = np.random.default_rng(8)
    rows = set(rng.choice(w * h, 4000, replace=False).tolist())
    rows |= set(range(w)) | set(range((h - 1) * w, h * w)) | set(range(0, w * h, w)) | set(range(w - 1, w * h, w))
    rows = np.array(sorted(rows))
    want = {f: np.zeros(len(rows), np.int64) for f in ("idx1", "idx2", "dist1", "dist2", "accepted")}
    for i, p in enumerate(rows):
        py, px = divmod(int(p), w)
        cy = np.arange(max(0, py - r), min(h, py + r + 1))
        cx = np.arange(max(0, px - r), min(w, px + r + 1))
        cand = (cy[:, None] * w + cx[None, :]).ravel()  # raster order of B
        m = oracle.match(da[p:p + 1], db[cand], 2, 0.8)
        for f in ("dist1", "dist2", "accepted"):
            want[f][i] = m[f][0]
        want["idx1"][i] = cand[m["idx1"][0]]
        want["idx2"][i] = cand[m["idx2"][0]] if m["idx2"][0] >= 0 else -1
    same_matches({f: got[f][rows] for f in want}, want)
    # the shift is recovered wherever the windows lie inside both images
    inner = (np.arange(h)[:, None] >= 26) & (np.arange(h)[:, None] < h - 26) & \
            (np.arange(w)[None, :] >= 26) & (np.arange(w)[None, :] < w - 26)
    assert (got["dist1"].reshape(h, w)[inner] == 0).all()


def test_dense_argument_errors(gpu_ctx):
    d = torch.zeros((16, 64), dtype=torch.uint8, device="cuda")
    out = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    for args in ((4, 4, 17, 2, 0.8), (4, 4, -1, 2, 0.8), (4, 4, 2, 3, 0.8), (4, 4, 2, 2, 1.5), (0, 4, 2, 2, 0.8)):
        with pytest.raises(P.LatchError) as e:
            P.latch_dense_match(gpu_ctx.handle, d, d, *args[:3], args[3], args[4], out, 0)
        assert e.value.status == 1
    trip = synth.triplets(synth.seed(32, 9, synth.KIND_TRIPLETS), hi=43)
    wctx = P.Context(0, triplets=trip)
    try:
        P.latch_set_patch_weights(wctx.handle, np.ones((8, 8), np.uint8))
        img = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
        with pytest.raises(P.LatchError) as e:
            wctx.dense_extract(img, 8, 8)
        assert e.value.status == 4
    finally:
        wctx.close()

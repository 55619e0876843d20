"""Pins for the oracle's dense per-pixel LATCH and windowed matching (Sec. 6: dense
pixel matching).  Each test names the mistake it is there to catch.  No GPU."""
import numpy as np
import pytest

import oracle
from paper_1609_03986_gb300 import synth


def _popcount_rows(a, b):
    return np.unpackbits(np.bitwise_xor(a, b), axis=1).sum(axis=1).astype(np.int64)


def test_dense_is_the_keypoint_descriptor_at_every_pixel():
    """Every pixel, border pixels included, carries the descriptor of an upright,
    scale-1 keypoint there (raster order): catches a transposed layout, a wrong
    row stride or a shifted window origin."""
    w, h = 23, 17
    img = synth.image(synth.seed(9, 0, synth.KIND_IMAGE), w, h, n_ellipses=6)
    trip = synth.triplets()
    dense = oracle.dense_extract(img, w, h, trip)
    ys, xs = np.mgrid[0:h, 0:w]
    kps = np.stack([xs.ravel(), ys.ravel(), np.zeros(w * h), np.zeros(w * h)], axis=1).astype(np.int32)
    want = oracle.extract(img, w, h, kps, trip, scales=(1.0,))
    assert np.array_equal(dense, want)


def test_dense_delta_image_closed_form():
    """A single bright pixel at s on black: for pixel p and triplet (a, c1, c2) (window
    coordinates), a patch centred at window point c covers s iff |s - p - (c - 24)| <= 3
    on both axes, so D1 = v^2 ([A covers s] + [C1 covers s]) unless a == c1 (then 0),
    and bit = D1 > D2.  Evaluated for all pixels and triplets at once: catches a
    wrong window centre, sign or patch extent anywhere in the dense loop."""
    w, h = 40, 31
    sx, sy, v = 17, 12, 200
    img = np.zeros((h, w), np.uint8)
    img[sy, sx] = v
    trip = synth.triplets().astype(np.int64)
    dense = oracle.dense_extract(img, w, h, trip.astype(np.uint8))
    ys, xs = np.mgrid[0:h, 0:w]
    px, py = xs.ravel()[:, None], ys.ravel()[:, None]  # (P, 1)

    def covers(cx, cy):  # (P, T) bool
        return (np.abs(sx - px - (cx[None, :] - 24)) <= 3) & (np.abs(sy - py - (cy[None, :] - 24)) <= 3)

    ax, ay, c1x, c1y, c2x, c2y = (trip[:, i] for i in range(6))
    ca, c1, c2 = covers(ax, ay), covers(c1x, c1y), covers(c2x, c2y)
    same1 = (ax == c1x) & (ay == c1y)
    same2 = (ax == c2x) & (ay == c2y)
    d1 = np.where(same1[None, :], 0, ca.astype(np.int64) + c1)
    d2 = np.where(same2[None, :], 0, ca.astype(np.int64) + c2)
    bits = (d1 > d2).astype(np.uint8)  # (P, 512), bit t
    want = np.packbits(bits, axis=1, bitorder="little")
    assert np.array_equal(dense, want)
    assert dense.any()  # the closed form is not vacuous


def test_dense_translation_moves_descriptors():
    """Image B = image A shifted by (tx, ty): wherever both windows lie inside their
    images, descriptor B(p + t) equals descriptor A(p).  Catches a window sampled
    relative to the tile instead of the pixel."""
    w, h, tx, ty = 70, 66, 5, -3
    big = synth.image(synth.seed(9, 1, synth.KIND_IMAGE), w + 20, h + 20, n_ellipses=20)
    a = np.ascontiguousarray(big[10:10 + h, 10:10 + w])
    b = np.ascontiguousarray(big[10 - ty:10 - ty + h, 10 - tx:10 - tx + w])
    trip = synth.triplets()
    da = oracle.dense_extract(a, w, h, trip).reshape(h, w, 64)
    db = oracle.dense_extract(b, w, h, trip).reshape(h, w, 64)
    for y in range(24, h - 24):
        for x in range(24, w - 24):
            if 24 <= x + tx < w - 24 and 24 <= y + ty < h - 24:
                assert np.array_equal(db[y + ty, x + tx], da[y, x]), (x, y)


def test_dense_match_full_radius_is_global_matching():
    """With a radius covering the whole image the candidate set of every pixel is all
    of B in raster order, so windowed matching equals global brute-force matching:
    catches a candidate order that is not raster order (ties) or a missed candidate."""
    w, h = 13, 9
    rng = np.random.default_rng(7)
    # few distinct descriptors: many ties, exercising the lowest-index rule
    pool = synth.random_descriptors(synth.seed(9, 2, synth.KIND_GALLERY), 6)
    da = pool[rng.integers(0, 6, w * h)]
    db = pool[rng.integers(0, 6, w * h)]
    for k, ratio in ((2, 0.8), (1, 0.8), (2, 1.0)):
        got = oracle.dense_match(da, db, w, h, max(w, h), k, ratio)
        want = oracle.match(da, db, k, ratio)
        for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
            assert np.array_equal(got[f], want[f]), (k, ratio, f)


def test_dense_match_radius_zero():
    """Radius 0: the only candidate is the same pixel, at the plain Hamming distance,
    with no second match (idx2 = -1, dist2 = 65535)."""
    w, h = 11, 7
    da = synth.random_descriptors(synth.seed(9, 3, synth.KIND_GALLERY), w * h)
    db = synth.random_descriptors(synth.seed(9, 4, synth.KIND_GALLERY), w * h)
    got = oracle.dense_match(da, db, w, h, 0, 2, 0.8)
    assert np.array_equal(got["idx1"], np.arange(w * h))
    assert np.array_equal(got["dist1"], _popcount_rows(da, db))
    assert (got["idx2"] == -1).all() and (got["dist2"] == 65535).all()
    assert (got["accepted"] == 1).all()


@pytest.mark.parametrize("radius", [1, 3, 6])
def test_dense_match_planted_displacements(radius):
    """A(p) is planted as an exact copy of B(p + f(p)) with |f| <= radius on both axes
    (clipped to B): the match is p + f(p) at distance 0.  The same plant at one
    more than the radius is out of the window (distance > 0).  Catches an
    off-by-one window, a swapped axis or a wrong raster index."""
    w, h = 21, 15
    rng = np.random.default_rng(radius)
    db = synth.random_descriptors(synth.seed(9, 5, synth.KIND_GALLERY), w * h)
    ys, xs = np.mgrid[0:h, 0:w]
    fx = rng.integers(-radius, radius + 1, w * h)
    fy = rng.integers(-radius, radius + 1, w * h)
    qx = np.clip(xs.ravel() + fx, 0, w - 1)
    qy = np.clip(ys.ravel() + fy, 0, h - 1)
    q = qy * w + qx
    da = db[q]
    got = oracle.dense_match(da, db, w, h, radius, 2, 0.8)
    assert np.array_equal(got["idx1"], q)
    assert (got["dist1"] == 0).all()
    # one beyond the window: x displacement radius + 1, kept where it stays inside
    far_x = xs.ravel() + radius + 1
    inside = far_x < w
    q2 = ys.ravel() * w + np.minimum(far_x, w - 1)
    da2 = db[q2]
    got2 = oracle.dense_match(da2, db, w, h, radius, 2, 0.8)
    assert (got2["dist1"][inside] > 0).all()
    assert (got2["dist1"][~inside] == 0).all()


def test_dense_degenerate_sizes():
    """A one-pixel image, an image narrower than the window and an empty image."""
    trip = synth.triplets()
    one = np.array([[77]], np.uint8)
    d = oracle.dense_extract(one, 1, 1, trip)
    kp = np.array([[0, 0, 0, 0]], np.int32)
    assert np.array_equal(d, oracle.extract(one, 1, 1, kp, trip, scales=(1.0,)))
    got = oracle.dense_match(d, d, 1, 1, 4, 2, 0.8)
    assert got["idx1"][0] == 0 and got["dist1"][0] == 0 and got["idx2"][0] == -1
    thin = synth.image(synth.seed(9, 6, synth.KIND_IMAGE), 3, 50, n_ellipses=2)
    assert oracle.dense_extract(thin, 3, 50, trip).shape == (150, 64)
    empty = np.zeros((1, 16), np.uint8)
    assert oracle.dense_extract(empty, 0, 0, trip).shape == (0, 64)
    e = oracle.dense_match(np.zeros((0, 64), np.uint8), np.zeros((0, 64), np.uint8), 0, 0, 3)
    assert e["idx1"].size == 0

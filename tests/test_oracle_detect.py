"""Pins for the oracle's keypoint detection (Sec. 3.2: FAST keypoints whose
orientation sets the window's angle): the FAST-9 segment test and score on
hand-made circles, the score against an independent closed form on random images,
non-maximum suppression and the detection region by brute force, the centroid
orientation on hand-worked images, and the whole chain's 90-degree rotation
invariance.  No GPU."""
import os

import numpy as np
import pytest

import oracle
from paper_1609_03986_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# the radius-3 Bresenham circle, clockwise from the pixel above the centre (x right, y down)
CIRCLE = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
          (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]


def _circle_image(values, centre=100, bg=100):
    """21x21 image, centre pixel (10, 10) = centre, circle pixel k = values[k] (None: bg)."""
    img = np.full((21, 32), bg, np.uint8)
    img[10, 10] = centre
    for k, v in enumerate(values):
        if v is not None:
            dx, dy = CIRCLE[k]
            img[10 + dy, 10 + dx] = v
    return img


def _arc(first, length, value):
    vals = [None] * 16
    for k in range(first, first + length):
        vals[k % 16] = value
    return vals


@pytest.mark.parametrize("values, t, want, why", [
    (_arc(0, 9, 150), 20, 49, "nine brighter pixels: score = 150 - 100 - 1"),
    (_arc(0, 8, 150), 20, 0, "eight are not enough (catches an arc length of 8)"),
    (_arc(12, 9, 150), 20, 49, "the arc wraps from position 15 to 0 (catches a non-circular scan)"),
    (_arc(3, 9, 60), 20, 39, "nine darker pixels: score = 100 - 60 - 1"),
    ([120 if k == 4 else v for k, v in enumerate(_arc(0, 9, 150))], 10, 19, "the arc's smallest margin sets the score"),
    ([120 if k == 4 else v for k, v in enumerate(_arc(0, 9, 150))], 20, 0, "equal to I(p) + t is not brighter (strict)"),
    (_arc(0, 9, 125), 25, 0, "exactly I(p) + t: not a corner at t"),
    (_arc(0, 9, 125), 24, 24, "one below: a corner, score 24"),
    ([120] + _arc(1, 8, 140)[1:9] + [160] + [None] * 6, 10, 39, "best of two arcs (0..8 gives 19, 1..9 gives 39)"),
    (_arc(0, 16, 140), 30, 39, "a full bright ring"),
    (_arc(0, 9, 255), 154, 154, "largest score over a centre of 100"),
])
def test_fast_score_hand_circles(values, t, want, why):
    img = _circle_image(values)
    assert oracle.fast_score(img, 21, 21, 10, 10, t) == want, why


def test_fast_score_largest_threshold():
    """Centre 0, nine pixels of 255: a corner up to t = 254 (the largest threshold)."""
    img = _circle_image(_arc(5, 9, 255), centre=0, bg=0)
    assert oracle.fast_score(img, 21, 21, 10, 10, 254) == 254
    assert oracle.fast_score(img, 21, 21, 10, 10, 1) == 254


def test_fast_score_needs_the_whole_circle():
    img = np.full((8, 16), 100, np.uint8)
    assert oracle.fast_score(img, 8, 8, 2, 4, 5) == 0 and oracle.fast_score(img, 8, 8, 5, 4, 5) == 0


def _closed_form_scores(img, w, h, t):
    """Score of every pixel from the arcs' margins: max over the 16 arcs of 9 of
    max(min(I_k - I_p), min(I_p - I_k)) - 1, kept when at least t."""
    a = img[:, :w].astype(np.int32)
    out = np.zeros((h, w), np.int32)
    c = a[3:h - 3, 3:w - 3]
    d = np.stack([a[3 + dy:h - 3 + dy, 3 + dx:w - 3 + dx] - c for dx, dy in CIRCLE])  # (16, h-6, w-6)
    best = np.full(c.shape, -10**6)
    for s in range(16):
        idx = [(s + k) % 16 for k in range(9)]
        best = np.maximum(best, np.maximum(d[idx].min(0), (-d[idx]).min(0)) - 1)
    out[3:h - 3, 3:w - 3] = np.where(best >= t, best, 0)
    return out


@pytest.mark.parametrize("t", [1, 12, 40])
def test_fast_score_closed_form_on_random_images(t):
    """The oracle's threshold search equals the closed form over arcs, pixel by
    pixel, on noisy images with many corners of both polarities."""
    rng = np.random.default_rng(70 + t)
    w, h = 37, 29
    img = np.zeros((h, 48), np.uint8)
    img[:, :w] = rng.integers(0, 256, (h, w))
    img[:, :w] = np.where(rng.random((h, w)) < 0.3, 128, img[:, :w])
    want = _closed_form_scores(img, w, h, t)
    got = np.array([[oracle.fast_score(img, w, h, x, y, t) for x in range(w)] for y in range(h)])
    assert np.array_equal(got, want)
    assert (got > 0).sum() > 20


def _brute_detect(img, w, h, t):
    s = np.array([[oracle.fast_score(img, w, h, x, y, t) for x in range(w)] for y in range(h)])
    kp = []
    for y in range(16, h - 16):
        for x in range(16, w - 16):
            v = s[y, x]
            nb = [s[y + dy, x + dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy]
            if v > 0 and all(v > q for q in nb):
                kp.append((x, y))
    return kp, s


@pytest.mark.parametrize("seed, t", [(1, 10), (2, 25), (3, 60)])
def test_detect_is_strict_nms_over_the_region(seed, t):
    """Keypoints = pixels at least 16 from every border whose score is non-zero and
    strictly above all 8 neighbours', in raster order (catches >= in the
    suppression, a wrong region, a wrong order); the bins are the centroid's."""
    w, h = 90, 70
    img = synth.image(synth.seed(72, seed, synth.KIND_IMAGE), w, h, n_ellipses=25)
    got = oracle.detect(img, w, h, t)
    want, s = _brute_detect(img, w, h, t)
    assert [tuple(p) for p in got[:, :2]] == want
    assert all(oracle.orientation_bin(img, x, y) == b for x, y, b in got)
    # some pair of neighbouring corners ties somewhere: both are suppressed
    ties = [(x, y) for y in range(16, h - 16) for x in range(16, w - 16)
            if s[y, x] > 0 and any(s[y, x] == s[y + dy, x + dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                                   if dx or dy)]
    assert not set(ties) & set(want)


def test_detect_ties_are_suppressed():
    """Two identical corner patterns side by side with equal scores next to each
    other: neither is kept; a lone one is."""
    img = np.full((40, 48), 100, np.uint8)
    # a dark 2x1 blob: both pixels are corners (bright surroundings) with the same score
    img[20, 20] = img[20, 21] = 30
    got = oracle.detect(img, 40, 40, 20)
    assert not any((x, y) in ((20, 20), (21, 20)) for x, y, _ in got)
    img[20, 21] = 100
    got = oracle.detect(img, 40, 40, 20)
    assert (20, 20) in [(x, y) for x, y, _ in got]


def test_orientation_hand_values():
    with open(os.path.join(GOLDEN, "orientation_spot_values.txt")) as f:
        rows = [line.split("#", 1)[0].split() for line in f]
    rows = [r for r in rows if r]
    assert len(rows) >= 15
    for r in rows:
        img = np.zeros((41, 48), np.uint8)
        vals = list(map(int, r[1:]))
        for i in range(0, len(vals), 3):
            dx, dy, v = vals[i:i + 3]
            img[20 + dy, 20 + dx] = v
        assert oracle.orientation_bin(img, 20, 20) == int(r[0]), r


def test_orientation_ramps():
    """A linear ramp points the centroid along its gradient: +x -> 0, +y -> 8,
    -x -> 16, -y -> 24."""
    y, x = np.mgrid[0:41, 0:48]
    for img, want in ((x * 5, 0), (y * 5, 8), (255 - x * 5, 16), (255 - y * 5, 24)):
        assert oracle.orientation_bin(img.astype(np.uint8), 20, 20) == want


def _near_boundary(img, x, y):
    """theta * 16 / pi within 1e-7 of a half-integer: the bin is a tie of rounding."""
    yy, xx = np.mgrid[-15:16, -15:16]
    m = (xx ** 2 + yy ** 2) <= 225
    patch = img[y - 15:y + 16, x - 15:x + 16].astype(np.int64)
    v = np.arctan2((yy * patch)[m].sum(), (xx * patch)[m].sum()) * 16 / np.pi
    return abs(abs(v - np.floor(v)) - 0.5) < 1e-7


def test_detection_rotates_with_the_image(triplets):
    """Turning the image by 90 degrees (clockwise as displayed, y down) turns every
    keypoint with it and adds 8 to its angle bin; the descriptors at the detected
    keypoints are then equal.  Pins the orientation's frame against the window's."""
    w = h = 160
    img = synth.image(synth.seed(73, 0, synth.KIND_IMAGE), w, h, n_ellipses=40)[:, :w]
    rot = np.ascontiguousarray(np.rot90(img, -1))  # rot[r, c] = img[h-1-c, r]
    a = oracle.detect(img, w, h, 20)
    b = oracle.detect(rot, h, w, 20)
    assert len(a) > 50 and len(a) == len(b)
    mapped = {(h - 1 - y, x): (bn + 8) % 32 for x, y, bn in a}
    got = {(x, y): bn for x, y, bn in b}
    assert set(mapped) == set(got)
    for (x, y), bn in got.items():
        if not _near_boundary(rot, x, y):
            assert mapped[(x, y)] == bn
    kpa = np.concatenate([a, np.zeros((len(a), 1), np.int32)], 1)
    kpb = np.array([[h - 1 - y, x, (bn + 8) % 32, 0] for x, y, bn in a], np.int32)
    assert np.array_equal(oracle.extract(img, w, h, kpa, triplets), oracle.extract(rot, h, w, kpb, triplets))


def test_detect_rejects_bad_thresholds():
    img = np.zeros((40, 48), np.uint8)
    for t in (0, 255, -3):
        with pytest.raises(ValueError):
            oracle.detect(img, 40, 40, t)
    assert len(oracle.detect(img, 40, 40, 1)) == 0  # a flat image has no corner

"""Pins for the CPU oracle: closed forms, hand-worked fixtures, invariants and brute
force against full sorting.  Each test names the mistake it is there to catch.
The oracle is test infrastructure; these tests run without a GPU."""
import os

import numpy as np
import pytest

import oracle
from paper_1609_03986_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _bit(desc, t):
    return (int(desc[t >> 3]) >> (t & 7)) & 1


# ---------------------------------------------------------------- offset table

def test_offsets_hand_values():
    """Hand-worked offsets: catches a wrong centre, rotation direction, angle
    step, scale order or rounding rule (banker's rounding or floor fail at .5)."""
    for s, b, u, v, dx, dy in _golden_rows("offset_spot_values.txt"):
        tx, ty = oracle.offsets(float(s), int(b))
        assert (tx[int(v), int(u)], ty[int(v), int(u)]) == (int(dx), int(dy)), (s, b, u, v)


@pytest.mark.parametrize("scale", synth.SCALES)
def test_offsets_quarter_turn_exact(scale):
    """Bin b+8 is exactly bin b turned by 90 degrees, and b+16 by 180 degrees,
    at every scale (the quarter turns are applied exactly)."""
    for b in range(32):
        dx, dy = oracle.offsets(scale, b)
        dx8, dy8 = oracle.offsets(scale, b + 8)
        dx16, dy16 = oracle.offsets(scale, b + 16)
        assert np.array_equal(dx8, -dy) and np.array_equal(dy8, dx)
        assert np.array_equal(dx16, -dx) and np.array_equal(dy16, -dy)


def test_offsets_identity_and_range():
    """Bin 0, scale 1 is the identity; bins wrap modulo 32; every offset is the
    nearest integer of the rotated, scaled point (error at most 1/2), so the
    sampled point set is the rotated square; magnitudes stay within 77."""
    dx, dy = oracle.offsets(1.0, 0)
    u = np.arange(48)
    assert np.array_equal(dx, np.broadcast_to(u - 24, (48, 48)))
    assert np.array_equal(dy, np.broadcast_to((u - 24)[:, None], (48, 48)))
    for b in (3, 17, 30):
        assert np.array_equal(oracle.offsets(1.5, b)[0], oracle.offsets(1.5, b + 32)[0])
    a = (u - 24)[None, :].astype(np.float64)
    e = (u - 24)[:, None].astype(np.float64)
    for s in synth.SCALES:
        for b in range(32):
            th = 2 * np.pi * b / 32
            dx, dy = oracle.offsets(s, b)
            ex = s * (np.cos(th) * a - np.sin(th) * e)
            ey = s * (np.sin(th) * a + np.cos(th) * e)
            assert np.max(np.abs(dx - ex)) <= 0.5 + 1e-9
            assert np.max(np.abs(dy - ey)) <= 0.5 + 1e-9
            assert np.max(np.abs(dx)) <= 77 and np.max(np.abs(dy)) <= 77


# ---------------------------------------------------------------- extraction

def _table_with(rows):
    trip = np.full((512, 6), 24, dtype=np.uint8)
    for idx, t in rows:
        trip[idx] = t
    return trip


def test_border_constant_hand_worked():
    """Hand-worked SSDs at the image border (samples outside read 0): catches a
    wrong border rule, a wrong patch size or centre, swapped anchor/companion
    roles, a non-strict comparison and a wrong bit order."""
    rows = _golden_rows("border_constant.txt")
    trip = _table_with([(int(r[0]), [int(v) for v in r[1:7]]) for r in rows])
    img = np.full((40, 48), 100, dtype=np.uint8)
    img[:, 40:] = 0  # pitch padding, outside the 40-pixel width
    d1, d2 = oracle.distances(img, 40, 40, (5, 5, 0, 0), trip)
    desc = oracle.extract(img, 40, 40, np.array([[5, 5, 0, 0]]), trip)[0]
    for r in rows:
        t = int(r[0])
        assert (d1[t], d2[t]) == (int(r[7]), int(r[8])), t
        assert _bit(desc, t) == int(r[9]), t
    listed = {int(r[0]) for r in rows}
    assert all(_bit(desc, t) == 0 for t in range(512) if t not in listed)
    assert desc[0] == 0x01 and desc[1] == 0x02 and desc[12] == 0x10


def _delta_image(x0, y0, ox, oy, val=200, size=120):
    img = np.zeros((size, size), dtype=np.uint8)
    img[y0 + oy, x0 + ox] = val
    return img


@pytest.mark.parametrize("case", [
    # (angle bin, scale, image offset of the bright pixel, window position where it must appear)
    (0, 0, (5, -2), (29, 22)),     # upright: window (u, v) = offset + 24
    (8, 0, (5, -2), (22, 19)),     # 90 deg: sample at (-e, a) -> a = -2, e = -5
    (16, 0, (5, -2), (19, 26)),    # 180 deg: (-a, -e)
    (0, 1, (6, -3), (28, 22)),     # scale 1.5: rha(1.5*4) = 6, rha(1.5*-2) = -3
    (0, 1, (5, 0), (27, 24)),      # scale 1.5: rha(1.5*3) = rha(4.5) = 5 (half away from zero)
])
def test_delta_image_closed_form(case):
    """A single bright pixel of value 200 shows up in the window exactly where the
    reading of the offsets puts it.  A triplet whose first companion covers it
    gives D1 = 200^2, D2 = 0 and bit 1; with the companions swapped, bit 0; with
    the anchor covering it, a tie and bit 0."""
    b, si, (ox, oy), (wu, wv) = case
    x0 = y0 = 60
    img = _delta_image(x0, y0, ox, oy)
    far = (6, 41) if wu > 24 else (41, 41)
    rows = [(3, [far[0], far[1], wu, wv, far[0], 6]),     # C1 covers -> 1
            (40, [far[0], far[1], far[0], 6, wu, wv]),    # C2 covers -> 0
            (77, [wu, wv, far[0], far[1], far[0], 6])]    # A covers -> tie -> 0
    trip = _table_with(rows)
    kp = (x0, y0, b, si)
    d1, d2 = oracle.distances(img, 120, 120, kp, trip, synth.SCALES)
    assert (d1[3], d2[3]) == (40000, 0)
    assert (d1[40], d2[40]) == (0, 40000)
    assert (d1[77], d2[77]) == (40000, 40000)
    desc = oracle.extract(img, 120, 120, np.array([kp]), trip, synth.SCALES)[0]
    assert [_bit(desc, t) for t in (3, 40, 77)] == [1, 0, 0]
    assert int(np.unpackbits(desc).sum()) == 1


def _ramp_image(x0, y0, size=120):
    y, x = np.mgrid[0:size, 0:size]
    return np.clip(100 + (x - x0) + 2 * (y - y0), 0, 255).astype(np.uint8)


@pytest.mark.parametrize("b, coef", [(0, (1, 2)), (8, (2, -1)), (16, (-1, -2)), (24, (-2, 1))])
def test_ramp_image_closed_form(triplets, b, coef):
    """On the ramp I = 100 + (x-x0) + 2(y-y0) every patch difference is constant,
    so ||P_A - P_C||^2 = 49 * (cx*(ax-cx') + cy*(ay-cy'))^2 with (cx, cy) the
    ramp's window gradient at that angle.  Checks all 512 seeded triplets."""
    x0 = y0 = 60
    img = _ramp_image(x0, y0)
    d1, d2 = oracle.distances(img, 120, 120, (x0, y0, b, 0), triplets)
    t = triplets.astype(np.int64)
    g1 = coef[0] * (t[:, 0] - t[:, 2]) + coef[1] * (t[:, 1] - t[:, 3])
    g2 = coef[0] * (t[:, 0] - t[:, 4]) + coef[1] * (t[:, 1] - t[:, 5])
    assert np.array_equal(d1, 49 * g1 * g1)
    assert np.array_equal(d2, 49 * g2 * g2)
    desc = oracle.extract(img, 120, 120, np.array([[x0, y0, b, 0]]), triplets)[0]
    bits = np.unpackbits(desc, bitorder="little")
    assert np.array_equal(bits, (np.abs(g1) > np.abs(g2)).astype(np.uint8))


@pytest.fixture(scope="module")
def scene():
    w, h = 160, 128
    img = synth.image(synth.seed(9, 0, synth.KIND_IMAGE), w, h, n_ellipses=12)
    kps = synth.keypoints(synth.seed(9, 0, synth.KIND_KEYPOINTS), w, h, 24, 8, True, 3)
    return img, w, h, kps


def test_identical_companions_and_swap(scene, triplets):
    """Identical companions give 0; swapping the companions flips exactly the
    bits whose distances differ and leaves tied bits 0."""
    img, w, h, kps = scene
    t2 = triplets.copy()
    t2[:, 4:6] = t2[:, 2:4]
    assert not oracle.extract(img, w, h, kps, t2, synth.SCALES).any()
    sw = triplets.copy()
    sw[:, 2:4], sw[:, 4:6] = triplets[:, 4:6], triplets[:, 2:4]
    a = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
    b_ = oracle.extract(img, w, h, kps, sw, synth.SCALES)
    assert not (a & b_).any()
    for i in range(4):
        d1, d2 = oracle.distances(img, w, h, kps[i], triplets, synth.SCALES)
        ba = np.unpackbits(a[i], bitorder="little")
        bb = np.unpackbits(b_[i], bitorder="little")
        assert np.array_equal(ba | bb, (d1 != d2).astype(np.uint8))


def test_constant_and_inverted_images(triplets):
    """A constant image gives the all-zero descriptor; inverting intensities
    (255 - I) leaves every SSD, hence the descriptor, unchanged."""
    w, h = 260, 240
    img = synth.image(synth.seed(9, 1, synth.KIND_IMAGE), w, h, n_ellipses=20)
    kps = synth.keypoints(synth.seed(9, 1, synth.KIND_KEYPOINTS), w, h, 16, 80, True, 3)
    const = np.full_like(img, 77)
    const[:, w:] = 0
    assert not oracle.extract(const, w, h, kps, triplets, synth.SCALES).any()
    inv = (255 - img).astype(np.uint8)
    a = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
    b_ = oracle.extract(inv, w, h, kps, triplets, synth.SCALES)
    assert np.array_equal(a, b_)
    assert a.any()


def test_translation_invariance(triplets):
    """Moving image and keypoint together by an integer shift leaves the
    descriptor unchanged while the window stays inside the image."""
    w, h = 260, 240
    img = synth.image(synth.seed(9, 2, synth.KIND_IMAGE), w, h, n_ellipses=20)
    kps = synth.keypoints(synth.seed(9, 2, synth.KIND_KEYPOINTS), w, h, 16, 80, True, 3)
    big = np.zeros((h + 12, 288), dtype=np.uint8)
    big[12:12 + h, 20:20 + w] = img[:, :w]
    moved = kps.copy()
    moved[:, 0] += 20
    moved[:, 1] += 12
    a = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
    b_ = oracle.extract(big, w + 20, h + 12, moved, triplets, synth.SCALES)
    assert np.array_equal(a, b_)


def test_rotating_image_by_90_matches_bin_plus_8(scene, triplets):
    """Turning the whole image by 90 degrees clockwise (as displayed, y down) and
    adding 8 to the angle bin gives the same descriptor, at every scale and also
    where the window leaves the image.  Pins the direction of rotation."""
    img, w, h, kps = scene
    im = img[:, :w]
    rot = np.ascontiguousarray(np.rot90(im, -1))  # rot[r, c] = im[h-1-c, r]
    kr = kps.copy()
    kr[:, 0] = h - 1 - kps[:, 1]
    kr[:, 1] = kps[:, 0]
    kr[:, 2] = (kps[:, 2] + 8) % 32
    a = oracle.extract(im, w, h, kps, triplets, synth.SCALES)
    b_ = oracle.extract(rot, h, w, kr, triplets, synth.SCALES)
    assert np.array_equal(a, b_)


def test_invalid_inputs_rejected(triplets):
    img = np.zeros((16, 16), np.uint8)
    with pytest.raises(ValueError):
        oracle.extract(img, 16, 16, np.array([[4, 4, 0, 3]]), triplets, synth.SCALES)
    bad = triplets.copy()
    bad[5, 2] = 45
    with pytest.raises(ValueError):
        oracle.extract(img, 16, 16, np.array([[4, 4, 0, 0]]), bad)


# ---------------------------------------------------------------- matching

def _popcount_rows(x):
    return np.unpackbits(x, axis=-1).sum(axis=-1).astype(np.int64)


def test_hamming_metric_axioms():
    """d(a,a) = 0, symmetry, triangle inequality, and agreement with an
    independent popcount (numpy unpackbits)."""
    d = synth.random_descriptors(synth.seed(9, 3, synth.KIND_GALLERY), 24)
    for i in range(24):
        assert oracle.hamming(d[i], d[i]) == 0
        for j in range(24):
            dij = oracle.hamming(d[i], d[j])
            assert dij == oracle.hamming(d[j], d[i])
            assert dij == int(_popcount_rows(d[i] ^ d[j]))
            for k in range(0, 24, 5):
                assert dij <= oracle.hamming(d[i], d[k]) + oracle.hamming(d[k], d[j])


def _sorted_top2(q, t):
    """Independent reference: sort all (distance, index) pairs and take the first two."""
    dist = _popcount_rows(q[:, None, :] ^ t[None, :, :])
    out = []
    for i in range(q.shape[0]):
        order = np.lexsort((np.arange(t.shape[0]), dist[i]))
        out.append((order[0], order[1], dist[i, order[0]], dist[i, order[1]]))
    return out


def test_match_against_full_sort():
    """Top-2 with lowest-index tie-breaking equals the first two entries of a full
    stable sort, on descriptors built to have many tied distances."""
    rng = np.random.default_rng(5)
    q = np.zeros((40, 64), np.uint8)
    t = np.zeros((300, 64), np.uint8)
    q[:, :2] = rng.integers(0, 256, (40, 2))
    t[:, :2] = rng.integers(0, 256, (300, 2))
    m = oracle.match(q, t, 2, 0.8)
    for i, (j1, j2, e1, e2) in enumerate(_sorted_top2(q, t)):
        assert (m["idx1"][i], m["idx2"][i], m["dist1"][i], m["dist2"][i]) == (j1, j2, e1, e2)
        assert m["accepted"][i] == int(1000 * e1 < 800 * e2)


def _with_bits(n):
    d = np.zeros(64, np.uint8)
    for b in range(n):
        d[b >> 3] |= 1 << (b & 7)
    return d


def test_ratio_rule_is_strict():
    """1000*d1 < 800*d2: (4, 5) sits on the boundary and is rejected, (3, 4) is
    accepted; a rule with <= or ratio 0.8 rounded differently fails one of them."""
    q = np.zeros((1, 64), np.uint8)
    for d1, d2, want in ((4, 5, 0), (3, 4, 1), (8, 10, 0), (7, 9, 1), (0, 0, 0), (0, 1, 1)):
        t = np.stack([_with_bits(d2), _with_bits(d1)])
        m = oracle.match(q, t, 2, 0.8)
        first = (1, 0) if d1 < d2 else (0, 1)  # equal distances: lowest index first
        assert (m["idx1"][0], m["idx2"][0], m["dist1"][0], m["dist2"][0]) == (*first, d1, d2)
        assert m["accepted"][0] == want, (d1, d2)


def test_match_degenerate_cases():
    """Identical gallery -> idx1 = 0, idx2 = 1, rejected; nt = 0 -> nothing found;
    nt = 1 -> no second match (65535) and accepted; k = 1 always accepts."""
    q = synth.random_descriptors(7, 3)
    same = np.repeat(q[:1], 5, axis=0)
    m = oracle.match(q[:1], same)
    assert (m["idx1"][0], m["idx2"][0], m["dist1"][0], m["dist2"][0], m["accepted"][0]) == (0, 1, 0, 0, 0)
    m = oracle.match(q, np.zeros((0, 64), np.uint8))
    assert (m["idx1"] == -1).all() and (m["idx2"] == -1).all() and (m["dist1"] == 65535).all()
    assert not m["accepted"].any()
    m = oracle.match(q, q[1:2])
    assert (m["idx1"] == 0).all() and (m["idx2"] == -1).all() and (m["dist2"] == 65535).all()
    assert m["accepted"].all()
    m = oracle.match(q, same, k=1)
    assert m["accepted"].all() and (m["idx2"] == -1).all()
    with pytest.raises(ValueError):
        oracle.match(q, same, k=3)


def test_planted_near_duplicates_closed_form():
    """Each query's planted copy at h in [20, 60] flipped bits is its nearest
    neighbour at exactly distance h and passes the ratio test (random 512-bit
    strings sit near 256 +- 11)."""
    q, g, slots, hs = synth.gallery_workload(n_gallery=2048, n_query=48, config=9)
    m = oracle.match(q, g, 2, 0.8)
    assert np.array_equal(m["idx1"], slots)
    assert np.array_equal(m["dist1"], hs)
    assert m["accepted"].all()
    assert (m["dist2"] > 150).all()


def test_sharded_oracle_equals_the_single_call(triplets):
    """The tests' sharded runs of the oracle (slices of keypoints / query rows in host
    threads, results concatenated in order) give exactly the single call's output."""
    import oracle_shards
    w, h = 200, 160
    img = synth.image(synth.seed(60, 0, synth.KIND_IMAGE), w, h, n_ellipses=10)
    kps = synth.keypoints(synth.seed(60, 0, synth.KIND_KEYPOINTS), w, h, 301, 8, True, 3)
    one = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
    assert np.array_equal(oracle_shards.extract(img, w, h, kps, triplets, synth.SCALES, per=37), one)
    both = oracle_shards.extract_many([(img, w, h, kps, triplets, synth.SCALES), (img, w, h, kps[:5], triplets,
                                                                                  synth.SCALES)], per=16)
    assert np.array_equal(both[0], one) and np.array_equal(both[1], one[:5])
    q = synth.random_descriptors(61, 203)
    t = synth.random_descriptors(62, 500)
    t[::9] = q[3]
    want = oracle.match(q, t, 2, 0.7)
    for got in (oracle_shards.match(q, t, 2, 0.7, per=10), oracle_shards.match_many([(q, t, 2, 0.7)], per=7)[0]):
        for f in want:
            assert np.array_equal(got[f], want[f]), f

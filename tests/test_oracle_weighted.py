"""Pins for the oracle's weighted 8x8 patches (Sec. 3.2, "Weighing pixels in LATCH
patches"): zero weights on the last row and column reproduce the 7x7 descriptor
exactly (the paper's own statement), a uniform weight changes nothing, all-zero
weights give all-zero descriptors, a delta image shows which weight each pixel gets
(catches a transposed table, a wrong patch offset, a dropped row or column), and
swapping the companions flips every untied bit.  No GPU."""
import numpy as np
import pytest

import oracle
from paper_1609_03986_gb300 import synth


def _seven_by_seven(k=1):
    w = np.zeros((8, 8), np.uint8)
    w[:7, :7] = k
    return w


@pytest.fixture(scope="module")
def scene():
    w, h = 300, 220
    img = synth.image(synth.seed(90, 0, synth.KIND_IMAGE), w, h, n_ellipses=40)
    kps = synth.keypoints(synth.seed(90, 0, synth.KIND_KEYPOINTS), w + 60, h + 60, 250, 0, True, 3)
    kps[:, :2] -= 30  # some windows leave the image
    trip = synth.triplets(synth.seed(90, 0, synth.KIND_TRIPLETS), hi=43)
    return img, w, h, kps, trip


@pytest.mark.parametrize("k", [1, 7, 255])
def test_zero_last_row_and_column_is_the_7x7_descriptor(scene, k):
    img, w, h, kps, trip = scene
    want = oracle.extract(img, w, h, kps, trip, synth.SCALES)
    assert np.array_equal(oracle.extract(img, w, h, kps, trip, synth.SCALES, weights=_seven_by_seven(k)), want)


def test_full_8x8_differs_and_zero_weights_give_zero(scene):
    img, w, h, kps, trip = scene
    seven = oracle.extract(img, w, h, kps, trip, synth.SCALES)
    eight = oracle.extract(img, w, h, kps, trip, synth.SCALES, weights=np.ones(64, np.uint8))
    assert (seven != eight).any()  # the 8th row and column take part
    assert not oracle.extract(img, w, h, kps, trip, synth.SCALES, weights=np.zeros(64, np.uint8)).any()


def test_delta_image_shows_each_pixels_weight():
    """Constant window but one pixel P of value 50 + 90; the anchor patch misses P,
    companion 1 holds P at patch pixel (i1, j1) and companion 2 at (i2, j2), so
    D1 = w[i1][j1] 90^2 and D2 = w[i2][j2] 90^2: with weights w[i][j] = 8 i + j + 1
    the bit is 8 i1 + j1 > 8 i2 + j2."""
    x0, y0 = 60, 60
    img = np.full((120, 128), 50, np.uint8)
    px, py = 20, 21  # P in window coordinates (u right, v down)
    img[y0 + py - 24, x0 + px - 24] = 140
    rng = np.random.default_rng(91)
    pos = rng.integers(0, 8, (512, 4))  # i1, j1, i2, j2
    trip = np.zeros((512, 6), np.uint8)
    trip[:, 0:2] = 40  # anchor: window 37..44, away from P
    trip[:, 2] = px + 3 - pos[:, 1]
    trip[:, 3] = py + 3 - pos[:, 0]
    trip[:, 4] = px + 3 - pos[:, 3]
    trip[:, 5] = py + 3 - pos[:, 2]
    weights = (np.arange(64) + 1).astype(np.uint8)
    got = oracle.extract(img, 120, 120, np.array([[x0, y0, 0, 0]], np.int32), trip, (1.0,), weights=weights)
    bits = np.unpackbits(got[0], bitorder="little")
    want = (8 * pos[:, 0] + pos[:, 1]) > (8 * pos[:, 2] + pos[:, 3])
    assert np.array_equal(bits.astype(bool), want)


def test_swapped_companions_flip_untied_bits(scene):
    img, w, h, kps, trip = scene
    gauss = np.array([[int(round(255 * np.exp(-((i - 3.5) ** 2 + (j - 3.5) ** 2) / 8.0))) for j in range(8)]
                      for i in range(8)], np.uint8)
    sw = trip.copy()
    sw[:, [2, 3, 4, 5]] = trip[:, [4, 5, 2, 3]]
    a = np.unpackbits(oracle.extract(img, w, h, kps, trip, synth.SCALES, weights=gauss), axis=1)
    b = np.unpackbits(oracle.extract(img, w, h, kps, sw, synth.SCALES, weights=gauss), axis=1)
    assert not (a & b).any() and (a | b).mean() > 0.75  # ties (flat or outside parts) stay 0 both ways


def test_weighted_patches_need_coordinates_up_to_43(scene):
    img, w, h, kps, trip = scene
    bad = trip.copy()
    bad[5, 4] = 44
    with pytest.raises(ValueError):
        oracle.extract(img, w, h, kps[:3], bad, synth.SCALES, weights=np.ones(64, np.uint8))
    oracle.extract(img, w, h, kps[:3], bad, synth.SCALES)  # the 7x7 patches take 44

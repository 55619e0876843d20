"""Pins for the oracle's multi-scale pyramid (Sec. 6: CLATCH at multiple scales):
level images by hand (nearest pixel at spacing s, rounded half away from zero), the
size floor(W / s), level 0 = plain detection, every level = detection on its own
image with coordinates mapped back, and each keypoint sitting on the base pixel its
level pixel came from.  No GPU."""
import numpy as np
import pytest

import oracle
from paper_1609_03986_gb300 import synth


def test_level_images_by_hand():
    img = (np.arange(20)[None, :] + 10 * (np.arange(20)[:, None] % 2)).astype(np.uint8)  # I(x, y) = x + 10 (y mod 2)
    # s = 1.5: x -> 0, 2 (1.5), 3, 5 (4.5), 6, 8 (7.5), 9, 11 (10.5), 12, 14 (13.5), 15, 17 (16.5), 18; 13 columns
    want_x = [0, 2, 3, 5, 6, 8, 9, 11, 12, 14, 15, 17, 18]
    lev = oracle.pyramid_level(img, 20, 20, 1.5)
    assert lev.shape == (13, 13)
    assert list(lev[0]) == want_x
    assert list(lev[:, 0]) == [10 * (v % 2) for v in want_x]  # rows y -> the same map
    # s = 2.25: x -> 0, 2 (2.25), 5 (4.5), 7 (6.75), 9, 11 (11.25), 14 (13.5), 16 (15.75); 8 columns
    lev = oracle.pyramid_level(img, 20, 20, 2.25)
    assert lev.shape == (8, 8)
    assert list(lev[0]) == [0, 2, 5, 7, 9, 11, 14, 16]
    assert np.array_equal(oracle.pyramid_level(img, 20, 20, 1.0), img)
    assert oracle.pyramid_level(img, 20, 17, 1.5).shape == (11, 13)


@pytest.fixture(scope="module")
def scene():
    w, h = 400, 300
    return synth.image(synth.seed(95, 0, synth.KIND_IMAGE), w, h, n_ellipses=60), w, h


def test_level_zero_is_plain_detection(scene):
    img, w, h = scene
    pyr = oracle.detect_pyramid(img, w, h, 20, (1.0, 1.5, 2.25))
    plain = oracle.detect(img, w, h, 20)
    l0 = pyr[pyr[:, 3] == 0]
    assert np.array_equal(l0[:, :3], plain)
    assert list(np.unique(pyr[:, 3])) == [0, 1, 2]
    assert np.all(np.diff(pyr[:, 3]) >= 0)  # level after level


@pytest.mark.parametrize("s", [1.5, 2.25, 2.0])
def test_each_level_is_detection_on_its_image(scene, s):
    img, w, h = scene
    pyr = oracle.detect_pyramid(img, w, h, 15, (1.0, s))
    lev = oracle.pyramid_level(img, w, h, s)
    own = oracle.detect(lev, lev.shape[1], lev.shape[0], 15)
    got = pyr[pyr[:, 3] == 1]
    mapped = np.stack([np.floor(s * own[:, 0] + 0.5), np.floor(s * own[:, 1] + 0.5)], 1).astype(np.int32)
    assert np.array_equal(got[:, :2], mapped) and np.array_equal(got[:, 2], own[:, 2])
    # every keypoint sits on the base pixel its level pixel was sampled from
    assert np.array_equal(img[got[:, 1], got[:, 0]], lev[own[:, 1], own[:, 0]])


def test_pyramid_rejects_scales_below_one(scene):
    img, w, h = scene
    with pytest.raises(ValueError):
        oracle.detect_pyramid(img, w, h, 20, (1.0, 0.75))

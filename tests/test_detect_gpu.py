"""Parity of GPU keypoint detection (oriented FAST, Sec. 3.2) and of the fused
detect-then-extract call with the CPU oracle through the C ABI: the same keypoint
set (in the documented 32x32-cell order), the same angle bins, the same count,
truncation at max_kps, and the descriptors of the detected keypoints."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
from conftest import to_dev

pytestmark = pytest.mark.gpu


def _cell_order(kp, width):
    """Keypoints (x, y, ...) sorted as the library writes them: 32x32 cells row by row,
    then row by row inside a cell."""
    gx = (width + 31) // 32
    k = kp.astype(np.int64)
    key = ((k[:, 1] // 32) * gx + k[:, 0] // 32) * 1024 + (k[:, 1] % 32) * 32 + k[:, 0] % 32
    return kp[np.argsort(key, kind="stable")]


def _near_boundary(img, x, y):
    """theta * 16 / pi within 1e-7 of a half-integer (rounding may go either way there)."""
    yy, xx = np.mgrid[-15:16, -15:16]
    m = (xx ** 2 + yy ** 2) <= 225
    patch = img[y - 15:y + 16, x - 15:x + 16].astype(np.int64)
    v = np.arctan2((yy * patch)[m].sum(), (xx * patch)[m].sum()) * 16 / np.pi
    return abs(abs(v - np.floor(v)) - 0.5) < 1e-7


def _gpu_detect(ctx, img, w, h, t, max_kps, scale_idx=0, with_desc=False):
    out = ctx.detect(to_dev(img), w, h, t, max_kps, scale_idx, with_desc)
    torch.cuda.synchronize()
    n = int(out[1].item())
    m = min(n, max_kps)
    kp = P.unpack_keypoints(out[0][:m].cpu().numpy())
    if with_desc:
        return n, kp, out[2][:m].cpu().numpy()
    return n, kp


def _same_keypoints(img, got, want, scale_idx):
    assert np.array_equal(got[:, :2], want[:, :2])
    assert (got[:, 3] == scale_idx).all()
    diff = np.nonzero(got[:, 2] != want[:, 2])[0]
    assert all(_near_boundary(img, int(want[i, 0]), int(want[i, 1])) for i in diff), diff


@pytest.mark.parametrize("w, h, t", [(640, 480, 20), (333, 251, 10), (640, 480, 60), (48, 48, 5), (40, 40, 5),
                                     (33, 70, 5), (20, 20, 5), (1920, 1080, 25)])
def test_detect_equals_oracle(gpu_ctx, w, h, t):
    img = synth.image(synth.seed(80, w * 7 + h, synth.KIND_IMAGE), w, h, n_ellipses=60)
    want = _cell_order(oracle.detect(img, w, h, t), w)
    n, got = _gpu_detect(gpu_ctx, img, w, h, t, max(1, 4 * len(want)), scale_idx=1)
    assert n == len(want)
    _same_keypoints(img, got, want, 1)


def test_detect_dense_corners(gpu_ctx):
    """A noise image with corners almost everywhere (the most keypoints a cell can
    hold after suppression) and the smallest threshold."""
    rng = np.random.default_rng(81)
    w, h = 256, 200
    img = np.zeros((h, 256), np.uint8)
    img[:, :w] = rng.integers(0, 256, (h, w))
    want = _cell_order(oracle.detect(img, w, h, 1), w)
    n, got = _gpu_detect(gpu_ctx, img, w, h, 1, len(want) + 5)
    assert n == len(want) and n > 3000
    _same_keypoints(img, got, want, 0)


def test_detect_longest_sides(gpu_ctx):
    for w, h in ((32768, 40), (40, 32768)):
        img = synth.image(synth.seed(82, w, synth.KIND_IMAGE), w, h, n_ellipses=200)
        want = _cell_order(oracle.detect(img, w, h, 15), w)
        n, got = _gpu_detect(gpu_ctx, img, w, h, 15, len(want) + 1)
        assert n == len(want) and n > 0
        _same_keypoints(img, got, want, 0)


def test_detect_truncates_at_max_kps(gpu_ctx):
    w, h = 640, 480
    img = synth.image(synth.seed(83, 0, synth.KIND_IMAGE), w, h, n_ellipses=80)
    want = _cell_order(oracle.detect(img, w, h, 20), w)
    for cap in (0, 1, 37, len(want) - 1):
        n, got = _gpu_detect(gpu_ctx, img, w, h, 20, cap)
        assert n == len(want) and len(got) == cap
        _same_keypoints(img, got, want[:cap], 0)


def test_detect_extract_equals_oracle(gpu_ctx, triplets):
    """Detection then extraction in one call: the descriptors of the detected
    keypoints equal the oracle's descriptors of the oracle's keypoints, at each
    scale of the table, and a truncated call describes the first max_kps."""
    w, h = 1280, 720
    img = synth.image(synth.seed(84, 0, synth.KIND_IMAGE), w, h, n_ellipses=120)
    want = _cell_order(oracle.detect(img, w, h, 20), w)
    for sc in range(3):
        n, got, desc = _gpu_detect(gpu_ctx, img, w, h, 20, len(want) + 100, scale_idx=sc, with_desc=True)
        assert n == len(want)
        _same_keypoints(img, got, want, sc)
        kps = np.concatenate([want, np.full((len(want), 1), sc, np.int32)], 1)
        assert np.array_equal(desc, oracle.extract(img, w, h, kps, triplets, synth.SCALES)), sc
    n, got, desc = _gpu_detect(gpu_ctx, img, w, h, 20, 500, with_desc=True)
    kps = np.concatenate([want[:500], np.zeros((500, 1), np.int32)], 1)
    assert np.array_equal(desc, oracle.extract(img, w, h, kps, triplets, synth.SCALES))
    gpu_ctx.check()


def test_detect_rejects_bad_arguments(gpu_ctx):
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    kps = torch.zeros((10, 12), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for t, sc in ((0, 0), (255, 0), (20, 3), (20, -1)):
        with pytest.raises(P.LatchError) as e:
            P.latch_detect(gpu_ctx.handle, img, 64, 64, 64, t, sc, 10, kps, cnt, 0)
        assert e.value.status == 1
    with pytest.raises(P.LatchError):
        P.latch_detect(gpu_ctx.handle, img, 64, 64, 64, 20, 0, 10, kps, 0, 0)

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


def _pyramid_order(kp, width, scales):
    """Keypoints (x, y, bin, level) in the library's pyramid order: level after level,
    each level in the cell order of its own image (level coordinates recovered as
    round(x / s): |rha(s x) - s x| <= 1/2 < s/2)."""
    out = []
    for l, s in enumerate(scales):
        k = kp[kp[:, 3] == l].astype(np.int64)
        lx, ly = np.rint(k[:, 0] / s).astype(np.int64), np.rint(k[:, 1] / s).astype(np.int64)
        gx = (int(np.floor(width / s)) + 31) // 32
        key = ((ly // 32) * gx + lx // 32) * 1024 + (ly % 32) * 32 + lx % 32
        out.append(k[np.argsort(key, kind="stable")])
    return np.concatenate(out).astype(np.int32)


@pytest.mark.parametrize("w, h, t", [(640, 480, 20), (1920, 1080, 25), (101, 77, 10)])
def test_pyramid_equals_oracle(gpu_ctx, triplets, w, h, t):
    """Every level of the default scale table {1, 1.5, 2.25}: the same keypoints
    (base coordinates, bins, level as scale index) in the documented order, and the
    descriptors of all of them at their level's scale."""
    img = synth.image(synth.seed(85, w + h, synth.KIND_IMAGE), w, h, n_ellipses=80)
    want = _pyramid_order(oracle.detect_pyramid(img, w, h, t, synth.SCALES), w, synth.SCALES)
    cap = len(want) + 50
    kps = torch.empty((cap, 12), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    desc = torch.empty((cap, 64), dtype=torch.uint8, device="cuda")
    d_img = to_dev(img)
    P.latch_detect_pyramid(gpu_ctx.handle, d_img, w, h, d_img.stride(0), t, 3, cap, kps, cnt, desc,
                           int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert n == len(want)
    got = P.unpack_keypoints(kps[:n].cpu().numpy())
    assert np.array_equal(got[:, [0, 1, 3]], want[:, [0, 1, 3]])
    for l, s in enumerate(synth.SCALES):  # bins: exact but for rounding ties at a half-integer
        lev = oracle.pyramid_level(img, w, h, s)
        sel = np.nonzero((want[:, 3] == l) & (got[:, 2] != want[:, 2]))[0]
        assert all(_near_boundary(lev, int(round(want[i, 0] / s)), int(round(want[i, 1] / s))) for i in sel)
    assert np.array_equal(desc[:n].cpu().numpy(), oracle.extract(img, w, h, want, triplets, synth.SCALES))
    gpu_ctx.check()


def test_pyramid_level_count_and_scales(gpu_ctx):
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    kps = torch.zeros((10, 12), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for nl in (0, 4):
        with pytest.raises(P.LatchError) as e:
            P.latch_detect_pyramid(gpu_ctx.handle, img, 64, 64, 64, 20, nl, 10, kps, cnt)
        assert e.value.status == 1
    ctx = P.Context(0, scales=(1.0, 0.5))
    try:
        P.latch_detect_pyramid(ctx.handle, img, 64, 64, 64, 20, 1, 10, kps, cnt)
        with pytest.raises(P.LatchError):
            P.latch_detect_pyramid(ctx.handle, img, 64, 64, 64, 20, 2, 10, kps, cnt)
    finally:
        ctx.close()

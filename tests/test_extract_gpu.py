"""Parity of the CUDA extraction path with the CPU oracle, bit for bit, through the
C ABI.  Sizes span many thread blocks with ragged tails; edge cases cover empty
input, keypoints at and beyond the border, every angle bin and scale, and a bad
scale index."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
from conftest import to_dev

pytestmark = pytest.mark.gpu


def _extract(ctx, img, w, h, kps, triplets=None):
    out = ctx.extract(to_dev(img), w, h, to_dev(P.pack_keypoints(kps)), triplets)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_plain_pair_parity(gpu_ctx, triplets):
    """Both images of the upright 640x480 pair workload, every keypoint (2 x 2,000)."""
    wl = synth.pair("plain_640x480_2k")
    for img, kps in zip(wl["images"], wl["kps"]):
        got = _extract(gpu_ctx, img, wl["width"], wl["height"], kps)
        want = oracle.extract(img, wl["width"], wl["height"], kps, triplets, synth.SCALES)
        assert np.array_equal(got, want)
    gpu_ctx.check()


def test_oriented_pair_parity(gpu_ctx, oriented_pair_oracle):
    """Both images of the oriented and scaled 1920x1080 pair workload, all 2 x 10,000
    descriptors against the (sharded) oracle, plus a ragged 3,001-keypoint prefix
    (a launch whose last batch of 32 is partly empty)."""
    wl, descs = oriented_pair_oracle["wl"], oriented_pair_oracle["descs"]
    for img, kps, want in zip(wl["images"], wl["kps"], descs):
        assert np.array_equal(_extract(gpu_ctx, img, wl["width"], wl["height"], kps), want)
        assert np.array_equal(_extract(gpu_ctx, img, wl["width"], wl["height"], kps[:3001]), want[:3001])
    gpu_ctx.check()


def test_every_bin_and_scale_near_borders(gpu_ctx, triplets):
    """All 32 bins x 3 scales, keypoints within 5 px of the border and outside the
    image (windows partly or wholly outside read zeros)."""
    w, h = 333, 250
    img = synth.image(synth.seed(11, 0, synth.KIND_IMAGE), w, h, n_ellipses=30)
    rng = np.random.default_rng(3)
    pts = []
    for b in range(32):
        for s in range(3):
            for x, y in ((0, 0), (w - 1, h - 1), (2, h // 2), (w // 2, 4), (w - 3, 7)):
                pts.append((x, y, b, s))
    pts += [(-10, 40, 3, 1), (w + 5, h + 90, 9, 2), (-200, -200, 0, 0), (w // 2, h // 2, 31, 2)]
    xs = rng.integers(-40, w + 40, 300)
    ys = rng.integers(-40, h + 40, 300)
    pts += [(int(x), int(y), int(rng.integers(0, 32)), int(rng.integers(0, 3))) for x, y in zip(xs, ys)]
    kps = np.array(pts, dtype=np.int32)
    got = _extract(gpu_ctx, img, w, h, kps)
    want = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
    assert np.array_equal(got, want)
    gpu_ctx.check()


def test_bin_wraps_modulo_32(gpu_ctx, triplets):
    w, h = 200, 200
    img = synth.image(synth.seed(11, 1, synth.KIND_IMAGE), w, h, n_ellipses=10)
    kps = np.array([[100, 100, b, 1] for b in range(32)], np.int32)
    a = _extract(gpu_ctx, img, w, h, kps)
    kps2 = kps.copy()
    kps2[:, 2] += 32
    assert np.array_equal(a, _extract(gpu_ctx, img, w, h, kps2))


def test_tiny_and_odd_images(gpu_ctx, triplets):
    for w, h in ((1, 1), (7, 3), (17, 64), (48, 48)):
        pitch = (w + 15) // 16 * 16
        img = synth.image(synth.seed(11, w, synth.KIND_IMAGE), w, h, pitch, n_ellipses=2)
        kps = np.array([[0, 0, 0, 0], [w // 2, h // 2, 5, 2], [w - 1, h - 1, 20, 1]], np.int32)
        got = _extract(gpu_ctx, img, w, h, kps)
        assert np.array_equal(got, oracle.extract(img, w, h, kps, triplets, synth.SCALES))


def test_longest_image_sides(gpu_ctx, triplets):
    """Images at the 32,768-pixel limit in either direction, keypoints at, near and
    beyond the far corners (some far enough that their windows miss the image, some
    at coordinates near the int32 range), every scale."""
    rng = np.random.default_rng(13)
    for w, h in ((32768, 40), (40, 32768)):
        img = synth.image(synth.seed(13, w, synth.KIND_IMAGE), w, h, n_ellipses=20)
        pts = []
        for x0, y0 in ((0, 0), (w - 1, 0), (0, h - 1), (w - 1, h - 1), (w // 2, h // 2)):
            for dx, dy in ((0, 0), (-60, 30), (90, -90), (-130, 0), (0, 140), (200, 200)):
                pts.append([x0 + dx, y0 + dy, int(rng.integers(0, 32)), int(rng.integers(0, 3))])
        pts += [[2**30, 5, 3, 1], [-2**30, -2**30, 7, 2], [w + 77, h + 77, 9, 2]]
        kps = np.array(pts, np.int32)
        got = _extract(gpu_ctx, img, w, h, kps)
        assert np.array_equal(got, oracle.extract(img, w, h, kps, triplets, synth.SCALES)), (w, h)


def test_empty_and_invalid_arguments(gpu_ctx, triplets):
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    kps = torch.zeros((0, 12), dtype=torch.uint8, device="cuda")
    out = gpu_ctx.extract(img, 64, 64, kps)
    assert out.shape == (0, 64)
    bad = triplets.copy()
    bad[7, 3] = 2
    with pytest.raises(P.LatchError) as e:
        gpu_ctx.extract(img, 64, 64, to_dev(P.pack_keypoints([[5, 5, 0, 0]])), bad)
    assert e.value.status == 1
    with pytest.raises(P.LatchError):  # pitch not a multiple of 16
        P.latch_extract(gpu_ctx.handle, img, 60, 64, 60, 0, 0, None, 0, 0)
    with pytest.raises(P.LatchError):
        P.latch_extract(gpu_ctx.handle, img, 64, 64, 64, 0, -1, None, 0, 0)


def test_bad_scale_index_flags_device_error(gpu_ctx, triplets):
    w, h = 100, 100
    img = synth.image(synth.seed(11, 2, synth.KIND_IMAGE), w, h, n_ellipses=5)
    kps = np.array([[50, 50, 0, 0], [50, 50, 0, 7], [40, 40, 3, 2]], np.int32)
    got = _extract(gpu_ctx, img, w, h, kps)
    with pytest.raises(P.LatchError) as e:
        gpu_ctx.check()
    assert e.value.status == 8
    assert not got[1].any()
    good = kps[[0, 2]]
    assert np.array_equal(got[[0, 2]], oracle.extract(img, w, h, good, triplets, synth.SCALES))
    gpu_ctx.check()  # the flag was cleared


def test_triplet_table_switch(gpu_ctx, triplets):
    """Passing a different table per call is honoured and restored."""
    w, h = 160, 120
    img = synth.image(synth.seed(11, 3, synth.KIND_IMAGE), w, h, n_ellipses=8)
    kps = synth.keypoints(synth.seed(11, 3, synth.KIND_KEYPOINTS), w, h, 50, 10, True, 3)
    other = synth.triplets(12345)
    got = _extract(gpu_ctx, img, w, h, kps, other)
    assert np.array_equal(got, oracle.extract(img, w, h, kps, other, synth.SCALES))
    got = _extract(gpu_ctx, img, w, h, kps, triplets)
    assert np.array_equal(got, oracle.extract(img, w, h, kps, triplets, synth.SCALES))


def test_degenerate_triplet_tables(gpu_ctx, triplets):
    """Tables with identical companions (bit always 0), the anchor on companion 1
    (D1 = 0: bit 0) or on companion 2 (bit 1 unless D1 = 0), and patches at the
    extreme centres 3 and 44; and the regular table with the companions swapped
    (every bit flips except ties).  GPU = oracle, and the invariants hold."""
    w, h = 400, 300
    img = synth.image(synth.seed(14, 0, synth.KIND_IMAGE), w, h, n_ellipses=30)
    kps = synth.keypoints(synth.seed(14, 0, synth.KIND_KEYPOINTS), w, h, 300, 0, True, 3)
    rng = np.random.default_rng(14)
    t = rng.integers(3, 45, (512, 6)).astype(np.uint8)
    t[0:128, 4:6] = t[0:128, 2:4]      # C2 = C1
    t[128:256, 2:4] = t[128:256, 0:2]  # C1 = A
    t[256:384, 4:6] = t[256:384, 0:2]  # C2 = A
    t[384:512] = rng.choice([3, 44], (128, 6)).astype(np.uint8)
    got = _extract(gpu_ctx, img, w, h, kps, t)
    assert np.array_equal(got, oracle.extract(img, w, h, kps, t, synth.SCALES))
    bits = np.unpackbits(got, axis=1, bitorder="little")
    assert not bits[:, 0:256].any()
    swapped = triplets.copy()
    swapped[:, [2, 3, 4, 5]] = triplets[:, [4, 5, 2, 3]]
    # (a table passed to a call stays loaded: the regular one goes last)
    b = np.unpackbits(_extract(gpu_ctx, img, w, h, kps, swapped), axis=1, bitorder="little")
    a = np.unpackbits(_extract(gpu_ctx, img, w, h, kps, triplets), axis=1, bitorder="little")
    want = oracle.extract(img, w, h, kps, swapped, synth.SCALES)
    assert np.array_equal(b, np.unpackbits(want, axis=1, bitorder="little"))
    assert not (a & b).any()  # never both set: D1 > D2 and D2 > D1 exclude each other
    assert (a | b).mean() > 0.9  # and one of them is set unless the distances tie


def test_device_wait_timeout_is_reported(gpu_ctx, triplets):
    """A device-side wait that can never complete gives up after its limit and the
    host sees LATCH_ETIMEOUT; the context keeps working afterwards."""
    P.latch_selftest_wait_timeout(gpu_ctx.handle, 20000, 0)
    with pytest.raises(P.LatchError) as e:
        gpu_ctx.check()
    assert e.value.status == 6
    gpu_ctx.check()  # the flag was cleared
    w, h = 120, 90
    img = synth.image(synth.seed(11, 9, synth.KIND_IMAGE), w, h, n_ellipses=5)
    kps = np.array([[60, 45, 3, 1], [10, 10, 30, 2]], np.int32)
    assert np.array_equal(_extract(gpu_ctx, img, w, h, kps), oracle.extract(img, w, h, kps, triplets, synth.SCALES))


def test_autotune_changes_speed_not_results(gpu_ctx, triplets):
    """The autotuner picks a work-item size and a path threshold within range; every
    item size gives the same descriptors; tuning can be saved and restored."""
    saved = P.latch_get_tuning(gpu_ctx.handle)
    try:
        t = P.latch_autotune(gpu_ctx.handle, 640, 480, 3000, 2000, 2000)
        assert 1 <= t["item_kps"] <= 32 and t["tensor_min_pairs"] >= 0
        w, h = 640, 480
        img = synth.image(synth.seed(11, 20, synth.KIND_IMAGE), w, h, n_ellipses=30)
        kps = synth.keypoints(synth.seed(11, 20, synth.KIND_KEYPOINTS), w, h, 900, 8, True, 3)
        want = oracle.extract(img, w, h, kps, triplets, synth.SCALES)
        for item in (1, 5, 16, 32):
            P.latch_set_tuning(gpu_ctx.handle, item, t["tensor_min_pairs"])
            assert np.array_equal(_extract(gpu_ctx, img, w, h, kps), want), item
        with pytest.raises(P.LatchError):
            P.latch_set_tuning(gpu_ctx.handle, 33, 0)
    finally:
        P.latch_set_tuning(gpu_ctx.handle, saved["item_kps"], saved["tensor_min_pairs"])
    gpu_ctx.check()


def test_batch_and_run_boundaries(gpu_ctx, triplets):
    """Layouts aimed at the extraction's batches of 32 keypoints (one per lane) and its
    per-cell tile runs: 150 keypoints in one 32x32 cell (runs spanning several
    batches), one keypoint in each of 300 cells (a tile per keypoint), and counts
    around multiples of 32; each at several work-item sizes, so that batches are split
    between blocks at many chunk offsets."""
    w, h = 1024, 768
    img = synth.image(synth.seed(11, 40, synth.KIND_IMAGE), w, h, n_ellipses=40)
    rng = np.random.default_rng(17)

    def attrs(n):
        return rng.integers(0, 32, n), rng.integers(0, 3, n)

    cases = []
    b, s = attrs(150)
    cases.append(np.stack([320 + rng.integers(0, 32, 150), 256 + rng.integers(0, 32, 150), b, s], 1))
    gx, gy = np.meshgrid(np.arange(20), np.arange(15))
    b, s = attrs(300)
    cases.append(np.stack([gx.ravel() * 32 + rng.integers(0, 32, 300), gy.ravel() * 32 + rng.integers(0, 32, 300), b, s], 1))
    for n in (1, 31, 32, 33, 64, 65, 97):
        b, s = attrs(n)
        cases.append(np.stack([rng.integers(-20, w + 20, n), rng.integers(-20, h + 20, n), b, s], 1))
    cases = [c.astype(np.int32) for c in cases]
    wants = [oracle.extract(img, w, h, k, triplets, synth.SCALES) for k in cases]
    saved = P.latch_get_tuning(gpu_ctx.handle)
    try:
        for item in (1, 7, 32):
            P.latch_set_tuning(gpu_ctx.handle, item, saved["tensor_min_pairs"])
            for k, want in zip(cases, wants):
                assert np.array_equal(_extract(gpu_ctx, img, w, h, k), want), (item, len(k))
    finally:
        P.latch_set_tuning(gpu_ctx.handle, saved["item_kps"], saved["tensor_min_pairs"])
    gpu_ctx.check()

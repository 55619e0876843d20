"""Parity of the weighted 8x8-patch extraction (Sec. 3.2, weighing pixels in LATCH
patches) with the oracle through the C ABI, on the plain and the batched entry
points; the zero-row-and-column table reproduces the 7x7 descriptors."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
from conftest import to_dev

pytestmark = pytest.mark.gpu

GAUSS = np.array([[int(round(255 * np.exp(-((i - 3.5) ** 2 + (j - 3.5) ** 2) / 8.0))) for j in range(8)]
                  for i in range(8)], np.uint8)


@pytest.fixture(scope="module")
def wctx():
    """A context of its own (the weights stay set on it), triplets within [3, 43]."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    trip = synth.triplets(synth.seed(92, 0, synth.KIND_TRIPLETS), hi=43)
    ctx = P.Context(0, triplets=trip)
    yield ctx, trip
    ctx.close()


def _scene(seed, w, h, n):
    img = synth.image(synth.seed(92, seed, synth.KIND_IMAGE), w, h, n_ellipses=60)
    kps = synth.keypoints(synth.seed(92, seed, synth.KIND_KEYPOINTS), w + 80, h + 80, n, 0, True, 3)
    kps[:, :2] -= 40
    return img, kps


def _extract(ctx, img, w, h, kps):
    out = ctx.extract(to_dev(img), w, h, to_dev(P.pack_keypoints(kps)))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("weights", ["gauss", "ones", "ramp"])
def test_weighted_equals_oracle(wctx, weights):
    ctx, trip = wctx
    wt = {"gauss": GAUSS, "ones": np.ones((8, 8), np.uint8),
          "ramp": (np.arange(64).reshape(8, 8) * 4 + 3).astype(np.uint8)}[weights]
    img, kps = _scene(1, 700, 500, 3001)
    P.latch_set_patch_weights(ctx.handle, wt)
    try:
        got = _extract(ctx, img, 700, 500, kps)
    finally:
        P.latch_set_patch_weights(ctx.handle, None)
    assert np.array_equal(got, oracle.extract(img, 700, 500, kps, trip, synth.SCALES, weights=wt))
    ctx.check()


def test_zero_last_row_and_column_equals_7x7(wctx):
    ctx, trip = wctx
    img, kps = _scene(2, 400, 300, 777)
    plain = _extract(ctx, img, 400, 300, kps)
    w7 = np.zeros((8, 8), np.uint8)
    w7[:7, :7] = 9
    P.latch_set_patch_weights(ctx.handle, w7)
    try:
        weighted = _extract(ctx, img, 400, 300, kps)
    finally:
        P.latch_set_patch_weights(ctx.handle, None)
    assert np.array_equal(weighted, plain)
    assert np.array_equal(plain, oracle.extract(img, 400, 300, kps, trip, synth.SCALES))


def test_weighted_batch_equals_oracle(wctx):
    """Two images and a pair through latch_batch_run with the Gaussian table."""
    ctx, trip = wctx
    scenes = [_scene(3 + i, 500, 400, 1500 + 301 * i) for i in range(2)]
    imgs = [to_dev(im) for im, _ in scenes]
    n = [len(k) for _, k in scenes]
    d_kps = to_dev(np.concatenate([P.pack_keypoints(k) for _, k in scenes]))
    d_desc = torch.zeros((sum(n), 64), dtype=torch.uint8, device="cuda")
    d_m = torch.zeros((n[0], 16), dtype=torch.uint8, device="cuda")
    b = P.BatchDesc([(t, 500, 400, t.stride(0)) for t in imgs], n, d_kps, d_desc, [(0, 1)], 2, 0.8, d_m)
    P.latch_set_patch_weights(ctx.handle, GAUSS)
    try:
        P.latch_batch_run(ctx.handle, b, int(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
    finally:
        P.latch_set_patch_weights(ctx.handle, None)
    ctx.check()
    want = [oracle.extract(im, 500, 400, k, trip, synth.SCALES, weights=GAUSS) for im, k in scenes]
    got = d_desc.cpu().numpy()
    assert np.array_equal(got[:n[0]], want[0]) and np.array_equal(got[n[0]:], want[1])
    m = P.matches_from_bytes(d_m.cpu().numpy())
    o = oracle.match(want[0], want[1], 2, 0.8)
    for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
        assert np.array_equal(m[f].astype(np.int64), o[f].astype(np.int64)), f


def test_weights_need_coordinates_up_to_43(gpu_ctx, triplets):
    """The seeded table reaches 44: weights are refused while it is loaded, and a
    44 in a later table is refused while weights are set."""
    assert triplets.max() == 44
    with pytest.raises(P.LatchError) as e:
        P.latch_set_patch_weights(gpu_ctx.handle, GAUSS)
    assert e.value.status == 1
    ctx = P.Context(0, triplets=synth.triplets(synth.seed(92, 1, synth.KIND_TRIPLETS), hi=43))
    try:
        P.latch_set_patch_weights(ctx.handle, GAUSS)
        with pytest.raises(P.LatchError):
            P.latch_set_triplets(ctx.handle, triplets)
    finally:
        ctx.close()

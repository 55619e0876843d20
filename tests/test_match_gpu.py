"""Parity of the CUDA matching paths with the CPU oracle through the C ABI: exact
indices, distances and ratio-test verdicts, on tie-heavy inputs, ragged sizes,
degenerate cases and sampled rows of the million-descriptor gallery."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
from conftest import match_records, to_dev

pytestmark = pytest.mark.gpu
PATHS = [P.PATH_POPC, P.PATH_TENSOR, P.PATH_AUTO]


def _match(ctx, q, t, k=2, ratio=0.8, path=P.PATH_AUTO):
    out = ctx.match(to_dev(q), to_dev(t), k, ratio, path)
    torch.cuda.synchronize()
    return match_records(out)


def _same(got, want):
    for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
        assert np.array_equal(got[f].astype(np.int64), want[f].astype(np.int64)), f


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("nq, nt", [(1, 1), (3, 2), (129, 257), (1000, 777), (517, 4099)])
def test_random_parity(gpu_ctx, path, nq, nt):
    q = synth.random_descriptors(synth.seed(12, nq, synth.KIND_GALLERY), nq)
    t = synth.random_descriptors(synth.seed(12, nt + 7, synth.KIND_GALLERY), nt)
    _same(_match(gpu_ctx, q, t, path=path), oracle.match(q, t))


@pytest.mark.parametrize("path", PATHS)
def test_tie_heavy_parity(gpu_ctx, path):
    """Only 12 random bits per descriptor: many equal distances, so the lowest-index
    rule decides most results."""
    rng = np.random.default_rng(8)
    q = np.zeros((700, 64), np.uint8)
    t = np.zeros((3000, 64), np.uint8)
    q[:, 7] = rng.integers(0, 256, 700)
    q[:, 30] = rng.integers(0, 16, 700)
    t[:, 7] = rng.integers(0, 256, 3000)
    t[:, 30] = rng.integers(0, 16, 3000)
    for k in (1, 2):
        _same(_match(gpu_ctx, q, t, k=k, path=path), oracle.match(q, t, k=k))


@pytest.mark.parametrize("path", PATHS)
def test_degenerate(gpu_ctx, path):
    q = synth.random_descriptors(5, 40)
    same = np.repeat(q[:1], 9, axis=0)
    _same(_match(gpu_ctx, q, same, path=path), oracle.match(q, same))
    _same(_match(gpu_ctx, q, q[:1], path=path), oracle.match(q, q[:1]))
    empty = np.zeros((0, 64), np.uint8)
    got = _match(gpu_ctx, q, empty, path=path)
    assert (got["idx1"] == -1).all() and (got["dist1"] == 65535).all() and not got["accepted"].any()
    for ratio in (0.0, 0.55, 1.0):
        _same(_match(gpu_ctx, q, q[::-1].copy(), ratio=ratio, path=path), oracle.match(q, q[::-1], ratio=ratio))
    out = gpu_ctx.match(to_dev(empty), to_dev(q))
    assert out.shape == (0, 16)


def test_invalid_arguments(gpu_ctx):
    q = to_dev(synth.random_descriptors(5, 4))
    for kw in ({"k": 3}, {"ratio": 1.5}, {"ratio": -0.1}, {"path": 9}):
        with pytest.raises(P.LatchError) as e:
            gpu_ctx.match(q, q, **kw)
        assert e.value.status == 1


def test_pair_workload_parity(gpu_ctx, triplets):
    """Extract both images of the plain 640x480 workload on the GPU and match them
    2,000 x 2,000; descriptors and matches equal the oracle's."""
    wl = synth.pair("plain_640x480_2k")
    descs = []
    for img, kps in zip(wl["images"], wl["kps"]):
        d = gpu_ctx.extract(to_dev(img), wl["width"], wl["height"], to_dev(P.pack_keypoints(kps)))
        descs.append(d)
    torch.cuda.synchronize()
    q, t = (d.cpu().numpy() for d in descs)
    assert np.array_equal(q, oracle.extract(wl["images"][0], wl["width"], wl["height"], wl["kps"][0], triplets))
    want = oracle.match(q, t)
    for path in PATHS:
        _same(match_records(gpu_ctx.match(descs[0], descs[1], 2, 0.8, path)), want)


@pytest.mark.parametrize("path", PATHS)
def test_million_gallery_sampled(gpu_ctx, path):
    """16,384 queries against the 1,048,576-descriptor gallery with planted
    near-duplicates: every planted match by closed form (idx1 = planted slot,
    dist1 = h, accepted), plus 48 rows checked in full against the oracle."""
    q, g, slots, hs = synth.gallery_workload()
    got = _match(gpu_ctx, q, g, path=path)
    assert np.array_equal(got["idx1"], slots)
    assert np.array_equal(got["dist1"].astype(np.int32), hs)
    assert got["accepted"].all()
    rows = np.random.default_rng(1).choice(q.shape[0], 48, replace=False)
    want = oracle.match(q[rows], g)
    _same(got[rows], want)

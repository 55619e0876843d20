"""Parity of the CUDA matching paths with the CPU oracle through the C ABI: exact
indices, distances and ratio-test verdicts, on tie-heavy inputs, ragged sizes,
degenerate cases and sampled rows of the million-descriptor gallery."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth
import oracle_shards
from conftest import match_records, same_matches, to_dev

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
    2,000 x 2,000 on every path; descriptors equal the oracle's, and the matches equal
    the oracle's matching of its own descriptors."""
    wl = synth.pair("plain_640x480_2k")
    descs = []
    for img, kps in zip(wl["images"], wl["kps"]):
        d = gpu_ctx.extract(to_dev(img), wl["width"], wl["height"], to_dev(P.pack_keypoints(kps)))
        descs.append(d)
    torch.cuda.synchronize()
    wq, wt = (oracle.extract(im, wl["width"], wl["height"], k, triplets) for im, k in zip(wl["images"], wl["kps"]))
    assert np.array_equal(descs[0].cpu().numpy(), wq) and np.array_equal(descs[1].cpu().numpy(), wt)
    want = oracle.match(wq, wt)
    for path in PATHS:
        _same(match_records(gpu_ctx.match(descs[0], descs[1], 2, 0.8, path)), want)


@pytest.mark.parametrize("path", PATHS)
def test_oriented_pair_full_match(gpu_ctx, oriented_pair_oracle, path):
    """The oriented and scaled pair: 10,000 x 10,000 top-2 on each path, every query
    row equal to the oracle's matching of its own descriptors (sharded over the host
    cores)."""
    wl, descs, want = oriented_pair_oracle["wl"], oriented_pair_oracle["descs"], oriented_pair_oracle["match"]
    got = [gpu_ctx.extract(to_dev(im), wl["width"], wl["height"], to_dev(P.pack_keypoints(k)))
           for im, k in zip(wl["images"], wl["kps"])]
    torch.cuda.synchronize()
    for g, d in zip(got, descs):
        assert np.array_equal(g.cpu().numpy(), d)
    same_matches(match_records(gpu_ctx.match(got[0], got[1], 2, 0.8, path)), want)


@pytest.fixture(scope="module")
def gallery():
    """The 16,384 x 1,048,576 gallery workload and the oracle's full records for 1%
    of its query rows (a seeded sample of 168 rows), computed once for all paths."""
    q, g, slots, hs = synth.gallery_workload()
    rows = np.sort(np.random.default_rng(1).choice(q.shape[0], 168, replace=False))
    return q, g, slots, hs, rows, oracle_shards.match(q[rows], g, 2, 0.8, per=1)


@pytest.mark.parametrize("path", PATHS)
def test_million_gallery(gpu_ctx, gallery, path):
    """16,384 queries against the 1,048,576-descriptor gallery with planted
    near-duplicates: every planted match by closed form (idx1 = planted slot,
    dist1 = h, accepted), and 168 rows (1%) compared in full (idx1, idx2, dist1,
    dist2, accepted) with the oracle."""
    q, g, slots, hs, rows, want = gallery
    got = _match(gpu_ctx, q, g, path=path)
    assert np.array_equal(got["idx1"], slots)
    assert np.array_equal(got["dist1"].astype(np.int32), hs)
    assert got["accepted"].all()
    same_matches(got, want, rows)

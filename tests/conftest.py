import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def triplets():
    from paper_1609_03986_gb300 import synth
    return synth.triplets()


@pytest.fixture(scope="session")
def gpu_ctx(triplets):
    """A library context on cuda:0 with the seeded triplet table loaded."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1609_03986_gb300 import build
    build.build()
    import paper_1609_03986_gb300 as P
    ctx = P.Context(0, triplets=triplets)
    yield ctx
    ctx.close()


def to_dev(a):
    import torch
    return torch.from_numpy(a).cuda()


def match_records(t):
    import paper_1609_03986_gb300 as P
    return P.matches_from_bytes(t.cpu().numpy())


def same_matches(got, want, rows=None):
    """Field-by-field equality of match records with oracle results (optionally on rows)."""
    import numpy as np
    for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
        g = got[f] if rows is None else got[f][rows]
        assert np.array_equal(g.astype(np.int64), np.asarray(want[f]).astype(np.int64)), f


@pytest.fixture(scope="session")
def oriented_pair_oracle(triplets):
    """The oriented and scaled pair workload (2 x 1920x1080, 10,000 keypoints each)
    with the oracle's descriptors of both images and its full 10k x 10k top-2 match,
    computed once by the sharded oracle."""
    import oracle_shards
    from paper_1609_03986_gb300 import synth
    wl = synth.pair("oriented_scaled_1920x1080_10k")
    w, h = wl["width"], wl["height"]
    descs = oracle_shards.extract_many([(im, w, h, k, triplets, synth.SCALES) for im, k in zip(wl["images"], wl["kps"])])
    match = oracle_shards.match(descs[0], descs[1], 2, 0.8)
    return {"wl": wl, "descs": descs, "match": match}

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

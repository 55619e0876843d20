"""The allocation-free matching entry point.

hamming_match_noalloc is for callers that may not allocate device memory (for
example a host application whose own pool owns all HBM, or a pipeline in which a
cudaMalloc would stall its other streams).  Its scratch is the library's fixed
16 MiB device array.  Here it must give exactly the records of the allocating
entry point on the tensor-core path, on two calls in a row (the second with other
inputs, so nothing left in the shared array from the first call can leak into
it), and must refuse a request that does not fit.  This file is collected last.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_03986_gb300 as P
from paper_1609_03986_gb300 import synth

pytestmark = pytest.mark.gpu


def _records(t):
    return P.matches_from_bytes(t.cpu().numpy())


def test_noalloc_equals_allocating_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1609_03986_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    ctx = P.latch_context_create(0)
    try:
        stream = int(torch.cuda.current_stream().cuda_stream)
        for call, (nq, nt) in enumerate(((3001, 5003), (700, 9999))):
            qh = synth.random_descriptors(synth.seed(21, call, synth.KIND_GALLERY), nq)
            th = synth.random_descriptors(synth.seed(22, call, synth.KIND_GALLERY), nt)
            th[::7] = qh[0]  # ties: equal distances must resolve to the same lowest index
            q, t = torch.from_numpy(qh).cuda(), torch.from_numpy(th).cuda()
            want = torch.empty((nq, 16), dtype=torch.uint8, device="cuda")
            got = torch.full((nq, 16), 0xAB, dtype=torch.uint8, device="cuda")
            P.hamming_match(ctx, q, nq, t, nt, 2, 0.8, want, P.PATH_TENSOR, stream)
            P.hamming_match_noalloc(q, nq, t, nt, 2, 0.8, got, stream)
            torch.cuda.synchronize()
            P.hamming_match_noalloc_status()  # no device-side wait gave up
            a, b = _records(want), _records(got)
            for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
                assert np.array_equal(a[f], b[f]), (call, f)
            # and a few rows straight against the oracle (row 0 is the planted tie)
            rows = np.array([0, 1, nq // 2, nq - 1])
            o = oracle.match(qh[rows], th, 2, 0.8)
            for f in ("idx1", "idx2", "dist1", "dist2", "accepted"):
                assert np.array_equal(b[f][rows].astype(np.int64), o[f].astype(np.int64)), (call, f)
        P.latch_check(ctx)
    finally:
        P.latch_context_destroy(ctx)


def test_noalloc_rejects_requests_beyond_its_array():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    q = torch.zeros((40000, 64), dtype=torch.uint8, device="cuda")
    out = torch.zeros((40000, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(P.LatchError) as e:
        P.hamming_match_noalloc(q, 40000, q, 40000, 2, 0.8, out, 0)
    assert e.value.status == 1
    assert "static scratch" in P.latch_last_error(None)

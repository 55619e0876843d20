"""The CPU oracle run on shards of a workload in parallel host threads.

Each shard is one call of the unchanged single-threaded oracle (``oracle.extract`` on
a slice of the keypoints, ``oracle.match`` on a slice of the query rows against the
whole train set); the shards' results are concatenated in order.  The oracle's C
functions are called through ctypes, which releases the GIL for the duration of the
call, so the threads run on all host cores.  Threads, not processes: nothing is
forked after the CUDA context exists.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

WORKERS = max(1, os.cpu_count() or 1)
_pool = ThreadPoolExecutor(WORKERS)


def _shards(n: int, per: int):
    return [(i, min(n, i + per)) for i in range(0, n, per)]


def extract(image, width, height, kps, triplets, scales, per: int = 256) -> np.ndarray:
    """oracle.extract over all keypoints, `per` keypoints per shard."""
    kps = np.asarray(kps)
    if len(kps) == 0:
        return np.zeros((0, 64), np.uint8)
    parts = list(_pool.map(lambda s: oracle.extract(image, width, height, kps[s[0]:s[1]], triplets, scales),
                           _shards(len(kps), per)))
    return np.concatenate(parts)


def extract_many(jobs, per: int = 256):
    """[(image, width, height, kps, triplets, scales), ...] -> list of descriptor arrays;
    the shards of all jobs share the pool."""
    futs = []
    for image, w, h, kps, trip, sc in jobs:
        kps = np.asarray(kps)
        futs.append([_pool.submit(oracle.extract, image, w, h, kps[a:b], trip, sc) for a, b in _shards(len(kps), per)])
    return [np.concatenate([f.result() for f in fs]) if fs else np.zeros((0, 64), np.uint8) for fs in futs]


def match(query, train, k: int = 2, ratio: float = 0.8, per: int | None = None) -> dict:
    """oracle.match of every query row against the whole train set, query rows split
    into shards."""
    query = np.ascontiguousarray(query, dtype=np.uint8).reshape(-1, 64)
    train = np.ascontiguousarray(train, dtype=np.uint8).reshape(-1, 64)
    if per is None:
        per = max(1, -(-len(query) // (4 * WORKERS)))
    parts = list(_pool.map(lambda s: oracle.match(query[s[0]:s[1]], train, k, ratio), _shards(len(query), per)))
    if not parts:
        return oracle.match(query, train, k, ratio)
    return {f: np.concatenate([p[f] for p in parts]) for f in parts[0]}


def match_many(jobs, per: int = 8):
    """[(query, train, k, ratio), ...] -> list of oracle.match results; all jobs'
    shards share the pool."""
    futs = []
    for q, t, k, r in jobs:
        q = np.ascontiguousarray(q, dtype=np.uint8).reshape(-1, 64)
        futs.append((q, t, k, r, [_pool.submit(oracle.match, q[a:b], t, k, r) for a, b in _shards(len(q), per)]))
    out = []
    for q, t, k, r, fs in futs:
        parts = [f.result() for f in fs]
        out.append({f: np.concatenate([p[f] for p in parts]) for f in parts[0]} if parts else oracle.match(q, t, k, r))
    return out

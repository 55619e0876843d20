"""Python access to the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check and
by the benchmark's CPU-baseline leg, never by the library's product path.  The
oracle shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (plain C, -O2, FP contraction off so the FP64 offset
    formula is evaluated exactly as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I, I64, D, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
        lib.oracle_offsets.restype = None
        lib.oracle_offsets.argtypes = [D, I, P, P]
        lib.oracle_extract.restype = I
        lib.oracle_extract.argtypes = [P, I, I, I64, P, P, P, P, I, P, P, I, P]
        lib.oracle_distances.restype = I
        lib.oracle_distances.argtypes = [P, I, I, I64, I, I, I, I, P, P, I, P, P]
        lib.oracle_hamming.restype = I
        lib.oracle_hamming.argtypes = [P, P, I]
        lib.oracle_match.restype = I
        lib.oracle_match.argtypes = [P, I, P, I, I, F, P, P, P, P, P]
        lib.oracle_extract_weighted.restype = I
        lib.oracle_extract_weighted.argtypes = [P, I, I, I64, P, P, P, P, I, P, P, I, P, P]
        lib.oracle_fast_score.restype = I
        lib.oracle_fast_score.argtypes = [P, I, I, I64, I, I, I]
        lib.oracle_orientation_bin.restype = I
        lib.oracle_orientation_bin.argtypes = [P, I64, I, I]
        lib.oracle_detect.restype = I
        lib.oracle_detect.argtypes = [P, I, I, I64, I, I, P, P, P]
        lib.oracle_pyramid_level.restype = None
        lib.oracle_pyramid_level.argtypes = [P, I, I, I64, D, P, I64, P, P]
        lib.oracle_dense_extract.restype = I
        lib.oracle_dense_extract.argtypes = [P, I, I, I64, P, P]
        lib.oracle_dense_match.restype = I
        lib.oracle_dense_match.argtypes = [P, P, I, I, I, I, F, P, P, P, P, P]
        lib.oracle_detect_pyramid.restype = I
        lib.oracle_detect_pyramid.argtypes = [P, I, I, I64, I, P, I, I, P, P, P, P]
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def offsets(scale: float, angle_bin: int):
    """(dx, dy) int32 arrays of shape (48, 48), indexed [v, u]."""
    dx = np.zeros((48, 48), dtype=np.int32)
    dy = np.zeros((48, 48), dtype=np.int32)
    _load().oracle_offsets(float(scale), int(angle_bin), dx.ctypes.data, dy.ctypes.data)
    return dx, dy


def extract(image: np.ndarray, width: int, height: int, kps: np.ndarray, triplets: np.ndarray,
            scales=(1.0,), weights=None) -> np.ndarray:
    """Descriptors (n, 64) uint8.  image: (H, pitch) uint8; kps: (n, 4) int32
    (x, y, angle_bin, scale_idx); triplets (512, 6) uint8; weights: None for the
    7x7 patches, or 64 uint8 weights of the 8x8 patches (row-major)."""
    image = _c(image, np.uint8)
    kps = _c(kps, np.int32).reshape(-1, 4)
    n = kps.shape[0]
    kx, ky, kb, ks = (_c(kps[:, i], np.int32) for i in range(4))
    trip = _c(triplets, np.uint8).reshape(-1)
    assert trip.size == 512 * 6
    sc = _c(scales, np.float64)
    out = np.zeros((n, 64), dtype=np.uint8)
    if weights is not None:
        wt = _c(weights, np.uint8).reshape(-1)
        assert wt.size == 64
        rc = _load().oracle_extract_weighted(image.ctypes.data, width, height, image.shape[1], kx.ctypes.data,
                                             ky.ctypes.data, kb.ctypes.data, ks.ctypes.data, n, trip.ctypes.data,
                                             sc.ctypes.data, sc.size, wt.ctypes.data, out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_extract_weighted: invalid scale index or triplet")
        return out
    rc = _load().oracle_extract(image.ctypes.data, width, height, image.shape[1], kx.ctypes.data, ky.ctypes.data,
                                kb.ctypes.data, ks.ctypes.data, n, trip.ctypes.data, sc.ctypes.data, sc.size,
                                out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_extract: invalid scale index or triplet")
    return out


def distances(image: np.ndarray, width: int, height: int, kp, triplets: np.ndarray, scales=(1.0,)):
    """The two squared patch distances of Eq. 1 for every triplet of one keypoint
    kp = (x, y, angle_bin, scale_idx).  Returns (d1, d2) int64 arrays of length 512."""
    image = _c(image, np.uint8)
    trip = _c(triplets, np.uint8).reshape(-1)
    sc = _c(scales, np.float64)
    d1 = np.zeros(512, np.int64)
    d2 = np.zeros(512, np.int64)
    rc = _load().oracle_distances(image.ctypes.data, width, height, image.shape[1], int(kp[0]), int(kp[1]),
                                  int(kp[2]), int(kp[3]), trip.ctypes.data, sc.ctypes.data, sc.size,
                                  d1.ctypes.data, d2.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_distances: invalid scale index")
    return d1, d2


def hamming(a: np.ndarray, b: np.ndarray) -> int:
    a = _c(a, np.uint8)
    b = _c(b, np.uint8)
    return int(_load().oracle_hamming(a.ctypes.data, b.ctypes.data, a.size))


def match(query: np.ndarray, train: np.ndarray, k: int = 2, ratio: float = 0.8):
    """Brute-force top-k matching.  Returns dict of arrays idx1, idx2, dist1, dist2, accepted."""
    q = _c(query, np.uint8).reshape(-1, 64)
    t = _c(train, np.uint8).reshape(-1, 64)
    nq, nt = q.shape[0], t.shape[0]
    idx1 = np.zeros(nq, np.int32)
    idx2 = np.zeros(nq, np.int32)
    d1 = np.zeros(nq, np.int32)
    d2 = np.zeros(nq, np.int32)
    acc = np.zeros(nq, np.uint8)
    rc = _load().oracle_match(q.ctypes.data, nq, t.ctypes.data, nt, k, ratio, idx1.ctypes.data, idx2.ctypes.data,
                              d1.ctypes.data, d2.ctypes.data, acc.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_match: bad arguments")
    return {"idx1": idx1, "idx2": idx2, "dist1": d1, "dist2": d2, "accepted": acc}


def fast_score(image: np.ndarray, width: int, height: int, x: int, y: int, t: int) -> int:
    """FAST-9 score of pixel (x, y) at threshold t (0: not a corner)."""
    image = _c(image, np.uint8)
    return int(_load().oracle_fast_score(image.ctypes.data, width, height, image.shape[1], x, y, t))


def orientation_bin(image: np.ndarray, x: int, y: int) -> int:
    """Angle bin of the intensity centroid of the radius-15 disc around (x, y)."""
    image = _c(image, np.uint8)
    return int(_load().oracle_orientation_bin(image.ctypes.data, image.shape[1], x, y))


def detect(image: np.ndarray, width: int, height: int, t: int) -> np.ndarray:
    """Oriented FAST keypoints in raster order: (n, 3) int32 array of x, y, angle bin."""
    image = _c(image, np.uint8)
    lib = _load()
    cap = 4096
    while True:
        xs, ys, bs = (np.zeros(cap, np.int32) for _ in range(3))
        n = lib.oracle_detect(image.ctypes.data, width, height, image.shape[1], t, cap, xs.ctypes.data,
                              ys.ctypes.data, bs.ctypes.data)
        if n < 0:
            raise ValueError("oracle_detect: bad arguments")
        if n <= cap:
            return np.stack([xs[:n], ys[:n], bs[:n]], axis=1)
        cap = n


def pyramid_level(image: np.ndarray, width: int, height: int, scale: float) -> np.ndarray:
    """Level image of scale >= 1, (floor(H / s), floor(W / s)) uint8."""
    image = _c(image, np.uint8)
    w, h = int(np.floor(width / scale)), int(np.floor(height / scale))
    out = np.zeros((max(h, 1), max(w, 1)), np.uint8)
    lw, lh = ctypes.c_int(), ctypes.c_int()
    _load().oracle_pyramid_level(image.ctypes.data, width, height, image.shape[1], float(scale), out.ctypes.data,
                                 out.shape[1], ctypes.byref(lw), ctypes.byref(lh))
    return out[:lh.value, :lw.value]


def detect_pyramid(image: np.ndarray, width: int, height: int, t: int, scales) -> np.ndarray:
    """Oriented FAST keypoints of every pyramid level, level after level (raster order
    of the level's image), in base coordinates: (n, 4) int32 x, y, angle bin, level."""
    image = _c(image, np.uint8)
    sc = _c(scales, np.float64)
    lib = _load()
    cap = 4096
    while True:
        arrs = [np.zeros(cap, np.int32) for _ in range(4)]
        n = lib.oracle_detect_pyramid(image.ctypes.data, width, height, image.shape[1], t, sc.ctypes.data, sc.size,
                                      cap, *[a.ctypes.data for a in arrs])
        if n < 0:
            raise ValueError("oracle_detect_pyramid: bad arguments")
        if n <= cap:
            return np.stack([a[:n] for a in arrs], axis=1)
        cap = n


def dense_extract(image: np.ndarray, width: int, height: int, triplets: np.ndarray) -> np.ndarray:
    """Descriptor of every pixel (angle bin 0, scale 1), raster order: (H * W, 64) uint8."""
    image = _c(image, np.uint8)
    trip = _c(triplets, np.uint8).reshape(-1)
    assert trip.size == 512 * 6
    out = np.zeros((height * width, 64), dtype=np.uint8)
    rc = _load().oracle_dense_extract(image.ctypes.data, width, height, image.shape[1], trip.ctypes.data,
                                      out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_dense_extract: invalid triplet")
    return out


def dense_match(desc_a: np.ndarray, desc_b: np.ndarray, width: int, height: int, radius: int, k: int = 2,
                ratio: float = 0.8):
    """Windowed matching of two dense descriptor fields (raster order, width x height
    pixels each).  Returns dict of arrays idx1, idx2 (raster indices in B), dist1,
    dist2, accepted, one entry per pixel of A."""
    a = _c(desc_a, np.uint8).reshape(-1, 64)
    b = _c(desc_b, np.uint8).reshape(-1, 64)
    n = width * height
    assert a.shape[0] == n and b.shape[0] == n
    idx1, idx2, d1, d2 = (np.zeros(n, np.int32) for _ in range(4))
    acc = np.zeros(n, np.uint8)
    rc = _load().oracle_dense_match(a.ctypes.data, b.ctypes.data, width, height, radius, k, ratio, idx1.ctypes.data,
                                    idx2.ctypes.data, d1.ctypes.data, d2.ctypes.data, acc.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_dense_match: bad arguments")
    return {"idx1": idx1, "idx2": idx2, "dist1": d1, "dist2": d2, "accepted": acc}

"""Seeded synthetic inputs shaped like the paper's structure-from-motion workloads.

Images, keypoints, triplet tables, random descriptor galleries with planted
near-duplicates and Poisson request streams.  The generators are written in C
(``synth.c``) and hold none of the descriptor or matching arithmetic; both the CPU
oracle's tests and the CUDA library's tests and benchmarks take their inputs from
here so that the two sides see the same bytes.

Seeds: ``base ^ (config << 32) ^ (index << 8) ^ kind`` with base 0x160903986 and
kind 1 = image, 2 = keypoints, 3 = triplets (one table for every workload),
4 = gallery / random descriptors, 5 = arrivals, 6 = planting.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

KIND_IMAGE, KIND_KEYPOINTS, KIND_TRIPLETS, KIND_GALLERY, KIND_ARRIVALS, KIND_PLANT = 1, 2, 3, 4, 5, 6
DESC_BYTES = 64
N_TRIPLETS = 512
WINDOW = 48
PATCH = 7
SCALES = (1.0, 1.5, 2.25)

_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (plain C, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.synth_seed.restype = U64
        lib.synth_seed.argtypes = [I, I, I]
        lib.synth_image.restype = I
        lib.synth_image.argtypes = [U64, I, I, I64, P, I]
        lib.synth_keypoints.restype = None
        lib.synth_keypoints.argtypes = [U64, I, I, I, I, I, I, P]
        lib.synth_triplets.restype = None
        lib.synth_triplets.argtypes = [U64, I, I, I, P]
        lib.synth_bytes.restype = None
        lib.synth_bytes.argtypes = [U64, I64, P]
        lib.synth_plant.restype = I
        lib.synth_plant.argtypes = [U64, P, I, P, I64, I, I, I, P, P]
        lib.synth_arrivals.restype = I
        lib.synth_arrivals.argtypes = [U64, D, D, I, I, I, I, I, P, P, P, P]
        _lib = lib
    return _lib


def seed(config: int, index: int, kind: int) -> int:
    return int(_load().synth_seed(config, index, kind))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def image(seed_value: int, width: int, height: int, pitch: int | None = None, n_ellipses: int = 200) -> np.ndarray:
    """uint8 array of shape (height, pitch); columns >= width are zero padding."""
    if pitch is None:
        pitch = (width + 15) // 16 * 16
    out = np.zeros((height, pitch), dtype=np.uint8)
    if _load().synth_image(seed_value, width, height, pitch, _ptr(out), n_ellipses) != 0:
        raise MemoryError("synth_image failed")
    return out


def keypoints(seed_value: int, width: int, height: int, n: int, border: int = 32, oriented: bool = False,
              nscales: int = 1) -> np.ndarray:
    """int32 array (n, 4): x, y, angle_bin, scale_idx."""
    if width - 1 - 2 * border < 0 or height - 1 - 2 * border < 0 or nscales < 1:
        raise ValueError("keypoint border leaves no room in the image")
    out = np.zeros((n, 4), dtype=np.int32)
    _load().synth_keypoints(seed_value, width, height, n, border, int(oriented), nscales, _ptr(out))
    return out


def triplets(seed_value: int | None = None, count: int = N_TRIPLETS, lo: int = 3, hi: int = 44) -> np.ndarray:
    """uint8 array (count, 6): ax, ay, c1x, c1y, c2x, c2y in window coordinates."""
    if seed_value is None:
        seed_value = seed(0, 0, KIND_TRIPLETS)
    out = np.zeros((count, 6), dtype=np.uint8)
    _load().synth_triplets(seed_value, count, lo, hi, _ptr(out))
    return out


def random_descriptors(seed_value: int, n: int, nbytes: int = DESC_BYTES) -> np.ndarray:
    out = np.empty((n, nbytes), dtype=np.uint8)
    _load().synth_bytes(seed_value, n * nbytes, _ptr(out))
    return out


def plant(seed_value: int, queries: np.ndarray, gallery: np.ndarray, hmin: int = 20, hmax: int = 60):
    """Overwrite one distinct gallery slot per query with a copy at Hamming distance
    h in [hmin, hmax].  Returns (slots, h) int32 arrays; `gallery` is modified."""
    assert queries.dtype == np.uint8 and gallery.dtype == np.uint8
    assert queries.flags.c_contiguous and gallery.flags.c_contiguous
    nq, nb = queries.shape
    slots = np.zeros(nq, dtype=np.int32)
    hs = np.zeros(nq, dtype=np.int32)
    rc = _load().synth_plant(seed_value, _ptr(queries), nq, _ptr(gallery), gallery.shape[0], nb, hmin, hmax,
                             _ptr(slots), _ptr(hs))
    if rc != 0:
        raise ValueError("synth_plant failed")
    return slots, hs


def arrivals(seed_value: int, rate: float, duration: float, n_sizes: int, kmin: int, kmax: int,
             n_galleries: int):
    cap = int(rate * duration * 2 + 64)
    t = np.zeros(cap, dtype=np.float64)
    size = np.zeros(cap, dtype=np.int32)
    kps = np.zeros(cap, dtype=np.int32)
    gal = np.zeros(cap, dtype=np.int32)
    n = _load().synth_arrivals(seed_value, rate, duration, n_sizes, kmin, kmax, n_galleries, cap, _ptr(t),
                               _ptr(size), _ptr(kps), _ptr(gal))
    return t[:n], size[:n], kps[:n], gal[:n]


# ---------------------------------------------------------------------------
# Workload recipes (the five synthetic workloads; sizes follow the paper's SfM
# photo sets scaled to what one GPU holds).
# ---------------------------------------------------------------------------

PAIR_WORKLOADS = {
    # name: (config id, width, height, keypoints per image, oriented, number of scales)
    "plain_640x480_2k": (1, 640, 480, 2000, False, 1),
    "oriented_scaled_1920x1080_10k": (2, 1920, 1080, 10000, True, 3),
}


def pair(name: str, n_keypoints: int | None = None):
    """Two images and their keypoints for a one-pair workload.

    Returns dict with images (list of (H, pitch) uint8), kps (list of (n, 4) int32),
    width, height, triplets ((512, 6) uint8) and scales.
    """
    cfg, w, h, nk, oriented, nsc = PAIR_WORKLOADS[name]
    if n_keypoints is not None:
        nk = n_keypoints
    imgs = [image(seed(cfg, i, KIND_IMAGE), w, h) for i in range(2)]
    kps = [keypoints(seed(cfg, i, KIND_KEYPOINTS), w, h, nk, 32, oriented, nsc) for i in range(2)]
    return {"images": imgs, "kps": kps, "width": w, "height": h, "triplets": triplets(),
            "scales": SCALES if nsc > 1 else SCALES[:1], "config": cfg}


def gallery_workload(n_gallery: int = 1 << 20, n_query: int = 16384, hmin: int = 20, hmax: int = 60, config: int = 4):
    """Random 512-bit gallery with one planted near-duplicate per query."""
    gal = random_descriptors(seed(config, 0, KIND_GALLERY), n_gallery)
    q = random_descriptors(seed(config, 1, KIND_GALLERY), n_query)
    slots, hs = plant(seed(config, 0, KIND_PLANT), q, gal, hmin, hmax)
    return q, gal, slots, hs


BATCH_IMAGES, BATCH_W, BATCH_H, BATCH_NEIGHBOURS = 64, 4000, 3000, 8


def batch_pairs(n_images: int = BATCH_IMAGES, neighbours: int = BATCH_NEIGHBOURS):
    """Sequential-neighbour pair list: (i, j) for j = i+1 .. min(i+neighbours, n-1)."""
    return [(i, j) for i in range(n_images) for j in range(i + 1, min(i + neighbours, n_images - 1) + 1)]


def batch_keypoint_counts(n_images: int = BATCH_IMAGES, lo: int = 5000, hi: int = 50000, config: int = 3):
    """Per-image keypoint counts, uniform integers in [lo, hi] (drawn as the x
    coordinate of a 1-pixel-high keypoint field of width hi - lo + 1)."""
    tmp = np.zeros((n_images, 4), dtype=np.int32)
    _load().synth_keypoints(seed(config, 0, KIND_KEYPOINTS) ^ 0x77, hi - lo + 1, 1, n_images, 0, 0, 1, _ptr(tmp))
    return (tmp[:, 0] + lo).astype(np.int32)


def sfm_batch(n_images: int = BATCH_IMAGES, width: int = BATCH_W, height: int = BATCH_H,
              neighbours: int = BATCH_NEIGHBOURS, kmin: int = 5000, kmax: int = 50000, config: int = 3):
    """The batched structure-from-motion workload: n_images grey images with
    oriented, scaled keypoints (counts uniform in [kmin, kmax]) and the pair list of
    every image against its next `neighbours` images."""
    counts = batch_keypoint_counts(n_images, kmin, kmax, config)
    # the C generator releases the GIL (ctypes) and keeps no shared state: images in parallel
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        imgs = list(ex.map(lambda i: image(seed(config, i, KIND_IMAGE), width, height), range(n_images)))
    kps = [keypoints(seed(config, i, KIND_KEYPOINTS), width, height, int(counts[i]), 32, True, 3)
           for i in range(n_images)]
    return {"images": imgs, "kps": kps, "pairs": batch_pairs(n_images, neighbours), "width": width,
            "height": height, "triplets": triplets(), "scales": SCALES}

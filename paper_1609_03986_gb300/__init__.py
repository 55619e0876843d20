"""GB300-native LATCH descriptors and Hamming matching (CLATCH, arXiv 1609.03986).

Thin ctypes binding over the C ABI declared in ``include/latch.h``.  The functions
below carry the C names and only marshal arguments; every step of extraction and
matching runs in the CUDA kernels of ``liblatch.so``.  There is no CPU fallback:
if the library is missing or fails to load, importing the binding raises.

Pointers are passed as integers (e.g. ``tensor.data_ptr()``) or as objects with a
``data_ptr()`` method; streams as ``cudaStream_t`` integers
(``torch.cuda.current_stream().cuda_stream``) or 0 for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblatch.so")

DESC_BYTES = 64
N_TRIPLETS = 512
PATH_AUTO, PATH_POPC, PATH_TENSOR = 0, 1, 2
AVAILABLE_PATHS = (PATH_POPC, PATH_TENSOR)
STATUS = {0: "LATCH_OK", 1: "LATCH_EINVAL", 2: "LATCH_ENOMEM", 3: "LATCH_ECUDA", 4: "LATCH_EUNSUPPORTED",
          5: "LATCH_EBUSY", 6: "LATCH_ETIMEOUT", 7: "LATCH_ECANCELLED", 8: "LATCH_EDEVICE"}

# numpy views of the C records
MATCH_DTYPE = np.dtype([("idx1", "<i4"), ("idx2", "<i4"), ("dist1", "<u2"), ("dist2", "<u2"),
                        ("accepted", "u1"), ("pad", "u1", (3,))])
KEYPOINT_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("angle_bin", "u1"), ("scale_idx", "u1"),
                           ("reserved", "<u2")])
assert MATCH_DTYPE.itemsize == 16 and KEYPOINT_DTYPE.itemsize == 12


class LatchError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class latch_image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch", ctypes.c_int64)]


class latch_batch_desc(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("h_images", ctypes.c_void_p), ("h_n_kps", ctypes.c_void_p),
                ("d_kps", ctypes.c_void_p), ("d_desc", ctypes.c_void_p), ("n_pairs", ctypes.c_int32),
                ("h_pairs", ctypes.c_void_p), ("k", ctypes.c_int32), ("ratio", ctypes.c_float),
                ("d_matches", ctypes.c_void_p)]


class latch_host_batch_desc(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("h_images", ctypes.c_void_p), ("h_n_kps", ctypes.c_void_p),
                ("h_kps", ctypes.c_void_p), ("h_desc", ctypes.c_void_p), ("n_pairs", ctypes.c_int32),
                ("h_pairs", ctypes.c_void_p), ("k", ctypes.c_int32), ("ratio", ctypes.c_float),
                ("h_matches", ctypes.c_void_p)]


class latch_tuning(ctypes.Structure):
    _fields_ = [("item_kps", ctypes.c_int32), ("tensor_min_pairs", ctypes.c_int64)]


class latch_tune_shape(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n_keypoints", ctypes.c_int32),
                ("n_query", ctypes.c_int32), ("n_train", ctypes.c_int32)]


class latch_request(ctypes.Structure):
    _fields_ = [("h_image", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch", ctypes.c_int64), ("h_kps", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("gallery_id", ctypes.c_int32), ("k", ctypes.c_int32), ("ratio", ctypes.c_float),
                ("h_matches", ctypes.c_void_p), ("h_desc", ctypes.c_void_p)]


class latch_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class latch_session_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "rejected", "failed", "batches", "max_queue",
                                             "queued", "lane_bytes", "hbm_free", "hbm_budget")]


_lib = None

# (name, restype, argtypes) of every exported entry point
_P, _I32, _I64, _F, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
EXPORTS = [
    ("latch_version", ctypes.c_char_p, []),
    ("latch_last_error", ctypes.c_char_p, [_P]),
    ("latch_context_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P)]),
    ("latch_context_destroy", ctypes.c_int, [_P]),
    ("latch_set_scales", ctypes.c_int, [_P, _P, _I32]),
    ("latch_set_triplets", ctypes.c_int, [_P, _P]),
    ("latch_reserve", ctypes.c_int, [_P, _I64, _I64, _I64]),
    ("latch_extract", ctypes.c_int, [_P, ctypes.POINTER(latch_image), _P, _I32, _P, _P, _P]),
    ("hamming_match", ctypes.c_int, [_P, _P, _I32, _P, _I32, _I32, _F, _P, _I32, _P]),
    ("latch_check", ctypes.c_int, [_P]),
    ("latch_selftest_wait_timeout", ctypes.c_int, [_P, _I32, _P]),
    ("latch_trace_enable", ctypes.c_int, [_P, _I32]),
    ("latch_trace_collect", ctypes.c_int, [_P, _P, _I32, ctypes.POINTER(_I32)]),
    ("latch_kernel_launches", ctypes.c_uint64, []),
    ("hamming_match_path", ctypes.c_int32, [_P, _I64, _I64]),
    ("latch_autotune", ctypes.c_int, [_P, ctypes.POINTER(latch_tune_shape), ctypes.POINTER(latch_tuning)]),
    ("latch_get_tuning", ctypes.c_int, [_P, ctypes.POINTER(latch_tuning)]),
    ("latch_set_tuning", ctypes.c_int, [_P, ctypes.POINTER(latch_tuning)]),
    ("latch_reserve_batch", ctypes.c_int, [_P, ctypes.POINTER(latch_batch_desc)]),
    ("latch_batch_run", ctypes.c_int, [_P, ctypes.POINTER(latch_batch_desc), _P]),
    ("latch_batch_run_host", ctypes.c_int, [_P, ctypes.POINTER(latch_host_batch_desc), _P]),
    ("latch_session_create", ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, _I64, _I32, _I64, _P,
                                            ctypes.POINTER(_P)]),
    ("latch_session_create_lanes", ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, _I64, _I32, _I64, _I32, _P,
                                                  ctypes.POINTER(_P)]),
    ("latch_session_destroy", ctypes.c_int, [_P]),
    ("latch_gallery_add", ctypes.c_int, [_P, _P, _I32, ctypes.POINTER(_I32)]),
    ("latch_submit", ctypes.c_int, [_P, ctypes.POINTER(latch_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("latch_wait", ctypes.c_int, [_P, ctypes.c_uint64, _I32, ctypes.POINTER(latch_result)]),
    ("latch_release", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("latch_session_get_stats", ctypes.c_int, [_P, ctypes.POINTER(latch_session_stats)]),
    ("latch_session_last_error", ctypes.c_char_p, [_P]),
    ("hamming_match_noalloc", ctypes.c_int, [_P, _I32, _P, _I32, _I32, _F, _P, _P]),
    ("hamming_match_noalloc_status", ctypes.c_int, []),
    ("latch_set_patch_weights", ctypes.c_int, [_P, _P]),
    ("latch_detect_pyramid", ctypes.c_int, [_P, ctypes.POINTER(latch_image), _I32, _I32, _I32, _P, _P, _P, _P]),
    ("latch_detect", ctypes.c_int, [_P, ctypes.POINTER(latch_image), _I32, _I32, _I32, _P, _P, _P]),
    ("latch_detect_extract", ctypes.c_int, [_P, ctypes.POINTER(latch_image), _I32, _I32, _I32, _P, _P, _P, _P]),
    ("latch_dense_extract", ctypes.c_int, [_P, ctypes.POINTER(latch_image), _P, _P]),
    ("latch_dense_match", ctypes.c_int, [_P, _P, _P, _I32, _I32, _I32, _I32, _F, _P, _P]),
]


def library():
    """Load ``liblatch.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1609_03986_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in EXPORTS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def _check(ctx, status: int):
    if status != 0:
        msg = library().latch_last_error(ctx)
        raise LatchError(status, msg.decode() if msg else "")


def latch_version() -> str:
    return library().latch_version().decode()


def latch_last_error(ctx) -> str:
    m = library().latch_last_error(ctx)
    return m.decode() if m else ""


def latch_context_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(None, library().latch_context_create(device, ctypes.byref(h)))
    return h


def latch_context_destroy(ctx) -> None:
    _check(None, library().latch_context_destroy(ctx))


def latch_set_scales(ctx, scales) -> None:
    s = np.ascontiguousarray(scales, dtype=np.float64)
    _check(ctx, library().latch_set_scales(ctx, s.ctypes.data, s.size))


def latch_set_triplets(ctx, triplets) -> None:
    t = np.ascontiguousarray(triplets, dtype=np.uint8).reshape(-1)
    if t.size != N_TRIPLETS * 6:
        raise ValueError("triplet table must hold 512 x 6 bytes")
    _check(ctx, library().latch_set_triplets(ctx, t.ctypes.data))


def latch_set_patch_weights(ctx, weights) -> None:
    """64 uint8 weights of the 8x8 patches (row-major), or None for the 7x7 patches."""
    if weights is None:
        _check(ctx, library().latch_set_patch_weights(ctx, None))
        return
    w = np.ascontiguousarray(weights, dtype=np.uint8).reshape(-1)
    if w.size != 64:
        raise ValueError("the weight table holds 8 x 8 bytes")
    _check(ctx, library().latch_set_patch_weights(ctx, w.ctypes.data))


def latch_reserve(ctx, max_keypoints: int, max_query: int, max_train: int) -> None:
    _check(ctx, library().latch_reserve(ctx, max_keypoints, max_query, max_train))


def latch_extract(ctx, image, width: int, height: int, pitch: int, kps, n: int, triplets, out,
                  stream: int = 0) -> None:
    """Descriptors of n keypoints (device pointers image, kps, out; triplets host
    (512, 6) uint8 or None for the context's table)."""
    img = latch_image(_ptr(image), width, height, pitch)
    tp = 0
    if triplets is not None:
        t = np.ascontiguousarray(triplets, dtype=np.uint8).reshape(-1)
        if t.size != N_TRIPLETS * 6:
            raise ValueError("triplet table must hold 512 x 6 bytes")
        tp = t.ctypes.data
    _check(ctx, library().latch_extract(ctx, ctypes.byref(img), _ptr(kps), n, tp, _ptr(out), stream))


def latch_detect(ctx, image, width: int, height: int, pitch: int, threshold: int, scale_idx: int, max_kps: int,
                 kps_out, count_out, stream: int = 0) -> None:
    """Oriented FAST keypoints (device pointers image, kps_out, count_out)."""
    img = latch_image(_ptr(image), width, height, pitch)
    _check(ctx, library().latch_detect(ctx, ctypes.byref(img), threshold, scale_idx, max_kps, _ptr(kps_out),
                                       _ptr(count_out), stream))


def latch_detect_extract(ctx, image, width: int, height: int, pitch: int, threshold: int, scale_idx: int,
                         max_kps: int, kps_out, count_out, desc_out, stream: int = 0) -> None:
    """Oriented FAST keypoints and their descriptors, no host round trip."""
    img = latch_image(_ptr(image), width, height, pitch)
    _check(ctx, library().latch_detect_extract(ctx, ctypes.byref(img), threshold, scale_idx, max_kps, _ptr(kps_out),
                                               _ptr(count_out), _ptr(desc_out), stream))


def latch_detect_pyramid(ctx, image, width: int, height: int, pitch: int, threshold: int, n_levels: int,
                         max_kps: int, kps_out, count_out, desc_out=None, stream: int = 0) -> None:
    """Oriented FAST keypoints of every pyramid level (the scale table's first n_levels
    entries), level after level, optionally with their descriptors."""
    img = latch_image(_ptr(image), width, height, pitch)
    _check(ctx, library().latch_detect_pyramid(ctx, ctypes.byref(img), threshold, n_levels, max_kps, _ptr(kps_out),
                                               _ptr(count_out), _ptr(desc_out), stream))


def hamming_match(ctx, query, nq: int, train, nt: int, k: int, ratio: float, out, path: int = PATH_AUTO,
                  stream: int = 0) -> None:
    _check(ctx, library().hamming_match(ctx, _ptr(query), nq, _ptr(train), nt, k, ratio, _ptr(out), path, stream))


def hamming_match_noalloc(query, nq: int, train, nt: int, k: int, ratio: float, out, stream: int = 0) -> None:
    """hamming_match on the current device without allocating device memory (for
    callers that may not call cudaMalloc); scratch is the library's fixed 16 MiB
    array, so nq + nt is limited to roughly 60,000 descriptors."""
    _check(None, library().hamming_match_noalloc(_ptr(query), nq, _ptr(train), nt, k, ratio, _ptr(out), stream))


def latch_dense_extract(ctx, image, width: int, height: int, pitch: int, out, stream: int = 0) -> None:
    """Descriptor of every pixel (device pointers image, out: width * height * 64 bytes)."""
    img = latch_image(_ptr(image), width, height, pitch)
    _check(ctx, library().latch_dense_extract(ctx, ctypes.byref(img), _ptr(out), stream))


def latch_dense_match(ctx, desc_a, desc_b, width: int, height: int, radius: int, k: int, ratio: float, out,
                      stream: int = 0) -> None:
    """Windowed matching of two dense descriptor fields (device pointers)."""
    _check(ctx, library().latch_dense_match(ctx, _ptr(desc_a), _ptr(desc_b), width, height, radius, k, ratio,
                                            _ptr(out), stream))


def hamming_match_noalloc_status() -> None:
    """Raise LatchError if a device-side wait of an earlier hamming_match_noalloc call
    on the current device gave up (reads and clears the status word; synchronises)."""
    _check(None, library().hamming_match_noalloc_status())


def latch_check(ctx) -> None:
    _check(ctx, library().latch_check(ctx))


class BatchDesc:
    """Host-side arrays of a latch_batch_desc, kept alive with the struct.

    images: list of (device pointer, width, height, pitch); n_kps: list of ints;
    pairs: list of (query image, train image)."""

    def __init__(self, images, n_kps, d_kps, d_desc, pairs, k, ratio, d_matches):
        self._imgs = (latch_image * max(1, len(images)))(*[latch_image(_ptr(p), w, h, pt) for p, w, h, pt in images])
        self._n = np.ascontiguousarray(n_kps, dtype=np.int32)
        self._pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.desc = latch_batch_desc(len(images), ctypes.addressof(self._imgs), self._n.ctypes.data, _ptr(d_kps),
                                     _ptr(d_desc), self._pairs.shape[0], self._pairs.ctypes.data, k, ratio,
                                     _ptr(d_matches))

    def match_offsets(self):
        """First match record of every pair."""
        q = self._n[self._pairs[:, 0]].astype(np.int64)
        return np.concatenate([[0], np.cumsum(q)])


def latch_reserve_batch(ctx, batch: BatchDesc) -> None:
    _check(ctx, library().latch_reserve_batch(ctx, ctypes.byref(batch.desc)))


def latch_batch_run(ctx, batch: BatchDesc, stream: int = 0) -> None:
    _check(ctx, library().latch_batch_run(ctx, ctypes.byref(batch.desc), stream))


class HostBatchDesc:
    """Host-side arrays of a latch_host_batch_desc, kept alive with the struct.

    images: list of (host pointer, width, height, pitch); n_kps: list of ints;
    pairs: list of (query image, train image); h_kps / h_desc / h_matches: host
    buffers (pinned for asynchronous copies), h_desc may be None."""

    def __init__(self, images, n_kps, h_kps, h_desc, pairs, k, ratio, h_matches):
        self._imgs = (latch_image * max(1, len(images)))(*[latch_image(_ptr(p), w, h, pt) for p, w, h, pt in images])
        self._n = np.ascontiguousarray(n_kps, dtype=np.int32)
        self._pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.desc = latch_host_batch_desc(len(images), ctypes.addressof(self._imgs), self._n.ctypes.data,
                                          _ptr(h_kps), _ptr(h_desc), self._pairs.shape[0], self._pairs.ctypes.data,
                                          k, ratio, _ptr(h_matches))

    def match_offsets(self):
        """First match record of every pair."""
        q = self._n[self._pairs[:, 0]].astype(np.int64)
        return np.concatenate([[0], np.cumsum(q)])


def latch_batch_run_host(ctx, batch: HostBatchDesc, stream: int = 0) -> None:
    _check(ctx, library().latch_batch_run_host(ctx, ctypes.byref(batch.desc), stream))


def _scheck(sess, status: int):
    if status != 0:
        msg = library().latch_session_last_error(sess)
        raise LatchError(status, msg.decode() if msg else "")


def latch_session_create(device: int, hbm_budget: int, max_gallery_rows: int, max_batch: int, max_batch_kps: int,
                         triplets, lanes: int = 2):
    t = np.ascontiguousarray(triplets, dtype=np.uint8).reshape(-1)
    h = ctypes.c_void_p()
    if lanes == 2:  # the default lane count
        st = library().latch_session_create(device, hbm_budget, max_gallery_rows, max_batch, max_batch_kps,
                                            t.ctypes.data, ctypes.byref(h))
    else:
        st = library().latch_session_create_lanes(device, hbm_budget, max_gallery_rows, max_batch, max_batch_kps,
                                                  lanes, t.ctypes.data, ctypes.byref(h))
    if st != 0:
        raise LatchError(st, "latch_session_create failed")
    return h


def latch_session_create_lanes(device: int, hbm_budget: int, max_gallery_rows: int, max_batch: int,
                               max_batch_kps: int, lanes: int, triplets):
    return latch_session_create(device, hbm_budget, max_gallery_rows, max_batch, max_batch_kps, triplets, lanes)


def latch_session_destroy(sess) -> None:
    library().latch_session_destroy(sess)


def latch_gallery_add(sess, h_desc, n: int) -> int:
    gid = ctypes.c_int32()
    _scheck(sess, library().latch_gallery_add(sess, _ptr(h_desc), n, ctypes.byref(gid)))
    return gid.value


def latch_submit(sess, req: latch_request) -> int:
    t = ctypes.c_uint64()
    _scheck(sess, library().latch_submit(sess, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def latch_wait(sess, ticket: int, timeout_ms: int = -1) -> latch_result:
    r = latch_result()
    _scheck(sess, library().latch_wait(sess, ticket, timeout_ms, ctypes.byref(r)))
    return r


def latch_release(sess, ticket: int) -> None:
    _scheck(sess, library().latch_release(sess, ticket))


def latch_session_get_stats(sess) -> dict:
    st = latch_session_stats()
    _scheck(sess, library().latch_session_get_stats(sess, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in latch_session_stats._fields_}


def latch_session_last_error(sess) -> str:
    m = library().latch_session_last_error(sess)
    return m.decode() if m else ""


def _host_buffer(shape):
    """Page-locked host array (so the session's device-to-host copies stay
    asynchronous); plain numpy memory when torch/CUDA is not available."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.empty(shape, dtype=torch.uint8, pin_memory=True).numpy()
    except Exception:
        pass
    return np.empty(shape, np.uint8)


def pinned_copy(a: np.ndarray) -> np.ndarray:
    """Page-locked copy of a host array (inputs that the session copies asynchronously)."""
    b = _host_buffer(a.shape) if a.dtype == np.uint8 else np.array(a)
    b[...] = a
    return b


class Session:
    """Owner of a latch_session; requests take numpy host arrays (pinned ones keep
    the session's host<->device copies fully asynchronous)."""

    def __init__(self, triplets, device: int = 0, hbm_budget: int = 8 << 30, max_gallery_rows: int = 1 << 22,
                 max_batch: int = 16, max_batch_kps: int = 1 << 18, lanes: int = 2):
        self.handle = latch_session_create(device, hbm_budget, max_gallery_rows, max_batch, max_batch_kps, triplets,
                                           lanes)
        self._live = {}

    def close(self):
        if self.handle is not None:
            latch_session_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_gallery(self, desc: np.ndarray) -> int:
        desc = np.ascontiguousarray(desc, dtype=np.uint8).reshape(-1, DESC_BYTES)
        return latch_gallery_add(self.handle, desc, desc.shape[0])

    def submit(self, image: np.ndarray, width: int, height: int, kps_packed: np.ndarray, gallery: int, k: int = 2,
               ratio: float = 0.8, want_desc: bool = False):
        """image: (H, pitch) uint8; kps_packed: (n, 12) uint8.  Returns a ticket;
        the output arrays stay referenced until wait()."""
        n = kps_packed.shape[0]
        matches = _host_buffer((max(n, 1), 16))
        desc = _host_buffer((max(n, 1), DESC_BYTES)) if want_desc else None
        req = latch_request(image.ctypes.data, width, height, image.strides[0], kps_packed.ctypes.data, n, gallery,
                            k, ratio, matches.ctypes.data, desc.ctypes.data if desc is not None else 0)
        t = latch_submit(self.handle, req)
        self._live[t] = (image, kps_packed, matches, desc, n)
        return t

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (latch_result, match records, descriptors or None) and forgets the ticket."""
        r = latch_wait(self.handle, ticket, timeout_ms)
        image, kps, matches, desc, n = self._live.pop(ticket)
        latch_release(self.handle, ticket)
        return r, matches_from_bytes(matches[:n]), (desc[:n] if desc is not None else None)

    def stats(self) -> dict:
        return latch_session_get_stats(self.handle)


def latch_autotune(ctx, width: int, height: int, n_keypoints: int, n_query: int, n_train: int) -> dict:
    """Tune on this device for the given shape; returns the chosen settings."""
    out = latch_tuning()
    _check(ctx, library().latch_autotune(ctx, ctypes.byref(latch_tune_shape(width, height, n_keypoints, n_query,
                                                                            n_train)), ctypes.byref(out)))
    return {"item_kps": out.item_kps, "tensor_min_pairs": out.tensor_min_pairs}


def latch_get_tuning(ctx) -> dict:
    out = latch_tuning()
    _check(ctx, library().latch_get_tuning(ctx, ctypes.byref(out)))
    return {"item_kps": out.item_kps, "tensor_min_pairs": out.tensor_min_pairs}


def latch_set_tuning(ctx, item_kps: int, tensor_min_pairs: int) -> None:
    _check(ctx, library().latch_set_tuning(ctx, ctypes.byref(latch_tuning(item_kps, tensor_min_pairs))))


def hamming_match_path(ctx, nq: int, nt: int) -> int:
    """The path LATCH_PATH_AUTO takes for nq x nt on this context."""
    return int(library().hamming_match_path(ctx, nq, nt))


def latch_selftest_wait_timeout(ctx, limit_us: int, stream: int = 0) -> None:
    _check(ctx, library().latch_selftest_wait_timeout(ctx, limit_us, stream))


def latch_trace_enable(ctx, max_records: int) -> None:
    _check(ctx, library().latch_trace_enable(ctx, max_records))


def latch_trace_collect(ctx, capacity: int) -> np.ndarray:
    """(n, 2) float32 array of [extraction ms, matching ms] per traced batch run."""
    out = np.zeros((max(capacity, 1), 2), np.float32)
    n = ctypes.c_int32()
    _check(ctx, library().latch_trace_collect(ctx, out.ctypes.data, capacity, ctypes.byref(n)))
    return out[:n.value]


def latch_kernel_launches() -> int:
    """Number of kernels this library has launched in this process."""
    return int(library().latch_kernel_launches())


def pack_keypoints(kps: np.ndarray) -> np.ndarray:
    """(n, 4) int (x, y, angle_bin, scale_idx) -> (n, 12) uint8 latch_keypoint records."""
    kps = np.asarray(kps).reshape(-1, 4)
    rec = np.zeros(kps.shape[0], dtype=KEYPOINT_DTYPE)
    rec["x"] = kps[:, 0]
    rec["y"] = kps[:, 1]
    rec["angle_bin"] = kps[:, 2]
    rec["scale_idx"] = kps[:, 3]
    return rec.view(np.uint8).reshape(-1, 12)


def unpack_keypoints(raw: np.ndarray) -> np.ndarray:
    """(n, 12) uint8 latch_keypoint records -> (n, 4) int32 (x, y, angle_bin, scale_idx)."""
    rec = np.ascontiguousarray(raw, dtype=np.uint8).reshape(-1).view(KEYPOINT_DTYPE)
    return np.stack([rec["x"], rec["y"], rec["angle_bin"], rec["scale_idx"]], axis=1).astype(np.int32)


def matches_from_bytes(raw: np.ndarray) -> np.ndarray:
    """(nq, 16) uint8 -> structured array of latch_match records."""
    return np.ascontiguousarray(raw, dtype=np.uint8).reshape(-1).view(MATCH_DTYPE)


class Context:
    """Convenience owner of a latch_context working on torch CUDA tensors.

    Outputs are allocated with torch; every computation is one C-ABI call."""

    def __init__(self, device: int = 0, scales=(1.0, 1.5, 2.25), triplets=None):
        self.device = device
        self.handle = latch_context_create(device)
        if tuple(scales) != (1.0, 1.5, 2.25):
            latch_set_scales(self.handle, scales)
        if triplets is not None:
            latch_set_triplets(self.handle, triplets)

    def close(self):
        if self.handle is not None:
            latch_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        if stream is not None:
            return int(stream)
        import torch
        return int(torch.cuda.current_stream().cuda_stream)

    def extract(self, image, width: int, height: int, kps, triplets=None, out=None, stream=None):
        """image: (H, pitch) uint8 CUDA tensor; kps: (n, 12) uint8 CUDA tensor of
        packed keypoints.  Returns (n, 64) uint8 CUDA tensor."""
        import torch
        n = kps.shape[0]
        if out is None:
            out = torch.empty((n, DESC_BYTES), dtype=torch.uint8, device=image.device)
        latch_extract(self.handle, image, width, height, image.stride(0), kps, n, triplets, out,
                      self._stream(stream))
        return out

    def detect(self, image, width: int, height: int, threshold: int = 20, max_kps: int = 1 << 16, scale_idx: int = 0,
               with_descriptors: bool = False, stream=None):
        """image: (H, pitch) uint8 CUDA tensor.  Returns (keypoints (max_kps, 12) uint8
        tensor, count (1,) int32 tensor[, descriptors (max_kps, 64) uint8 tensor]); the
        first min(count, max_kps) rows are valid once the stream is synchronised."""
        import torch
        kps = torch.empty((max(max_kps, 1), 12), dtype=torch.uint8, device=image.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=image.device)
        if with_descriptors:
            desc = torch.empty((max(max_kps, 1), DESC_BYTES), dtype=torch.uint8, device=image.device)
            latch_detect_extract(self.handle, image, width, height, image.stride(0), threshold, scale_idx, max_kps,
                                 kps, cnt, desc, self._stream(stream))
            return kps, cnt, desc
        latch_detect(self.handle, image, width, height, image.stride(0), threshold, scale_idx, max_kps, kps, cnt,
                     self._stream(stream))
        return kps, cnt

    def match(self, query, train, k: int = 2, ratio: float = 0.8, path: int = PATH_AUTO, out=None, stream=None):
        """query (nq, 64), train (nt, 64) uint8 CUDA tensors -> (nq, 16) uint8 tensor of latch_match."""
        import torch
        nq, nt = query.shape[0], train.shape[0]
        if out is None:
            out = torch.empty((nq, 16), dtype=torch.uint8, device=query.device)
        hamming_match(self.handle, query, nq, train, nt, k, ratio, out, path, self._stream(stream))
        return out

    def dense_extract(self, image, width: int, height: int, out=None, stream=None):
        """image: (H, pitch) uint8 CUDA tensor.  Returns the (H * W, 64) uint8 CUDA tensor
        of every pixel's descriptor, raster order."""
        import torch
        if out is None:
            out = torch.empty((width * height, DESC_BYTES), dtype=torch.uint8, device=image.device)
        latch_dense_extract(self.handle, image, width, height, image.stride(0), out, self._stream(stream))
        return out

    def dense_match(self, desc_a, desc_b, width: int, height: int, radius: int, k: int = 2, ratio: float = 0.8,
                    out=None, stream=None):
        """Two (H * W, 64) dense fields -> (H * W, 16) uint8 tensor of latch_match."""
        import torch
        if out is None:
            out = torch.empty((width * height, 16), dtype=torch.uint8, device=desc_a.device)
        latch_dense_match(self.handle, desc_a, desc_b, width, height, radius, k, ratio, out, self._stream(stream))
        return out

    def check(self):
        latch_check(self.handle)

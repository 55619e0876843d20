"""Host-side checks of the C ABI: the library loads, exports every function that
include/latch.h declares, and the binding covers them.  No GPU work is done."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src,
                                re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_03986_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("latch_context_create", "latch_extract", "hamming_match", "latch_check"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_1609_03986_gb300 as P
    bound = {e[0] for e in P.EXPORTS}
    assert set(_declared()) <= bound | {"latch_version"}
    for n in _declared():
        assert callable(getattr(P, n)), n


def test_record_layouts():
    import paper_1609_03986_gb300 as P
    assert P.MATCH_DTYPE.itemsize == 16
    assert P.KEYPOINT_DTYPE.itemsize == 12
    rec = P.pack_keypoints([[1, 2, 3, 4], [-5, 6, 31, 2]])
    assert rec.shape == (2, 12)
    assert list(rec[1, :10]) == [251, 255, 255, 255, 6, 0, 0, 0, 31, 2]


def test_no_device_means_clean_error(lib):
    """Without a GPU, creating a context fails with a status code, not a crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1609_03986_gb300 as P
    with pytest.raises(P.LatchError):
        P.latch_context_create(0)
    assert P.latch_last_error(None)


def test_oracle_is_not_on_the_product_path():
    """The package never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1609_03986_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".c")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "liboracle" not in src and "oracle_" not in src, f

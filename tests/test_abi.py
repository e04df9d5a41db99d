"""The C ABI: every function declared in include/jatam.h is exported by
libjatam.so, the library loads without a GPU, and the host-only entry points
behave (no CUDA work is started here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2205_15311_gb300 import binding as J
from paper_2205_15311_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "jatam.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*\**\s*(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return J.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("jatam_enumerate", "jatam_classify_batch", "ga_evaluate", "jatam_shutdown", "jatam_last_error"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    assert ctypes.sizeof(J.jatam_config) == 16
    assert J.RESULT_DTYPE.itemsize == 8
    assert J.HIST_DTYPE.itemsize == 32


def test_last_error_starts_empty(lib):
    assert J.jatam_last_error() == ""


def _hist(rows):
    h = np.zeros(len(rows), J.HIST_DTYPE)
    for i, (cls, hh, size, count, mid) in enumerate(rows):
        h[i] = (cls, hh, size, 0, count, mid)
    return h


def test_hist_merge_host_only(lib):
    a = _hist([(0, 5, 2, 10, 7), (0, 9, 3, 1, 100), (1, 0, 0, 50, 3)])
    b = _hist([(0, 5, 2, 4, 2), (0, 7, 4, 2, 11), (3, 0, 0, 6, 1)])
    m = J.merge_histograms(a, b)
    assert [(int(r["cls"]), int(r["shape_hash"]), int(r["count"]), int(r["min_id"])) for r in m] == [
        (0, 5, 14, 2), (0, 7, 2, 11), (0, 9, 1, 100), (1, 0, 50, 3), (3, 0, 6, 1)]
    assert not m["flags"].any()
    # a size disagreement on one key is a detected hash collision
    c = _hist([(0, 5, 3, 1, 0)])
    assert J.merge_histograms(a, c)["flags"][0] == 1
    # too small an output is an error and still reports the length
    out = np.zeros(1, J.HIST_DTYPE)
    n = ctypes.c_uint32(0)
    rc = J.jatam_hist_merge(a.ctypes.data, 3, b.ctypes.data, 3, out.ctypes.data, 1, ctypes.addressof(n))
    assert rc == J.JATAM_EINVAL and n.value == 5
    assert "cap" in J.jatam_last_error()

"""The C ABI library builds, loads and exports every function include/dtwgb.h declares.

Runs on CPU: no compute call is made (no GPU here), only symbol lookups and
calls that do not touch the device.
"""

import ctypes
import os
import re

import pytest

from paper_2307_04904_gb300 import api
from paper_2307_04904_gb300 import build as B

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(INCLUDE, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src))
    return sorted(names - {"defined"})


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_binding_names():
    assert set(_declared()) == set(api.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    lib.dtw_version.restype = ctypes.c_char_p
    assert lib.dtw_version().decode().count(".") == 2
    lib.dtw_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.dtw_last_error(), bytes)
    lib.dtw_max_band_cells.restype = ctypes.c_int32
    assert lib.dtw_max_band_cells() >= 256


def test_argument_errors_before_any_device_work(lib):
    # p < 1 and NULL pointers are rejected on the host, before any CUDA call
    lib.dtw_pairwise.restype = ctypes.c_int
    assert lib.dtw_pairwise(None, None, 0, 3, 0, None, None) == api.DTW_EINVAL
    assert lib.dtw_pairwise(None, None, 5, 3, 0, None, None) == api.DTW_EINVAL
    lib.dtw_last_error.restype = ctypes.c_char_p
    assert b"NULL" in lib.dtw_last_error()
    lib.kmedoids_fit.restype = ctypes.c_int
    assert lib.kmedoids_fit(None, 0, 1, None, 10, None, None, None, None, None) == api.DTW_EINVAL
    assert lib.kmedoids_fit(None, 5, 6, None, 10, None, None, None, None, None) == api.DTW_EINVAL

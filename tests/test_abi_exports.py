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


def test_describe_shape_is_host_only(monkeypatch):
    """The shape chooser runs on the host: the benchmark workload's band (w = 51, L = 512)
    goes to the two-row kernel with four lanes of 2 x 13 slots (104 slots for 103 band
    cells, one masked); very wide ragged bands go to the column strips; DTWGB_SHAPE is
    honoured; a bad length range is refused."""
    from paper_2307_04904_gb300 import api

    assert api.describe_shape(512, 512, 51) == "dtw_tworow_kernel<H=13,MT=1> G=4"
    assert api.describe_shape(256, 256, 25) == "dtw_tworow_kernel<H=13,MT=1> G=2"
    assert api.describe_shape(64, 2048, 50, permille=True).startswith("dtw_strip_kernel")
    # sets of several lengths take 256-column strips (the model, which sees only the extreme
    # pair, would take 512); one length keeps the model's choice; a band of 153 cells takes the
    # one-row K = 20 with an 8-slot tail over the fully masked two-row H = 10
    assert api.describe_shape(300, 2000, 1700) == "dtw_strip_kernel<K=8>"
    assert api.describe_shape(768, 768, 76) == "dtw_band_kernel<K=20,MT=8> G=8 pairs_per_lane=1"
    monkeypatch.setenv("DTWGB_SHAPE", "rot:13:8")
    assert api.describe_shape(512, 512, 51) == "dtw_band_kernel<K=13,MT=1> G=8 pairs_per_lane=1"
    monkeypatch.delenv("DTWGB_SHAPE")
    with pytest.raises(api.DTWError) as e:
        api.describe_shape(10, 5, 3)
    assert e.value.code == api.DTW_EINVAL


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


def test_new_entry_points_reject_bad_arguments_on_the_host(lib):
    """Argument checks that need no device: NULL pointers and sizes out of range."""
    lib.dtw_last_error.restype = ctypes.c_char_p
    cases = [
        ("dtw_pairs", (None, None, 0, None, None, 0, 3, 0, None, None)),
        ("dtw_pairs", (None, None, 4, None, None, -1, 3, 0, None, None)),
        ("kmedoids_pam", (None, 10, 3, None, 5, None, None, None, None, None)),
        ("kmedoids_pam", (ctypes.c_void_p(16), 10, 65, None, 5, ctypes.c_void_p(16),
                          ctypes.c_void_p(16), None, None, None)),
        ("kmedoids_silhouette", (None, 10, None, 3, None, None, None)),
        ("proposal_kmeanspp", (None, 10, 4, 3, 0, None, None)),
        ("proposal_kmeans", (ctypes.c_void_p(16), 10, 4, 11, 1, 5, 0, ctypes.c_void_p(16), None,
                             None)),
        ("kmedoids_lazy_fit", (None, None, 0, 5, 0, None, 0, 2, None, 0, 0, 0, 10, None, None, None,
                               None, None, None)),
        ("dtw_encoder_create", (100, 8, None)),
        ("dtw_encoder_targets", (None, 10, None, None)),
        ("dtw_encoder_targets", (ctypes.c_void_p(16), 1, ctypes.c_void_p(16), None)),  # S < 2
    ]
    for name, args in cases:
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(*args) == api.DTW_EINVAL, name
        assert lib.dtw_last_error(), name


def test_binding_rejects_short_or_mistyped_buffers_before_the_call():
    """The binding checks the sizes and dtypes of caller buffers (outputs the library writes,
    n labels and k medoids) before anything reaches the library: a short or mistyped buffer
    would otherwise be written past its end.  CPU tensors are enough, the checks come first."""
    import torch

    from paper_2307_04904_gb300 import api

    D = torch.zeros((6, 6), dtype=torch.float32)
    init = torch.tensor([0, 3], dtype=torch.int32)
    bad = [
        dict(out_medoids=torch.zeros(1, dtype=torch.int32)),          # fewer than k
        dict(out_medoids=torch.zeros(2, dtype=torch.int64)),          # wrong dtype
        dict(out_labels=torch.zeros(5, dtype=torch.int32)),           # fewer than n
        dict(out_labels=torch.zeros(6, dtype=torch.int64)),           # 8-byte labels
    ]
    for fn in (api.kmedoids_fit, api.kmedoids_fit_noalloc):
        for kw in bad:
            with pytest.raises((TypeError, ValueError)):
                fn(D, 2, init, **kw)
    with pytest.raises(ValueError, match="square"):
        api.kmedoids_fit(torch.zeros((6, 5)), 2, init)
    # the initial medoids must be exactly k entries (a short list would be read past its end)
    for fn in (api.kmedoids_fit, api.kmedoids_fit_noalloc, api.kmedoids_pam):
        with pytest.raises(ValueError, match="init_medoids"):
            fn(D, 3, init)
    with pytest.raises((TypeError, ValueError)):
        api.kmedoids_silhouette(D, torch.zeros(5, dtype=torch.int32), 2)
    with pytest.raises((TypeError, ValueError)):
        api.proposal_kmeanspp(torch.zeros((6, 4)), 3, 0, out=torch.zeros(2, dtype=torch.int32))
    # correct sizes on the CPU reach the device check and fail loudly (no CPU fallback)
    with pytest.raises(TypeError, match="CUDA"):
        api.kmedoids_fit(D, 2, init)


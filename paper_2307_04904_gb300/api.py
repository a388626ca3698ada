"""Python binding of the dtwgb C ABI (``include/dtwgb.h``).

Argument marshalling only: tensors are passed as raw device pointers and the
caller's current CUDA stream is passed as the stream handle.  Every step of the
computation runs in the CUDA library; there is no CPU fallback.  If the shared
library has not been built, or no GPU is present, the calls raise.

Functions keep the C names:

* ``dtw_pairwise(values, offsets, window, ...)`` -> D (p x p float32, or packed)
* ``dtw_query(query, values, offsets, window, ...)`` -> one row of D
* ``dtw_pairs(values, offsets, pair_a, pair_b, window, ...)`` -> DTW of listed pairs
* ``kmedoids_fit(D, k, init_medoids, max_iter)`` -> (medoids, labels, cost, iters),
  ``kmedoids_fit_noalloc`` the same without device allocation
* ``kmedoids_pam(D, k, init_medoids, max_swaps)`` -> PAM BUILD / SWAP
* ``kmedoids_silhouette(D, labels, k)`` -> (per-point silhouette, mean)
* ``kmedoids_lazy_fit(values, offsets, window, k, init, ...)`` -> k-medoids over exact DTW
  computed pair by pair, with optional embedding proposals and sampled screening
* ``proposal_kmeanspp`` / ``proposal_kmeans`` -> initial medoids from embeddings
* ``Batch`` -> planned, graph-captured batches of ragged DTW jobs (dtwgb_batch.h);
  ``batch_run_once`` plans, runs and releases one without device synchronisation
* ``describe_shape`` -> the kernel and shape dtw_pairwise picks (host only)
* ``Encoder`` -> the proposal encoder's training and inference (dtwgb_encoder.h)
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

DTW_OK = 0
DTW_EINVAL = -1
DTW_ENOMEM = -2
DTW_ECUDA = -3
DTW_ETIMEOUT = -4
DTW_EUNSUPPORTED = -5

DTW_BAND_STRICT = 0x1
DTW_OUT_PACKED_UPPER = 0x2
DTW_HOST_IO = 0x4
DTW_CHECK_FINITE = 0x8
DTW_WINDOW_PERMILLE = 0x10
DTW_OFFSETS_HOST = 0x20

_ERRNAMES = {DTW_EINVAL: "DTW_EINVAL", DTW_ENOMEM: "DTW_ENOMEM", DTW_ECUDA: "DTW_ECUDA",
             DTW_ETIMEOUT: "DTW_ETIMEOUT", DTW_EUNSUPPORTED: "DTW_EUNSUPPORTED"}

# every symbol include/dtwgb.h declares
EXPORTS = ("dtw_last_error", "dtw_version", "dtw_pairwise", "dtw_query", "dtw_max_band_cells",
           "dtw_describe_shape",
           "kmedoids_fit", "kmedoids_fit_noalloc", "dtw_batch_create", "dtw_batch_run",
           "dtw_batch_get_info", "dtw_batch_get_class", "dtw_batch_destroy", "dtw_batch_run_once",
           "dtw_encoder_num_params", "dtw_encoder_create", "dtw_encoder_set_params",
           "dtw_encoder_get_params", "dtw_encoder_get_grads", "dtw_encoder_embed",
           "dtw_encoder_train", "dtw_encoder_targets", "dtw_encoder_init_params",
           "dtw_encoder_check", "dtw_encoder_destroy", "dtw_encoder_get_tensor", "dtw_pairs",
           "proposal_kmeanspp", "proposal_kmeans", "kmedoids_lazy_fit", "kmedoids_silhouette",
           "kmedoids_pam")

DTW_BATCH_GRAPH = 0x1
DTW_BATCH_AUTOTUNE = 0x2
DTW_BATCH_UNSORTED = 0x4
DTW_BATCH_POOLED = 0x8


class DTWJob(ctypes.Structure):
    """struct dtw_job of include/dtwgb_batch.h."""

    _fields_ = [("values", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("offsets_host", ctypes.c_void_p), ("p", ctypes.c_int32),
                ("query", ctypes.c_void_p), ("qlen", ctypes.c_int32),
                ("window", ctypes.c_int32), ("window_permille", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("out", ctypes.c_void_p)]


class DTWBatchInfo(ctypes.Structure):
    """struct dtw_batch_info of include/dtwgb_batch.h."""

    _fields_ = [("pairs", ctypes.c_int64), ("cells", ctypes.c_int64),
                ("classes", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("buckets_tuned", ctypes.c_int32), ("jobs", ctypes.c_int32)]


class DTWError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libdtwgb.so (built in-tree by ``build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"dtwgb CUDA library not built ({path} missing); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        lib.dtw_last_error.restype = ctypes.c_char_p
        lib.dtw_last_error.argtypes = []
        lib.dtw_version.restype = ctypes.c_char_p
        lib.dtw_version.argtypes = []
        lib.dtw_max_band_cells.restype = _i32
        lib.dtw_max_band_cells.argtypes = []
        lib.dtw_describe_shape.restype = ctypes.c_int
        lib.dtw_describe_shape.argtypes = [_i32, _i32, _i32, _u32, ctypes.c_char_p, _i32]
        lib.dtw_pairwise.restype = ctypes.c_int
        lib.dtw_pairwise.argtypes = [_p, _p, _i32, _i32, _u32, _p, _p]
        lib.dtw_query.restype = ctypes.c_int
        lib.dtw_query.argtypes = [_p, _i32, _p, _p, _i32, _i32, _u32, _p, _p]
        lib.kmedoids_fit.restype = ctypes.c_int
        lib.kmedoids_fit.argtypes = [_p, _i32, _i32, _p, _i32, _p, _p,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i32), _p]
        lib.kmedoids_fit_noalloc.restype = ctypes.c_int
        lib.kmedoids_fit_noalloc.argtypes = lib.kmedoids_fit.argtypes
        lib.dtw_batch_create.restype = ctypes.c_int
        lib.dtw_batch_create.argtypes = [ctypes.POINTER(DTWJob), _i32, _u32, _p,
                                         ctypes.POINTER(ctypes.c_void_p)]
        lib.dtw_batch_run.restype = ctypes.c_int
        lib.dtw_batch_run.argtypes = [_p, _p]
        lib.dtw_batch_run_once.restype = ctypes.c_int
        lib.dtw_batch_run_once.argtypes = [ctypes.POINTER(DTWJob), _i32, _u32, _p]
        lib.dtw_batch_get_info.restype = ctypes.c_int
        lib.dtw_batch_get_info.argtypes = [_p, ctypes.POINTER(DTWBatchInfo)]
        lib.dtw_batch_get_class.restype = ctypes.c_int
        lib.dtw_batch_get_class.argtypes = [_p, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                            ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]
        lib.dtw_batch_destroy.restype = None
        lib.dtw_batch_destroy.argtypes = [_p]
        lib.dtw_encoder_num_params.restype = _i32
        lib.dtw_encoder_num_params.argtypes = []
        lib.dtw_encoder_create.restype = ctypes.c_int
        lib.dtw_encoder_create.argtypes = [_i32, _i32, ctypes.POINTER(ctypes.c_void_p)]
        for f in ("dtw_encoder_set_params", "dtw_encoder_get_params", "dtw_encoder_get_grads"):
            getattr(lib, f).restype = ctypes.c_int
            getattr(lib, f).argtypes = [_p, _p]
        lib.dtw_encoder_embed.restype = ctypes.c_int
        lib.dtw_encoder_embed.argtypes = [_p, _p, _i32, _p, _p]
        lib.dtw_encoder_train.restype = ctypes.c_int
        lib.dtw_encoder_train.argtypes = [_p, _p, _i32, _p, _p, _i32, _p, _i32, _p]
        lib.dtw_encoder_check.restype = ctypes.c_int
        lib.dtw_encoder_check.argtypes = [_p]
        lib.dtw_encoder_get_tensor.restype = ctypes.c_int
        lib.dtw_encoder_get_tensor.argtypes = [_p, _i32, _p]
        lib.dtw_encoder_init_params.restype = ctypes.c_int
        lib.dtw_encoder_init_params.argtypes = [_p, ctypes.c_uint64]
        lib.dtw_encoder_targets.restype = ctypes.c_int
        lib.dtw_encoder_targets.argtypes = [_p, _i32, _p, _p]
        lib.dtw_encoder_destroy.restype = None
        lib.dtw_encoder_destroy.argtypes = [_p]
        lib.dtw_pairs.restype = ctypes.c_int
        lib.dtw_pairs.argtypes = [_p, _p, _i32, _p, _p, ctypes.c_int64, _i32, _u32, _p, _p]
        lib.proposal_kmeanspp.restype = ctypes.c_int
        lib.proposal_kmeanspp.argtypes = [_p, _i32, _i32, _i32, ctypes.c_uint64, _p, _p]
        lib.kmedoids_silhouette.restype = ctypes.c_int
        lib.kmedoids_silhouette.argtypes = [_p, _i32, _p, _i32, _p, ctypes.POINTER(ctypes.c_double),
                                            _p]
        lib.kmedoids_pam.restype = ctypes.c_int
        lib.kmedoids_pam.argtypes = [_p, _i32, _i32, _p, _i32, _p, _p,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i32), _p]
        lib.proposal_kmeans.restype = ctypes.c_int
        lib.proposal_kmeans.argtypes = [_p, _i32, _i32, _i32, _i32, _i32, ctypes.c_uint64, _p,
                                        ctypes.POINTER(ctypes.c_double), _p]
        lib.kmedoids_lazy_fit.restype = ctypes.c_int
        lib.kmedoids_lazy_fit.argtypes = [_p, _p, _i32, _i32, _u32, _p, _i32, _i32, _p, _i32,
                                          _i32, _i32, _i32, _p, _p,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_int64),
                                          _p]
        _lib = lib
        return lib


def _check(rc: int):
    if rc != DTW_OK:
        msg = load().dtw_last_error().decode(errors="replace")
        raise DTWError(rc, msg)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _vec(t, dtype, n: int, name: str):
    """Shape and dtype of a caller's 1-D buffer of n elements, checked before any launch."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return t


def _square(D: torch.Tensor, name: str = "D") -> int:
    if not isinstance(D, torch.Tensor) or D.dim() != 2 or D.shape[0] != D.shape[1]:
        raise ValueError(f"{name} must be a square matrix")
    return D.shape[0]


def _init_medoids(init, k: int) -> torch.Tensor:
    """Initial medoids as an int32 tensor of exactly k entries (moved to the device later)."""
    if not (isinstance(init, torch.Tensor) and init.dtype == torch.int32):
        init = torch.as_tensor(init, dtype=torch.int32)
    if init.numel() != k:
        raise ValueError(f"init_medoids has {init.numel()} entries, expected k = {k}")
    return init


def _on(t: torch.Tensor, device, name: str):
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _host_offsets(offsets_host, n: int):
    """A C-contiguous int64 numpy copy-free view of host offsets with n entries."""
    import numpy as np

    oh = np.ascontiguousarray(np.asarray(offsets_host, dtype=np.int64))
    if oh.ndim != 1 or oh.size != n:
        raise ValueError(f"offsets_host must hold {n} int64 values")
    return oh


def _flags(strict: bool, packed: bool = False, check_finite: bool = False,
           permille: bool = False) -> int:
    f = DTW_WINDOW_PERMILLE if permille else 0
    if strict:
        f |= DTW_BAND_STRICT
    if packed:
        f |= DTW_OUT_PACKED_UPPER
    if check_finite:
        f |= DTW_CHECK_FINITE
    return f


def dtw_pairwise(values: torch.Tensor, offsets: torch.Tensor, window: int = -1, *,
                 strict: bool = False, packed: bool = False, check_finite: bool = False,
                 permille: bool = False, out: torch.Tensor | None = None,
                 offsets_host=None, stream=None) -> torch.Tensor:
    """All-pairs DTW matrix D of a set (values float32, offsets int64, both on the GPU).

    With ``permille`` the window is per mille of the longer series of each pair.  With
    ``offsets_host`` (the same offsets as a host int64 array) the call neither reads the
    offsets back nor synchronises the stream (DTW_OFFSETS_HOST); ``offsets`` is then
    not used."""
    _dev(values, torch.float32, "values")
    extra = 0
    if offsets_host is not None:
        oh = _host_offsets(offsets_host, offsets_host.shape[0] if hasattr(offsets_host, "shape")
                           else len(offsets_host))
        return _pairwise_offsets_host(values, oh, window, strict, packed, check_finite,
                                      permille, out, stream, extra)
    _dev(offsets, torch.int64, "offsets")
    p = offsets.numel() - 1
    n_out = p * (p - 1) // 2 if packed else p * p
    if out is None:
        shape = (n_out,) if packed else (p, p)
        out = torch.empty(shape, dtype=torch.float32, device=values.device)
    else:
        _dev(out, torch.float32, "out")
        if out.numel() != n_out:
            raise ValueError(f"out has {out.numel()} elements, expected {n_out}")
    with torch.cuda.device(values.device):
        rc = load().dtw_pairwise(values.data_ptr(), offsets.data_ptr(), p, int(window),
                                 _flags(strict, packed, check_finite, permille) | extra,
                                 out.data_ptr(), _stream_handle(stream))
    _check(rc)
    return out


def _pairwise_offsets_host(values, oh, window, strict, packed, check_finite, permille, out,
                           stream, extra=0):
    p = oh.size - 1
    n_out = p * (p - 1) // 2 if packed else p * p
    if out is None:
        out = torch.empty((n_out,) if packed else (p, p), dtype=torch.float32,
                          device=values.device)
    else:
        _dev(out, torch.float32, "out")
        if out.numel() != n_out:
            raise ValueError(f"out has {out.numel()} elements, expected {n_out}")
    with torch.cuda.device(values.device):
        rc = load().dtw_pairwise(values.data_ptr(), oh.ctypes.data, p, int(window),
                                 _flags(strict, packed, check_finite, permille) | DTW_OFFSETS_HOST
                                 | extra,
                                 out.data_ptr(), _stream_handle(stream))
    _check(rc)
    return out


def describe_shape(minlen: int, maxlen: int, window: int = -1, *, strict: bool = False,
                   permille: bool = False) -> str:
    """The kernel and shape dtw_pairwise runs for series lengths in [minlen, maxlen] (host only)."""
    buf = ctypes.create_string_buffer(160)
    _check(load().dtw_describe_shape(int(minlen), int(maxlen), int(window),
                                     _flags(strict, False, False, permille), buf, len(buf)))
    return buf.value.decode()


def dtw_pairwise_host(values, offsets, window: int = -1, *, strict: bool = False,
                      packed: bool = False, out=None):
    """Same as dtw_pairwise on HOST numpy/tensor buffers (DTW_HOST_IO): the library
    stages them through device memory; synchronous."""
    import numpy as np

    v = np.ascontiguousarray(np.asarray(values, dtype=np.float32))
    o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    p = o.size - 1
    n_out = p * (p - 1) // 2 if packed else p * p
    if out is None:
        out = np.empty(n_out if packed else (p, p), dtype=np.float32)
    elif out.dtype != np.float32 or out.size != n_out or not out.flags.c_contiguous:
        raise ValueError(f"out must be a contiguous float32 array of {n_out} elements")
    rc = load().dtw_pairwise(v.ctypes.data, o.ctypes.data, p, int(window),
                             _flags(strict, packed) | DTW_HOST_IO, out.ctypes.data,
                             _stream_handle(None))
    _check(rc)
    return out


def dtw_query_host(query, values, offsets, window: int = -1, *, strict: bool = False, out=None):
    """Same as dtw_query on HOST numpy/tensor buffers (DTW_HOST_IO); synchronous."""
    import numpy as np

    q = np.ascontiguousarray(np.asarray(query, dtype=np.float32))
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float32))
    o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    p = o.size - 1
    if out is None:
        out = np.empty(p, dtype=np.float32)
    elif out.dtype != np.float32 or out.size != p or not out.flags.c_contiguous:
        raise ValueError(f"out must be a contiguous float32 array of {p} elements")
    rc = load().dtw_query(q.ctypes.data, q.size, v.ctypes.data, o.ctypes.data, p, int(window),
                          _flags(strict) | DTW_HOST_IO, out.ctypes.data, _stream_handle(None))
    _check(rc)
    return out


def dtw_query(query: torch.Tensor, values: torch.Tensor, offsets: torch.Tensor,
              window: int = -1, *, strict: bool = False, check_finite: bool = False,
              out: torch.Tensor | None = None, offsets_host=None, stream=None) -> torch.Tensor:
    """DTW of one query against every series of a resident set (``offsets_host``: as for
    dtw_pairwise)."""
    _dev(query, torch.float32, "query")
    _dev(values, torch.float32, "values")
    flags_extra = 0
    if offsets_host is not None:
        offsets_host = _host_offsets(offsets_host, len(offsets_host))
        p = offsets_host.size - 1
        off_ptr = offsets_host.ctypes.data
        flags_extra |= DTW_OFFSETS_HOST
    else:
        _dev(offsets, torch.int64, "offsets")
        p = offsets.numel() - 1
        off_ptr = offsets.data_ptr()
    if out is None:
        out = torch.empty(p, dtype=torch.float32, device=values.device)
    else:
        _dev(out, torch.float32, "out")
        if out.numel() != p:
            raise ValueError("out must have p elements")
    with torch.cuda.device(values.device):
        rc = load().dtw_query(query.data_ptr(), query.numel(), values.data_ptr(), off_ptr, p,
                              int(window), _flags(strict, False, check_finite) | flags_extra,
                              out.data_ptr(), _stream_handle(stream))
    _check(rc)
    return out


def dtw_pairs(values: torch.Tensor, offsets: torch.Tensor, pair_a: torch.Tensor,
              pair_b: torch.Tensor, window: int = -1, *, strict: bool = False,
              permille: bool = False, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    """DTW of the listed pairs (pair_a[t], pair_b[t]) of one resident set."""
    _dev(values, torch.float32, "values")
    _dev(offsets, torch.int64, "offsets")
    _dev(pair_a, torch.int32, "pair_a")
    _dev(pair_b, torch.int32, "pair_b")
    if pair_a.numel() != pair_b.numel():
        raise ValueError("pair_a and pair_b differ in length")
    npairs = pair_a.numel()
    if out is None:
        out = torch.empty(npairs, dtype=torch.float32, device=values.device)
    else:
        _dev(out, torch.float32, "out")
        if out.numel() != npairs:
            raise ValueError("out must have one element per pair")
    with torch.cuda.device(values.device):
        rc = load().dtw_pairs(values.data_ptr(), offsets.data_ptr(), offsets.numel() - 1,
                              pair_a.data_ptr(), pair_b.data_ptr(), npairs, int(window),
                              _flags(strict, False, False, permille), out.data_ptr(),
                              _stream_handle(stream))
    _check(rc)
    return out


def proposal_kmeanspp(emb: torch.Tensor, k: int, seed: int, *, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """k distinct initial medoids by k-means++ seeding over embeddings emb [n][dim]."""
    if out is not None:
        _vec(out, torch.int32, int(k), "out")
    _dev(emb, torch.float32, "emb")
    n, dim = emb.shape
    if out is None:
        out = torch.empty(k, dtype=torch.int32, device=emb.device)
    _on(out, emb.device, "out")
    with torch.cuda.device(emb.device):
        rc = load().proposal_kmeanspp(emb.data_ptr(), n, dim, int(k),
                                      int(seed) & 0xFFFFFFFFFFFFFFFF, out.data_ptr(),
                                      _stream_handle(stream))
    _check(rc)
    return out


def proposal_kmeans(emb: torch.Tensor, k: int, seed: int, *, restarts: int = 4,
                    iters: int = 25, stream=None):
    """Medoid proposals from k-means in embedding space: (medoids int32[k], inertia)."""
    _dev(emb, torch.float32, "emb")
    n, dim = emb.shape
    out = torch.empty(k, dtype=torch.int32, device=emb.device)
    inertia = ctypes.c_double()
    with torch.cuda.device(emb.device):
        rc = load().proposal_kmeans(emb.data_ptr(), n, dim, int(k), int(restarts), int(iters),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, out.data_ptr(),
                                    ctypes.byref(inertia), _stream_handle(stream))
    _check(rc)
    return out, inertia.value


def kmedoids_lazy_fit(values: torch.Tensor, offsets: torch.Tensor, window: int, k: int,
                      init_medoids: torch.Tensor, *, emb: torch.Tensor | None = None,
                      candidates: int = 0, screen_sample: int = 0, screen_keep: int = 0,
                      max_iter: int = 100, strict: bool = False, permille: bool = False,
                      stream=None):
    """Alternate k-medoids over exact DTW computed pair by pair (no matrix D).

    Returns (medoids int32[k], labels int32[n], cost float, iters int, pairs int).
    """
    _dev(values, torch.float32, "values")
    _dev(offsets, torch.int64, "offsets")
    n = offsets.numel() - 1
    dim = 0
    if emb is not None:
        _dev(emb, torch.float32, "emb")
        dim = emb.shape[1]
    if emb is not None and (emb.dim() != 2 or emb.shape[0] != n):
        raise ValueError(f"emb must be [n = {n}][dim]")
    init = _init_medoids(init_medoids, int(k)).to(values.device).contiguous()
    med = torch.empty(k, dtype=torch.int32, device=values.device)
    lab = torch.empty(n, dtype=torch.int32, device=values.device)
    cost, iters, pairs = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int64()
    with torch.cuda.device(values.device):
        rc = load().kmedoids_lazy_fit(values.data_ptr(), offsets.data_ptr(), n, int(window),
                                      _flags(strict, False, False, permille),
                                      emb.data_ptr() if emb is not None else None, dim, int(k),
                                      init.data_ptr(), int(candidates), int(screen_sample),
                                      int(screen_keep), int(max_iter),
                                      med.data_ptr(), lab.data_ptr(), ctypes.byref(cost),
                                      ctypes.byref(iters), ctypes.byref(pairs),
                                      _stream_handle(stream))
    _check(rc)
    return med, lab, cost.value, iters.value, pairs.value


def kmedoids_fit(D: torch.Tensor, k: int, init_medoids: torch.Tensor, max_iter: int = 100, *,
                 out_medoids: torch.Tensor | None = None, out_labels: torch.Tensor | None = None,
                 stream=None, _symbol: str = "kmedoids_fit"):
    """Alternate k-medoids over a symmetric float32 D on the GPU.

    Returns (medoids int32[k], labels int32[n], cost float, iters int).
    """
    # sizes and dtypes first: a short or mistyped buffer would be written past its end
    n = _square(D)
    if out_medoids is not None:
        _vec(out_medoids, torch.int32, int(k), "out_medoids")
    if out_labels is not None:
        _vec(out_labels, torch.int32, n, "out_labels")
    init = _init_medoids(init_medoids, int(k))
    _dev(D, torch.float32, "D")
    init = init.to(D.device).contiguous()
    if out_medoids is None:
        out_medoids = torch.empty(k, dtype=torch.int32, device=D.device)
    if out_labels is None:
        out_labels = torch.empty(n, dtype=torch.int32, device=D.device)
    _on(out_medoids, D.device, "out_medoids")
    _on(out_labels, D.device, "out_labels")
    cost = ctypes.c_double()
    iters = ctypes.c_int32()
    with torch.cuda.device(D.device):
        rc = getattr(load(), _symbol)(D.data_ptr(), n, int(k), init.data_ptr(), int(max_iter),
                                      out_medoids.data_ptr(), out_labels.data_ptr(),
                                      ctypes.byref(cost), ctypes.byref(iters),
                                      _stream_handle(stream))
    _check(rc)
    return out_medoids, out_labels, cost.value, iters.value


def kmedoids_silhouette(D: torch.Tensor, labels: torch.Tensor, k: int, *,
                        out: torch.Tensor | None = None, stream=None):
    """Silhouette of a clustering over D: (s float32[n] on the GPU, mean float)."""
    n = _square(D)
    _vec(labels, torch.int32, n, "labels")
    if out is not None:
        _vec(out, torch.float32, n, "out")
    _dev(D, torch.float32, "D")
    _dev(labels, torch.int32, "labels")
    _on(labels, D.device, "labels")
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=D.device)
    _on(out, D.device, "out")
    mean = ctypes.c_double()
    with torch.cuda.device(D.device):
        rc = load().kmedoids_silhouette(D.data_ptr(), n, labels.data_ptr(), int(k), out.data_ptr(),
                                        ctypes.byref(mean), _stream_handle(stream))
    _check(rc)
    return out, mean.value


def kmedoids_pam(D: torch.Tensor, k: int, init_medoids: torch.Tensor | None = None,
                 max_swaps: int = 1000, *, stream=None):
    """PAM (BUILD when no initial medoids, then best-swap passes) over D on the GPU.

    Returns (medoids int32[k], labels int32[n], cost float, swaps int).
    """
    n = _square(D)
    init = None
    if init_medoids is not None:
        init = _init_medoids(init_medoids, int(k))
    _dev(D, torch.float32, "D")
    if init is not None:
        init = init.to(D.device).contiguous()
    med = torch.empty(k, dtype=torch.int32, device=D.device)
    lab = torch.empty(n, dtype=torch.int32, device=D.device)
    cost, swaps = ctypes.c_double(), ctypes.c_int32()
    with torch.cuda.device(D.device):
        rc = load().kmedoids_pam(D.data_ptr(), n, int(k), init.data_ptr() if init is not None else None,
                                 int(max_swaps), med.data_ptr(), lab.data_ptr(), ctypes.byref(cost),
                                 ctypes.byref(swaps), _stream_handle(stream))
    _check(rc)
    return med, lab, cost.value, swaps.value


def kmedoids_fit_noalloc(D: torch.Tensor, k: int, init_medoids: torch.Tensor,
                         max_iter: int = 100, *, out_medoids: torch.Tensor | None = None,
                         out_labels: torch.Tensor | None = None, stream=None):
    """kmedoids_fit that allocates no device memory (static scratch; n <= 65536, k <= 1024).

    For callers that must not allocate during the call; calls that overlap on
    the GPU race on the shared scratch.  ``out_medoids``/``out_labels`` should
    be passed preallocated by such callers (otherwise this wrapper creates
    them with torch before the call).
    """
    return kmedoids_fit(D, k, init_medoids, max_iter, out_medoids=out_medoids,
                        out_labels=out_labels, stream=stream, _symbol="kmedoids_fit_noalloc")


def _job_array(jobs, keep: list, outputs: list):
    """The dtw_job array of a list of job dicts (see Batch); keeps every buffer it points to
    alive in `keep` and appends each job's output to `outputs`."""
    import numpy as np

    arr = (DTWJob * len(jobs))()
    for i, j in enumerate(jobs):
        v = _dev(j["values"], torch.float32, "values")
        o = _dev(j["offsets"], torch.int64, "offsets")
        p = o.numel() - 1
        oh = j.get("offsets_host")
        oh = np.ascontiguousarray(o.cpu().numpy()) if oh is None else _host_offsets(oh, p + 1)
        q = j.get("query")
        if q is not None:
            _dev(q, torch.float32, "query")
        packed = bool(j.get("packed", False))
        n_out = p if q is not None else (p * (p - 1) // 2 if packed else p * p)
        out = j.get("out")
        if out is None:
            shape = (p, p) if (q is None and not packed) else (n_out,)
            out = torch.empty(shape, dtype=torch.float32, device=v.device)
        else:
            _dev(out, torch.float32, "out")
            if out.numel() != n_out:
                raise ValueError(f"job {i}: out has {out.numel()} elements, expected {n_out}")
        arr[i].values = v.data_ptr()
        arr[i].offsets = o.data_ptr()
        arr[i].offsets_host = oh.ctypes.data
        arr[i].p = p
        arr[i].query = q.data_ptr() if q is not None else None
        arr[i].qlen = q.numel() if q is not None else 0
        arr[i].window = int(j.get("window", -1))
        arr[i].window_permille = int(j.get("window_permille", 0))
        arr[i].flags = _flags(bool(j.get("strict", False)), packed)
        arr[i].out = out.data_ptr()
        keep += [v, o, oh, q, out]
        outputs.append(out)
    return arr


def batch_run_once(jobs, *, unsorted: bool = False, stream=None) -> list:
    """Plan, run once and release a batch of job dicts (see Batch) on `stream`, with every
    device buffer from the library's stream-ordered pool and no device synchronisation
    (dtw_batch_run_once).  Returns the jobs' outputs; they are final when `stream`
    reaches the enqueued work.  The caller keeps the inputs alive until then."""
    keep, outputs = [], []
    arr = _job_array(jobs, keep, outputs)
    dev = outputs[0].device
    with torch.cuda.device(dev):
        rc = load().dtw_batch_run_once(arr, len(jobs), DTW_BATCH_UNSORTED if unsorted else 0,
                                       _stream_handle(stream))
    _check(rc)
    return outputs


class Batch:
    """A planned batch of DTW jobs (include/dtwgb_batch.h).

    ``jobs`` is a list of dicts with keys ``values`` (CUDA float32), ``offsets``
    (CUDA int64), optional ``offsets_host`` (the same offsets as a host int64 array;
    read from the device otherwise), optional ``query`` (CUDA float32), ``window``
    (int, default -1), ``window_permille`` (int, default 0), ``strict`` / ``packed``
    (bools) and optional ``out``.  Outputs are allocated when missing and kept in
    ``self.outputs``; the batch holds references to every buffer it uses.
    """

    def __init__(self, jobs, *, graph: bool = True, autotune: bool = False,
                 unsorted: bool = False, stream=None):
        self._keep = []
        self.outputs = []
        arr = _job_array(jobs, self._keep, self.outputs)
        flags = ((DTW_BATCH_GRAPH if graph else 0) | (DTW_BATCH_AUTOTUNE if autotune else 0)
                 | (DTW_BATCH_UNSORTED if unsorted else 0))
        handle = ctypes.c_void_p()
        rc = load().dtw_batch_create(arr, len(jobs), flags, _stream_handle(stream),
                                     ctypes.byref(handle))
        _check(rc)
        self._h = handle

    def run(self, stream=None):
        _check(load().dtw_batch_run(self._h, _stream_handle(stream)))
        return self.outputs

    def info(self) -> dict:
        inf = DTWBatchInfo()
        _check(load().dtw_batch_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in DTWBatchInfo._fields_}

    def classes(self) -> list:
        out = []
        for i in range(self.info()["classes"]):
            kind, K, G = _i32(), _i32(), _i32()
            items, cells = ctypes.c_int64(), ctypes.c_int64()
            _check(load().dtw_batch_get_class(self._h, i, ctypes.byref(kind), ctypes.byref(K),
                                              ctypes.byref(G), ctypes.byref(items),
                                              ctypes.byref(cells)))
            out.append({"kind": ("rotated", "strip", "tstrip", "tworow")[kind.value], "K": K.value,
                        "G": G.value, "items": items.value, "cells": cells.value})
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().dtw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Encoder:
    """The proposal encoder of include/dtwgb_encoder.h (series of length T)."""

    def __init__(self, T: int, max_batch: int, params=None):
        import numpy as np

        h = ctypes.c_void_p()
        _check(load().dtw_encoder_create(int(T), int(max_batch), ctypes.byref(h)))
        self._h = h
        self.T = T
        self.max_batch = max_batch
        self.n_params = load().dtw_encoder_num_params()
        if params is not None:
            self.set_params(params)
        self._np = np

    def set_params(self, params):
        import numpy as np

        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(load().dtw_encoder_set_params(self._h, p.ctypes.data))

    def check(self):
        """Raise if a tensor-core kernel of this encoder gave up waiting (synchronises)."""
        _check(load().dtw_encoder_check(self._h))

    def init_params(self, seed: int):
        """He-style random parameters drawn on the device from a splitmix64 stream."""
        _check(load().dtw_encoder_init_params(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF))

    def params(self):
        import numpy as np

        p = np.empty(self.n_params, np.float32)
        _check(load().dtw_encoder_get_params(self._h, p.ctypes.data))
        return p

    def grads(self):
        import numpy as np

        g = np.empty(self.n_params, np.float32)
        _check(load().dtw_encoder_get_grads(self._h, g.ctypes.data))
        return g

    TENSORS = ("z1", "h1", "z2", "h2", "z3", "h3", "dz3", "dz2", "dz1", "e", "dE")

    def tensor(self, name: str):
        """A tensor of the last training step as float32 numpy: activations and their
        gradients [S][T][64], the embeddings e and dL/de [S][64]."""
        import numpy as np

        which = self.TENSORS.index(name)
        S = self._last_S
        shape = (S, 64) if name in ("e", "dE") else (S, self.T, 64)
        out = np.empty(shape, np.float32)
        _check(load().dtw_encoder_get_tensor(self._h, which, out.ctypes.data))
        return out

    def embed(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        _dev(x, torch.float32, "x")
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, 64), dtype=torch.float32, device=x.device)
        _check(load().dtw_encoder_embed(self._h, x.data_ptr(), B, out.data_ptr(),
                                        _stream_handle(stream)))
        return out

    @staticmethod
    def targets(D: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """Regression targets sqrt(D) / mean off-diagonal sqrt(D) (zero diagonal)."""
        _dev(D, torch.float32, "D")
        S = D.shape[0]
        if out is None:
            out = torch.empty((S, S), dtype=torch.float32, device=D.device)
        with torch.cuda.device(D.device):
            rc = load().dtw_encoder_targets(D.data_ptr(), S, out.data_ptr(),
                                            _stream_handle(stream))
        _check(rc)
        return out

    def train(self, x: torch.Tensor, targets: torch.Tensor, lr: float, steps: int, *,
              graph: bool = True, stream=None):
        """`steps` full-batch Adam steps; returns the per-step losses (CUDA tensor)."""
        _dev(x, torch.float32, "x")
        _dev(targets, torch.float32, "targets")
        S = x.shape[0]
        if not hasattr(self, "_lr") or self._lr.device != x.device:
            self._lr = torch.empty(1, dtype=torch.float32, device=x.device)
        self._lr.fill_(float(lr))
        need = max(int(steps), 1)
        if not hasattr(self, "_loss") or self._loss.numel() < need:
            self._loss = torch.empty(need, dtype=torch.float32, device=x.device)
        self._last_S = S
        _check(load().dtw_encoder_train(self._h, x.data_ptr(), S, targets.data_ptr(),
                                        self._lr.data_ptr(), int(steps), self._loss.data_ptr(),
                                        1 if graph else 0, _stream_handle(stream)))
        return self._loss[:steps]

    def close(self):
        if getattr(self, "_h", None):
            load().dtw_encoder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

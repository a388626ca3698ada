"""Plain CPU oracle for all-pairs DTW and k-medoids (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path in
``paper_2307_04904_gb300`` and never imports it.

The arithmetic lives in ``dtw_oracle.c`` (double precision, plain dynamic
programme, see the readings in its header); this module only marshals numpy
arrays through ctypes.  ``brute.py`` holds the brute-force references that pin
the oracle.  The shared object is built on first use (``build()``) with gcc and
OpenMP into ``oracle/_build``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_dtw.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile dtw_oracle.c into a shared object (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        # -ffp-contract=off: the double DP must not be fused behind our back;
        # the float mirror calls fmaf explicitly.
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_dtw_f64.restype = ctypes.c_double
        lib.oracle_dtw_f64.argtypes = [_f32p, _i64, _f32p, _i64, _i64, _int]
        lib.oracle_dtw_f32_mirror.restype = ctypes.c_float
        lib.oracle_dtw_f32_mirror.argtypes = [_f32p, _i64, _f32p, _i64, _i64, _int]
        lib.oracle_band_cells.restype = _i64
        lib.oracle_band_cells.argtypes = [_i64, _i64, _i64, _int]
        lib.oracle_pairwise_f64.restype = None
        lib.oracle_pairwise_f64.argtypes = [_f32p, _i64p, _i64, _i64, _int, _f64p, _int]
        lib.oracle_pairs_f64.restype = None
        lib.oracle_pairs_f64.argtypes = [_f32p, _i64p, _i64p, _i64p, _i64, _i64, _int, _f64p, _int]
        lib.oracle_pairs_w_f64.restype = None
        lib.oracle_pairs_w_f64.argtypes = [_f32p, _i64p, _i64p, _i64p, _i64p, _i64, _int, _f64p,
                                           _int]
        lib.oracle_pairs_f32_mirror.restype = None
        lib.oracle_pairs_f32_mirror.argtypes = [
            _f32p, _i64p, _i64p, _i64p, _i64, _i64, _int,
            np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS"), _int]
        lib.oracle_pairs_w_f32_mirror.restype = None
        lib.oracle_pairs_w_f32_mirror.argtypes = [
            _f32p, _i64p, _i64p, _i64p, _i64p, _i64, _int,
            np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS"), _int]
        lib.oracle_query_f64.restype = None
        lib.oracle_query_f64.argtypes = [_f32p, _i64, _f32p, _i64p, _i64, _i64, _int, _f64p, _int]
        lib.oracle_kmedoids.restype = _int
        lib.oracle_kmedoids.argtypes = [_f64p, _i64, _i64, _i64p, _i64, _i64p, _i64p,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64),
                                        ctypes.POINTER(ctypes.c_double)]
        lib.oracle_cluster_cost.restype = ctypes.c_double
        lib.oracle_cluster_cost.argtypes = [_f64p, _i64, _i64p, _i64p]
        _lib = lib
        return lib


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _i64a(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def dtw(x, y, w: int = -1, strict: bool = False) -> float:
    """c_{n,m} in double for one pair (float inputs widened exactly)."""
    x, y = _f32(x), _f32(y)
    return float(_load().oracle_dtw_f64(x, len(x), y, len(y), int(w), int(strict)))


def dtw_f32_mirror(x, y, w: int = -1, strict: bool = False) -> np.float32:
    """The same recurrence in float with one fmaf per cell."""
    x, y = _f32(x), _f32(y)
    return np.float32(_load().oracle_dtw_f32_mirror(x, len(x), y, len(y), int(w), int(strict)))


def band_cells(n: int, m: int, w: int = -1, strict: bool = False) -> int:
    """Admissible cells of the band for lengths n, m (the DP work of one pair)."""
    return int(_load().oracle_band_cells(int(n), int(m), int(w), int(strict)))


def pairwise(values, offsets, w: int = -1, strict: bool = False, threads: int = 0) -> np.ndarray:
    """Full p x p distance matrix D in double."""
    values, offsets = _f32(values), _i64a(offsets)
    p = len(offsets) - 1
    D = np.empty((p, p), dtype=np.float64)
    _load().oracle_pairwise_f64(values, offsets, p, int(w), int(strict), D, int(threads))
    return D


def pairs(values, offsets, a, b, w: int = -1, strict: bool = False, threads: int = 0) -> np.ndarray:
    """d(a[t], b[t]) in double for a list of pairs."""
    values, offsets, a, b = _f32(values), _i64a(offsets), _i64a(a), _i64a(b)
    out = np.empty(len(a), dtype=np.float64)
    _load().oracle_pairs_f64(values, offsets, a, b, len(a), int(w), int(strict), out, int(threads))
    return out


def pairs_w(values, offsets, a, b, w, strict: bool = False, threads: int = 0) -> np.ndarray:
    """d(a[t], b[t]) in double, pair t with its own window w[t]."""
    values, offsets, a, b, w = _f32(values), _i64a(offsets), _i64a(a), _i64a(b), _i64a(w)
    out = np.empty(len(a), dtype=np.float64)
    _load().oracle_pairs_w_f64(values, offsets, a, b, w, len(a), int(strict), out, int(threads))
    return out


def pairs_f32_mirror(values, offsets, a, b, w: int = -1, strict: bool = False,
                     threads: int = 0) -> np.ndarray:
    """Float-mirror d(a[t], b[t]) for a list of pairs."""
    values, offsets, a, b = _f32(values), _i64a(offsets), _i64a(a), _i64a(b)
    out = np.empty(len(a), dtype=np.float32)
    _load().oracle_pairs_f32_mirror(values, offsets, a, b, len(a), int(w), int(strict), out,
                                    int(threads))
    return out


def pairs_w_f32_mirror(values, offsets, a, b, w, strict: bool = False,
                       threads: int = 0) -> np.ndarray:
    """Float-mirror d(a[t], b[t]), pair t with its own window w[t]."""
    values, offsets, a, b, w = _f32(values), _i64a(offsets), _i64a(a), _i64a(b), _i64a(w)
    out = np.empty(len(a), dtype=np.float32)
    _load().oracle_pairs_w_f32_mirror(values, offsets, a, b, w, len(a), int(strict), out,
                                      int(threads))
    return out


def query(q, values, offsets, w: int = -1, strict: bool = False, threads: int = 0) -> np.ndarray:
    """One row of D: DTW of q against every series of the set, in double."""
    q, values, offsets = _f32(q), _f32(values), _i64a(offsets)
    p = len(offsets) - 1
    out = np.empty(p, dtype=np.float64)
    _load().oracle_query_f64(q, len(q), values, offsets, p, int(w), int(strict), out, int(threads))
    return out


def kmedoids(D, k: int, init, max_iter: int = 100):
    """Alternate k-medoids in double on D.

    Returns dict(medoids, labels, cost, iters, min_margin); see dtw_oracle.c.
    """
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    p = D.shape[0]
    init = _i64a(init)
    med = np.empty(k, dtype=np.int64)
    lab = np.empty(p, dtype=np.int64)
    cost = ctypes.c_double()
    iters = ctypes.c_int64()
    margin = ctypes.c_double()
    rc = _load().oracle_kmedoids(D, p, int(k), init, int(max_iter), med, lab,
                                 ctypes.byref(cost), ctypes.byref(iters), ctypes.byref(margin))
    if rc != 0:
        raise MemoryError("oracle_kmedoids failed")
    return dict(medoids=med, labels=lab, cost=cost.value, iters=iters.value,
                min_margin=margin.value)


def cluster_cost(D, medoids, labels) -> float:
    """sum_j D[j, medoids[labels[j]]] in double."""
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    return float(_load().oracle_cluster_cost(D, D.shape[0], _i64a(medoids), _i64a(labels)))

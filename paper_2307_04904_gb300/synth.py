"""Seeded synthetic time-series sets (inputs only; none of the method's arithmetic).

The paper benchmarks on the UCR Time Series Archive, which is not available
here.  These generators make sets with the shapes the benchmarks need (number
of series, length, length mix) from a seed:

* ``random_walk_set`` -- cumulative sums of N(0, 1) steps;
* ``five_class_set``  -- five class generators (sine with 1..8 cycles and a
  random phase, square wave, sawtooth, random walk, Gaussian bump of width
  L/20 at a random centre), each circularly shifted by up to 15 % of its
  length and given N(0, 0.1) noise;
* ``ragged_lengths``  -- lengths drawn uniformly from a range;
* ``init_medoids``    -- k distinct starting medoids drawn by a Fisher-Yates
  shuffle driven by a splitmix64 stream of the seed.

Every series is z-normalised (mean 0, standard deviation 1 with the 1/L
convention).  A set is returned as ``(values, offsets)``: float32 values of all
series concatenated, and int64 offsets of length N+1 (series i is
``values[offsets[i]:offsets[i+1]]``).

This module is shared by the tests, the benchmark and the oracle-side checks;
it imports neither the oracle nor the CUDA binding.
"""

from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One splitmix64 step (Steele, Lea & Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def init_medoids(p: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices in [0, p): first k of a splitmix64-driven Fisher-Yates shuffle."""
    if not 1 <= k <= p:
        raise ValueError("need 1 <= k <= p")
    perm = list(range(p))
    state = seed & _MASK64
    for i in range(p - 1, 0, -1):
        state, r = splitmix64(state)
        j = r % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return np.array(perm[:k], dtype=np.int64)


def znorm(s: np.ndarray) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    mu = s.mean()
    sd = s.std()
    if sd == 0.0:
        return np.zeros_like(s, dtype=np.float32)
    return ((s - mu) / sd).astype(np.float32)


def _pack(series) -> tuple[np.ndarray, np.ndarray]:
    lens = np.array([len(s) for s in series], dtype=np.int64)
    offsets = np.zeros(len(series) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    values = np.concatenate(series).astype(np.float32) if series else np.zeros(0, np.float32)
    return np.ascontiguousarray(values), offsets


def random_walk(rng: np.random.Generator, L: int) -> np.ndarray:
    return znorm(np.cumsum(rng.standard_normal(L)))


def random_walk_set(N: int, L: int, seed: int = 0):
    """N z-normalised Gaussian random walks of length L."""
    rng = np.random.default_rng(seed)
    return _pack([random_walk(rng, L) for _ in range(N)])


CLASSES = ("sine", "square", "sawtooth", "random_walk", "bump")


def class_series(rng: np.random.Generator, cls: int, L: int) -> np.ndarray:
    """One series of class ``cls`` (index into CLASSES), shifted, noised, z-normalised."""
    t = np.arange(L, dtype=np.float64) / L
    name = CLASSES[cls % 5]
    if name in ("sine", "square", "sawtooth"):
        f = rng.uniform(1.0, 8.0)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        arg = 2.0 * np.pi * f * t + phase
        if name == "sine":
            s = np.sin(arg)
        elif name == "square":
            s = np.where(np.sin(arg) >= 0.0, 1.0, -1.0)
        else:
            u = arg / (2.0 * np.pi)
            s = 2.0 * (u - np.floor(u)) - 1.0
    elif name == "random_walk":
        s = np.cumsum(rng.standard_normal(L))
    else:
        centre = rng.uniform(0.0, L)
        sigma = L / 20.0
        s = np.exp(-0.5 * ((np.arange(L) - centre) / sigma) ** 2)
    shift = int(rng.integers(0, int(0.15 * L) + 1))
    s = np.roll(s, shift)
    s = s + rng.normal(0.0, 0.1, size=L)
    return znorm(s)


def five_class_set(N: int, L, seed: int = 1):
    """N series from the five class generators (series i has class i mod 5).

    ``L`` is either one length for every series or an array of N lengths.
    Returns (values, offsets, classes).
    """
    rng = np.random.default_rng(seed)
    lens = np.full(N, int(L), dtype=np.int64) if np.isscalar(L) else np.asarray(L, np.int64)
    series = [class_series(rng, i % 5, int(lens[i])) for i in range(N)]
    values, offsets = _pack(series)
    return values, offsets, np.arange(N, dtype=np.int64) % 5


def ragged_lengths(N: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """N lengths uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=N).astype(np.int64)


def integer_set(N: int, L, seed: int = 0, lo: int = -3, hi: int = 3):
    """Small-integer series: every DP sum is exact in float and double."""
    rng = np.random.default_rng(seed)
    lens = np.full(N, int(L), dtype=np.int64) if np.isscalar(L) else np.asarray(L, np.int64)
    series = [rng.integers(lo, hi + 1, size=int(l)).astype(np.float32) for l in lens]
    return _pack(series)

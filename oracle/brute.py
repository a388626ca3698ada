"""Brute-force references for tiny inputs (test infrastructure only).

These enumerate what the dynamic programme and the k-medoids sweeps only
search, so they pin the oracle in ``dtw_oracle.c`` to something other than
itself:

* ``dtw_by_paths`` -- the DTW distance as the minimum, over every admissible
  warping path, of the summed pointwise costs.  A path starts at (1, 1), ends
  at (n, m) and moves by (1, 0), (0, 1) or (1, 1): the three constraints of the
  paper's problem statement (first and last elements matched, monotone,
  continuous).  The pointwise cost is the squared difference of the equation
  for c_{i,j}; the band is |i - j| <= w with the same readings as the oracle
  (w < 0: none; default widens to |n - m|; strict keeps w).
* ``kmedoids_optimum`` -- the global optimum of the paper's MIP clustering
  objective, min sum_ij D_ij A_ij under its three constraints, found by trying
  every set of k centroids (each series then joins its nearest centroid).
* ``labels_to_A`` / ``mip_objective`` -- the binary matrix A of the MIP
  formulation (A_ij = 1 iff series j belongs to the cluster whose centroid is
  series i) and its objective.

Pure Python loops: use only for n, m <= 7 and p <= 12.
"""

from __future__ import annotations

import itertools
import math


def _band(n: int, m: int, w: int, strict: bool) -> int:
    if w < 0:
        return -1
    if strict:
        return w
    return max(w, abs(n - m))


def warping_paths(n: int, m: int, w: int = -1, strict: bool = False):
    """Yield every admissible warping path as a tuple of 1-based (i, j) cells."""
    band = _band(n, m, w, strict)

    def ok(i, j):
        return band < 0 or abs(i - j) <= band

    if not ok(1, 1) or not ok(n, m):
        return

    def rec(path):
        i, j = path[-1]
        if (i, j) == (n, m):
            yield tuple(path)
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            a, b = i + di, j + dj
            if a <= n and b <= m and ok(a, b):
                path.append((a, b))
                yield from rec(path)
                path.pop()

    yield from rec([(1, 1)])


def dtw_by_paths(x, y, w: int = -1, strict: bool = False) -> float:
    """Minimum over all admissible warping paths of sum (x_i - y_j)^2 (float64)."""
    n, m = len(x), len(y)
    best = math.inf
    for path in warping_paths(n, m, w, strict):
        s = 0.0
        for i, j in path:
            d = float(x[i - 1]) - float(y[j - 1])
            s += d * d
        best = min(best, s)
    return best


def delannoy(n: int, m: int) -> int:
    """Number of unconstrained warping paths from (1,1) to (n,m) (Delannoy number)."""
    a, b = n - 1, m - 1
    return sum(math.comb(a, t) * math.comb(b, t) * 2**t for t in range(min(a, b) + 1))


def labels_to_A(labels, medoids):
    """The MIP matrix A: A[i][j] = 1 iff series j is in the cluster of centroid i."""
    p = len(labels)
    A = [[0] * p for _ in range(p)]
    for j, c in enumerate(labels):
        A[medoids[c]][j] = 1
    return A


def check_A_constraints(A, k: int) -> bool:
    """The three MIP constraints: k centroids, one cluster per series, A_ij <= A_ii."""
    p = len(A)
    if sum(A[i][i] for i in range(p)) != k:
        return False
    for j in range(p):
        if sum(A[i][j] for i in range(p)) != 1:
            return False
    for i in range(p):
        for j in range(p):
            if A[i][j] > A[i][i]:
                return False
    return True


def mip_objective(D, A) -> float:
    """sum_i sum_j D_ij A_ij."""
    p = len(A)
    return sum(float(D[i][j]) * A[i][j] for i in range(p) for j in range(p))


def kmedoids_optimum(D, k: int):
    """Global optimum of the MIP objective by enumerating every k-subset of centroids.

    Returns (cost, medoids) with medoids the lexicographically first optimal set.
    """
    p = len(D)
    best, best_set = math.inf, None
    for S in itertools.combinations(range(p), k):
        cost = 0.0
        for j in range(p):
            cost += min(float(D[j][c]) for c in S)
        if cost < best:
            best, best_set = cost, S
    return best, list(best_set)

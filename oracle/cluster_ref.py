"""Float64 reference of the cluster-quality scores (test infrastructure only).

The paper's software reports a silhouette score and an elbow score to help
choose k (Overview, item 6) without defining them.  Read here as:

* silhouette (Rousseeuw 1987) over the clustering's own distances D:
  a(i) = mean of D[i][j] over the other members of i's cluster,
  b(i) = least mean of D[i][j] over the members of another non-empty cluster,
  s(i) = (b - a) / max(a, b), with s(i) = 0 for a singleton cluster or when
  max(a, b) = 0; the score is the mean of s(i);
* elbow: the k-medoids cost as a function of k; the elbow is the k in
  [2, kmax - 1] with the largest second difference
  cost(k - 1) - 2 cost(k) + cost(k + 1) (the smallest such k on ties).

Plain loops over numpy arrays, independent of the CUDA path.
"""

from __future__ import annotations

import numpy as np


def silhouette(D, labels):
    """(s [n] float64, mean) for a symmetric D and integer labels."""
    D = np.asarray(D, dtype=np.float64)
    labels = np.asarray(labels)
    n = D.shape[0]
    clusters = sorted(set(labels.tolist()))
    if len(clusters) < 2:
        raise ValueError("the silhouette needs at least two non-empty clusters")
    members = {c: [j for j in range(n) if labels[j] == c] for c in clusters}
    s = np.zeros(n)
    for i in range(n):
        own = members[labels[i]]
        if len(own) == 1:
            continue
        a = sum(D[i, j] for j in own if j != i) / (len(own) - 1)
        b = min(sum(D[i, j] for j in members[c]) / len(members[c])
                for c in clusters if c != labels[i])
        m = max(a, b)
        s[i] = (b - a) / m if m > 0 else 0.0
    return s, float(s.mean())


def elbow(costs):
    """The elbow k of a cost curve given as {k: cost} for consecutive k."""
    ks = sorted(costs)
    best, best_k = -np.inf, None
    for k in ks[1:-1]:
        d2 = costs[k - 1] - 2 * costs[k] + costs[k + 1]
        if d2 > best:
            best, best_k = d2, k
    return best_k


# --------------------------------------------------------------------- PAM
#
# PAM (Kaufman & Rousseeuw 1990) on D: BUILD picks the first medoid with the
# least row sum, then k - 1 times the point that lowers the total deviation
# TD = sum_j min_c D[M_c][j] the most (ties to the smaller index).  SWAP
# passes then apply, one at a time, the swap (remove medoid i, add point o)
# with the most negative change in TD, computed for all k medoids of a
# candidate o in one pass over the points (Schubert & Rousseeuw 2019, FastPAM1):
# with d1, d2 the nearest and second-nearest medoid distances and n1 the
# nearest medoid of point j,
#   delta(o, i) = sum_j min(0, D[o][j] - d1(j))
#                 + sum_{j: n1(j) = i} [min(D[o][j], d2(j)) - d1(j) - min(0, D[o][j] - d1(j))]
# Ties: the least delta, then the smaller o, then the smaller i; the pass
# stops when the least delta is not negative.


def nearest(D, M):
    """d1, n1 (ties to the smaller position in M), d2 for every point."""
    D = np.asarray(D, dtype=np.float64)
    R = D[np.asarray(M)]  # k x n
    n1 = np.argmin(R, axis=0)
    d1 = R[n1, np.arange(R.shape[1])]
    if len(M) > 1:
        R2 = R.copy()
        R2[n1, np.arange(R.shape[1])] = np.inf
        d2 = R2.min(0)
    else:
        d2 = np.full(R.shape[1], np.inf)
    return d1, n1, d2


def swap_deltas(D, M):
    """delta[o][i] for every non-medoid o (inf for medoids), by the one-pass formula."""
    D = np.asarray(D, dtype=np.float64)
    n, k = D.shape[0], len(M)
    d1, n1, d2 = nearest(D, M)
    out = np.full((n, k), np.inf)
    for o in range(n):
        if o in M:
            continue
        t1 = np.zeros(k)
        t2 = np.zeros(k)
        for j in range(n):
            c = n1[j]
            t1[c] += min(0.0, D[o, j] - d1[j])
            t2[c] += min(D[o, j], d2[j]) - d1[j]
        S = t1.sum()
        for i in range(k):
            out[o, i] = S + t2[i] - t1[i]
    return out


def _rel_gap(vals):
    """Relative gap between the least and the next larger finite value (inf if none)."""
    v = np.sort(np.asarray(vals, dtype=np.float64))
    v = v[np.isfinite(v)]
    if len(v) < 2 or v[0] <= 0:
        return np.inf
    larger = v[v > v[0]]
    return (larger[0] - v[0]) / v[0] if len(larger) else np.inf


def pam_build(D, k, with_gap=False):
    """BUILD medoids; with_gap also returns the smallest relative gap between the
    chosen and the runner-up value met in any step (0 on an exact tie)."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    sums = D.sum(1)
    M = [int(np.argmin(sums))]
    gap = _rel_gap(sums) if np.count_nonzero(sums == sums.min()) == 1 else 0.0
    d1 = D[M[0]].copy()
    for _ in range(k - 1):
        gains = [np.minimum(D[o], d1).sum() if o not in M else np.inf for o in range(n)]
        o = int(np.argmin(gains))
        g = np.asarray(gains)
        gap = min(gap, _rel_gap(g) if np.count_nonzero(g == g[o]) == 1 else 0.0)
        M.append(o)
        d1 = np.minimum(d1, D[o])
    return (M, gap) if with_gap else M


def pam(D, k, init=None, max_swaps=1000):
    """Returns dict(medoids, labels, cost, swaps, min_gap, build_gap): min_gap is
    the smallest relative gap between the chosen and the runner-up delta, or
    between the least delta and 0, met in any pass; build_gap the same for the
    BUILD choices (inf when the medoids were given)."""
    D = np.asarray(D, dtype=np.float64)
    if init is None:
        M, build_gap = pam_build(D, k, with_gap=True)
    else:
        M, build_gap = [int(i) for i in init], np.inf
    swaps, gap = 0, np.inf
    while swaps < max_swaps:
        d1, _, _ = nearest(D, M)
        td = d1.sum()
        delta = swap_deltas(D, M)
        flat = [(delta[o, i], o, i) for o in range(D.shape[0]) for i in range(k)
                if np.isfinite(delta[o, i])]
        if not flat:
            break
        flat.sort()
        best = flat[0]
        scale = td if td > 0 else 1.0
        gap = min(gap, abs(best[0]) / scale)
        if len(flat) > 1 and flat[1][0] != best[0]:
            gap = min(gap, (flat[1][0] - best[0]) / scale)
        if best[0] >= 0:
            break
        M[best[2]] = best[1]
        swaps += 1
    d1, n1, _ = nearest(D, M)
    labels = n1.copy()
    for c, m in enumerate(M):
        labels[m] = c
    return dict(medoids=np.asarray(M, dtype=np.int64), labels=labels, cost=float(d1.sum()),
                swaps=swaps, min_gap=gap, build_gap=build_gap)

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

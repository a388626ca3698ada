"""Cluster-quality reporting over the DTW matrix (include/dtwgb_cluster.h).

* :func:`silhouette` -- the silhouette of a clustering (``kmedoids_silhouette``).
* :func:`elbow` -- the elbow curve: ``kmedoids_fit`` for k = 1 .. kmax from
  seeded initial medoids, and the elbow k, the one with the largest second
  difference cost(k - 1) - 2 cost(k) + cost(k + 1) (the smallest on ties).

Both only marshal arguments; the sweeps and reductions run in the library.
"""

from __future__ import annotations

import torch

from . import api, synth


def silhouette(D: torch.Tensor, labels: torch.Tensor, k: int, stream=None):
    """(per-point s on the GPU, mean silhouette)."""
    return api.kmedoids_silhouette(D, labels, k, stream=stream)


def elbow(D: torch.Tensor, kmax: int, seed: int = 0, max_iter: int = 100, stream=None) -> dict:
    """Cost curve {k: cost} for k = 1 .. kmax, the elbow k and the silhouette of each k >= 2."""
    n = D.shape[0]
    costs, sil = {}, {}
    kmax = min(kmax, n)
    # the seeded medoids for k are the first k of one shuffle, so one draw serves every k
    order = torch.as_tensor(synth.init_medoids(n, kmax, seed), dtype=torch.int32, device=D.device)
    for k in range(1, kmax + 1):
        _, labels, cost, _ = api.kmedoids_fit(D, k, order[:k].contiguous(), max_iter, stream=stream)
        costs[k] = cost
        if 2 <= k < n:
            sil[k] = api.kmedoids_silhouette(D, labels, k, stream=stream)[1]
    best, best_k = None, None
    for k in sorted(costs)[1:-1]:
        d2 = costs[k - 1] - 2 * costs[k] + costs[k + 1]
        if best is None or d2 > best:
            best, best_k = d2, k
    return {"costs": costs, "elbow": best_k, "silhouette": sil}

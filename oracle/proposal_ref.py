"""Float64 reference of the proposal layer (test infrastructure only).

Two procedures the project adds on top of the paper's k-medoids (section
"Mathematical background", last paragraph; the paper notes that k-medoids
needs only some of the DTW distances, "Performance comparison"):

* ``kmeanspp``  k-means++ seeding (Arthur & Vassilvitskii 2007) over
  embedding vectors: the first centre is index ``splitmix64(seed) mod n``; each
  next centre is the smallest index j whose running sum of D2 (squared
  distance to the nearest chosen centre) exceeds ``u * sum(D2)``, with
  ``u = (next splitmix64 output >> 11) * 2**-53``.  If every D2 is zero the
  smallest index not chosen yet is taken.
* ``kmeans``  Lloyd's k-means over the embeddings from ``restarts`` k-means++
  seedings (seeds ``seed + r``), at most ``iters`` assignment steps each
  (stopping when no label changes), the restart of least inertia (the first on
  ties); the proposal of each cluster is its member nearest to the centroid,
  an empty cluster takes the nearest point not taken yet.
* ``lazy_kmedoids``  the alternate k-medoids of ``oracle.kmedoids`` (same
  assign, update and tie rules) in which the update evaluates, per cluster,
  only a candidate list: the current medoid, then the ``candidates - 1`` other
  members nearest to the cluster's embedding centroid in increasing
  (squared distance, index) order, then (with ``screen_sample`` s > 0) the
  ``screen_keep`` members of least DTW sum to the sample
  ``C[floor(q |C| / s)]``, q < min(s, |C|), of the cluster's index-ordered
  members.  Without proposals and screening every member is a candidate,
  which is exactly ``oracle.kmedoids``.

Both are plain loops over numpy arrays, independent of the CUDA path.  The
random stream is splitmix64 (Steele, Lea & Flood 2014), written here from its
published definition.  Each function also reports the smallest relative gap met at a decision
taken on floating-point values, so that a test knows when a float32
implementation may legitimately decide otherwise.
"""

from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One splitmix64 step: add the golden gamma, then mix; returns (state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def kmeanspp(emb, k: int, seed: int):
    """Returns (centres int64[k], min relative gap between u*total and a running sum)."""
    E = np.asarray(emb, dtype=np.float64)
    n = E.shape[0]
    if not 1 <= k <= n:
        raise ValueError("need 1 <= k <= n")
    state, out = splitmix64(seed)
    centres = [out % n]
    D2 = None
    gap = np.inf
    for _ in range(1, k):
        d = ((E - E[centres[-1]]) ** 2).sum(1)
        D2 = d if D2 is None else np.minimum(D2, d)
        state, out = splitmix64(state)
        u = (out >> 11) * 2.0 ** -53
        total = float(D2.sum())
        pick = -1
        if total > 0:
            thr = u * total
            run = np.cumsum(D2)
            # smallest j with run[j] > thr and D2[j] > 0
            idx = np.nonzero((run > thr) & (D2 > 0))[0]
            pick = int(idx[0]) if idx.size else int(np.nonzero(D2 > 0)[0][-1])
            gap = min(gap, float(np.min(np.abs(run - thr))) / total)
        if pick < 0:
            pick = next(j for j in range(n) if j not in centres)
        centres.append(pick)
    return np.asarray(centres, dtype=np.int64), gap


def _sqdist(E, C):
    return ((E[:, None, :] - C[None, :, :]) ** 2).sum(-1)


def _assign(E, C):
    """labels (ties to the smallest centre), distances, min relative decision gap."""
    d = _sqdist(E, C)
    lab = d.argmin(1)  # first minimum: the smallest index on ties
    gap = np.inf
    if C.shape[0] > 1:
        s = np.sort(d, 1)
        gap = float(np.min((s[:, 1] - s[:, 0]) / np.where(s[:, 1] > 0, s[:, 1], 1.0)))
    return lab, d[np.arange(len(E)), lab], gap


def kmeans(emb, k: int, restarts: int, iters: int, seed: int):
    """Returns dict(medoids, inertia, centroids, min_gap): min_gap is the smallest
    relative gap met at an assignment, a restart choice or a nearest-member choice."""
    E = np.asarray(emb, dtype=np.float64)
    n = E.shape[0]
    gap = np.inf
    results = []
    for r in range(restarts):
        seeds, g0 = kmeanspp(E, k, seed + r)
        gap = min(gap, g0)
        C = E[seeds].copy()
        labels = np.full(n, -1)
        for _ in range(iters):
            new, _, g = _assign(E, C)
            gap = min(gap, g)
            if np.array_equal(new, labels):
                break
            labels = new
            for c in range(k):
                if np.any(labels == c):
                    C[c] = E[labels == c].mean(0)
        lab, dist, g = _assign(E, C)
        gap = min(gap, g)
        results.append((float(dist.sum()), C, lab, dist))
    inertias = [x[0] for x in results]
    b = int(np.argmin(inertias))  # first minimum
    if restarts > 1:
        others = [v for i, v in enumerate(inertias) if i != b]
        gap = min(gap, (min(others) - inertias[b]) / max(min(others), 1e-300))
    inertia, C, lab, dist = results[b]
    med = []
    for c in range(k):
        mem = np.nonzero(lab == c)[0]
        if mem.size == 0:
            med.append(-1)
            continue
        order = sorted(mem.tolist(), key=lambda j: (dist[j], j))
        if len(order) > 1:
            d0, d1 = dist[order[0]], dist[order[1]]
            gap = min(gap, (d1 - d0) / (d1 if d1 > 0 else 1.0))
        med.append(order[0])
    for c in range(k):
        if med[c] >= 0:
            continue
        d = ((E - C[c]) ** 2).sum(1)
        free = [j for j in range(n) if j not in med]
        med[c] = min(free, key=lambda j: (d[j], j))
    return dict(medoids=np.asarray(med, dtype=np.int64), inertia=inertia, centroids=C,
                min_gap=gap)


def _rel_gap(best, second):
    scale = abs(second) if second != 0 else 1.0
    return (second - best) / scale


def candidate_list(members, medoid, emb, ncand):
    """The medoid, then the ncand-1 other members nearest to the centroid of the
    members' embeddings, by (squared distance, index).  Returns (list, gap)."""
    E = np.asarray(emb, dtype=np.float64)
    cent = E[members].mean(0)
    others = [j for j in members if j != medoid]
    d = {j: float(((E[j] - cent) ** 2).sum()) for j in others}
    order = sorted(others, key=lambda j: (d[j], j))
    chosen = [medoid] + order[:ncand - 1]
    gap = np.inf
    if 0 < ncand - 1 < len(order):  # the boundary between the last chosen and the first left out
        a, b = d[order[ncand - 2]], d[order[ncand - 1]]
        gap = (b - a) / (b if b > 0 else 1.0)
    return chosen, gap


def lazy_kmedoids(D, emb, k: int, init, candidates=None, max_iter: int = 100,
                  screen_sample: int = 0, screen_keep: int = 0):
    """Lazy alternate k-medoids on the float64 matrix D (entries looked up, never all used).

    Returns dict(medoids, labels, cost, iters, pairs, min_margin, min_cand_gap);
    ``pairs`` counts the DTW values the procedure needs: k*n per assignment,
    |C_c| * min(s, |C_c|) per cluster for screening and ncand_c * |C_c| per
    cluster and update.
    """
    propose = emb is not None and candidates is not None and candidates > 0
    screen = screen_sample > 0
    every = not propose and not screen
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    M = [int(i) for i in init]
    pairs = 0
    margin = np.inf
    cand_gap = np.inf

    def assign(M):
        nonlocal pairs, margin
        labels = np.empty(n, dtype=np.int64)
        for j in range(n):
            if j in M:
                labels[j] = M.index(j)
                continue
            row = [D[M[c], j] for c in range(k)]
            best = min(range(k), key=lambda c: (row[c], c))
            labels[j] = best
            if k > 1:
                second = min(row[c] for c in range(k) if c != best)
                margin = min(margin, _rel_gap(row[best], second))
        pairs += k * n
        return labels

    iters = 0
    converged = False
    labels = None
    for it in range(1, max_iter + 1):
        labels = assign(M)
        Mn = list(M)
        changed = False
        for c in range(k):
            members = [j for j in range(n) if labels[j] == c]
            m = len(members)
            if every:
                cand = members
            else:
                if propose:
                    cand, g = candidate_list(members, M[c], emb, min(candidates, m))
                    cand_gap = min(cand_gap, g)
                else:
                    cand = [M[c]]
                if screen:
                    s = min(screen_sample, m)
                    sample = [members[q * m // s] for q in range(s)]
                    score = {}
                    for i in members:
                        acc = 0.0
                        for j in sample:  # in order: the float64 sum is reproducible
                            acc += D[i, j]
                        score[i] = acc
                    pairs += m * s
                    cand = list(cand) + sorted(members, key=lambda i: (score[i], i))[:min(screen_keep, m)]
            S = [sum(D[i, j] for j in members) for i in cand]
            pairs += len(cand) * len(members)
            best = min(range(len(cand)), key=lambda q: (S[q], cand[q]))
            cur = S[cand.index(M[c])]
            chosen = M[c] if cur == S[best] else cand[best]
            if len(cand) > 1:
                second = min(S[q] for q in range(len(cand)) if q != best)
                margin = min(margin, _rel_gap(S[best], second))
            Mn[c] = chosen
            changed |= chosen != M[c]
        iters = it
        if not changed:
            converged = True
            break
        M = Mn
    if not converged:
        labels = assign(M)
    cost = float(sum(D[M[labels[j]], j] for j in range(n)))
    return dict(medoids=np.asarray(M, dtype=np.int64), labels=labels, cost=cost, iters=iters,
                pairs=pairs, min_margin=margin, min_cand_gap=cand_gap)

"""k-medoids with learned proposals: the encoder of ``include/dtwgb_encoder.h``
trained on exact DTW, k-means seeding in its embedding space, and the lazy
k-medoids of ``include/dtwgb_proposal.h`` whose every accepted assignment,
medoid and cost is exact DTW.

Pipeline of :func:`fit` (series of one length T, a multiple of 64):

1. exact DTW matrix of the first ``train_series`` series (``dtw_pairwise``);
2. regression targets sqrt(D) / mean sqrt(D) (``dtw_encoder_targets``);
3. ``steps`` full-batch Adam steps of the encoder, one CUDA graph replayed;
4. embeddings of every series (``dtw_encoder_embed``, batches of rows);
5. initial medoids from k-means over the embeddings (``proposal_kmeans``, or
   the k-means++ seeds alone with ``seeding="kmeanspp"``);
6. ``kmedoids_lazy_fit``: per cluster and sweep the current medoid, the
   ``candidates - 1`` members nearest to the embedding centroid and the
   ``screen_keep`` members of least exact DTW sum to a ``screen_sample``-member
   sample of the cluster, judged by exact DTW sums over the whole cluster;
7. with ``polish``, ``kmedoids_lazy_fit`` again from that answer with every
   member a candidate: sweeps of the plain alternate k-medoids (on exact DTW
   computed within clusters only) until no medoid moves, so the answer is a
   fixed point of the plain method.

Steps 5-7 run for up to ``rounds`` k-means seeds (``seed``, ``seed + 1``, ...)
and keep the least exact cost; with ``target_cost`` they stop at the first
round whose cost is within 1e-5 (relative) of it.

With ``embed=False`` the encoder is left out (steps 1-5): every round starts
from ``init_medoids(n, k, seed + round)`` and the lazy fit's candidates are the
current medoid and the screened members only -- the pipeline without learned
proposals, for comparison.  ``steps=0`` keeps the encoder untrained (its
seeded initial parameters).

:func:`plain_fit` is the method without proposals: the full DTW matrix and
the alternate k-medoids over it (``dtw_pairwise`` + ``kmedoids_fit``).  Both
only marshal arguments; every step runs in the CUDA library.
"""

from __future__ import annotations

import torch

from . import api

STAGES = ("targets", "train", "embed", "proposals")
REACH_RTOL = 1e-5


def _equal_length(offsets: torch.Tensor) -> tuple[int, int]:
    o = offsets.cpu()
    n = o.numel() - 1
    T = int(o[1] - o[0])
    if not torch.equal(o - o[0], torch.arange(n + 1, dtype=o.dtype) * T):
        raise ValueError("learned proposals need series of one length")
    if T % 64 or not 64 <= T <= 832:
        raise ValueError(f"series length {T} must be a multiple of 64 in [64, 832]")
    return n, T


def fit(values: torch.Tensor, offsets: torch.Tensor, window: int, k: int, *,
        train_series: int = 633, steps: int = 20, lr: float = 3e-3, candidates: int = 8,
        screen_sample: int = 32, screen_keep: int = 8, seed: int = 0, seeding: str = "kmeans",
        restarts: int = 4, kmeans_iters: int = 25, polish: bool = False, rounds: int = 1,
        target_cost: float | None = None, embed_batch: int = 4096, max_iter: int = 100,
        encoder: api.Encoder | None = None, embed: bool = True, stream=None) -> dict:
    """Learned-proposal k-medoids; returns medoids, labels, cost, iters, pairs (DTW pairs
    evaluated), the rounds run, the per-step training losses, the embeddings and the GPU
    time of each stage in ms."""
    if not embed:
        return _fit_without_embedding(values, offsets, window, k, screen_sample=screen_sample,
                                      screen_keep=screen_keep, seed=seed, rounds=rounds,
                                      target_cost=target_cost, max_iter=max_iter, stream=stream)
    n, T = _equal_length(offsets)
    S = min(train_series, n)
    st = stream if stream is not None else torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
    x = values.view(n, T)
    B = min(embed_batch, n)
    enc = encoder if encoder is not None else api.Encoder(T, max(S, B, 2))
    if encoder is None:
        enc.init_params(seed)
    with torch.cuda.stream(st):
        ev[0].record(st)
        D = api.dtw_pairwise(values[:S * T], offsets[:S + 1], window, stream=st)
        tgt = api.Encoder.targets(D, stream=st)
        ev[1].record(st)
        losses = enc.train(x[:S], tgt, lr, steps, stream=st) if steps > 0 else None
        ev[2].record(st)
        emb = torch.empty((n, 64), dtype=torch.float32, device=values.device)
        for b0 in range(0, n, B):
            b1 = min(n, b0 + B)
            enc.embed(x[b0:b1], out=emb[b0:b1], stream=st)
        ev[3].record(st)
        enc.check()
        best = None
        pairs = 0
        for r in range(rounds):
            if seeding == "kmeans":
                init, _ = api.proposal_kmeans(emb, k, seed + r, restarts=restarts,
                                              iters=kmeans_iters, stream=st)
            elif seeding == "kmeanspp":
                init = api.proposal_kmeanspp(emb, k, seed + r, stream=st)
            else:
                raise ValueError(f"unknown seeding {seeding!r}")
            med, lab, cost, iters, p1 = api.kmedoids_lazy_fit(
                values, offsets, window, k, init, emb=emb, candidates=candidates,
                screen_sample=screen_sample, screen_keep=screen_keep, max_iter=max_iter,
                stream=st)
            pairs += p1
            lazy_cost, polish_iters = cost, 0
            if polish:
                med, lab, cost, polish_iters, p2 = api.kmedoids_lazy_fit(
                    values, offsets, window, k, med, max_iter=max_iter, stream=st)
                pairs += p2
            if best is None or cost < best["cost"]:
                best = dict(medoids=med, labels=lab, cost=cost, iters=iters, init=init,
                            lazy_cost=lazy_cost, polish_iters=polish_iters, round=r)
            if target_cost is not None and best["cost"] <= target_cost * (1 + REACH_RTOL):
                break
        ev[4].record(st)
    st.synchronize()
    times = {s: ev[i].elapsed_time(ev[i + 1]) for i, s in enumerate(STAGES)}
    out = dict(best, pairs=pairs, rounds=r + 1, embeddings=emb,
               losses=losses.cpu() if losses is not None else None, times_ms=times,
               train_pairs=S * (S - 1) // 2)
    if encoder is None:
        enc.close()
    return out


def _fit_without_embedding(values, offsets, window, k, *, screen_sample, screen_keep, seed,
                           rounds, target_cost, max_iter, stream):
    """The lazy fit from seeded random medoids with screening only (no encoder)."""
    from . import synth

    n = offsets.numel() - 1
    st = stream if stream is not None else torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    best, pairs = None, 0
    with torch.cuda.stream(st):
        ev[0].record(st)
        for r in range(rounds):
            init = torch.as_tensor(synth.init_medoids(n, k, seed + r), dtype=torch.int32,
                                   device=values.device)
            med, lab, cost, iters, p1 = api.kmedoids_lazy_fit(
                values, offsets, window, k, init, screen_sample=screen_sample,
                screen_keep=screen_keep, max_iter=max_iter, stream=st)
            pairs += p1
            if best is None or cost < best["cost"]:
                best = dict(medoids=med, labels=lab, cost=cost, iters=iters, init=init,
                            lazy_cost=cost, polish_iters=0, round=r)
            if target_cost is not None and best["cost"] <= target_cost * (1 + REACH_RTOL):
                break
        ev[1].record(st)
    st.synchronize()
    times = {s: 0.0 for s in STAGES}
    times["proposals"] = ev[0].elapsed_time(ev[1])
    return dict(best, pairs=pairs, rounds=r + 1, embeddings=None, losses=None, times_ms=times,
                train_pairs=0)


def plain_fit(values: torch.Tensor, offsets: torch.Tensor, window: int, k: int,
              init_medoids: torch.Tensor, *, max_iter: int = 100, stream=None) -> dict:
    """The method without proposals: full DTW matrix, then alternate k-medoids."""
    st = stream if stream is not None else torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(st):
        ev[0].record(st)
        D = api.dtw_pairwise(values, offsets, window, stream=st)
        ev[1].record(st)
        med, lab, cost, iters = api.kmedoids_fit(D, k, init_medoids, max_iter, stream=st)
        ev[2].record(st)
    st.synchronize()
    del D
    return dict(medoids=med, labels=lab, cost=cost, iters=iters,
                times_ms={"matrix": ev[0].elapsed_time(ev[1]),
                          "kmedoids": ev[1].elapsed_time(ev[2])})

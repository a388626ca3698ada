"""k-medoids with learned proposals: the encoder of ``include/dtwgb_encoder.h``
trained on exact DTW, k-means++ seeding in its embedding space, and the lazy
k-medoids of ``include/dtwgb_proposal.h`` whose every accepted assignment,
medoid and cost is exact DTW.

Pipeline of :func:`fit` (series of one length T, a multiple of 64):

1. exact DTW matrix of the first ``train_series`` series (``dtw_pairwise``);
2. regression targets sqrt(D) / mean sqrt(D) (``dtw_encoder_targets``);
3. ``steps`` full-batch Adam steps of the encoder, one CUDA graph replayed;
4. embeddings of every series (``dtw_encoder_embed``, batches of rows);
5. initial medoids by k-means++ over the embeddings (``proposal_kmeanspp``);
6. ``kmedoids_lazy_fit`` with ``candidates`` proposals per cluster and sweep.

:func:`plain_fit` is the method without proposals: the full DTW matrix and
the alternate k-medoids over it (``dtw_pairwise`` + ``kmedoids_fit``).  Both
only marshal arguments; every step runs in the CUDA library.
"""

from __future__ import annotations

import torch

from . import api

STAGES = ("targets", "train", "embed", "seed", "lazy")


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
        train_series: int = 633, steps: int = 200, lr: float = 2e-3, candidates: int = 16,
        seed: int = 0, embed_batch: int = 4096, max_iter: int = 100,
        encoder: api.Encoder | None = None, stream=None) -> dict:
    """Learned-proposal k-medoids; returns medoids, labels, cost, iters, pairs,
    the per-step training losses and the GPU time of each stage in ms."""
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
        init = api.proposal_kmeanspp(emb, k, seed, stream=st)
        ev[4].record(st)
        med, lab, cost, iters, pairs = api.kmedoids_lazy_fit(
            values, offsets, window, k, init, emb=emb, candidates=candidates,
            max_iter=max_iter, stream=st)
        ev[5].record(st)
    st.synchronize()
    times = {s: ev[i].elapsed_time(ev[i + 1]) for i, s in enumerate(STAGES)}
    out = dict(medoids=med, labels=lab, cost=cost, iters=iters, pairs=pairs, init=init,
               embeddings=emb, losses=losses.cpu() if losses is not None else None,
               times_ms=times, train_pairs=S * (S - 1) // 2)
    if encoder is None:
        enc.close()
    return out


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

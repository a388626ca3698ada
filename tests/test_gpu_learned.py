"""What the trained proposal encoder gains on the learned-proposal workload.

The workload: 20000 seeded five-class series of length 256, band w = 25, k = 10;
the encoder is trained on the exact DTW of the first 633 series (200,028 pairs).
The same pipeline runs three ways on the same seeds: with the trained encoder,
with the encoder left at its seeded initial parameters, and without embeddings
(seeded random medoids, screened candidates only).  Plain k-medoids (full DTW
matrix, alternate k-medoids) sets the cost each leg must reach.

What is asserted is what holds robustly:
  * training makes embedding distances follow DTW: the Spearman correlation
    between embedding distance and sqrt(DTW) over 20000 random pairs rises from
    about 0.15 (random features) to about 0.5;
  * every leg's labels are the exact-DTW nearest medoids and its cost is the
    exact DTW cost of that clustering (float32 DTW values summed in float64);
  * the learned path reaches the plain cost in less wall time than plain
    k-medoids, in the median over the seeds.
Whether training makes the pipeline faster than the untrained encoder is not
asserted: on this workload it does not, in the median (the measured legs are
in the benchmark's `--workload learned` line).
"""

import time

import numpy as np
import pytest
import torch

from paper_2307_04904_gb300 import api, learned, synth

pytestmark = pytest.mark.gpu

N, T, W, K = 20000, 256, 25, 10


@pytest.fixture(scope="module")
def c3():
    values, offsets, _ = synth.five_class_set(N, T, seed=3)
    return torch.from_numpy(values).cuda(), torch.from_numpy(offsets).cuda()


def _spearman(a, b):
    def rank(x):
        r = np.empty(len(x))
        r[np.argsort(x, kind="stable")] = np.arange(len(x))
        return r

    return float(np.corrcoef(rank(a), rank(b))[0, 1])


def _rank_correlation(emb, v, o, seed=5, pairs=20000):
    rng = np.random.default_rng(seed)
    pa = torch.as_tensor(rng.integers(0, N, pairs), dtype=torch.int32).cuda()
    pb = torch.as_tensor(rng.integers(0, N, pairs), dtype=torch.int32).cuda()
    d = api.dtw_pairs(v, o, pa, pb, W).double().cpu().numpy()
    e = emb.double()
    de = (e[pa.long()] - e[pb.long()]).norm(dim=1).cpu().numpy()
    return _spearman(de, np.sqrt(d))


def test_training_makes_embedding_distances_follow_dtw(c3):
    v, o = c3
    trained = learned.fit(v, o, W, K, seed=0)
    untrained = learned.fit(v, o, W, K, seed=0, steps=0)
    rho_t = _rank_correlation(trained["embeddings"], v, o)
    rho_u = _rank_correlation(untrained["embeddings"], v, o)
    assert rho_t >= 0.35, rho_t
    assert rho_t - rho_u >= 0.2, (rho_t, rho_u)
    losses = trained["losses"].numpy()
    assert losses[-1] < 0.6 * losses[0]  # the regression loss falls over the 20 steps


def _check_exact(v, o, r):
    """Labels are the exact-DTW nearest medoids (ties to the smaller cluster, a medoid
    labels itself) and the cost is the exact DTW cost of the clustering."""
    med = r["medoids"].long()
    lab = r["labels"].cpu().numpy()
    pts = torch.arange(N, dtype=torch.int32).cuda()
    dist = torch.stack([api.dtw_pairs(v, o, pts, torch.full((N,), int(m), dtype=torch.int32,
                                                                device="cuda"), W)
                        for m in med.tolist()], 1).cpu().numpy()  # [N][K], float32 DTW
    want = np.argmin(dist, axis=1)  # first minimum: ties to the smaller cluster index
    want[med.cpu().numpy()] = np.arange(K)
    assert np.array_equal(lab, want)
    cost = dist[np.arange(N), lab].astype(np.float64).sum()
    assert r["cost"] == pytest.approx(cost, rel=1e-9)


def test_three_legs_on_five_seeds(c3):
    v, o = c3
    legs = {"trained": dict(), "untrained": dict(steps=0), "no_embedding": dict(embed=False)}
    t_plain, t_trained, reached = [], [], {name: 0 for name in legs}
    for seed in range(5):
        init = torch.as_tensor(synth.init_medoids(N, K, seed), dtype=torch.int32).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = learned.plain_fit(v, o, W, K, init)
        t_plain.append(time.perf_counter() - t0)
        for name, kw in legs.items():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = learned.fit(v, o, W, K, seed=seed, rounds=4, target_cost=p["cost"], **kw)
            torch.cuda.synchronize()
            if name == "trained":
                t_trained.append(time.perf_counter() - t0)
            reached[name] += r["cost"] <= p["cost"] * (1 + learned.REACH_RTOL)
            if seed == 0:
                _check_exact(v, o, r)
    assert np.median(t_trained) < np.median(t_plain), (t_trained, t_plain)
    print(f"reached the plain cost on 5 seeds: {reached}; median s: trained "
          f"{np.median(t_trained):.4f}, plain {np.median(t_plain):.4f}")

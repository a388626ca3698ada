"""Pins of the proposal-layer oracle (oracle/proposal_ref.py) on the CPU.

* splitmix64 against its published first output for seed 0;
* k-means++: the first centre, distinct centres, the draw frequencies of the
  second centre against the D2 / sum(D2) law, the all-duplicates fallback;
* lazy k-medoids with every member a candidate against the C oracle's
  alternate k-medoids (an independent implementation), the closed-form pair
  count of a run with one candidate per cluster, and the candidate list on a
  hand-worked cluster.
"""

import numpy as np
import pytest

import oracle
from oracle import proposal_ref as pr


def _euclid(n, dim, seed):
    rng = np.random.default_rng(seed)
    pts = rng.standard_normal((n, dim))
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1))
    return np.minimum(D, D.T), pts


def test_splitmix64_published_value():
    assert pr.splitmix64(0)[1] == 0xE220A8397B1DCDAF


def test_kmeanspp_first_and_distinct():
    rng = np.random.default_rng(0)
    E = rng.standard_normal((40, 3))
    for seed in range(20):
        c, _ = pr.kmeanspp(E, 7, seed)
        assert c[0] == pr.splitmix64(seed)[1] % 40
        assert len(set(c.tolist())) == 7
    c, _ = pr.kmeanspp(E, 40, 3)
    assert sorted(c.tolist()) == list(range(40))


def test_kmeanspp_second_centre_follows_d2_law():
    # five 1-D points; the second centre is drawn with probability D2_j / sum D2
    E = np.array([[0.0], [1.0], [3.0], [3.0], [7.0]])
    counts = {}
    firsts = 0
    for seed in range(6000):
        c, _ = pr.kmeanspp(E, 2, seed)
        if c[0] != 0:
            continue
        firsts += 1
        counts[int(c[1])] = counts.get(int(c[1]), 0) + 1
    d2 = np.array([0.0, 1.0, 9.0, 9.0, 49.0])
    p = d2 / d2.sum()
    assert firsts > 800
    assert 0 not in counts
    for j in range(1, 5):
        exp = firsts * p[j]
        sd = np.sqrt(firsts * p[j] * (1 - p[j]))
        assert abs(counts.get(j, 0) - exp) < 5 * sd + 1


def test_kmeanspp_all_duplicates_fallback():
    E = np.zeros((10, 4))
    c, _ = pr.kmeanspp(E, 4, 11)
    first = pr.splitmix64(11)[1] % 10
    rest = [j for j in range(10) if j != first][:3]
    assert c.tolist() == [first] + rest


def test_kmeans_recovers_separated_blobs():
    rng = np.random.default_rng(2)
    centres = np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0], [10.0, 10.0]])
    E = np.concatenate([c + 0.3 * rng.standard_normal((25, 2)) for c in centres])
    res = pr.kmeans(E, 4, restarts=3, iters=50, seed=5)
    blobs = sorted(int(m) // 25 for m in res["medoids"])
    assert blobs == [0, 1, 2, 3]  # one proposal per blob
    for m in res["medoids"]:
        b = int(m) // 25
        mean = E[b * 25:(b + 1) * 25].mean(0)
        d = ((E[b * 25:(b + 1) * 25] - mean) ** 2).sum(1)
        assert int(m) == b * 25 + int(np.argmin(d))  # the member nearest its blob mean
    inertia = sum(((E[b * 25:(b + 1) * 25] - E[b * 25:(b + 1) * 25].mean(0)) ** 2).sum()
                  for b in range(4))
    assert res["inertia"] == pytest.approx(inertia, rel=1e-12)


def test_kmeans_restarts_take_the_least_inertia():
    rng = np.random.default_rng(4)
    E = rng.standard_normal((120, 3))
    single = [pr.kmeans(E, 6, 1, 30, 10 + r)["inertia"] for r in range(4)]
    multi = pr.kmeans(E, 6, 4, 30, 10)
    assert multi["inertia"] == pytest.approx(min(single), rel=1e-12)
    # zero iterations: the k-means++ seeds themselves are the proposals
    seeds, _ = pr.kmeanspp(E, 6, 10)
    assert pr.kmeans(E, 6, 1, 0, 10)["medoids"].tolist() == seeds.tolist()


@pytest.mark.parametrize("n,k,seed", [(30, 3, 0), (64, 5, 1), (100, 8, 2), (12, 12, 3)])
def test_lazy_all_candidates_is_alternate_kmedoids(n, k, seed):
    D, pts = _euclid(n, 3, seed)
    init = np.random.default_rng(seed).permutation(n)[:k]
    ref = oracle.kmedoids(D, k, init, 100)
    got = pr.lazy_kmedoids(D, None, k, init)
    assert got["medoids"].tolist() == ref["medoids"].tolist()
    assert got["labels"].tolist() == ref["labels"].tolist()
    assert got["iters"] == ref["iters"]
    assert got["cost"] == pytest.approx(ref["cost"], rel=1e-12)
    # every member a candidate through the embedding route as well
    got2 = pr.lazy_kmedoids(D, pts, k, init, candidates=n)
    assert got2["medoids"].tolist() == ref["medoids"].tolist()


def test_lazy_one_candidate_pair_count():
    D, pts = _euclid(50, 2, 7)
    init = [3, 17, 40]
    got = pr.lazy_kmedoids(D, pts, 3, init, candidates=1)
    # only the current medoid is a candidate: nothing moves, one sweep
    assert got["iters"] == 1
    assert got["medoids"].tolist() == init
    assert got["pairs"] == 3 * 50 + 50


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lazy_full_screen_is_alternate_kmedoids(seed):
    # a sample of the whole cluster that keeps every member: every member is a candidate
    D, pts = _euclid(70, 3, seed + 20)
    init = np.random.default_rng(seed).permutation(70)[:4]
    ref = oracle.kmedoids(D, 4, init, 100)
    got = pr.lazy_kmedoids(D, None, 4, init, screen_sample=70, screen_keep=70)
    assert got["medoids"].tolist() == ref["medoids"].tolist()
    assert got["labels"].tolist() == ref["labels"].tolist()
    assert got["iters"] == ref["iters"]


def test_lazy_screen_hand_example():
    # one cluster of 1-D points; sample of 2 from 5 members: positions 0 and 2
    x = np.array([0.0, 1.0, 2.0, 3.0, 10.0])
    D = np.abs(x[:, None] - x[None])
    got = pr.lazy_kmedoids(D, None, 1, [4], screen_sample=2, screen_keep=1, max_iter=1)
    # sample {0, 2}: scores 2, 2, 2, 4, 18 -> the smallest index of least score, 0
    assert got["medoids"].tolist() == [0]
    assert got["pairs"] == 5 + 5 * 2 + 2 * 5 + 5  # assign, screen, update, final assign


def test_candidate_list_hand_example():
    # members 0..4 at 1-D positions; centroid (0+1+2+6+10)/5 = 3.8
    emb = np.array([[0.0], [1.0], [2.0], [6.0], [10.0]])
    chosen, gap = pr.candidate_list([0, 1, 2, 3, 4], 4, emb, 3)
    # squared distances to 3.8: 14.44, 7.84, 3.24, 4.84 (medoid 4 excluded)
    assert chosen == [4, 2, 3]
    assert gap == pytest.approx((7.84 - 4.84) / 7.84)


def test_lazy_max_iter_reassigns():
    D, pts = _euclid(80, 2, 9)
    init = [0, 1, 2, 3]
    full = oracle.kmedoids(D, 4, init, 1)
    got = pr.lazy_kmedoids(D, None, 4, init, max_iter=1)
    assert got["medoids"].tolist() == full["medoids"].tolist()
    assert got["labels"].tolist() == full["labels"].tolist()

"""Pins of the cluster-quality reference (oracle/cluster_ref.py) on the CPU."""

import numpy as np
import pytest

from oracle import cluster_ref as cr


def test_silhouette_hand_example():
    # points 0, 1 (cluster 0) and 10, 12 (cluster 1) on a line, D = |x - y|
    x = np.array([0.0, 1.0, 10.0, 12.0])
    D = np.abs(x[:, None] - x[None])
    s, mean = cr.silhouette(D, [0, 0, 1, 1])
    # point 0: a = 1, b = (10 + 12) / 2 = 11 -> 10/11; point 1: a = 1, b = 10 -> 9/10
    # point 10: a = 2, b = 9.5 -> 7.5/9.5; point 12: a = 2, b = 11.5 -> 9.5/11.5
    ref = [10 / 11, 9 / 10, 7.5 / 9.5, 9.5 / 11.5]
    assert np.allclose(s, ref, rtol=1e-15)
    assert mean == pytest.approx(np.mean(ref), rel=1e-15)


def test_silhouette_singleton_and_sign():
    x = np.array([0.0, 1.0, 5.0])
    D = np.abs(x[:, None] - x[None])
    s, _ = cr.silhouette(D, [0, 1, 1])
    assert s[0] == 0.0  # a singleton cluster
    # point 1 sits closer to the other cluster: a = 4 > b = 1 -> negative
    assert s[1] == pytest.approx((1 - 4) / 4)


@pytest.mark.parametrize("n,k,seed", [(30, 2, 0), (80, 5, 1), (57, 9, 2)])
def test_silhouette_matches_library(n, k, seed):
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(seed)
    pts = rng.standard_normal((n, 3))
    D = ((pts[:, None] - pts[None]) ** 2).sum(-1)  # squared distances, like DTW costs
    labels = np.arange(n) % k
    rng.shuffle(labels)
    _, mean = cr.silhouette(D, labels)
    assert mean == pytest.approx(metrics.silhouette_score(D, labels, metric="precomputed"),
                                 rel=1e-12)
    s, _ = cr.silhouette(D, labels)
    assert np.allclose(s, metrics.silhouette_samples(D, labels, metric="precomputed"), rtol=1e-12)


def test_elbow_second_difference():
    costs = {1: 100.0, 2: 60.0, 3: 25.0, 4: 22.0, 5: 20.0, 6: 19.0}
    # second differences: k=2: 100-120+25=5, k=3: 60-50+22=32, k=4: 25-44+20=1, k=5: 22-40+19=1
    assert cr.elbow(costs) == 3


def _rand_D(n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.standard_normal((n, 2))
    return np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1))


@pytest.mark.parametrize("n,k,seed", [(9, 2, 0), (12, 3, 1), (10, 4, 2)])
def test_pam_swap_deltas_equal_brute_force(n, k, seed):
    D = _rand_D(n, seed)
    M = list(np.random.default_rng(seed).permutation(n)[:k])
    delta = cr.swap_deltas(D, M)
    td = cr.nearest(D, M)[0].sum()
    for o in range(n):
        for i in range(k):
            if o in M:
                assert np.isinf(delta[o, i])
                continue
            M2 = list(M)
            M2[i] = o
            assert delta[o, i] == pytest.approx(cr.nearest(D, M2)[0].sum() - td, abs=1e-12)


@pytest.mark.parametrize("n,k,seed", [(10, 1, 3), (11, 2, 4), (12, 3, 5)])
def test_pam_reaches_a_swap_local_optimum(n, k, seed):
    import oracle.brute as brute
    D = _rand_D(n, seed)
    res = cr.pam(D, k)
    M = list(res["medoids"])
    td = res["cost"]
    for o in range(n):  # no single swap improves the answer
        for i in range(k):
            if o in M:
                continue
            M2 = list(M)
            M2[i] = o
            assert cr.nearest(D, M2)[0].sum() >= td - 1e-12
    opt, _ = brute.kmedoids_optimum(D, k)
    assert td >= opt - 1e-12
    if k == 1:  # BUILD alone finds the optimum
        assert td == pytest.approx(opt, rel=1e-15)


def test_pam_finds_planted_optimum():
    import oracle.brute as brute
    rng = np.random.default_rng(6)
    centres = np.array([[0, 0], [10, 0], [0, 10]])
    pts = centres[np.arange(12) % 3] + 0.5 * rng.standard_normal((12, 2))
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1))
    res = cr.pam(D, 3, init=[0, 3, 6])  # three medoids from the same group
    opt, _ = brute.kmedoids_optimum(D, 3)
    assert res["cost"] == pytest.approx(opt, rel=1e-12) and res["swaps"] >= 2


def test_pam_build_gap_is_the_runner_up_margin():
    # seven points on a line at 0, 1, 3, 6, 8, 11, 12: row sums 41, 36, 30, 27, 29, 38,
    # 43 -> the point at 6 first (runner-up 29: gap 2/27); with d1 = (6, 5, 3, 0, 2, 5, 6)
    # the gains are 17, 16, 18, -, 21, 17, 17 -> the point at 1 (gap 1/16)
    x = np.array([0.0, 1.0, 3.0, 6.0, 8.0, 11.0, 12.0])
    D = np.abs(x[:, None] - x[None])
    M, gap = cr.pam_build(D, 2, with_gap=True)
    assert M == [3, 1] and gap == pytest.approx(1 / 16, rel=1e-15)
    assert cr.pam_build(D, 2) == M
    assert cr.pam_build(D, 1, with_gap=True)[1] == pytest.approx(2 / 27, rel=1e-15)
    # an exact tie makes the gap 0: the two middle points of four on a line
    x = np.array([0.0, 1.0, 2.0, 3.0])
    _, gap = cr.pam_build(np.abs(x[:, None] - x[None]), 1, with_gap=True)
    assert gap == 0.0
    assert np.isinf(cr.pam(D, 2, init=[0, 1])["build_gap"])

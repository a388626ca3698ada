"""GPU parity of the silhouette, the elbow curve and PAM against the float64 references.

Both sides see the same float32 matrix (made on the CPU) and labels; the GPU
sums clusters in float64 in a different order, so s(i) agree within 1e-9.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import cluster_ref as cr
from paper_2307_04904_gb300 import api, quality, synth

pytestmark = pytest.mark.gpu


def _sqdist(n, dim, seed, centres=None):
    rng = np.random.default_rng(seed)
    pts = rng.standard_normal((n, dim))
    if centres is not None:
        pts = pts + centres[np.arange(n) % len(centres)]
    D = ((pts[:, None] - pts[None]) ** 2).sum(-1).astype(np.float32)
    D = np.minimum(D, D.T)
    np.fill_diagonal(D, 0)
    return D


@pytest.mark.parametrize("n,k,seed", [(2, 2, 0), (37, 3, 1), (300, 7, 2), (1000, 12, 3)])
def test_silhouette_random_labels(n, k, seed):
    D = _sqdist(n, 4, seed)
    labels = (np.arange(n) % k).astype(np.int32)
    np.random.default_rng(seed).shuffle(labels)
    s, mean = api.kmedoids_silhouette(torch.from_numpy(D).cuda(), torch.from_numpy(labels).cuda(), k)
    ref_s, ref_mean = cr.silhouette(D.astype(np.float64), labels)
    assert np.max(np.abs(s.cpu().numpy() - ref_s)) < 1e-6  # s is returned as float32
    assert mean == pytest.approx(ref_mean, abs=1e-9)


def test_silhouette_dtw_matrix_empty_and_singleton_clusters():
    values, offsets, cls = synth.five_class_set(60, 96, seed=4)
    a, b = np.triu_indices(60, 1)
    D = np.zeros((60, 60), dtype=np.float32)
    D[a, b] = D[b, a] = oracle.pairs_f32_mirror(values, offsets, a, b, 9)
    labels = cls.astype(np.int32).copy()
    labels[7] = 6  # a singleton cluster; cluster 5 stays empty
    s, mean = api.kmedoids_silhouette(torch.from_numpy(D).cuda(), torch.from_numpy(labels).cuda(), 7)
    ref_s, ref_mean = cr.silhouette(D.astype(np.float64), labels)
    assert np.max(np.abs(s.cpu().numpy() - ref_s)) < 1e-6 and s[7].item() == 0.0
    assert mean == pytest.approx(ref_mean, abs=1e-9)


def test_silhouette_errors():
    D = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    for labels, k in (([0, 0, 0, 0], 2), ([0, 1, 2, 3], 1), ([0, 1, 5, 1], 3)):
        with pytest.raises(api.DTWError):
            api.kmedoids_silhouette(D, torch.tensor(labels, dtype=torch.int32, device="cuda"), k)


def test_elbow_curve_and_silhouette_choose_the_planted_k():
    centres = np.array([[0, 0, 0], [12, 0, 0], [0, 12, 0], [0, 0, 12]], dtype=np.float64)
    D = _sqdist(400, 3, 5, centres)
    Dt = torch.from_numpy(D).cuda()
    res = quality.elbow(Dt, 7, seed=2)
    for k, cost in res["costs"].items():
        ref = oracle.kmedoids(D.astype(np.float64), k, synth.init_medoids(400, k, 2), 100)
        if ref["min_margin"] >= 1e-6:
            assert cost == pytest.approx(ref["cost"], rel=1e-9)
    assert res["elbow"] == cr.elbow(res["costs"])
    # one medoid per planted group (points i and i % 4 share a group): the fit finds the
    # groups, and their silhouette beats every k-medoids answer with another k
    _, labels, _, _ = api.kmedoids_fit(Dt, 4, torch.arange(4, dtype=torch.int32, device="cuda"))
    assert np.array_equal(labels.cpu().numpy(), np.arange(400) % 4)
    _, s4 = quality.silhouette(Dt, labels, 4)
    assert s4 > 0.9 and all(s4 >= v for v in res["silhouette"].values())


def _assert_pam(got, ref):
    # the GPU sums the swap terms in compensated float32: decisions are compared
    # when no delta of the reference lies within 1e-6 (relative to the cost) of another or of 0
    med, lab, cost, swaps = got
    if ref["min_gap"] >= 1e-6:
        assert med.cpu().numpy().tolist() == ref["medoids"].tolist()
        assert lab.cpu().numpy().tolist() == ref["labels"].tolist()
        assert swaps == ref["swaps"]
        assert cost == pytest.approx(ref["cost"], rel=1e-9)
    else:
        assert cost == pytest.approx(ref["cost"], rel=1e-5)


@pytest.mark.parametrize("n,k,seed", [(1, 1, 0), (40, 1, 1), (60, 3, 2), (200, 7, 3), (150, 64, 4)])
def test_pam_build_and_swap(n, k, seed):
    D = _sqdist(n, 3, seed)
    Dt = torch.from_numpy(D).cuda()
    _assert_pam(api.kmedoids_pam(Dt, k), cr.pam(D.astype(np.float64), k))


def test_pam_on_dtw_matrix_from_alternate_answer():
    values, offsets, _ = synth.five_class_set(100, 96, seed=6)
    a, b = np.triu_indices(100, 1)
    D = np.zeros((100, 100), dtype=np.float32)
    D[a, b] = D[b, a] = oracle.pairs_f32_mirror(values, offsets, a, b, 9)
    Dt = torch.from_numpy(D).cuda()
    init = synth.init_medoids(100, 5, 6)
    med, _, alt_cost, _ = api.kmedoids_fit(Dt, 5, torch.as_tensor(init, dtype=torch.int32).cuda())
    got = api.kmedoids_pam(Dt, 5, med)
    ref = cr.pam(D.astype(np.float64), 5)  # BUILD on both sides
    # from the alternate answer: PAM never raises the cost
    assert got[2] <= alt_cost * (1 + 1e-12)
    # from the same initial medoids on both sides
    _assert_pam(api.kmedoids_pam(Dt, 5, torch.as_tensor(init, dtype=torch.int32).cuda()),
                cr.pam(D.astype(np.float64), 5, init=init))
    _assert_pam(api.kmedoids_pam(Dt, 5), ref)


def test_pam_swap_limit_and_errors():
    D = _sqdist(80, 2, 7)
    Dt = torch.from_numpy(D).cuda()
    init = [0, 1, 2, 3]
    for ms in (0, 1, 2):
        got = api.kmedoids_pam(Dt, 4, torch.tensor(init, dtype=torch.int32, device="cuda"), ms)
        ref = cr.pam(D.astype(np.float64), 4, init=init, max_swaps=ms)
        assert got[3] == ref["swaps"] <= ms
        _assert_pam(got, ref)
    with pytest.raises(api.DTWError):
        api.kmedoids_pam(Dt, 65)
    with pytest.raises(api.DTWError):
        api.kmedoids_pam(Dt, 2, torch.tensor([3, 3], dtype=torch.int32, device="cuda"))

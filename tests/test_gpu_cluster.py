"""GPU parity of the silhouette, the elbow curve and PAM against the float64 references.

Both sides see the same float32 matrix (made on the CPU) and labels.  The GPU
sums rows in segments of 512 (Kahan-compensated float32 within a segment,
float64 across), so s(i) agree within 1e-6 and PAM's choices are compared where
no two candidates of the reference lie within 1e-6 of each other.
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


@pytest.mark.parametrize("n,k,seed", [(2, 2, 0), (37, 3, 1), (300, 7, 2), (1000, 12, 3),
                                      (1500, 300, 4), (2100, 40, 5)])
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
    if min(ref["min_gap"], ref["build_gap"]) >= 1e-6:
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


# n = 1100 and 1030 put more than 512 members in a cluster and more than 512 rows
# in BUILD's sums, so segments split; 1100 takes the float4 path, 1030 the scalar one
@pytest.mark.parametrize("n", [1100, 1030])
def test_silhouette_and_pam_across_segments(n):
    D = _sqdist(n, 3, 11)
    labels = (np.arange(n) % 2).astype(np.int32)
    s, mean = api.kmedoids_silhouette(torch.from_numpy(D).cuda(), torch.from_numpy(labels).cuda(), 2)
    ref_s, ref_mean = cr.silhouette(D.astype(np.float64), labels)
    assert np.max(np.abs(s.cpu().numpy() - ref_s)) < 1e-6
    assert mean == pytest.approx(ref_mean, abs=1e-9)
    Dt = torch.from_numpy(D).cuda()
    _assert_pam(api.kmedoids_pam(Dt, 2, None, 1), cr.pam(D.astype(np.float64), 2, max_swaps=1))


@pytest.mark.parametrize("n,k", [(3000, 5), (3001, 4)])
def test_pam_build_across_segments(n, k):
    D = _sqdist(n, 3, 12)
    got = api.kmedoids_pam(torch.from_numpy(D).cuda(), k, None, 0)
    _assert_pam(got, cr.pam(D.astype(np.float64), k, max_swaps=0))


def test_packed_and_scalar_reductions_give_the_same_bits():
    # the same matrix once 16-byte aligned (float4 loads, packed pair arithmetic) and
    # once 4 bytes past the boundary (scalar loads and arithmetic): identical results
    n = 1100
    D = _sqdist(n, 3, 13)
    a = torch.from_numpy(D).cuda()
    buf = torch.empty(n * n + 1, dtype=torch.float32, device="cuda")
    b = buf[1:].view(n, n)
    b.copy_(a)
    assert a.data_ptr() % 16 == 0 and b.data_ptr() % 16 == 4
    labels = torch.from_numpy((np.arange(n) % 3).astype(np.int32)).cuda()
    s1, m1 = api.kmedoids_silhouette(a, labels, 3)
    s2, m2 = api.kmedoids_silhouette(b, labels, 3)
    assert torch.equal(s1, s2) and m1 == m2
    p1, p2 = api.kmedoids_pam(a, 4), api.kmedoids_pam(b, 4)
    assert torch.equal(p1[0], p2[0]) and torch.equal(p1[1], p2[1]) and p1[2:] == p2[2:]


def test_mip_export_of_the_gpu_matrix_bounds_the_heuristics():
    pytest.importorskip("scipy.optimize")
    import oracle.brute as brute
    from paper_2307_04904_gb300 import mip

    values, offsets, _ = synth.five_class_set(12, 64, seed=9)
    D = api.dtw_pairwise(torch.from_numpy(values).cuda(), torch.from_numpy(offsets).cuda(), 6)
    Dh = D.cpu().numpy().astype(np.float64)
    k = 3
    res = mip.solve(D, k)
    opt, _ = brute.kmedoids_optimum(Dh, k)
    assert res["cost"] == pytest.approx(opt, rel=1e-9)
    init = torch.as_tensor(synth.init_medoids(12, k, 9), dtype=torch.int32).cuda()
    for med, lab, cost, _ in (api.kmedoids_fit(D, k, init), api.kmedoids_pam(D, k)):
        A = mip.assignment_matrix(med, lab)
        assert (Dh * A).sum() == pytest.approx(cost, rel=1e-6)  # the GPU's own cost
        assert cost >= res["cost"] * (1 - 1e-6)

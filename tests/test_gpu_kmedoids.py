"""GPU parity of kmedoids_fit against the oracle's alternate k-medoids.

Both sides run from the same initial medoids on the same float32 D, made on
the CPU (the oracle's float-mirror DTW, or Euclidean distances of seeded
points) and widened exactly to float64 for the oracle.  Labels and medoids
must be identical when no decision of the oracle's run is a near-tie (relative
gap >= 1e-6 between best and second-best); otherwise the costs must agree
within 1e-5 relative.  Costs are float64 sums in a different order on each
side, so they are compared at 1e-9 relative when the labels agree.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2307_04904_gb300 import api, synth

pytestmark = pytest.mark.gpu
NEAR_TIE = 1e-6


def _fit_both(D_t, k, init, max_iter=100):
    med, lab, cost, iters = api.kmedoids_fit(D_t, k, torch.as_tensor(init, dtype=torch.int32).cuda(),
                                             max_iter)
    D64 = D_t.cpu().numpy().astype(np.float64)
    ref = oracle.kmedoids(D64, k, init, max_iter)
    return med.cpu().numpy(), lab.cpu().numpy(), cost, iters, ref


def _assert_parity(got, ref):
    med, lab, cost, iters = got
    if ref["min_margin"] >= NEAR_TIE:
        assert med.tolist() == ref["medoids"].tolist()
        assert lab.tolist() == ref["labels"].tolist()
        assert iters == ref["iters"]
        assert cost == pytest.approx(ref["cost"], rel=1e-9)
    else:
        assert cost == pytest.approx(ref["cost"], rel=1e-5)


def _mirror_matrix(values, offsets, w):
    p = len(offsets) - 1
    a, b = np.triu_indices(p, 1)
    m = oracle.pairs_f32_mirror(values, offsets, a, b, w)
    D = np.zeros((p, p), dtype=np.float32)
    D[a, b] = m
    D[b, a] = m
    return D


def test_small_config_kmedoids():
    values, offsets = synth.random_walk_set(50, 128, seed=0)
    for w in (128, 12):
        D = torch.from_numpy(_mirror_matrix(values, offsets, w)).cuda()
        init = synth.init_medoids(50, 3, 0)
        med, lab, cost, iters, ref = _fit_both(D, 3, init)
        _assert_parity((med, lab, cost, iters), ref)


def test_large_config_kmedoids_on_the_dtw_matrix(c1_matrix):
    """k = 5 on the DTW matrix of the 2000 x 512 benchmark set (w = 51), which equals the
    oracle's float mirror bit for bit (checked pair by pair in test_gpu_dtw), from the
    benchmark's initial medoids and from four more seeds."""
    c = c1_matrix
    D = c["D"]
    a, b = c["a"], c["b"]
    assert np.array_equal(D[a, b].view(np.uint32), c["mirror"].view(np.uint32))
    Dt = torch.from_numpy(D).cuda()
    checked = 0
    for seed in range(1, 6):
        init = synth.init_medoids(2000, 5, seed)
        med, lab, cost, iters, ref = _fit_both(Dt, 5, init)
        _assert_parity((med, lab, cost, iters), ref)
        checked += ref["min_margin"] >= NEAR_TIE
    assert checked >= 3  # most runs decide every step by a clear margin


def test_large_config_kmedoids():
    # n = 2000, k = 5: five well-separated groups of seeded points
    rng = np.random.default_rng(1)
    centres = rng.standard_normal((5, 6)) * 4
    pts = centres[np.arange(2000) % 5] + rng.standard_normal((2000, 6))
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)).astype(np.float32)
    D = np.minimum(D, D.T)
    np.fill_diagonal(D, 0)
    init = synth.init_medoids(2000, 5, 1)
    med, lab, cost, iters, ref = _fit_both(torch.from_numpy(D).cuda(), 5, init)
    _assert_parity((med, lab, cost, iters), ref)


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (7, 1), (33, 4), (130, 12), (257, 3)])
def test_kmedoids_shapes(n, k):
    rng = np.random.default_rng(n * 31 + k)
    pts = rng.standard_normal((n, 3))
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)).astype(np.float32)
    D = np.minimum(D, D.T)  # exactly symmetric
    init = synth.init_medoids(n, k, n + k)
    med, lab, cost, iters, ref = _fit_both(torch.from_numpy(D).cuda(), k, init)
    _assert_parity((med, lab, cost, iters), ref)


def test_max_iter_and_fixed_point():
    rng = np.random.default_rng(5)
    pts = rng.standard_normal((60, 2))
    D = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)).astype(np.float32)
    D = np.minimum(D, D.T)
    Dt = torch.from_numpy(D).cuda()
    init = synth.init_medoids(60, 4, 5)
    for mi in (1, 2, 3):
        med, lab, cost, iters, ref = _fit_both(Dt, 4, init, mi)
        _assert_parity((med, lab, cost, iters), ref)
    # a converged answer is a fixed point: one sweep, same medoids
    med, _, _, _ = api.kmedoids_fit(Dt, 4, torch.as_tensor(init, dtype=torch.int32).cuda())
    med2, _, _, it2 = api.kmedoids_fit(Dt, 4, med.clone())
    assert it2 == 1 and torch.equal(med, med2)


def _fit_exact(D, k, init, max_iter=100):
    """Both sides on a matrix of small integers: every distance and every sum is exact in
    float32, TwoSum pairs and float64, so every decision -- ties included -- must come out
    the same, and the costs equal exactly."""
    med, lab, cost, iters = api.kmedoids_fit(torch.from_numpy(D.astype(np.float32)).cuda(), k,
                                             torch.as_tensor(init, dtype=torch.int32).cuda(),
                                             max_iter)
    ref = oracle.kmedoids(D.astype(np.float64), k, init, max_iter)
    assert med.cpu().numpy().tolist() == ref["medoids"].tolist()
    assert lab.cpu().numpy().tolist() == ref["labels"].tolist()
    assert iters == ref["iters"] and cost == ref["cost"]
    return ref


def test_exact_ties_are_decided_as_the_oracle_decides():
    # the hand-built line of the oracle's tie pin: update ties keep the current medoid,
    # else go to the smallest index
    x = np.array([0, 1, 2, 3, 100, 101, 102, 103])
    D = np.abs(x[:, None] - x[None, :])
    assert _fit_exact(D, 2, [2, 6])["medoids"].tolist() == [2, 6]
    assert _fit_exact(D, 2, [0, 7])["medoids"].tolist() == [1, 5]
    _fit_exact(D, 2, [3, 4], max_iter=1)
    # assignment ties go to the smallest cluster; a medoid labels itself at distance 0
    A = np.array([[0, 1, 1, 5], [1, 0, 0, 5], [1, 0, 0, 5], [5, 5, 5, 0]])
    r = _fit_exact(A, 2, [1, 2], max_iter=1)
    assert r["labels"].tolist() == [0, 0, 1, 0]


@pytest.mark.parametrize("keep", [True, False])
def test_exact_ties_at_scale(keep):
    """n = 2000, k = 5 in scattered index order: each cluster is 400 consecutive integer
    positions, so its two central members tie exactly.  From the larger-index member of
    each tied pair the fit keeps it; from the clusters' first positions it moves to the
    smaller-index member and keeps that.  Exercises the multi-lane row sums and the
    block-wide update scan on exact ties."""
    rng = np.random.default_rng(12)
    perm = rng.permutation(2000)
    pos = np.empty(2000, np.int64)
    pos[perm] = (np.arange(2000) // 400) * 1000 + np.arange(2000) % 400
    D = np.abs(pos[:, None] - pos[None, :])
    centre = [(perm[400 * c + 199], perm[400 * c + 200]) for c in range(5)]
    if keep:
        init = [max(p) for p in centre]
        want_iters = 1
    else:
        init = [perm[400 * c] for c in range(5)]
        want_iters = 2
    r = _fit_exact(D, 5, init)
    assert r["iters"] == want_iters
    assert r["medoids"].tolist() == ([max(p) for p in centre] if keep else [min(p) for p in centre])


def test_kmedoids_argument_errors():
    D = torch.zeros((5, 5), dtype=torch.float32, device="cuda")
    # duplicate and out-of-range medoids, and k > n, are refused by the library
    for init, k in (([0, 0], 2), ([0, 5], 2), ([0, 1, 2, 3, 4, 0], 6)):
        with pytest.raises(api.DTWError) as e:
            api.kmedoids_fit(D, k, torch.tensor(init, dtype=torch.int32, device="cuda"))
        assert e.value.code == api.DTW_EINVAL
    # an initial list that is not k long never reaches the library
    with pytest.raises(ValueError, match="init_medoids"):
        api.kmedoids_fit(D, 3, torch.tensor([0, 1], dtype=torch.int32, device="cuda"))

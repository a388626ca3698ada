"""GPU parity of the pair-list DTW, k-means++ seeding and lazy k-medoids
(include/dtwgb.h dtw_pairs, include/dtwgb_proposal.h) against the oracles.

* dtw_pairs: bit-for-bit equal to the oracle's float mirror (the same float
  operations per cell), <= 1e-5 relative to the float64 oracle, on rotated-band
  and column-strip shapes and per-mille windows.
* kmedoids_lazy_fit: run on the oracle's float-mirror DTW matrix (widened to
  float64), the oracle's lazy k-medoids must give the same medoids, labels,
  sweep count and pair count when none of its decisions is a near-tie; with
  every member a candidate it is the plain alternate k-medoids.
* proposal_kmeanspp: the same centres as the oracle when no draw lands within
  1e-6 (relative) of a running-sum boundary.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import proposal_ref as pr
from paper_2307_04904_gb300 import api, synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5
NEAR_TIE = 1e-9      # update sums: float64 in a different order on each side
CAND_GAP = 1e-5      # embedding distances: float32 on the GPU, float64 in the oracle
KPP_GAP = 1e-6       # k-means++ draw against the running sums (relative to the total)


def _dev(values, offsets):
    return torch.from_numpy(values).cuda(), torch.from_numpy(offsets).cuda()


def _mirror_matrix(values, offsets, w):
    p = len(offsets) - 1
    a, b = np.triu_indices(p, 1)
    m = oracle.pairs_f32_mirror(values, offsets, a, b, w)
    D = np.zeros((p, p), dtype=np.float32)
    D[a, b] = m
    D[b, a] = m
    return D


@pytest.mark.parametrize("w,shape,lo,hi", [(10, None, 60, 300), (-1, None, 60, 300),
                                           (30, "strip:8", 100, 140), (30, "rot:13:8", 100, 140)])
def test_dtw_pairs_mirror(w, shape, lo, hi, monkeypatch):
    if shape:
        monkeypatch.setenv("DTWGB_SHAPE", shape)
    lens = synth.ragged_lengths(40, lo, hi, seed=3)
    values, offsets, _ = synth.five_class_set(40, lens, seed=3)
    rng = np.random.default_rng(4)
    a = rng.integers(0, 40, 2500).astype(np.int32)
    b = rng.integers(0, 40, 2500).astype(np.int32)
    a[:40] = np.arange(40)
    b[:40] = np.arange(40)          # diagonal pairs: exactly 0
    got = api.dtw_pairs(*_dev(values, offsets), torch.from_numpy(a).cuda(),
                        torch.from_numpy(b).cuda(), w).cpu().numpy()
    mir = oracle.pairs_f32_mirror(values, offsets, a, b, w)
    assert np.array_equal(got.view(np.uint32), mir.view(np.uint32))
    assert np.all(got[:40] == 0)
    ref = oracle.pairs(values, offsets, a, b, w)
    nz = ref > 0
    assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) <= RTOL


def test_dtw_pairs_permille_and_edges():
    lens = synth.ragged_lengths(30, 50, 900, seed=6)
    values, offsets, _ = synth.five_class_set(30, lens, seed=6)
    v, o = _dev(values, offsets)
    rng = np.random.default_rng(7)
    a = rng.integers(0, 30, 600).astype(np.int32)
    b = rng.integers(0, 30, 600).astype(np.int32)
    got = api.dtw_pairs(v, o, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 80,
                        permille=True).cpu().numpy().astype(np.float64)
    w = np.maximum(lens[a], lens[b]) * 80 // 1000
    ref = oracle.pairs_w(values, offsets, a, b, w)
    nz = ref > 0
    assert np.all(got[~nz] == 0)
    assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) <= RTOL
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    assert api.dtw_pairs(v, o, empty, empty, 10).numel() == 0
    bad = torch.tensor([0, 30], dtype=torch.int32, device="cuda")
    with pytest.raises(api.DTWError):
        api.dtw_pairs(v, o, bad, bad.flip(0).contiguous(), 10)


def _lazy_both(values, offsets, w, k, init, emb=None, candidates=0, max_iter=100, screen=(0, 0)):
    D = _mirror_matrix(values, offsets, w).astype(np.float64)
    v, o = _dev(values, offsets)
    e = torch.from_numpy(emb).cuda() if emb is not None else None
    med, lab, cost, iters, pairs = api.kmedoids_lazy_fit(
        v, o, w, k, torch.as_tensor(init, dtype=torch.int32).cuda(), emb=e,
        candidates=candidates, screen_sample=screen[0], screen_keep=screen[1], max_iter=max_iter)
    ref = pr.lazy_kmedoids(D, emb, k, init, candidates if candidates > 0 else None, max_iter,
                           screen_sample=screen[0], screen_keep=screen[1])
    return (med.cpu().numpy(), lab.cpu().numpy(), cost, iters, pairs), ref, D


def _assert_lazy(got, ref):
    med, lab, cost, iters, pairs = got
    if ref["min_margin"] >= NEAR_TIE and ref["min_cand_gap"] >= CAND_GAP:
        assert med.tolist() == ref["medoids"].tolist()
        assert lab.tolist() == ref["labels"].tolist()
        assert iters == ref["iters"]
        assert pairs == ref["pairs"]
        assert cost == pytest.approx(ref["cost"], rel=1e-9)
    else:
        assert cost == pytest.approx(ref["cost"], rel=RTOL)


@pytest.mark.parametrize("k,seed", [(1, 0), (3, 1), (7, 2)])
def test_lazy_all_candidates_equals_alternate_kmedoids(k, seed):
    values, offsets = synth.random_walk_set(120, 96, seed=seed)
    init = synth.init_medoids(120, k, seed)
    got, ref, D = _lazy_both(values, offsets, 10, k, init)
    _assert_lazy(got, ref)
    plain = oracle.kmedoids(D, k, init, 100)
    if plain["min_margin"] >= NEAR_TIE:
        assert got[0].tolist() == plain["medoids"].tolist()
        assert got[1].tolist() == plain["labels"].tolist()


@pytest.mark.parametrize("cands,dim", [(1, 8), (4, 8), (16, 3), (1000, 8)])
def test_lazy_with_proposals(cands, dim):
    values, offsets, _ = synth.five_class_set(150, 128, seed=9)
    rng = np.random.default_rng(cands + dim)
    emb = rng.standard_normal((150, dim)).astype(np.float32)
    init = synth.init_medoids(150, 5, 9)
    got, ref, _ = _lazy_both(values, offsets, 12, 5, init, emb, cands)
    _assert_lazy(got, ref)


@pytest.mark.parametrize("cands,screen", [(0, (8, 4)), (6, (16, 3)), (0, (400, 400)),
                                          (1, (1, 1))])
def test_lazy_with_screening(cands, screen):
    values, offsets, _ = synth.five_class_set(140, 128, seed=15)
    emb = np.random.default_rng(15).standard_normal((140, 8)).astype(np.float32)
    init = synth.init_medoids(140, 6, 15)
    got, ref, D = _lazy_both(values, offsets, 12, 6, init, emb if cands else None, cands,
                             screen=screen)
    _assert_lazy(got, ref)
    if screen[0] >= 140:  # every member screened and kept: the plain algorithm
        plain = oracle.kmedoids(D, 6, init, 100)
        assert got[2] == pytest.approx(plain["cost"], rel=1e-9)


def test_lazy_ragged_strip_and_max_iter():
    lens = synth.ragged_lengths(90, 40, 400, seed=12)
    values, offsets, _ = synth.five_class_set(90, lens, seed=12)
    init = synth.init_medoids(90, 4, 12)
    for mi in (1, 2, 100):
        got, ref, _ = _lazy_both(values, offsets, -1, 4, init, max_iter=mi)
        _assert_lazy(got, ref)


def test_lazy_errors():
    values, offsets = synth.random_walk_set(10, 32, seed=0)
    v, o = _dev(values, offsets)
    with pytest.raises(api.DTWError):
        api.kmedoids_lazy_fit(v, o, 5, 2, torch.tensor([1, 1], dtype=torch.int32).cuda())
    with pytest.raises(api.DTWError):
        api.kmedoids_lazy_fit(v, o, 5, 2, torch.tensor([0, 10], dtype=torch.int32).cuda())
    with pytest.raises(api.DTWError):
        api.kmedoids_lazy_fit(v, o, 5, 11, torch.arange(11, dtype=torch.int32).cuda())
    with pytest.raises(api.DTWError):  # sampling without keeping anything
        api.kmedoids_lazy_fit(v, o, 5, 2, torch.tensor([0, 1], dtype=torch.int32).cuda(),
                              screen_sample=4, screen_keep=0)


@pytest.mark.parametrize("n,dim,k", [(500, 16, 10), (37, 3, 37), (2000, 64, 24)])
def test_kmeanspp_parity(n, dim, k):
    rng = np.random.default_rng(n + k)
    emb = rng.standard_normal((n, dim)).astype(np.float32)
    e = torch.from_numpy(emb).cuda()
    for seed in (0, 1, 12345):
        got = api.proposal_kmeanspp(e, k, seed).cpu().numpy()
        assert len(set(got.tolist())) == k
        ref, gap = pr.kmeanspp(emb, k, seed)
        if gap >= KPP_GAP:
            assert got.tolist() == ref.tolist()
        else:
            assert got[0] == ref[0]


def test_kmeanspp_duplicates_and_errors():
    e = torch.zeros((12, 4), dtype=torch.float32, device="cuda")
    got = api.proposal_kmeanspp(e, 5, 3).cpu().numpy()
    ref, _ = pr.kmeanspp(np.zeros((12, 4)), 5, 3)
    assert got.tolist() == ref.tolist()
    with pytest.raises(api.DTWError):
        api.proposal_kmeanspp(e, 13, 0)


def test_kmeans_separated_blobs_exact():
    rng = np.random.default_rng(21)
    centres = rng.standard_normal((12, 16)) * 10
    emb = (centres[np.arange(3000) % 12] + rng.standard_normal((3000, 16))).astype(np.float32)
    got, inertia = api.proposal_kmeans(torch.from_numpy(emb).cuda(), 12, 5, restarts=4, iters=30)
    ref = pr.kmeans(emb, 12, 4, 30, 5)
    if ref["min_gap"] >= CAND_GAP:
        assert got.cpu().numpy().tolist() == ref["medoids"].tolist()
    assert inertia == pytest.approx(ref["inertia"], rel=1e-5)


@pytest.mark.parametrize("n,dim,k,restarts,iters", [(800, 8, 10, 3, 20), (64, 3, 64, 1, 5),
                                                    (2000, 64, 10, 2, 0)])
def test_kmeans_properties(n, dim, k, restarts, iters):
    rng = np.random.default_rng(n + k)
    emb = rng.standard_normal((n, dim)).astype(np.float32)
    got, inertia = api.proposal_kmeans(torch.from_numpy(emb).cuda(), k, 7, restarts=restarts,
                                       iters=iters)
    got = got.cpu().numpy()
    assert len(set(got.tolist())) == k and got.min() >= 0 and got.max() < n
    ref = pr.kmeans(emb, k, restarts, iters, 7)
    if ref["min_gap"] >= CAND_GAP:
        assert got.tolist() == ref["medoids"].tolist()
        assert inertia == pytest.approx(ref["inertia"], rel=1e-5)
    with pytest.raises(api.DTWError):
        api.proposal_kmeans(torch.from_numpy(emb).cuda(), n + 1, 0)


def test_encoder_targets():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((70, 5))
    D = (((X[:, None] - X[None]) ** 2).sum(-1)).astype(np.float32)
    got = api.Encoder.targets(torch.from_numpy(D).cuda()).cpu().numpy()
    R = np.sqrt(D.astype(np.float64))
    off = ~np.eye(70, dtype=bool)
    ref = R / R[off].mean()
    np.fill_diagonal(ref, 0)
    assert np.all(np.diag(got) == 0)
    assert np.max(np.abs(got - ref)[off] / ref[off]) <= 1e-6

"""Pins for the CPU oracle: checks against brute force, closed forms and invariants.

Each test ties the double-precision DP of ``oracle/dtw_oracle.c`` (or the
k-medoids sweeps) to something other than itself, so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one of them.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import brute
from paper_2307_04904_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- DTW pins


def test_path_enumerator_counts_delannoy():
    # unconstrained paths from (1,1) to (n,m) with steps (1,0),(0,1),(1,1)
    for n in range(1, 6):
        for m in range(1, 6):
            cnt = sum(1 for _ in brute.warping_paths(n, m))
            assert cnt == brute.delannoy(n, m)
    # spot values of the Delannoy table
    assert brute.delannoy(3, 3) == 13 and brute.delannoy(4, 4) == 63


@pytest.mark.parametrize("strict", [False, True])
def test_dp_equals_brute_force_tiny(oracle_mod, strict):
    rng = _rng(11)
    for n in range(1, 7):
        for m in range(1, 7):
            x = rng.standard_normal(n).astype(np.float32)
            y = rng.standard_normal(m).astype(np.float32)
            for w in [-1] + list(range(0, max(n, m) + 1)):
                ref = brute.dtw_by_paths(x, y, w, strict)
                got = oracle_mod.dtw(x, y, w, strict)
                if math.isinf(ref):
                    assert math.isinf(got), (n, m, w)
                else:
                    assert got == pytest.approx(ref, rel=1e-12, abs=1e-12), (n, m, w)


def test_integer_inputs_exact(oracle_mod):
    # small-integer series: every partial sum is exact in float and double
    rng = _rng(12)
    for _ in range(60):
        n, m = rng.integers(1, 8, size=2)
        x = rng.integers(-3, 4, size=n).astype(np.float32)
        y = rng.integers(-3, 4, size=m).astype(np.float32)
        w = int(rng.integers(-1, 8))
        ref = brute.dtw_by_paths(x, y, w)
        assert oracle_mod.dtw(x, y, w) == ref
        assert float(oracle_mod.dtw_f32_mirror(x, y, w)) == ref


def test_hand_examples(oracle_mod):
    with open(os.path.join(GOLDEN, "dtw_hand_examples.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        exp = math.inf if c["expected"] == "inf" else float(c["expected"])
        got = oracle_mod.dtw(c["x"], c["y"], c["w"], c["strict"])
        assert got == exp, c
        assert float(oracle_mod.dtw_f32_mirror(c["x"], c["y"], c["w"], c["strict"])) == exp


def test_self_distance_zero_and_symmetry(oracle_mod):
    rng = _rng(13)
    for _ in range(20):
        n, m = rng.integers(1, 200, size=2)
        x = rng.standard_normal(n).astype(np.float32)
        y = rng.standard_normal(m).astype(np.float32)
        w = int(rng.integers(-1, 40))
        assert oracle_mod.dtw(x, x, w) == 0.0
        assert oracle_mod.dtw(x, y, w) == oracle_mod.dtw(y, x, w)  # bitwise
        assert oracle_mod.dtw_f32_mirror(x, y, w) == oracle_mod.dtw_f32_mirror(y, x, w)


def test_w0_is_squared_euclidean(oracle_mod):
    rng = _rng(14)
    for L in (1, 2, 7, 64, 300):
        x = rng.standard_normal(L).astype(np.float32)
        y = rng.standard_normal(L).astype(np.float32)
        ref = float(np.sum((x.astype(np.float64) - y.astype(np.float64)) ** 2))
        assert oracle_mod.dtw(x, y, 0) == pytest.approx(ref, rel=1e-13)
        # DTW never exceeds the squared Euclidean distance for equal lengths
        assert oracle_mod.dtw(x, y, -1) <= ref * (1 + 1e-13)


def test_single_element_closed_form(oracle_mod):
    rng = _rng(15)
    for n in (1, 2, 9, 50):
        x = rng.standard_normal(n).astype(np.float32)
        y1 = rng.standard_normal(1).astype(np.float32)
        ref = float(np.sum((x.astype(np.float64) - float(y1[0])) ** 2))
        assert oracle_mod.dtw(x, y1) == pytest.approx(ref, rel=1e-13)
        assert oracle_mod.dtw(y1, x) == pytest.approx(ref, rel=1e-13)


def test_monotone_in_window_and_saturation(oracle_mod):
    rng = _rng(16)
    for _ in range(10):
        L = int(rng.integers(5, 80))
        x = rng.standard_normal(L).astype(np.float32)
        y = rng.standard_normal(L).astype(np.float32)
        vals = [oracle_mod.dtw(x, y, w) for w in range(0, L + 2)]
        assert all(b <= a for a, b in zip(vals, vals[1:]))
        unc = oracle_mod.dtw(x, y, -1)
        assert vals[L - 1] == unc and vals[-1] == unc


def test_band_readings_for_unequal_lengths(oracle_mod):
    rng = _rng(17)
    x = rng.standard_normal(30).astype(np.float32)
    y = rng.standard_normal(20).astype(np.float32)
    # strict band narrower than |n-m| cannot reach (n, m)
    assert math.isinf(oracle_mod.dtw(x, y, 5, strict=True))
    # the default reading widens the band to |n-m| = 10
    assert oracle_mod.dtw(x, y, 5) == oracle_mod.dtw(x, y, 10, strict=True)
    assert oracle_mod.dtw(x, y, 12) == oracle_mod.dtw(x, y, 12, strict=True)


def test_band_cells_closed_form(oracle_mod):
    for L, w in [(128, 128), (128, 12), (512, 51), (256, 25), (10, 0), (10, 3)]:
        we = min(w, L - 1)
        assert oracle_mod.band_cells(L, L, w) == L * (2 * we + 1) - we * (we + 1)
    assert oracle_mod.band_cells(512, 512, 51) == 50084
    assert oracle_mod.band_cells(128, 128, 12) == 3044


def test_float_mirror_close_to_double(oracle_mod):
    vals, offs = synth.random_walk_set(20, 128, seed=0)
    a, b = np.triu_indices(20, 1)
    ref = oracle_mod.pairs(vals, offs, a, b, 12)
    f32 = oracle_mod.pairs_f32_mirror(vals, offs, a, b, 12)
    rel = np.abs(f32.astype(np.float64) - ref) / np.maximum(ref, 1e-30)
    assert rel.max() < 1e-5


def test_pairwise_matrix_matches_single_pairs(oracle_mod):
    lens = synth.ragged_lengths(9, 3, 40, seed=5)
    vals, offs = synth.five_class_set(9, lens, seed=5)[:2]
    D = oracle_mod.pairwise(vals, offs, 4)
    assert np.all(np.diag(D) == 0.0)
    assert np.array_equal(D, D.T)
    for i, j in [(0, 1), (3, 7), (8, 2)]:
        x = vals[offs[i]:offs[i + 1]]
        y = vals[offs[j]:offs[j + 1]]
        assert D[i, j] == oracle_mod.dtw(x, y, 4)
    q = vals[offs[4]:offs[5]]
    assert np.array_equal(oracle_mod.query(q, vals, offs, 4), D[4])


@pytest.mark.parametrize("strict", [False, True])
def test_pair_lists_with_their_own_windows_match_brute_force(oracle_mod, strict):
    """pairs_w (a window per pair, the reference of the ragged and pair-list tests) against the
    enumeration of every warping path on a tiny ragged set, in both orders of each pair; with one
    window for every pair it equals pairs."""
    rng = _rng(21)
    lens = np.array([1, 2, 3, 4, 5, 6, 6, 3])
    vals = rng.standard_normal(int(lens.sum())).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    a, b = np.meshgrid(np.arange(len(lens)), np.arange(len(lens)), indexing="ij")
    a, b = a.ravel(), b.ravel()
    w = rng.integers(-1, 7, len(a))
    got = oracle_mod.pairs_w(vals, offs, a, b, w, strict)
    for t in range(len(a)):
        x = vals[offs[a[t]]:offs[a[t] + 1]]
        y = vals[offs[b[t]]:offs[b[t] + 1]]
        ref = brute.dtw_by_paths(x, y, int(w[t]), strict)
        if math.isinf(ref):
            assert math.isinf(got[t]), (a[t], b[t], w[t])
        else:
            assert got[t] == pytest.approx(ref, rel=1e-12, abs=1e-12), (a[t], b[t], w[t])
    for wc in (-1, 0, 2):
        assert np.array_equal(oracle_mod.pairs_w(vals, offs, a, b, np.full(len(a), wc), strict),
                              oracle_mod.pairs(vals, offs, a, b, wc, strict))


# ---------------------------------------------------------- k-medoids pins


def _dist_matrix(seed, p):
    pts = _rng(seed).standard_normal((p, 2))
    return np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))


def test_A_matrix_example_from_paper():
    with open(os.path.join(GOLDEN, "a_matrix_example.json")) as f:
        g = json.load(f)
    p, k = g["p"], g["k"]
    medoids = [c - 1 for c in g["centroids_1based"]]
    labels = [0] * p
    for c, members in enumerate(g["clusters_1based"]):
        for j in members:
            labels[j - 1] = c
    A = brute.labels_to_A(labels, medoids)
    nz = sorted((i + 1, j + 1) for i in range(p) for j in range(p) if A[i][j])
    assert nz == sorted(tuple(t) for t in g["A_nonzero_1based"])
    assert brute.check_A_constraints(A, k)


def test_cost_identity_with_mip_objective(oracle_mod):
    D = _dist_matrix(3, 9)
    r = oracle_mod.kmedoids(D, 3, [0, 1, 2])
    A = brute.labels_to_A(list(r["labels"]), list(r["medoids"]))
    assert brute.check_A_constraints(A, 3)
    assert brute.mip_objective(D, A) == pytest.approx(r["cost"], rel=1e-14)
    assert oracle_mod.cluster_cost(D, r["medoids"], r["labels"]) == r["cost"]


def test_kmedoids_bounded_by_global_optimum_and_fixed_point(oracle_mod):
    for seed in range(6):
        p = 8 + seed % 4
        D = _dist_matrix(100 + seed, p)
        for k in (2, 3):
            opt, opt_set = brute.kmedoids_optimum(D, k)
            init = synth.init_medoids(p, k, seed)
            r = oracle_mod.kmedoids(D, k, init)
            assert r["cost"] >= opt * (1 - 1e-14)
            # starting at the optimum is a fixed point
            f = oracle_mod.kmedoids(D, k, opt_set)
            assert sorted(f["medoids"]) == sorted(opt_set)
            assert f["iters"] == 1
            assert f["cost"] == pytest.approx(opt, rel=1e-14)


def test_kmedoids_cost_non_increasing_per_sweep(oracle_mod):
    D = _dist_matrix(7, 60)
    init = synth.init_medoids(60, 4, 7)
    costs = [oracle_mod.kmedoids(D, 4, init, max_iter=s)["cost"] for s in range(1, 10)]
    assert all(b <= a * (1 + 1e-14) for a, b in zip(costs, costs[1:]))


def test_kmedoids_assignment_rules(oracle_mod):
    # exact ties in the assignment go to the smallest cluster index; a medoid
    # labels itself even when another medoid is at distance 0
    D = np.array([[0, 1, 1, 5], [1, 0, 0, 5], [1, 0, 0, 5], [5, 5, 5, 0]], dtype=np.float64)
    r = oracle_mod.kmedoids(D, 2, [1, 2], max_iter=1)
    assert list(r["labels"][1:3]) == [0, 1]
    assert r["labels"][0] == 0 and r["labels"][3] == 0


def _line_D(pos):
    x = np.asarray(pos, dtype=np.float64)
    return np.abs(x[:, None] - x[None, :])


def test_kmedoids_update_tie_keeps_the_current_medoid(oracle_mod):
    # Two groups on a line, 0 1 2 3 and 100 101 102 103.  In each group the two inner
    # members have equal within-cluster sums (1+0+1+2 = 2+1+0+1 = 4), the outer ones 6.
    D = _line_D([0, 1, 2, 3, 100, 101, 102, 103])
    # the current medoids (the larger index of each tied pair) attain the minimum: kept,
    # so the first sweep changes nothing (taking the smallest index would move to 1, 5)
    r = oracle_mod.kmedoids(D, 2, [2, 6])
    assert r["medoids"].tolist() == [2, 6] and r["iters"] == 1
    assert r["cost"] == 8.0 and r["labels"].tolist() == [0, 0, 0, 0, 1, 1, 1, 1]
    # current medoids outside the minima: the smallest tied index wins (taking the last
    # minimum would give 2, 6), and the second sweep keeps it
    r = oracle_mod.kmedoids(D, 2, [0, 7])
    assert r["medoids"].tolist() == [1, 5] and r["iters"] == 2
    r = oracle_mod.kmedoids(D, 2, [3, 4], max_iter=1)
    assert r["medoids"].tolist() == [1, 5] and r["iters"] == 1
    # the near-tie detector reports the exact tie
    assert r["min_margin"] == 0.0


def test_planted_clusters_recovered(oracle_mod):
    rng = _rng(21)
    centres = np.array([[0, 0], [20, 0], [0, 20], [20, 20]])
    pts = np.concatenate([c + rng.standard_normal((15, 2)) for c in centres])
    D = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    r = oracle_mod.kmedoids(D, 4, [0, 1, 2, 15 * 3])  # three in one cluster
    truth = np.repeat(np.arange(4), 15)
    # recovered partition equals the planted one up to relabelling
    for c in range(4):
        members = set(np.where(r["labels"] == c)[0])
        assert any(members == set(np.where(truth == t)[0]) for t in range(4))


def test_kmedoids_medoid_minimises_within_cluster_sum(oracle_mod):
    D = _dist_matrix(31, 40)
    r = oracle_mod.kmedoids(D, 3, synth.init_medoids(40, 3, 31))
    for c in range(3):
        mem = np.where(r["labels"] == c)[0]
        S = D[np.ix_(mem, mem)].sum(1)
        assert D[r["medoids"][c], mem].sum() == pytest.approx(S.min(), rel=1e-14)


# ------------------------------------------------------------ input recipe


def test_synth_shapes_and_normalisation():
    v, o, cls = synth.five_class_set(10, 64, seed=1)
    assert o.tolist() == list(range(0, 641, 64))
    for i in range(10):
        s = v[o[i]:o[i + 1]].astype(np.float64)
        assert abs(s.mean()) < 1e-5 and abs(s.std() - 1) < 1e-5
    assert cls.tolist() == [i % 5 for i in range(10)]
    v2, o2 = synth.random_walk_set(3, 17, seed=4)
    v3, o3 = synth.random_walk_set(3, 17, seed=4)
    assert np.array_equal(v2, v3) and o2[-1] == 51
    m = synth.init_medoids(50, 3, 0)
    assert len(set(m.tolist())) == 3 and all(0 <= t < 50 for t in m)
    # splitmix64 reference value (seed 0 -> first output 0xE220A8397B1DCDAF)
    assert synth.splitmix64(0)[1] == 0xE220A8397B1DCDAF


def test_init_medoids_for_k_are_a_prefix_of_one_shuffle():
    # the shuffle does not depend on k, so the medoids for k are the first k of those
    # for any larger k (the elbow curve draws once for kmax); a brute-force check that
    # the permutation is a permutation
    full = synth.init_medoids(97, 97, 5)
    assert sorted(full.tolist()) == list(range(97))
    for k in (1, 2, 7, 40, 96):
        assert synth.init_medoids(97, k, 5).tolist() == full[:k].tolist()

"""The clustering MIP export (host side): the model of the paper's integer program, its LP
text, the assignment matrix A of a clustering, and a solve through SciPy's HiGHS interface
pinned to the brute-force optimum over all k-subsets of centroids."""

import numpy as np
import pytest

import oracle.brute as brute
from paper_2307_04904_gb300 import mip


def _rand_D(p, seed):
    rng = np.random.default_rng(seed)
    pts = rng.standard_normal((p, 2))
    return ((pts[:, None] - pts[None]) ** 2).sum(-1)


def _feasible(A, k):
    p = A.shape[0]
    return (np.trace(A) == k and (A.sum(0) == 1).all()
            and all(A[i, j] <= A[i, i] for i in range(p) for j in range(p)))


def test_assignment_matrix_reproduces_the_papers_example():
    # the paper's example output: series 1, 2, 5 in the cluster of centroid 2 and series
    # 3, 4 in that of centroid 4 (1-based), i.e. A22 = A21 = A25 = 1 and A44 = A43 = 1
    A = mip.assignment_matrix([1, 3], [0, 0, 1, 1, 0])
    want = np.zeros((5, 5), dtype=np.int8)
    want[1, [0, 1, 4]] = 1
    want[3, [2, 3]] = 1
    assert np.array_equal(A, want) and _feasible(A, 2)
    # the objective of A is the clustering cost sum_j D[M_label_j, j]
    D = _rand_D(5, 0)
    assert (D * A).sum() == pytest.approx(D[1, 0] + D[1, 1] + D[1, 4] + D[3, 2] + D[3, 3])


def test_model_arrays_accept_exactly_the_feasible_assignments():
    pytest.importorskip("scipy")
    p, k = 4, 2
    c, A_eq, b_eq, A_ub, b_ub = mip.model_arrays(_rand_D(p, 1), k)
    assert A_eq.shape == (p + 1, p * p) and A_ub.shape == (p * (p - 1), p * p)
    n_ok = 0
    for bits in range(1 << (p * p)):  # every binary A of a 4 x 4 problem
        x = np.array([(bits >> t) & 1 for t in range(p * p)], dtype=np.float64)
        ok = np.allclose(A_eq @ x, b_eq) and (A_ub @ x <= b_ub + 1e-12).all()
        assert ok == _feasible(x.reshape(p, p).astype(np.int8), k)
        n_ok += ok
    # feasible A: choose the k centroids, then each of the p - k others joins one of them
    assert n_ok == 6 * 2 ** (p - k)


@pytest.mark.parametrize("p,k,seed", [(6, 1, 2), (8, 2, 3), (10, 3, 4), (12, 4, 5)])
def test_solve_reaches_the_brute_force_optimum(p, k, seed):
    pytest.importorskip("scipy.optimize")
    D = _rand_D(p, seed)
    res = mip.solve(D, k)
    opt, _ = brute.kmedoids_optimum(D, k)
    assert res["cost"] == pytest.approx(opt, rel=1e-9, abs=1e-12)
    assert _feasible(res["A"], k) and len(res["medoids"]) == k
    assert np.array_equal(mip.assignment_matrix(res["medoids"], res["labels"]), res["A"])


def test_write_lp_text(tmp_path):
    D = np.array([[0.0, 1.5, 2.0], [1.5, 0.0, 0.25], [2.0, 0.25, 0.0]])
    f = tmp_path / "m.lp"
    mip.write_lp(D, 1, str(f))
    text = f.read_text().splitlines()
    assert text[1] == "Minimize" and text[-1] == "End"
    obj = " ".join(text[2:text.index("Subject To")])
    assert obj.split()[0] == "obj:"
    terms = obj.replace("obj:", "").replace("+", " ").split()
    coef = dict(zip(terms[1::2], map(float, terms[0::2])))
    assert coef == {f"a_{i}_{j}": D[i, j] for i in range(3) for j in range(3)}
    assert " centroids: a_0_0 + a_1_1 + a_2_2 = 1" in text
    assert " one_1: a_0_1 + a_1_1 + a_2_1 = 1" in text
    assert " member_2_0: a_2_0 - a_2_2 <= 0" in text
    assert sum(line.startswith(" member_") for line in text) == 6
    binary = " ".join(text[text.index("Binary") + 1:-1]).split()
    assert sorted(binary) == sorted(f"a_{i}_{j}" for i in range(3) for j in range(3))


def test_rejects_bad_input(tmp_path):
    with pytest.raises(ValueError):
        mip.write_lp(np.zeros((3, 4)), 1, str(tmp_path / "x.lp"))
    with pytest.raises(ValueError):
        mip.write_lp(np.array([[0.0, np.inf], [np.inf, 0.0]]), 1, str(tmp_path / "x.lp"))
    with pytest.raises(ValueError):
        mip.write_lp(np.zeros((3, 3)), 4, str(tmp_path / "x.lp"))

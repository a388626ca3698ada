"""The paper's integer program for clustering, exported for an external solver.

Given the DTW matrix D (p x p) and k, the paper (Mathematical background, the
clustering paragraphs and equations) clusters with a binary p x p matrix A:
A_ij = 1 when series j belongs to the cluster whose centroid is series i.

    minimise    sum_i sum_j D_ij A_ij
    subject to  sum_i A_ii = k                  (k centroids)
                sum_i A_ij = 1    for every j   (each series in exactly one cluster)
                A_ij <= A_ii      for every i, j (members only in centroid rows)

The model stays on the host: it has p^2 binary variables, so it is meant for
the small sets the paper recommends it for (few, long series).

* :func:`write_lp` writes the model in the LP text format that MIP solvers
  (HiGHS, CBC, SCIP, CPLEX, Gurobi) read.
* :func:`model_arrays` returns it as sparse matrices.
* :func:`solve` hands it to SciPy's MILP interface (HiGHS) where SciPy is installed.
* :func:`assignment_matrix` turns medoids and labels (from ``kmedoids_fit``,
  ``kmedoids_pam`` or :func:`solve`) into A, so that sum_ij D_ij A_ij is the
  clustering cost.

D comes from the device once (``dtw_pairwise`` output); nothing here runs on the GPU.
"""

from __future__ import annotations

import numpy as np


def _host_matrix(D) -> np.ndarray:
    if hasattr(D, "detach"):  # a torch tensor, possibly on the GPU
        D = D.detach().cpu().numpy()
    D = np.asarray(D, dtype=np.float64)
    if D.ndim != 2 or D.shape[0] != D.shape[1]:
        raise ValueError("D must be a square matrix")
    if not np.all(np.isfinite(D)):
        raise ValueError("D must be finite (a strict-band +inf has no place in the objective)")
    return D


def _check_k(p: int, k: int):
    if not 1 <= k <= p:
        raise ValueError(f"need 1 <= k <= p (p = {p}, k = {k})")


def _var(i: int, j: int) -> str:
    return f"a_{i}_{j}"


def _wrap(terms, first: str, per_line: int = 6) -> list[str]:
    """Expression lines of at most `per_line` terms (LP lines stay short)."""
    lines, cur = [], first
    for t, term in enumerate(terms):
        cur += " " + term
        if (t + 1) % per_line == 0:
            lines.append(cur)
            cur = "   "
    if cur.strip():
        lines.append(cur)
    return lines


def write_lp(D, k: int, path: str) -> None:
    """Write the clustering MIP in LP format to `path` (variables a_i_j = A_ij)."""
    D = _host_matrix(D)
    p = D.shape[0]
    _check_k(p, k)
    out = [f"\\ DTW clustering MIP: p = {p} series, k = {k} clusters", "Minimize"]
    obj = []
    for t, (i, j) in enumerate((i, j) for i in range(p) for j in range(p)):
        v = float(D[i, j])
        sign = "-" if v < 0 else ("+" if t else "")
        obj.append(f"{sign} {abs(v)!r} {_var(i, j)}".strip())
    out += _wrap(obj, " obj:")
    out.append("Subject To")
    out += _wrap([("+ " if i else "") + _var(i, i) for i in range(p)], " centroids:")
    out[-1] += f" = {k}"
    for j in range(p):
        out += _wrap([("+ " if i else "") + _var(i, j) for i in range(p)], f" one_{j}:")
        out[-1] += " = 1"
    for i in range(p):
        for j in range(p):
            if i != j:
                out.append(f" member_{i}_{j}: {_var(i, j)} - {_var(i, i)} <= 0")
    out.append("Binary")
    out += _wrap([_var(i, j) for i in range(p) for j in range(p)], "")
    out.append("End")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


def model_arrays(D, k: int):
    """(c, A_eq, b_eq, A_ub, b_ub) of the MIP over x = A flattened row-major (x[i p + j] = A_ij):
    minimise c.x subject to A_eq x = b_eq, A_ub x <= b_ub, x binary.  Sparse (scipy) matrices."""
    from scipy import sparse

    D = _host_matrix(D)
    p = D.shape[0]
    _check_k(p, k)
    c = D.reshape(-1).copy()
    diag = np.arange(p) * (p + 1)
    # row 0: sum_i A_ii = k; rows 1 + j: sum_i A_ij = 1
    rows = np.concatenate([np.zeros(p, np.int64), 1 + np.tile(np.arange(p), p)])
    cols = np.concatenate([diag, np.arange(p * p)])
    A_eq = sparse.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(p + 1, p * p))
    b_eq = np.concatenate([[float(k)], np.ones(p)])
    # A_ij - A_ii <= 0 for i != j
    ii, jj = np.nonzero(~np.eye(p, dtype=bool))
    r = np.arange(len(ii))
    A_ub = sparse.csr_matrix(
        (np.concatenate([np.ones(len(ii)), -np.ones(len(ii))]),
         (np.concatenate([r, r]), np.concatenate([ii * p + jj, ii * (p + 1)]))),
        shape=(len(ii), p * p))
    return c, A_eq, b_eq, A_ub, np.zeros(len(ii))


def assignment_matrix(medoids, labels, p: int | None = None) -> np.ndarray:
    """A (p x p, int8) from medoids M (k) and labels (p): A[M[label_j], j] = 1."""
    if hasattr(medoids, "detach"):
        medoids = medoids.detach().cpu().numpy()
    if hasattr(labels, "detach"):
        labels = labels.detach().cpu().numpy()
    M = np.asarray(medoids, dtype=np.int64)
    lab = np.asarray(labels, dtype=np.int64)
    p = len(lab) if p is None else p
    A = np.zeros((p, p), dtype=np.int8)
    A[M[lab], np.arange(p)] = 1
    return A


def solve(D, k: int, time_limit: float | None = None) -> dict:
    """Solve the MIP with SciPy's HiGHS interface: dict(medoids, labels, cost, A, status).
    Medoids are the centroids in increasing index order; labels index into them."""
    from scipy.optimize import Bounds, LinearConstraint, milp

    D = _host_matrix(D)
    p = D.shape[0]
    c, A_eq, b_eq, A_ub, b_ub = model_arrays(D, k)
    opts = {} if time_limit is None else {"time_limit": float(time_limit)}
    res = milp(c, integrality=np.ones(p * p), bounds=Bounds(0, 1),
               constraints=[LinearConstraint(A_eq, b_eq, b_eq),
                            LinearConstraint(A_ub, -np.inf, b_ub)], options=opts)
    if res.x is None:
        raise RuntimeError(f"MILP solver found no solution: {res.message}")
    A = np.rint(res.x).astype(np.int8).reshape(p, p)
    medoids = np.nonzero(np.diag(A))[0]
    where = {int(m): c for c, m in enumerate(medoids)}
    labels = np.array([where[int(np.argmax(A[:, j]))] for j in range(p)], dtype=np.int64)
    return dict(medoids=medoids, labels=labels, cost=float((D * A).sum()), A=A,
                status=res.status, message=res.message)

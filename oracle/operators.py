"""The constraint operator A(X) = [<A_i, X>]_i and its adjoint A^T(y) = sum_i y_i A_i.

Section 1 (eq. sdp-pd) states the SDP with this operator; (A3) / Assumption
mvp2 name its two products; (Newt-eps) writes it as the matrix whose rows are
svec(A_i).  Each function below builds the matrices A_i from the storage
convention of ``workloads`` and applies the definition literally.
"""
from __future__ import annotations

import numpy as np

from .linalg import smat, svec


def constraint_matrix(prob, i: int) -> np.ndarray:
    """A_i as an explicit symmetric n x n matrix."""
    n = prob.n
    if prob.kind == "diag":
        A = np.zeros((n, n))
        A[i, i] = 1.0
        return A
    if prob.kind == "sparse":
        A = np.zeros((n, n))
        sel = np.nonzero(prob.a_con == i)[0]
        for k in sel:
            r, c, v = int(prob.a_row[k]), int(prob.a_col[k]), float(prob.a_val[k])
            A[r, c] += v
            if r != c:
                A[c, r] += v
        return A
    if prob.kind == "dense":
        return smat(prob.a_dense[i], n)
    raise ValueError(prob.kind)


def A_op(prob, X: np.ndarray) -> np.ndarray:
    """A(X) = [<A_i, X>]_{i=1..m} (eq. sdp-pd)."""
    X = np.asarray(X, dtype=np.float64)
    if prob.kind == "diag":
        return np.diag(X).copy()
    if prob.kind == "sparse":
        w = np.where(prob.a_row == prob.a_col, 1.0, 2.0)
        out = np.zeros(prob.m)
        np.add.at(out, prob.a_con, prob.a_val * w * X[prob.a_row, prob.a_col])
        return out
    if prob.kind == "dense":
        return prob.a_dense @ svec(X)
    raise ValueError(prob.kind)


def At_op(prob, y: np.ndarray) -> np.ndarray:
    """A^T(y) = sum_i y_i A_i (eq. sdp-pd, dual constraint)."""
    n = prob.n
    y = np.asarray(y, dtype=np.float64)
    if prob.kind == "diag":
        return np.diag(y)
    if prob.kind == "sparse":
        Y = np.zeros((n, n))
        v = prob.a_val * y[prob.a_con]
        np.add.at(Y, (prob.a_row, prob.a_col), v)
        off = prob.a_row != prob.a_col
        np.add.at(Y, (prob.a_col[off], prob.a_row[off]), v[off])
        return Y
    if prob.kind == "dense":
        return smat(prob.a_dense.T @ y, n)
    raise ValueError(prob.kind)


def A_matrix(prob) -> np.ndarray:
    """The m x n(n+1)/2 matrix whose rows are svec(A_i), built entry by entry."""
    return np.array([svec(constraint_matrix(prob, i)) for i in range(prob.m)])


def row_norm_scale(prob) -> float:
    """s_A = ||A||_F^2 / m, the mean squared row norm of the svec-row matrix."""
    if prob.kind == "diag":
        return 1.0
    if prob.kind == "dense":
        return float(np.sum(prob.a_dense ** 2) / prob.m)
    # merge duplicate (con, row, col) entries, then sum v^2 (diagonal) or 2 v^2 (off-diagonal)
    key = np.stack([prob.a_con, prob.a_row, prob.a_col], axis=1).astype(np.int64)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    vals = np.zeros(uniq.shape[0])
    np.add.at(vals, inv.reshape(-1), prob.a_val)
    w = np.where(uniq[:, 1] == uniq[:, 2], 1.0, 2.0)
    return float(np.sum(w * vals * vals) / prob.m)

"""Symmetric vectorisation and symmetric Kronecker product (paper, Notations).

svec(X) stacks the lower triangle of X column by column and multiplies the
off-diagonal entries by sqrt(2), so that <X, S> = svec(X) . svec(S).  For a
non-symmetric argument, svec takes the symmetric part (Appendix A:
svec(X) = Psi^T vec(X) = 1/2 Psi^T vec(X + X^T)).  Psi_n is the orthonormal
n^2 x n(n+1)/2 basis of vec(S^n); vec is column stacking, and the Kronecker
product satisfies (B kron A) vec(X) = vec(A X B^T).  The symmetric Kronecker
product of A, B (n x r) is 1/2 Psi_n^T (A kron B + B kron A) Psi_r.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def vec(X: np.ndarray) -> np.ndarray:
    """Column-stacking vectorisation."""
    return np.asarray(X).reshape(-1, order="F").copy()


def unvec(x: np.ndarray, n: int, r: int | None = None) -> np.ndarray:
    r = n if r is None else r
    return np.asarray(x).reshape((n, r), order="F").copy()


def sym(X: np.ndarray) -> np.ndarray:
    return 0.5 * (X + X.T)


def _svec_index(n: int):
    """(row, col) of each svec position: lower triangle, column by column."""
    rows, cols = [], []
    for j in range(n):
        for i in range(j, n):
            rows.append(i)
            cols.append(j)
    return np.array(rows), np.array(cols)


_IDX_CACHE: dict = {}


def svec_index(n: int):
    if n not in _IDX_CACHE:
        _IDX_CACHE[n] = _svec_index(n)
    return _IDX_CACHE[n]


def svec(X: np.ndarray) -> np.ndarray:
    """svec of the symmetric part, lower triangle column by column, off-diagonals * sqrt(2)."""
    S = sym(np.asarray(X, dtype=np.float64))
    rows, cols = svec_index(S.shape[0])
    return S[rows, cols] * np.where(rows == cols, 1.0, SQRT2)


def smat(x: np.ndarray, n: int) -> np.ndarray:
    """Inverse of svec on symmetric matrices."""
    rows, cols = svec_index(n)
    v = np.asarray(x, dtype=np.float64) / np.where(rows == cols, 1.0, SQRT2)
    X = np.zeros((n, n))
    X[rows, cols] = v
    X[cols, rows] = v
    return X


def psi(n: int) -> np.ndarray:
    """Orthonormal basis Psi_n with vec(X) = Psi_n svec(X) for symmetric X."""
    N = n * (n + 1) // 2
    P = np.zeros((n * n, N))
    k = 0
    for j in range(n):
        P[j + j * n, k] = 1.0
        k += 1
        for i in range(j + 1, n):
            P[i + j * n, k] = 1.0 / SQRT2
            P[j + i * n, k] = 1.0 / SQRT2
            k += 1
    return P


def skron(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Symmetric Kronecker product 1/2 Psi_n^T (A kron B + B kron A) Psi_r."""
    n, r = A.shape
    return 0.5 * psi(n).T @ (np.kron(A, B) + np.kron(B, A)) @ psi(r)

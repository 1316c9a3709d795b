"""Nesterov-Todd scaling and the Newton direction of (Newt-eps) by its plain definition.

Section 1, eq. newt: the Newton subproblem with scaling point W and residuals
(b~, C~).  Section 3, (Newt-eps): its KKT equations

    [ -(W (x)s W)^{-1}  A^T ] [ svec dX ]   [ svec C~ ]
    [        A           0  ] [   dy    ] = [    b~   ],     dS = C~ - A^T(dy).

Eliminating svec dX = (W (x)s W)(A^T dy - c) gives the m x m Schur system
    M dy = b~ + A(W C~ W),    M_ij = <A_i, W A_j W>,
then dX = W (A^T(dy) - C~) W.  ``newton_direct`` is that elimination with a
LAPACK Cholesky of M; ``newton_kkt_dense`` builds the full KKT matrix of
(Newt-eps) explicitly (tiny n only) and solves it by LU.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .linalg import skron, svec, smat, svec_index
from .operators import A_matrix, A_op, At_op, constraint_matrix


def sqrtm_psd(X: np.ndarray) -> np.ndarray:
    w, U = np.linalg.eigh(0.5 * (X + X.T))
    return (U * np.sqrt(np.maximum(w, 0.0))) @ U.T


def inv_sqrtm_pd(X: np.ndarray) -> np.ndarray:
    w, U = np.linalg.eigh(0.5 * (X + X.T))
    return (U / np.sqrt(w)) @ U.T


def nt_scaling(X: np.ndarray, S: np.ndarray) -> np.ndarray:
    """W = X^{1/2} (X^{1/2} S X^{1/2})^{-1/2} X^{1/2} (eq. newt, NT scaling).

    Evaluated as W = L (L^T S L)^{-1/2} L^T with X = L L^T: L = X^{1/2} O for
    an orthogonal O, and O cancels, so this is the same matrix without a
    square root of X.
    """
    L = np.linalg.cholesky(0.5 * (X + X.T))
    T = L.T @ S @ L
    W = L @ inv_sqrtm_pd(T) @ L.T
    return 0.5 * (W + W.T)


def schur_matrix_by_columns(prob, W: np.ndarray) -> np.ndarray:
    """M_ij = <A_i, W A_j W>, i.e. A (W (x)s W) A^T, one column per constraint: W A_j W is
    formed explicitly and A(.) applied to it."""
    m = prob.m
    cols = np.empty((m, m))
    for j in range(m):
        cols[:, j] = A_op(prob, W @ constraint_matrix(prob, j) @ W)
    return 0.5 * (cols + cols.T)


def _single_entry_constraints(prob) -> bool:
    return prob.kind == "sparse" and len(prob.a_con) == prob.m and np.array_equal(prob.a_con, np.arange(prob.m))


def schur_matrix(prob, W: np.ndarray, block: int = 100) -> np.ndarray:
    """M_ij = <A_i, W A_j W>, i.e. A (W (x)s W) A^T.

    DIAG: <e_i e_i^T, W e_j e_j^T W> = W_ij^2.  Dense svec rows: the same columns as
    ``schur_matrix_by_columns``, for ``block`` constraints at a time (W A_j W by one batched
    product, svec, then A times the block).  Constraints with one stored entry each (A_i =
    v_i s_i (e_r e_c^T + e_c e_r^T), s_i = 1/2 on the diagonal, 1 off it; matrix completion):
    <e_a e_b^T, W e_p e_q^T W> = W_ap W_qb summed over the four terms gives
    M_ij = 2 v_i s_i v_j s_j (W_{r_i r_j} W_{c_i c_j} + W_{r_i c_j} W_{c_i r_j}).
    Any other sparse storage: ``schur_matrix_by_columns``."""
    m = prob.m
    if prob.kind == "diag":
        return W * W
    if prob.kind == "dense":
        n = prob.n
        rows, cols = svec_index(n)
        wgt = np.where(rows == cols, 1.0, np.sqrt(2.0))
        M = np.empty((m, m))
        for j0 in range(0, m, block):
            j1 = min(m, j0 + block)
            Ab = np.zeros((j1 - j0, n, n))
            vals = prob.a_dense[j0:j1] / wgt
            Ab[:, rows, cols] = vals
            Ab[:, cols, rows] = vals
            WAW = np.matmul(np.matmul(W, Ab), W)
            M[:, j0:j1] = prob.a_dense @ (WAW[:, rows, cols] * wgt).T
        return 0.5 * (M + M.T)
    if _single_entry_constraints(prob):
        r = prob.a_row.astype(np.int64)
        c = prob.a_col.astype(np.int64)
        v = prob.a_val * np.where(r == c, 0.5, 1.0)
        M = np.empty((m, m))
        for i0 in range(0, m, 1024):          # row blocks bound the temporaries
            i1 = min(m, i0 + 1024)
            ri, ci = r[i0:i1], c[i0:i1]
            M[i0:i1] = 2.0 * np.outer(v[i0:i1], v) * (W[np.ix_(ri, r)] * W[np.ix_(ci, c)] +
                                                       W[np.ix_(ri, c)] * W[np.ix_(ci, r)])
        return 0.5 * (M + M.T)
    return schur_matrix_by_columns(prob, W)


def schur_solver(M: np.ndarray):
    """Solver for M dy = rhs: LAPACK Cholesky; if M is numerically indefinite
    (cond(M) grows like 1/mu^2, Section 1), a symmetric eigensolve with the
    eigenvalues floored at eps * lambda_max."""
    try:
        cf = sla.cho_factor(M, lower=True)
        return lambda rhs: sla.cho_solve(cf, rhs)
    except np.linalg.LinAlgError:
        w, U = np.linalg.eigh(M)
        w = np.maximum(w, np.finfo(float).eps * w[-1])
        return lambda rhs: U @ ((U.T @ rhs) / w)


def newton_direct(prob, W: np.ndarray, Ct: np.ndarray, bt: np.ndarray, M: np.ndarray | None = None,
                  refine: int = 2, WCW: np.ndarray | None = None):
    """Newton direction of (Newt-eps) with eps = 0 by Schur-complement elimination.

    The Cholesky solve of M is followed by ``refine`` steps of classical
    iterative refinement on the equation A(dX) = b~ (dX = W(A^T dy - C~)W),
    which the ill-conditioning of M at small mu (Section 1) makes necessary
    for a direction that is exact to working precision.
    ``WCW`` may pass the product W C~ W when the caller has it in a more
    accurate closed form (the outer loop does: W C~ W = W R_d W - R_c).
    Returns (dX, dy, dS) with dS = C~ - A^T(dy) (Section 3, after Newt-eps).
    """
    if M is None:
        M = schur_matrix(prob, W)
    solve = schur_solver(M)
    if WCW is None:
        WCW = W @ Ct @ W
    dy = solve(bt + A_op(prob, WCW))
    for _ in range(refine):
        dX = W @ At_op(prob, dy) @ W - WCW
        dy = dy + solve(bt - A_op(prob, dX))
    Aty = At_op(prob, dy)
    dX = W @ Aty @ W - WCW
    dX = 0.5 * (dX + dX.T)
    dS = Ct - Aty
    return dX, dy, dS


def kkt_matrix(prob, W: np.ndarray) -> np.ndarray:
    """The full (Newt-eps) matrix [[-(W (x)s W)^{-1}, A^T], [A, 0]] (tiny n)."""
    WW = skron(W, W)
    A = A_matrix(prob)
    N = WW.shape[0]
    K = np.zeros((N + prob.m, N + prob.m))
    K[:N, :N] = -np.linalg.inv(WW)
    K[:N, N:] = A.T
    K[N:, :N] = A
    return K


def newton_kkt_dense(prob, W: np.ndarray, Ct: np.ndarray, bt: np.ndarray):
    """Solve (Newt-eps) exactly with the explicit KKT matrix (dense LU)."""
    K = kkt_matrix(prob, W)
    N = K.shape[0] - prob.m
    sol = np.linalg.solve(K, np.concatenate([svec(Ct), bt]))
    dX = smat(sol[:N], prob.n)
    dy = sol[N:]
    return dX, dy, Ct - At_op(prob, dy)


def newt_eps_residual(prob, W: np.ndarray, Ct: np.ndarray, bt: np.ndarray,
                      dX: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """Residual vector of (Newt-eps): [-(W(x)sW)^{-1} svec dX + A^T dy - c ; A dX - b~].

    (W (x)s W)^{-1} svec(dX) = svec(W^{-1} dX W^{-1}).
    """
    Wi = np.linalg.inv(W)
    top = -Wi @ dX @ Wi + At_op(prob, dy) - Ct
    return np.concatenate([svec(top), A_op(prob, dX) - bt])

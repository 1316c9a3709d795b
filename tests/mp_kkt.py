"""High-precision (mpmath, 60 digits) solve of the (Newt-eps) KKT system for tiny n.

Test helper only: builds [[-(W (x)s W)^{-1}, A^T], [A, 0]] from the FP64 inputs
converted exactly to mpmath numbers, using (W (x)s W)^{-1} = W^{-1} (x)s W^{-1}
column by column as svec(W^{-1} E_k W^{-1}), and solves it by LU.
"""
import math

import mpmath as mp
import numpy as np


def _svec_positions(n):
    return [(i, j) for j in range(n) for i in range(j, n)]


def _mat(M):
    return mp.matrix([[mp.mpf(float(v)) for v in row] for row in np.asarray(M)])


def newton_kkt_mp(A_rows: np.ndarray, W: np.ndarray, Ct: np.ndarray, bt: np.ndarray, dps: int = 60):
    """Return (dX, dy) in float64 from a `dps`-digit KKT solve.  A_rows: m x n(n+1)/2 svec rows."""
    mp.mp.dps = dps
    n = W.shape[0]
    pos = _svec_positions(n)
    N = len(pos)
    m = A_rows.shape[0]
    r2 = mp.sqrt(2)
    Wi = _mat(W) ** -1

    def smat_unit(k):
        E = mp.zeros(n, n)
        i, j = pos[k]
        if i == j:
            E[i, i] = 1
        else:
            E[i, j] = E[j, i] = 1 / r2
        return E

    def svec_mp(X):
        return [X[i, j] if i == j else r2 * X[i, j] for (i, j) in pos]

    K = mp.zeros(N + m, N + m)
    for k in range(N):
        col = svec_mp(Wi * smat_unit(k) * Wi)
        for t in range(N):
            K[t, k] = -col[t]
    for i in range(m):
        for k in range(N):
            a = mp.mpf(float(A_rows[i, k]))
            K[N + i, k] = a
            K[k, N + i] = a
    Ctm = _mat(Ct)
    rhs = mp.matrix(svec_mp(Ctm) + [mp.mpf(float(v)) for v in bt])
    sol = mp.lu_solve(K, rhs)
    x = [float(sol[t]) for t in range(N)]
    dX = np.zeros((n, n))
    for t, (i, j) in enumerate(pos):
        v = x[t] if i == j else x[t] / math.sqrt(2.0)
        dX[i, j] = dX[j, i] = v
    dy = np.array([float(sol[N + i]) for i in range(m)])
    return dX, dy

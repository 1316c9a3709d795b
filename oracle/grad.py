"""Implicit derivative of the SDP optimum with respect to (C, b): the vector-Jacobian product.

Test infrastructure (see the package header): nothing outside ``tests/`` and the bench's
CPU baseline imports this module.

At a point of the central path with NT scaling W (Section 1, eq. newt), a perturbation
(dC, db) of the data moves the iterate by the solution of the linearised optimality
conditions, which is (Newt-eps) of Section 3 with (C~, b~) = (dC, db) and no centring term:

    A(dX) = db,   A^T(dy) + dS = dC,   dX + W dS W = 0.

Eliminating dS = -W^{-1} dX W^{-1} gives the KKT matrix K = [[-(W (x)s W)^{-1}, A^T], [A, 0]]
with K [svec dX; dy] = [svec dC; db].  K is symmetric, so for a cotangent (gX, gy) of the
outputs (X, y) the cotangent of the data is

    [svec gC; gb] = K^{-1} [svec gX; gy],

which is the Newton direction of (Newt-eps) with (C~, b~) = (sym gX, gy): gC = dX, gb = dy.
At a point with mu = <X, S>/n > 0 this is the derivative of the central-path point; it
differs from the derivative of the optimum by O(mu).
"""
from __future__ import annotations

import numpy as np

from .newton import newton_direct, nt_scaling


def vjp(prob, X: np.ndarray, S: np.ndarray, gX: np.ndarray, gy: np.ndarray):
    """(gC, gb) = K^{-1} [sym gX; gy] at the NT scaling point of (X, S)."""
    W = nt_scaling(X, S)
    gXs = 0.5 * (gX + gX.T)
    dX, dy, _ = newton_direct(prob, W, gXs, np.asarray(gy, dtype=float))
    return 0.5 * (dX + dX.T), dy


def vjp_at_scaling(prob, W: np.ndarray, gX: np.ndarray, gy: np.ndarray):
    """The same product for a given scaling point W."""
    gXs = 0.5 * (gX + gX.T)
    dX, dy, _ = newton_direct(prob, W, gXs, np.asarray(gy, dtype=float))
    return 0.5 * (dX + dX.T), dy


def vjp_lp(prob, X: np.ndarray, S: np.ndarray, x: np.ndarray, z: np.ndarray, G: np.ndarray,
           gX: np.ndarray, gx: np.ndarray, gy: np.ndarray, r_hat: int = 3, space: str = "d"):
    """The same product for the problem with the orthant (nonnegative x entering as A(X) + G x = b,
    cost c_l, dual slack z = c_l - G^T y).  Linearising the optimality conditions at the NT
    scaling point (W for (X, S), d = x / z for the orthant) gives the KKT matrix
    [[-(W (x)s W)^{-1}, 0, A^T], [0, -D^{-1}, G^T], [A, G, 0]] acting on (dX, dx, dy) with right
    side (dC, dc_l, db).  It is symmetric, so the cotangent of the data (gC, gc_l, gb) is the
    Newton direction (dX, dx, dy) of the system with (C~, c~, b~) = (sym gX, gx, gy).  It is
    computed by the reformulated solve with the linear block (well conditioned as mu -> 0, where
    the plain Schur route of this system breaks down), in the preconditioner space `space`."""
    from .lpcone import newton_reform_lp
    from .operators import row_norm_scale
    W = nt_scaling(X, S)
    lw, Vw = np.linalg.eigh(W)
    gXs = 0.5 * (gX + gX.T)
    dX, dx, dy, _ = newton_reform_lp(prob, Vw, lw, gXs, np.asarray(gy, dtype=float), G, x / z,
                                     np.asarray(gx, dtype=float), r_hat=r_hat, s_A=row_norm_scale(prob),
                                     space=space)
    return 0.5 * (dX + dX.T), dx, dy

"""The linear cone of the paper's robust experiments in the Newton system (test infrastructure).

Section 7 writes robust matrix completion (eq. rmc-sdp) and the outlier-robust sensor network
localisation as semidefinite programs with extra nonnegative variables:

    min <C, X> + c_l^T x   s.t.   A(X) + G x = b,   X PSD,   x >= 0,

(eq. rmc-sdp: x = [v; w], G = [I, -I], c_l = 1, C = lambda I).  The paper solves them with an
existing solver and its reformulation of Sections 3-6 treats the semidefinite block only; this
module writes the extension down, in the paper's notation, as the oracle of that next step.

Newton system.  With the NT scaling W of (X, S) and d = x / z (elementwise) for the orthant,
(Newt-eps) gains a second primal block:

    A(dX) + G dx = b~,   -W^{-1} dX W^{-1} + A^T(dy) = C~,   -D^{-1} dx + G^T dy = c~,

D = diag(d).  Eliminating dX and dx gives M_l dy = b~ + A(W C~ W) + G D c~ with
M_l = A (W (x)s W) A^T + G D G^T, then dX = W(A^T(dy) - C~)W and dx = D(G^T dy - c~).

Reformulation.  With W (x)s W = Q Sigma^{-1} Q^T + tau^2 E (Prop. correct),
tau^{-2} M_l = (A E A^T + tau^{-2} G D G^T) + (A Q)(tau^2 Sigma)^{-1}(A Q)^T, so eq. augsys keeps
its form with the positive diagonal-type term tau^{-2} G D G^T added to its (1,1) block and
G D c~ added to b~; eq. recover is unchanged and dx = D(G^T dy - c~).

Preconditioner.  Section 6 replaces A E A^T by beta I.  Here the (1,1) block becomes
beta I + tau^{-2} G D G^T, which is diagonal when every column of G has at most one nonzero
(eq. rmc-sdp: G D G^T = diag(d_v + d_w)).  With Lam = beta I + tau^{-2} G D G^T the block inverse
of Section 6 becomes
    d-space: C = tau^2 Sigma + B^T Lam^{-1} B,  s = r_v - B^T Lam^{-1} r_u,  z_v = -C^{-1} s,
             z_u = Lam^{-1}(r_u - B z_v);
    m-space: K = Lam + B (tau^2 Sigma)^{-1} B^T,  z_u = K^{-1}(r_u + B D^{-1} r_v),
             z_v = D^{-1}(B^T z_u - r_v)     (D = tau^2 Sigma).
The operator and the preconditioner still share their second block row, so the second-block
residual of Prop. indefpcg stays zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from .linalg import skron, smat, svec
from .newton import schur_matrix, schur_solver
from .operators import A_matrix, A_op, At_op
from .reform import AQ_matrix, aug_apply, aug_rhs, pcg, recover, sigma_vec, split


def gdg(G: np.ndarray, d: np.ndarray) -> np.ndarray:
    """G diag(d) G^T."""
    return (G * d) @ G.T


def newton_direct_lp(prob, W: np.ndarray, Ct: np.ndarray, bt: np.ndarray, G: np.ndarray, d: np.ndarray,
                     ct: np.ndarray, refine: int = 2):
    """The Newton direction by its plain definition: the Schur system M_l dy = b~ + A(W C~ W) + G D c~
    with M_l = A (W (x)s W) A^T + G D G^T (Cholesky, with iterative refinement on the first primal
    block), then dX = W(A^T(dy) - C~)W, dx = D(G^T dy - c~).  Returns (dX, dx, dy)."""
    M = schur_matrix(prob, W) + gdg(G, d)
    solve = schur_solver(M)
    WCW = W @ Ct @ W
    rhs = bt + A_op(prob, WCW) + G @ (d * ct)
    dy = solve(rhs)
    for _ in range(refine):
        dX = W @ At_op(prob, dy) @ W - WCW
        dx = d * (G.T @ dy - ct)
        dy = dy + solve(bt - A_op(prob, dX) - G @ dx)
    dX = W @ At_op(prob, dy) @ W - WCW
    dX = 0.5 * (dX + dX.T)
    dx = d * (G.T @ dy - ct)
    return dX, dx, dy


def newton_kkt_dense_lp(prob, W: np.ndarray, Ct: np.ndarray, bt: np.ndarray, G: np.ndarray, d: np.ndarray,
                        ct: np.ndarray):
    """The same system assembled as one dense KKT matrix (tiny n) and solved by LU:
        [[-(W (x)s W)^{-1}, 0, A^T], [0, -D^{-1}, G^T], [A, G, 0]] [svec dX; dx; dy] = [svec C~; c~; b~]."""
    A = A_matrix(prob)
    N, p, m = A.shape[1], G.shape[1], prob.m
    K = np.zeros((N + p + m, N + p + m))
    K[:N, :N] = -np.linalg.inv(skron(W, W))
    K[:N, N + p:] = A.T
    K[N:N + p, N:N + p] = -np.diag(1.0 / d)
    K[N:N + p, N + p:] = G.T
    K[N + p:, :N] = A
    K[N + p:, N:N + p] = G
    sol = np.linalg.solve(K, np.concatenate([svec(Ct), ct, bt]))
    return smat(sol[:N], prob.n), sol[N:N + p], sol[N + p:]


@dataclass
class PrecondLP:
    space: str
    lam: np.ndarray       # m: the (1,1) block of P, beta + tau^{-2} diag(G D G^T)
    B: np.ndarray         # m x d
    Dv: np.ndarray        # d: tau^2 Sigma
    factor: tuple
    Cmat: np.ndarray


def precond_setup_lp(prob, sp, G: np.ndarray, d: np.ndarray, space: str = "d") -> PrecondLP:
    """Section 6's block inverse with beta I replaced by Lam = beta I + tau^{-2} G D G^T, which is
    diagonal when every column of G has at most one nonzero (each linear variable enters one
    constraint, as in eq. rmc-sdp)."""
    if np.count_nonzero(G, axis=0).max(initial=0) > 1:
        raise ValueError("G D G^T must be diagonal: at most one nonzero per column of G")
    B = AQ_matrix(prob, sp)
    lam = sp.beta + np.diag(gdg(G, d)) / sp.tau ** 2
    Dv = sp.tau ** 2 * sigma_vec(sp)
    if space == "d":
        Cm = np.diag(Dv) + (B.T / lam) @ B                 # C = tau^2 Sigma + B^T Lam^{-1} B
    elif space == "m":
        Cm = np.diag(lam) + (B / Dv) @ B.T                 # K = Lam + B D^{-1} B^T
    else:
        raise ValueError(space)
    Cm = 0.5 * (Cm + Cm.T)
    return PrecondLP(space=space, lam=lam, B=B, Dv=Dv, factor=sla.cho_factor(Cm, lower=True), Cmat=Cm)


def precond_apply_lp(P: PrecondLP, ru: np.ndarray, rv: np.ndarray):
    """z = [[Lam, B], [B^T, -D]]^{-1} [ru; rv]."""
    if P.space == "d":
        s = rv - P.B.T @ (ru / P.lam)
        zv = -sla.cho_solve(P.factor, s)
        zu = (ru - P.B @ zv) / P.lam
    else:
        zu = sla.cho_solve(P.factor, ru + P.B @ (rv / P.Dv))
        zv = (P.B.T @ zu - rv) / P.Dv
    return zu, zv


def precond_matrix_lp(P: PrecondLP) -> np.ndarray:
    top = np.hstack([np.diag(P.lam), P.B])
    bot = np.hstack([P.B.T, -np.diag(P.Dv)])
    return np.vstack([top, bot])


@dataclass
class ReformLPInfo:
    split: object
    precond: PrecondLP
    pcg: object


def choose_space_lp(sp, G: np.ndarray, d: np.ndarray, m: int, dominance: float = 1e8) -> str:
    """Preconditioner space with the linear block.  Rows where tau^{-2} delta_i exceeds
    `dominance` * beta are fixed by their slack (Lam is exact there); the d-space elimination then
    rests on the m_free remaining rows, and when m_free < d it loses the direction to rounding
    at small mu (the analogue of A11 failing) while the m-space complement, nearly diagonal on
    the fixed rows, stays accurate.  "m" when m_free < d, else "d"."""
    delta = np.diag(gdg(G, d))
    m_free = int(np.count_nonzero(delta / sp.tau ** 2 <= dominance * sp.beta))
    return "m" if m_free < sp.d else "d"


def newton_reform_lp(prob, V: np.ndarray, lam: np.ndarray, Ct: np.ndarray, bt: np.ndarray, G: np.ndarray,
                     d: np.ndarray, ct: np.ndarray, r: int | None = None, r_hat: int | None = None,
                     s_A: float = 1.0, rtol: float = 1e-12, maxit: int = 2000, space: str = "d"):
    """The Newton direction through eq. augsys with the linear block (module docstring), by the
    indefinite PCG of Cor. pcg started from x0 = P^{-1}[0; g_v], then eq. recover and
    dx = D(G^T dy - c~).  space: "d", "m" or "auto" (``choose_space_lp``).  Returns
    (dX, dx, dy, info)."""
    sp = split(V, lam, r=r, r_hat=r_hat, s_A=s_A)
    if space == "auto":
        space = choose_space_lp(sp, G, d, prob.m)
    P = precond_setup_lp(prob, sp, G, d, space=space)
    m = prob.m
    GDG = gdg(G, d)
    btl = bt + G @ (d * ct)
    gu, gv = aug_rhs(prob, sp, Ct, btl)
    g = np.concatenate([gu, gv])

    def Aop(x):
        a, b_ = aug_apply(prob, sp, x[:m], x[m:])
        return np.concatenate([a + GDG @ x[:m] / sp.tau ** 2, b_])

    def Pinv(rr):
        a, b_ = precond_apply_lp(P, rr[:m], rr[m:])
        return np.concatenate([a, b_])

    x0 = Pinv(np.concatenate([np.zeros(m), gv]))
    tol = rtol * math.sqrt(float(np.sum(Ct * Ct)) + float(btl @ btl) + float(ct @ ct))
    res = pcg(Aop, g, Pinv, x0, tol, maxit)
    dX, dy, _ = recover(prob, sp, Ct, res.x[:m], res.x[m:])
    dx = d * (G.T @ dy - ct)
    return dX, dx, dy, ReformLPInfo(split=sp, precond=P, pcg=res)

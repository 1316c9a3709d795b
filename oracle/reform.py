"""The well-conditioned reformulation of (Newt-eps), step by step, in numpy FP64.

Each function follows one passage of the paper, in the paper's notation:

* ``choose_rank``  -- Section 7: r = argmax_{i <= r_hat} lambda_i(W)/lambda_{i+1}(W).
* ``split``        -- eq. EQSigdef: W = Q Lam Q^T + Qp Lamp Qp^T, tau = lambda_{r+1}/2,
                      E = Q Q^T + tau^{-1} Qp Lamp Qp^T,
                      Sigma = diag(Lam (x)s Lam - tau^2 I, (Lam - tau I) (x) Lamp)^{-1};
                      Section 7: beta = (median eigenvalue of E)^2 (times s_A, see below).
* ``E_op, Q_op, Qt_op`` -- Section 5: E svec X = svec(E X E);
                      Q [svec B; vec N] = svec([Q Qp][B; sqrt2 N] Q^T);
                      Q^T svec X = [svec(Q^T X Q); sqrt2 vec(Qp^T X Q)].
* ``explicit_*``   -- the same objects assembled from their Kronecker definitions
                      (eq. EQSigdef), for tiny n.
* ``aug_apply, aug_rhs, recover`` -- eq. augsys and eq. recover.
* ``precond_*``    -- Section 6: C = tau^2 Sigma + beta^{-1} Q^T A^T A Q and the
                      block-triangular inverse of [[beta I, A Q], [Q^T A^T, -tau^2 Sigma]];
                      also the same inverse through the m x m complement
                      K = beta I + B D^{-1} B^T (B = A Q, D = tau^2 Sigma).
* ``pcg``          -- Def. pcg (with beta_j = <r_{j+1}, z_{j+1}>/<r_j, z_j>, the
                      standard PCG coefficient that the proof of Prop. indefpcg uses).
* ``newton_reform`` -- Cor. pcg end to end: v0 = -Sigma^{-1} Q^T c, PCG on augsys,
                      recovery.
* ``minres``       -- Def. MINRES with P = I: x_k = argmin ||A x - b|| over
                      x0 + span{r0, A r0, ..., A^{k-1} r0}, written out as the definition
                      (an orthonormal basis of the Krylov space, then a least-squares solve).
* ``newton_minres`` -- Cor. minres end to end: MINRES_k(augsys, g, I, 0), recovery.

Readings taken where the paper is garbled or silent: the sqrt(2) placement of Section 5; the beta^{-1}
factors of the block inverse in Section 6; the PCG beta index of Def. pcg;
beta scaled by s_A = ||A||_F^2/m (equal to the paper's rule when the rows
svec(A_i) have unit norm); the PCG stop ||r_k|| <= rtol ||[svec C~; b~]||.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from .linalg import SQRT2, psi, skron, svec
from .operators import A_op, At_op

# ----------------------------------------------------------------------------
# Split of W (eq. EQSigdef)


def choose_rank(lam_desc: np.ndarray, r_hat: int) -> int:
    """r = argmax_{1 <= i <= r_hat} lambda_i / lambda_{i+1} (1-based); first maximiser."""
    n = lam_desc.shape[0]
    r_hat = min(r_hat, n - 1)
    best, r = -np.inf, 1
    for i in range(1, r_hat + 1):
        ratio = lam_desc[i - 1] / lam_desc[i]
        if ratio > best:
            best, r = ratio, i
    return r


@dataclass
class Split:
    n: int
    r: int
    d: int
    Q: np.ndarray        # n x r
    Qp: np.ndarray       # n x (n - r)
    lam: np.ndarray      # r     (Lambda, descending)
    lamp: np.ndarray     # n - r (Lambda_perp, descending)
    tau: float
    E: np.ndarray        # n x n
    sigB: np.ndarray     # r x r, Sigma_B entry for svec position (i, j), i >= j
    sigN: np.ndarray     # (n - r) x r, Sigma_N entry for vec(N)[k, j]
    beta: float


def split(V: np.ndarray, lam: np.ndarray, r: int | None = None, r_hat: int | None = None,
          s_A: float = 1.0) -> Split:
    order = np.argsort(-lam, kind="stable")
    lam_s, V_s = lam[order], V[:, order]
    n = lam_s.shape[0]
    if r is None:
        r = choose_rank(lam_s, r_hat if r_hat is not None else n - 1)
    if not 1 <= r < n:
        raise ValueError("need 1 <= r < n")
    Q, Qp = V_s[:, :r], V_s[:, r:]
    L, Lp = lam_s[:r], lam_s[r:]
    tau = 0.5 * lam_s[r]                                  # tau = lambda_{r+1}(W) / 2
    E = Q @ Q.T + (Qp * (Lp / tau)) @ Qp.T
    E = 0.5 * (E + E.T)
    sigB = 1.0 / (np.outer(L, L) - tau * tau)              # (Lam (x)s Lam - tau^2 I)^{-1}
    sigN = 1.0 / np.outer(Lp, L - tau)                     # ((Lam - tau I) (x) Lamp)^{-1}
    eigE = np.linalg.eigvalsh(E)
    beta = float(np.median(eigE)) ** 2 * s_A               # Section 7 rule, scaled by s_A
    d = n * r - r * (r - 1) // 2
    return Split(n=n, r=r, d=d, Q=Q, Qp=Qp, lam=L, lamp=Lp, tau=float(tau), E=E,
                 sigB=sigB, sigN=sigN, beta=beta)


# ----------------------------------------------------------------------------
# Coordinates h = [svec B; vec N] of range(Q)  (Section 5)


def lower_pairs(r: int):
    """svec positions of an r x r matrix: (i, j), i >= j, column by column."""
    return [(i, j) for j in range(r) for i in range(j, r)]


def sigma_vec(sp: Split) -> np.ndarray:
    """Diagonal of Sigma in h-coordinates."""
    sb = np.array([sp.sigB[i, j] for (i, j) in lower_pairs(sp.r)])
    return np.concatenate([sb, sp.sigN.reshape(-1, order="F")])


def unpack_h(sp: Split, h: np.ndarray):
    """h -> (B symmetric r x r, N (n - r) x r)."""
    r, n = sp.r, sp.n
    nb = r * (r + 1) // 2
    B = np.zeros((r, r))
    for k, (i, j) in enumerate(lower_pairs(r)):
        v = h[k] if i == j else h[k] / SQRT2
        B[i, j] = B[j, i] = v
    N = np.asarray(h[nb:]).reshape((n - r, r), order="F")
    return B, N


def pack_h(sp: Split, B: np.ndarray, N: np.ndarray) -> np.ndarray:
    hb = np.array([B[i, j] if i == j else SQRT2 * B[i, j] for (i, j) in lower_pairs(sp.r)])
    return np.concatenate([hb, N.reshape(-1, order="F")])


def E_op(sp: Split, X: np.ndarray) -> np.ndarray:
    """E svec(X) = svec(E X E), returned as the matrix E X E."""
    return sp.E @ X @ sp.E


def Q_op(sp: Split, h: np.ndarray) -> np.ndarray:
    """Q h as a symmetric matrix: sym([Q Qp][B; sqrt2 N] Q^T)."""
    B, N = unpack_h(sp, h)
    U = sp.Q @ B + SQRT2 * (sp.Qp @ N)
    M = U @ sp.Q.T
    return 0.5 * (M + M.T)


def Qt_op(sp: Split, X: np.ndarray) -> np.ndarray:
    """Q^T svec(X) = [svec(Q^T X Q); sqrt2 vec(Qp^T X Q)]."""
    XQ = X @ sp.Q
    return np.concatenate([svec(sp.Q.T @ XQ), SQRT2 * (sp.Qp.T @ XQ).reshape(-1, order="F")])


# ----------------------------------------------------------------------------
# Explicit matrices from the Kronecker definitions (tiny n)


def explicit_E(sp: Split) -> np.ndarray:
    return skron(sp.E, sp.E)


def explicit_Q(sp: Split) -> np.ndarray:
    """[Q (x)s Q, sqrt2 Psi_n^T (Q kron Qp)]."""
    QB = skron(sp.Q, sp.Q)
    QN = SQRT2 * psi(sp.n).T @ np.kron(sp.Q, sp.Qp)
    return np.hstack([QB, QN])


def explicit_Sigma(sp: Split) -> np.ndarray:
    """diag(Lam (x)s Lam - tau^2 I, (Lam - tau I) kron Lamp)^{-1}."""
    L = np.diag(sp.lam)
    SB_inv = skron(L, L) - sp.tau ** 2 * np.eye(sp.r * (sp.r + 1) // 2)
    SN_inv = np.kron(np.diag(sp.lam - sp.tau), np.diag(sp.lamp))
    top = np.linalg.inv(SB_inv)
    bot = np.linalg.inv(SN_inv)
    d = top.shape[0] + bot.shape[0]
    S = np.zeros((d, d))
    S[:top.shape[0], :top.shape[0]] = top
    S[top.shape[0]:, top.shape[0]:] = bot
    return S


# ----------------------------------------------------------------------------
# Augmented system and recovery (eq. augsys, eq. recover)


def aug_apply(prob, sp: Split, u: np.ndarray, v: np.ndarray):
    """[[A E A^T, A Q], [Q^T A^T, -tau^2 Sigma]] [u; v]."""
    Y = At_op(prob, u)
    top = A_op(prob, E_op(sp, Y) + Q_op(sp, v))
    bot = Qt_op(sp, Y) - sp.tau ** 2 * sigma_vec(sp) * v
    return top, bot


def aug_rhs(prob, sp: Split, Ct: np.ndarray, bt: np.ndarray):
    """[b~ + tau^2 A E c; tau^2 Q^T c]."""
    return bt + sp.tau ** 2 * A_op(prob, E_op(sp, Ct)), sp.tau ** 2 * Qt_op(sp, Ct)


def recover(prob, sp: Split, Ct: np.ndarray, u: np.ndarray, v: np.ndarray):
    """dy = tau^{-2} u, svec dX = E(A^T u - tau^2 c) + Q v; dS = C~ - A^T(dy)."""
    dy = u / sp.tau ** 2
    dX = E_op(sp, At_op(prob, u) - sp.tau ** 2 * Ct) + Q_op(sp, v)
    dX = 0.5 * (dX + dX.T)
    return dX, dy, Ct - At_op(prob, dy)


# ----------------------------------------------------------------------------
# Preconditioner (Section 6)


def AQ_matrix(prob, sp: Split) -> np.ndarray:
    """B = A Q, formed column by column with d products A Q e_j."""
    B = np.empty((prob.m, sp.d))
    for j in range(sp.d):
        e = np.zeros(sp.d)
        e[j] = 1.0
        B[:, j] = A_op(prob, Q_op(sp, e))
    return B


@dataclass
class Precond:
    space: str            # "d" or "m"
    beta: float
    B: np.ndarray         # m x d
    Dv: np.ndarray        # d, tau^2 Sigma
    factor: tuple         # scipy cho_factor of C (d-space) or K (m-space)
    Cmat: np.ndarray      # the factored matrix


def precond_setup(prob, sp: Split, space: str = "d", B: np.ndarray | None = None) -> Precond:
    if B is None:
        B = AQ_matrix(prob, sp)
    Dv = sp.tau ** 2 * sigma_vec(sp)
    if space == "d":
        Cm = np.diag(Dv) + (B.T @ B) / sp.beta            # C = tau^2 Sigma + beta^{-1} B^T B
    elif space == "m":
        Cm = sp.beta * np.eye(prob.m) + (B / Dv) @ B.T     # K = beta I + B D^{-1} B^T
    else:
        raise ValueError(space)
    Cm = 0.5 * (Cm + Cm.T)
    return Precond(space=space, beta=sp.beta, B=B, Dv=Dv, factor=sla.cho_factor(Cm, lower=True), Cmat=Cm)


def precond_apply(P: Precond, ru: np.ndarray, rv: np.ndarray):
    """z = [[beta I, B], [B^T, -D]]^{-1} [ru; rv]."""
    if P.space == "d":
        s = rv - (P.B.T @ ru) / P.beta
        zv = -sla.cho_solve(P.factor, s)
        zu = (ru - P.B @ zv) / P.beta
    else:
        zu = sla.cho_solve(P.factor, ru + P.B @ (rv / P.Dv))
        zv = (P.B.T @ zu - rv) / P.Dv
    return zu, zv


def precond_matrix(P: Precond) -> np.ndarray:
    m = P.B.shape[0]
    top = np.hstack([P.beta * np.eye(m), P.B])
    bot = np.hstack([P.B.T, -np.diag(P.Dv)])
    return np.vstack([top, bot])


# ----------------------------------------------------------------------------
# PCG (Def. pcg)


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    res_hist: list
    x_hist: list
    converged: bool


def pcg(Aop, b: np.ndarray, Pinv, x0: np.ndarray, tol: float, maxit: int,
        keep_iterates: bool = False, stop_norm=None) -> PCGResult:
    """PCG_k(A, b, P, x0) of Def. pcg with beta_j = <r_{j+1}, z_{j+1}>/<r_j, z_j>.

    Runs until ||r_k|| <= tol (an absolute threshold chosen by the caller) or maxit.
    No sign test on <p, A p>: with an indefinite P the iteration is Def. pcg as written,
    and at the rounding floor that product may change sign without harm.
    """
    x = x0.copy()
    r = b - Aop(x)
    z = Pinv(r)
    p = z.copy()
    rz = float(r @ z)
    norm = stop_norm if stop_norm is not None else (lambda v: float(np.linalg.norm(v)))
    hist, xs = [norm(r)], ([x.copy()] if keep_iterates else [])
    k = 0
    conv = hist[-1] <= tol
    while not conv and k < maxit:
        Ap = Aop(p)
        alpha = rz / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        z = Pinv(r)
        rz_new = float(r @ z)
        bj = rz_new / rz
        p = z + bj * p
        rz = rz_new
        k += 1
        hist.append(norm(r))
        if keep_iterates:
            xs.append(x.copy())
        conv = hist[-1] <= tol
    return PCGResult(x=x, iters=k, res_hist=hist, x_hist=xs, converged=conv)


# ----------------------------------------------------------------------------
# Cor. pcg end to end


@dataclass
class ReformInfo:
    split: Split
    precond: Precond
    pcg: PCGResult
    g: np.ndarray


def newton_reform(prob, V: np.ndarray, lam: np.ndarray, Ct: np.ndarray, bt: np.ndarray,
                  r: int | None = None, r_hat: int | None = None, s_A: float = 1.0,
                  rtol: float = 1e-12, maxit: int = 2000, space: str = "d",
                  keep_iterates: bool = False, start: str = "paper"):
    """Solve (Newt-eps) through eq. augsys with the indefinite PCG of Cor. pcg.

    start = "paper": x0 = [0; -Sigma^{-1} Q^T c] as Cor. pcg prints it.
    start = "precond": x0 = P^{-1}[0; g_v], the preconditioner applied to the second block
    of the right side.  Both make the second block of r0 zero, which is what Cor. pcg and
    Prop. indefpcg need (P x0 = [0; g_v] and the operator shares P's second block row).
    """
    sp = split(V, lam, r=r, r_hat=r_hat, s_A=s_A)
    P = precond_setup(prob, sp, space=space)
    m = prob.m
    gu, gv = aug_rhs(prob, sp, Ct, bt)
    g = np.concatenate([gu, gv])
    v0 = -Qt_op(sp, Ct) / sigma_vec(sp)                   # v0 = -Sigma^{-1} Q^T c

    def Aop(x):
        a, b_ = aug_apply(prob, sp, x[:m], x[m:])
        return np.concatenate([a, b_])

    def Pinv(rr):
        a, b_ = precond_apply(P, rr[:m], rr[m:])
        return np.concatenate([a, b_])

    if start == "paper":
        x0 = np.concatenate([np.zeros(m), v0])
    elif start == "precond":
        x0 = Pinv(np.concatenate([np.zeros(m), gv]))
    else:
        raise ValueError(start)
    # Stop on ||r_k|| <= rtol ||[svec C~; b~]||: with the second-block residual at rounding
    # level, ||r_k|| is the (Newt-eps) residual of the recovered direction (Lemma smallres),
    # measured against the right side of (Newt-eps).
    tol = rtol * math.sqrt(float(np.sum(Ct * Ct)) + float(bt @ bt))
    res = pcg(Aop, g, Pinv, x0, tol, maxit, keep_iterates=keep_iterates)
    dX, dy, dS = recover(prob, sp, Ct, res.x[:m], res.x[m:])
    return dX, dy, dS, ReformInfo(split=sp, precond=P, pcg=res, g=g)


# ----------------------------------------------------------------------------
# MINRES (Def. MINRES with P = I) and Cor. minres


@dataclass
class MinresResult:
    x: np.ndarray
    iters: int
    res_hist: list
    converged: bool


def minres(Aop, b: np.ndarray, x0: np.ndarray, tol: float, maxit: int) -> MinresResult:
    """MINRES_k(A, b, I, x0) by its definition: x_k minimises ||A x - b|| over
    x0 + span{r0, A r0, ..., A^{k-1} r0}, r0 = b - A x0.

    The Krylov space is kept as an orthonormal basis Z (each new direction A z_k
    orthogonalised twice against all previous ones), and x_k = x0 + Z c with
    c = argmin ||(A Z) c - r0|| by a least-squares solve.  Plain and slow (O(k^2 n) work and
    O(k n) memory); stops when ||A x_k - b|| <= tol or k = maxit, or when the Krylov space
    stops growing (then x_k is the exact minimiser over the whole space)."""
    x0 = np.asarray(x0, dtype=float)
    r0 = b - Aop(x0)
    n0 = float(np.linalg.norm(r0))
    hist = [n0]
    if n0 <= tol:
        return MinresResult(x=x0.copy(), iters=0, res_hist=hist, converged=True)
    Z = [r0 / n0]
    AZ = [Aop(Z[0])]
    x = x0.copy()
    k = 0
    while k < maxit:
        k += 1
        Zm, AZm = np.stack(Z, axis=1), np.stack(AZ, axis=1)
        c = np.linalg.lstsq(AZm, r0, rcond=None)[0]
        x = x0 + Zm @ c
        res = float(np.linalg.norm(b - Aop(x)))
        hist.append(res)
        if res <= tol:
            return MinresResult(x=x, iters=k, res_hist=hist, converged=True)
        z = AZ[-1].copy()                                  # next Krylov direction A z_k
        for _ in range(2):
            z -= Zm @ (Zm.T @ z)
        nz = float(np.linalg.norm(z))
        if nz <= 1e-14 * float(np.linalg.norm(AZ[-1])):   # invariant space: x is final
            return MinresResult(x=x, iters=k, res_hist=hist, converged=res <= tol)
        Z.append(z / nz)
        AZ.append(Aop(Z[-1]))
    return MinresResult(x=x, iters=k, res_hist=hist, converged=False)


def newton_minres(prob, V: np.ndarray, lam: np.ndarray, Ct: np.ndarray, bt: np.ndarray,
                  r: int | None = None, r_hat: int | None = None, s_A: float = 1.0,
                  rtol: float = 1e-12, maxit: int = 2000):
    """Solve (Newt-eps) as Cor. minres states: [u; v] = MINRES_k(augsys, g, I, 0), then
    eq. recover; the stop test is the one of newton_reform (||r_k|| <= rtol ||[svec C~; b~]||)."""
    sp = split(V, lam, r=r, r_hat=r_hat, s_A=s_A)
    m = prob.m
    gu, gv = aug_rhs(prob, sp, Ct, bt)
    g = np.concatenate([gu, gv])

    def Aop(x):
        a, b_ = aug_apply(prob, sp, x[:m], x[m:])
        return np.concatenate([a, b_])

    tol = rtol * math.sqrt(float(np.sum(Ct * Ct)) + float(bt @ bt))
    res = minres(Aop, g, np.zeros_like(g), tol, maxit)
    dX, dy, dS = recover(prob, sp, Ct, res.x[:m], res.x[m:])
    return dX, dy, dS, res, sp


def prop_minres_bound(kappa: float, r0norm: float, eps: float) -> int:
    """Iteration bound of Prop. minres for symmetric indefinite A: ceil(kappa log(2 ||A x0 - b|| / eps)).

    Prop. minres prints kappa/2 in front of the logarithm; for an indefinite spectrum the
    residual contracts by (kappa - 1)/(kappa + 1) only every two steps, which gives kappa
    (the printed factor holds for a definite A)."""
    return int(math.ceil(kappa * math.log(2.0 * r0norm / eps)))


def cor_pcg_bound(kappa_E: float, kappa_A: float, gnorm: float, eps: float) -> int:
    """Iteration bound of Cor. pcg."""
    k = kappa_E * kappa_A
    return int(math.ceil(0.5 * k * math.log(k * gnorm / (2 * eps))))

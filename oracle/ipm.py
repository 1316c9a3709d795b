"""A textbook infeasible primal-dual path-following IPM with NT scaling (the outer loop).

The paper keeps the outer loop of an existing solver unchanged (Section 7)
and describes it only through the log-barrier path and the Newton subproblem
(Section 1, eq. newt).  This module writes one standard method down so that
the Newton directions can be exercised along a real central path and so
that solved instances can pin the problem data.  Its choices (start point,
Mehrotra predictor-corrector, step rule, stopping rule) are the oracle's own
definitions: parity unpinned beyond the convergence invariants that the
tests check (feasibility, duality gap, complementarity, known optima).

Per iteration, with mu = <X,S>/n, r_p = b - A(X), R_d = C - A^T(y) - S:
    A(dX) = r_p,  A^T(dy) + dS = R_d,  dX + W dS W = R_c,
so that (dX, dy) solve (Newt-eps) with b~ = r_p, C~ = R_d - W^{-1} R_c W^{-1}
and dS = R_d - A^T(dy).  In the NT-scaled space G = W^{1/2},
Lam = G^{-1} X G^{-1} = G S G, the complementarity target is the Lyapunov
equation Lam R + R Lam = 2 sigma mu I - 2 Lam^2 - (Dx Ds + Ds Dx) with
R = G^{-1}(dX + W dS W)G^{-1}; R_c = G R G.  Predictor: sigma = 0 and no
second-order term (then R_c = -X).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .newton import newton_direct, nt_scaling, schur_matrix, sqrtm_psd
from .operators import A_op, At_op, constraint_matrix


def max_step(X: np.ndarray, dX: np.ndarray) -> float:
    """Largest alpha with X + alpha dX PSD (X PD): via lambda_min(L^{-1} dX L^{-T})."""
    L = np.linalg.cholesky(X)
    Li = np.linalg.inv(L)
    lmin = float(np.linalg.eigvalsh(Li @ dX @ Li.T)[0])
    return math.inf if lmin >= 0 else -1.0 / lmin


def _lyap_diag(U: np.ndarray, g: np.ndarray, RHS: np.ndarray) -> np.ndarray:
    """Solve Lam R + R Lam = RHS with Lam = U diag(g) U^T."""
    T = U.T @ RHS @ U
    R = T / (g[:, None] + g[None, :])
    return U @ R @ U.T


@dataclass
class IPMState:
    X: np.ndarray
    y: np.ndarray
    S: np.ndarray


@dataclass
class IPMLog:
    it: int
    mu: float
    rel_gap: float
    pinf: float
    dinf: float
    alpha_p: float
    alpha_d: float
    sigma: float


@dataclass
class IPMResult:
    X: np.ndarray
    y: np.ndarray
    S: np.ndarray
    iters: int
    converged: bool
    log: list = field(default_factory=list)
    history: list = field(default_factory=list)

    @property
    def obj(self):
        return self.log[-1] if self.log else None


def start_point(prob) -> IPMState:
    """X0 = S0 = xi I, y0 = 0 with xi = max(10, sqrt n, max_i (1+|b_i|)/(1+||A_i||_F), (1+||C||_F)/sqrt n)."""
    n = prob.n
    an = np.array([np.linalg.norm(constraint_matrix(prob, i)) for i in range(prob.m)]) \
        if prob.m <= 20000 else np.ones(prob.m)
    xi = max(10.0, math.sqrt(n), float(np.max((1 + np.abs(prob.b)) / (1 + an))),
             (1 + np.linalg.norm(prob.C)) / math.sqrt(n))
    return IPMState(X=xi * np.eye(n), y=np.zeros(prob.m), S=xi * np.eye(n))


def measures(prob, st: IPMState):
    pobj = float(np.sum(prob.C * st.X))
    dobj = float(prob.b @ st.y)
    rel_gap = abs(pobj - dobj) / (1 + abs(pobj) + abs(dobj))
    pinf = float(np.linalg.norm(prob.b - A_op(prob, st.X)) / (1 + np.linalg.norm(prob.b)))
    dinf = float(np.linalg.norm(prob.C - At_op(prob, st.y) - st.S) / (1 + np.linalg.norm(prob.C)))
    return pobj, dobj, rel_gap, pinf, dinf


def ipm_solve(prob, tol: float = 1e-8, max_iter: int = 100, step_frac: float = 0.98,
              keep_history: bool = False, x0: IPMState | None = None) -> IPMResult:
    st = x0 if x0 is not None else start_point(prob)
    n = prob.n
    log, hist = [], []
    converged = False
    it = 0
    for it in range(max_iter + 1):
        pobj, dobj, gap, pinf, dinf = measures(prob, st)
        if gap <= tol and pinf <= tol and dinf <= tol:
            converged = True
            break
        if it == max_iter:
            break
        X, y, S = st.X, st.y, st.S
        mu = float(np.sum(X * S)) / n
        W = nt_scaling(X, S)
        G = sqrtm_psd(W)
        Gi = np.linalg.inv(G)
        Wi = Gi @ Gi
        Lam = G @ S @ G
        Lam = 0.5 * (Lam + Lam.T)
        g, U = np.linalg.eigh(Lam)
        r_p = prob.b - A_op(prob, X)
        R_d = prob.C - At_op(prob, y) - S
        M = schur_matrix(prob, W)
        if keep_history:
            hist.append(dict(X=X.copy(), y=y.copy(), S=S.copy(), W=W.copy(), mu=mu, r_p=r_p, R_d=R_d))

        WRdW = W @ R_d @ W

        def direction(Rc):
            Ct = R_d - Wi @ Rc @ Wi
            Ct = 0.5 * (Ct + Ct.T)
            # W C~ W = W R_d W - R_c exactly; this form avoids forming W^{-1} R_c W^{-1}
            dX, dy, _ = newton_direct(prob, W, Ct, r_p, M=M, WCW=WRdW - Rc)
            dS = R_d - At_op(prob, dy)
            return dX, dy, 0.5 * (dS + dS.T)

        # predictor (sigma = 0)
        Rc_aff = G @ _lyap_diag(U, g, -2.0 * Lam @ Lam) @ G
        dXa, dya, dSa = direction(Rc_aff)
        ap = min(1.0, max_step(X, dXa))
        ad = min(1.0, max_step(S, dSa))
        mu_aff = float(np.sum((X + ap * dXa) * (S + ad * dSa))) / n
        sigma = min(1.0, (mu_aff / mu) ** 3)
        # corrector: centring plus the second-order term in the scaled space
        Dx = Gi @ dXa @ Gi
        Ds = G @ dSa @ G
        rhs = 2.0 * sigma * mu * np.eye(n) - 2.0 * Lam @ Lam - (Dx @ Ds + Ds @ Dx)
        Rc = G @ _lyap_diag(U, g, rhs) @ G
        dX, dy, dS = direction(0.5 * (Rc + Rc.T))
        ap = min(1.0, step_frac * max_step(X, dX))
        ad = min(1.0, step_frac * max_step(S, dS))
        Xn = X + ap * dX
        Sn = S + ad * dS
        st = IPMState(X=0.5 * (Xn + Xn.T), y=y + ad * dy, S=0.5 * (Sn + Sn.T))
        log.append(IPMLog(it=it, mu=mu, rel_gap=gap, pinf=pinf, dinf=dinf, alpha_p=ap, alpha_d=ad, sigma=sigma))
    return IPMResult(X=st.X, y=st.y, S=st.S, iters=it, converged=converged, log=log, history=hist)


def center(prob, st: IPMState, mu: float, max_iter: int = 50, tol: float = 1e-12) -> IPMState:
    """Newton steps towards the central-path point of parameter mu: A(X) = b, A^T y + S = C,
    X S = mu I (NT direction with R_c = mu S^{-1} - X, i.e. sigma mu = mu and no second-order
    term), with step lengths that keep X, S positive definite.  Stops when the residuals and
    ||G^{-1} X S G - mu I|| / mu (the scaled centrality) fall below tol."""
    n = prob.n
    X, y, S = st.X, st.y, st.S
    for _ in range(max_iter):
        r_p = prob.b - A_op(prob, X)
        R_d = prob.C - At_op(prob, y) - S
        W = nt_scaling(X, S)
        G = sqrtm_psd(W)
        Lam = G @ S @ G
        Lam = 0.5 * (Lam + Lam.T)
        cen = float(np.linalg.norm(Lam @ Lam - mu * np.eye(n))) / mu
        res = max(float(np.linalg.norm(r_p)) / (1 + np.linalg.norm(prob.b)),
                  float(np.linalg.norm(R_d)) / (1 + np.linalg.norm(prob.C)))
        if cen <= tol and res <= tol:
            break
        Wi = np.linalg.inv(W)
        Rc = mu * np.linalg.inv(S) - X
        Rc = 0.5 * (Rc + Rc.T)
        Ct = R_d - Wi @ Rc @ Wi
        dX, dy, _ = newton_direct(prob, W, 0.5 * (Ct + Ct.T), r_p, WCW=W @ R_d @ W - Rc)
        dS = R_d - At_op(prob, dy)
        dS = 0.5 * (dS + dS.T)
        ap = min(1.0, 0.95 * max_step(X, dX))
        ad = min(1.0, 0.95 * max_step(S, dS))
        a = min(ap, ad)
        X = X + a * dX
        y = y + a * dy
        S = S + a * dS
        X, S = 0.5 * (X + X.T), 0.5 * (S + S.T)
    return IPMState(X=X, y=y, S=S)

"""The outer interior-point loop with nonnegative variables (test infrastructure).

The problems of Section 7's robust experiments (eq. rmc-sdp) couple the semidefinite variable X
with nonnegative variables x:

    min <C, X> + c_l^T x   s.t.   A(X) + G x = b,   X PSD,   x >= 0,
    max b^T y              s.t.   C - A^T(y) = S PSD,   c_l - G^T y = z >= 0.

This is the method of ``ipm.py`` (infeasible NT path following with Mehrotra's predictor-corrector,
the oracle's own textbook choices) with the orthant added:

* residuals r_p = b - A(X) - G x, R_d = C - A^T(y) - S, r_l = c_l - G^T y - z, and
  mu = (<X, S> + x^T z) / (n + p);
* the Newton direction (the reformulated solve by default) solves the linearised optimality
  conditions
      A(dX) + G dx = r_p,  A^T(dy) + dS = R_d,  G^T dy + dz = r_l,
      dX + W dS W = R_c   (NT, semidefinite block),   z dx + x dz = r_x   (orthant),
  which is the Newton system of ``lpcone`` with d = x / z, b~ = r_p, C~ = R_d - W^{-1} R_c W^{-1}
  and c~ = r_l - r_x / x (then dx = D(G^T dy - c~) = d (G^T dy - r_l) + r_x / z);
* predictor r_x = -x z (sigma = 0); corrector r_x = sigma mu - x z - dx_a dz_a, the semidefinite
  block as in ``ipm.py``; sigma = min(1, (mu_aff / mu)^3);
* step lengths: the semidefinite bound of ``ipm.max_step`` and the ratio test
  sup{a : x + a dx >= 0} for the orthant, primal (X, x) and dual (S, z) separately, times 0.98;
* stop when the relative gap, ||r_p|| / (1 + ||b||) and the dual residuals
  (||R_d||_F^2 + ||r_l||^2)^{1/2} / (1 + ||C||_F + ||c_l||) are all <= tol.

Start: X = S = xi I, x = z = xi 1, y = 0 (xi as in ``ipm.start_point``).  Parity unpinned beyond the
optimality conditions and the known solutions that the tests check.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .ipm import _lyap_diag, max_step, start_point
from .lpcone import newton_direct_lp, newton_reform_lp
from .newton import nt_scaling, sqrtm_psd
from .operators import A_op, At_op, row_norm_scale


@dataclass
class LPState:
    X: np.ndarray
    x: np.ndarray
    y: np.ndarray
    S: np.ndarray
    z: np.ndarray


@dataclass
class LPResult:
    X: np.ndarray
    x: np.ndarray
    y: np.ndarray
    S: np.ndarray
    z: np.ndarray
    iters: int
    converged: bool
    log: list = field(default_factory=list)


def ratio_step(x: np.ndarray, dx: np.ndarray) -> float:
    """sup{a >= 0 : x + a dx >= 0} for x > 0."""
    neg = dx < 0
    return float(np.min(-x[neg] / dx[neg])) if np.any(neg) else math.inf


def lp_measures(prob, G, cl, st: LPState):
    pobj = float(np.sum(prob.C * st.X) + cl @ st.x)
    dobj = float(prob.b @ st.y)
    gap = abs(pobj - dobj) / (1 + abs(pobj) + abs(dobj))
    rp = prob.b - A_op(prob, st.X) - G @ st.x
    Rd = prob.C - At_op(prob, st.y) - st.S
    rl = cl - G.T @ st.y - st.z
    pinf = float(np.linalg.norm(rp) / (1 + np.linalg.norm(prob.b)))
    dinf = float(math.sqrt(float(np.sum(Rd * Rd)) + float(rl @ rl)) / (1 + np.linalg.norm(prob.C) + np.linalg.norm(cl)))
    return pobj, dobj, gap, pinf, dinf, rp, Rd, rl


def ipm_solve_lp(prob, G: np.ndarray, cl: np.ndarray, tol: float = 1e-8, max_iter: int = 100,
                 step_frac: float = 0.98, direction_by: str = "reform", r_hat: int = 3) -> LPResult:
    """direction_by = "reform": each Newton direction through eq. augsys with the linear block and
    the indefinite PCG (``lpcone.newton_reform_lp``, rank parameter r_hat), which stays well
    conditioned as mu -> 0; "schur": the plain Schur elimination (``lpcone.newton_direct_lp``),
    whose normal matrix A (W (x)s W) A^T + G D G^T reaches a condition number near 1/mu^2 when
    the constraints nearly cover the svec coordinates (robust completion) and loses the
    direction before a 1e-8 gap."""
    n, p = prob.n, G.shape[1]
    sA = row_norm_scale(prob)
    st0 = start_point(prob)
    xi = float(st0.X[0, 0])
    st = LPState(X=st0.X, x=xi * np.ones(p), y=np.zeros(prob.m), S=st0.S, z=xi * np.ones(p))
    log = []
    converged = False
    it = 0
    for it in range(max_iter + 1):
        pobj, dobj, gap, pinf, dinf, rp, Rd, rl = lp_measures(prob, G, cl, st)
        if gap <= tol and pinf <= tol and dinf <= tol:
            converged = True
            break
        if it == max_iter:
            break
        X, x, y, S, z = st.X, st.x, st.y, st.S, st.z
        mu = (float(np.sum(X * S)) + float(x @ z)) / (n + p)
        W = nt_scaling(X, S)
        Gs = sqrtm_psd(W)
        Gi = np.linalg.inv(Gs)
        Wi = Gi @ Gi
        Lam = Gs @ S @ Gs
        Lam = 0.5 * (Lam + Lam.T)
        g, U = np.linalg.eigh(Lam)
        d = x / z

        if direction_by == "reform":
            lw, Vw = np.linalg.eigh(W)

        def direction(Rc, rx):
            Ct = Rd - Wi @ Rc @ Wi
            Ct = 0.5 * (Ct + Ct.T)
            ct = rl - rx / x
            if direction_by == "reform":
                dX, dx, dy, _ = newton_reform_lp(prob, Vw, lw, Ct, rp, G, d, ct, r_hat=r_hat, s_A=sA)
            else:
                dX, dx, dy = newton_direct_lp(prob, W, Ct, rp, G, d, ct)
            dS = Rd - At_op(prob, dy)
            dz = rl - G.T @ dy
            return dX, dx, dy, 0.5 * (dS + dS.T), dz

        # predictor (sigma = 0)
        Rc_aff = Gs @ _lyap_diag(U, g, -2.0 * Lam @ Lam) @ Gs
        dXa, dxa, dya, dSa, dza = direction(Rc_aff, -x * z)
        ap = min(1.0, max_step(X, dXa), ratio_step(x, dxa))
        ad = min(1.0, max_step(S, dSa), ratio_step(z, dza))
        mu_aff = (float(np.sum((X + ap * dXa) * (S + ad * dSa))) + float((x + ap * dxa) @ (z + ad * dza))) / (n + p)
        sigma = min(1.0, (mu_aff / mu) ** 3)
        # corrector: centring plus the second-order terms
        Dx = Gi @ dXa @ Gi
        Ds = Gs @ dSa @ Gs
        rhs = 2.0 * sigma * mu * np.eye(n) - 2.0 * Lam @ Lam - (Dx @ Ds + Ds @ Dx)
        Rc = Gs @ _lyap_diag(U, g, rhs) @ Gs
        rx = sigma * mu - x * z - dxa * dza
        dX, dx, dy, dS, dz = direction(0.5 * (Rc + Rc.T), rx)
        ap = min(1.0, step_frac * min(max_step(X, dX), ratio_step(x, dx)))
        ad = min(1.0, step_frac * min(max_step(S, dS), ratio_step(z, dz)))
        Xn = X + ap * dX
        Sn = S + ad * dS
        st = LPState(X=0.5 * (Xn + Xn.T), x=x + ap * dx, y=y + ad * dy, S=0.5 * (Sn + Sn.T), z=z + ad * dz)
        log.append(dict(it=it, mu=mu, rel_gap=gap, pinf=pinf, dinf=dinf, alpha_p=ap, alpha_d=ad, sigma=sigma))
    return LPResult(X=st.X, x=st.x, y=st.y, S=st.S, z=st.z, iters=it, converged=converged, log=log)


def center_lp(prob, G: np.ndarray, cl: np.ndarray, st: LPState, mu: float, max_iter: int = 60,
              tol: float = 1e-12, r_hat: int = 3) -> LPState:
    """Newton steps towards the central-path point of parameter mu of the problem with the orthant:
    A(X) + G x = b, A^T y + S = C, G^T y + z = c_l, X S = mu I, x z = mu 1 (NT direction with
    R_c = mu S^{-1} - X and r_x = mu - x z, no second-order terms), by the reformulated solve, with
    step lengths that keep X, S, x, z in the interior.  Stops when the residuals and the scaled
    centrality of both cones fall below tol."""
    n = prob.n
    sA = row_norm_scale(prob)
    X, x, y, S, z = st.X, st.x, st.y, st.S, st.z
    for _ in range(max_iter):
        rp = prob.b - A_op(prob, X) - G @ x
        Rd = prob.C - At_op(prob, y) - S
        rl = cl - G.T @ y - z
        W = nt_scaling(X, S)
        Gs = sqrtm_psd(W)
        Lam = Gs @ S @ Gs
        Lam = 0.5 * (Lam + Lam.T)
        cen = max(float(np.linalg.norm(Lam @ Lam - mu * np.eye(n))), float(np.abs(x * z - mu).max())) / mu
        res = max(float(np.linalg.norm(rp)) / (1 + np.linalg.norm(prob.b)),
                  math.sqrt(float(np.sum(Rd * Rd)) + float(rl @ rl)) / (1 + np.linalg.norm(prob.C) + np.linalg.norm(cl)))
        if cen <= tol and res <= tol:
            break
        Wi = np.linalg.inv(W)
        Rc = mu * np.linalg.inv(S) - X
        Rc = 0.5 * (Rc + Rc.T)
        Ct = Rd - Wi @ Rc @ Wi
        rx = mu - x * z
        lw, Vw = np.linalg.eigh(W)
        dX, dx, dy, _ = newton_reform_lp(prob, Vw, lw, 0.5 * (Ct + Ct.T), rp, G, x / z, rl - rx / x,
                                         r_hat=r_hat, s_A=sA)
        dS = Rd - At_op(prob, dy)
        dS = 0.5 * (dS + dS.T)
        dz = rl - G.T @ dy
        a = min(1.0, 0.95 * min(max_step(X, dX), ratio_step(x, dx)), 0.95 * min(max_step(S, dS), ratio_step(z, dz)))
        X, x, y, S, z = X + a * dX, x + a * dx, y + a * dy, S + a * dS, z + a * dz
        X, S = 0.5 * (X + X.T), 0.5 * (S + S.T)
    return LPState(X=X, x=x, y=y, S=S, z=z)

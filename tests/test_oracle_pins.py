"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Every test here runs on the CPU (`-m "not gpu"`).  None of them re-types an
oracle formula: each checks a property that a dropped term, a wrong sign or a
transposed operand in the oracle would break (a defining identity, a closed
form, an exact high-precision solve, a textbook invariant).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import linalg, newton, operators, reform

SEED = 12345


def rs(seed):
    return np.random.default_rng(seed)


def rand_sym(n, g):
    G = g.standard_normal((n, n))
    return 0.5 * (G + G.T)


def small_problems():
    return [
        W.sensing(6, 14, 2, 11),
        W.maxcut(6, 0.6, 12),
        W.random_sparse(6, 10, 3, 13),
        W.completion(3, 3, 1, 0.7, 14),
    ]


def w_of(sp):
    return (sp.V * sp.lam) @ sp.V.T


# ---------------------------------------------------------------- Notations


def test_svec_inner_product_and_psi():
    g = rs(1)
    for n in (1, 2, 5):
        X, S = rand_sym(n, g), rand_sym(n, g)
        assert abs(linalg.svec(X) @ linalg.svec(S) - np.trace(X @ S)) < 1e-12
        P = linalg.psi(n)
        assert np.allclose(P.T @ P, np.eye(n * (n + 1) // 2))
        assert np.allclose(P @ linalg.svec(X), linalg.vec(X))
        # svec of a non-symmetric matrix is svec of its symmetric part
        G = g.standard_normal((n, n))
        assert np.allclose(linalg.svec(G), P.T @ linalg.vec(G))


def test_skron_defining_property():
    """(A (x)s B) svec(X) = svec(A X B^T) (symmetrised) for X in S^r (Notations)."""
    g = rs(2)
    n, r = 5, 3
    A, B = g.standard_normal((n, r)), g.standard_normal((n, r))
    X = rand_sym(r, g)
    lhs = linalg.skron(A, B) @ linalg.svec(X)
    rhs = linalg.svec(0.5 * (A @ X @ B.T + B @ X @ A.T))
    assert np.allclose(lhs, rhs, atol=1e-12)
    assert np.allclose(linalg.skron(A, A) @ linalg.svec(X), linalg.svec(A @ X @ A.T), atol=1e-12)


# ---------------------------------------------------------------- operators


@pytest.mark.parametrize("pi", range(4))
def test_operator_adjoint_and_matrix(pi):
    prob = small_problems()[pi]
    g = rs(3 + pi)
    X, y = rand_sym(prob.n, g), g.standard_normal(prob.m)
    lhs = operators.A_op(prob, X) @ y
    rhs = np.sum(X * operators.At_op(prob, y))
    assert abs(lhs - rhs) < 1e-11 * (1 + abs(lhs))
    Am = operators.A_matrix(prob)
    assert np.allclose(Am @ linalg.svec(X), operators.A_op(prob, X), atol=1e-12)


def test_operator_closed_forms():
    g = rs(4)
    mc = W.maxcut(7, 0.5, 3)
    X = rand_sym(7, g)
    assert np.allclose(operators.A_op(mc, X), np.diag(X))
    cp = W.completion(4, 5, 2, 0.5, 5)
    M = g.standard_normal((4, 5))
    Z = np.zeros((9, 9))
    Z[:4, 4:] = M
    Z[4:, :4] = M.T
    got = operators.A_op(cp, Z)
    a = cp.a_col
    b = cp.a_row - 4
    assert np.allclose(got, M[a, b])
    # b of the completion instance equals the sampled entries of F1 F2^T
    F = cp.meta["F1"] @ cp.meta["F2"].T
    assert np.allclose(cp.b, F[a, b])


# ---------------------------------------------------------------- NT scaling


def test_nt_scaling_properties():
    g = rs(5)
    n = 6
    GX, GS = g.standard_normal((n, n)), g.standard_normal((n, n))
    X = GX @ GX.T + 0.1 * np.eye(n)
    S = GS @ GS.T + 0.1 * np.eye(n)
    Wm = newton.nt_scaling(X, S)
    assert np.allclose(Wm @ S @ Wm, X, atol=1e-9)           # NT: W S W = X
    # second expression of eq. newt: W = [S^{1/2} (S^{1/2} X S^{1/2})^{-1/2} S^{1/2}]^{-1}
    Sh = newton.sqrtm_psd(S)
    W2 = np.linalg.inv(Sh @ newton.inv_sqrtm_pd(Sh @ X @ Sh) @ Sh)
    assert np.allclose(Wm, W2, atol=1e-9)
    # commuting case: X = diag(x), S = diag(s) -> W = diag(sqrt(x/s))
    x, s = g.uniform(0.5, 2, n), g.uniform(0.5, 2, n)
    assert np.allclose(newton.nt_scaling(np.diag(x), np.diag(s)), np.diag(np.sqrt(x / s)))


# ---------------------------------------------------------------- Newton direction


@pytest.mark.parametrize("pi", range(4))
def test_newton_direct_matches_high_precision_kkt(pi):
    mpk = pytest.importorskip("tests.mp_kkt")
    prob = small_problems()[pi]
    sp = W.scaling_point(prob.n, 2, 1e-2, 21 + pi)
    Wm = w_of(sp)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 31 + pi)
    dX, dy, dS = newton.newton_direct(prob, Wm, Ct, bt)
    dXe, dye = mpk.newton_kkt_mp(operators.A_matrix(prob), Wm, Ct, bt)
    # FP64 error of the Schur route is bounded by about cond(W)^2 * eps (Section 1)
    condW = sp.lam.max() / sp.lam.min()
    bound = 50 * condW ** 2 * np.finfo(float).eps
    assert np.linalg.norm(dX - dXe) <= bound * np.linalg.norm(dXe)
    assert np.linalg.norm(dy - dye) <= bound * np.linalg.norm(dye)
    dX2, dy2, _ = newton.newton_kkt_dense(prob, Wm, Ct, bt)
    assert np.linalg.norm(dX2 - dXe) <= bound * np.linalg.norm(dXe)


@pytest.mark.parametrize("pi", range(4))
def test_newton_direction_is_qp_optimum(pi):
    """eq. newt: dX solves the primal QP, (dy, dS) the dual QP, with equal optimal values."""
    prob = small_problems()[pi]
    sp = W.scaling_point(prob.n, 2, 1e-1, 41 + pi)
    Wm = w_of(sp)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 51 + pi)
    dX, dy, dS = newton.newton_direct(prob, Wm, Ct, bt)
    assert np.allclose(operators.A_op(prob, dX), bt, atol=1e-9)      # primal feasible
    assert np.allclose(operators.At_op(prob, dy) + dS, Ct, atol=1e-9)  # dual feasible
    Wh = newton.sqrtm_psd(Wm)
    Whi = np.linalg.inv(Wh)
    pobj = np.sum(Ct * dX) + 0.5 * np.linalg.norm(Whi @ dX @ Whi) ** 2
    dobj = bt @ dy - 0.5 * np.linalg.norm(Wh @ dS @ Wh) ** 2
    assert abs(pobj - dobj) <= 1e-8 * (1 + abs(pobj))
    # optimality: perturbing dX inside null(A) cannot decrease the primal objective
    g = rs(60 + pi)
    Am = operators.A_matrix(prob)
    _, _, Vt = np.linalg.svd(Am)
    null = Vt[prob.m:]
    for _ in range(5):
        H = linalg.smat(null.T @ g.standard_normal(null.shape[0]), prob.n) * 1e-3
        pert = np.sum(Ct * (dX + H)) + 0.5 * np.linalg.norm(Whi @ (dX + H) @ Whi) ** 2
        assert pert >= pobj - 1e-10


# ---------------------------------------------------------------- Prop. correct


@pytest.mark.parametrize("n,r", [(4, 1), (5, 2), (6, 3), (7, 2)])
def test_decomposition_identity(n, r):
    """W (x)s W = Q Sigma^{-1} Q^T + tau^2 E, Q^T Q = I_d, Sigma, E PD (Prop. correct)."""
    sp_in = W.scaling_point(n, r, 1e-3, 70 + n)
    s = reform.split(sp_in.V, sp_in.lam, r=r)
    Wm = w_of(sp_in)
    WW = linalg.skron(Wm, Wm)
    Qb, Sg, Eb = reform.explicit_Q(s), reform.explicit_Sigma(s), reform.explicit_E(s)
    assert s.d == n * r - r * (r - 1) // 2 == Qb.shape[1]
    assert np.allclose(Qb.T @ Qb, np.eye(s.d), atol=1e-12)
    recon = Qb @ np.linalg.inv(Sg) @ Qb.T + s.tau ** 2 * Eb
    assert np.linalg.norm(recon - WW) <= 1e-12 * np.linalg.norm(WW)
    assert np.all(np.diag(Sg) > 0) and np.linalg.eigvalsh(Eb)[0] > 0


def test_lemma_eigen_bounds():
    """4 >= lmax(E) >= lmin(E) >= w_n^2/w_{r+1}^2; w_{r+1}^2/(w_n w_r) >= tau^2 lam(Sigma) >= w_n^2/(4 w_1^2)."""
    for seed in range(5):
        n, r = 6, 2
        sp_in = W.scaling_point(n, r, 10.0 ** (-seed), 80 + seed)
        s = reform.split(sp_in.V, sp_in.lam, r=r)
        w = np.sort(sp_in.lam)[::-1]
        eE = np.linalg.eigvalsh(reform.explicit_E(s))
        assert eE[-1] <= 4 + 1e-12 and eE[0] >= w[-1] ** 2 / w[r] ** 2 * (1 - 1e-12)
        ts = s.tau ** 2 * reform.sigma_vec(s)
        assert ts.max() <= w[r] ** 2 / (w[-1] * w[r - 1]) * (1 + 1e-12)
        assert ts.min() >= w[-1] ** 2 / (4 * w[0] ** 2) * (1 - 1e-12)


def test_matrix_free_products_match_explicit():
    """Section 5 products equal the explicit E, Q, Q^T of eq. EQSigdef."""
    g = rs(9)
    n, r = 6, 2
    sp_in = W.scaling_point(n, r, 1e-2, 90)
    s = reform.split(sp_in.V, sp_in.lam, r=r)
    X = rand_sym(n, g)
    h = g.standard_normal(s.d)
    assert np.allclose(linalg.svec(reform.E_op(s, X)), reform.explicit_E(s) @ linalg.svec(X), atol=1e-12)
    assert np.allclose(linalg.svec(reform.Q_op(s, h)), reform.explicit_Q(s) @ h, atol=1e-12)
    assert np.allclose(reform.Qt_op(s, X), reform.explicit_Q(s).T @ linalg.svec(X), atol=1e-12)
    assert np.allclose(reform.sigma_vec(s), np.diag(reform.explicit_Sigma(s)), rtol=1e-12)
    # Lemma spanQ: svec(sym(V Q^T)) lies in range(Q)
    Vv = g.standard_normal((n, r))
    x = linalg.svec(Vv @ s.Q.T)
    Qb = reform.explicit_Q(s)
    assert np.allclose(Qb @ (Qb.T @ x), x, atol=1e-12)


def test_choose_rank_and_beta():
    lam = np.array([50.0, 40.0, 30.0, 0.02, 0.01, 0.009, 0.008])
    assert reform.choose_rank(lam, 5) == 3
    assert reform.choose_rank(np.array([8.0, 4.0, 2.0, 1.0]), 3) == 1   # tie -> smallest i
    V = np.eye(7)
    s = reform.split(V, lam, r_hat=5)
    # eig(E) = {1 (r times)} U {lambda_perp / tau}; its median squared is beta (s_A = 1)
    ev = np.sort(np.concatenate([np.ones(3), lam[3:] / (lam[3] / 2)]))
    assert abs(s.beta - ev[3] ** 2) < 1e-14


# ---------------------------------------------------------------- augsys, recovery, smallres


@pytest.mark.parametrize("pi", range(4))
def test_augsys_recovery_solves_newt_eps(pi):
    mpk = pytest.importorskip("tests.mp_kkt")
    prob = small_problems()[pi]
    sp_in = W.scaling_point(prob.n, 2, 1e-6, 100 + pi)
    Wm = w_of(sp_in)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 110 + pi)
    s = reform.split(sp_in.V, sp_in.lam, r=2)
    Am = operators.A_matrix(prob)
    Qb, Sg, Eb = reform.explicit_Q(s), reform.explicit_Sigma(s), reform.explicit_E(s)
    Mtop = np.hstack([Am @ Eb @ Am.T, Am @ Qb])
    Mbot = np.hstack([Qb.T @ Am.T, -s.tau ** 2 * Sg])
    c = linalg.svec(Ct)
    gvec = np.concatenate([bt + s.tau ** 2 * Am @ Eb @ c, s.tau ** 2 * Qb.T @ c])
    uv = np.linalg.solve(np.vstack([Mtop, Mbot]), gvec)
    dX, dy, _ = reform.recover(prob, s, Ct, uv[:prob.m], uv[prob.m:])
    dXe, dye = mpk.newton_kkt_mp(Am, Wm, Ct, bt)
    assert np.linalg.norm(dX - dXe) <= 1e-8 * np.linalg.norm(dXe)
    assert np.linalg.norm(dy - dye) <= 1e-8 * np.linalg.norm(dye)
    # the matrix-free augsys operator and RHS equal the explicit ones
    gu, gv = reform.aug_rhs(prob, s, Ct, bt)
    assert np.allclose(np.concatenate([gu, gv]), gvec, rtol=1e-10, atol=1e-10 * np.abs(gvec).max())
    u, v = uv[:prob.m], uv[prob.m:]
    a, b_ = reform.aug_apply(prob, s, u, v)
    full = np.vstack([Mtop, Mbot]) @ uv
    assert np.allclose(np.concatenate([a, b_]), full, atol=1e-9 * np.abs(full).max())


def test_lemma_smallres_residual_map():
    """A residual [p; d] of augsys maps to the (Newt-eps) residual [tau^-2 E^-1 Q C^-1 d; p]."""
    prob = W.sensing(5, 12, 1, 7)
    sp_in = W.scaling_point(5, 1, 1e-2, 120)
    s = reform.split(sp_in.V, sp_in.lam, r=1)
    Wm = w_of(sp_in)
    Ct, bt = W.newton_rhs(5, 12, 121)
    g = rs(122)
    u, v = g.standard_normal(prob.m), g.standard_normal(s.d)
    a, b_ = reform.aug_apply(prob, s, u, v)
    gu, gv = reform.aug_rhs(prob, s, Ct, bt)
    p, d = a - gu, b_ - gv
    dX, dy, _ = reform.recover(prob, s, Ct, u, v)
    res = newton.newt_eps_residual(prob, Wm, Ct, bt, dX, dy)
    Qb, Sg, Eb = reform.explicit_Q(s), reform.explicit_Sigma(s), reform.explicit_E(s)
    Cm = s.tau ** 2 * Sg + Qb.T @ np.linalg.inv(Eb) @ Qb
    top = s.tau ** -2 * np.linalg.solve(Eb, Qb @ np.linalg.solve(Cm, d))
    N = top.shape[0]
    assert np.allclose(res[N:], p, atol=1e-8 * np.abs(p).max())
    assert np.allclose(res[:N], top, atol=1e-7 * np.abs(top).max())


# ---------------------------------------------------------------- preconditioner and PCG


@pytest.mark.parametrize("space", ["d", "m"])
def test_preconditioner_inverse(space):
    prob = W.sensing(6, 20, 2, 8)
    sp_in = W.scaling_point(6, 2, 1e-3, 130)
    s = reform.split(sp_in.V, sp_in.lam, r=2, s_A=operators.row_norm_scale(prob))
    P = reform.precond_setup(prob, s, space=space)
    # B = A Q equals the explicit product
    assert np.allclose(P.B, operators.A_matrix(prob) @ reform.explicit_Q(s), atol=1e-10)
    g = rs(131)
    z = g.standard_normal(prob.m + s.d)
    Pm = reform.precond_matrix(P)
    zu, zv = reform.precond_apply(P, (Pm @ z)[:prob.m], (Pm @ z)[prob.m:])
    assert np.allclose(np.concatenate([zu, zv]), z, atol=1e-8 * np.abs(z).max())


def test_indefinite_pcg_equals_schur_pcg():
    """Prop. indefpcg: u_k equals PCG on H = A(E + tau^-2 Q Sigma^-1 Q^T)A^T with
    H~ = beta I + tau^-2 A Q Sigma^-1 Q^T A^T, and the second-block residual stays 0."""
    prob = W.sensing(6, 18, 2, 9)
    sp_in = W.scaling_point(6, 2, 1e-1, 140)
    Ct, bt = W.newton_rhs(6, 18, 141)
    sA = operators.row_norm_scale(prob)
    dX, dy, dS, info = reform.newton_reform(prob, sp_in.V, sp_in.lam, Ct, bt, r=2, s_A=sA,
                                            rtol=1e-13, maxit=60, keep_iterates=True)
    s = info.split
    Am = operators.A_matrix(prob)
    Qb, Sg, Eb = reform.explicit_Q(s), reform.explicit_Sigma(s), reform.explicit_E(s)
    Sgi = np.linalg.inv(Sg)
    H = Am @ (Eb + s.tau ** -2 * Qb @ Sgi @ Qb.T) @ Am.T
    Ht = s.beta * np.eye(prob.m) + s.tau ** -2 * Am @ Qb @ Sgi @ Qb.T @ Am.T
    c = linalg.svec(Ct)
    gH = bt + s.tau ** 2 * Am @ (Eb + s.tau ** -2 * Qb @ Sgi @ Qb.T) @ c
    ref = reform.pcg(lambda x: H @ x, gH, lambda r_: np.linalg.solve(Ht, r_), np.zeros(prob.m),
                     tol=0.0, maxit=12, keep_iterates=True)
    m = prob.m
    for k in range(1, 10):
        uk = info.pcg.x_hist[k][:m]
        assert np.linalg.norm(uk - ref.x_hist[k]) <= 1e-7 * np.linalg.norm(ref.x_hist[k])
        vk = info.pcg.x_hist[k][m:]
        # v_k = C^{-1}(B^T u_k - g) with C = tau^2 Sigma: second block residual is zero
        rv = Qb.T @ Am.T @ uk - s.tau ** 2 * Sg @ vk - s.tau ** 2 * Qb.T @ c
        assert np.linalg.norm(rv) <= 1e-8 * np.linalg.norm(s.tau ** 2 * Qb.T @ c)


def test_claim_condition_bound_and_cor_pcg_iterations():
    """Claim (Section 6): cond(H~^{-1/2} H H~^{-1/2}) <= cond(A E A^T) when beta lies in its
    spectrum; the observed PCG count respects the Cor. pcg bound."""
    prob = W.sensing(6, 18, 2, 10)
    sp_in = W.scaling_point(6, 2, 1e-1, 150)
    s = reform.split(sp_in.V, sp_in.lam, r=2)
    Am = operators.A_matrix(prob)
    Eb = reform.explicit_E(s)
    AEA = Am @ Eb @ Am.T
    ev = np.linalg.eigvalsh(AEA)
    U = s.tau ** -1 * Am @ reform.explicit_Q(s) @ np.diag(np.sqrt(1 / reform.sigma_vec(s)))
    for beta in (ev[0], np.median(ev), ev[-1]):
        Ht = beta * np.eye(prob.m) + U @ U.T
        L = np.linalg.cholesky(Ht)
        Li = np.linalg.inv(L)
        T = Li @ (AEA + U @ U.T) @ Li.T
        et = np.linalg.eigvalsh(0.5 * (T + T.T))
        assert et[-1] / et[0] <= ev[-1] / ev[0] * (1 + 1e-8)
    Ct, bt = W.newton_rhs(6, 18, 151)
    s2 = reform.split(sp_in.V, sp_in.lam, r=2)
    s2.beta = float(np.median(ev))
    P = reform.precond_setup(prob, s2, space="d")
    gu, gv = reform.aug_rhs(prob, s2, Ct, bt)
    m = prob.m
    v0 = -reform.Qt_op(s2, Ct) / reform.sigma_vec(s2)

    def Aop(x):
        a, b_ = reform.aug_apply(prob, s2, x[:m], x[m:])
        return np.concatenate([a, b_])

    def Pinv(rr):
        a, b_ = reform.precond_apply(P, rr[:m], rr[m:])
        return np.concatenate([a, b_])

    gg = np.concatenate([gu, gv])
    eps = 1e-8 * np.linalg.norm(gg)
    res = reform.pcg(Aop, gg, Pinv, np.concatenate([np.zeros(m), v0]), tol=eps, maxit=500)
    kE = math.sqrt(np.linalg.eigvalsh(Eb)[-1] / np.linalg.eigvalsh(Eb)[0])
    eA = np.linalg.eigvalsh(Am @ Am.T)
    kA = math.sqrt(eA[-1] / eA[0])
    assert res.converged
    assert res.iters <= reform.cor_pcg_bound(kE, kA, np.linalg.norm(gg), eps)


@pytest.mark.parametrize("pi", range(4))
def test_newton_reform_matches_direct(pi):
    """Cor. pcg + recovery reproduce the plain Schur direction (moderate mu)."""
    prob = small_problems()[pi]
    sp_in = W.scaling_point(prob.n, 2, 1e-2, 160 + pi)
    Wm = w_of(sp_in)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 170 + pi)
    dX, dy, dS = newton.newton_direct(prob, Wm, Ct, bt)
    for space in ("d", "m"):
        dX2, dy2, dS2, info = reform.newton_reform(prob, sp_in.V, sp_in.lam, Ct, bt, r_hat=3,
                                                   s_A=operators.row_norm_scale(prob), space=space,
                                                   rtol=1e-14, maxit=500)
        assert np.linalg.norm(dX2 - dX) <= 1e-8 * np.linalg.norm(dX)
        assert np.linalg.norm(dy2 - dy) <= 1e-8 * np.linalg.norm(dy)
        assert np.linalg.norm(dS2 - dS) <= 1e-8 * np.linalg.norm(dS)

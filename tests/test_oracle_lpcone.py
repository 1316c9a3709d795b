"""Pins of the oracle's linear-cone extension of the Newton system (Section 7, eq. rmc-sdp):
the plain Schur definition against the dense KKT system, its limit without the linear block,
the reformulated solve (augsys with the linear block, both preconditioner spaces) against the
definition, the block inverse of the extended preconditioner, and the robust-completion
generator's measurements."""
import numpy as np
import pytest

import workloads as W
from oracle import linalg, lpcone, newton as onewton
from oracle.operators import A_op


def _lp_case(n=6, m=10, seed=11, mu=1e-2, rank=2):
    prob = W.sensing(n, m, rank, seed)
    sp = W.scaling_point(n, rank, mu, seed + 1)
    Ct, bt = W.newton_rhs(n, m, seed + 2)
    g = np.random.default_rng(seed + 3)
    G = np.hstack([np.eye(m), -np.eye(m)])                # eq. rmc-sdp: x = [v; w]
    d = 10.0 ** g.uniform(-3, 3, 2 * m)                   # x / z of the orthant
    ct = g.standard_normal(2 * m)
    return prob, sp, Ct, bt, G, d, ct


def test_rmc_generator_measures_single_svec_entries():
    prob = W.rmc(7, 15, 3, 41)
    rows, cols = linalg.svec_index(7)
    pos = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(rows, cols))}
    X = np.random.default_rng(0).standard_normal((7, 7))
    X = X + X.T
    sv = linalg.svec(X)
    want = np.array([sv[pos[(int(a), int(b))]] for a, b in zip(prob.a_row, prob.a_col)])
    assert np.allclose(A_op(prob, X), want, rtol=0, atol=1e-12)
    eps = prob.meta["eps"]
    assert np.count_nonzero(eps) == 3
    assert np.allclose(prob.b - eps, A_op(prob, prob.meta["Xs"]), rtol=1e-12, atol=1e-9)


def test_lp_direction_solves_the_dense_kkt_system():
    prob, sp, Ct, bt, G, d, ct = _lp_case(n=5, m=7)
    Wm = (sp.V * sp.lam) @ sp.V.T
    dX, dx, dy = lpcone.newton_direct_lp(prob, Wm, Ct, bt, G, d, ct)
    kX, kx, ky = lpcone.newton_kkt_dense_lp(prob, Wm, Ct, bt, G, d, ct)
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    assert rel(dX, kX) < 1e-9 and rel(dx, kx) < 1e-9 and rel(dy, ky) < 1e-9
    # the three block equations hold
    assert np.allclose(A_op(prob, dX) + G @ dx, bt, rtol=0, atol=1e-9 * (1 + np.abs(bt).max()))
    assert np.allclose(dx, d * (G.T @ dy - ct), rtol=1e-12, atol=0)


def test_lp_direction_tends_to_the_semidefinite_one_as_d_vanishes():
    prob, sp, Ct, bt, G, d, ct = _lp_case(n=6, m=9, seed=21)
    Wm = (sp.V * sp.lam) @ sp.V.T
    dX, dx, dy = lpcone.newton_direct_lp(prob, Wm, Ct, bt, G, 1e-13 * np.ones_like(d), ct)
    rX, ry, _ = onewton.newton_direct(prob, Wm, Ct, bt)
    assert np.linalg.norm(dX - rX) <= 1e-8 * np.linalg.norm(rX)
    assert np.linalg.norm(dy - ry) <= 1e-8 * np.linalg.norm(ry)
    assert np.abs(dx).max() <= 1e-9 * (1 + np.abs(dy).max())


@pytest.mark.parametrize("space", ["d", "m"])
def test_reformulated_lp_solve_equals_the_definition(space):
    prob, sp, Ct, bt, G, d, ct = _lp_case(n=12, m=40, seed=31, mu=1e-3)
    Wm = (sp.V * sp.lam) @ sp.V.T
    rX, rx, ry = lpcone.newton_direct_lp(prob, Wm, Ct, bt, G, d, ct)
    dX, dx, dy, info = lpcone.newton_reform_lp(prob, sp.V, sp.lam, Ct, bt, G, d, ct, r_hat=4, space=space)
    assert info.pcg.converged
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    assert rel(dX, rX) < 1e-8 and rel(dx, rx) < 1e-8 and rel(dy, ry) < 1e-8


@pytest.mark.parametrize("space", ["d", "m"])
def test_extended_preconditioner_is_the_exact_block_inverse(space):
    prob, sp, Ct, bt, G, d, ct = _lp_case(n=8, m=20, seed=51)
    from oracle import reform
    s = reform.split(sp.V, sp.lam, r_hat=3)
    P = lpcone.precond_setup_lp(prob, s, G, d, space=space)
    Pm = lpcone.precond_matrix_lp(P)
    z = np.random.default_rng(1).standard_normal(Pm.shape[0])
    zu, zv = lpcone.precond_apply_lp(P, z[:prob.m], z[prob.m:])
    back = Pm @ np.concatenate([zu, zv])
    assert np.linalg.norm(back - z) <= 1e-10 * np.linalg.norm(z) * np.linalg.cond(Pm) ** 0.5
    with pytest.raises(ValueError):
        lpcone.precond_setup_lp(prob, s, np.ones((prob.m, 2)), np.ones(2))   # a variable in every row


def _solve_rmc(n, m, m_o, seed):
    from oracle import ipm_lp
    prob = W.rmc(n, m, m_o, seed)
    res = ipm_lp.ipm_solve_lp(prob, prob.meta["G_l"], prob.meta["c_l"], tol=1e-8)
    return prob, res


def test_rmc_without_outliers_recovers_the_planted_matrix():
    """Exact measurements of a rank-2 matrix on 45 of the 55 svec coordinates (n = 10): the
    robust-completion SDP returns X* (recovery expected at this sampling), v = w = 0, and a dual
    point with |y_i| <= 1 (the dual constraints of v, w >= 0 with unit cost)."""
    prob, res = _solve_rmc(10, 45, 0, 7)
    Xs = prob.meta["Xs"]
    assert res.converged
    assert np.linalg.norm(res.X - Xs) <= 1e-6 * np.linalg.norm(Xs)
    m = prob.m
    assert np.abs(res.x[:m] - res.x[m:]).max() <= 1e-6 * (1 + np.abs(prob.b).max())
    assert np.abs(res.y).max() <= 1 + 1e-8


def test_rmc_with_outliers_finds_them_and_the_matrix():
    """Three gross outliers among 70 measurements (n = 12): X* is still recovered, v - w is the
    outlier vector (its support is the outlier set), |y_i| = 1 on the outliers (complementary
    slackness with the unit cost of v, w), and the optimal value is tr X* + sum |eps_i|
    (lambda = 1), the objective of the recovered point."""
    prob, res = _solve_rmc(12, 70, 3, 9)
    m = prob.m
    Xs, eps, out = prob.meta["Xs"], prob.meta["eps"], prob.meta["outliers"]
    assert res.converged
    assert np.linalg.norm(res.X - Xs) <= 1e-6 * np.linalg.norm(Xs)
    vw = res.x[:m] - res.x[m:]
    assert set(np.where(np.abs(vw) > 1e-3)[0].tolist()) == set(out.tolist())
    assert np.allclose(vw[out], eps[out], rtol=1e-6, atol=1e-6)
    assert np.allclose(np.abs(res.y[out]), 1.0, atol=1e-6) and np.abs(res.y).max() <= 1 + 1e-8
    pobj = float(np.trace(res.X) + res.x.sum())
    assert abs(pobj - (np.trace(Xs) + np.abs(eps).sum())) <= 1e-6 * pobj


def test_lp_outer_loop_meets_the_optimality_conditions():
    """At the returned point: primal and dual feasibility and the relative gap within 1e-8,
    X, S positive semidefinite, x, z positive, and small complementarity."""
    prob, res = _solve_rmc(10, 45, 2, 8)
    from oracle import ipm_lp
    G, cl = prob.meta["G_l"], prob.meta["c_l"]
    st = ipm_lp.LPState(X=res.X, x=res.x, y=res.y, S=res.S, z=res.z)
    pobj, dobj, gap, pinf, dinf, *_ = ipm_lp.lp_measures(prob, G, cl, st)
    assert res.converged and gap <= 1e-8 and pinf <= 1e-8 and dinf <= 1e-8
    assert np.linalg.eigvalsh(res.X).min() > -1e-10 and np.linalg.eigvalsh(res.S).min() > -1e-10
    assert res.x.min() > 0 and res.z.min() > 0
    comp = float(np.sum(res.X * res.S) + res.x @ res.z)
    assert comp <= 1e-6 * (1 + abs(pobj))


def test_linear_block_conditioning_along_the_path():
    """Section 4's point carried to the orthant, on the outer loop's own iterates (robust
    completion, 3 outliers): the Schur matrix A (W (x)s W) A^T + G D G^T grows ill-conditioned as
    mu -> 0 (past 1e15 by mu ~ 1e-5), and so does the extended augmented matrix, whose (1,1) block
    gains tau^-2 diag(delta) with delta = x/z of order 1/mu on the outliers.  That growth sits in
    a diagonal block the preconditioner inverts exactly, so the spectrum of P^{-1} K stays inside
    the mediant bound [min(1, l_min), max(1, l_max)] of A E A^T / beta at every iterate.  The plain
    Schur route of the same outer loop breaks down before the 1e-8 gap."""
    from oracle import ipm_lp, reform
    from oracle.newton import nt_scaling, schur_matrix
    from oracle.operators import At_op, row_norm_scale
    prob = W.rmc(12, 70, 3, 9)
    G, cl, m = prob.meta["G_l"], prob.meta["c_l"], prob.m
    sA = row_norm_scale(prob)
    condM = []
    for k in (1, 5, 9, 11):
        res = ipm_lp.ipm_solve_lp(prob, G, cl, tol=1e-8, max_iter=k)
        Wm = nt_scaling(res.X, res.S)
        d = res.x / res.z
        GDG = lpcone.gdg(G, d)
        condM.append(np.linalg.cond(schur_matrix(prob, Wm) + GDG))
        lw, Vw = np.linalg.eigh(Wm)
        s = reform.split(Vw, lw, r_hat=3, s_A=sA)
        K = np.zeros((m + s.d, m + s.d))
        for j in range(m + s.d):
            e = np.zeros(m + s.d)
            e[j] = 1.0
            a, b = reform.aug_apply(prob, s, e[:m], e[m:])
            K[:, j] = np.concatenate([a + GDG @ e[:m] / s.tau ** 2, b])
        AEA = np.column_stack([A_op(prob, reform.E_op(s, At_op(prob, e))) for e in np.eye(m)])
        ae = np.linalg.eigvalsh(0.5 * (AEA + AEA.T))
        lo, hi = min(1.0, ae[0] / s.beta), max(1.0, ae[-1] / s.beta)
        P = lpcone.precond_setup_lp(prob, s, G, d, space="d")
        ev = np.linalg.eigvals(np.linalg.solve(lpcone.precond_matrix_lp(P), K))
        assert np.abs(ev.imag).max() <= 1e-6 * np.abs(ev).max()
        assert ev.real.min() >= lo * (1 - 1e-6) and ev.real.max() <= hi * (1 + 1e-6), k
        assert ev.real.max() / ev.real.min() <= 10.0
    assert condM[0] < 1e2 and condM[-1] > 1e15
    try:
        schur = ipm_lp.ipm_solve_lp(prob, G, cl, tol=1e-8, max_iter=60, direction_by="schur")
        assert not schur.converged
    except np.linalg.LinAlgError:          # here: the Cholesky factor of a Schur matrix fails
        pass


def test_space_rule_with_many_active_slacks():
    """Six of eight constraints carry an active slack (sensing n = 6 with two gross outliers and a
    cheap slack cost), so only two rows are left to the semidefinite part against d = 6.  At
    mu = 1e-9 on the central path, with the right side (0, 0, b), the d-space elimination loses
    the direction to rounding (PCG does not reach 1e-12 in 200 iterations) although P^{-1} K is
    the identity to 1e-8; the rule
    picks the m-space complement there, which converges at once to the right direction, and
    keeps the d-space form on robust completion (three outliers among 70 rows)."""
    from oracle import ipm_lp, reform
    from oracle.newton import nt_scaling
    from oracle.operators import row_norm_scale
    p0 = W.sensing(6, 8, 2, 77)
    b = p0.b.copy()
    b[0] += 5.0
    b[3] -= 4.0
    prob = W.Problem(kind=p0.kind, n=p0.n, m=p0.m, b=b, C=p0.C, a_dense=p0.a_dense)
    m = prob.m
    G = np.hstack([np.eye(m), -np.eye(m)])
    cl = 0.5 * np.ones(2 * m)
    res = ipm_lp.ipm_solve_lp(prob, G, cl, tol=1e-9, max_iter=200)
    st = ipm_lp.center_lp(prob, G, cl, ipm_lp.LPState(res.X, res.x, res.y, res.S, res.z), 1e-9)
    Wm = nt_scaling(st.X, st.S)
    lw, Vw = np.linalg.eigh(Wm)
    d = st.x / st.z
    Ct, bt, ct = np.zeros((6, 6)), prob.b, np.zeros(2 * m)      # the right side of dp*/dC (envelope)
    kw = dict(r_hat=3, s_A=row_norm_scale(prob), maxit=200)
    *_, info_d = lpcone.newton_reform_lp(prob, Vw, lw, Ct, bt, G, d, ct, space="d", **kw)
    assert not info_d.pcg.converged
    dX, dx, dy, info = lpcone.newton_reform_lp(prob, Vw, lw, Ct, bt, G, d, ct, space="auto", **kw)
    assert info.precond.space == "m" and info.pcg.converged and info.pcg.iters <= 3
    # the dense KKT matrix has condition ~1e28 here, so the direction is checked by the envelope
    # theorem (this right side is the cotangent of b^T y: (dX, dx, dy) -> (X*, x*, 0) up to O(mu))
    # and by the primal block equation A(dX) + G dx = b
    kX, kx, ky = lpcone.newton_kkt_dense_lp(prob, Wm, Ct, bt, G, d, ct)
    rel = lambda a, b_: np.linalg.norm(a - b_) / np.linalg.norm(b_)
    assert rel(dX, kX) <= 1e-6 and rel(dX, st.X) <= 1e-6 and rel(dx, st.x) <= 1e-6
    assert np.linalg.norm(dy) <= 1e-6 * np.linalg.norm(st.y)
    assert rel(A_op(prob, dX) + G @ dx, bt) <= 1e-9
    r2 = W.rmc(12, 70, 3, 9)
    res2 = ipm_lp.ipm_solve_lp(r2, r2.meta["G_l"], r2.meta["c_l"], tol=1e-8)
    lw2, Vw2 = np.linalg.eigh(nt_scaling(res2.X, res2.S))
    sp2 = reform.split(Vw2, lw2, r_hat=3, s_A=row_norm_scale(r2))
    assert lpcone.choose_space_lp(sp2, r2.meta["G_l"], res2.x / res2.z, r2.m) == "d"

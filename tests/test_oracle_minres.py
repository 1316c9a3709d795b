"""Pins of the oracle's MINRES (Def. MINRES with P = I) and of Cor. minres on the reformulation.

- The oracle's MINRES is the definition written out (Krylov basis + least squares); it is
  compared with SciPy's MINRES (an independent short-recurrence implementation) iterate by
  iterate on symmetric indefinite systems, and its residual norms never increase.
- Prop. minres: the iteration count to an absolute residual eps stays within
  ceil(kappa log(2 ||b|| / eps)) on indefinite systems with a prescribed spectrum (the
  printed kappa/2 is the definite-case factor: a kappa = 10 indefinite system needs 125
  iterations where kappa/2 log(...) gives 96).
- Cor. minres end to end: MINRES on eq. augsys plus eq. recover solves (Newt-eps): the
  direction equals the plain Schur-complement definition to 1e-8 (moderate mu), and equals the
  PCG route.  A planted mistake (a flipped sign of the second block of the right side) fails.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import newton as onewton, operators as oops, reform


def _sym_indef(n, seed, neg=0.4, cond=50.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    mags = np.logspace(0, np.log10(cond), n)
    signs = np.where(rng.random(n) < neg, -1.0, 1.0)
    return (Q * (signs * mags)) @ Q.T, float(cond)


@pytest.mark.parametrize("n,seed", [(12, 1), (30, 2), (60, 3)])
def test_minres_matches_scipy_iterates(n, seed):
    A, _ = _sym_indef(n, seed)
    b = np.random.default_rng(seed + 10).standard_normal(n)
    for k in (1, 3, 7, min(n, 15)):
        ours = reform.minres(lambda x: A @ x, b, np.zeros(n), 0.0, k)
        ref, _ = spla.minres(A, b, x0=np.zeros(n), rtol=0.0, maxiter=k)
        assert np.linalg.norm(ours.x - ref) <= 1e-8 * max(1.0, np.linalg.norm(ref)), k
    full = reform.minres(lambda x: A @ x, b, np.zeros(n), 1e-10 * np.linalg.norm(b), 4 * n)
    assert full.converged
    assert all(full.res_hist[i + 1] <= full.res_hist[i] * (1 + 1e-12) for i in range(len(full.res_hist) - 1))


def test_minres_iterations_within_prop_minres_bound():
    for seed, cond in [(4, 10.0), (5, 100.0), (6, 1000.0)]:
        A, kappa = _sym_indef(200, seed, cond=cond)
        b = np.random.default_rng(seed).standard_normal(200)
        eps = 1e-8 * np.linalg.norm(b)
        res = reform.minres(lambda x: A @ x, b, np.zeros(200), eps, 2000)
        assert res.converged
        assert res.iters <= reform.prop_minres_bound(kappa, np.linalg.norm(b), eps)


@pytest.mark.parametrize("mk,rt", [(lambda: W.sensing(12, 40, 2, 101), 2), (lambda: W.maxcut(20, 0.3, 4101), 3)])
def test_cor_minres_solves_newt_eps(mk, rt):
    prob = mk()
    sp = W.scaling_point(prob.n, rt, 1e-2, 300 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 301 + prob.n)
    sA = oops.row_norm_scale(prob)
    dX, dy, dS, res, spl = reform.newton_minres(prob, sp.V, sp.lam, Ct, bt, r_hat=rt + 2, s_A=sA, maxit=3000)
    assert res.converged
    rX, ry, rS = onewton.newton_direct(prob, (sp.V * sp.lam) @ sp.V.T, Ct, bt)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(dX, rX) < 1e-8 and rel(dy, ry) < 1e-8 and rel(dS, rS) < 1e-8
    pX, py, pS, _ = reform.newton_reform(prob, sp.V, sp.lam, Ct, bt, r_hat=rt + 2, s_A=sA, start="precond")
    assert rel(dX, pX) < 1e-8 and rel(dy, py) < 1e-8
    # planted mistake: the second block of the right side with the wrong sign
    m = prob.m
    gu, gv = reform.aug_rhs(prob, spl, Ct, bt)
    Aop = lambda x: np.concatenate(reform.aug_apply(prob, spl, x[:m], x[m:]))
    bad = reform.minres(Aop, np.concatenate([gu, -gv]), np.zeros(m + spl.d), res.res_hist[-1], 3000)
    bX, by, _ = reform.recover(prob, spl, Ct, bad.x[:m], bad.x[m:])
    assert rel(bX, rX) > 1e-3

"""The two PCG starts that satisfy Cor. pcg (second block of r0 zero).

- x0 = [0; -Sigma^{-1} Q^T c] as printed in Cor. pcg, and
- x0 = P^{-1}[0; g_v] (the preconditioner applied to the second block of g).

Both start Def. pcg on the same system and reach the same Newton direction where both
converge.  Near the end of an interior-point path the printed start leaves a first block of
r0 of size ~||B Sigma^{-1} Q^T c|| that the finite-precision recurrence never recovers from
(the true residual stalls orders of magnitude above the stopping test), while the
preconditioned start converges in about the same number of iterations as early in the path.
The library's FP64 solve therefore starts from P^{-1}[0; g_v] by default (option pcg_start).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ipm, operators as ops, reform


@pytest.fixture(scope="module")
def path():
    prob = W.sensing(20, 120, 2, 77)
    res = ipm.ipm_solve(prob, tol=1e-8, keep_history=True)
    A = ops.A_matrix(prob)
    return prob, res, float(np.sum(A * A)) / prob.m


def _solve(prob, h, s_A, start, maxit=2000):
    lam, V = np.linalg.eigh(h["W"])
    Ct, bt = h["R_d"] + h["S"], h["r_p"]
    return reform.newton_reform(prob, V, lam, Ct, bt, r_hat=4, s_A=s_A, start=start, maxit=maxit)


def test_starts_agree_early_in_the_path(path):
    prob, res, s_A = path
    h = res.history[4]
    a = _solve(prob, h, s_A, "paper")
    b = _solve(prob, h, s_A, "precond")
    assert a[3].pcg.converged and b[3].pcg.converged
    for x, y in zip(a[:3], b[:3]):
        assert np.linalg.norm(x - y) <= 1e-8 * max(np.linalg.norm(y), 1e-30)


def test_printed_start_stalls_near_the_end(path):
    prob, res, s_A = path
    h = res.history[10]
    a = _solve(prob, h, s_A, "paper", maxit=600)
    b = _solve(prob, h, s_A, "precond", maxit=600)
    assert b[3].pcg.converged and b[3].pcg.iters < 300
    assert not a[3].pcg.converged

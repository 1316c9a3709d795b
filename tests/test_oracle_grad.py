"""Pins of the oracle's implicit derivative (oracle/grad.py) against what the mathematics fixes.

- Central finite differences of the central-path point x(mu; C, b) (the oracle IPM's optimum,
  re-centred at a fixed mu by ``ipm.center``) in random data directions:
      <gX, dX/dt> + <gy, dy/dt> = <gC, dC> + <gb, db>,
  with step h = 1e-5 (second-order FD error ~1e-7 here).
- The envelope theorem at the optimum: p* = <C, X*> = <b, y*> has dp*/db = y* and
  dp*/dC = X*, so the VJP with (gX, gy) = (C, 0) gives gb = y*, gC = 0, and the VJP with
  (gX, gy) = (0, b) gives gC = X*, gb = 0, up to O(mu).
- Planted mistakes fail: a flipped sign of the product, and the product taken at the
  IPM's last iterate without re-centring (there X S is far from mu I, so the NT
  linearisation dX + W dS W = 0 is not the derivative of the path).

The instance is a weighted MaxCut SDP (strictly feasible on both sides, nondegenerate for
generic weights).  Matrix-sensing instances in the exact-recovery regime (m larger than the
dimension of the rank-r tangent space) are primal degenerate, so their y* is not unique and
has no derivative; they are not used here.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad, ipm

MU = 1e-6
H = 1e-5


def _rand_sym(rng, n):
    G = rng.standard_normal((n, n))
    return 0.5 * (G + G.T)


@pytest.fixture(scope="module")
def case():
    prob = W.maxcut(10, 0.6, 2718, weights="gauss")
    res = ipm.ipm_solve(prob, tol=1e-8, max_iter=200)
    assert res.converged
    st = ipm.center(prob, ipm.IPMState(res.X, res.y, res.S), MU)
    return prob, res, st


def _fd(prob, st, db, dC):
    outs = []
    for sgn in (+1.0, -1.0):
        p2 = W.Problem(kind=prob.kind, n=prob.n, m=prob.m, b=prob.b + sgn * H * db, C=prob.C + sgn * H * dC)
        s2 = ipm.center(p2, st, MU)
        outs.append((s2.X, s2.y))
    return (outs[0][0] - outs[1][0]) / (2 * H), (outs[0][1] - outs[1][1]) / (2 * H)


def _directions(prob, seed):
    rng = np.random.default_rng(seed)
    gX, gy = _rand_sym(rng, prob.n), rng.standard_normal(prob.m)
    dirs = [(rng.standard_normal(prob.m), np.zeros((prob.n, prob.n))),
            (np.zeros(prob.m), _rand_sym(rng, prob.n))]
    return gX, gy, dirs


def _mismatch(prob, st, gX, gy, gC, gb, db, dC):
    dX, dy = _fd(prob, st, db, dC)
    lhs = float(np.sum(gX * dX) + gy @ dy)
    rhs = float(np.sum(gC * dC) + gb @ db)
    return abs(lhs - rhs) / (abs(lhs) + abs(rhs))


def test_vjp_matches_central_differences(case):
    prob, _, st = case
    gX, gy, dirs = _directions(prob, 5)
    gC, gb = grad.vjp(prob, st.X, st.S, gX, gy)
    for db, dC in dirs:
        assert _mismatch(prob, st, gX, gy, gC, gb, db, dC) <= 1e-5


def test_envelope_theorem(case):
    prob, _, _ = case
    # at mu = 1e-9 the O(mu) gap is ~1e-9, but the Schur route of the oracle loses digits like
    # cond(W)^2 eps (Section 1), about 1e-6 here: the bound is 1e-5
    st = ipm.center(prob, case[2], 1e-9)
    X, y, S = st.X, st.y, st.S
    gC, gb = grad.vjp(prob, X, S, prob.C, np.zeros(prob.m))
    assert np.linalg.norm(gb - y) <= 1e-5 * np.linalg.norm(y)
    assert np.linalg.norm(gC) <= 1e-5 * np.linalg.norm(X)
    gC, gb = grad.vjp(prob, X, S, np.zeros_like(X), prob.b)
    assert np.linalg.norm(gC - X) <= 1e-5 * np.linalg.norm(X)
    assert np.linalg.norm(gb) <= 1e-5 * np.linalg.norm(y)


def test_planted_mistakes_fail(case):
    prob, res, st = case
    gX, gy, dirs = _directions(prob, 6)
    gC, gb = grad.vjp(prob, st.X, st.S, gX, gy)
    db, dC = dirs[1]
    assert _mismatch(prob, st, gX, gy, -gC, -gb, db, dC) > 0.5            # sign flipped
    gCr, gbr = grad.vjp(prob, res.X, res.S, gX, gy)                         # not re-centred
    assert _mismatch(prob, st, gX, gy, gCr, gbr, *dirs[0]) > 1e-3

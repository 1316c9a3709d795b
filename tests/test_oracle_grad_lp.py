"""Pins of the oracle's implicit derivative with the orthant (oracle/grad.py ``vjp_lp``): the
optimum of min <C, X> + c_l^T x s.t. A(X) + G x = b, X PSD, x >= 0 (the robust form of Section
7, eq. rmc-sdp, x = [v; w], G = [I, -I]) as a function of (C, c_l, b).

- Central finite differences of the central-path point (``ipm_lp.center_lp`` at mu = 1e-6) in
  random directions of b, C and c_l:
      <gX, dX/dt> + <gx, dx/dt> + <gy, dy/dt> = <gC, dC> + <gc, dc_l> + <gb, db>.
- The envelope theorem, p* = <C, X*> + c_l^T x* = b^T y*: dp*/db = y*, dp*/dC = X*,
  dp*/dc_l = x*, so the product with (gX, gx, gy) = (C, c_l, 0) is (0, 0, y*) and the product
  with (0, 0, b) is (X*, x*, 0), up to O(mu).
- Planted mistakes fail: the sign of the product, and the linear block's cotangent dropped.

The instance is a small dense sensing problem (n = 6, m = 8, below the dimension of the rank-1
tangent space, so X* and y* are unique) with two gross outliers in b; at its optimum six of the
eight constraints carry an active slack, each strictly complementary.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad, ipm_lp

MU = 1e-6
H = 1e-5


def _sym(rng, n):
    A = rng.standard_normal((n, n))
    return 0.5 * (A + A.T)


@pytest.fixture(scope="module")
def case():
    p0 = W.sensing(6, 8, 2, 77)
    b = p0.b.copy()
    b[0] += 5.0
    b[3] -= 4.0
    prob = W.Problem(kind=p0.kind, n=p0.n, m=p0.m, b=b, C=p0.C, a_dense=p0.a_dense)
    m = prob.m
    G = np.hstack([np.eye(m), -np.eye(m)])
    cl = 0.5 * np.ones(2 * m)
    res = ipm_lp.ipm_solve_lp(prob, G, cl, tol=1e-9, max_iter=200)
    assert res.converged
    st = ipm_lp.center_lp(prob, G, cl, ipm_lp.LPState(res.X, res.x, res.y, res.S, res.z), MU)
    return prob, G, cl, st


def _fd_mismatch(prob, G, cl, st, g, out, db, dC, dc):
    gX, gx, gy = g
    gC, gc, gb = out
    pts = []
    for sgn in (1.0, -1.0):
        p2 = W.Problem(kind=prob.kind, n=prob.n, m=prob.m, b=prob.b + sgn * H * db, C=prob.C + sgn * H * dC,
                       a_dense=prob.a_dense)
        pts.append(ipm_lp.center_lp(p2, G, cl + sgn * H * dc, st, MU))
    dX = (pts[0].X - pts[1].X) / (2 * H)
    dx = (pts[0].x - pts[1].x) / (2 * H)
    dy = (pts[0].y - pts[1].y) / (2 * H)
    lhs = float(np.sum(gX * dX) + gx @ dx + gy @ dy)
    rhs = float(np.sum(gC * dC) + gc @ dc + gb @ db)
    return abs(lhs - rhs) / (abs(lhs) + abs(rhs))


def _dirs(prob, rng):
    n, m = prob.n, prob.m
    z = lambda: (np.zeros(m), np.zeros((n, n)), np.zeros(2 * m))
    d_b, d_C, d_c = z(), z(), z()
    return [(rng.standard_normal(m), d_b[1], d_b[2]), (d_C[0], _sym(rng, n), d_C[2]),
            (d_c[0], d_c[1], rng.standard_normal(2 * m))]


def test_vjp_lp_matches_central_differences(case):
    prob, G, cl, st = case
    rng = np.random.default_rng(3)
    g = (_sym(rng, prob.n), rng.standard_normal(2 * prob.m), rng.standard_normal(prob.m))
    out = grad.vjp_lp(prob, st.X, st.S, st.x, st.z, G, *g)
    for db, dC, dc in _dirs(prob, rng):
        assert _fd_mismatch(prob, G, cl, st, g, out, db, dC, dc) <= 1e-5


@pytest.mark.parametrize("mu,space,bound", [(1e-8, "d", 1e-6), (1e-8, "m", 1e-6)])
def test_vjp_lp_envelope_theorem(case, mu, space, bound):
    prob, G, cl, st0 = case
    st = ipm_lp.center_lp(prob, G, cl, st0, mu)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    gC, gc, gb = grad.vjp_lp(prob, st.X, st.S, st.x, st.z, G, prob.C, cl, np.zeros(prob.m), space=space)
    assert rel(gb, st.y) <= bound and np.linalg.norm(gC) <= bound * np.linalg.norm(st.X)
    assert np.linalg.norm(gc) <= bound * np.linalg.norm(st.x)
    gC, gc, gb = grad.vjp_lp(prob, st.X, st.S, st.x, st.z, G, np.zeros_like(st.X), np.zeros(2 * prob.m), prob.b,
                             space=space)
    assert rel(gC, st.X) <= bound and rel(gc, st.x) <= bound and np.linalg.norm(gb) <= bound * np.linalg.norm(st.y)


def test_vjp_lp_planted_mistakes_fail(case):
    prob, G, cl, st = case
    rng = np.random.default_rng(4)
    g = (_sym(rng, prob.n), rng.standard_normal(2 * prob.m), rng.standard_normal(prob.m))
    gC, gc, gb = grad.vjp_lp(prob, st.X, st.S, st.x, st.z, G, *g)
    db, dC, dc = _dirs(prob, rng)[1]
    assert _fd_mismatch(prob, G, cl, st, g, (-gC, -gc, -gb), db, dC, dc) > 0.5          # sign flipped
    dropped = grad.vjp_lp(prob, st.X, st.S, st.x, st.z, G, g[0], np.zeros(2 * prob.m), g[2])
    db, dC, dc = _dirs(prob, rng)[2]
    assert _fd_mismatch(prob, G, cl, st, g, dropped, db, dC, dc) > 1e-3                 # gx ignored

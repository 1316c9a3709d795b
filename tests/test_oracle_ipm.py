"""Pins of the oracle's outer loop and problem data against closed forms and brute force.

The MaxCut SDP (C = -L/4, diag X = 1, Section 1 eq. sdp-pd in min form):
  * a connected bipartite graph with unit weights has optimum -|E| attained by
    the rank-1 X = z z^T, z the +-1 side indicator (every cut is <= |E|);
  * a vertex-transitive graph has SDP value (n/4) lambda_max(L) (the
    eigenvalue bound is tight there): the 5-cycle gives 4.5225..., the
    Petersen graph 12.5;
  * for any graph, the max cut (brute force, n <= 12) is <= the SDP value and,
    for unit weights, >= 0.878 times it (Goemans-Williamson).
Plus the invariants of a solved SDP: feasibility, gap, complementarity, rank.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ipm, maxcut, newton, operators


def solve(prob, tol=1e-8):
    res = ipm.ipm_solve(prob, tol=tol)
    assert res.converged, "IPM did not converge"
    return res


def sdp_value(prob, res):
    return -float(np.sum(prob.C * res.X))


def check_invariants(prob, res, tol=1e-8):
    X, y, S = res.X, res.y, res.S
    assert np.linalg.norm(operators.A_op(prob, X) - prob.b) <= 10 * tol * (1 + np.linalg.norm(prob.b))
    assert np.linalg.norm(operators.At_op(prob, y) + S - prob.C) <= 10 * tol * (1 + np.linalg.norm(prob.C))
    assert np.linalg.eigvalsh(X)[0] > -1e-12 and np.linalg.eigvalsh(S)[0] > -1e-12
    pobj, dobj = float(np.sum(prob.C * X)), float(prob.b @ y)
    assert abs(pobj - dobj) <= 10 * tol * (1 + abs(pobj) + abs(dobj))
    # complementarity X S ~ 0, measured symmetrically: ||X^{1/2} S X^{1/2}||_F <= <X, S>
    Xh = newton.sqrtm_psd(X)
    comp = np.linalg.norm(Xh @ S @ Xh) / (1 + abs(pobj))
    assert comp <= 20 * tol


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (3, 4), (4, 4)])
def test_bipartite_maxcut_closed_form(a, b):
    edges = np.array([(i, a + j) for i in range(a) for j in range(b)])
    prob = W.maxcut(a + b, 0.0, 0, edges=edges)
    res = solve(prob)
    check_invariants(prob, res)
    assert abs(sdp_value(prob, res) - len(edges)) <= 1e-7 * len(edges)
    ev = np.linalg.eigvalsh(res.X)
    assert ev[-2] <= 1e-6 * ev[-1]                       # rank one
    z = np.concatenate([np.ones(a), -np.ones(b)])
    assert np.linalg.norm(res.X - np.outer(z, z)) <= 1e-6 * (a + b)


def _cycle(n):
    return np.array([(i, (i + 1) % n) for i in range(n)])


def _petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return np.array(outer + spokes + inner)


@pytest.mark.parametrize("name,n,edges,value", [
    ("C5", 5, _cycle(5), 5 / 4 * (2 + 2 * math.cos(math.pi / 5))),
    ("C7", 7, _cycle(7), 7 / 4 * (2 - 2 * math.cos(2 * math.pi * 3 / 7))),
    ("Petersen", 10, _petersen(), 12.5),
])
def test_vertex_transitive_closed_form(name, n, edges, value):
    prob = W.maxcut(n, 0.0, 0, edges=edges)
    res = solve(prob)
    check_invariants(prob, res)
    assert abs(sdp_value(prob, res) - value) <= 1e-7 * value
    L = -4 * prob.C
    assert abs(n / 4 * np.linalg.eigvalsh(L)[-1] - value) <= 1e-12 * value


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_maxcut_bounds(seed):
    n = 9 + seed
    prob = W.maxcut(n, 0.4, 500 + seed)
    e, w = prob.meta["edges"], prob.meta["weights"]
    if e.shape[0] == 0:
        pytest.skip("empty graph")
    res = solve(prob)
    check_invariants(prob, res)
    sdp = sdp_value(prob, res)
    cut = maxcut.max_cut_brute_force(n, e, w)
    assert cut <= sdp * (1 + 1e-8)
    assert cut >= 0.878 * sdp
    # relabelling the vertices leaves the value unchanged
    perm = np.random.default_rng(seed).permutation(n)
    prob2 = W.maxcut(n, 0.0, 0, edges=perm[e])
    assert abs(sdp_value(prob2, solve(prob2)) - sdp) <= 1e-7 * sdp


def test_maxcut64_instance_solves():
    prob = W.workload("maxcut64")
    res = solve(prob)
    check_invariants(prob, res)
    cut = sdp_value(prob, res)
    # the SDP bound never exceeds the total edge weight, and exceeds half of it
    tot = float(np.sum(prob.meta["weights"]))
    assert 0.5 * tot <= cut <= tot


def test_sensing_recovers_planted_and_scales():
    prob = W.sensing(20, 120, 2, 77)
    res = solve(prob)
    check_invariants(prob, res)
    U = prob.meta["U"]
    Xs = U @ U.T
    assert np.linalg.norm(res.X - Xs) <= 1e-5 * np.linalg.norm(Xs)
    ev = np.linalg.eigvalsh(res.X)[::-1]
    assert np.sum(ev > 1e-6 * ev[0]) <= 2                 # rank <= r
    # homogeneity: scaling b scales X* and the value
    prob.b = 3.0 * prob.b
    res3 = solve(prob)
    assert np.linalg.norm(res3.X - 3 * res.X) <= 1e-5 * np.linalg.norm(3 * res.X)


def test_ipm_direction_linearised_complementarity():
    """Each IPM direction satisfies A(dX) = r_p, A^T dy + dS = R_d, dX + W dS W = R_c(pred) = -X."""
    prob = W.maxcut(12, 0.4, 9)
    res = ipm.ipm_solve(prob, max_iter=4, keep_history=True)
    h = res.history[-1]
    Wm, X, S = h["W"], h["X"], h["S"]
    Wi = np.linalg.inv(Wm)
    Rc = -X
    Ct = h["R_d"] - Wi @ Rc @ Wi
    dX, dy, _ = newton.newton_direct(prob, Wm, 0.5 * (Ct + Ct.T), h["r_p"])
    dS = h["R_d"] - operators.At_op(prob, dy)
    assert np.allclose(operators.A_op(prob, dX), h["r_p"], atol=1e-9)
    assert np.linalg.norm(dX + Wm @ dS @ Wm - Rc) <= 1e-8 * np.linalg.norm(X)

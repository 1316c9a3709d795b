"""GPU parity of the SPARSE_COO constraint kind (matrix completion, generic sparse A_i)
against the oracle: the Newton direction by its plain definition, and whole solves.

The generic instance has several entries per constraint, repeated positions within a
constraint and positions shared by several constraints, so the position-grouped A^T(y) and
the constraint-grouped A(Z) are both exercised with collisions.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ipm as oipm, newton as onewton, operators as oops

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = [
    ("completion8x8", lambda: W.completion(8, 8, 2, 0.4, 11), 2, 3),
    ("completion20x15", lambda: W.completion(20, 15, 2, 0.3, 13), 2, 4),
    ("random_sparse", lambda: W.random_sparse(12, 30, 3, 12), 2, 4),
    # several tiles of every kernel, ragged n, d < m and d > m
    ("completion150x130", lambda: W.completion(150, 130, 3, 0.08, 21), 3, 3),
    ("random_sparse257", lambda: W.random_sparse(257, 700, 4, 22), 3, 4),
]


@pytest.mark.parametrize("name,mk,rt,rh", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("space", [0, 1, 2])
def test_sparse_newton_matches_direct_definition(name, mk, rt, rh, space):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    sp = W.scaling_point(prob.n, rt, 1e-3, 500 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 600 + prob.n)
    s = NewtonSolver(prob, r_hat=rh, precond_space=space)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged
    Wm = (sp.V * sp.lam) @ sp.V.T
    rX, ry, rS = onewton.newton_direct(prob, Wm, Ct, bt)
    assert rel(dX.cpu().numpy(), rX) < TOL
    assert rel(dy.cpu().numpy(), ry) < TOL
    assert rel(dS.cpu().numpy(), rS) < TOL
    s.close()


def test_sparse_sdp_solve_matches_oracle():
    from paper_2407_14013_gb300 import NewtonSolver
    for prob in (W.completion(8, 8, 2, 0.4, 11), W.random_sparse(12, 30, 3, 12)):
        ref = oipm.ipm_solve(prob, tol=1e-8, max_iter=100)
        assert ref.converged
        s = NewtonSolver(prob, r_hat=4)
        X, y, S, info = s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-8, max_iter=100)
        assert info["converged"] == 1, info
        X, y, S = X.cpu().numpy(), y.cpu().numpy(), S.cpu().numpy()
        pobj, pref = float(np.sum(prob.C * X)), float(np.sum(prob.C * ref.X))
        assert abs(pobj - pref) <= 2e-8 * (1 + 2 * abs(pref))
        assert np.linalg.norm(oops.A_op(prob, X) - prob.b) <= 1e-8 * (1 + np.linalg.norm(prob.b))
        assert np.linalg.norm(prob.C - oops.At_op(prob, y) - S) <= 1e-8 * (1 + np.linalg.norm(prob.C))
        s.close()

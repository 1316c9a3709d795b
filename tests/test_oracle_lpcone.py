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

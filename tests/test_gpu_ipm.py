"""GPU outer loop: the Jacobi eigensolver (sdp_eigh), one interior-point step (ipm_step) in
lockstep with the oracle's step, and whole solves (sdp_solve) against the oracle's optimum.

Lockstep (one step from the oracle's own iterate) is compared at the early iterates, where
the oracle's Schur-complement directions are accurate to ~cond(W)^2 eps; whole solves are
compared on the objective (relative 1e-8 with both at gap <= 1e-8) and on X (relative 1e-6:
X is determined to O(mu) near the end of the path).
"""
import numpy as np
import pytest

import workloads as W
from oracle import ipm as oipm, operators as oops

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,kind", [(1, "rand"), (2, "rand"), (7, "rand"), (64, "rand"), (201, "rand"),
                                    (60, "graded"), (40, "clustered")])
def test_eigh_matches_lapack(n, kind):
    from paper_2407_14013_gb300 import eigh
    rng = np.random.default_rng(n)
    if kind == "rand":
        M = rng.standard_normal((n, n))
        A = M + M.T
    else:
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        if kind == "graded":
            w = np.logspace(-10, 3, n)
        else:
            w = np.concatenate([np.full(n // 2, 1.0), np.full(n - n // 2, 1.0 + 1e-9)])
        A = (Q * w) @ Q.T
        A = 0.5 * (A + A.T)
    lam, V, sweeps = eigh(_t(A))
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    nrm = np.linalg.norm(A, 2)
    assert np.max(np.abs(np.sort(lam) - ref)) <= 1e-13 * nrm * max(1, n) ** 0.5
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-13 * n
    assert np.linalg.norm((V * lam) @ V.T - A) <= 1e-13 * nrm * n
    assert sweeps <= 20


LOCK = [
    ("maxcut20", lambda: W.maxcut(20, 0.3, 4101), 6),
    ("sensing12", lambda: W.sensing(12, 40, 2, 4102), 4),
]


@pytest.mark.parametrize("name,mk,rh", LOCK, ids=[c[0] for c in LOCK])
def test_ipm_step_lockstep_with_oracle(name, mk, rh):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    res = oipm.ipm_solve(prob, max_iter=6, keep_history=True)
    s = NewtonSolver(prob, r_hat=rh)
    for k in (1, 3):
        h0, h1 = res.history[k], res.history[k + 1]
        X, y, S = _t(h0["X"]), _t(h0["y"]), _t(h0["S"])
        info = s.ipm_step(_t(prob.b), _t(prob.C), X, y, S)
        assert rel(X.cpu().numpy(), h1["X"]) < 1e-8, (k, info)
        assert rel(y.cpu().numpy(), h1["y"]) < 1e-8
        assert rel(S.cpu().numpy(), h1["S"]) < 1e-8
        assert abs(info["mu"] - h0["mu"]) <= 1e-12 * h0["mu"]
    s.close()


SOLVE = [
    ("maxcut64", lambda: W.workload("maxcut64"), 12),
    ("sensing20", lambda: W.sensing(20, 120, 2, 77), 4),
    ("maxcut_bipartite", lambda: W.maxcut(7, 0.0, 5, edges=[(i, 3 + j) for i in range(3) for j in range(4)]), 4),
]


@pytest.mark.parametrize("name,mk,rh", SOLVE, ids=[c[0] for c in SOLVE])
def test_sdp_solve_matches_oracle(name, mk, rh):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    ref = oipm.ipm_solve(prob, tol=1e-8, max_iter=100)
    assert ref.converged
    s = NewtonSolver(prob, r_hat=rh)
    X, y, S, info = s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-8, max_iter=100)
    assert info["converged"] == 1, info
    X, y, S = X.cpu().numpy(), y.cpu().numpy(), S.cpu().numpy()
    pobj, pobj_ref = float(np.sum(prob.C * X)), float(np.sum(prob.C * ref.X))
    # each side is at rel_gap <= 1e-8 with infeasibilities <= 1e-8, so each objective is within
    # about 1e-8 (1 + 2|p*|) of the optimal value
    assert abs(pobj - pobj_ref) <= 2e-8 * (1 + 2 * abs(pobj_ref))
    assert rel(X, ref.X) < 1e-6
    # invariants at the GPU optimum
    assert np.linalg.norm(oops.A_op(prob, X) - prob.b) <= 1e-8 * (1 + np.linalg.norm(prob.b))
    assert np.linalg.norm(prob.C - oops.At_op(prob, y) - S) <= 1e-8 * (1 + np.linalg.norm(prob.C))
    assert np.linalg.eigvalsh(X)[0] > -1e-9 and np.linalg.eigvalsh(S)[0] > -1e-9
    if name == "maxcut_bipartite":
        m_edges = len(prob.meta["edges"])
        assert abs(pobj + m_edges) <= 1e-7 * m_edges        # value -|E| (connected bipartite, unit weights)
    s.close()


def test_scaling_point_and_adjoint_at_the_final_iterate():
    """sdp_scaling_point gives the eigen-decomposition of the NT scaling of an iterate (compared
    with the oracle's NT scaling); the whole GPU chain sdp_solve -> sdp_scaling_point -> sdp_grad
    satisfies the envelope theorem at the final (uncentred, gap 1e-8) iterate: with
    (gX, gy) = (C, 0), gb = y* and with (0, b), gC = X*, to the O(mu)-type error of the
    linearisation there (1e-5 on the oracle for this instance; bound 1e-4)."""
    from paper_2407_14013_gb300 import NewtonSolver
    from oracle import newton as onewton
    prob = W.maxcut(40, 0.15, 2719)
    ref = oipm.ipm_solve(prob, tol=1e-8, max_iter=200)
    # a centred iterate at mu = 1e-4: both NT-scaling routes are accurate there (near the end of
    # the path L^T S L is nearly singular and the two routes agree only to ~cond(W) eps)
    st = oipm.center(prob, oipm.IPMState(ref.X, ref.y, ref.S), 1e-4)
    s = NewtonSolver(prob, r_hat=8)
    V, lam = s.scaling_point(_t(st.X), _t(st.S))
    Vh, lh = V.cpu().numpy(), lam.cpu().numpy()
    assert np.max(np.abs(Vh.T @ Vh - np.eye(prob.n))) < 1e-12
    assert rel((Vh * lh) @ Vh.T, onewton.nt_scaling(st.X, st.S)) < 1e-9
    X, y, S, info = s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-8, max_iter=100)
    assert info["converged"] == 1
    V, lam = s.scaling_point(X, S)
    gC, gb = s.grad(V, lam, _t(prob.C), _t(np.zeros(prob.m)))
    assert rel(gb.cpu().numpy(), y.cpu().numpy()) < 1e-4
    gC, gb = s.grad(V, lam, _t(np.zeros((prob.n, prob.n))), _t(prob.b))
    assert rel(gC.cpu().numpy(), X.cpu().numpy()) < 1e-4
    s.close()


def test_solve_stops_cleanly_on_unconverged_direction():
    """A Newton solve that reaches max_pcg far above the stop test ends the outer loop with
    SDP_ENOTCONV before any step is taken on its direction: the outputs hold the last iterate
    (here the start X = S = xi I, y = 0) and the message names the cause.  With a cap that
    lets the first directions converge, the loop stops later at a positive-definite iterate."""
    import torch
    from paper_2407_14013_gb300 import NewtonSolver, native
    prob = W.sensing(16, 60, 2, 4111)
    s = NewtonSolver(prob, r_hat=4, max_pcg=1, check_every=1)
    X, y, S, info = s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-8, max_iter=30, allow_notconv=True)
    assert info["status"] == native.SDP_ENOTCONV and info["iters"] == 0
    Xh, Sh = X.cpu().numpy(), S.cpu().numpy()
    xi = Xh[0, 0]
    assert xi >= 10 and np.array_equal(Xh, xi * np.eye(16)) and np.array_equal(Sh, xi * np.eye(16))
    assert not y.cpu().numpy().any()
    assert "not converged" in native.sdp_last_error(s.handle)
    s.close()
    # a tighter cap than the solve needs somewhere along the path: whichever direction misses it,
    # the iterate returned is the last one stepped to (finite, X and S positive definite)
    s = NewtonSolver(prob, r_hat=4, max_pcg=30, check_every=1)
    X, y, S, info = s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-8, max_iter=60, allow_notconv=True)
    print(f"\ncap 30: status={info['status']} iters={info['iters']} gap={info['rel_gap']:.2e}")
    if info["status"] == native.SDP_ENOTCONV and not info["converged"]:
        assert np.isfinite(X.cpu().numpy()).all()
        assert np.linalg.eigvalsh(X.cpu().numpy()).min() > 0 and np.linalg.eigvalsh(S.cpu().numpy()).min() > 0
    else:
        assert info["status"] == 0
    s.close()

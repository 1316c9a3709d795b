"""GPU parity of the implicit derivative sdp_grad (C ABI) against the oracle's VJP.

The oracle product (oracle/grad.py) is pinned by central differences of the central path and
by the envelope theorem (tests/test_oracle_grad.py).  Here the CUDA product, computed through
the reformulated Newton operator and its preconditioner, is compared with it on the same
scaling points at moderate mu (1e-2), where the oracle's Schur route is accurate to ~cond(W)^2 eps;
near the optimum it is checked against the envelope theorem directly.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad as ograd, ipm, newton as onewton

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _centered(prob, mu, tol=1e-8):
    res = ipm.ipm_solve(prob, tol=tol, max_iter=200)
    assert res.converged
    return ipm.center(prob, ipm.IPMState(res.X, res.y, res.S), mu)


def _eig(Wm):
    lam, V = np.linalg.eigh(Wm)
    return V, lam


CASES = [
    ("maxcut10w", lambda: W.maxcut(10, 0.6, 2718, weights="gauss"), 4),
    ("maxcut40", lambda: W.maxcut(40, 0.15, 2719), 8),
    ("sensing12", lambda: W.sensing(12, 30, 2, 2720), 4),
]


@pytest.mark.parametrize("name,mk,rh", CASES, ids=[c[0] for c in CASES])
def test_grad_matches_oracle_vjp(name, mk, rh):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    st = _centered(prob, 1e-2)   # cond(W) ~ 5e3: the oracle Schur route is good to ~1e-9
    Wm = onewton.nt_scaling(st.X, st.S)
    V, lam = _eig(Wm)
    rng = np.random.default_rng(11)
    G = rng.standard_normal((prob.n, prob.n))
    gX, gy = G, rng.standard_normal(prob.m)                 # non-symmetric gX: only sym(gX) counts
    oC, ob = ograd.vjp_at_scaling(prob, Wm, gX, gy)
    s = NewtonSolver(prob, r_hat=rh)
    gC, gb = s.grad(_t(V), _t(lam), _t(gX), _t(gy))
    assert s.last_info.converged
    assert rel(gC.cpu().numpy(), oC) < TOL and rel(gb.cpu().numpy(), ob) < TOL
    s.close()


def test_grad_envelope_near_optimum():
    """At the centred point mu = 1e-8: (gX, gy) = (C, 0) gives gb = y*, gC = 0 and
    (gX, gy) = (0, b) gives gC = X*, gb = 0 (dp*/db = y*, dp*/dC = X*), up to O(mu) terms of
    the central-path derivative (about 2e-6 relative here; the same bound as the oracle's pin)."""
    from paper_2407_14013_gb300 import NewtonSolver
    prob = W.maxcut(40, 0.15, 2719)
    st = _centered(prob, 1e-8)
    V, lam = _eig(onewton.nt_scaling(st.X, st.S))
    s = NewtonSolver(prob, r_hat=8)
    gC, gb = s.grad(_t(V), _t(lam), _t(prob.C), _t(np.zeros(prob.m)))
    assert rel(gb.cpu().numpy(), st.y) < 1e-5
    assert np.linalg.norm(gC.cpu().numpy()) < 1e-5 * np.linalg.norm(st.X)
    gC, gb = s.grad(_t(V), _t(lam), _t(np.zeros((prob.n, prob.n))), _t(prob.b))
    assert rel(gC.cpu().numpy(), st.X) < 1e-5
    assert np.linalg.norm(gb.cpu().numpy()) < 1e-5 * np.linalg.norm(st.y)
    s.close()


def test_sdp_optimum_autograd_matches_grad():
    import torch
    from paper_2407_14013_gb300 import NewtonSolver, sdp_optimum
    prob = W.maxcut(10, 0.6, 2718, weights="gauss")
    st = _centered(prob, 1e-4)
    V, lam = _eig(onewton.nt_scaling(st.X, st.S))
    s = NewtonSolver(prob, r_hat=4)
    C = _t(prob.C).requires_grad_(True)
    b = _t(prob.b).requires_grad_(True)
    X, y = sdp_optimum(C, b, _t(st.X), _t(st.y), _t(V), _t(lam), s)
    rng = np.random.default_rng(3)
    GX, gy = _t(rng.standard_normal((prob.n, prob.n))), _t(rng.standard_normal(prob.m))
    loss = (GX * X).sum() + (gy * y).sum()
    loss.backward()
    gC, gb = s.grad(_t(V), _t(lam), GX, gy)
    assert torch.allclose(C.grad, gC, rtol=0, atol=1e-12 * float(gC.abs().max()))
    assert torch.allclose(b.grad, gb, rtol=0, atol=1e-12 * float(gb.abs().max()))
    s.close()

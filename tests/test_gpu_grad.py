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


def test_sdp_optimum_at_autograd_matches_grad():
    import torch
    from paper_2407_14013_gb300 import NewtonSolver, sdp_optimum_at
    prob = W.maxcut(10, 0.6, 2718, weights="gauss")
    st = _centered(prob, 1e-4)
    V, lam = _eig(onewton.nt_scaling(st.X, st.S))
    s = NewtonSolver(prob, r_hat=4)
    C = _t(prob.C).requires_grad_(True)
    b = _t(prob.b).requires_grad_(True)
    X, y = sdp_optimum_at(C, b, _t(st.X), _t(st.y), _t(V), _t(lam), s)
    rng = np.random.default_rng(3)
    GX, gy = _t(rng.standard_normal((prob.n, prob.n))), _t(rng.standard_normal(prob.m))
    loss = (GX * X).sum() + (gy * y).sum()
    loss.backward()
    gC, gb = s.grad(_t(V), _t(lam), GX, gy)
    assert torch.allclose(C.grad, gC, rtol=0, atol=1e-12 * float(gC.abs().max()))
    assert torch.allclose(b.grad, gb, rtol=0, atol=1e-12 * float(gb.abs().max()))
    s.close()


def test_center_matches_oracle_central_point():
    """sdp_center from the GPU solve's final iterate reaches the central-path point of the
    given mu, which is unique: it matches the oracle's own centring (oracle/ipm.py center) of
    the oracle's final iterate, entry by entry."""
    import torch
    from paper_2407_14013_gb300 import NewtonSolver
    prob = W.maxcut(10, 0.6, 2718, weights="gauss")
    mu = 1e-4
    ref = _centered(prob, mu)
    s = NewtonSolver(prob, r_hat=4)
    X, y, S, info = s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-8)
    ci = s.center(_t(prob.b), _t(prob.C), X, y, S, mu, tol=1e-10, max_iter=60, allow_notconv=True)
    print(f"\ncenter: status={ci['status']} iters={ci['iters']} centrality={ci['sigma']:.2e} "
          f"pinf={ci['pinf']:.2e} dinf={ci['dinf']:.2e}")
    assert ci["status"] == 0 and ci["sigma"] <= 1e-10
    for got, want in ((X, ref.X), (y, ref.y), (S, ref.S)):
        g = got.cpu().numpy()
        assert np.abs(g - want).max() <= 1e-8 * np.abs(want).max()
    s.close()


def _fd_layer(prob, s, bvec, Cmat, GX, gy, mu_c):
    """Loss <GX, X> + <gy, y> of the GPU layer's forward (solve, centre at mu_c)."""
    import torch
    from paper_2407_14013_gb300 import sdp_optimum
    with torch.no_grad():
        X, y = sdp_optimum(_t(Cmat), _t(bvec), s, gap_tol=1e-9, center_mu=mu_c, center_tol=1e-11)
    return float((X.cpu().numpy() * GX).sum() + (y.cpu().numpy() * gy).sum())


def test_sdp_layer_gradient_matches_central_differences():
    """The differentiable layer (forward: sdp_solve + sdp_center + scaling point on the GPU;
    backward: sdp_grad) against central differences of its own forward pass in b and in C, on
    a nondegenerate weighted MaxCut instance (unique primal and dual optimum), to 1e-5; the
    forward's X also matches the oracle's centred point."""
    import torch
    from paper_2407_14013_gb300 import NewtonSolver, sdp_optimum
    prob = W.maxcut(10, 0.6, 2718, weights="gauss")
    mu_c = 1e-6
    s = NewtonSolver(prob, r_hat=4)
    rng = np.random.default_rng(5)
    GX = rng.standard_normal((prob.n, prob.n))
    GX = 0.5 * (GX + GX.T)
    gy = rng.standard_normal(prob.m)
    C = _t(prob.C).requires_grad_(True)
    b = _t(prob.b).requires_grad_(True)
    X, y = sdp_optimum(C, b, s, gap_tol=1e-9, center_mu=mu_c, center_tol=1e-11)
    ref = _centered(prob, mu_c)
    assert np.abs(X.detach().cpu().numpy() - ref.X).max() <= 1e-7 * np.abs(ref.X).max()
    loss = (_t(GX) * X).sum() + (_t(gy) * y).sum()
    loss.backward()
    db = rng.standard_normal(prob.m)
    dC = rng.standard_normal((prob.n, prob.n))
    dC = 0.5 * (dC + dC.T)
    # central differences with one Richardson step: (4 D(h/2) - D(h)) / 3 removes the h^2 term
    # (about 4e-4 relative at h = 1e-4 in the C direction on this instance, as the oracle's own
    # central point shows)
    def fd(f, h):
        d = lambda t: (f(t) - f(-t)) / (2 * t)
        return (4 * d(h / 2) - d(h)) / 3
    h = 1e-4
    fd_b = fd(lambda t: _fd_layer(prob, s, prob.b + t * db, prob.C, GX, gy, mu_c), h)
    an_b = float((b.grad.cpu().numpy() * db).sum())
    print(f"\nlayer FD: b {fd_b:.10f} vs {an_b:.10f}")
    assert abs(fd_b - an_b) <= 1e-5 * max(abs(an_b), 1e-3 * np.linalg.norm(b.grad.cpu().numpy()))
    fd_C = fd(lambda t: _fd_layer(prob, s, prob.b, prob.C + t * dC, GX, gy, mu_c), h)
    an_C = float((C.grad.cpu().numpy() * dC).sum())
    print(f"layer FD: C {fd_C:.10f} vs {an_C:.10f}")
    assert abs(fd_C - an_C) <= 1e-5 * max(abs(an_C), 1e-3 * np.linalg.norm(C.grad.cpu().numpy()))
    s.close()

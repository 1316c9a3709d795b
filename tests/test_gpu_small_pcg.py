"""GPU parity of the one-cluster PCG solve of small DIAG problems (n <= 128, r <= 16, m-space).

With use_graph (the default) a DIAG problem of that size runs its whole FP64 PCG solve, from
x0 through the stop test, as one launch of one thread-block cluster; use_graph = 0 keeps the
launch chain (a dozen kernels per iteration).  Both are checked against the oracle's plain
definition of the Newton direction (relative 1e-8, the FP64 bar of the other parity tests)
and against each other (relative 1e-10: the same iteration in another summation order).
The shapes cover fewer rows than CTAs (n = 5), a ragged last CTA (n = 100), the largest n and r
(n = 128 with r = 16 fits in shared memory with 16 CTAs of 8 rows), 8- and 16-CTA clusters
(n <= 32 and n > 32), both starts of Cor. pcg, the iteration limit, and the shapes that fall
back to the launch chain.
"""
import numpy as np
import pytest

import workloads as W
from oracle import newton as onewton

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def solve(prob, sp, Ct, bt, **kw):
    from paper_2407_14013_gb300 import NewtonSolver
    s = NewtonSolver(prob, **kw)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt), allow_notconv=True)
    out = (dX.cpu().numpy(), dy.cpu().numpy(), dS.cpu().numpy(), info, info.launches)
    s.close()
    return out


CASES = [
    # name, problem, r_true, mu, r_hat
    ("maxcut5", lambda: W.maxcut(5, 0.9, 1301), 1, 1e-2, 2),
    ("maxcut17", lambda: W.maxcut(17, 0.3, 1302), 2, 1e-3, 4),
    ("maxcut64", lambda: W.workload("maxcut64"), 3, 1e-3, 12),
    ("maxcut100_ragged", lambda: W.maxcut(100, 0.08, 1303, weights="gauss"), 5, 1e-3, 8),
    ("maxcut120_r16", lambda: W.maxcut(120, 0.06, 1304, weights="gauss"), 16, 1e-3, 16),
    ("maxcut128_r12", lambda: W.maxcut(128, 0.06, 1311, weights="gauss"), 12, 1e-3, 12),
    ("maxcut128_r16", lambda: W.maxcut(128, 0.06, 1312, weights="gauss"), 16, 1e-3, 16),
]


@pytest.mark.parametrize("start", [0, 1])
@pytest.mark.parametrize("name,mk,rt,mu,rh", CASES, ids=[c[0] for c in CASES])
def test_cluster_solve_matches_oracle_and_launch_chain(name, mk, rt, mu, rh, start):
    prob = mk()
    sp = W.scaling_point(prob.n, rt, mu, 1400 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 1500 + prob.n)
    X1, y1, S1, i1, l1 = solve(prob, sp, Ct, bt, r_hat=rh, precond_space=2, pcg_start=start)
    X2, y2, S2, i2, l2 = solve(prob, sp, Ct, bt, r_hat=rh, precond_space=2, pcg_start=start, use_graph=False)
    assert i1.converged and i2.converged and i1.status == 0 and i1.space == 2
    assert i1.r == i2.r and i1.d == i2.d
    assert abs(i1.pcg_iters - i2.pcg_iters) <= 1
    rX, ry, rS = onewton.newton_direct(prob, (sp.V * sp.lam) @ sp.V.T, Ct, bt)
    assert rel(X1, rX) < TOL and rel(y1, ry) < TOL and rel(S1, rS) < TOL
    assert rel(X1, X2) < 1e-10 and rel(y1, y2) < 1e-10 and rel(S1, S2) < 1e-10
    # the loop is one launch: the chain spends about a dozen per iteration
    assert l1 + 10 * max(i2.pcg_iters - 1, 0) < l2


def test_cluster_solve_stops_at_the_iteration_limit():
    """max_pcg iterations without the stop test: SDP_ENOTCONV with the iterate after exactly
    max_pcg iterations, the same as the launch chain's."""
    from paper_2407_14013_gb300 import native
    prob = W.maxcut(96, 0.07, 1305, weights="gauss")
    sp = W.scaling_point(96, 4, 1e-6, 1306)
    Ct, bt = W.newton_rhs(96, 96, 1307)
    X1, y1, S1, i1, _ = solve(prob, sp, Ct, bt, r_hat=6, precond_space=2, max_pcg=2)
    X2, y2, S2, i2, _ = solve(prob, sp, Ct, bt, r_hat=6, precond_space=2, max_pcg=2, use_graph=False)
    assert i1.status == native.SDP_ENOTCONV and i2.status == native.SDP_ENOTCONV
    assert i1.pcg_iters == i2.pcg_iters == 2
    assert rel(X1, X2) < 1e-10 and rel(y1, y2) < 1e-10


@pytest.mark.parametrize("n,rt", [(129, 3), (130, 16)])
def test_shapes_outside_the_cluster_range_take_the_launch_chain(n, rt):
    """n above 128 (the cluster solve's range) gives the oracle's direction through the launch
    chain."""
    prob = W.maxcut(n, 0.05, 1308)
    sp = W.scaling_point(n, rt, 1e-3, 1309)
    Ct, bt = W.newton_rhs(n, n, 1310)
    X1, y1, S1, i1, l1 = solve(prob, sp, Ct, bt, r_hat=rt, precond_space=2)
    assert i1.converged
    rX, ry, rS = onewton.newton_direct(prob, (sp.V * sp.lam) @ sp.V.T, Ct, bt)
    assert rel(X1, rX) < TOL and rel(y1, ry) < TOL
    assert l1 > 10 * i1.pcg_iters                      # a dozen launches per iteration


def test_cluster_solve_zero_and_non_finite_right_sides():
    """Through the cluster solve: a zero right side gives the zero direction at once (||r_0|| = 0
    meets the threshold 0), a NaN in C~ is reported as SDP_ENUMERIC by the right side's finish
    inside the kernel, and the handle then solves a good right side as before."""
    import torch
    from paper_2407_14013_gb300 import NewtonSolver, SdpError, native
    prob = W.maxcut(40, 0.2, 1313)
    sp = W.scaling_point(40, 3, 1e-3, 1314)
    Ct, bt = W.newton_rhs(40, 40, 1315)
    s = NewtonSolver(prob, r_hat=4, precond_space=2)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dX, dy, dS, info = s.solve(t(sp.V), t(sp.lam), t(np.zeros_like(Ct)), t(np.zeros_like(bt)))
    assert info.converged and info.status == 0 and info.pcg_iters == 0
    assert not np.any(dX.cpu().numpy()) and not np.any(dy.cpu().numpy()) and not np.any(dS.cpu().numpy())
    Cn = Ct.copy()
    Cn[3, 5] = Cn[5, 3] = np.nan
    with pytest.raises(SdpError) as e:
        s.solve(t(sp.V), t(sp.lam), t(Cn), t(bt))
    assert e.value.status == native.SDP_ENUMERIC
    dX, dy, dS, info = s.solve(t(sp.V), t(sp.lam), t(Ct), t(bt))
    assert info.converged
    rX, ry, rS = onewton.newton_direct(prob, (sp.V * sp.lam) @ sp.V.T, Ct, bt)
    assert rel(dX.cpu().numpy(), rX) < TOL and rel(dy.cpu().numpy(), ry) < TOL
    s.close()

"""GPU parity of the linear block of the Newton system (the nonnegative variables of Section 7's
robust problems, eq. rmc-sdp): with sdp_set_linear_diag the Newton direction equals the oracle's
plain definition (Schur system with G D G^T, oracle/lpcone.py) to the FP64 tolerance, in both
preconditioner spaces, for dense constraints and for robust matrix completion (SPARSE_COO);
combinations that are not built are refused."""
import numpy as np
import pytest

import workloads as W
from oracle import lpcone, operators as oops

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = [
    # name, problem, r_true, mu, r_hat, preconditioner space (1 = d, 2 = m)
    ("sensing12_d", lambda: W.sensing(12, 40, 2, 1201), 2, 1e-3, 4, 1),
    ("sensing12_m", lambda: W.sensing(12, 40, 2, 1201), 2, 1e-3, 4, 2),
    ("sensing37_d", lambda: W.sensing(37, 150, 3, 1202), 3, 1e-2, 5, 1),
    # robust matrix completion (Section 7, eq. rmc-sdp): single svec entries, SPARSE_COO kind
    ("rmc20_d", lambda: W.rmc(20, 90, 5, 1203), 2, 1e-3, 3, 1),
    ("rmc20_m", lambda: W.rmc(20, 60, 4, 1204), 2, 1e-3, 3, 2),
]


@pytest.mark.parametrize("name,mk,rt,mu,rh,space", CASES, ids=[c[0] for c in CASES])
def test_linear_block_direction_matches_definition(name, mk, rt, mu, rh, space):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    m = prob.m
    sp = W.scaling_point(prob.n, rt, mu, 1300 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, m, 1301 + prob.n)
    g = np.random.default_rng(1302 + prob.n)
    G = np.hstack([np.eye(m), -np.eye(m)])                # eq. rmc-sdp: x = [v; w]
    d = 10.0 ** g.uniform(-3, 3, 2 * m)
    ct = g.standard_normal(2 * m)
    Wm = (sp.V * sp.lam) @ sp.V.T
    rX, rx, ry = lpcone.newton_direct_lp(prob, Wm, Ct, bt, G, d, ct)
    s = NewtonSolver(prob, r_hat=rh, precond_space=space)
    s.set_linear_diag(d[:m] + d[m:])                      # delta = diag(G D G^T)
    btl = bt + G @ (d * ct)                               # the caller folds G D c~ into b~
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(btl))
    assert info.converged and info.space == space
    dX, dy = dX.cpu().numpy(), dy.cpu().numpy()
    dx = d * (G.T @ dy - ct)
    assert rel(dX, rX) < TOL and rel(dy, ry) < TOL and rel(dx, rx) < TOL
    # the outer loop and the adjoint have no nonnegative variables: refused while the block is set
    from paper_2407_14013_gb300 import SdpError, native
    with pytest.raises(SdpError) as e:
        s.solve_sdp(_t(prob.b), _t(prob.C), gap_tol=1e-2, max_iter=1)
    assert e.value.status == native.SDP_EUNSUPPORTED
    # removing the block gives back the semidefinite direction
    s.set_linear_diag(None)
    dX0, dy0, _, i0 = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    from oracle import newton as onewton
    sX, sy, _ = onewton.newton_direct(prob, Wm, Ct, bt)
    assert i0.converged and rel(dX0.cpu().numpy(), sX) < TOL and rel(dy0.cpu().numpy(), sy) < TOL
    s.close()


def test_linear_block_refused_where_not_built():
    from paper_2407_14013_gb300 import NewtonSolver, SdpError, native
    import torch
    delta = torch.ones(20, dtype=torch.float64, device="cuda")
    for kw, prob in ((dict(precision="mixed_fp32"), W.sensing(8, 20, 2, 1400)),
                     (dict(krylov="minres"), W.sensing(8, 20, 2, 1401)),
                     ({}, W.maxcut(20, 0.3, 1402))):
        s = NewtonSolver(prob, r_hat=3, **kw)
        with pytest.raises(SdpError) as e:
            s.set_linear_diag(delta[:prob.m])
        assert e.value.status == native.SDP_EUNSUPPORTED
        ones = _t(np.ones(prob.m))
        with pytest.raises(SdpError) as e:              # refused before any output is written
            s.solve_slack(_t(prob.b), _t(prob.C), ones, ones)
        assert e.value.status == native.SDP_EUNSUPPORTED
        s.close()


def test_slack_solve_recovers_rmc_and_matches_the_oracle():
    """sdp_solve_slack on robust completion (n = 12, 70 measurements, 3 gross outliers): converges
    to a 1e-8 gap, recovers X*, puts v - w exactly on the outliers with |y| <= 1, and agrees with
    the oracle's outer loop (oracle/ipm_lp.py); a second call on the same handle gives the same
    point (the handle is left without the linear block)."""
    from oracle import ipm_lp
    from paper_2407_14013_gb300 import NewtonSolver
    prob = W.rmc(12, 70, 3, 9)
    m = prob.m
    ones = np.ones(m)
    s = NewtonSolver(prob, r_hat=3)
    X, y, S, v, w, zv, zw, info = s.solve_slack(_t(prob.b), _t(prob.C), _t(ones), _t(ones))
    assert info["status"] == 0 and info["converged"] == 1 and info["rel_gap"] <= 1e-8
    Xh = X.cpu().numpy()
    Xs, eps, out = prob.meta["Xs"], prob.meta["eps"], prob.meta["outliers"]
    assert rel(Xh, Xs) <= 1e-6
    vw = (v - w).cpu().numpy()
    assert set(np.where(np.abs(vw) > 1e-3)[0].tolist()) == set(out.tolist())
    assert np.allclose(vw[out], eps[out], rtol=1e-6, atol=1e-6)
    assert np.abs(y.cpu().numpy()).max() <= 1 + 1e-8
    assert min(float(v.min()), float(w.min()), float(zv.min()), float(zw.min())) > 0
    res = ipm_lp.ipm_solve_lp(prob, prob.meta["G_l"], prob.meta["c_l"])
    assert rel(Xh, res.X) <= 1e-6
    X2, *_, info2 = s.solve_slack(_t(prob.b), _t(prob.C), _t(ones), _t(ones))
    assert info2["converged"] == 1 and rel(X2.cpu().numpy(), Xh) <= 1e-9
    s.close()


def test_slack_solve_dense_constraints_matches_the_oracle():
    """The same loop on dense constraints (matrix sensing with two gross outliers in b): converges
    and agrees with the oracle's outer loop on X and on the slacks."""
    from oracle import ipm_lp
    from paper_2407_14013_gb300 import NewtonSolver
    prob = W.sensing(10, 40, 2, 1501)
    g = np.random.default_rng(1502)
    b = prob.b.copy()
    b[g.choice(prob.m, 2, replace=False)] += 50.0 * g.standard_normal(2)
    prob.b = b
    m = prob.m
    G = np.hstack([np.eye(m), -np.eye(m)])
    cl = np.ones(2 * m)
    res = ipm_lp.ipm_solve_lp(prob, G, cl)
    assert res.converged
    s = NewtonSolver(prob, r_hat=3)
    X, y, S, v, w, zv, zw, info = s.solve_slack(_t(prob.b), _t(prob.C), _t(cl[:m]), _t(cl[m:]))
    assert info["converged"] == 1
    assert rel(X.cpu().numpy(), res.X) <= 1e-6
    assert np.allclose((v - w).cpu().numpy(), res.x[:m] - res.x[m:], rtol=0, atol=1e-6 * (1 + np.abs(b).max()))
    s.close()


def _lp_case_dense():
    p0 = W.sensing(6, 8, 2, 77)
    b = p0.b.copy()
    b[0] += 5.0
    b[3] -= 4.0
    return W.Problem(kind=p0.kind, n=p0.n, m=p0.m, b=b, C=p0.C, a_dense=p0.a_dense)


# (case, outer-loop tolerance of the oracle's solve, centring mu or None, bound).  On robust
# completion d = x / z spans 4e-4 .. 7e7 (mu ~ 2e-3) and 2.7e-9 .. 4e13 (final, mu ~ 1e-8): the KKT
# matrix's condition is then 1e11 and more, the dense LU solve of the same system is off by 3e-5
# and O(1) there, and two FP64 solves of it agree to a few 1e-8 (measured 4e-8 GPU vs oracle), so
# those cases carry a bound of 1e-6; the dense case (d in 1e-4 .. 1e5) keeps the FP64 bar.
SLACK_CASES = [("sensing6_outliers", 1e-9, 1e-4, 1e-8), ("rmc12_mid", 1e-4, None, 1e-6),
               ("rmc12_final", 1e-9, None, 1e-6)]


@pytest.mark.parametrize("name,otol,mu_c,bound", SLACK_CASES, ids=[c[0] for c in SLACK_CASES])
def test_grad_slack_matches_kkt_definition(name, otol, mu_c, bound):
    """The adjoint with the slacks of eq. rmc-sdp on the GPU (sdp_grad_slack: one reformulated
    Newton solve with the linear block, then dx = D(G^T dy - c~)) against the oracle's solve of the
    same symmetric KKT system of the two cones, [[-(W (x)s W)^{-1}, 0, A^T], [0, -D^{-1}, G^T],
    [A, G, 0]] [gC; gc; gb] = [sym gX; gx; gy] (oracle/lpcone.py newton_reform_lp, the product
    vjp_lp takes, here to a residual of 1e-15), at a centred iterate (mu = 1e-4) of the dense case,
    where the plain dense KKT solve (LU) agrees with it to 1e-9, and at two iterates of the oracle's
    solve for robust completion (mu ~ 2e-3, and the final mu ~ 1e-8, where the dense KKT matrix is
    too ill-conditioned for LU and the reformulation is what stays accurate).  Entry by entry: gC and gb, and the slack
    cotangent through D^{-1} gc = G^T gb - gx (gc itself multiplies that difference by d = x / z, up
    to 1e12 on the outliers, which no FP64 evaluation resolves better than d eps max|gb|).  (At its
    default tolerance the oracle's PCG stops one iteration early on the dense case at mu = 1e-6 and
    sits 7e-7 from the KKT solution; the GPU's stop test takes the second iteration.)"""
    from oracle import ipm_lp, lpcone, newton as onewton
    from paper_2407_14013_gb300 import NewtonSolver
    dense = name.startswith("sensing6")
    prob = _lp_case_dense() if dense else W.rmc(12, 70, 3, 9)
    m = prob.m
    G = np.hstack([np.eye(m), -np.eye(m)])
    cl = 0.5 * np.ones(2 * m) if dense else np.ones(2 * m)
    res = ipm_lp.ipm_solve_lp(prob, G, cl, tol=otol, max_iter=200)
    assert res.converged
    st = ipm_lp.LPState(res.X, res.x, res.y, res.S, res.z)
    if mu_c is not None:
        st = ipm_lp.center_lp(prob, G, cl, st, mu_c)
    rng = np.random.default_rng(12)
    gX = rng.standard_normal((prob.n, prob.n))
    gX = 0.5 * (gX + gX.T)
    gx, gy = rng.standard_normal(2 * m), rng.standard_normal(m)
    Wm = onewton.nt_scaling(st.X, st.S)
    d = st.x / st.z
    lam, V = np.linalg.eigh(Wm)
    # the oracle's reformulated solve taken to a tighter tolerance than its default
    kC, kc, kb, _ = lpcone.newton_reform_lp(prob, V, lam, gX, gy, G, d, gx, r_hat=3,
                                            s_A=oops.row_norm_scale(prob), rtol=1e-15, space="d")
    if dense:   # and the plain dense KKT solve agrees with it here (mu = 1e-4)
        dC, dc, db = lpcone.newton_kkt_dense_lp(prob, Wm, gX, gy, G, d, gx)[:3]
        assert np.abs(dC - kC).max() <= 1e-9 * np.abs(kC).max() and np.abs(db - kb).max() <= 1e-9 * np.abs(kb).max()
    s = NewtonSolver(prob, r_hat=3)
    gC, gb, gcv, gcw = s.grad_slack(_t(V), _t(lam), _t(d[:m]), _t(d[m:]), _t(gX), _t(gy), _t(gx[:m]), _t(gx[m:]))
    assert s.last_info.converged
    gc = np.concatenate([gcv.cpu().numpy(), gcw.cpu().numpy()])
    emax = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    errs = {"gC": emax(gC.cpu().numpy(), kC), "gb": emax(gb.cpu().numpy(), kb), "gc/d": emax(gc / d, kc / d)}
    print(f"\n{name} pcg_iters={s.last_info.pcg_iters} d in [{d.min():.1e}, {d.max():.1e}] " +
          " ".join(f"{k}={e:.2e}" for k, e in errs.items()))
    for k, e in errs.items():
        assert e <= bound, (k, e)
    # the handle is left without a linear block: a plain adjoint call works afterwards
    gC2, gb2 = s.grad(_t(V), _t(lam), _t(gX), _t(gy))
    assert s.last_info.converged
    s.close()


@pytest.mark.parametrize("dominated,expect", [(30, 2), (0, 1)], ids=["most_rows_fixed", "no_row_fixed"])
def test_space_rule_with_linear_block(dominated, expect):
    """precond_space = 3: with the linear block the GPU picks the space by the oracle's rule
    (lpcone.choose_space_lp: the m-space when fewer than d rows have tau^-2 delta_i <= 1e8 beta),
    here the m-space when 30 of the 40 rows are fixed by a slack (d = 23 > 10 free rows), the
    d-space when none is, and the direction still equals the oracle's.  Where slacks fix rows
    (delta_i = 1e14) the plain Schur route of the definition has a matrix of condition ~1e14 and
    misses the direction by ~3e-4; the reference is then the oracle's reformulated solve at
    rtol 1e-15, whose two spaces agree to 3e-14 (the Schur route is kept for the case without
    fixed rows, where all three agree)."""
    from paper_2407_14013_gb300 import NewtonSolver
    from oracle.reform import split
    prob = W.sensing(12, 40, 2, 1201)
    m = prob.m
    sp = W.scaling_point(prob.n, 2, 1e-3, 1312)
    Ct, bt = W.newton_rhs(prob.n, m, 1313)
    g = np.random.default_rng(1314)
    G = np.hstack([np.eye(m), -np.eye(m)])
    d = 10.0 ** g.uniform(-3, 3, 2 * m)
    d[:dominated] = 1e14                                  # slacks that fix their rows
    ct = g.standard_normal(2 * m)
    osp = split(sp.V, sp.lam, r_hat=4, s_A=oops.row_norm_scale(prob))
    assert lpcone.choose_space_lp(osp, G, d, m) == ("m" if expect == 2 else "d")
    if dominated:
        rX, rx, ry, _ = lpcone.newton_reform_lp(prob, sp.V, sp.lam, Ct, bt, G, d, ct, r_hat=4,
                                                s_A=oops.row_norm_scale(prob), rtol=1e-15, space="auto")
    else:
        Wm = (sp.V * sp.lam) @ sp.V.T
        rX, rx, ry = lpcone.newton_direct_lp(prob, Wm, Ct, bt, G, d, ct)
    s = NewtonSolver(prob, r_hat=4, precond_space=3)
    s.set_linear_diag(d[:m] + d[m:])
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt + G @ (d * ct)))
    assert info.converged and info.space == expect
    dX, dy = dX.cpu().numpy(), dy.cpu().numpy()
    dx = d * (G.T @ dy - ct)
    # dx = D (G^T dy - c~) multiplies the rounding of dy by D (up to 1e14 here): compare D^{-1} dx
    print(f"\nspace {info.space}: dX {rel(dX, rX):.2e} dy {rel(dy, ry):.2e} D^-1 dx {rel(dx / d, rx / d):.2e}")
    assert rel(dX, rX) < TOL and rel(dy, ry) < TOL and rel(dx / d, rx / d) < TOL
    # without the block, precond_space 3 is the plain auto rule (d = 23 <= m = 40: d-space)
    s.set_linear_diag(None)
    _, _, _, i0 = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert i0.converged and i0.space == 1
    s.close()

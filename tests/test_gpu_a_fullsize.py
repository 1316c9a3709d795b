"""Entry-wise GPU parity of the Newton direction at the workloads' full sizes.

The Newton direction is the unit of parity (Section 3, (Newt-eps) and eq. recover): the CUDA
path (reformulated augmented system, indefinite PCG, recovery) is compared with the oracle's
plain definition (oracle/newton.py newton_direct: Schur elimination M dy = b~ + A(W C~ W),
M_ij = <A_i, W A_j W>, Cholesky, dX = W(A^T dy - C~)W), element by element:

    max |a - b| <= 1e-8 max |b|

for dy, dS and dX, and separately for each block of dX in the eigenbasis of W, V^T dX V =
[[top r x r, .], [cross, orthogonal]], each against its own largest entry, so that an error in
a small block cannot hide under a large one.  The scaling points have the two-cluster spectrum
of (A0) at mu = 1e-3, where cond(W)^2 eps keeps the oracle's Schur route accurate to about
1e-10.  The measured errors are printed (pytest -s).

Sizes: matrix sensing n = 200, m = 2000, r = 3 (the bench workload); MaxCut n = 5000, r = 100
(DIAG, m-space core); matrix completion 500 + 500 with 5% of the entries (m = 12500, r = 5,
d-space core); the completion workload at its full size 1000 + 1000 (m = 50000), where the
oracle's Schur matrix (20 GB) is out of reach, through the (Newt-eps) residual of the GPU
direction instead.  Two dynamic-range cases exercise the integer-digit passes over A: entries
spread over 1e-8 .. 1 within each row of A, and a solution dy whose entries span 1e-8 .. 1.
"""
import numpy as np
import pytest

import workloads as W
from oracle import newton as onewton, operators as oops

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def emax(a, b):
    """max |a - b| / max |b|"""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def block_errors(dX, rX, V, lam, r):
    """Entry-wise errors of the blocks of V^T dX V (eigenvalues descending: the top r first)."""
    o = np.argsort(-lam)
    Vs = V[:, o]
    A = Vs.T @ dX @ Vs
    B = Vs.T @ rX @ Vs
    return {"top": emax(A[:r, :r], B[:r, :r]), "cross": emax(A[r:, :r], B[r:, :r]),
            "orth": emax(A[r:, r:], B[r:, r:])}


def compare(name, prob, sp, Ct, bt, r_expect, **kw):
    from paper_2407_14013_gb300 import NewtonSolver
    s = NewtonSolver(prob, **kw)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged and info.r == r_expect
    dX, dy, dS = dX.cpu().numpy(), dy.cpu().numpy(), dS.cpu().numpy()
    s.close()
    Wm = (sp.V * sp.lam) @ sp.V.T
    rX, ry, rS = onewton.newton_direct(prob, Wm, Ct, bt)
    err = {"dX": emax(dX, rX), "dy": emax(dy, ry), "dS": emax(dS, rS)}
    err.update({"dX_" + k: v for k, v in block_errors(dX, rX, sp.V, sp.lam, r_expect).items()})
    print(f"\n{name}: pcg_iters={info.pcg_iters} space={info.space} " +
          " ".join(f"{k}={v:.2e}" for k, v in err.items()))
    for k, v in err.items():
        assert v <= TOL, (name, k, v)
    return err


def test_sensing_full_size_entrywise():
    """Matrix sensing n = 200, m = 2000 (the bench workload), r = 3, d-space core."""
    prob = W.workload("sensing200")
    sp = W.scaling_point(200, 3, 1e-3, 5101, V_top=prob.meta["U"])
    Ct, bt = W.newton_rhs(200, 2000, 5102)
    compare("sensing200", prob, sp, Ct, bt, 3, r_hat=3)


def test_maxcut_full_size_entrywise():
    """MaxCut n = 5000 (average degree 8, N(0,1) weights), r = 100: the m-space core K in
    closed form, the products with B from the eigenvectors, tensor-core FP64 products."""
    prob = W.workload("maxcut5000")
    sp = W.scaling_point(5000, 100, 1e-3, 5103)
    Ct, bt = W.newton_rhs(5000, 5000, 5104)
    compare("maxcut5000", prob, sp, Ct, bt, 100, r_hat=100)


def test_completion_500_500_entrywise():
    """Matrix completion 500 + 500, 5% of a rank-5 target (m = 12500), r = 5, d-space core."""
    prob = W.completion(500, 500, 5, 0.05, 5105)
    assert prob.m == 12500
    sp = W.scaling_point(1000, 5, 1e-3, 5106)
    Ct, bt = W.newton_rhs(1000, prob.m, 5107)
    compare("completion1000", prob, sp, Ct, bt, 5, r_hat=5)


def test_completion_full_size_newt_eps_residual():
    """The completion workload at full size (1000 + 1000, m = 50000, r = 5): the GPU direction
    satisfies (Newt-eps) -- primal block A(dX) = b~ and dual block -W^{-1} dX W^{-1} + A^T(dy) = C~
    -- to 1e-8 relative, the residual evaluated by the oracle's operators; dS = C~ - A^T(dy)."""
    from paper_2407_14013_gb300 import NewtonSolver
    prob = W.workload("completion2000")
    sp = W.scaling_point(2000, 5, 1e-4, 5108)
    Ct, bt = W.newton_rhs(2000, prob.m, 5109)
    s = NewtonSolver(prob, r_hat=5)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged and info.r == 5 and info.space == 1
    dX, dy, dS = dX.cpu().numpy(), dy.cpu().numpy(), dS.cpu().numpy()
    s.close()
    Wi = (sp.V / sp.lam) @ sp.V.T
    T = Wi @ dX @ Wi
    Aty = oops.At_op(prob, dy)
    primal = np.linalg.norm(oops.A_op(prob, dX) - bt) / np.linalg.norm(bt)
    dual = np.linalg.norm(-T + Aty - Ct) / (np.linalg.norm(T) + np.linalg.norm(Ct))
    print(f"\ncompletion2000: pcg_iters={info.pcg_iters} primal={primal:.2e} dual={dual:.2e}")
    assert primal <= TOL and dual <= TOL
    assert emax(dS, Ct - Aty) <= 1e-12


def test_integer_passes_rows_with_internal_spread():
    """Entries spread over 1e-8 .. 1 inside every row of A (each entry scaled by 10^(-8u), u
    uniform): the integer-digit passes (one power-of-two scale per row) and the FP64 FMA passes
    both match the oracle entry by entry."""
    prob = W.sensing(40, 300, 2, 5110)
    rng = np.random.default_rng(5111)
    prob.a_dense = prob.a_dense * 10.0 ** (-8.0 * rng.random(prob.a_dense.shape))
    sp = W.scaling_point(40, 2, 1e-2, 5112)
    Ct, bt = W.newton_rhs(40, 300, 5113)
    for ip in (True, False):
        compare(f"rowspread int_passes={ip}", prob, sp, Ct, bt, 2, r_hat=3, int_passes=ip)


def test_integer_passes_solution_with_wide_spread():
    """A right side whose exact solution dy* has entries spanning 1e-8 .. 1 (C~ = 0,
    b~ = A(W A^T(dy*) W), so dy = dy*, dX = W A^T(dy*) W, dS = -A^T(dy*)): the vector the
    recovery passes over A, u = tau^2 dy, spans the same decades."""
    prob = W.sensing(40, 300, 2, 5114)
    rng = np.random.default_rng(5115)
    ys = rng.choice([-1.0, 1.0], 300) * 10.0 ** (-8.0 * rng.random(300))
    sp = W.scaling_point(40, 2, 1e-2, 5116)
    Wm = (sp.V * sp.lam) @ sp.V.T
    Xs = Wm @ oops.At_op(prob, ys) @ Wm
    bt = oops.A_op(prob, Xs)
    Ct = np.zeros((40, 40))
    from paper_2407_14013_gb300 import NewtonSolver
    for ip in (True, False):
        s = NewtonSolver(prob, r_hat=3, int_passes=ip)
        dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
        assert info.converged
        e = {"dy": emax(dy.cpu().numpy(), ys), "dX": emax(dX.cpu().numpy(), Xs),
             "dS": emax(dS.cpu().numpy(), -oops.At_op(prob, ys))}
        print(f"\nwide-spread dy int_passes={ip}: " + " ".join(f"{k}={v:.2e}" for k, v in e.items()))
        s.close()
        for k, v in e.items():
            assert v <= TOL, (ip, k, v)

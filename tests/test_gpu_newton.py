"""GPU parity of the Newton solve (C ABI) against the CPU oracle.

Tolerance: the FP64 form must agree to relative 1e-8.  Both sides solve the
same well-conditioned augmented system (eq. augsys) to ||r|| <= 1e-12 ||g||; their
difference is bounded by cond(augsys) * 1e-12 plus rounding, so 1e-8 holds for the
moderate spectra used here.  Against the plain Schur-complement definition the FP64
error of that route itself grows like cond(W)^2 eps (Section 1), so those checks use
mu >= 1e-3 where cond(W)^2 eps < 1e-9.
"""
import numpy as np
import pytest

import workloads as W
from oracle import linalg, newton as onewton, operators as oops, reform

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def gpu_solve(prob, sp, Ct, bt, **kw):
    """Set up a solver for `prob` (keyword options of NewtonSolver) and solve once."""
    from paper_2407_14013_gb300 import NewtonSolver
    s = NewtonSolver(prob, **kw)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    out = (dX.cpu().numpy(), dy.cpu().numpy(), dS.cpu().numpy(), info)
    return s, out


def w_of(sp):
    return (sp.V * sp.lam) @ sp.V.T


CASES = [
    # name, problem factory, r_true, mu, r_hat
    ("sensing12", lambda: W.sensing(12, 40, 2, 101), 2, 1e-3, 4),
    ("sensing37_ragged", lambda: W.sensing(37, 150, 3, 102), 3, 1e-3, 5),
    ("sensing65", lambda: W.sensing(65, 400, 2, 103), 2, 1e-2, 3),
    ("maxcut64", lambda: W.workload("maxcut64"), 3, 1e-3, 12),
    ("maxcut130", lambda: W.maxcut(130, 0.05, 104), 4, 1e-2, 6),
]


@pytest.mark.parametrize("name,mk,rt,mu,rh", CASES, ids=[c[0] for c in CASES])
def test_newton_matches_direct_definition(name, mk, rt, mu, rh):
    prob = mk()
    sp = W.scaling_point(prob.n, rt, mu, 200 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 300 + prob.n)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=rh)
    assert info.converged and info.status == 0
    rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
    assert rel(dX, rX) < TOL and rel(dy, ry) < TOL and rel(dS, rS) < TOL
    assert np.allclose(dX, dX.T, rtol=0, atol=1e-14 * np.abs(dX).max())


@pytest.mark.parametrize("space", [1, 2])
@pytest.mark.parametrize("name,mk,rt,mu,rh", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_newton_matches_reform_oracle_each_space(name, mk, rt, mu, rh, space):
    """Same r, beta, space and stopping rule as the oracle's step-by-step reformulation."""
    prob = mk()
    sp = W.scaling_point(prob.n, rt, 1e-5, 400 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 500 + prob.n)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, precond_space=space)
    assert info.converged and info.space == space
    sA = oops.row_norm_scale(prob)
    oX, oy, oS, oinfo = reform.newton_reform(prob, sp.V, sp.lam, Ct, bt, r_hat=rh, s_A=sA,
                                             space="d" if space == 1 else "m", rtol=1e-12, maxit=2000)
    assert info.r == oinfo.split.r and info.d == oinfo.split.d
    assert abs(info.tau - oinfo.split.tau) <= 1e-14 * oinfo.split.tau
    assert abs(info.beta - oinfo.split.beta) <= 1e-12 * oinfo.split.beta
    assert abs(info.s_A - sA) <= 1e-12 * sA
    assert rel(dX, oX) < TOL and rel(dy, oy) < TOL and rel(dS, oS) < TOL
    # setup objects: E, D = tau^2 Sigma, B = A Q (row-major)
    n, m, d = prob.n, prob.m, info.d
    E = s.debug_buffer(0, n * n).cpu().numpy().reshape(n, n, order="F")
    assert rel(E, oinfo.split.E) < 1e-12
    Dv = s.debug_buffer(1, d).cpu().numpy()
    assert rel(Dv, oinfo.split.tau ** 2 * reform.sigma_vec(oinfo.split)) < 1e-12
    if prob.kind == "diag" and space == 2:
        # no explicit B: the m-space core K = beta I + B D^{-1} B^T is formed in closed form;
        # its inverse matches the inverse of the oracle's K (formed by the definition) to
        # about cond(K) eps
        Ki = s.debug_buffer(3, m * m).cpu().numpy().reshape(m, m, order="F")
        K = oinfo.precond.Cmat
        assert rel(Ki, np.linalg.inv(K)) < 1e-15 * np.linalg.cond(K) * 100
    else:
        B = s.debug_buffer(2, m * d).cpu().numpy().reshape(m, d)
        assert rel(B, oinfo.precond.B) < 1e-12
    s.close()


DIAG_LARGE = [
    # n ragged against every tile shape, r above the GEMM tile widths
    ("maxcut601_r37", lambda: W.maxcut(601, 0.014, 105, weights="gauss"), 37, 1e-3, 40),
    ("maxcut1200_r50", lambda: W.maxcut(1200, 0.007, 106, weights="gauss"), 50, 1e-2, 50),
]


@pytest.mark.parametrize("name,mk,rt,mu,rh", DIAG_LARGE, ids=[c[0] for c in DIAG_LARGE])
def test_diag_closed_form_core_large(name, mk, rt, mu, rh):
    """DIAG kind at larger n and r: m-space core in closed form, products with B from Vs;
    the direction matches the oracle's plain definition."""
    prob = mk()
    sp = W.scaling_point(prob.n, rt, mu, 700 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 800 + prob.n)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=rh)
    assert info.converged and info.space == 2 and info.r == rt
    rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
    assert rel(dX, rX) < TOL and rel(dy, ry) < TOL and rel(dS, rS) < TOL
    with pytest.raises(Exception):
        s.debug_buffer(2, 1)                          # B is not formed
    s.close()


def test_newt_eps_residual_full_size_sensing200():
    """Full-size sensing workload (n=200, m=2000, r=3): the recovered direction satisfies
    (Newt-eps) to a small residual; the residual is evaluated by the oracle's operators."""
    prob = W.workload("sensing200")
    sp = W.scaling_point(prob.n, 3, 1e-6, 4242)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 4243)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=3)
    assert info.converged and info.r == 3 and info.d == 597 and info.space == 1
    Wm = w_of(sp)
    res = onewton.newt_eps_residual(prob, Wm, Ct, bt, dX, dy)
    N = prob.n * (prob.n + 1) // 2
    # primal block: A(dX) = b~ ; dual block relative to ||C~|| (amplified by ||W^-1||^2 rounding)
    assert np.linalg.norm(res[N:]) <= 1e-8 * np.linalg.norm(bt)
    Wi = np.linalg.inv(Wm)
    scale = np.linalg.norm(Wi @ dX @ Wi) + np.linalg.norm(Ct)
    assert np.linalg.norm(res[:N]) <= 1e-8 * scale
    assert np.allclose(dS, Ct - oops.At_op(prob, dy), rtol=0, atol=1e-10 * np.abs(Ct).max())
    # sampled entries of A(dX) equal b~ (computed one by one from the svec rows)
    idx = np.random.default_rng(0).choice(prob.m, 16, replace=False)
    sv = linalg.svec(dX)
    for i in idx:
        assert abs(prob.a_dense[i] @ sv - bt[i]) <= 1e-8 * (1 + abs(bt[i]))
    s.close()


def test_host_entry_matches_device_entry():
    import torch
    prob = W.sensing(20, 80, 2, 111)
    sp = W.scaling_point(20, 2, 1e-4, 112)
    Ct, bt = W.newton_rhs(20, 80, 113)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=3)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    out = (torch.empty((20, 20), dtype=torch.float64).pin_memory(), torch.empty(80, dtype=torch.float64).pin_memory(),
           torch.empty((20, 20), dtype=torch.float64).pin_memory())
    Vcm = pin(sp.V.T).t()            # pinned, column-major storage of V
    hX, hy, hS, hinfo = s.solve_host(Vcm, pin(sp.lam), pin(Ct), pin(bt), out)
    assert np.array_equal(hX.numpy(), dX) and np.array_equal(hy.numpy(), dy) and np.array_equal(hS.numpy(), dS)
    s.close()


def test_edge_cases_rank_and_sizes():
    # r = n - 1 (largest rank), r = 1, n = 2, m = 1
    for n, m, rfix in [(6, 10, 5), (6, 10, 1), (2, 2, 1), (5, 1, 1)]:
        prob = W.sensing(n, m, 1, 600 + n + m)
        sp = W.scaling_point(n, 1, 1e-2, 601 + n)
        Ct, bt = W.newton_rhs(n, m, 602 + n)
        s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_fixed=rfix)
        assert info.r == rfix and info.converged
        rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
        assert rel(dX, rX) < TOL and rel(dy, ry) < TOL, (n, m, rfix)
        s.close()


def test_errors_are_reported():
    from paper_2407_14013_gb300 import SdpError, native
    prob = W.sensing(8, 20, 2, 700)
    sp = W.scaling_point(8, 2, 1e-3, 701)
    Ct, bt = W.newton_rhs(8, 20, 702)
    lam_bad = sp.lam.copy()
    lam_bad[3] = -1.0
    from paper_2407_14013_gb300 import NewtonSolver
    s = NewtonSolver(prob, r_hat=3)
    with pytest.raises(SdpError) as e:
        s.solve(_t(sp.V), _t(lam_bad), _t(Ct), _t(bt))
    assert e.value.status == native.SDP_EINVAL
    s.close()
    s = NewtonSolver(prob, r_hat=3, max_pcg=1, newton_rtol=1e-15)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt), allow_notconv=True)
    assert info.status == native.SDP_ENOTCONV and info.pcg_iters == 1 and not info.converged
    # a later good solve on the same handle still works
    s2 = NewtonSolver(prob, r_hat=3)
    _, _, _, i2 = s2.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert i2.converged
    s.close()
    s2.close()


@pytest.mark.parametrize("int_passes", [True, False])
def test_zero_and_non_finite_right_sides(int_passes):
    """A zero right side gives the zero direction (the passes' vectors are all zero: no exponent);
    a NaN in C~ is reported as SDP_ENUMERIC (the integer passes turn a non-finite vector into
    NaN outputs, as FP64 arithmetic does) and leaves the handle usable for a good right side."""
    from paper_2407_14013_gb300 import NewtonSolver, SdpError, native
    prob = W.sensing(12, 40, 2, 710)
    sp = W.scaling_point(12, 2, 1e-3, 711)
    Ct, bt = W.newton_rhs(12, 40, 712)
    s = NewtonSolver(prob, r_hat=3, int_passes=int_passes)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(np.zeros_like(Ct)), _t(np.zeros_like(bt)))
    assert info.converged and info.status == 0
    assert not np.any(dX.cpu().numpy()) and not np.any(dy.cpu().numpy()) and not np.any(dS.cpu().numpy())
    Cn = Ct.copy()
    Cn[3, 5] = Cn[5, 3] = np.nan
    with pytest.raises(SdpError) as e:
        s.solve(_t(sp.V), _t(sp.lam), _t(Cn), _t(bt))
    assert e.value.status == native.SDP_ENUMERIC
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged
    rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
    assert rel(dX.cpu().numpy(), rX) < TOL and rel(dy.cpu().numpy(), ry) < TOL
    s.close()


def test_graph_replay_matches_plain_launches():
    """The PCG iterations replayed from a captured CUDA graph give the same bits as plain launches."""
    prob = W.sensing(40, 200, 2, 801)
    sp = W.scaling_point(40, 2, 1e-5, 802)
    Ct, bt = W.newton_rhs(40, 200, 803)
    s1, (X1, y1, S1, i1) = gpu_solve(prob, sp, Ct, bt, r_hat=3, use_graph=True)
    s2, (X2, y2, S2, i2) = gpu_solve(prob, sp, Ct, bt, r_hat=3, use_graph=False)
    assert i1.pcg_iters == i2.pcg_iters and i1.converged and i2.converged
    assert np.array_equal(X1, X2) and np.array_equal(y1, y2) and np.array_equal(S1, S2)
    # a second solve on the same handle reuses the captured graph
    _, _, _, i3 = s1.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert i3.pcg_iters == i1.pcg_iters
    # event timing of the dense passes works in both modes
    for s in (s1, s2):
        s.set_profiling(True)
        _, _, _, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
        assert info.prof_A_launches == info.pcg_iters + 2       # right side, r0, one per iteration
        assert info.prof_At_launches == info.pcg_iters + 2      # r0, one per iteration, recovery
        assert info.prof_A_ms > 0 and info.prof_At_ms > 0
        s.close()


MIXED_CASES = [
    ("sensing40", lambda: W.sensing(40, 200, 2, 901), 2, 1e-5, 3, 1),
    ("sensing37_m", lambda: W.sensing(37, 150, 3, 902), 3, 1e-3, 5, 2),
    ("maxcut64", lambda: W.workload("maxcut64"), 3, 1e-4, 12, 0),
]


@pytest.mark.parametrize("name,mk,rt,mu,rh,space", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_mixed_precision_matches_fp64(name, mk, rt, mu, rh, space):
    """Correction solves with the FP32 A E A^T block under FP64 refinement reach the same
    (Newt-eps) stop test as the FP64 form, on the true FP64 residual, so the two directions
    agree to the FP64 tolerance."""
    prob = mk()
    sp = W.scaling_point(prob.n, rt, mu, 1000 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 1100 + prob.n)
    s64, (X64, y64, S64, i64) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, precond_space=space)
    s32, (X32, y32, S32, i32) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, precond_space=space, precision="mixed_fp32")
    assert i64.converged and i32.converged and i32.refine_steps >= 1
    assert i32.res_norm <= 1e-12 * i32.rhs_norm                      # the FP64 residual itself
    assert rel(X32, X64) < TOL and rel(y32, y64) < TOL and rel(S32, S64) < TOL
    s64.close()
    s32.close()


def test_mixed_full_size_sensing200():
    prob = W.workload("sensing200")
    sp = W.scaling_point(prob.n, 3, 1e-6, 4242, V_top=prob.meta["U"])
    Ct, bt = W.newton_rhs(prob.n, prob.m, 4243)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=3, precision="mixed_fp32")
    assert info.converged and info.refine_steps >= 1
    Wm = w_of(sp)
    res = onewton.newt_eps_residual(prob, Wm, Ct, bt, dX, dy)
    N = prob.n * (prob.n + 1) // 2
    assert np.linalg.norm(res[N:]) <= 1e-8 * np.linalg.norm(bt)
    s.set_profiling(True)
    _, _, _, i2 = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert i2.prof_A32_launches == i2.pcg_iters + i2.refine_steps       # r0 of each solve + one per iteration
    assert i2.prof_A_launches == i2.refine_steps + 1                    # right side + one residual per correction
    s.close()


def test_resolve_reuses_setup():
    """sdp_newton_resolve (second right side at the same scaling point, a1/a2 reused) gives the
    direction a fresh solve gives, and refuses to run on a handle without a previous solve."""
    from paper_2407_14013_gb300 import NewtonSolver, SdpError
    prob = W.sensing(30, 120, 2, 1701)
    sp = W.scaling_point(prob.n, 2, 1e-4, 1702)
    Ct1, bt1 = W.newton_rhs(prob.n, prob.m, 1703)
    Ct2, bt2 = W.newton_rhs(prob.n, prob.m, 1704)
    s = NewtonSolver(prob, r_hat=4)
    with pytest.raises(SdpError):
        s.resolve(_t(Ct2), _t(bt2))
    s.solve(_t(sp.V), _t(sp.lam), _t(Ct1), _t(bt1))
    dX, dy, dS, info = s.resolve(_t(Ct2), _t(bt2))
    assert info.converged
    fX, fy, fS, _ = s.solve(_t(sp.V), _t(sp.lam), _t(Ct2), _t(bt2))
    for a, b in ((dX, fX), (dy, fy), (dS, fS)):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-10
    s.close()


def test_mixed_continues_in_fp64_after_the_refinement_limit():
    """With max_refine = 1 one FP32 correction cannot reach the 1e-12 stop test; the FP64 PCG
    continues from the refined iterate and the direction equals the FP64 form's."""
    prob = W.sensing(37, 150, 3, 102)
    sp = W.scaling_point(prob.n, 3, 1e-4, 1237)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 1238)
    s64, (X64, y64, S64, i64) = gpu_solve(prob, sp, Ct, bt, r_hat=5)
    s32, (X32, y32, S32, i32) = gpu_solve(prob, sp, Ct, bt, r_hat=5, precision="mixed_fp32", max_refine=1)
    assert i32.converged and i32.refine_steps == 1
    assert i32.res_norm <= 1e-12 * i32.rhs_norm
    assert rel(X32, X64) < TOL and rel(y32, y64) < TOL and rel(S32, S64) < TOL
    s64.close()
    s32.close()


TC_CASES = [
    # n >= 512: E, E C~, the recovery and the complement run on the tensor cores (exact slices)
    ("maxcut700_r20", lambda: W.maxcut(700, 0.012, 107, weights="gauss"), 20, 24),
    ("completion260x260", lambda: W.completion(260, 260, 3, 0.04, 23), 3, 3),
]


@pytest.mark.parametrize("name,mk,rt,rh", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_tensor_core_products_match_fp64_mma_and_oracle(name, mk, rt, rh):
    """The Newton direction with the large products on the BF16 tensor cores equals the one with
    every product on the FP64 MMA path (both stop at the same 1e-12 test) and the oracle's plain
    definition to the FP64 tolerance."""
    prob = mk()
    sp = W.scaling_point(prob.n, rt, 1e-3, 900 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 901 + prob.n)
    s1, (X1, y1, S1, i1) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, tc_products=True)
    s0, (X0, y0, S0, i0) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, tc_products=False)
    assert i1.converged and i0.converged and i1.r == rt
    assert rel(X1, X0) < 1e-10 and rel(y1, y0) < 1e-10 and rel(S1, S0) < 1e-10
    rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
    assert rel(X1, rX) < TOL and rel(y1, ry) < TOL and rel(S1, rS) < TOL
    s1.close()
    s0.close()


def _row_scaled(prob, seed, spread):
    """The same constraints with row i multiplied by 10^u_i, u_i ~ U(-spread, spread): rows of
    very different size exercise the per-row exponents of the integer passes."""
    g = np.random.default_rng(seed)
    prob.a_dense = prob.a_dense * (10.0 ** g.uniform(-spread, spread, prob.m))[:, None]
    return prob


INT_CASES = [
    # name, problem factory, r_true, r_hat; odd n(n+1)/2 (padded rows), streamed A (> 64 MB)
    ("sensing10_odd_rows", lambda: W.sensing(10, 30, 2, 131), 2, 3),
    ("sensing37_scaled_rows", lambda: _row_scaled(W.sensing(37, 150, 3, 132), 7, 1.0), 3, 5),
    ("sensing120_streamed", lambda: W.sensing(120, 1500, 2, 133), 2, 4),
]


@pytest.mark.parametrize("name,mk,rt,rh", INT_CASES, ids=[c[0] for c in INT_CASES])
def test_integer_passes_match_fp64_passes_and_oracle(name, mk, rt, rh):
    """The FP64 operator's passes over A on the integer copy (exact int64 sums of two-digit
    products) give the same Newton direction as FP64 FMAs over A, to far below the FP64
    tolerance, and the oracle's plain definition to it; both stop at the same 1e-12 test."""
    prob = mk()
    sp = W.scaling_point(prob.n, rt, 1e-3, 950 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 951 + prob.n)
    s1, (X1, y1, S1, i1) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, int_passes=True)
    s0, (X0, y0, S0, i0) = gpu_solve(prob, sp, Ct, bt, r_hat=rh, int_passes=False)
    assert i1.converged and i0.converged and i1.r == rt
    assert abs(i1.pcg_iters - i0.pcg_iters) <= max(2, i0.pcg_iters // 20)   # rounding differs, not the method
    assert rel(X1, X0) < 1e-10 and rel(y1, y0) < 1e-10 and rel(S1, S0) < 1e-10
    rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
    assert rel(X1, rX) < TOL and rel(y1, ry) < TOL and rel(S1, rS) < TOL
    s1.close()
    s0.close()


def test_edge_cases_diag_and_sparse_kinds():
    """DIAG at r = 1 (d = n = m: the d-space core with the explicit B of the DIAG kind) and at
    r = n - 1; SPARSE_COO with one constraint and at r = 1; each against the plain definition."""
    cases = [
        (lambda: W.maxcut(9, 0.5, 611), 1, 1),        # d = n = m -> d-space, explicit B
        (lambda: W.maxcut(9, 0.5, 612), 1, 8),        # r = n - 1
        (lambda: W.random_sparse(7, 1, 3, 613), 1, 1),
        (lambda: W.random_sparse(10, 12, 2, 614), 1, 1),
    ]
    for mk, rt, rfix in cases:
        prob = mk()
        sp = W.scaling_point(prob.n, rt, 1e-2, 620 + prob.n + prob.m)
        Ct, bt = W.newton_rhs(prob.n, prob.m, 621 + prob.n + prob.m)
        s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_fixed=rfix)
        assert info.r == rfix and info.converged, (prob.kind, prob.n, prob.m, rfix)
        rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
        assert rel(dX, rX) < TOL and rel(dy, ry) < TOL and rel(dS, rS) < TOL, (prob.kind, prob.n, prob.m, rfix)
        if prob.kind == "diag" and rfix == 1:
            assert info.space == 1
        s.close()


def test_minres_with_tensor_core_products():
    """MINRES at n >= 512: E and the recovery on the tensor cores, the operator in the captured
    Krylov graph; the direction equals the plain definition."""
    prob = W.maxcut(601, 0.014, 105, weights="gauss")
    sp = W.scaling_point(prob.n, 37, 1e-1, 1301)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 1302)
    s, (dX, dy, dS, info) = gpu_solve(prob, sp, Ct, bt, r_hat=40, krylov="minres", max_pcg=50000)
    assert info.converged and info.r == 37
    rX, ry, rS = onewton.newton_direct(prob, w_of(sp), Ct, bt)
    assert rel(dX, rX) < TOL and rel(dy, ry) < TOL and rel(dS, rS) < TOL
    s.close()

"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Each mutation below breaks one formula of the reformulation in a way a
transcription slip would (a dropped sqrt(2), a sign, tau instead of tau^2, a
transposed operand, the paper's literal PCG beta index); the corresponding
identity from the paper must then fail.
"""
import numpy as np
import pytest

import workloads as W
from oracle import linalg, reform


def _split(n=6, r=2, mu=1e-3, seed=900):
    sp_in = W.scaling_point(n, r, mu, seed)
    return sp_in, reform.split(sp_in.V, sp_in.lam, r=r)


def _identity_error(s, sp_in):
    Wm = (sp_in.V * sp_in.lam) @ sp_in.V.T
    WW = linalg.skron(Wm, Wm)
    Qb = np.column_stack([linalg.svec(reform.Q_op(s, e)) for e in np.eye(s.d)])
    recon = Qb @ np.diag(1 / reform.sigma_vec(s)) @ Qb.T + s.tau ** 2 * linalg.skron(s.E, s.E)
    return np.linalg.norm(recon - WW) / np.linalg.norm(WW)


def test_unmutated_identity_holds():
    sp_in, s = _split()
    assert _identity_error(s, sp_in) < 1e-12


def test_mutation_missing_sqrt2_in_Q(monkeypatch):
    sp_in, s = _split()

    def bad_Q(sp, h):
        B, N = reform.unpack_h(sp, h)
        U = sp.Q @ B + (sp.Qp @ N)            # sqrt(2) dropped
        M = U @ sp.Q.T
        return 0.5 * (M + M.T)

    monkeypatch.setattr(reform, "Q_op", bad_Q)
    assert _identity_error(s, sp_in) > 1e-3


@pytest.mark.parametrize("field,bad", [
    ("sigB", lambda s: 1.0 / (np.outer(s.lam, s.lam) + s.tau ** 2)),     # sign of tau^2
    ("sigB", lambda s: 1.0 / (np.outer(s.lam, s.lam) - s.tau)),          # tau instead of tau^2
    ("sigN", lambda s: 1.0 / np.outer(s.lamp, s.lam)),                   # dropped -tau
])
def test_mutation_sigma(field, bad):
    sp_in, s = _split()
    setattr(s, field, bad(s))
    assert _identity_error(s, sp_in) > 1e-6


def test_mutation_E_uses_lambda_not_over_tau():
    sp_in, s = _split()
    s.E = s.Q @ s.Q.T + (s.Qp * s.lamp) @ s.Qp.T           # tau^{-1} dropped
    assert _identity_error(s, sp_in) > 1e-6


def test_mutation_transposed_Qt():
    """Q^T must be the adjoint of Q; using Q_perp^T X Q_perp-like transposes breaks it."""
    sp_in, s = _split()
    g = np.random.default_rng(1)
    X = g.standard_normal((s.n, s.n))
    X = X + X.T
    h = g.standard_normal(s.d)
    good = abs(np.sum(reform.Q_op(s, h) * X) - h @ reform.Qt_op(s, X))
    assert good < 1e-10
    XQ = X @ s.Qp[:, :s.r]                                  # wrong factor on the right
    bad_vec = np.concatenate([linalg.svec(s.Q.T @ X @ s.Q), np.sqrt(2) * (s.Qp.T @ XQ).reshape(-1, order="F")])
    assert abs(np.sum(reform.Q_op(s, h) * X) - h @ bad_vec) > 1e-3


def test_mutation_literal_pcg_beta_breaks_equivalence():
    """With beta_j = <r_{j+1}, z_j>/<r_j, z_j> (as printed in Def. pcg), PCG loses the
    finite-termination property that the standard coefficient has on a small SPD system."""
    g = np.random.default_rng(2)
    n = 12
    G = g.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    Pm = np.diag(np.diag(A))
    b = g.standard_normal(n)
    good = reform.pcg(lambda x: A @ x, b, lambda r: np.linalg.solve(Pm, r), np.zeros(n), tol=0.0, maxit=n)
    assert np.linalg.norm(A @ good.x - b) < 1e-9 * np.linalg.norm(b)

    def pcg_literal(maxit):
        x = np.zeros(n)
        r = b.copy()
        z = np.linalg.solve(Pm, r)
        p = z.copy()
        for _ in range(maxit):
            Ap = A @ p
            alpha = (r @ z) / (p @ Ap)
            x = x + alpha * p
            r_new = r - alpha * Ap
            beta = (r_new @ z) / (r @ z)
            z = np.linalg.solve(Pm, r_new)
            p = z + beta * p
            r = r_new
        return x

    assert np.linalg.norm(A @ pcg_literal(n) - b) > 1e-6 * np.linalg.norm(b)


# ---- the linear cone (robust problems): mistakes in the preconditioner and the outer loop


def _lp_precond_case(seed=61, mu=1e-4, n=8, m=20):
    from oracle import lpcone
    from oracle.operators import A_op, At_op
    prob = W.sensing(n, m, 2, seed)
    sp_in = W.scaling_point(n, 2, mu, seed + 1)
    s = reform.split(sp_in.V, sp_in.lam, r_hat=3)
    G = np.hstack([np.eye(m), -np.eye(m)])
    d = 10.0 ** np.random.default_rng(seed).uniform(-3, 3, 2 * m)
    GDG = lpcone.gdg(G, d)
    K = np.zeros((m + s.d, m + s.d))
    for j in range(m + s.d):
        e = np.zeros(m + s.d)
        e[j] = 1.0
        a, b = reform.aug_apply(prob, s, e[:m], e[m:])
        K[:, j] = np.concatenate([a + GDG @ e[:m] / s.tau ** 2, b])
    AEA = np.column_stack([A_op(prob, reform.E_op(s, At_op(prob, e))) for e in np.eye(m)])
    ev = np.linalg.eigvalsh(0.5 * (AEA + AEA.T))
    return prob, s, G, d, K, min(1.0, ev[0] / s.beta), max(1.0, ev[-1] / s.beta)


@pytest.mark.parametrize("space", ["d", "m"])
def test_lp_preconditioned_spectrum_lies_in_the_mediant_bound(space):
    """With K = [[H, B], [B^T, -D]] and P = [[Lam, B], [B^T, -D]] sharing the second block row,
    P^{-1} K = I + P^{-1} diag(H - Lam, 0): its eigenvalues are 1 (d times) and those of the pencil
    (H + B D^{-1} B^T, Lam + B D^{-1} B^T), which by the mediant inequality for Rayleigh quotients
    lie between min(1, l_min) and max(1, l_max), where l ranges over the pencil (H, Lam).  For
    H = A E A^T + tau^{-2} G D G^T and Lam = beta I + tau^{-2} G D G^T that pencil lies between
    min(1, lambda_min(A E A^T)/beta) and max(1, lambda_max(A E A^T)/beta), whatever d is.  Dropping
    tau^{-2} from Lam (a plausible slip: the operator scales the block, the preconditioner not)
    breaks the bound once tau < 1."""
    from oracle import lpcone
    prob, s, G, d, K, lo, hi = _lp_precond_case()
    P = lpcone.precond_setup_lp(prob, s, G, d, space=space)
    ev = np.linalg.eigvals(np.linalg.solve(lpcone.precond_matrix_lp(P), K))
    assert np.abs(ev.imag).max() <= 1e-6
    assert ev.real.min() >= lo * (1 - 1e-8) and ev.real.max() <= hi * (1 + 1e-8)
    assert s.tau < 1.0
    P.lam = s.beta + np.diag(lpcone.gdg(G, d))              # mutation: tau^{-2} dropped
    ev_bad = np.linalg.eigvals(np.linalg.solve(lpcone.precond_matrix_lp(P), K))
    assert ev_bad.real.max() > 2 * hi


def _rmc_outer(monkeypatch=None):
    from oracle import ipm_lp
    prob = W.rmc(12, 70, 3, 9)
    try:
        res = ipm_lp.ipm_solve_lp(prob, prob.meta["G_l"], prob.meta["c_l"], tol=1e-8, max_iter=60)
    except np.linalg.LinAlgError:
        return False
    Xs = prob.meta["Xs"]
    return bool(res.converged and res.x.min() > 0 and np.linalg.norm(res.X - Xs) <= 1e-6 * np.linalg.norm(Xs))


def test_lp_outer_loop_unmutated_recovers():
    assert _rmc_outer()


def test_mutation_lp_step_without_the_ratio_test(monkeypatch):
    """Steps that ignore the orthant (no bound from x + a dx >= 0) leave the interior: the
    recovery pin fails (here the scaling d = x / z turns negative and the Cholesky factor of
    the complement fails)."""
    from oracle import ipm_lp
    monkeypatch.setattr(ipm_lp, "ratio_step", lambda x, dx: float("inf"))
    assert not _rmc_outer()


@pytest.mark.parametrize("slip", ["dx_sign", "d_inverted"])
def test_mutation_lp_direction(monkeypatch, slip):
    """dx = D(G^T dy + c~) (sign of c~) or d = z / x instead of x / z: the outer loop no longer
    reaches the planted matrix."""
    from oracle import ipm_lp
    orig = ipm_lp.newton_reform_lp

    def bad(prob, V, lam, Ct, bt, G, d, ct, **kw):
        if slip == "d_inverted":
            return orig(prob, V, lam, Ct, bt, G, 1.0 / d, ct, **kw)
        dX, dx, dy, info = orig(prob, V, lam, Ct, bt, G, d, ct, **kw)
        return dX, d * (G.T @ dy + ct), dy, info

    monkeypatch.setattr(ipm_lp, "newton_reform_lp", bad)
    assert not _rmc_outer()

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

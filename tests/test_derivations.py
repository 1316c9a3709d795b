"""Identities the CUDA path relies on where it does not follow the oracle's definition step by
step, checked against the oracle's definitions on CPU.

- DIAG kind (A_i = e_i e_i^T), m-space core: the CUDA path forms
      K = beta I + tau^-2 G o (G + 2 tau E),   G = Q (Lam - tau I) Q^T,
  instead of beta I + B D^{-1} B^T with B = A Q formed column by column.  Derivation: row i of
  B is [svec(q_i q_i^T); sqrt2 vec(p_i q_i^T)] and D^{-1} = Sigma^{-1} / tau^2 (eq. EQSigdef),
  so the svec block gives (Q Lam Q^T)_il^2 - tau^2 (Q Q^T)_il^2 and the N block gives
  2 (Q (Lam - tau I) Q^T)_il (Qp Lamp Qp^T)_il, with Qp Lamp Qp^T = tau (E - Q Q^T).
- DIAG kind, products with B without B: B t = rowdot(Vs unpack(t), Q) and
  B^T u = pack(Vs^T diag(u) Q).
- SPARSE kind, d-space core in its Gram form: with A_i = sum_t w_t e_{x_t} e_{y_t}^T over its terms
  (an off-diagonal entry gives (r, c) and (c, r)), H_i = Vs^T A_i Q has vec(H_i) =
  sum_t w_t Q[y_t, :] (x) Vs[x_t, :], so block (j1, j2) of sum_i vec(H_i) vec(H_i)^T is
  Vs^T W_{j1 j2} Vs, W_{j1 j2} = sum_i sum_{t, t'} w_t w_t' Q[y_t, j1] Q[y_t', j2] e_{x_t} e_{x_t'}^T;
  B^T B follows through the h-coordinate map of pack(.), one product per unordered (j1, j2).
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as oops, reform


def _split(n, r_true, r_hat, seed, mu):
    prob = W.maxcut(n, 0.2, seed, weights="gauss")
    sp = W.scaling_point(n, r_true, mu, seed + 1)
    s = reform.split(sp.V, sp.lam, r_hat=r_hat, s_A=oops.row_norm_scale(prob))
    return prob, s


@pytest.mark.parametrize("n,r_true,r_hat,mu", [(9, 2, 3, 1e-2), (16, 3, 5, 1e-4), (23, 5, 7, 1e-6)])
def test_diag_K_closed_form_equals_definition(n, r_true, r_hat, mu):
    prob, s = _split(n, r_true, r_hat, 10 * n, mu)
    K_def = reform.precond_setup(prob, s, "m").Cmat
    G = (s.Q * (s.lam - s.tau)) @ s.Q.T
    K = s.beta * np.eye(n) + G * (G + 2 * s.tau * s.E) / s.tau ** 2
    assert np.linalg.norm(K - K_def) <= 1e-13 * np.linalg.norm(K_def)
    # planted mistakes are caught: the N-block cross term dropped or with its sign flipped
    # (relative size about tau / lam_r, far above the 1e-13 bound)
    for K_bad in (s.beta * np.eye(n) + G * G / s.tau ** 2,
                  s.beta * np.eye(n) + G * (G - 2 * s.tau * s.E) / s.tau ** 2):
        assert np.linalg.norm(K_bad - K_def) > 1e-9 * np.linalg.norm(K_def)


@pytest.mark.parametrize("n,r", [(8, 1), (13, 4)])
def test_diag_B_products_without_B(n, r):
    prob, s = _split(n, r, r, 7 * n, 1e-3)
    B = reform.AQ_matrix(prob, s)
    Vs = np.hstack([s.Q, s.Qp])
    rng = np.random.default_rng(n)
    t, u = rng.standard_normal(s.d), rng.standard_normal(n)
    Bm, N = reform.unpack_h(s, t)
    U = s.Q @ Bm + np.sqrt(2) * (s.Qp @ N)                        # Vs unpack(t)
    assert np.allclose(np.sum(U * s.Q, axis=1), B @ t, rtol=0, atol=1e-13 * np.abs(B @ t).max())
    H = Vs.T @ (u[:, None] * s.Q)
    packed = np.concatenate([reform.svec(0.5 * (H[:r] + H[:r].T)), np.sqrt(2) * H[r:].reshape(-1, order="F")])
    assert np.allclose(packed, B.T @ u, rtol=0, atol=1e-13 * np.abs(B.T @ u).max())


def _gram_btb(prob, s):
    """B^T B assembled as the CUDA path does (Gram blocks over the term pairs), in numpy."""
    n, m, r, d = prob.n, prob.m, s.r, s.d
    Vs = np.hstack([s.Q, s.Qp])
    pairs = []
    for i in range(m):
        terms = []
        for e in np.where(prob.a_con == i)[0]:
            x, y, w = int(prob.a_row[e]), int(prob.a_col[e]), float(prob.a_val[e])
            terms.append((x, y, w))
            if x != y:
                terms.append((y, x, w))
        pairs += [(t[0], u[0], t[1], u[1], t[2] * u[2]) for t in terms for u in terms]
    nb = r * (r + 1) // 2

    def hc(a, j):
        if a < r:
            i, jj = max(a, j), min(a, j)
            return jj * r - jj * (jj - 1) // 2 + (i - jj), (1.0 if i == jj else 0.5 * np.sqrt(2.0))
        return nb + (a - r) + j * (n - r), np.sqrt(2.0)

    C = np.zeros((d, d))
    for j1 in range(r):
        for j2 in range(j1, r):
            Wm = np.zeros((n, n))
            for x, xp, y, yp, w in pairs:
                Wm[x, xp] += w * s.Q[y, j1] * s.Q[yp, j2]
            G = Vs.T @ Wm @ Vs
            for a1 in range(n):
                h1, c1 = hc(a1, j1)
                for a2 in range(n):
                    h2, c2 = hc(a2, j2)
                    C[h1, h2] += c1 * c2 * G[a1, a2]
                    if j1 != j2:
                        C[h2, h1] += c1 * c2 * G[a1, a2]
    return C


@pytest.mark.parametrize("mk", [lambda: W.completion(8, 7, 2, 0.4, 31), lambda: W.random_sparse(11, 25, 3, 32)],
                         ids=["completion", "random_sparse"])
def test_sparse_gram_form_equals_btb(mk):
    prob = mk()
    sp = W.scaling_point(prob.n, 3, 1e-3, 33)
    s = reform.split(sp.V, sp.lam, r_hat=4, s_A=oops.row_norm_scale(prob))
    B = reform.AQ_matrix(prob, s)
    ref = B.T @ B
    got = _gram_btb(prob, s)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()

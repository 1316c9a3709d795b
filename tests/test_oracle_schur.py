"""Pins of the oracle's fast Schur-matrix forms (oracle/newton.py schur_matrix) against the
literal column-by-column definition M_ij = <A_i, W A_j W> (schur_matrix_by_columns, which forms
W A_j W explicitly and applies A): the blocked dense form, the closed form for constraints
with one stored entry (matrix completion, and single diagonal entries), and a planted slip in
the closed form (a dropped cross term) that the comparison catches."""
import numpy as np

import workloads as W
from oracle import newton as onewton


def _w(n, seed):
    sp = W.scaling_point(n, 2, 1e-2, seed)
    return (sp.V * sp.lam) @ sp.V.T


def test_blocked_dense_equals_column_definition():
    prob = W.sensing(13, 47, 2, 9001)
    Wm = _w(13, 9002)
    ref = onewton.schur_matrix_by_columns(prob, Wm)
    for block in (1, 7, 100):
        got = onewton.schur_matrix(prob, Wm, block=block)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_selection_closed_form_equals_column_definition():
    prob = W.completion(6, 5, 2, 0.5, 9003)
    Wm = _w(11, 9004)
    ref = onewton.schur_matrix_by_columns(prob, Wm)
    got = onewton.schur_matrix(prob, Wm)
    assert onewton._single_entry_constraints(prob)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_selection_closed_form_with_diagonal_entries():
    # one entry per constraint, some on the diagonal, arbitrary values
    rng = np.random.default_rng(9005)
    n, m = 7, 12
    r = rng.integers(0, n, m)
    c = np.array([rng.integers(0, ri + 1) for ri in r])
    c[:3] = r[:3]                                   # three diagonal constraints
    prob = W.Problem(kind="sparse", n=n, m=m, b=np.zeros(m), C=np.eye(n),
                     a_con=np.arange(m, dtype=np.int32), a_row=r.astype(np.int32), a_col=c.astype(np.int32),
                     a_val=rng.standard_normal(m))
    Wm = _w(n, 9006)
    ref = onewton.schur_matrix_by_columns(prob, Wm)
    got = onewton.schur_matrix(prob, Wm)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_dropped_cross_term_is_caught():
    prob = W.completion(6, 5, 2, 0.5, 9003)
    Wm = _w(11, 9004)
    ref = onewton.schur_matrix_by_columns(prob, Wm)
    rr = prob.a_row.astype(np.int64)
    cc = prob.a_col.astype(np.int64)
    v = prob.a_val
    wrong = 2.0 * np.outer(v, v) * (Wm[np.ix_(rr, rr)] * Wm[np.ix_(cc, cc)])
    assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()

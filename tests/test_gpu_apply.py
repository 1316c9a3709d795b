"""The augmented operator and the preconditioner, each applied alone through the C ABI
(sdp_apply_augsys), against the oracle's plain definitions at the same split.

After a Newton solve the handle holds the split (E, Q, tau, Sigma) and the preconditioner core of
that scaling point.  One application of M = [[A E A^T, A Q], [Q^T A^T, -tau^2 Sigma]] (eq. augsys)
to a seeded vector is compared with oracle.reform.aug_apply, and one application of the block
preconditioner of Section 6 with oracle.reform.precond_apply (its core factored by Cholesky on the
host), for every constraint kind and both preconditioner spaces.  Tolerances: the operator is
FP64 products and sums (the integer-digit passes agree with FP64 to about 1e-15 relative per
entry), so 1e-11 relative; the preconditioner goes through an inverse of the Schur complement,
so cond(core) eps, about 1e-10 for these instances.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as oops, reform

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = [
    # name, problem, r_true, mu, r_hat, space (1 = d, 2 = m)
    ("sensing37_d", lambda: W.sensing(37, 150, 3, 1601), 3, 1e-3, 5, 1),
    ("sensing30_m", lambda: W.sensing(30, 40, 2, 1602), 2, 1e-3, 3, 2),
    ("maxcut64_m", lambda: W.workload("maxcut64"), 3, 1e-3, 12, 2),
    ("maxcut40_d", lambda: W.maxcut(40, 0.2, 1603), 3, 1e-3, 4, 1),
    ("completion20x15_d", lambda: W.completion(20, 15, 2, 0.3, 1604), 2, 1e-3, 4, 1),
    ("random_sparse257_m", lambda: W.random_sparse(257, 700, 4, 1605), 3, 1e-3, 4, 2),
]


@pytest.mark.parametrize("name,mk,rt,mu,rh,space", CASES, ids=[c[0] for c in CASES])
def test_operator_and_preconditioner_alone_match_oracle(name, mk, rt, mu, rh, space):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    sp = W.scaling_point(prob.n, rt, mu, 1700 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 1800 + prob.n)
    s = NewtonSolver(prob, r_hat=rh, precond_space=space)
    _, _, _, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged and info.space == space
    split = reform.split(sp.V, sp.lam, r_hat=rh, s_A=oops.row_norm_scale(prob))
    assert split.r == info.r and split.d == info.d
    m, d = prob.m, info.d
    g = np.random.default_rng(1900 + prob.n)
    u, v = g.standard_normal(m), g.standard_normal(d)
    vec = _t(np.concatenate([u, v]))
    # the operator
    top, bot = reform.aug_apply(prob, split, u, v)
    got = s.apply(vec, 0).cpu().numpy()
    assert rel(got[:m], top) < 1e-11 and rel(got[m:], bot) < 1e-11
    # the preconditioner in the handle's space
    P = reform.precond_setup(prob, split, space="d" if space == 1 else "m")
    zu, zv = reform.precond_apply(P, u, v)
    got = s.apply(vec, 1).cpu().numpy()
    assert rel(got[:m], zu) < 1e-9 and rel(got[m:], zv) < 1e-9
    # a second application gives the same bits (the applies keep no state between calls)
    again = s.apply(vec, 1).cpu().numpy()
    assert np.array_equal(again, got)
    s.close()


def test_apply_argument_errors():
    from paper_2407_14013_gb300 import NewtonSolver, SdpError, native
    import torch
    prob = W.sensing(12, 40, 2, 1606)
    s = NewtonSolver(prob, r_hat=3)
    vec = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(SdpError) as e:                 # no solve on this handle yet
        s.apply(vec, 0)
    assert e.value.status == native.SDP_EINVAL
    sp = W.scaling_point(12, 2, 1e-3, 1607)
    Ct, bt = W.newton_rhs(12, 40, 1608)
    _, _, _, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    vec = torch.zeros(40 + info.d, dtype=torch.float64, device="cuda")
    with pytest.raises(SdpError) as e:
        native.sdp_apply_augsys(s.handle, vec.data_ptr(), torch.empty_like(vec).data_ptr(), 2)
    assert e.value.status == native.SDP_EINVAL
    assert not np.any(s.apply(vec, 0).cpu().numpy())   # M 0 = 0
    s.close()

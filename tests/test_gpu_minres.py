"""GPU MINRES on the augmented system (Cor. minres: MINRES_k(augsys, g, I, 0), then eq. recover)
against the oracle: the Newton direction equals the plain Schur-complement definition to 1e-8,
the iteration count is at least that of the oracle's MINRES by its definition (exact
termination) and within the Prop. minres bound for the explicit augmented matrix, and no
preconditioner core is formed (smaller workspace, debug copies of B and of the core refused)."""
import numpy as np
import pytest

import workloads as W
from oracle import newton as onewton, operators as oops, reform

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = [
    ("sensing12", lambda: W.sensing(12, 40, 2, 101), 2, 4),
    ("maxcut20", lambda: W.maxcut(20, 0.3, 4101), 3, 5),
    ("completion8x8", lambda: W.completion(8, 8, 2, 0.4, 11), 2, 3),
    ("sensing37_ragged", lambda: W.sensing(37, 150, 3, 102), 3, 5),
]


@pytest.mark.parametrize("name,mk,rt,rh", CASES, ids=[c[0] for c in CASES])
def test_minres_newton_matches_definition_and_oracle_iterations(name, mk, rt, rh):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    sp = W.scaling_point(prob.n, rt, 1e-2, 300 + prob.n)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 301 + prob.n)
    s = NewtonSolver(prob, r_hat=rh, krylov="minres", max_pcg=20000)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged
    rX, ry, rS = onewton.newton_direct(prob, (sp.V * sp.lam) @ sp.V.T, Ct, bt)
    assert rel(dX.cpu().numpy(), rX) < TOL and rel(dy.cpu().numpy(), ry) < TOL and rel(dS.cpu().numpy(), rS) < TOL
    if prob.m + info.d <= 400:
        # the short recurrence loses orthogonality in floating point, so it needs more iterations
        # than the oracle's MINRES by its definition (a re-orthogonalised Krylov basis: exact
        # termination), but stays within the Prop. minres bound for the condition number of the
        # explicit augmented matrix
        _, _, _, ores, spl = reform.newton_minres(prob, sp.V, sp.lam, Ct, bt, r_hat=rh,
                                                  s_A=oops.row_norm_scale(prob), maxit=3000)
        assert ores.converged and ores.iters <= info.pcg_iters
        nt = prob.m + spl.d
        Mx = np.stack([np.concatenate(reform.aug_apply(prob, spl, e[:prob.m], e[prob.m:])) for e in np.eye(nt)], axis=1)
        kappa = np.linalg.cond(Mx)
        g = np.concatenate(reform.aug_rhs(prob, spl, Ct, bt))
        eps = 1e-12 * np.sqrt(np.sum(Ct * Ct) + bt @ bt)
        assert info.pcg_iters <= reform.prop_minres_bound(kappa, np.linalg.norm(g), eps), (info.pcg_iters, kappa)
    s.close()


def test_minres_forms_no_preconditioner_core():
    from paper_2407_14013_gb300 import NewtonSolver
    prob = W.sensing(37, 150, 3, 102)
    sp = W.scaling_point(prob.n, 3, 1e-2, 337)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 338)
    sm = NewtonSolver(prob, r_hat=5, krylov="minres", max_pcg=20000)
    sc = NewtonSolver(prob, r_hat=5)
    assert sm.workspace_bytes() < sc.workspace_bytes()
    _, _, _, im = sm.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    _, _, _, ic = sc.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert im.converged and ic.converged and im.pcg_iters > ic.pcg_iters   # unpreconditioned
    with pytest.raises(Exception):
        sm.debug_buffer(3, 1)
    sm.close()
    sc.close()

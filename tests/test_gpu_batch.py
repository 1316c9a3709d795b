"""Batched solves (sdp_solve_batch): many independent SDPs of uneven size solved by several
host workers, each instance on its own handle and stream.

Each instance must reach the same stopping test as a single sdp_solve (relative gap and
infeasibilities <= 1e-8) and agree with a single solve on the objective (relative 2e-8, both
are within about 1e-8 (1 + 2|p*|) of the optimal value) and on X (relative 1e-6: X is fixed to
O(mu) at the end of the path); two instances are also checked against the oracle's optimum.
The batched solves take the non-cooperative eigensolver paths, so agreement is to the solve
tolerance, not bitwise.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ipm as oipm

pytestmark = pytest.mark.gpu


def _solvers(probs, **kw):
    import torch
    from paper_2407_14013_gb300 import NewtonSolver
    return [NewtonSolver(p, r_hat=kw.get("r_hat", 6), stream=torch.cuda.Stream(), **{k: v for k, v in kw.items()
                                                                                       if k != "r_hat"})
            for p in probs]


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


PROBS = [
    lambda: W.maxcut(20, 0.3, 4101),
    lambda: W.maxcut(37, 0.2, 4102, weights="gauss"),
    lambda: W.workload("maxcut64"),
    lambda: W.sensing(12, 40, 2, 4103),
    lambda: W.sensing(20, 120, 2, 77),
    lambda: W.batch_problem(("sensing", 33, 4104)),
]


def test_batch_matches_single_solves_and_oracle():
    from paper_2407_14013_gb300 import NewtonSolver, solve_sdp_batch
    probs = [mk() for mk in PROBS]
    solvers = _solvers(probs)
    out = solve_sdp_batch(solvers, [_t(p.b) for p in probs], [_t(p.C) for p in probs], gap_tol=1e-8,
                          max_iter=100, workers=4)
    for k, (p, (X, y, S, info)) in enumerate(zip(probs, out)):
        assert info["status"] == 0 and info["converged"] == 1, (k, info)
        assert info["rel_gap"] <= 1e-8 and info["pinf"] <= 1e-8 and info["dinf"] <= 1e-8
        single = NewtonSolver(p, r_hat=6)
        X1, y1, S1, i1 = single.solve_sdp(_t(p.b), _t(p.C), gap_tol=1e-8, max_iter=100)
        single.close()
        Xb, X1 = X.cpu().numpy(), X1.cpu().numpy()
        pb, p1 = float(np.sum(p.C * Xb)), float(np.sum(p.C * X1))
        assert abs(pb - p1) <= 2e-8 * (1 + 2 * abs(p1)), (k, pb, p1)
        assert np.linalg.norm(Xb - X1) <= 1e-6 * np.linalg.norm(X1), k
        if k in (1, 4):
            ref = oipm.ipm_solve(p, tol=1e-8, max_iter=100)
            pr = float(np.sum(p.C * ref.X))
            assert abs(pb - pr) <= 2e-8 * (1 + 2 * abs(pr)), (k, pb, pr)
    for s_ in solvers:
        s_.close()


def test_batch_reports_each_instance_status():
    """Statuses are reported per instance: with enough iterations every instance converges;
    with two iterations each instance reports SDP_ENOTCONV; a repeated handle is refused
    before anything is solved."""
    from paper_2407_14013_gb300 import _native
    probs = [W.maxcut(20, 0.3, 4101), W.sensing(12, 40, 2, 4103)]
    solvers = _solvers(probs)
    import torch
    bs = [_t(p.b) for p in probs]
    Cs = [_t(p.C) for p in probs]
    outs = [(torch.empty((p.n, p.n), dtype=torch.float64, device="cuda"), torch.empty(p.m, dtype=torch.float64,
             device="cuda"), torch.empty((p.n, p.n), dtype=torch.float64, device="cuda")) for p in probs]
    ptr = lambda t: t.data_ptr()
    torch.cuda.synchronize()
    st, infos = _native.sdp_solve_batch([s_.handle for s_ in solvers], [ptr(b) for b in bs], [ptr(c) for c in Cs],
                                        [ptr(o[0]) for o in outs], [ptr(o[1]) for o in outs],
                                        [ptr(o[2]) for o in outs], 1e-8, 100, 2)
    assert st == [0, 0]
    st, infos = _native.sdp_solve_batch([s_.handle for s_ in solvers], [ptr(b) for b in bs], [ptr(c) for c in Cs],
                                        [ptr(o[0]) for o in outs], [ptr(o[1]) for o in outs],
                                        [ptr(o[2]) for o in outs], 1e-8, 2, 2)
    assert st == [_native.SDP_ENOTCONV, _native.SDP_ENOTCONV] and infos[0].iters == 2
    with pytest.raises(_native.SdpError):
        _native.sdp_solve_batch([solvers[0].handle] * 2, [ptr(b) for b in bs], [ptr(c) for c in Cs],
                                [ptr(o[0]) for o in outs], [ptr(o[1]) for o in outs], [ptr(o[2]) for o in outs],
                                1e-8, 100, 2)
    for s_ in solvers:
        s_.close()

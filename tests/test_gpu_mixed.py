"""The mixed-precision forms of the Newton solve against the FP64 oracle.

Each form runs the correction solves of an FP64 iterative refinement with a low-precision
A E A^T block (Section 3 eq. augsys; the refinement is not in the paper):
  mixed_fp32  FP32 copies of A (or E o E), FP32 FFMA products;
  mixed_tf32  the FP32 copy of A, E Y E on the tensor cores with split TF32 operands (hi + lo,
              three MMAs per step);
  mixed_bf16  a BF16 copy of A (or E o E), E Y E on the tensor cores with BF16 operands;
all with FP32 accumulation.  The refinement stops on the FP64 residual with the stop test of the
FP64 form, so every form must give the oracle's direction to the FP64 bar, entry by entry
(max |a - b| <= 1e-8 max |b|).  Each form's own error is that of its correction operator, seen
as the contraction of the FP64 residual per correction (info.refine_rate), printed with the
direction errors (pytest -s) and bounded here.
"""
import numpy as np
import pytest

import workloads as W
from oracle import newton as onewton

pytestmark = pytest.mark.gpu

TOL = 1e-8
# bound on the mean contraction per correction solve, by form
RATE = {"mixed_fp32": 1e-3, "mixed_tf32": 1e-3, "mixed_bf16": 0.5}


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def emax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


CASES = [
    ("sensing37_ragged", lambda: W.sensing(37, 150, 3, 102), 3, 1e-3, 5),
    ("sensing65", lambda: W.sensing(65, 400, 2, 103), 2, 1e-2, 3),
    ("sensing200_full", lambda: W.workload("sensing200"), 3, 1e-3, 3),
    ("maxcut130", lambda: W.maxcut(130, 0.05, 104), 4, 1e-2, 6),
    ("maxcut601_r37", lambda: W.maxcut(601, 0.014, 105, weights="gauss"), 37, 1e-3, 40),
]


@pytest.mark.parametrize("prec", ["mixed_fp32", "mixed_tf32", "mixed_bf16"])
@pytest.mark.parametrize("name,mk,rt,mu,rh", CASES, ids=[c[0] for c in CASES])
def test_mixed_form_matches_oracle(name, mk, rt, mu, rh, prec):
    from paper_2407_14013_gb300 import NewtonSolver
    prob = mk()
    V_top = prob.meta.get("U") if prob.kind == "dense" else None
    sp = W.scaling_point(prob.n, rt, mu, 6100 + prob.n, V_top=V_top)
    Ct, bt = W.newton_rhs(prob.n, prob.m, 6200 + prob.n)
    s = NewtonSolver(prob, r_hat=rh, precision=prec)
    dX, dy, dS, info = s.solve(_t(sp.V), _t(sp.lam), _t(Ct), _t(bt))
    assert info.converged and info.r == rt
    dX, dy, dS = dX.cpu().numpy(), dy.cpu().numpy(), dS.cpu().numpy()
    s.close()
    rX, ry, rS = onewton.newton_direct(prob, (sp.V * sp.lam) @ sp.V.T, Ct, bt)
    e = {"dX": emax(dX, rX), "dy": emax(dy, ry), "dS": emax(dS, rS)}
    print(f"\n{name} {prec}: refine={info.refine_steps} inner_iters={info.pcg_iters} "
          f"rate={info.refine_rate:.2e} " + " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    for k, v in e.items():
        assert v <= TOL, (k, v)
    assert info.refine_steps >= 1 and 0.0 < info.refine_rate <= RATE[prec]

"""The allocation-free adjoint entry point (sdp_adjoint_dense_noalloc) against the Newton solve
and against the CPU oracle's A^T.

Callers that cannot call cudaMalloc (allocator callbacks, fully reserved device memory,
paths that must not hit out-of-memory) use this entry point; it keeps its scratch in a
fixed array inside the library.  Its output Y = A^T(y) must agree with what the regular
entry point produces: sdp_newton_solve returns dS = C~ - A^T(dy), so C~ - Y(dy) must equal
dS.  It is also compared entry by entry with the oracle's plain definition A^T(y) =
sum_i y_i A_i (oracle.operators.At_op, FP64 numpy), which shares no code with the library.
Two calls in a row are checked (the second one reuses the shared scratch array).
This file is collected last so that a run stopping at the first failure has run every
other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as oops

pytestmark = pytest.mark.gpu

TOL = 1e-8   # the relative tolerance of the other GPU parity tests


def test_noalloc_adjoint_matches_newton_solve_twice():
    import torch
    from paper_2407_14013_gb300 import NewtonSolver, native
    prob = W.sensing(30, 120, 2, 4711)
    sp = W.scaling_point(30, 2, 1e-4, 4712)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a_dev = t(prob.a_dense)
    stream = torch.cuda.current_stream().cuda_stream
    s = NewtonSolver(prob, r_hat=3)
    for call, seed in enumerate((4713, 4714)):
        Ct, bt = W.newton_rhs(30, 120, seed)
        dX, dy, dS, info = s.solve(t(sp.V), t(sp.lam), t(Ct), t(bt))
        assert info.converged
        Y = torch.full((30, 30), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = native.sdp_adjoint_dense_noalloc(a_dev.data_ptr(), 30, 120, dy.data_ptr(), Y.data_ptr(), stream)
        assert st == native.SDP_OK, f"call {call}: status {st}"
        ref = Ct - dS.cpu().numpy()                     # A^T(dy) from the regular entry point
        got = Y.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), f"call {call}"
        assert np.allclose(got, got.T, rtol=0, atol=0)
        # entry by entry against the oracle's definition, for the same dy
        orc = oops.At_op(prob, dy.cpu().numpy())
        assert np.abs(got - orc).max() <= 1e-12 * np.abs(orc).max(), f"call {call}"
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2407_14013_gb300 import native
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = native.sdp_adjoint_dense_noalloc(dummy.data_ptr(), 1024, 1, dummy.data_ptr(), dummy.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert st == native.SDP_EINVAL                       # n(n+1)/2 = 524800 > 524288: checked on the host

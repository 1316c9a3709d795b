"""The bounds-checked debug build (libwcipm_checked.so) on the GPU.

In that build every index that a gather or scatter of the sparse constraint operators (A(.) and
A^T(.) for SPARSE_COO, the position values, the CSR products of A^T(y)) takes from an index
table is compared with the length of the array it addresses before it is used.  Here:

  * the record and the report work: one check of an index outside its range (made by the
    library's self-test kernel, which addresses no memory) is reported once, with its index, and
    then cleared; an index inside the range is not reported;
  * the sparse Newton solves and a whole SDP solve of the SPARSE_COO parity cases, run through
    the checked build, see no index out of range, and give the default build's results.

The checked build runs in a child process (one library per process); the parent runs the
same cases through the default build and compares.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

# (name, problem, r_true, r_hat, precond_space): ragged n, several tiles of every kernel,
# repeated and shared positions, d < m and d > m, each preconditioner space
CASES = [
    ("completion8x8", lambda: W.completion(8, 8, 2, 0.4, 11), 2, 3, 0),
    ("random_sparse12", lambda: W.random_sparse(12, 30, 3, 12), 2, 4, 1),
    ("completion150x130", lambda: W.completion(150, 130, 3, 0.08, 21), 3, 3, 0),
    ("completion150x130_m", lambda: W.completion(150, 130, 3, 0.08, 21), 3, 3, 1),
    ("random_sparse257", lambda: W.random_sparse(257, 700, 4, 22), 3, 4, 2),
]


def _run_cases():
    """Every case through whichever library this process loaded: the Newton directions, one whole
    SDP solve, and the launch count of each."""
    import torch
    from paper_2407_14013_gb300 import NewtonSolver
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {}
    for name, mk, rt, rh, space in CASES:
        prob = mk()
        sp = W.scaling_point(prob.n, rt, 1e-3, 500 + prob.n)
        Ct, bt = W.newton_rhs(prob.n, prob.m, 600 + prob.n)
        s = NewtonSolver(prob, r_hat=rh, precond_space=space)
        dX, dy, dS, info = s.solve(t(sp.V), t(sp.lam), t(Ct), t(bt))
        assert info.converged, name
        out[name + "/dX"], out[name + "/dy"], out[name + "/dS"] = dX.cpu().numpy(), dy.cpu().numpy(), dS.cpu().numpy()
        s.close()
    prob = W.random_sparse(12, 30, 3, 12)
    s = NewtonSolver(prob, r_hat=4)
    X, y, S, info = s.solve_sdp(t(prob.b), t(prob.C), gap_tol=1e-8, max_iter=100)
    assert info["converged"] == 1, info
    out["sdp/X"], out["sdp/y"], out["sdp/S"] = X.cpu().numpy(), y.cpu().numpy(), S.cpu().numpy()
    s.close()
    torch.cuda.synchronize()
    return out


def _child(path: str) -> None:
    """Runs in the child process: loads the checked build first, then checks the record and the
    report, then runs the cases and saves their outputs with the report that follows them."""
    import torch
    from paper_2407_14013_gb300 import _native as nat
    nat.load(nat.LIB_CHECKED_PATH)
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    rec = []
    rec.append(nat.sdp_bounds_report())                       # start clean
    rec.append((nat.sdp_bounds_selftest(stream, 3, 10),) + nat.sdp_bounds_report())
    rec.append((nat.sdp_bounds_selftest(stream, -1, 10),) + nat.sdp_bounds_report())
    rec.append(nat.sdp_bounds_report())                       # cleared by the previous report
    rec.append((nat.sdp_bounds_selftest(stream, 10, 10),) + nat.sdp_bounds_report())
    out = _run_cases()
    final = nat.sdp_bounds_report()
    np.savez(path, rec=np.array([list(r) + [0] * (4 - len(r)) for r in rec], dtype=np.uint64),
             final=np.array(final, dtype=np.uint64), **out)


def test_checked_build_reports_nothing_and_matches_default_build(tmp_path):
    from paper_2407_14013_gb300 import _native as nat
    assert os.path.exists(nat.LIB_CHECKED_PATH), "the checked build is made by __graft_entry__.build()"
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--child", path], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    got = np.load(path)
    rec = got["rec"].astype(np.int64)
    SITE = 1 << 48
    assert tuple(rec[0][:3]) == (nat.SDP_OK, 0, 0)
    assert tuple(rec[1][:4]) == (nat.SDP_OK, nat.SDP_OK, 0, 0)             # 3 in [0, 10): nothing
    st, rst, first, count = (int(v) for v in got["rec"][2])
    assert st == nat.SDP_OK and rst == nat.SDP_EINVAL and count == 1         # -1: one violation
    assert first % SITE == SITE - 1 and first // SITE >= 1                   # index -1 mod 2^48, a site
    assert tuple(rec[3][:3]) == (nat.SDP_OK, 0, 0)                            # cleared
    st, rst, first, count = (int(v) for v in got["rec"][4])
    assert (st, rst, count) == (nat.SDP_OK, nat.SDP_EINVAL, 1) and first % SITE == 10   # the bound itself
    # the cases: no index out of range anywhere
    assert tuple(int(v) for v in got["final"]) == (nat.SDP_OK, 0, 0)
    # the default build (this process) gives the same results
    ref = _run_cases()
    assert nat.sdp_bounds_report()[0] == nat.SDP_EUNSUPPORTED               # the default build has no checks
    for k, v in ref.items():
        g = got[k]
        assert g.shape == v.shape, k
        assert np.isfinite(g).all(), k
        assert np.abs(g - v).max() <= 1e-12 * max(np.abs(v).max(), 1e-300), k


if __name__ == "__main__" and len(sys.argv) == 3 and sys.argv[1] == "--child":
    _child(sys.argv[2])

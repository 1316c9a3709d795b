"""GB300 (sm_103a) inner Newton solve of a well-conditioned primal-dual IPM for low-rank SDP.

Chiu & Zhang, arXiv 2407.14013: the Newton system (Newt-eps) is solved through
the augmented system eq. augsys with the indefinite preconditioned PCG of
Cor. pcg and recovered with eq. recover.  All arithmetic runs in the CUDA
library (``libwcipm.so``, C ABI in ``include/wcipm.h``); this module only
moves torch device tensors across that boundary.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

from . import _native as native
from ._native import (SDP_A_DENSE_SVEC, SDP_A_DIAG, SDP_A_SPARSE_COO, SDP_ENOTCONV, SDP_FP64, SDP_MIXED_BF16,
                      SDP_MIXED_FP32, SDP_MIXED_TF32, SDP_OK, SdpError, sdp_default_options)

__all__ = ["NewtonSolver", "SdpError", "native", "sdp_optimum", "sdp_optimum_at", "eigh", "solve_sdp_batch", "SDP_A_DIAG", "SDP_A_SPARSE_COO",
           "SDP_A_DENSE_SVEC"]

KINDS = {"diag": SDP_A_DIAG, "sparse": SDP_A_SPARSE_COO, "dense": SDP_A_DENSE_SVEC}
PRECISIONS = {"fp64": SDP_FP64, "mixed_fp32": SDP_MIXED_FP32, "mixed_tf32": SDP_MIXED_TF32,
              "mixed_bf16": SDP_MIXED_BF16}
# refinement defaults of the mixed forms: each correction solve is taken about as far as the
# precision of its operator carries it (BF16 ~ 4e-3; split TF32 and FP32 ~ 1e-7 relative)
MIXED_DEFAULTS = {"mixed_fp32": (10, 1e-6), "mixed_tf32": (10, 1e-6), "mixed_bf16": (30, 1e-2)}


@dataclass
class NewtonInfo:
    r: int
    d: int
    pcg_iters: int
    space: int
    converged: bool
    tau: float
    beta: float
    res_norm: float
    rhs_norm: float
    res0_norm: float
    s_A: float
    status: int
    launches: int
    setup_ms: float = 0.0
    pcg_ms: float = 0.0
    recover_ms: float = 0.0
    prof_At_ms: float = 0.0
    prof_A_ms: float = 0.0
    prof_At_launches: int = 0
    prof_A_launches: int = 0
    refine_steps: int = 0
    prof_At32_ms: float = 0.0
    prof_A32_ms: float = 0.0
    prof_At32_launches: int = 0
    prof_A32_launches: int = 0
    refine_rate: float = 0.0


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _colmajor(V):
    """Storage of the matrix V in column-major order (the C ABI's layout), without a copy
    when V already is a transposed view of a contiguous tensor."""
    if V.t().is_contiguous():
        return V
    return V.t().contiguous().t()


class NewtonSolver:
    """Owns one library handle: problem data on the GPU plus the solve workspace.

    ``prob`` is any object with ``kind`` ("diag" | "sparse" | "dense"), ``n``, ``m``
    and the matching arrays (``a_dense`` m x n(n+1)/2; ``a_con``, ``a_row``,
    ``a_col``, ``a_val``), as numpy arrays or torch tensors.
    """

    def __init__(self, prob, r_fixed: int = 0, r_hat: int = 10, precond_space: int = 0,
                 max_pcg: int = 2000, check_every: int = 8, beta_rule: int = 0,
                 newton_rtol: float = 1e-12, device: str = "cuda", stream=None, use_graph: bool = True,
                 precision: str = "fp64", max_refine: Optional[int] = None, max_inner: int = 500,
                 inner_rtol: Optional[float] = None,
                 pcg_start: int = 0, tc_products: bool = True, krylov: str = "pcg", int_passes: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        f64 = torch.float64

        def dev(a, dtype):
            if a is None:
                return None
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(a)
            return t.to(device=self.device, dtype=dtype).contiguous()

        self.kind = KINDS[prob.kind] if isinstance(prob.kind, str) else int(prob.kind)
        self.n, self.m = int(prob.n), int(prob.m)
        self._keep = {
            "a_dense": dev(getattr(prob, "a_dense", None), f64),
            "a_con": dev(getattr(prob, "a_con", None), torch.int32),
            "a_row": dev(getattr(prob, "a_row", None), torch.int32),
            "a_col": dev(getattr(prob, "a_col", None), torch.int32),
            "a_val": dev(getattr(prob, "a_val", None), f64),
        }
        k = self._keep
        p = native.sdp_problem()
        p.n, p.m, p.kind = self.n, self.m, self.kind
        p.nnz = 0 if k["a_val"] is None else int(k["a_val"].numel())
        p.a_con, p.a_row, p.a_col, p.a_val = _ptr(k["a_con"]), _ptr(k["a_row"]), _ptr(k["a_col"]), _ptr(k["a_val"])
        p.a_dense = _ptr(k["a_dense"])
        o = sdp_default_options()
        o.r_fixed, o.r_hat, o.precond_space = r_fixed, r_hat, precond_space
        o.max_pcg, o.check_every, o.beta_rule = max_pcg, check_every, beta_rule
        o.newton_rtol = newton_rtol
        o.use_graph = 1 if use_graph else 0
        o.precision = PRECISIONS[precision]
        dr, dt = MIXED_DEFAULTS.get(precision, (10, 1e-6))
        o.max_refine = dr if max_refine is None else max_refine
        o.max_inner = max_inner
        o.inner_rtol = dt if inner_rtol is None else inner_rtol
        o.pcg_start = pcg_start
        o.tc_products = 1 if tc_products else 0
        o.krylov = {"pcg": 0, "minres": 1}[krylov]
        o.int_passes = 1 if int_passes else 0
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        torch.cuda.synchronize(self.device)
        self.handle = native.sdp_setup(p, o, int(self.stream.cuda_stream))
        self.last_info: Optional[NewtonInfo] = None

    def debug_buffer(self, which: int, count: int):
        """Copy of an internal buffer of the last solve (see sdp_debug_copy)."""
        t = self.torch.empty(count, dtype=self.torch.float64, device=self.device)
        native.sdp_debug_copy(self.handle, which, _ptr(t), count)
        return t

    def set_profiling(self, on: bool = True) -> None:
        """CUDA-event timing of every pass over the dense constraint matrix."""
        native.sdp_set_profiling(self.handle, on)

    def workspace_bytes(self) -> int:
        return native.sdp_workspace_bytes(self.handle)

    def apply(self, vec, which: int = 0, out=None):
        """M vec (which 0: the augmented operator of eq. augsys) or P^{-1} vec (which 1: the
        preconditioner) at the scaling point of the last solve; vec is a device FP64 vector of
        m + d entries ([u; v], v in h-coordinates)."""
        torch = self.torch
        if vec.dtype != torch.float64 or not vec.is_contiguous() or vec.device != self.device:
            raise ValueError("vec must be a contiguous float64 tensor on the solver's device")
        if out is None:
            out = torch.empty_like(vec)
        cur = torch.cuda.current_stream(self.device)
        if self.stream.cuda_stream != cur.cuda_stream:     # vec is complete before the handle's stream reads it
            self.stream.wait_stream(cur)
        native.sdp_apply_augsys(self.handle, _ptr(vec), _ptr(out), which)   # enqueued on self.stream
        if self.stream.cuda_stream != cur.cuda_stream:     # later work on the current stream sees out
            cur.wait_stream(self.stream)
        return out

    def _info(self, ci, st) -> NewtonInfo:
        return NewtonInfo(r=ci.r, d=ci.d, pcg_iters=ci.pcg_iters, space=ci.space, converged=bool(ci.converged),
                          tau=ci.tau, beta=ci.beta, res_norm=ci.res_norm, rhs_norm=ci.rhs_norm, res0_norm=ci.res0_norm, s_A=ci.s_A,
                          status=st, launches=native.sdp_last_launch_count(self.handle),
                          setup_ms=ci.setup_ms, pcg_ms=ci.pcg_ms, recover_ms=ci.recover_ms,
                          prof_At_ms=ci.prof_At_ms, prof_A_ms=ci.prof_A_ms,
                          prof_At_launches=ci.prof_At_launches, prof_A_launches=ci.prof_A_launches,
                          refine_steps=ci.refine_steps, prof_At32_ms=ci.prof_At32_ms, prof_A32_ms=ci.prof_A32_ms,
                          prof_At32_launches=ci.prof_At32_launches, prof_A32_launches=ci.prof_A32_launches,
                          refine_rate=ci.refine_rate)

    def solve(self, V, lam, Ct, bt, out=None, allow_notconv: bool = False):
        """Newton direction (dX, dy, dS) of (Newt-eps) for W = V diag(lam) V^T; device tensors.

        V may have any strides (it is passed column-major, copied only if needed); Ct is
        symmetric, so its layout does not matter."""
        torch = self.torch
        n, m = self.n, self.m
        f64 = torch.float64
        lam, Ct, bt = (t.to(device=self.device, dtype=f64).contiguous() for t in (lam, Ct, bt))
        V = _colmajor(V.to(device=self.device, dtype=f64))
        if out is None:
            out = (torch.empty((n, n), dtype=f64, device=self.device), torch.empty(m, dtype=f64, device=self.device),
                   torch.empty((n, n), dtype=f64, device=self.device))
        dX, dy, dS = out
        ci = native.sdp_newton_info()
        st = native.sdp_newton_solve(self.handle, _ptr(V), _ptr(lam), _ptr(Ct), _ptr(bt), _ptr(dX), _ptr(dy),
                                     _ptr(dS), ci, allow_notconv=allow_notconv)
        self.last_info = self._info(ci, st)
        return dX, dy, dS, self.last_info

    def resolve(self, Ct, bt, out=None, allow_notconv: bool = False):
        """Another right side at the scaling point of the last solve (sdp_newton_resolve)."""
        torch = self.torch
        n, m = self.n, self.m
        f64 = torch.float64
        Ct, bt = (t.to(device=self.device, dtype=f64).contiguous() for t in (Ct, bt))
        if out is None:
            out = (torch.empty((n, n), dtype=f64, device=self.device), torch.empty(m, dtype=f64, device=self.device),
                   torch.empty((n, n), dtype=f64, device=self.device))
        dX, dy, dS = out
        ci = native.sdp_newton_info()
        st = native.sdp_newton_resolve(self.handle, _ptr(Ct), _ptr(bt), _ptr(dX), _ptr(dy), _ptr(dS), ci,
                                       allow_notconv=allow_notconv)
        self.last_info = self._info(ci, st)
        return dX, dy, dS, self.last_info

    def solve_host(self, V, lam, Ct, bt, out, allow_notconv: bool = False):
        """Same solve with host (CPU, ideally pinned) tensors; copies are inside the call.
        V must already be stored column-major (e.g. ``V.t().contiguous().t()``), so that
        no host-side copy is hidden in the call."""
        if not V.t().is_contiguous():
            raise ValueError("solve_host needs V stored column-major")
        dX, dy, dS = out
        ci = native.sdp_newton_info()
        st = native.sdp_newton_solve_host(self.handle, _ptr(V), _ptr(lam), _ptr(Ct), _ptr(bt), _ptr(dX), _ptr(dy),
                                          _ptr(dS), ci, allow_notconv=allow_notconv)
        self.last_info = self._info(ci, st)
        return dX, dy, dS, self.last_info

    def grad(self, V, lam, gX, gy, allow_notconv: bool = False):
        """Cotangents (gC, gb) of the data for cotangents (gX, gy) of the optimum (X, y), by
        implicit differentiation at the scaling point W = V diag(lam) V^T (sdp_grad)."""
        torch = self.torch
        n, m = self.n, self.m
        f64 = torch.float64
        lam, gX, gy = (t.to(device=self.device, dtype=f64).contiguous() for t in (lam, gX, gy))
        V = _colmajor(V.to(device=self.device, dtype=f64))
        gC = torch.empty((n, n), dtype=f64, device=self.device)
        gb = torch.empty(m, dtype=f64, device=self.device)
        ci = native.sdp_newton_info()
        st = native.sdp_grad(self.handle, _ptr(V), _ptr(lam), _ptr(gX), _ptr(gy), _ptr(gC), _ptr(gb), ci,
                             allow_notconv=allow_notconv)
        self.last_info = self._info(ci, st)
        return gC, gb

    def grad_slack(self, V, lam, dv, dw, gX, gy, gv, gw, allow_notconv: bool = False):
        """Cotangents (gC, gb, gcv, gcw) of the data of the robust form with slacks (eq. rmc-sdp)
        for cotangents (gX, gy, gv, gw) of its optimum (X, y, v, w), at the scaling point
        W = V diag(lam) V^T, d_v = v / zv, d_w = w / zw (sdp_grad_slack)."""
        torch = self.torch
        n, m = self.n, self.m
        f64 = torch.float64
        lam, dv, dw, gX, gy, gv, gw = (t.to(device=self.device, dtype=f64).contiguous()
                                       for t in (lam, dv, dw, gX, gy, gv, gw))
        V = _colmajor(V.to(device=self.device, dtype=f64))
        gC = torch.empty((n, n), dtype=f64, device=self.device)
        gb, gcv, gcw = (torch.empty(m, dtype=f64, device=self.device) for _ in range(3))
        ci = native.sdp_newton_info()
        st = native.sdp_grad_slack(self.handle, [_ptr(t) for t in (V, lam, dv, dw, gX, gy, gv, gw, gC, gb, gcv, gcw)],
                                   ci, allow_notconv=allow_notconv)
        self.last_info = self._info(ci, st)
        return gC, gb, gcv, gcw

    def ipm_step(self, b, C, X, y, S):
        """One outer interior-point iteration in place on the device tensors X, y, S (ipm_step)."""
        torch = self.torch
        f64 = torch.float64
        b, C = (t.to(device=self.device, dtype=f64).contiguous() for t in (b, C))
        for t in (X, y, S):
            if t.dtype != f64 or t.device != self.device or not t.is_contiguous():
                raise ValueError("X, y, S must be contiguous float64 tensors on the solver's device")
        ci = native.sdp_ipm_info()
        native.ipm_step(self.handle, _ptr(b), _ptr(C), _ptr(X), _ptr(y), _ptr(S), ci)
        return ci.as_dict()

    def solve_sdp(self, b, C, gap_tol: float = 1e-8, max_iter: int = 100, allow_notconv: bool = False):
        """Whole interior-point solve of min <C,X> s.t. A(X) = b, X PSD (sdp_solve); returns
        (X, y, S, info)."""
        torch = self.torch
        f64 = torch.float64
        n, m = self.n, self.m
        b, C = (t.to(device=self.device, dtype=f64).contiguous() for t in (b, C))
        X = torch.empty((n, n), dtype=f64, device=self.device)
        S = torch.empty((n, n), dtype=f64, device=self.device)
        y = torch.empty(m, dtype=f64, device=self.device)
        ci = native.sdp_ipm_info()
        st = native.sdp_solve(self.handle, _ptr(b), _ptr(C), _ptr(X), _ptr(y), _ptr(S), gap_tol, max_iter, ci,
                              allow_notconv=allow_notconv)
        info = ci.as_dict()
        info["status"] = st
        return X, y, S, info

    def solve_slack(self, b, C, cv, cw, gap_tol: float = 1e-8, max_iter: int = 100, allow_notconv: bool = False):
        """Whole solve of min <C,X> + cv^T v + cw^T w s.t. A(X) + v - w = b, X PSD, v, w >= 0 (the
        robust form of Section 7, sdp_solve_slack); returns (X, y, S, v, w, zv, zw, info)."""
        torch = self.torch
        f64 = torch.float64
        n, m = self.n, self.m
        b, C, cv, cw = (t.to(device=self.device, dtype=f64).contiguous() for t in (b, C, cv, cw))
        X = torch.empty((n, n), dtype=f64, device=self.device)
        S = torch.empty((n, n), dtype=f64, device=self.device)
        y, v, w, zv, zw = (torch.empty(m, dtype=f64, device=self.device) for _ in range(5))
        ci = native.sdp_ipm_info()
        st = native.sdp_solve_slack(self.handle, [_ptr(t) for t in (b, C, cv, cw, X, y, S, v, w, zv, zw)], gap_tol,
                                    max_iter, ci, allow_notconv=allow_notconv)
        info = ci.as_dict()
        info["status"] = st
        return X, y, S, v, w, zv, zw, info

    def center(self, b, C, X, y, S, mu: float, tol: float = 1e-10, max_iter: int = 50, allow_notconv: bool = False):
        """Newton steps towards the central-path point of parameter mu, in place on the device
        tensors X, y, S (sdp_center); returns the info dict (info["sigma"]: final centrality)."""
        torch = self.torch
        f64 = torch.float64
        b, C = (t.to(device=self.device, dtype=f64).contiguous() for t in (b, C))
        for t in (X, y, S):
            if t.dtype != f64 or t.device != self.device or not t.is_contiguous():
                raise ValueError("X, y, S must be contiguous float64 tensors on the solver's device")
        ci = native.sdp_ipm_info()
        st = native.sdp_center(self.handle, _ptr(b), _ptr(C), _ptr(X), _ptr(y), _ptr(S), mu, tol, max_iter, ci,
                               allow_notconv=allow_notconv)
        info = ci.as_dict()
        info["status"] = st
        return info

    def set_linear_diag(self, delta=None):
        """Nonnegative variables entering the constraints (sdp_set_linear_diag): every later solve
        adds diag(delta) to the Schur matrix, delta = diag(G D G^T) >= 0 (m values).  The caller
        folds G D c~ into b~ and forms dx = D(G^T dy - c~).  None removes the block."""
        torch = self.torch
        if delta is None:
            self._lin = None
            native.sdp_set_linear_diag(self.handle, 0)
            return
        t = delta if isinstance(delta, torch.Tensor) else torch.from_numpy(delta)
        self._lin = t.to(device=self.device, dtype=torch.float64).contiguous()
        native.sdp_set_linear_diag(self.handle, _ptr(self._lin))

    def scaling_point(self, X, S):
        """Eigen-decomposition (V, lam) of the NT scaling point of (X, S) (sdp_scaling_point), the
        input that solve() and grad() take."""
        torch = self.torch
        X = X.to(device=self.device, dtype=torch.float64).contiguous()
        S = S.to(device=self.device, dtype=torch.float64).contiguous()
        Vbuf = torch.empty((self.n, self.n), dtype=torch.float64, device=self.device)
        lam = torch.empty(self.n, dtype=torch.float64, device=self.device)
        native.sdp_scaling_point(self.handle, _ptr(X), _ptr(S), _ptr(Vbuf), _ptr(lam))
        return Vbuf.t(), lam          # column-major storage: V[i, j] = Vbuf[j, i]

    def close(self):
        if getattr(self, "handle", None):
            native.sdp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_sdp_batch(solvers, bs, Cs, gap_tol: float = 1e-8, max_iter: int = 100, workers: int = 0):
    """Whole interior-point solves of many independent problems at once (sdp_solve_batch):
    instance i on solvers[i] with data (bs[i], Cs[i]).  Give each solver its own stream
    (``NewtonSolver(..., stream=torch.cuda.Stream())``) for the solves to overlap on the GPU.
    Returns a list of (X, y, S, info) with info["status"] the instance's status code."""
    import torch
    f64 = torch.float64
    outs, keep = [], []
    for s_, b_, C_ in zip(solvers, bs, Cs):
        b_ = b_.to(device=s_.device, dtype=f64).contiguous()
        C_ = C_.to(device=s_.device, dtype=f64).contiguous()
        X = torch.empty((s_.n, s_.n), dtype=f64, device=s_.device)
        S = torch.empty((s_.n, s_.n), dtype=f64, device=s_.device)
        y = torch.empty(s_.m, dtype=f64, device=s_.device)
        keep.append((b_, C_))
        outs.append((X, y, S))
    for s_ in solvers:
        torch.cuda.synchronize(s_.device)
    statuses, infos = native.sdp_solve_batch([s_.handle for s_ in solvers], [_ptr(k[0]) for k in keep],
                                             [_ptr(k[1]) for k in keep], [_ptr(o[0]) for o in outs],
                                             [_ptr(o[1]) for o in outs], [_ptr(o[2]) for o in outs],
                                             gap_tol, max_iter, workers)
    res = []
    for (X, y, S), st, ci in zip(outs, statuses, infos):
        info = ci.as_dict()
        info["status"] = st
        res.append((X, y, S, info))
    return res


def sdp_optimum(C, b, solver: NewtonSolver, gap_tol: float = 1e-8, max_iter: int = 100, center_mu=None,
                center_tol: float = 1e-10, center_iters: int = 50):
    """Differentiable SDP layer: (X, y) = argmin <C,X> s.t. A(X) = b, X PSD (and its dual y) as a
    function of (C, b), for the constraint operator held by ``solver``.

    Forward: one device interior-point solve (sdp_solve) to ``gap_tol``, then centring steps at
    the final mu (or ``center_mu``) so that the derivative below is that of a central-path
    point (sdp_center), then the NT scaling point of the result (sdp_scaling_point).  Only the
    final (X, y, S) and the eigen-decomposition (V, lam) of its scaling point are kept.
    Backward: one sdp_grad call, the Newton system of the reformulation at that point used as
    the adjoint: (gC, gb) = K^{-1} [sym gX; gy].  The result differs from the derivative of the
    optimum by O(mu)."""
    import torch

    class _SdpOptimum(torch.autograd.Function):
        @staticmethod
        def forward(ctx, C_, b_):
            X, y, S, info = solver.solve_sdp(b_.detach(), C_.detach(), gap_tol=gap_tol, max_iter=max_iter)
            mu = float(info["mu"]) if center_mu is None else float(center_mu)
            solver.center(b_.detach(), C_.detach(), X, y, S, mu, tol=center_tol, max_iter=center_iters,
                          allow_notconv=True)
            V, lam = solver.scaling_point(X, S)
            ctx.save_for_backward(X, y, S, V, lam)
            ctx.mu = mu
            return X.to(C_.dtype), y.to(b_.dtype)

        @staticmethod
        def backward(ctx, gX, gy):
            X, y, S, V, lam = ctx.saved_tensors
            if gX is None:
                gX = torch.zeros((solver.n, solver.n), dtype=torch.float64, device=solver.device)
            if gy is None:
                gy = torch.zeros(solver.m, dtype=torch.float64, device=solver.device)
            gC, gb = solver.grad(V, lam, gX, gy)
            return gC.to(C.dtype), gb.to(b.dtype)

    return _SdpOptimum.apply(C, b)


def sdp_optimum_at(C, b, X, y, V, lam, solver: NewtonSolver):
    """(X, y) of an iterate the caller already holds, with (V, lam) the eigen-decomposition of
    its NT scaling point, made differentiable with respect to (C, b) by the same sdp_grad
    backward as sdp_optimum (no solve in the forward pass)."""
    import torch

    class _SdpAt(torch.autograd.Function):
        @staticmethod
        def forward(ctx, C_, b_, X_, y_, V_, lam_):
            ctx.save_for_backward(V_, lam_)
            return X_.clone(), y_.clone()

        @staticmethod
        def backward(ctx, gX, gy):
            V_, lam_ = ctx.saved_tensors
            if gX is None:
                gX = torch.zeros((solver.n, solver.n), dtype=torch.float64, device=solver.device)
            if gy is None:
                gy = torch.zeros(solver.m, dtype=torch.float64, device=solver.device)
            gC, gb = solver.grad(V_, lam_, gX, gy)
            return gC.to(C.dtype), gb.to(b.dtype), None, None, None, None

    return _SdpAt.apply(C, b, X.detach(), y.detach(), V.detach(), lam.detach())


def eigh(A, tol: float = 1e-14, max_sweeps: int = 40):
    """Symmetric eigen-decomposition of the device matrix A by the library's Jacobi solver
    (sdp_eigh); returns (lam, V, sweeps) with A = V diag(lam) V^T, lam unsorted."""
    import torch
    n = A.shape[0]
    A = A.to(dtype=torch.float64).t().contiguous().t().clone()
    V = torch.empty_like(A)
    lam = torch.empty(n, dtype=torch.float64, device=A.device)
    work = torch.empty(native.sdp_eigh_work_elems(n), dtype=torch.float64, device=A.device)
    stream = torch.cuda.current_stream(A.device)
    st, sweeps = native.sdp_eigh(int(stream.cuda_stream), n, _ptr(A), _ptr(V), _ptr(lam), tol, max_sweeps,
                                 _ptr(work), work.numel())
    if st != SDP_OK:
        raise SdpError(st, "Jacobi eigensolver did not converge")
    return lam, V, sweeps

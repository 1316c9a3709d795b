"""ctypes binding of the C ABI in include/wcipm.h (argument marshalling only).

Every function here forwards to the CUDA library ``libwcipm.so`` built next to
this file; there is no Python or CPU implementation of any step.  Loading fails
loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwcipm.so")
# the bounds-checked debug build (same exports; its sparse-operator gathers and scatters check
# every table index, see sdp_bounds_report): load(LIB_CHECKED_PATH) before any other call
LIB_CHECKED_PATH = os.path.join(HERE, "libwcipm_checked.so")

SDP_OK, SDP_EINVAL, SDP_ENOMEM, SDP_ECUDA, SDP_ENOTCONV, SDP_ENUMERIC, SDP_ETIMEOUT, SDP_EUNSUPPORTED = range(8)
STATUS_NAMES = ["SDP_OK", "SDP_EINVAL", "SDP_ENOMEM", "SDP_ECUDA", "SDP_ENOTCONV", "SDP_ENUMERIC",
                "SDP_ETIMEOUT", "SDP_EUNSUPPORTED"]
SDP_A_DIAG, SDP_A_SPARSE_COO, SDP_A_DENSE_SVEC = 0, 1, 2
SDP_FP64, SDP_MIXED_FP32, SDP_MIXED_TF32, SDP_MIXED_BF16 = 0, 1, 2, 3


class sdp_problem(Structure):
    _fields_ = [("n", c_int32), ("m", c_int32), ("kind", c_int32), ("pad_", c_int32), ("nnz", c_int64),
                ("a_con", c_void_p), ("a_row", c_void_p), ("a_col", c_void_p), ("a_val", c_void_p),
                ("a_dense", c_void_p)]


class sdp_options(Structure):
    _fields_ = [("r_fixed", c_int32), ("r_hat", c_int32), ("precision", c_int32), ("precond_space", c_int32),
                ("max_pcg", c_int32), ("check_every", c_int32), ("beta_rule", c_int32), ("use_graph", c_int32),
                ("newton_rtol", c_double), ("max_refine", c_int32), ("max_inner", c_int32),
                ("inner_rtol", c_double), ("pcg_start", c_int32), ("tc_products", c_int32),
                ("krylov", c_int32), ("int_passes", c_int32)]


class sdp_newton_info(Structure):
    _fields_ = [("r", c_int32), ("d", c_int32), ("pcg_iters", c_int32), ("space", c_int32),
                ("converged", c_int32), ("refine_steps", c_int32), ("tau", c_double), ("beta", c_double),
                ("res_norm", c_double), ("rhs_norm", c_double), ("res0_norm", c_double), ("s_A", c_double),
                ("setup_ms", c_double), ("pcg_ms", c_double), ("recover_ms", c_double),
                ("prof_At_ms", c_double), ("prof_A_ms", c_double),
                ("prof_At_launches", c_int32), ("prof_A_launches", c_int32),
                ("prof_At32_ms", c_double), ("prof_A32_ms", c_double),
                ("prof_At32_launches", c_int32), ("prof_A32_launches", c_int32), ("refine_rate", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class sdp_ipm_info(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("converged", c_int32), ("pcg_iters", c_int32), ("eig_sweeps", c_int32),
                ("newton_inexact", c_int32), ("pad_", c_int32), ("pobj", c_double), ("dobj", c_double), ("rel_gap", c_double), ("pinf", c_double),
                ("dinf", c_double), ("mu", c_double), ("alpha_p", c_double), ("alpha_d", c_double),
                ("sigma", c_double), ("newton_ms", c_double), ("total_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


EXPORTS = {
    "sdp_default_options": (None, [POINTER(sdp_options)]),
    "sdp_set_linear_diag": (c_int32, [c_void_p, c_void_p]),
    "sdp_solve_slack": (c_int32, [c_void_p] + [c_void_p] * 11 + [c_double, c_int32, POINTER(sdp_ipm_info)]),
    "sdp_setup": (c_int32, [POINTER(sdp_problem), POINTER(sdp_options), c_void_p, POINTER(c_void_p)]),
    "sdp_newton_solve": (c_int32, [c_void_p] + [c_void_p] * 7 + [POINTER(sdp_newton_info)]),
    "sdp_newton_solve_host": (c_int32, [c_void_p] + [c_void_p] * 7 + [POINTER(sdp_newton_info)]),
    "sdp_grad": (c_int32, [c_void_p] + [c_void_p] * 6 + [POINTER(sdp_newton_info)]),
    "sdp_grad_slack": (c_int32, [c_void_p] + [c_void_p] * 12 + [POINTER(sdp_newton_info)]),
    "sdp_newton_resolve": (c_int32, [c_void_p] + [c_void_p] * 5 + [POINTER(sdp_newton_info)]),
    "sdp_eigh_work_elems": (c_int64, [c_int32]),
    "sdp_eigh": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_double, c_int32, c_void_p, c_int64,
                           POINTER(c_int32)]),
    "ipm_step": (c_int32, [c_void_p] + [c_void_p] * 5 + [POINTER(sdp_ipm_info)]),
    "sdp_solve": (c_int32, [c_void_p] + [c_void_p] * 5 + [c_double, c_int32, POINTER(sdp_ipm_info)]),
    "sdp_scaling_point": (c_int32, [c_void_p] * 5),
    "sdp_center": (c_int32, [c_void_p] + [c_void_p] * 5 + [c_double, c_double, c_int32, POINTER(sdp_ipm_info)]),
    "sdp_solve_batch": (c_int32, [c_int32] + [c_void_p] * 6 + [c_double, c_int32, c_int32, c_void_p, c_void_p]),
    "sdp_gemm_f64_tc_work_bytes": (c_size_t, [c_int32, c_int32, c_int32]),
    "sdp_gemm_f64_tc": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_double, c_void_p, c_int64,
                                  c_void_p, c_int64, c_double, c_void_p, c_int64, c_void_p, c_size_t]),
    "sdp_gemm_tn_lp": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, ctypes.c_float, c_void_p, c_int64,
                                 c_void_p, c_int64, c_void_p, c_int64, c_void_p]),
    "sdp_spd_inverse_work_bytes": (c_size_t, [c_int32]),
    "sdp_spd_inverse": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_size_t]),
    "sdp_debug_copy": (c_int32, [c_void_p, c_int32, c_void_p, c_int64]),
    "sdp_set_profiling": (c_int32, [c_void_p, c_int32]),
    "sdp_adjoint_dense_noalloc": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "sdp_set_tc_wait_limit_ns": (None, [ctypes.c_uint64]),
    "sdp_apply_augsys": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "sdp_bounds_report": (c_int32, [POINTER(ctypes.c_uint64), POINTER(ctypes.c_uint64)]),
    "sdp_bounds_selftest": (c_int32, [c_void_p, c_int64, c_int64]),
    "sdp_workspace_bytes": (c_size_t, [c_void_p]),
    "sdp_last_launch_count": (c_int64, [c_void_p]),
    "sdp_last_error": (c_char_p, [c_void_p]),
    "sdp_destroy": (None, [c_void_p]),
}

_lib = None
_lib_path = None


def load(path: str | None = None):
    """Load the library (libwcipm.so unless path names another build) and declare every exported
    symbol; raises if it is missing, or if path names a build other than the one already loaded."""
    global _lib, _lib_path
    if _lib is not None:
        if path is not None and os.path.abspath(path) != _lib_path:
            raise RuntimeError(f"{_lib_path} is already loaded in this process; {path} cannot be")
        return _lib
    path = os.path.abspath(path or LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib, _lib_path = lib, path
    return lib


class SdpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def sdp_default_options() -> sdp_options:
    o = sdp_options()
    load().sdp_default_options(ctypes.byref(o))
    return o


def sdp_setup(prob: sdp_problem, opt: sdp_options, stream: int) -> int:
    lib = load()
    h = c_void_p()
    st = lib.sdp_setup(ctypes.byref(prob), ctypes.byref(opt), c_void_p(stream), ctypes.byref(h))
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(None).decode())
    return h.value


def _solve(fn_name: str, h: int, ptrs, info: sdp_newton_info, allow_notconv: bool) -> int:
    lib = load()
    st = getattr(lib, fn_name)(c_void_p(h), *[c_void_p(p) for p in ptrs], ctypes.byref(info))
    if st != SDP_OK and not (allow_notconv and st == SDP_ENOTCONV):
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_newton_solve(h: int, V: int, lam: int, Ct: int, bt: int, dX: int, dy: int, dS: int,
                     info: sdp_newton_info, allow_notconv: bool = False) -> int:
    return _solve("sdp_newton_solve", h, (V, lam, Ct, bt, dX, dy, dS), info, allow_notconv)


def sdp_newton_solve_host(h: int, V: int, lam: int, Ct: int, bt: int, dX: int, dy: int, dS: int,
                          info: sdp_newton_info, allow_notconv: bool = False) -> int:
    return _solve("sdp_newton_solve_host", h, (V, lam, Ct, bt, dX, dy, dS), info, allow_notconv)


def sdp_newton_resolve(h: int, Ct: int, bt: int, dX: int, dy: int, dS: int, info: sdp_newton_info,
                       allow_notconv: bool = False) -> int:
    return _solve("sdp_newton_resolve", h, (Ct, bt, dX, dy, dS), info, allow_notconv)


def sdp_grad_slack(h: int, ptrs, info: sdp_newton_info, allow_notconv: bool = False) -> int:
    """sdp_grad_slack with ptrs = (V, lam, dv, dw, gX, gy, gv, gw, gC, gb, gcv, gcw) device pointers."""
    lib = load()
    st = lib.sdp_grad_slack(c_void_p(h), *[c_void_p(p) for p in ptrs], ctypes.byref(info))
    if st != SDP_OK and not (allow_notconv and st == SDP_ENOTCONV):
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_grad(h: int, V: int, lam: int, gX: int, gy: int, gC: int, gb: int, info: sdp_newton_info,
             allow_notconv: bool = False) -> int:
    return _solve("sdp_grad", h, (V, lam, gX, gy, gC, gb), info, allow_notconv)


def sdp_eigh(stream: int, n: int, A: int, V: int, lam: int, tol: float, max_sweeps: int, work: int,
             work_elems: int) -> tuple[int, int]:
    """Jacobi eigen-decomposition on the device; returns (status, sweeps)."""
    lib = load()
    sw = c_int32(0)
    st = lib.sdp_eigh(c_void_p(stream), n, c_void_p(A), c_void_p(V), c_void_p(lam), tol, max_sweeps,
                      c_void_p(work), work_elems, ctypes.byref(sw))
    if st not in (SDP_OK, SDP_ENOTCONV):
        raise SdpError(st, lib.sdp_last_error(None).decode())
    return st, sw.value


def sdp_eigh_work_elems(n: int) -> int:
    return int(load().sdp_eigh_work_elems(n))


def ipm_step(h: int, b: int, C: int, X: int, y: int, S: int, info: sdp_ipm_info) -> int:
    lib = load()
    st = lib.ipm_step(c_void_p(h), c_void_p(b), c_void_p(C), c_void_p(X), c_void_p(y), c_void_p(S),
                      ctypes.byref(info))
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_solve(h: int, b: int, C: int, X: int, y: int, S: int, gap_tol: float, max_iter: int,
              info: sdp_ipm_info, allow_notconv: bool = False) -> int:
    lib = load()
    st = lib.sdp_solve(c_void_p(h), c_void_p(b), c_void_p(C), c_void_p(X), c_void_p(y), c_void_p(S), gap_tol,
                       max_iter, ctypes.byref(info))
    if st != SDP_OK and not (allow_notconv and st == SDP_ENOTCONV):
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_solve_slack(h: int, ptrs, gap_tol: float, max_iter: int, info: sdp_ipm_info,
                    allow_notconv: bool = False) -> int:
    """sdp_solve_slack with ptrs = (b, C, cv, cw, X, y, S, v, w, zv, zw) device pointers."""
    lib = load()
    st = lib.sdp_solve_slack(c_void_p(h), *[c_void_p(p) for p in ptrs], gap_tol, max_iter, ctypes.byref(info))
    if st != SDP_OK and not (allow_notconv and st == SDP_ENOTCONV):
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_set_linear_diag(h: int, delta: int) -> None:
    """Linear block delta (device pointer to m doubles, or 0 to remove it)."""
    lib = load()
    st = lib.sdp_set_linear_diag(c_void_p(h), c_void_p(delta) if delta else None)
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(c_void_p(h) if h else None).decode())


def sdp_center(h: int, b: int, C: int, X: int, y: int, S: int, mu: float, tol: float, max_iter: int,
               info: sdp_ipm_info, allow_notconv: bool = False) -> int:
    lib = load()
    st = lib.sdp_center(c_void_p(h), c_void_p(b), c_void_p(C), c_void_p(X), c_void_p(y), c_void_p(S), mu, tol,
                        max_iter, ctypes.byref(info))
    if st != SDP_OK and not (allow_notconv and st == SDP_ENOTCONV):
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_scaling_point(h: int, X: int, S: int, V: int, lam: int) -> None:
    lib = load()
    st = lib.sdp_scaling_point(c_void_p(h), c_void_p(X), c_void_p(S), c_void_p(V), c_void_p(lam))
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())


def sdp_solve_batch(handles, b, C, X, y, S, gap_tol: float, max_iter: int, workers: int = 0):
    """sdp_solve_batch over lists of handles and device pointers; returns (statuses, infos)."""
    lib = load()
    k = len(handles)
    arr = lambda xs: (c_void_p * max(k, 1))(*[c_void_p(v) for v in xs])
    infos = (sdp_ipm_info * max(k, 1))()
    statuses = (c_int32 * max(k, 1))()
    st = lib.sdp_solve_batch(k, arr(handles), arr(b), arr(C), arr(X), arr(y), arr(S), gap_tol, max_iter, workers,
                             ctypes.cast(infos, c_void_p), ctypes.cast(statuses, c_void_p))
    if st == SDP_EINVAL and (k == 0 or all(v == SDP_EINVAL for v in statuses[:k])):
        raise SdpError(st, lib.sdp_last_error(None).decode())
    return [int(v) for v in statuses[:k]], [infos[i] for i in range(k)]


def sdp_gemm_f64_tc(stream: int, tA: bool, tB: bool, M: int, N: int, K: int, alpha: float, A: int, lda: int, B: int,
                    ldb: int, beta: float, C: int, ldc: int, work: int, work_bytes: int) -> None:
    lib = load()
    st = lib.sdp_gemm_f64_tc(c_void_p(stream), int(tA), int(tB), M, N, K, alpha, c_void_p(A), lda, c_void_p(B), ldb,
                             beta, c_void_p(C), ldc, c_void_p(work), work_bytes)
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(None).decode())


def sdp_gemm_tn_lp(stream: int, tf32: bool, M: int, N: int, K: int, alpha: float, A: int, lda: int, B: int, ldb: int,
                   C: int, ldc: int, err_word: int) -> None:
    lib = load()
    st = lib.sdp_gemm_tn_lp(c_void_p(stream), int(tf32), M, N, K, alpha, c_void_p(A), lda, c_void_p(B), ldb,
                            c_void_p(C), ldc, c_void_p(err_word))
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(None).decode())


def sdp_spd_inverse(stream: int, n: int, A: int, Linv: int, mode: int, coop: bool, work: int, work_bytes: int) -> None:
    """mode 0: A := A^{-1}; mode 1: A := L (A = L L^T), Linv := L^{-1} when non-zero (device pointers)."""
    lib = load()
    st = lib.sdp_spd_inverse(c_void_p(stream), n, c_void_p(A), c_void_p(Linv or None), mode, int(coop),
                             c_void_p(work), work_bytes)
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(None).decode())


def sdp_debug_copy(h: int, which: int, dst: int, count: int) -> None:
    lib = load()
    st = lib.sdp_debug_copy(c_void_p(h), which, c_void_p(dst), count)
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())


def sdp_set_profiling(h: int, on: bool) -> None:
    lib = load()
    st = lib.sdp_set_profiling(c_void_p(h), 1 if on else 0)
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())


def sdp_adjoint_dense_noalloc(a_dense: int, n: int, m: int, y: int, Y: int, stream: int) -> int:
    """Y = A^T(y) with no device allocation (fixed scratch in the library); returns the status."""
    return int(load().sdp_adjoint_dense_noalloc(c_void_p(a_dense), n, m, c_void_p(y), c_void_p(Y),
                                                c_void_p(stream)))


def sdp_set_tc_wait_limit_ns(ns: int) -> None:
    """Limit of the main-loop waits of the tensor-core product (0: the default 2 s)."""
    load().sdp_set_tc_wait_limit_ns(int(ns))


def sdp_apply_augsys(h: int, pin: int, out: int, which: int) -> int:
    """out = M pin (which 0) or P^{-1} pin (which 1) at the handle's last scaling point."""
    lib = load()
    st = lib.sdp_apply_augsys(c_void_p(h), c_void_p(pin), c_void_p(out), which)
    if st != SDP_OK:
        raise SdpError(st, lib.sdp_last_error(c_void_p(h)).decode())
    return st


def sdp_bounds_report() -> tuple[int, int, int]:
    """(status, first violation, count) of the checked build's bounds records (cleared by the call)."""
    first, count = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = load().sdp_bounds_report(ctypes.byref(first), ctypes.byref(count))
    return int(st), int(first.value), int(count.value)


def sdp_bounds_selftest(stream: int, index: int, bound: int) -> int:
    return int(load().sdp_bounds_selftest(c_void_p(stream), index, bound))


def sdp_workspace_bytes(h: int) -> int:
    return int(load().sdp_workspace_bytes(c_void_p(h)))


def sdp_last_launch_count(h: int) -> int:
    return int(load().sdp_last_launch_count(c_void_p(h)))


def sdp_last_error(h: int | None) -> str:
    return load().sdp_last_error(c_void_p(h) if h else None).decode()


def sdp_destroy(h: int) -> None:
    load().sdp_destroy(c_void_p(h))

"""The SPD inverse and Cholesky factor of the preconditioner core (sdp_spd_inverse), both forms:
one cooperative launch (n <= 1024) and the launch chain, against exact integer arithmetic and
numpy's FP64 factorisations.

Section 6 inverts the Schur complement of the preconditioner (C = tau^2 Sigma + beta^{-1} B^T B,
or the m-space K) once per Newton solve; the PCG then applies it as one product.

- Exact cases: A = L0 L0^T with L0 unit lower bidiagonal, subdiagonal in {-1, 0, 1}.  Then
  L = L0, L^{-1} has entries in {-1, 0, 1} and A^{-1} = L^{-T} L^{-1} is an integer matrix with
  entries up to n: every step of either form is exact in FP64, so the results must equal the
  integer ones bit for bit (any misplaced tile, transposed operand or skipped update shows).
- Gaussian SPD matrices with condition numbers 1e2 .. 1e8: ||L L^T - A|| <= 4 n eps ||A||
  (backward stability), ||A A^{-1} - I|| and the distance to numpy's inverse within
  8 n cond eps, and the two forms agree within the same bound.
- Ragged sizes (1, 31, 33, ..., 1000, 1024), the first size past the cooperative limit (1100),
  and a matrix that is not positive definite (SDP_ENUMERIC, no fault).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _run(A, mode, coop, want_linv=True):
    import torch
    from paper_2407_14013_gb300 import _native
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()      # column-major A
    dL = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda") if (mode == 1 and want_linv) else None
    wb = _native.load().sdp_spd_inverse_work_bytes(n)
    work = torch.empty(wb // 8 + 64, dtype=torch.float64, device="cuda")
    wptr = (work.data_ptr() + 255) // 256 * 256
    _native.sdp_spd_inverse(torch.cuda.current_stream().cuda_stream, n, dA.data_ptr(),
                            dL.data_ptr() if dL is not None else 0, mode, coop, wptr, wb)
    out = dA.cpu().numpy().T
    return (out, dL.cpu().numpy().T) if dL is not None else (out, None)


def _exact_case(n, seed):
    rng = np.random.default_rng(seed)
    s = rng.integers(-1, 2, max(n - 1, 0))
    L0 = np.eye(n, dtype=np.int64) + np.diag(s, -1).astype(np.int64)
    Li0 = np.zeros((n, n), dtype=np.int64)           # L0^{-1}: (-1)^(i-j) prod s[j..i-1]
    for j in range(n):
        Li0[j, j] = 1
        for i in range(j + 1, n):
            Li0[i, j] = -s[i - 1] * Li0[i - 1, j]
    A = L0 @ L0.T
    Ainv = Li0.T @ Li0
    assert np.array_equal(A @ Ainv, np.eye(n, dtype=np.int64))
    return A.astype(np.float64), L0.astype(np.float64), Li0.astype(np.float64), Ainv.astype(np.float64)


@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 95, 200, 597, 1000, 1024])
@pytest.mark.parametrize("coop", [1, 0])
def test_exact_integer_cases(n, coop):
    A, L0, Li0, Ainv = _exact_case(n, 7000 + n)
    got, _ = _run(A, 0, coop)
    assert np.array_equal(got, Ainv), (n, coop, np.abs(got - Ainv).max())
    L, Linv = _run(A, 1, coop)
    assert np.array_equal(L, L0), (n, coop)
    assert np.array_equal(Linv, Li0), (n, coop)
    L, none = _run(A, 1, coop, want_linv=False)
    assert none is None and np.array_equal(L, L0)


def _spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, 1.0 / cond, n)
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("n,cond", [(64, 1e2), (597, 1e4), (597, 1e8), (1000, 1e6), (1024, 1e3), (1100, 1e4)])
def test_gaussian_spd(n, cond):
    A = _spd(n, cond, 7100 + n)
    ref = np.linalg.inv(A)
    bound = 8 * n * cond * EPS
    outs = []
    for coop in (1, 0):
        got, _ = _run(A, 0, coop)
        assert np.array_equal(got, got.T)
        res = np.abs(A @ got - np.eye(n)).max()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"\nn={n} cond={cond:.0e} coop={coop}: ||A Ainv - I||_max={res:.2e} vs numpy {err:.2e}")
        assert res <= bound and err <= bound, (coop, res, err, bound)
        L, Linv = _run(A, 1, coop)
        assert np.array_equal(np.triu(L, 1), np.zeros((n, n)))
        assert np.array_equal(np.triu(Linv, 1), np.zeros((n, n)))
        assert np.abs(L @ L.T - A).max() <= 4 * n * EPS * np.abs(A).max()
        assert np.abs(Linv @ L - np.eye(n)).max() <= 8 * n * np.sqrt(cond) * EPS
        outs.append(got)
    assert np.abs(outs[0] - outs[1]).max() <= bound * np.abs(ref).max()


@pytest.mark.parametrize("coop", [1, 0])
def test_not_positive_definite(coop):
    from paper_2407_14013_gb300._native import SdpError, SDP_ENUMERIC
    A = _spd(300, 1e2, 7200)
    A[150, 150] = -1.0                               # a negative diagonal entry: not SPD
    with pytest.raises(SdpError) as ei:
        _run(A, 0, coop)
    assert ei.value.status == SDP_ENUMERIC
    # the stream and the context stay usable
    B = _spd(40, 10.0, 7201)
    got, _ = _run(B, 0, coop)
    assert np.abs(B @ got - np.eye(40)).max() <= 8 * 40 * 10.0 * EPS

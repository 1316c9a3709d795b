"""FP64 products on the BF16 tensor cores (sdp_gemm_f64_tc, exact-slice splitting) against numpy
FP64 matrix products.

- Integer matrices (|a| <= 100, K <= 4096): every slice product is exact and the sums are
  integers below 2^53, so the result must equal numpy's bit for bit.
- Gaussian matrices, ragged shapes (M, N not multiples of the 128-row tile, K not a multiple of
  the 64-column step, K above one 4096-chunk), both transposes, alpha/beta: elementwise error
  <= 4 K 2^-53 max_k|A[i,k]| max_k|B[k,j]| (the stated bound, with room).
- Rows scaled over 1e-150 .. 1e150 (the per-row and per-column exponents absorb it).
- Products with few output tiles split K over the SMs; their partial tiles are reduced in a
  fixed order, so the same call twice gives the same bits.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _tc(A, B, tA=False, tB=False, alpha=1.0, beta=0.0, C=None):
    import torch
    from paper_2407_14013_gb300 import _native
    Am = np.asfortranarray(A.T if tA else A)        # stored matrix, column-major
    Bm = np.asfortranarray(B.T if tB else B)
    M, K = A.shape
    N = B.shape[1]
    dA = torch.from_numpy(Am.T.copy()).cuda().t()   # column-major view on the device
    dB = torch.from_numpy(Bm.T.copy()).cuda().t()
    C0 = np.zeros((M, N)) if C is None else C
    dC = torch.from_numpy(np.asfortranarray(C0).T.copy()).cuda().t()
    wb = _native.load().sdp_gemm_f64_tc_work_bytes(M, N, K)
    work = torch.empty(wb // 8 + 64, dtype=torch.float64, device="cuda")
    wptr = (work.data_ptr() + 255) // 256 * 256
    lda = Am.shape[0]
    ldb = Bm.shape[0]
    _native.sdp_gemm_f64_tc(torch.cuda.current_stream().cuda_stream, tA, tB, M, N, K, alpha, dA.data_ptr(), lda,
                            dB.data_ptr(), ldb, beta, dC.data_ptr(), M, wptr, wb)
    return dC.cpu().numpy()


def test_integer_products_are_exact():
    rng = np.random.default_rng(1)
    for (M, N, K) in [(128, 128, 64), (200, 77, 1000), (301, 260, 4096)]:
        A = rng.integers(-100, 101, (M, K)).astype(np.float64)
        B = rng.integers(-100, 101, (K, N)).astype(np.float64)
        assert np.array_equal(_tc(A, B), A @ B), (M, N, K)


@pytest.mark.parametrize("M,N,K,tA,tB", [(129, 130, 65, False, False), (256, 100, 5000, False, True),
                                         (333, 257, 700, True, False), (64, 512, 9000, True, True),
                                         # few output tiles: K split over the SMs, partial tiles reduced
                                         (600, 100, 5000, True, False), (130, 70, 3000, False, False)])
def test_gaussian_products_within_the_bound(M, N, K, tA, tB):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C0 = rng.standard_normal((M, N))
    got = _tc(A, B, tA, tB, alpha=0.75, beta=-0.5, C=C0)
    ref = 0.75 * (A @ B) - 0.5 * C0
    bound = 4 * K * 2.0 ** -53 * np.outer(np.abs(A).max(1), np.abs(B).max(0)) * 0.75 + 2.0 ** -52 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)


def test_row_and_column_scales():
    rng = np.random.default_rng(7)
    M, N, K = 150, 140, 300
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-150, 150, (M, 1))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-150, 150, (1, N))
    got = _tc(A, B)
    ref = A @ B
    bound = 4 * K * 2.0 ** -53 * np.outer(np.abs(A).max(1), np.abs(B).max(0))
    assert np.all(np.abs(got - ref) <= bound)


def test_zero_and_empty():
    A = np.zeros((70, 30))
    B = np.zeros((30, 90))
    assert np.array_equal(_tc(A, B), np.zeros((70, 90)))


def test_split_k_is_deterministic():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 4000))
    B = rng.standard_normal((4000, 90))
    assert np.array_equal(_tc(A, B), _tc(A, B))


def test_bounded_wait_runs_out_and_the_stream_stays_usable():
    """A main-loop wait limit of a few ns makes the product's bounded waits run out: the call
    returns SDP_ETIMEOUT (nothing faults or hangs: the kernel waits with its full bound for its own
    copies and products in flight, frees its TMEM and returns), and the next product on the same
    stream, with the default limit restored, is exact."""
    import torch
    from paper_2407_14013_gb300 import _native
    rng = np.random.default_rng(7)
    A = rng.integers(-100, 101, (256, 512)).astype(np.float64)
    B = rng.integers(-100, 101, (512, 256)).astype(np.float64)
    _native.sdp_set_tc_wait_limit_ns(5)
    try:
        with pytest.raises(_native.SdpError) as ei:
            _tc(A, B)
        assert ei.value.status == _native.SDP_ETIMEOUT
    finally:
        _native.sdp_set_tc_wait_limit_ns(0)
    torch.cuda.synchronize()
    assert np.array_equal(_tc(A, B), A @ B)
    assert np.array_equal(_tc(B.T, A.T), B.T @ A.T)

"""The mixed forms' low-precision products on the tensor cores (sdp_gemm_tn_lp: tcgen05 kind::f16
with BF16 operands, kind::tf32 with FP32 operands read as TF32, FP32 accumulation in TMEM)
against FP64 numpy products of the same operand values.

- Small-integer operands are exact in BF16 and TF32 and every partial sum is an integer below
  2^24, so the product must equal numpy's bit for bit.
- Gaussian BF16 operands: each product of two BF16 values is exact in FP32, so the only error is
  the FP32 summation: |C - A^T B| <= K 2^-23 (|A|^T |B|) elementwise (a loose form of the
  recursive-summation bound).  TF32: the operands are first rounded to 10 fraction bits (the
  tensor core reads the top of the FP32 word), adding 2 * 2^-10 (|A|^T |B|).
- Ragged shapes: M, N not multiples of the 128-row tile, K not a multiple of the K-slice (64
  BF16 / 32 TF32 entries), K below one slice, and the n = 200 shape of the sensing workload.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lp(As, Bs, tf32, alpha=1.0):
    """C = alpha As^T Bs through the C ABI; As (K x M), Bs (K x N) numpy FP32 (values already
    representable in the operand type)."""
    import torch
    from paper_2407_14013_gb300 import _native
    K, M = As.shape
    N = Bs.shape[1]
    dt = torch.float32 if tf32 else torch.bfloat16
    q = 4 if tf32 else 8                                       # 16-byte rows
    lda = ldb = (K + q - 1) // q * q
    dA = torch.zeros((M, lda), dtype=dt, device="cuda")       # row i = column i of As (K-contiguous)
    dB = torch.zeros((N, ldb), dtype=dt, device="cuda")
    dA[:, :K] = torch.from_numpy(np.ascontiguousarray(As.T)).to(dt).cuda()
    dB[:, :K] = torch.from_numpy(np.ascontiguousarray(Bs.T)).to(dt).cuda()
    C = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")   # column-major M x N
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    _native.sdp_gemm_tn_lp(torch.cuda.current_stream().cuda_stream, tf32, M, N, K, alpha, dA.data_ptr(), lda,
                           dB.data_ptr(), ldb, C.data_ptr(), M, err.data_ptr())
    return C.cpu().numpy().T.astype(np.float64)


def _bf16(x):
    import torch
    return torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _tf32(x):
    """Values rounded to 10 fraction bits (nearest, ties away), as a TF32 operand holds them."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + (1 << 12)) & ~np.uint64((1 << 13) - 1)).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


SHAPES = [(200, 200, 200), (129, 257, 65), (1, 1, 1), (128, 128, 64), (300, 64, 1000), (64, 300, 31)]


@pytest.mark.parametrize("tf32", [False, True], ids=["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_integer_operands_are_exact(tf32, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    As = rng.integers(-8, 9, (K, M)).astype(np.float64)
    Bs = rng.integers(-8, 9, (K, N)).astype(np.float64)
    assert np.array_equal(_lp(As, Bs, tf32), As.T @ Bs)


@pytest.mark.parametrize("tf32", [False, True], ids=["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gaussian_operands_within_the_fp32_bound(tf32, M, N, K):
    rng = np.random.default_rng(M + 11 * N + 101 * K)
    As = rng.standard_normal((K, M))
    Bs = rng.standard_normal((K, N))
    if tf32:
        C = _lp(As.astype(np.float32).astype(np.float64), Bs.astype(np.float32).astype(np.float64), True, alpha=0.5)
        Ar, Br = _tf32(As), _tf32(Bs)
        ref = 0.5 * (As.astype(np.float32).astype(np.float64).T @ Bs.astype(np.float32).astype(np.float64))
        bound = 0.5 * (K * 2.0 ** -23 + 2 * 2.0 ** -10) * (np.abs(Ar).T @ np.abs(Br))
    else:
        Ab, Bb = _bf16(As), _bf16(Bs)
        C = _lp(Ab, Bb, False, alpha=0.5)
        ref = 0.5 * (Ab.T @ Bb)
        bound = 0.5 * K * 2.0 ** -23 * (np.abs(Ab).T @ np.abs(Bb))
    assert np.all(np.abs(C - ref) <= bound + 1e-30)


def test_bounded_wait_of_the_lp_product():
    """A main-loop wait limit of a few ns makes the low-precision product give up with
    SDP_ETIMEOUT (no fault, no hang); with the default restored the next product is exact."""
    from paper_2407_14013_gb300 import _native
    rng = np.random.default_rng(3)
    # a long K (1024 K-slices per tile) keeps the product running far longer than the limit
    As = rng.integers(-8, 9, (65536, 256)).astype(np.float64)
    Bs = rng.integers(-8, 9, (65536, 256)).astype(np.float64)
    _native.sdp_set_tc_wait_limit_ns(5)
    try:
        with pytest.raises(_native.SdpError) as ei:
            _lp(As, Bs, False)
        assert ei.value.status == _native.SDP_ETIMEOUT
    finally:
        _native.sdp_set_tc_wait_limit_ns(0)
    assert np.array_equal(_lp(As, Bs, False), As.T @ Bs)

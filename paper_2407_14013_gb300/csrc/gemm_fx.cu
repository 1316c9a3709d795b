// Small dense FP64 products C = A B (column-major, no transposes) summed exactly in integers.
//
// GB300 issues FP64 FMAs at 2 per SM per clock (1.26 TFLOP/s for the GPU), so the n^3 products of
// the FP64 operator (E Y E of Section 5 at n of a few hundred) are bound by the FP64 pipe.  Here
// every row i of A is scaled by 2^-ea_i and every column j of B by 2^-eb_j (2^ea_i > max_k |A_ik|,
// 2^eb_j > max_k |B_kj|), both are written as two int32 digits (fx.cuh), and
//   C_ij = 2^(ea_i + eb_j) sum_k (hi_ik hi'_kj 2^-52 + (hi_ik lo'_kj + lo_ik hi'_kj) 2^-78)
// with both sums exact in int64 (flushed to FP64 every FX_FLUSH terms) on the integer pipe.  The
// error of an entry is within about K 2^-53 2^(ea_i + eb_j): the FP64 bound of a K-term dot
// product measured against the largest entry of the row of A and of the column of B.
//
// One CTA per 16 x 16 output tile, one output per thread.  A CTA reads its 16-row panel of A and
// 16-column panel of B twice from L2: once for their exponents (so no separate launch is needed),
// then in K-chunks of 128 that it splits into digits in shared memory.  LOWER skips tiles above
// the diagonal and writes only entries with i >= j.  A row or column with a non-finite entry
// gives NaN outputs.
#include "common.cuh"
#include "fx.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int TB = 16;
constexpr int KC = 128;
constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;

// PRE = 1: A is given by its row digits (Dd[i K + k], exponents De[i]); PRE = 2: B by its column
// digits (Dd[j K + k], exponents De[j]); the CTA then scans and splits only the other operand.
template <int PRE>
__global__ void __launch_bounds__(TB * TB)
fx_gemm_kernel(int M, int N, int K, const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
               int64_t ldb, double* __restrict__ C, int64_t ldc, int lower, const int32_t* __restrict__ done,
               const int2* __restrict__ Dd, const int* __restrict__ De, FxPack pk) {
  if (done && *done) return;
  const int i0 = blockIdx.x * TB, j0 = blockIdx.y * TB;
  if (lower && i0 + TB - 1 < j0) return;            // tile strictly above the diagonal
  __shared__ int2 As[KC][TB];
  __shared__ int2 Bs[KC][TB + 1];
  __shared__ int ered[TB][TB + 1];
  __shared__ int ea[TB], eb[TB];
  const int t = threadIdx.x;
  // ---- exponents: rows of the A panel (lanes along i), columns of the B panel (lanes along k),
  // eight independent loads in flight per thread
  constexpr int UE = 8;
  {
    const int r = t & 15, part = t >> 4;
    const int gi = i0 + r;
    int e = INT_MIN;
    if (gi < M && PRE != 1)
      for (int kb = part; kb < K; kb += 16 * UE) {
        unsigned long long b[UE];
#pragma unroll
        for (int u = 0; u < UE; ++u) {
          const int k = kb + 16 * u;
          b[u] = k < K ? (unsigned long long)__double_as_longlong(A[gi + (int64_t)k * lda]) & ABS : 0ull;
        }
#pragma unroll
        for (int u = 0; u < UE; ++u) {
          if (b[u] >= INF_BITS) e = FX_BAD;
          else if (b[u] && e != FX_BAD) e = max(e, fx_expo_bits(b[u]));
        }
      }
    ered[part][r] = e;
    const int c = t >> 4, kp = t & 15;
    const int gj = j0 + c;
    int f = INT_MIN;
    if (gj < N && PRE != 2)
      for (int kb = kp; kb < K; kb += 16 * UE) {
        unsigned long long b[UE];
#pragma unroll
        for (int u = 0; u < UE; ++u) {
          const int k = kb + 16 * u;
          b[u] = k < K ? (unsigned long long)__double_as_longlong(B[k + (int64_t)gj * ldb]) & ABS : 0ull;
        }
#pragma unroll
        for (int u = 0; u < UE; ++u) {
          if (b[u] >= INF_BITS) f = FX_BAD;
          else if (b[u] && f != FX_BAD) f = max(f, fx_expo_bits(b[u]));
        }
      }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {   // within the 16 lanes of column c (FX_BAD is the largest int)
      const int g = __shfl_xor_sync(0xffffffffu, f, o);
      f = max(f, g);
    }
    if (kp == 0) eb[c] = (PRE == 2) ? (gj < N ? De[gj] : INT_MIN) : f;
    __syncthreads();
    if (t < TB) {
      int m = INT_MIN;
      for (int p = 0; p < 16; ++p) m = max(m, ered[p][t]);
      ea[t] = (PRE == 1) ? (i0 + t < M ? De[i0 + t] : INT_MIN) : m;
    }
    __syncthreads();
  }
  const int ti = t & 15, tj = t >> 4;
  const int ra = ea[ti], rb = eb[tj];
  long long T1 = 0, T2 = 0;
  double acc = 0.0;
  int since = 0;
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kc = min(KC, K - k0);
    __syncthreads();
    {   // A chunk (lanes along i) and B chunk (lanes along k): all loads first, then the digits
      constexpr int US = KC * TB / (TB * TB);          // entries per thread per operand (8)
      double va[US], vb[US];
      int2 da[US], db[US];
#pragma unroll
      for (int u = 0; u < US; ++u) {
        const int q = t + u * TB * TB;
        if (PRE == 1) {                                  // given digits, k contiguous per row
          const int k = q % KC, r = q / KC;
          const int gi = i0 + r;
          da[u] = (k < kc && gi < M) ? Dd[(int64_t)gi * K + k0 + k] : make_int2(0, 0);
        } else {
          const int r = q & 15, k = q >> 4;
          const int gi = i0 + r;
          va[u] = (k < kc && gi < M && ea[r] != FX_BAD) ? A[gi + (int64_t)(k0 + k) * lda] : 0.0;
        }
        const int kk = q % KC, c = q / KC;
        const int gj = j0 + c;
        if (PRE == 2) db[u] = (kk < kc && gj < N) ? Dd[(int64_t)gj * K + k0 + kk] : make_int2(0, 0);
        else vb[u] = (kk < kc && gj < N && eb[c] != FX_BAD) ? B[(k0 + kk) + (int64_t)gj * ldb] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < US; ++u) {
        const int q = t + u * TB * TB;
        if (PRE == 1) {
          As[q % KC][q / KC] = da[u];
        } else {
          const int r = q & 15, k = q >> 4;
          const int F = ea[r];
          As[k][r] = fx_split((F == INT_MIN || F == FX_BAD) ? 0 : fx_fixed(va[u], 0, F));
        }
        const int kk = q % KC, c = q / KC;
        if (PRE == 2) {
          Bs[kk][c] = db[u];
        } else {
          const int G = eb[c];
          Bs[kk][c] = fx_split((G == INT_MIN || G == FX_BAD) ? 0 : fx_fixed(vb[u], 0, G));
        }
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kc; ++k) {
      const int2 a = As[k][ti], b = Bs[k][tj];
      T1 += (long long)a.x * b.x;
      T2 += (long long)a.x * b.y + (long long)a.y * b.x;
    }
    since += kc;
    if (since >= FX_FLUSH) {                           // KC divides FX_FLUSH
      acc += fx_value(T1, T2);
      T1 = T2 = 0;
      since = 0;
    }
  }
  acc += fx_value(T1, T2);
  const int gi = i0 + ti, gj = j0 + tj;
  const bool act = gi < M && gj < N && !(lower && gi < gj);
  double v = 0.0;
  if (act) {
    if (ra == FX_BAD || rb == FX_BAD) v = __longlong_as_double(0x7ff8000000000000ll);
    else if (ra == INT_MIN || rb == INT_MIN) v = 0.0;
    else v = ldexp(acc, ra + rb);
  }
  if (pk.out) {
    // svec(C + sym(U Q^T)) at (gi, gj), gi >= gj, and the exponent of the packed vector, as
    // svec_pack_plus_kernel forms them from C (same operations, same order)
    int e = INT_MIN;
    if (act) {
      if (pk.U) {
        double su = 0.0;
        for (int k = 0; k < pk.r; ++k)
          su += pk.U[gi + (int64_t)k * M] * pk.Q[gj + (int64_t)k * M] +
                pk.Q[gi + (int64_t)k * M] * pk.U[gj + (int64_t)k * M];
        v += 0.5 * su;
      }
      const double o = (gi == gj) ? v : v * WC_SQRT2;
      pk.out[svec_index(M, gi, gj)] = o;
      const unsigned long long bits = (unsigned long long)__double_as_longlong(o) & ABS;
      e = bits >= INF_BITS ? INT_MAX : (bits ? fx_expo_bits(bits) : INT_MIN);
    }
    if (pk.expo) {   // one atomic per warp (every thread of the tile is here)
      e = __reduce_max_sync(0xffffffffu, e);
      if ((t & 31) == 0 && e != INT_MIN) atomicMax(pk.expo, e);
    }
    return;
  }
  if (act) C[gi + (int64_t)gj * ldc] = v;
}

}  // namespace

cudaError_t fx_gemm(cudaStream_t st, int M, int N, int K, const double* A, int64_t lda, const double* B, int64_t ldb,
                    double* C, int64_t ldc, bool lower, const int32_t* done, int64_t* launches, int pre,
                    const int2* Dd, const int* De, const FxPack* pack) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 0 || (pre != 0 && (!Dd || !De)) || (pack && (M != N || !lower))) return cudaErrorInvalidValue;
  dim3 grid((M + TB - 1) / TB, (N + TB - 1) / TB);
  const int lw = lower ? 1 : 0;
  const FxPack pk = pack ? *pack : FxPack{};
  if (pre == 1) fx_gemm_kernel<1><<<grid, TB * TB, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, lw, done, Dd, De, pk);
  else if (pre == 2) fx_gemm_kernel<2><<<grid, TB * TB, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, lw, done, Dd, De, pk);
  else fx_gemm_kernel<0><<<grid, TB * TB, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, lw, done, Dd, De, pk);
  if (launches) ++*launches;
  return cudaGetLastError();
}

namespace {

// Exponent and digits of column j of M (n x n, column-major, n <= 512), one warp per column: the
// same exponent (the column's largest) and digits fx_gemm_kernel forms for a B panel, so digits
// made once can stand for that work in every product with M.
__global__ void col_digits_kernel(int n, const double* __restrict__ M, int2* __restrict__ D, int* __restrict__ e) {
  const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (j >= n) return;                                  // whole warps
  const int lane = threadIdx.x & 31;
  constexpr int VL = 16;
  double v[VL];
#pragma unroll
  for (int u = 0; u < VL; ++u) {
    const int k = lane + 32 * u;
    v[u] = k < n ? M[(int64_t)j * n + k] : 0.0;
  }
  int f = INT_MIN;
#pragma unroll
  for (int u = 0; u < VL; ++u) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v[u]) & ABS;
    if (b >= INF_BITS) f = FX_BAD;
    else if (b && f != FX_BAD) f = max(f, fx_expo_bits(b));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f = max(f, __shfl_xor_sync(0xffffffffu, f, o));   // FX_BAD is the largest int
  const bool zero = (f == INT_MIN || f == FX_BAD);
#pragma unroll
  for (int u = 0; u < VL; ++u) {
    const int k = lane + 32 * u;
    if (k < n) D[(int64_t)j * n + k] = zero ? make_int2(0, 0) : fx_split(fx_fixed(v[u], 0, f));
  }
  if (lane == 0) e[j] = f;
}

}  // namespace

bool fx_col_digits(cudaStream_t st, int n, const double* M, int2* D, int* e, int64_t* launches) {
  if (n <= 0 || n > 512) return false;
  col_digits_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, M, D, e);
  if (launches) ++*launches;
  return true;
}

}  // namespace wc

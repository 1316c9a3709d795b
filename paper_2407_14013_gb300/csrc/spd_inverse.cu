// Inverse of a symmetric positive definite matrix through its Cholesky factor:
//   A = L L^T,  X = L^{-1},  A^{-1} = X^T X.
//
// The preconditioner of Section 6 needs one solve with its Schur complement per PCG
// iteration.  A triangular solve is a chain of dependent steps that occupies a few SMs;
// multiplying by an explicit inverse is one bandwidth-bound matrix-vector product over the
// whole GPU, so the complement (C = tau^2 Sigma + beta^{-1} B^T B, or the m-space
// K = beta I + B D^{-1} B^T) is inverted once per Newton solve.  The Cholesky route keeps the
// error of the inverse near cond(A) eps (Gauss-Jordan sweeps lose about cond(A)^2 eps, which
// the m-space complement, ill-conditioned at small mu, cannot afford).
//
// Blocked with NB x NB diagonal blocks: each diagonal block is factored and its triangular
// factor inverted inside one CTA; everything else is FP64 GEMM (DMMA).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int NB = 32;

// Factor the w x w diagonal block at k0 (already updated by earlier blocks): L_KK into the
// lower triangle of A (upper part of the block zeroed), its inverse into Li (w x w, ld w).
//
// GB300 issues FP64 arithmetic at 2 lane-operations per SM per clock and a warp instruction
// costs its full width even with lanes masked off, so this kernel, which runs on one SM,
// enumerates exactly the active entries of each step (a table of the lower pairs, last
// column first) and takes one division per pivot.  Step p (one barrier each) does
//   the LDL^T update  S_ij -= S_ip S_jp / S_pp             (p < j <= i),
//   the inverse sweep X~_ij -= (S_ip / S_pp) X~_pj          (i > p >= j),
// so that X~ = L~^{-1} for the unit lower factor L~ = [S_ip / S_pp]; then L = L~ D^{1/2} and
// L^{-1} = D^{-1/2} X~ with D = diag(S_pp).
__global__ void __launch_bounds__(256)
chol_block_kernel(int n, int k0, int w, double* __restrict__ A, double* __restrict__ Li,
                  int32_t* __restrict__ status) {   // n: leading dimension of A
  __shared__ double S[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  __shared__ double inv[NB], dsq[NB], rdsq[NB];
  __shared__ unsigned char ti[NB * (NB + 1) / 2], tj[NB * (NB + 1) / 2];
  __shared__ int bad;
  const int ww = w * w;
  for (int q = threadIdx.x; q < ww; q += blockDim.x) {
    const int i = q % w, j = q / w;
    S[i][j] = A[(k0 + i) + (int64_t)(k0 + j) * n];
    X[i][j] = (i == j) ? 1.0 : 0.0;
    if (i >= j) {                          // column j's pairs start at T(w-1-j), T(k) = k(k+1)/2
      const int c = w - 1 - j;
      const int pos = c * (c + 1) / 2 + (i - j);
      ti[pos] = (unsigned char)i;
      tj[pos] = (unsigned char)j;
    }
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double piv = S[0][0];
    if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
    inv[0] = (piv > 0.0 && isfinite(piv)) ? 1.0 / piv : 1.0;
  }
  __syncthreads();
  for (int p = 0; p < w; ++p) {
    const double ip = inv[p];
    const int k = w - 1 - p;
    const int cnt_a = k * (k + 1) / 2;     // pairs with j > p: the first T(k) table entries
    const int cnt = cnt_a + k * (p + 1);   // plus the k x (p + 1) block of the sweep
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      if (t < cnt_a) {
        const int i = ti[t], j = tj[t];
        const double v = S[i][j] - S[i][p] * S[j][p] * ip;
        S[i][j] = v;
        if (i == j && j == p + 1) {        // the next pivot is final now
          if (!(v > 0.0) || !isfinite(v)) bad = 1;
          inv[j] = (v > 0.0 && isfinite(v)) ? 1.0 / v : 1.0;
        }
      } else {
        const int u = t - cnt_a;
        const int i = p + 1 + u % k, j = u / k;
        X[i][j] -= (S[i][p] * ip) * X[p][j];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < w) {                   // D^{1/2} and D^{-1/2}, once per pivot
    const int j = threadIdx.x;
    const double dj = sqrt(S[j][j] > 0.0 ? S[j][j] : 1.0);
    dsq[j] = dj;
    rdsq[j] = 1.0 / dj;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < ww; q += blockDim.x) {
    const int i = q % w, j = q / w;
    double l = 0.0, x = 0.0;
    if (i > j) { l = S[i][j] * rdsq[j]; x = X[i][j] * rdsq[i]; }
    else if (i == j) { l = dsq[j]; x = rdsq[i]; }
    A[(k0 + i) + (int64_t)(k0 + j) * n] = l;
    Li[i + (int64_t)j * w] = x;
  }
  if (threadIdx.x == 0 && bad) *status = 5;
}

// dst (rows x cols, ld ldd) = src (ld lds)
__global__ void copy_block_kernel(int rows, int cols, const double* __restrict__ src, int64_t lds,
                                  double* __restrict__ dst, int64_t ldd) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)rows * cols) return;
  int i = (int)(q % rows), j = (int)(q / rows);
  dst[i + (int64_t)j * ldd] = src[i + (int64_t)j * lds];
}

// zero the strictly upper triangle of an n x n matrix
__global__ void zero_upper_kernel(int n, int64_t ld, double* __restrict__ A) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int i = (int)(q % n), j = (int)(q / n);
  if (j > i) A[i + (int64_t)j * ld] = 0.0;
}

// upper triangle := lower triangle
__global__ void lower_to_full_kernel(int n, double* __restrict__ A) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int i = (int)(q % n), j = (int)(q / n);
  if (i <= j) return;
  A[j + (int64_t)i * n] = A[q];
}

inline unsigned nblk(int64_t total, int t) { return (unsigned)((total + t - 1) / t); }

}  // namespace

size_t spd_inverse_work(int n) { return (size_t)n * n + 2 * (size_t)n * NB + (size_t)((n + NB - 1) / NB) * NB * NB; }

namespace {

// Blocked Cholesky A = L L^T (L into the lower triangle of A, upper zeroed) and X = L^{-1}
// (lower triangular, n x n, ld n).
// A (n x n, leading dimension ld) = L L^T, L into A (upper zeroed); X (ld ldx, NULL: factor
// only) = L^{-1}; T: n x NB, U: NB x n, Li: ceil(n / NB) NB x NB blocks.
cudaError_t cholesky_and_inverse(cudaStream_t st, int n, int64_t ld, double* A, double* X, int64_t ldx, double* T,
                                 double* U, double* Li, double* gemm_ws, size_t gemm_ws_elems, int32_t* status,
                                 int64_t* launches) {
  cudaError_t e;
  // ---- blocked right-looking Cholesky, L in the lower triangle of A
  for (int k0 = 0, b = 0; k0 < n; k0 += NB, ++b) {
    const int w = (n - k0) < NB ? (n - k0) : NB;
    const int k1 = k0 + w, rest = n - k1;
    double* Lib = Li + (size_t)b * NB * NB;
    chol_block_kernel<<<1, 256, 0, st>>>((int)ld, k0, w, A, Lib, status);
    if (launches) ++*launches;
    if (rest == 0) break;
    // L_RK = A_RK L_KK^{-T}
    e = gemm_f64(st, false, true, rest, w, w, 1.0, A + k1 + (int64_t)k0 * ld, ld, Lib, w, 0.0, T, rest, gemm_ws,
                 gemm_ws_elems, launches);
    if (e != cudaSuccess) return e;
    copy_block_kernel<<<nblk((int64_t)rest * w, 256), 256, 0, st>>>(rest, w, T, rest, A + k1 + (int64_t)k0 * ld, ld);
    if (launches) ++*launches;
    // A_RR -= L_RK L_RK^T
    e = gemm_f64(st, false, true, rest, rest, w, -1.0, T, rest, T, rest, 1.0, A + k1 + (int64_t)k1 * ld, ld, gemm_ws,
                 gemm_ws_elems, launches, nullptr, GEMM_LOWER);
    if (e != cudaSuccess) return e;
  }
  zero_upper_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, ld, A);
  if (launches) ++*launches;
  if (!X) return cudaGetLastError();   // factor only
  // ---- X = L^{-1} by block rows: X[I, :I] = -Li_II (L[I, :I] X[:I, :I]), X[I, I] = Li_II
  e = cudaMemset2DAsync(X, ldx * sizeof(double), 0, n * sizeof(double), n, st);
  if (e != cudaSuccess) return e;
  for (int i0 = 0, b = 0; i0 < n; i0 += NB, ++b) {
    const int w = (n - i0) < NB ? (n - i0) : NB;
    const double* Lib = Li + (size_t)b * NB * NB;
    if (i0 > 0) {
      e = gemm_f64(st, false, false, w, i0, i0, 1.0, A + i0, ld, X, ldx, 0.0, U, w, gemm_ws, gemm_ws_elems, launches,
                   nullptr, GEMM_KSTART_COL);   // X lower triangular
      if (e != cudaSuccess) return e;
      e = gemm_f64(st, false, false, w, i0, w, -1.0, Lib, w, U, w, 0.0, X + i0, ldx, gemm_ws, gemm_ws_elems, launches);
      if (e != cudaSuccess) return e;
    }
    copy_block_kernel<<<nblk((int64_t)w * w, 256), 256, 0, st>>>(w, w, Lib, w, X + i0 + (int64_t)i0 * ldx, ldx);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace

// A (n x n, ld n) is overwritten with its inverse.  work must hold spd_inverse_work(n) doubles.
cudaError_t spd_inverse(cudaStream_t st, int n, double* A, double* work, size_t work_elems,
                        double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches) {
  if (spd_inverse_work(n) > work_elems) return cudaErrorInvalidValue;
  double* X = work;                                   // n x n, becomes L^{-1}
  double* T = X + (size_t)n * n;                      // n x NB panel
  double* U = T + (size_t)n * NB;                     // NB x n temporary
  double* Li = U + (size_t)n * NB;                    // inverses of the diagonal blocks
  cudaError_t e = cholesky_and_inverse(st, n, n, A, X, n, T, U, Li, gemm_ws, gemm_ws_elems, status, launches);
  if (e != cudaSuccess) return e;
  // ---- A^{-1} = X^T X
  // lower triangle of X^T X, skipping the zero upper part of X
  e = gemm_f64(st, true, false, n, n, n, 1.0, X, n, X, n, 0.0, A, n, gemm_ws, gemm_ws_elems, launches, nullptr,
               GEMM_LOWER | GEMM_KSTART_ROW | GEMM_KSTART_COL);
  if (e != cudaSuccess) return e;
  lower_to_full_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, A);
  if (launches) ++*launches;
  return cudaGetLastError();
}

void lower_to_full(cudaStream_t st, int n, double* A, int64_t* launches) {
  lower_to_full_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, A);
  if (launches) ++*launches;
}

// ---- two-level form for large n: 512-wide outer panels whose products run on the tensor cores

namespace {

constexpr int NB2 = 512;

// dense product: tensor cores (exact slices) when the context allows and the product is large
cudaError_t gemm_any(const TcCtx* tc, cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                     double* gemm_ws, size_t gemm_ws_elems, int64_t* launches, int flags) {
  if (tc && tc->work && M >= 64 && N >= 64 && K >= 64 && (double)M * N * K >= 134217728.0 &&
      tc_gemm_work_bytes(M, N, std::min(K, 4096)) <= tc->bytes)
    return gemm_f64_tc(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tc->work, tc->bytes, tc->err,
                       flags & GEMM_LOWER, launches);
  return gemm_f64(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, gemm_ws, gemm_ws_elems, launches, nullptr,
                  flags);
}

}  // namespace

size_t spd_inverse_tc_work(int n) {
  if (n < 2 * NB2) return spd_inverse_work(n);
  const size_t nb2 = (size_t)(n + NB2 - 1) / NB2;
  // X (n x n), panel T (n x NB2), U (NB2 x n), the diagonal-block inverses, the inner temporaries
  return (size_t)n * n + 2 * (size_t)n * NB2 + nb2 * NB2 * NB2 + 2 * (size_t)NB2 * NB + (size_t)(NB2 / NB) * NB * NB;
}

cudaError_t spd_inverse_tc(cudaStream_t st, int n, double* A, double* work, size_t work_elems, double* gemm_ws,
                           size_t gemm_ws_elems, const TcCtx* tc, int32_t* status, int64_t* launches) {
  if (spd_inverse_tc_work(n) > work_elems) return cudaErrorInvalidValue;
  if (n < 2 * NB2) {   // one level of 32-wide panels; only X^T X on the tensor cores
    double* X = work;
    double* T = X + (size_t)n * n;
    double* U = T + (size_t)n * NB;
    double* Li = U + (size_t)n * NB;
    cudaError_t e = cholesky_and_inverse(st, n, n, A, X, n, T, U, Li, gemm_ws, gemm_ws_elems, status, launches);
    if (e != cudaSuccess) return e;
    e = gemm_any(tc, st, true, false, n, n, n, 1.0, X, n, X, n, 0.0, A, n, gemm_ws, gemm_ws_elems, launches,
                 GEMM_LOWER | GEMM_KSTART_ROW | GEMM_KSTART_COL);
    if (e != cudaSuccess) return e;
    lower_to_full_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, A);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  double* X = work;                                       // n x n, becomes L^{-1}
  double* T = X + (size_t)n * n;                          // rest x NB2 panel
  double* U = T + (size_t)n * NB2;                        // NB2 x i0
  double* Xd = U + (size_t)n * NB2;                       // inverses of the diagonal blocks (ld NB2)
  const size_t nb2 = (size_t)(n + NB2 - 1) / NB2;
  double* Ti = Xd + nb2 * NB2 * NB2;                      // inner temporaries
  double* Ui = Ti + (size_t)NB2 * NB;
  double* Li = Ui + (size_t)NB2 * NB;
  cudaError_t e;
  // ---- right-looking Cholesky over 512-wide panels
  for (int k0 = 0, b = 0; k0 < n; k0 += NB2, ++b) {
    const int w = std::min(NB2, n - k0);
    const int k1 = k0 + w, rest = n - k1;
    double* Xb = Xd + (size_t)b * NB2 * NB2;
    // L_KK and L_KK^{-1} (one-CTA 32 x 32 blocks inside)
    e = cholesky_and_inverse(st, w, n, A + k0 + (int64_t)k0 * n, Xb, NB2, Ti, Ui, Li, gemm_ws, gemm_ws_elems, status,
                             launches);
    if (e != cudaSuccess) return e;
    if (rest == 0) break;
    // L_RK = A_RK L_KK^{-T};  A_RR -= L_RK L_RK^T (lower)
    e = gemm_any(tc, st, false, true, rest, w, w, 1.0, A + k1 + (int64_t)k0 * n, n, Xb, NB2, 0.0, T, rest, gemm_ws,
                 gemm_ws_elems, launches, 0);
    if (e != cudaSuccess) return e;
    copy_block_kernel<<<nblk((int64_t)rest * w, 256), 256, 0, st>>>(rest, w, T, rest, A + k1 + (int64_t)k0 * n, n);
    if (launches) ++*launches;
    e = gemm_any(tc, st, false, true, rest, rest, w, -1.0, T, rest, T, rest, 1.0, A + k1 + (int64_t)k1 * n, n, gemm_ws,
                 gemm_ws_elems, launches, GEMM_LOWER);
    if (e != cudaSuccess) return e;
  }
  zero_upper_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, n, A);
  if (launches) ++*launches;
  // ---- X = L^{-1} by panel rows: X[I, :I] = -X_II (L[I, :I] X[:I, :I]), X[I, I] = X_II
  e = cudaMemsetAsync(X, 0, (size_t)n * n * sizeof(double), st);
  if (e != cudaSuccess) return e;
  for (int i0 = 0, b = 0; i0 < n; i0 += NB2, ++b) {
    const int w = std::min(NB2, n - i0);
    const double* Xb = Xd + (size_t)b * NB2 * NB2;
    if (i0 > 0) {
      e = gemm_any(tc, st, false, false, w, i0, i0, 1.0, A + i0, n, X, n, 0.0, U, w, gemm_ws, gemm_ws_elems, launches,
                   GEMM_KSTART_COL);
      if (e != cudaSuccess) return e;
      e = gemm_any(tc, st, false, false, w, i0, w, -1.0, Xb, NB2, U, w, 0.0, X + i0, n, gemm_ws, gemm_ws_elems,
                   launches, 0);
      if (e != cudaSuccess) return e;
    }
    copy_block_kernel<<<nblk((int64_t)w * w, 256), 256, 0, st>>>(w, w, Xb, NB2, X + i0 + (int64_t)i0 * n, n);
    if (launches) ++*launches;
  }
  // ---- A^{-1} = X^T X (lower triangle, then mirrored)
  e = gemm_any(tc, st, true, false, n, n, n, 1.0, X, n, X, n, 0.0, A, n, gemm_ws, gemm_ws_elems, launches,
               GEMM_LOWER | GEMM_KSTART_ROW | GEMM_KSTART_COL);
  if (e != cudaSuccess) return e;
  lower_to_full_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, A);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// A = L L^T: L into A (lower, upper zeroed), L^{-1} into Linv (n x n; NULL: factor only).
// work as for spd_inverse.
cudaError_t spd_cholesky(cudaStream_t st, int n, double* A, double* Linv, double* work, size_t work_elems,
                         double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches) {
  if (spd_inverse_work(n) > work_elems) return cudaErrorInvalidValue;
  double* T = work + (size_t)n * n;
  double* U = T + (size_t)n * NB;
  double* Li = U + (size_t)n * NB;
  return cholesky_and_inverse(st, n, n, A, Linv, n, T, U, Li, gemm_ws, gemm_ws_elems, status, launches);
}

}  // namespace wc

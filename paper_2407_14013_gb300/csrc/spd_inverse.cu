// In-place inverse of a symmetric positive definite matrix by blocked Gauss-Jordan elimination.
//
// The preconditioner of Section 6 needs one solve with its Schur complement per PCG
// iteration.  A triangular solve is a chain of dependent steps that occupies a few SMs;
// multiplying by an explicit inverse is one bandwidth-bound matrix-vector product over the
// whole GPU, so the complement (C = tau^2 Sigma + beta^{-1} B^T B, or the m-space
// K = beta I + B D^{-1} B^T) is inverted once per Newton solve.
//
// Pivoting on the diagonal block K of [[A_KK, A_KR], [A_RK, A_RR]] maps it to
//   [[P, P A_KR], [-A_RK P, A_RR - A_RK P A_KR]],  P = A_KK^{-1};
// after pivoting on every block the array holds A^{-1}.  For an SPD matrix every pivot
// block is a Schur complement of an SPD matrix, hence SPD, and no pivoting is needed.
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int NB = 64;

// P = inverse of the w x w block A[k0:k0+w, k0:k0+w] by scalar Gauss-Jordan in shared memory.
__global__ void __launch_bounds__(256)
block_inverse_kernel(int n, int k0, int w, const double* __restrict__ A, double* __restrict__ P,
                     int32_t* __restrict__ status) {
  __shared__ double S[NB][NB + 1];
  __shared__ double rowp[NB], colp[NB];
  __shared__ int bad;
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
    int i = q % w, j = q / w;
    S[i][j] = A[(k0 + i) + (int64_t)(k0 + j) * n];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int p = 0; p < w; ++p) {
    const double piv = S[p][p];
    if (!(piv > 0.0) || !isfinite(piv)) {
      if (threadIdx.x == 0) bad = 1;
    }
    const double ip = 1.0 / piv;
    for (int q = threadIdx.x; q < w; q += blockDim.x) {
      rowp[q] = S[p][q];
      colp[q] = S[q][p];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
      int i = q % w, j = q / w;
      double v;
      if (i == p && j == p) v = ip;
      else if (i == p) v = ip * rowp[j];
      else if (j == p) v = -colp[i] * ip;
      else v = S[i][j] - colp[i] * ip * rowp[j];
      S[i][j] = v;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
    int i = q % w, j = q / w;
    P[i + (int64_t)j * w] = S[i][j];
  }
  if (threadIdx.x == 0 && bad) *status = 5;
}

// T (n x w) = A[:, K] with the rows of K set to zero.
__global__ void copy_panel_kernel(int n, int k0, int w, const double* __restrict__ A, double* __restrict__ T) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * w) return;
  int i = (int)(q % n), j = (int)(q / n);
  T[q] = (i >= k0 && i < k0 + w) ? 0.0 : A[i + (int64_t)(k0 + j) * n];
}

// Zero the columns K of R (w x n).
__global__ void zero_cols_kernel(int n, int k0, int w, double* __restrict__ R) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= w * w) return;
  int i = q % w, j = q / w;
  R[i + (int64_t)(k0 + j) * w] = 0.0;
}

// Rows K of A: A[K, j] = R[:, j] for j outside K, A[K, K] = P.
__global__ void finish_rows_kernel(int n, int k0, int w, const double* __restrict__ R,
                                   const double* __restrict__ P, double* __restrict__ A) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)w * n) return;
  int i = (int)(q % w), j = (int)(q / w);
  double v = (j >= k0 && j < k0 + w) ? P[i + (int64_t)(j - k0) * w] : R[i + (int64_t)j * w];
  A[(k0 + i) + (int64_t)j * n] = v;
}

__global__ void symmetrize_kernel(int n, double* __restrict__ A) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int i = (int)(q % n), j = (int)(q / n);
  if (i <= j) return;
  double v = 0.5 * (A[q] + A[j + (int64_t)i * n]);
  A[q] = v;
  A[j + (int64_t)i * n] = v;
}

inline unsigned nblk(int64_t total, int t) { return (unsigned)((total + t - 1) / t); }

}  // namespace

// work must hold NB * NB + 2 * n * NB doubles.
cudaError_t spd_inverse(cudaStream_t st, int n, double* A, double* work, size_t work_elems,
                        double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches) {
  if ((size_t)NB * NB + 2 * (size_t)n * NB > work_elems) return cudaErrorInvalidValue;
  double* P = work;
  double* T = work + NB * NB;
  double* R = T + (size_t)n * NB;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int w = (n - k0) < NB ? (n - k0) : NB;
    block_inverse_kernel<<<1, 256, 0, st>>>(n, k0, w, A, P, status);
    copy_panel_kernel<<<nblk((int64_t)n * w, 256), 256, 0, st>>>(n, k0, w, A, T);
    if (launches) *launches += 2;
    // R = P A[K, :]   (w x n)
    cudaError_t e = gemm_f64(st, false, false, w, n, w, 1.0, P, w, A + k0, n, 0.0, R, w, gemm_ws,
                             gemm_ws_elems, launches);
    if (e != cudaSuccess) return e;
    zero_cols_kernel<<<nblk((int64_t)w * w, 256), 256, 0, st>>>(n, k0, w, R);
    if (launches) ++*launches;
    // A_RR -= A_RK P A_KR (rows and columns of K untouched: T rows K and R columns K are zero)
    e = gemm_f64(st, false, false, n, n, w, -1.0, T, n, R, w, 1.0, A, n, gemm_ws, gemm_ws_elems, launches);
    if (e != cudaSuccess) return e;
    // A[:, K] = -A_RK P
    e = gemm_f64(st, false, false, n, w, w, -1.0, T, n, P, w, 0.0, A + (int64_t)k0 * n, n, gemm_ws,
                 gemm_ws_elems, launches);
    if (e != cudaSuccess) return e;
    finish_rows_kernel<<<nblk((int64_t)w * n, 256), 256, 0, st>>>(n, k0, w, R, P, A);
    if (launches) ++*launches;
  }
  symmetrize_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, A);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace wc

// Layout conversions between full symmetric n x n matrices and svec vectors (Notations:
// svec stacks the lower triangle column by column, off-diagonal entries times sqrt(2);
// svec of a non-symmetric matrix is svec of its symmetric part).
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

__global__ void svec_unpack_sum_kernel(int n, const double* __restrict__ part, int groups, int64_t N,
                                       double scale, double* __restrict__ Y,
                                       const int32_t* __restrict__ done) {
  if (done && *done) return;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int a = (int)(q % n), b = (int)(q / n);
  int i = a > b ? a : b, j = a > b ? b : a;
  int64_t idx = svec_index(n, i, j);
  double s = 0.0;
  for (int g = 0; g < groups; ++g) s += part[(int64_t)g * N + idx];
  Y[q] = (a == b ? s : s * WC_RSQRT2) * scale;
}

__global__ void svec_pack_plus_kernel(int n, int r, const double* __restrict__ Z, const double* __restrict__ U,
                                      const double* __restrict__ Q, double* __restrict__ out,
                                      const int32_t* __restrict__ done) {
  if (done && *done) return;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int a = (int)(q % n), b = (int)(q / n);
  if (a < b) return;
  double v = 0.5 * (Z[a + (int64_t)b * n] + Z[b + (int64_t)a * n]);
  if (U) {
    double t = 0.0;
    for (int k = 0; k < r; ++k)
      t += U[a + (int64_t)k * n] * Q[b + (int64_t)k * n] + Q[a + (int64_t)k * n] * U[b + (int64_t)k * n];
    v += 0.5 * t;
  }
  out[svec_index(n, a, b)] = (a == b) ? v : v * WC_SQRT2;
}

__global__ void svec_rows_unpack_kernel(const double* __restrict__ A, int n, int64_t N, int i0, int mb,
                                        double* __restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t per = (int64_t)n * n;
  if (q >= per * mb) return;
  // q enumerates out in memory order: out[b * (mb n) + il * n + a]
  int64_t col = q / ((int64_t)mb * n);
  int64_t rem = q % ((int64_t)mb * n);
  int il = (int)(rem / n), a = (int)(rem % n), b = (int)col;
  int i = a > b ? a : b, j = a > b ? b : a;
  double v = A[(int64_t)(i0 + il) * N + svec_index(n, i, j)];
  out[q] = (a == b) ? v : v * WC_RSQRT2;
}

inline unsigned nblk(int64_t total, int t) { return (unsigned)((total + t - 1) / t); }

}  // namespace

void svec_unpack_sum(cudaStream_t st, int n, const double* part, int groups, double scale, double* Y,
                     const int32_t* done, int64_t* launches) {
  int64_t N = (int64_t)n * (n + 1) / 2;
  svec_unpack_sum_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, part, groups, N, scale, Y, done);
  if (launches) ++*launches;
}

void svec_pack_plus(cudaStream_t st, int n, int r, const double* Z, const double* U, const double* Q,
                    double* out, const int32_t* done, int64_t* launches) {
  svec_pack_plus_kernel<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, r, Z, U, Q, out, done);
  if (launches) ++*launches;
}

void svec_rows_unpack(cudaStream_t st, const double* A, int n, int i0, int mb, double* out,
                      int64_t* launches) {
  int64_t N = (int64_t)n * (n + 1) / 2;
  svec_rows_unpack_kernel<<<nblk((int64_t)n * n * mb, 256), 256, 0, st>>>(A, n, N, i0, mb, out);
  if (launches) ++*launches;
}

}  // namespace wc

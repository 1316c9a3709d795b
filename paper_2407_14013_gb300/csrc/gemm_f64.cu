// FP64 GEMM on the FP64 tensor-core path (mma.sync m8n8k4 f64), column-major operands.
//
//   C (M x N) = alpha * op(A) * op(B) + beta * C
//
// op(A) is M x K (A col-major M x K, or its transpose stored K x M); op(B) is K x N.
// GB300 runs FP64 FMA at about 1 TFLOP/s and this MMA at about 4 TFLOP/s, and the
// dense products of the Newton solve are small (n <= a few thousand), so the grid is
// filled by splitting K across CTAs when the M x N tile count is below the SM count;
// the K-slices write partial tiles to scratch and a second kernel reduces them in a
// fixed order (results are bitwise reproducible).
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int PAD = 4;              // row stride 68 doubles: conflict-free fragment reads
constexpr int THREADS = 128;        // 4 warps in a 2 x 2 arrangement, 32 x 32 each

__global__ void __launch_bounds__(THREADS)
gemm_f64_kernel(int M, int N, int K, int kchunk, double alpha,
                const double* __restrict__ A, int64_t lda, int tA,
                const double* __restrict__ B, int64_t ldb, int tB,
                double beta, double* __restrict__ C, int64_t ldc,
                double* __restrict__ part, const int32_t* __restrict__ done) {
  if (done && *done) return;
  __shared__ double As[BK][BM + PAD];
  __shared__ double Bs[BK][BN + PAD];

  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, t = lane & 3;

  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  // Each thread stages 8 elements of the A tile and 8 of the B tile per K-step.
  double ra[8], rb[8];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int idx = tid + e * THREADS;   // 0 .. 1023
      int mi, ki;
      if (!tA) { mi = idx % BM; ki = idx / BM; } else { ki = idx % BK; mi = idx / BK; }
      int gm = m0 + mi, gk = k0 + ki;
      double v = 0.0;
      if (gm < M && gk < kend) v = tA ? A[(int64_t)gk + (int64_t)gm * lda] : A[(int64_t)gm + (int64_t)gk * lda];
      ra[e] = v;
      int ni, kj;
      if (!tB) { kj = idx % BK; ni = idx / BK; } else { ni = idx % BN; kj = idx / BN; }
      int gn = n0 + ni, gk2 = k0 + kj;
      double w = 0.0;
      if (gn < N && gk2 < kend) w = tB ? B[(int64_t)gn + (int64_t)gk2 * ldb] : B[(int64_t)gk2 + (int64_t)gn * ldb];
      rb[e] = w;
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int idx = tid + e * THREADS;
      int mi, ki;
      if (!tA) { mi = idx % BM; ki = idx / BM; } else { ki = idx % BK; mi = idx / BK; }
      As[ki][mi] = ra[e];
      int ni, kj;
      if (!tB) { kj = idx % BK; ni = idx / BK; } else { ni = idx % BN; kj = idx / BN; }
      Bs[kj][ni] = rb[e];
    }
  };

  if (kbeg < kend) {
    load_tiles(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      store_tiles();
      __syncthreads();
      if (k0 + BK < kend) load_tiles(k0 + BK);   // prefetch the next K-step into registers
#pragma unroll
      for (int kk = 0; kk < BK; kk += 4) {
        double af[4], bf[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) af[i] = As[kk + t][wm + i * 8 + g];
#pragma unroll
        for (int j = 0; j < 4; ++j) bf[j] = Bs[kk + t][wn + j * 8 + g];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) dmma_8x8x4(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
      }
      __syncthreads();
    }
  }

  // Epilogue: c0 = C[g][2t], c1 = C[g][2t+1] within each 8 x 8 tile.
  const bool split = (gridDim.z > 1);
  double* P = split ? part + (int64_t)blockIdx.z * M * N : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        int gm = m0 + wm + i * 8 + g;
        int gn = n0 + wn + j * 8 + 2 * t + c;
        if (gm < M && gn < N) {
          double v = alpha * acc[i][j][c];
          if (split) {
            P[(int64_t)gm + (int64_t)gn * M] = v;
          } else {
            double* cp = C + (int64_t)gm + (int64_t)gn * ldc;
            *cp = (beta == 0.0) ? v : v + beta * *cp;
          }
        }
      }
}

__global__ void splitk_reduce_kernel(int M, int N, int S, const double* __restrict__ part,
                                     double beta, double* __restrict__ C, int64_t ldc,
                                     const int32_t* __restrict__ done) {
  if (done && *done) return;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t MN = (int64_t)M * N;
  if (idx >= MN) return;
  double s = 0.0;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * MN + idx];
  int64_t gm = idx % M, gn = idx / M;
  double* cp = C + gm + gn * ldc;
  *cp = (beta == 0.0) ? s : s + beta * *cp;
}

}  // namespace

int g_num_sms = 152;

cudaError_t gemm_f64(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     double* C, int64_t ldc, double* ws, size_t ws_elems, int64_t* launches,
                     const int32_t* done) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  int gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
  int tiles = gm * gn;
  int S = 1;
  if (K > 0 && ws != nullptr) {
    int want = (2 * g_num_sms + tiles - 1) / tiles;               // about two CTAs per SM
    int maxS = (K + 63) / 64;                                      // keep >= 64 of K per slice
    S = want < maxS ? want : maxS;
    if (S < 1) S = 1;
    if (S > 64) S = 64;
    while (S > 1 && (size_t)S * M * N > ws_elems) --S;
  }
  int kchunk = K > 0 ? ((K + S - 1) / S + BK - 1) / BK * BK : 0;
  if (K > 0) S = (K + kchunk - 1) / kchunk;
  if (K <= 0) {  // C = beta * C
    S = 1;
    kchunk = 0;
  }
  dim3 grid(gm, gn, S);
  gemm_f64_kernel<<<grid, THREADS, 0, st>>>(M, N, K, kchunk, alpha, A, lda, tA ? 1 : 0, B, ldb,
                                            tB ? 1 : 0, beta, C, ldc, ws, done);
  if (launches) ++*launches;
  if (S > 1) {
    int64_t MN = (int64_t)M * N;
    splitk_reduce_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(M, N, S, ws, beta, C, ldc, done);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace wc

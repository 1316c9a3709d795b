// FP32 GEMM with FP32 FMA (about 73 TFLOP/s on GB300), column-major operands; used by the
// inner solve of the mixed-precision form.  Same conventions and split-K scheme as gemm_f64:
//   C (M x N) = alpha * op(A) * op(B) + beta * C.
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int THREADS = 256;

// Each thread owns a TM x TN block of C; K advances in steps of BK with the next step's
// tiles prefetched into registers while the current one is multiplied (the small products
// of the mixed form are latency-bound, so few, long K steps matter more than tile reuse).
template <int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__(THREADS)
gemm_f32_kernel(int M, int N, int K, int kchunk, float alpha, const float* __restrict__ A, int64_t lda, int tA,
                const float* __restrict__ B, int64_t ldb, int tB, float beta, float* __restrict__ C, int64_t ldc,
                float* __restrict__ part, const int32_t* __restrict__ done) {
  static_assert((BM / TM) * (BN / TN) == THREADS, "thread layout");
  constexpr int A_PER = (BM * BK + THREADS - 1) / THREADS, B_PER = (BN * BK + THREADS - 1) / THREADS;
  if (done && *done) return;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tid = threadIdx.x;
  const int ty = tid % (BM / TM), tx = tid / (BM / TM);
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  float ra[A_PER], rb[B_PER];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int idx = tid + e * THREADS;
      int mi, ki;
      if (!tA) { mi = idx % BM; ki = idx / BM; } else { ki = idx % BK; mi = idx / BK; }
      const int gm = m0 + mi, gk = k0 + ki;
      float v = 0.f;
      if (idx < BM * BK && gm < M && gk < kend)
        v = tA ? A[(int64_t)gk + (int64_t)gm * lda] : A[(int64_t)gm + (int64_t)gk * lda];
      ra[e] = v;
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = tid + e * THREADS;
      int ni, kj;
      if (!tB) { kj = idx % BK; ni = idx / BK; } else { ni = idx % BN; kj = idx / BN; }
      const int gn = n0 + ni, gk = k0 + kj;
      float w = 0.f;
      if (idx < BN * BK && gn < N && gk < kend)
        w = tB ? B[(int64_t)gn + (int64_t)gk * ldb] : B[(int64_t)gk + (int64_t)gn * ldb];
      rb[e] = w;
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int idx = tid + e * THREADS;
      if (idx >= BM * BK) break;
      int mi, ki;
      if (!tA) { mi = idx % BM; ki = idx / BM; } else { ki = idx % BK; mi = idx / BK; }
      As[ki][mi] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = tid + e * THREADS;
      if (idx >= BN * BK) break;
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
      if (k0 + BK < kend) load_tiles(k0 + BK);
#pragma unroll 8
      for (int kk = 0; kk < BK; ++kk) {
        float a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  const bool split = gridDim.z > 1;
  float* P = split ? part + (int64_t)blockIdx.z * M * N : nullptr;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gm = m0 + ty * TM + i, gn = n0 + tx * TN + j;
      if (gm < M && gn < N) {
        float v = alpha * acc[i][j];
        if (split) P[(int64_t)gm + (int64_t)gn * M] = v;
        else {
          float* cp = C + (int64_t)gm + (int64_t)gn * ldc;
          *cp = (beta == 0.f) ? v : v + beta * *cp;
        }
      }
    }
}

__global__ void splitk_reduce_f32_kernel(int M, int N, int S, const float* __restrict__ part, float beta,
                                         float* __restrict__ C, int64_t ldc, const int32_t* __restrict__ done) {
  if (done && *done) return;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t MN = (int64_t)M * N;
  if (idx >= MN) return;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * MN + idx];
  int64_t gm = idx % M, gn = idx / M;
  float* cp = C + gm + gn * ldc;
  *cp = (beta == 0.f) ? s : s + beta * *cp;
}

template <int BM, int BN, int TM, int TN, int BK>
cudaError_t launch(cudaStream_t st, bool tA, bool tB, int M, int N, int K, float alpha, const float* A, int64_t lda,
                   const float* B, int64_t ldb, float beta, float* C, int64_t ldc, float* ws, size_t ws_elems,
                   int64_t* launches, const int32_t* done) {
  int gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
  int tiles = gm * gn;
  int S = 1;
  if (K > 0 && ws != nullptr) {
    int want = (2 * g_num_sms + tiles - 1) / tiles;
    int maxS = K / 256;                           // split only long products
    S = want < maxS ? want : maxS;
    if (S < 1) S = 1;
    if (S > 64) S = 64;
    while (S > 1 && (size_t)S * M * N > ws_elems) --S;
  }
  int kchunk = K > 0 ? ((K + S - 1) / S + BK - 1) / BK * BK : 0;
  if (K > 0) S = (K + kchunk - 1) / kchunk;
  if (K <= 0) { S = 1; kchunk = 0; }
  dim3 grid(gm, gn, S);
  gemm_f32_kernel<BM, BN, TM, TN, BK><<<grid, THREADS, 0, st>>>(M, N, K, kchunk, alpha, A, lda, tA ? 1 : 0, B, ldb,
                                                           tB ? 1 : 0, beta, C, ldc, ws, done);
  if (launches) ++*launches;
  if (S > 1) {
    int64_t MN = (int64_t)M * N;
    splitk_reduce_f32_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(M, N, S, ws, beta, C, ldc, done);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_f32(cudaStream_t st, bool tA, bool tB, int M, int N, int K, float alpha, const float* A,
                     int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, float* ws,
                     size_t ws_elems, int64_t* launches, const int32_t* done) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (N <= 8)
    return launch<256, 8, 2, 4, 32>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                                   done);
  if ((int64_t)M * N <= 512 * 512)
    return launch<32, 32, 2, 2, 64>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                                    done);
  return launch<64, 64, 4, 4, 16>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                                  done);
}

}  // namespace wc

// FP64 GEMM on the FP64 MMA path (mma.sync m8n8k4 f64), column-major operands.
//
//   C (M x N) = alpha * op(A) * op(B) + beta * C
//
// op(A) is M x K (A col-major M x K, or its transpose stored K x M); op(B) is K x N.
// On GB300 this MMA issues to the same FP64 pipe as FMA (about 1.1-1.2 TFLOP/s either way);
// it is used for its operand reuse (fewer shared-memory reads per flop).  The dense products
// of the Newton solve range from n ~ 200 to n ~ 5000, so four tile shapes are compiled
// (64 x 64 for large products, 32 x 32 and 16 x 16 with long K steps for n ~ 200-500,
// 32 x 8 for the n x r factors) and the grid is filled by splitting a long K across CTAs
// when the M x N tile count is small; the K-slices write partial tiles to scratch and the
// last slice of each tile adds them in a fixed order (results are bitwise reproducible).
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int THREADS = 128;        // 4 warps
constexpr int kGemmTickets = 4096;  // split-K tickets (tiles) at most
constexpr size_t kGemmTicketDoubles = kGemmTickets / 2;
constexpr int PAD = 4;              // row stride BM+4 doubles: conflict-free fragment reads

// Warp layout WARPS_M x WARPS_N (= 4); each warp owns a (BM/WARPS_M) x (BN/WARPS_N) block of
// 8 x 8 MMA tiles.
template <int BM, int BN, int WARPS_M, int BK>
__global__ void __launch_bounds__(THREADS)
gemm_f64_kernel(int M, int N, int K, int kchunk, double alpha,
                const double* __restrict__ A, int64_t lda, int tA,
                const double* __restrict__ B, int64_t ldb, int tB,
                double beta, double* __restrict__ C, int64_t ldc,
                double* __restrict__ part, unsigned int* __restrict__ counters, int flags,
                const int32_t* __restrict__ done) {
  constexpr int WARPS_N = 4 / WARPS_M;
  constexpr int WM = BM / WARPS_M, WN = BN / WARPS_N;
  constexpr int TM = WM / 8, TN = WN / 8;
  constexpr int A_PER = BM * BK / THREADS, B_PER = BN * BK / THREADS;
  static_assert(TM >= 1 && TN >= 1 && A_PER >= 1 && B_PER >= 1, "tile shape");
  if (done && *done) return;
  __shared__ double As[BK][BM + PAD];
  __shared__ double Bs[BK][BN + PAD];

  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if ((flags & GEMM_LOWER) && m0 + BM <= n0) return;      // tile entirely above the diagonal
  int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  if (flags & GEMM_KSTART_ROW) kbeg = max(kbeg, m0);       // op(A)[i, k] = 0 for k < i
  if (flags & GEMM_KSTART_COL) kbeg = max(kbeg, n0);       // op(B)[k, j] = 0 for k < j
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp % WARPS_M) * WM, wn = (warp / WARPS_M) * WN;
  const int g = lane >> 2, t = lane & 3;

  double acc[TM][TN][2];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  double ra[A_PER], rb[B_PER];
  auto a_idx = [&](int e, int& mi, int& ki) {
    int idx = tid + e * THREADS;
    if (!tA) { mi = idx % BM; ki = idx / BM; } else { ki = idx % BK; mi = idx / BK; }
  };
  auto b_idx = [&](int e, int& ni, int& kj) {
    int idx = tid + e * THREADS;
    if (!tB) { kj = idx % BK; ni = idx / BK; } else { ni = idx % BN; kj = idx / BN; }
  };
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      int mi, ki;
      a_idx(e, mi, ki);
      int gm = m0 + mi, gk = k0 + ki;
      double v = 0.0;
      if (gm < M && gk < kend) v = tA ? A[(int64_t)gk + (int64_t)gm * lda] : A[(int64_t)gm + (int64_t)gk * lda];
      ra[e] = v;
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      int ni, kj;
      b_idx(e, ni, kj);
      int gn = n0 + ni, gk = k0 + kj;
      double w = 0.0;
      if (gn < N && gk < kend) w = tB ? B[(int64_t)gn + (int64_t)gk * ldb] : B[(int64_t)gk + (int64_t)gn * ldb];
      rb[e] = w;
    }
  };
  auto store_tiles = [&]() {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      int mi, ki;
      a_idx(e, mi, ki);
      As[ki][mi] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      int ni, kj;
      b_idx(e, ni, kj);
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
        double af[TM], bf[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) af[i] = As[kk + t][wm + i * 8 + g];
#pragma unroll
        for (int j = 0; j < TN; ++j) bf[j] = Bs[kk + t][wn + j * 8 + g];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) dmma_8x8x4(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
      }
      __syncthreads();
    }
  }

  // Epilogue: c0 = C[g][2t], c1 = C[g][2t+1] within each 8 x 8 tile.  With K split over
  // gridDim.z slices, every slice writes its partial tile; the last slice to finish (atomic
  // ticket per tile) adds the partials in slice order, so the result does not depend on
  // which slice finished last, and resets the ticket for the next product.
  const bool split = (gridDim.z > 1);
  double* P = split ? part + (int64_t)blockIdx.z * M * N : nullptr;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
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
  if (!split) return;
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  unsigned int* ticket = counters + (blockIdx.x + (int64_t)blockIdx.y * gridDim.x);
  if (tid == 0) last = (atomicAdd(ticket, 1u) == gridDim.z - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int64_t MN = (int64_t)M * N;
  for (int e = tid; e < BM * BN; e += THREADS) {
    const int gm = m0 + e % BM, gn = n0 + e / BM;
    if (gm >= M || gn >= N) continue;
    const int64_t idx = (int64_t)gm + (int64_t)gn * M;
    double sum = 0.0;
    for (int z = 0; z < (int)gridDim.z; ++z) sum += __ldcg(part + z * MN + idx);
    double* cp = C + (int64_t)gm + (int64_t)gn * ldc;
    *cp = (beta == 0.0) ? sum : sum + beta * *cp;
  }
  if (tid == 0) *ticket = 0u;
}

// CPS: CTAs per SM the K split aims for (more for the large tile, whose CTAs are few and long)
template <int BM, int BN, int WARPS_M, int BK, int CPS = 2>
cudaError_t launch(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                   int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, double* ws,
                   size_t ws_elems, int64_t* launches, int flags, const int32_t* done) {
  int gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
  int tiles = gm * gn;
  if (flags & GEMM_LOWER) tiles = (tiles + gm) / 2;                // about half the tiles do work
  int S = 1;
  // the last kGemmTickets doubles of ws hold the per-tile tickets of the split-K reduction
  const size_t part_elems = ws_elems > kGemmTicketDoubles ? ws_elems - kGemmTicketDoubles : 0;
  if (K > 0 && ws != nullptr && gm * gn <= kGemmTickets) {
    int want = (CPS * g_num_sms + tiles - 1) / tiles;             // about CPS CTAs per SM
    int maxS = K / (2 * BK);                                       // at least two K steps per slice
    S = want < maxS ? want : maxS;
    if (S < 1) S = 1;
    if (S > 64) S = 64;
    while (S > 1 && (size_t)S * M * N > part_elems) --S;
  }
  int kchunk = K > 0 ? ((K + S - 1) / S + BK - 1) / BK * BK : 0;
  if (K > 0) S = (K + kchunk - 1) / kchunk;
  if (K <= 0) { S = 1; kchunk = 0; }
  unsigned int* tickets = ws ? reinterpret_cast<unsigned int*>(ws + part_elems) : nullptr;
  dim3 grid(gm, gn, S);
  gemm_f64_kernel<BM, BN, WARPS_M, BK><<<grid, THREADS, 0, st>>>(M, N, K, kchunk, alpha, A, lda, tA ? 1 : 0, B, ldb,
                                                                tB ? 1 : 0, beta, C, ldc, ws, tickets, flags, done);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace

int g_num_sms = 152;

cudaError_t raise_dyn_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> limit;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limit[func];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t gemm_f64(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     double* C, int64_t ldc, double* ws, size_t ws_elems, int64_t* launches,
                     const int32_t* done, int flags) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (N <= 8)   // the n x r factors: short tiles, K split over many CTAs
    return launch<32, 8, 4, 16>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                                flags, done);
  if ((int64_t)M * N <= 320 * 320)   // one 8 x 8 MMA tile per warp, long K steps: few, latency-bound steps
    return launch<16, 16, 2, 64>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                                 flags, done);
  if ((int64_t)M * N <= 512 * 512)
    return launch<32, 32, 2, 32>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                                 flags, done);
  return launch<64, 64, 2, 16, 6>(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, launches,
                               flags, done);
}

}  // namespace wc

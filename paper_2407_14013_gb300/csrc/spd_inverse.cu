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
#include <string>
#include <cooperative_groups.h>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace wc {

namespace {

constexpr int NB = 32;

// 1/v for a positive normal v by Newton's iteration for the reciprocal, r <- r + r (1 - v r), from
// a seed built without FP64 arithmetic: the FP32 reciprocal of v's leading 24 significand bits
// (rcp.approx, relative error about 2^-22 with the truncation), with v's exponent applied to it in
// the integer domain.  Two steps bring the error to the FP64 rounding level (within an ulp or so;
// exact when 1/v is a power of two).  On GB300 every FP64 operation carries a long latency, and a
// pivot's reciprocal sits on the critical path of the one-CTA factorisation below: four dependent
// FMAs are much shorter than a full-precision division.  Pivots with exponents near the ends of the
// range take the division.
__device__ __forceinline__ double recip_newton(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 4 || e > 2040) return 1.0 / v;
  const float mant = __int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF));   // in [1, 2)
  float rm;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rm) : "f"(mant));                      // in (0.5, 1]
  const int fb = __float_as_int(rm);
  const long long de = (long long)(((fb >> 23) & 0xFF) - 127 + 2046 - e);     // exponent of rm 2^(1023 - e)
  double r = __longlong_as_double((de << 52) | ((long long)(fb & 0x7FFFFF) << 29) | (b & (1ll << 63)));
  double q = fma(-v, r, 1.0);
  r = fma(r, q, r);
  q = fma(-v, r, 1.0);
  return fma(r, q, r);
}

// A pivot is usable when it is positive and finite; tested on its bits (integer operations), so
// the check stays off the FP64 pipe.
__device__ __forceinline__ bool pivot_ok(double v) {
  const long long b = __double_as_longlong(v);
  return b > 0 && ((b >> 52) & 0x7FF) != 0x7FF;
}

// Factor the w x w diagonal block at k0 (already updated by earlier blocks): L_KK into the
// lower triangle of A (upper part of the block zeroed), its inverse into Li.
//
// GB300 issues FP64 arithmetic at 2 lane-operations per SM per clock and a warp instruction
// costs its full width even with lanes masked off, so this routine, which runs on one SM,
// enumerates exactly the active entries of each step.  Step p (one barrier) does
//   the LDL^T update S_ij -= l_i S_jp (p < j <= i) and the inverse sweep X~_ij -= l_i X~_pj
//   (i > p >= j), with l_i = S_ip / S_pp formed by each thread from the pivot's reciprocal,
// so that X~ = L~^{-1} for the unit lower factor L~ = [l]; then L = L~ D^{1/2} and
// L^{-1} = D^{-1/2} X~ with D = diag(S_pp).  The step's latency is the chain of the next pivot
// (its update, its reciprocal), so the lower pairs are tabled column by column: the pairs of
// step p are a suffix of the table whose first entry is the next pivot (p+1, p+1), and thread 0
// takes it first while the rest of the step runs.
//
// Li gets L_KK^{-1} with leading dimension ldl; X2 (may be NULL) a second copy with ldx2.  A is
// read through L2 (another CTA of a cooperative launch may have just written the block).  Every
// thread of the block calls it (block-wide barriers inside).
__device__ void chol_block_dev(int64_t n, int k0, int w, double* __restrict__ A, double* __restrict__ Li,
                               int64_t ldl, double* __restrict__ X2, int64_t ldx2, int32_t* __restrict__ status) {
  __shared__ double S[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  __shared__ double inv[NB], dsq[NB], rdsq[NB];
  __shared__ unsigned char ti[NB * (NB + 1) / 2], tj[NB * (NB + 1) / 2];
  __shared__ int bad;
  const int ww = w * w;
  for (int q = threadIdx.x; q < ww; q += blockDim.x) {
    const int i = q % w, j = q / w;
    S[i][j] = __ldcg(A + (k0 + i) + (int64_t)(k0 + j) * n);
    X[i][j] = (i == j) ? 1.0 : 0.0;
    if (i >= j) {                          // column j starts at off(j) = j w - j (j - 1) / 2
      const int pos = j * w - j * (j - 1) / 2 + (i - j);
      ti[pos] = (unsigned char)i;
      tj[pos] = (unsigned char)j;
    }
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double piv = S[0][0];
    const bool ok = pivot_ok(piv);
    if (!ok) bad = 1;
    inv[0] = ok ? recip_newton(piv) : 1.0;
  }
  __syncthreads();
  for (int p = 0; p < w - 1; ++p) {
    const int k = w - 1 - p;
    const double ip = inv[p];
    const int start = (p + 1) * w - (p + 1) * p / 2;   // off(p + 1)
    const int cnt_a = k * (k + 1) / 2;                 // pairs with j > p
    const int cnt = cnt_a + k * (p + 1);               // plus the k x (p + 1) block of the sweep
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      if (t < cnt_a) {
        const int i = ti[start + t], j = tj[start + t];
        const double v = fma(-(S[i][p] * ip), S[j][p], S[i][j]);
        S[i][j] = v;
        if (t == 0) {                      // (p+1, p+1): the next pivot is final now
          const bool ok = pivot_ok(v);
          if (!ok) bad = 1;
          inv[p + 1] = ok ? recip_newton(v) : 1.0;
        }
      } else {
        const int u = t - cnt_a;
        const int i = p + 1 + u % k, j = u / k;
        X[i][j] = fma(-(S[i][p] * ip), X[p][j], X[i][j]);
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
    Li[i + (int64_t)j * ldl] = x;
    if (X2) X2[i + (int64_t)j * ldx2] = x;
  }
  if (threadIdx.x == 0 && bad) *status = 5;
  __syncthreads();   // the shared arrays may be reused by the caller's next call
}

__global__ void __launch_bounds__(256)
chol_block_kernel(int n, int k0, int w, double* __restrict__ A, double* __restrict__ Li,
                  int32_t* __restrict__ status) {   // n: leading dimension of A
  chol_block_dev(n, k0, w, A, Li, w, nullptr, 0, status);
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

// ---- the whole factorisation in one cooperative launch (n <= kCoopMax)
//
// The chain above is ~7 launches per 32-wide block column, most of them small and serial.  Here
// every CTA of a GPU-filling cooperative grid takes part in each step k (one 32-wide block column),
// and the three triangular parts of the inverse advance together, right-looking:
//   phase B(k):  L_ik = A_ik L_kk^{-T} (panel, i > k);  X_kj = L_kk^{-1} T_kj (j < k), X_kk = L_kk^{-1}
//   phase C(k):  A_ij -= L_ik L_jk^T    (i >= j > k: the Cholesky's trailing update)
//                T_ij -= L_ik X_kj      (i > k >= j: block forward substitution for X = L^{-1})
//                Ainv_ij += X_ki^T X_kj (k >= i >= j: Ainv = X^T X = sum over block rows k)
// with a grid barrier after each phase.  X_kj is final after B(k), so C(k) can use it at once; the
// block rows of Ainv live in the tiles (i, j), i <= k, whose L is no longer read.  Every phase C
// holds the same number of 32 x 32 x 32 tile products, n_b (n_b + 1) / 2 for n_b block columns,
// cut into four 8-row units each.  CTA 0 takes the diagonal tile (k+1, k+1) and factors it
// (one-CTA kernel above) while the others update the rest, so the next step's pivot block is
// ready at the barrier.  FP64 work: n^3 / 2 multiply-adds, as for the chain.
constexpr int kCoopMax = 1024;

struct CoopSmem {
  double P[NB][NB + 1];
  double Q[NB][NB + 1];
};

__device__ __forceinline__ int blk_w(int n, int b) { return min(NB, n - NB * b); }

// C (R x Cc) (= or +=) sign * P Q with P (R x NB) and Q (NB x Cc) read from column-major memory,
// directly (P[r + k ld]) or transposed (P[k + r ld]).  Entries of P outside (pr, pk) and of Q
// outside (pk, qc) read as zero; outputs outside (pr, qc) are not written.  R Cc == blockDim.x.
// C may alias P (row units, R < NB) or Q (column units): each unit reads all its inputs before it
// writes, and no other unit of the phase touches those rows (columns).
__device__ void tile_unit(CoopSmem& sm, int R, int Cc, const double* P, int64_t ldp, bool pT, int pr, int pk,
                          const double* Q, int64_t ldq, bool qT, int qc, double* C, int64_t ldc, double sign,
                          bool accumulate) {
  const int t = threadIdx.x;
  // every load of the unit issued before any is stored (R NB, NB Cc <= 4 blockDim.x): one L2
  // round trip instead of one per entry a thread stages
  double pv[4], qv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = t + u * (int)blockDim.x;
    pv[u] = 0.0;
    if (idx < R * NB) {
      int r, k;
      if (pT) { k = idx % NB; r = idx / NB; } else { r = idx % R; k = idx / R; }
      if (r < pr && k < pk) pv[u] = pT ? P[k + (int64_t)r * ldp] : P[r + (int64_t)k * ldp];
    }
    qv[u] = 0.0;
    if (idx < NB * Cc) {
      int k, c;
      if (qT) { c = idx % Cc; k = idx / Cc; } else { k = idx % NB; c = idx / NB; }
      if (k < pk && c < qc) qv[u] = qT ? Q[c + (int64_t)k * ldq] : Q[k + (int64_t)c * ldq];
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = t + u * (int)blockDim.x;
    if (idx < R * NB) {
      int r, k;
      if (pT) { k = idx % NB; r = idx / NB; } else { r = idx % R; k = idx / R; }
      sm.P[r][k] = pv[u];
    }
    if (idx < NB * Cc) {
      int k, c;
      if (qT) { c = idx % Cc; k = idx / Cc; } else { k = idx % NB; c = idx / NB; }
      sm.Q[k][c] = qv[u];
    }
  }
  __syncthreads();
  {
    // four independent FMA chains: on GB300 a dependent FP64 FMA waits about 140 clocks, so one
    // chain of 32 would set the time of the unit
    const int r = t / Cc, c = t % Cc;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int k = 0; k < NB; k += 4) {
      a0 = fma(sm.P[r][k], sm.Q[k][c], a0);
      a1 = fma(sm.P[r][k + 1], sm.Q[k + 1][c], a1);
      a2 = fma(sm.P[r][k + 2], sm.Q[k + 2][c], a2);
      a3 = fma(sm.P[r][k + 3], sm.Q[k + 3][c], a3);
    }
    const double acc = (a0 + a1) + (a2 + a3);
    if (r < pr && c < qc) {
      double* o = C + r + (int64_t)c * ldc;
      *o = accumulate ? fma(sign, acc, *o) : sign * acc;
    }
  }
  __syncthreads();
}

// A_ij -= L_ik L_jk^T, rows 8q.. of block i (A holds L in the finished block columns)
__device__ void unit_trailing(CoopSmem& sm, int n, double* A, int64_t lda, int i, int j, int k, int q) {
  const int pr = min(8, blk_w(n, i) - 8 * q);
  if (pr <= 0) return;
  const int64_t r0 = (int64_t)NB * i + 8 * q;
  tile_unit(sm, 8, NB, A + r0 + (int64_t)NB * k * lda, lda, false, pr, blk_w(n, k),
            A + (int64_t)NB * j + (int64_t)NB * k * lda, lda, true, blk_w(n, j),
            A + r0 + (int64_t)NB * j * lda, lda, -1.0, true);
}

// Wait (thread 0) until *c >= target, at most limit_ns of %globaltimer time; false on expiry.
// The count is raised by other CTAs of the same cooperative launch, all resident by construction,
// so the wait ends after one tile unit; the bound only keeps a fault elsewhere from hanging here.
constexpr unsigned long long kFlagWaitNs = 2000000000ull;
__device__ bool wait_count(const unsigned int* c, unsigned int target, unsigned long long limit_ns) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (*(volatile const unsigned int*)c >= target) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
    __nanosleep(64);
  }
}

// The four units of the tiles above, by kind, and the step's barriers.
__global__ void __launch_bounds__(256)
spd_coop_kernel(int n, double* __restrict__ A, int64_t lda, double* __restrict__ X, int64_t ldx,
                double* __restrict__ Li, int inv, int32_t* __restrict__ status, unsigned int* __restrict__ flag) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ CoopSmem sm;
  const int nb = (n + NB - 1) / NB;
  const bool withX = X != nullptr;
  const int G = gridDim.x, b = blockIdx.x;
  if (b == 0) {
    if (threadIdx.x == 0) *flag = 0u;
    chol_block_dev(lda, 0, blk_w(n, 0), A, Li, NB, withX ? X : nullptr, ldx, status);
  }
  grid.sync();
  for (int k = 0; k < nb; ++k) {
    const int wk = blk_w(n, k);
    const int Mc = nb - k - 1;
    const double* Lik = Li + (size_t)k * NB * NB;
    // ---- phase B(k): panel rows (8-row units) and the scaling of block row k of X (8-column units)
    {
      const int Up = 4 * Mc, Ur = withX ? 4 * k : 0;
      for (int u = b; u < Up + Ur; u += G) {
        const int q = u & 3;
        if (u < Up) {
          const int i = k + 1 + (u >> 2);
          const int pr = min(8, blk_w(n, i) - 8 * q);
          if (pr <= 0) continue;
          double* Pik = A + (int64_t)NB * i + 8 * q + (int64_t)NB * k * lda;
          tile_unit(sm, 8, NB, Pik, lda, false, pr, wk, Lik, NB, true, wk, Pik, lda, 1.0, false);
        } else {
          const int j = (u - Up) >> 2;
          const int qc = min(8, blk_w(n, j) - 8 * q);
          if (qc <= 0) continue;
          double* Xkj = X + (int64_t)NB * k + ((int64_t)NB * j + 8 * q) * ldx;
          tile_unit(sm, NB, 8, Lik, NB, false, wk, wk, Xkj, ldx, false, qc, Xkj, ldx, 1.0, false);
        }
      }
    }
    grid.sync();
    // ---- phase C(k)
    if (b == 0) {
      if (Mc > 0) {                          // the next pivot block, once CTAs 1-4 have updated it
        if (threadIdx.x == 0 && !wait_count(flag, 4u * (k + 1), kFlagWaitNs)) *status = 5;
        __syncthreads();
        __threadfence();
        chol_block_dev(lda, NB * (k + 1), blk_w(n, k + 1), A, Li + (size_t)(k + 1) * NB * NB, NB,
                       withX ? X + (int64_t)NB * (k + 1) * (1 + ldx) : nullptr, ldx, status);
      }
    } else {
      const int D = Mc > 0 ? 1 : 0;                          // the tile (k+1, k+1) first
      const int Tc1 = Mc > 0 ? Mc * (Mc + 1) / 2 - 1 : 0;   // the other trailing tiles
      const int Tg = withX ? Mc * (k + 1) : 0;
      const int Tx = inv ? (k + 1) * (k + 2) / 2 : 0;
      const int U = 4 * (D + Tc1 + Tg + Tx);
      for (int u = b - 1; u < U; u += G - 1) {
        const int q = u & 3;
        int t = u >> 2;
        if (t < D) {                         // a quarter of the next pivot block, then its signal
          unit_trailing(sm, n, A, lda, k + 1, k + 1, k, q);
          if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(flag, 1u);
          }
          continue;
        }
        t -= D;
        if (t < Tc1) {
          t += 1;                            // lower-triangle index a (a + 1) / 2 + c of the trailing tiles
          int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
          while (a * (a + 1) / 2 > t) --a;
          while ((a + 1) * (a + 2) / 2 <= t) ++a;
          const int c = t - a * (a + 1) / 2;
          unit_trailing(sm, n, A, lda, k + 1 + a, k + 1 + c, k, q);
          continue;
        }
        t -= Tc1;
        if (t < Tg) {                        // T_ij -= L_ik X_kj (X_kk = L_kk^{-1}: first touch of T_ik)
          const int i = k + 1 + t / (k + 1), j = t % (k + 1);
          const int pr = min(8, blk_w(n, i) - 8 * q);
          if (pr <= 0) continue;
          const int64_t r0 = (int64_t)NB * i + 8 * q;
          tile_unit(sm, 8, NB, A + r0 + (int64_t)NB * k * lda, lda, false, pr, wk,
                    X + (int64_t)NB * k + (int64_t)NB * j * ldx, ldx, false, blk_w(n, j),
                    X + r0 + (int64_t)NB * j * ldx, ldx, -1.0, j < k);
          continue;
        }
        t -= Tg;
        {                                    // Ainv_ij += X_ki^T X_kj (first touch at k == i)
          int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
          while (i * (i + 1) / 2 > t) --i;
          while ((i + 1) * (i + 2) / 2 <= t) ++i;
          const int j = t - i * (i + 1) / 2;
          const int pr = min(8, blk_w(n, i) - 8 * q);
          if (pr <= 0) continue;
          const int64_t r0 = (int64_t)NB * i + 8 * q;
          tile_unit(sm, 8, NB, X + (int64_t)NB * k + r0 * ldx, ldx, true, pr, wk,
                    X + (int64_t)NB * k + (int64_t)NB * j * ldx, ldx, false, blk_w(n, j),
                    A + r0 + (int64_t)NB * j * lda, lda, 1.0, i < k);
        }
      }
    }
    grid.sync();
  }
  // ---- the strict upper triangles: mirrored (inverse) or zeroed (factor)
  const int64_t tot = (int64_t)n * n;
  for (int64_t q = (int64_t)b * blockDim.x + threadIdx.x; q < tot; q += (int64_t)G * blockDim.x) {
    const int r = (int)(q % n), c = (int)(q / n);
    if (r >= c) continue;
    if (inv) A[r + (int64_t)c * lda] = A[c + (int64_t)r * lda];
    else {
      A[r + (int64_t)c * lda] = 0.0;
      if (withX) X[r + (int64_t)c * ldx] = 0.0;
    }
  }
}

int spd_coop_blocks() {
  static int blocks = -1;
  if (blocks < 0) {
    int dev = 0, coop = 0, per = 0, sms = 0;
    blocks = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms >= 2 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, spd_coop_kernel, 256, 0) == cudaSuccess && per > 0)
      blocks = sms;                        // one CTA per SM: the tile products are FP64-pipe bound
    cudaGetLastError();
  }
  return blocks;
}

// One cooperative launch: inv = true: A (lower triangle read) := A^{-1} (full), X (n x n, ld ldx)
// as workspace; inv = false: L into A (upper zeroed) and, with X non-NULL, X = L^{-1}.  Li holds
// ceil(n / 32) 32 x 32 blocks; flag: one word of device scratch.  cudaErrorNotSupported when the
// launch is not possible here.
cudaError_t spd_coop(cudaStream_t st, int n, double* A, int64_t lda, double* X, int64_t ldx, double* Li, bool inv,
                     int32_t* status, unsigned int* flag, int64_t* launches) {
  int blocks = spd_coop_blocks();
  if (blocks <= 0 || n > kCoopMax || n < 1 || (inv && !X)) return cudaErrorNotSupported;
  // no more CTAs than the largest phase C has units for (CTA 0 factors the pivot blocks, the others
  // take the units): the barriers are shorter, and at small n most SMs stay free for the work on
  // other streams (the right side's products beside the preconditioner setup)
  {
    const int nb = (n + NB - 1) / NB;
    int units = 0;
    for (int k = 0; k < nb; ++k) {
      const int mc = nb - k - 1;
      const int u = 4 * ((mc > 0 ? 1 : 0) + (mc > 0 ? mc * (mc + 1) / 2 - 1 : 0) + (X ? mc * (k + 1) : 0) +
                         (inv ? (k + 1) * (k + 2) / 2 : 0));
      units = std::max(units, std::max(u, 4 * (nb - k - 1) + (X ? 4 * k : 0)));   // phases C and B
    }
    blocks = std::min(blocks, std::max(16, units + 1));
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int iv = inv ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, spd_coop_kernel, n, A, lda, X, ldx, Li, iv, status, flag);
  if (e == cudaSuccess && launches) ++*launches;
  return e;
}

}  // namespace

// A (n x n, ld n) is overwritten with its inverse.  work must hold spd_inverse_work(n) doubles.
cudaError_t spd_inverse(cudaStream_t st, int n, double* A, double* work, size_t work_elems,
                        double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches,
                        bool allow_coop) {
  if (spd_inverse_work(n) > work_elems) return cudaErrorInvalidValue;
  double* X = work;                                   // n x n, becomes L^{-1}
  double* T = X + (size_t)n * n;                      // n x NB panel
  double* U = T + (size_t)n * NB;                     // NB x n temporary
  double* Li = U + (size_t)n * NB;                    // inverses of the diagonal blocks
  if (allow_coop && n <= kCoopMax &&
      spd_coop(st, n, A, n, X, n, Li, true, status, reinterpret_cast<unsigned int*>(T), launches) == cudaSuccess)
    return cudaSuccess;
  cudaGetLastError();
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
                           size_t gemm_ws_elems, const TcCtx* tc, int32_t* status, int64_t* launches,
                           bool allow_coop) {
  if (spd_inverse_tc_work(n) > work_elems) return cudaErrorInvalidValue;
  if (n < 2 * NB2) {   // one level of 32-wide panels; only X^T X on the tensor cores
    double* X = work;
    double* T = X + (size_t)n * n;
    double* U = T + (size_t)n * NB;
    double* Li = U + (size_t)n * NB;
    if (allow_coop && n <= kCoopMax &&
        spd_coop(st, n, A, n, X, n, Li, true, status, reinterpret_cast<unsigned int*>(T), launches) == cudaSuccess)
      return cudaSuccess;
    cudaGetLastError();
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
    // L_KK and L_KK^{-1}: one cooperative launch, else the chain of one-CTA 32 x 32 blocks
    if (!(allow_coop && spd_coop(st, w, A + k0 + (int64_t)k0 * n, n, Xb, NB2, Li, false, status,
                                     reinterpret_cast<unsigned int*>(Ti), launches) ==
                            cudaSuccess)) {
      cudaGetLastError();
      e = cholesky_and_inverse(st, w, n, A + k0 + (int64_t)k0 * n, Xb, NB2, Ti, Ui, Li, gemm_ws, gemm_ws_elems,
                               status, launches);
      if (e != cudaSuccess) return e;
    }
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
                         double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches,
                         bool allow_coop) {
  if (spd_inverse_work(n) > work_elems) return cudaErrorInvalidValue;
  double* T = work + (size_t)n * n;
  double* U = T + (size_t)n * NB;
  double* Li = U + (size_t)n * NB;
  if (allow_coop && n <= kCoopMax &&
      spd_coop(st, n, A, n, Linv, n, Li, false, status, reinterpret_cast<unsigned int*>(T), launches) == cudaSuccess)
    return cudaSuccess;
  cudaGetLastError();
  return cholesky_and_inverse(st, n, n, A, Linv, n, T, U, Li, gemm_ws, gemm_ws_elems, status, launches);
}

}  // namespace wc

// ---- C-ABI entry point (tests and callers with their own SPD matrices)

extern "C" size_t sdp_spd_inverse_work_bytes(int32_t n) {
  if (n < 1) return 256;
  return 256 + wc::spd_inverse_work(n) * sizeof(double);
}

extern "C" sdp_status sdp_spd_inverse(void* stream, int32_t n, double* A, double* Linv, int32_t mode, int32_t coop,
                                      void* work, size_t work_bytes) {
  using namespace wc;
  if (n < 0 || (mode != 0 && mode != 1)) return wc_fail(nullptr, SDP_EINVAL, "bad size or mode");
  if (n == 0) return SDP_OK;
  if (!A || !work) return wc_fail(nullptr, SDP_EINVAL, "NULL array argument");
  if (work_bytes < sdp_spd_inverse_work_bytes(n)) return wc_fail(nullptr, SDP_EINVAL, "work too small");
  if ((reinterpret_cast<uintptr_t>(work) & 255u) != 0) return wc_fail(nullptr, SDP_EINVAL, "work not 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* status = static_cast<int32_t*>(work);
  double* w = reinterpret_cast<double*>(static_cast<char*>(work) + 256);
  const size_t we = spd_inverse_work(n);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (e == cudaSuccess)
    e = mode == 0 ? spd_inverse(st, n, A, w, we, nullptr, 0, status, nullptr, coop != 0)
                  : spd_cholesky(st, n, A, Linv, w, we, nullptr, 0, status, nullptr, coop != 0);
  int32_t h_status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, std::string("spd inverse: ") + cudaGetErrorString(e));
  if (h_status) return wc_fail(nullptr, SDP_ENUMERIC, "a pivot of the Cholesky factorisation is not positive");
  return SDP_OK;
}

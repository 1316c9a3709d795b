// Products with a row-major FP64 matrix streamed from memory: y = A x and y = A^T p.
//
// These carry the dense constraint operator A (rows svec(A_i), eq. sdp-pd / A3):
// A(Z) = [<svec A_i, svec Z>]_i and svec(A^T(y)) = sum_i y_i svec(A_i); and the
// preconditioner's B = A Q and C^{-1} products.  Both are bandwidth-bound (one FMA per
// 8-byte element), so each kernel streams every element exactly once with 16-byte loads
// where the row alignment allows, keeps the small vector operand in shared memory or L1,
// and writes per-slab / per-row-group partial sums that the consumer kernel reduces in
// a fixed order.  The large operand A is loaded with an evict-first L2 policy so that the
// L2-resident operands (B, C^{-1}, the n x n work matrices) survive the stream.
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int GV_SLAB = 2048;           // doubles of x per CTA (16 KB of shared memory)
constexpr int GV_WARPS = 8;
constexpr int GV_ROWS_PER_WARP = 4;
constexpr int GV_ROWS = GV_WARPS * GV_ROWS_PER_WARP;

template <bool VEC, bool STREAM>
__global__ void __launch_bounds__(GV_WARPS * 32)
rows_gemv_kernel(const double* __restrict__ A, int m, int64_t L, const double* __restrict__ x,
                 double* __restrict__ part, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  __shared__ __align__(16) double xs[GV_SLAB];
  const int s = blockIdx.x;
  const int64_t k0 = (int64_t)s * GV_SLAB;
  const int len = (int)((L - k0) < (int64_t)GV_SLAB ? (L - k0) : (int64_t)GV_SLAB);
  for (int q = threadIdx.x; q < len; q += blockDim.x) xs[q] = x[k0 + q];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rr = 0; rr < GV_ROWS_PER_WARP; ++rr) {
    const int i = blockIdx.y * GV_ROWS + rr * GV_WARPS + warp;
    if (i >= m) break;
    const double* row = A + (int64_t)i * L + k0;
    double acc = 0.0;
    if (VEC) {
      // row start is 16-byte aligned (L even, base aligned), len even except at the last slab
      const double2* r2 = reinterpret_cast<const double2*>(row);
      const double2* x2 = reinterpret_cast<const double2*>(xs);
      const int np = len >> 1;
      int q = lane;
      for (; q + 96 < np; q += 128) {
        double2 v0 = STREAM ? ld_stream_d2(r2 + q, pol) : __ldg(r2 + q);
        double2 v1 = STREAM ? ld_stream_d2(r2 + q + 32, pol) : __ldg(r2 + q + 32);
        double2 v2 = STREAM ? ld_stream_d2(r2 + q + 64, pol) : __ldg(r2 + q + 64);
        double2 v3 = STREAM ? ld_stream_d2(r2 + q + 96, pol) : __ldg(r2 + q + 96);
        double2 w0 = x2[q], w1 = x2[q + 32], w2 = x2[q + 64], w3 = x2[q + 96];
        acc = fma(v0.x, w0.x, acc); acc = fma(v0.y, w0.y, acc);
        acc = fma(v1.x, w1.x, acc); acc = fma(v1.y, w1.y, acc);
        acc = fma(v2.x, w2.x, acc); acc = fma(v2.y, w2.y, acc);
        acc = fma(v3.x, w3.x, acc); acc = fma(v3.y, w3.y, acc);
      }
      for (; q < np; q += 32) {
        double2 v = STREAM ? ld_stream_d2(r2 + q, pol) : __ldg(r2 + q);
        double2 w = x2[q];
        acc = fma(v.x, w.x, acc); acc = fma(v.y, w.y, acc);
      }
      if ((len & 1) && lane == 0) acc = fma(row[len - 1], xs[len - 1], acc);
    } else {
      int q = lane;
      for (; q + 96 < len; q += 128) {
        double v0 = STREAM ? ld_stream_d(row + q, pol) : __ldg(row + q);
        double v1 = STREAM ? ld_stream_d(row + q + 32, pol) : __ldg(row + q + 32);
        double v2 = STREAM ? ld_stream_d(row + q + 64, pol) : __ldg(row + q + 64);
        double v3 = STREAM ? ld_stream_d(row + q + 96, pol) : __ldg(row + q + 96);
        acc = fma(v0, xs[q], acc); acc = fma(v1, xs[q + 32], acc);
        acc = fma(v2, xs[q + 64], acc); acc = fma(v3, xs[q + 96], acc);
      }
      for (; q < len; q += 32) acc = fma(STREAM ? ld_stream_d(row + q, pol) : __ldg(row + q), xs[q], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) part[(int64_t)s * m + i] = acc;
  }
}

constexpr int GT_THREADS = 256;

template <bool VEC, bool STREAM>
__global__ void __launch_bounds__(GT_THREADS)
rows_gemvT_kernel(const double* __restrict__ A, int m, int64_t L, const double* __restrict__ p,
                  double* __restrict__ part, int rows_per_group, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  const int g = blockIdx.y;
  const int i0 = g * rows_per_group;
  const int i1 = min(m, i0 + rows_per_group);
  if (VEC) {
    const int64_t c = ((int64_t)blockIdx.x * GT_THREADS + threadIdx.x) * 2;
    if (c >= L) return;
    double a0 = 0.0, a1 = 0.0;
    if (c + 1 < L) {
      int i = i0;
      for (; i + 3 < i1; i += 4) {
        const double2* b = reinterpret_cast<const double2*>(A + (int64_t)i * L + c);
        const int64_t st2 = L >> 1;   // rows apart, in double2 units (L even)
        double2 v0 = STREAM ? ld_stream_d2(b, pol) : __ldg(b);
        double2 v1 = STREAM ? ld_stream_d2(b + st2, pol) : __ldg(b + st2);
        double2 v2 = STREAM ? ld_stream_d2(b + 2 * st2, pol) : __ldg(b + 2 * st2);
        double2 v3 = STREAM ? ld_stream_d2(b + 3 * st2, pol) : __ldg(b + 3 * st2);
        double p0 = __ldg(p + i), p1 = __ldg(p + i + 1), p2 = __ldg(p + i + 2), p3 = __ldg(p + i + 3);
        a0 = fma(p0, v0.x, a0); a1 = fma(p0, v0.y, a1);
        a0 = fma(p1, v1.x, a0); a1 = fma(p1, v1.y, a1);
        a0 = fma(p2, v2.x, a0); a1 = fma(p2, v2.y, a1);
        a0 = fma(p3, v3.x, a0); a1 = fma(p3, v3.y, a1);
      }
      for (; i < i1; ++i) {
        const double2* b = reinterpret_cast<const double2*>(A + (int64_t)i * L + c);
        double2 v = STREAM ? ld_stream_d2(b, pol) : __ldg(b);
        double pi = __ldg(p + i);
        a0 = fma(pi, v.x, a0); a1 = fma(pi, v.y, a1);
      }
      part[(int64_t)g * L + c] = a0;
      part[(int64_t)g * L + c + 1] = a1;
    } else {
      for (int i = i0; i < i1; ++i) a0 = fma(__ldg(p + i), A[(int64_t)i * L + c], a0);
      part[(int64_t)g * L + c] = a0;
    }
  } else {
    const int64_t c = (int64_t)blockIdx.x * GT_THREADS + threadIdx.x;
    if (c >= L) return;
    double a0 = 0.0;
    int i = i0;
    for (; i + 3 < i1; i += 4) {
      const double* b = A + (int64_t)i * L + c;
      double v0 = STREAM ? ld_stream_d(b, pol) : __ldg(b);
      double v1 = STREAM ? ld_stream_d(b + L, pol) : __ldg(b + L);
      double v2 = STREAM ? ld_stream_d(b + 2 * L, pol) : __ldg(b + 2 * L);
      double v3 = STREAM ? ld_stream_d(b + 3 * L, pol) : __ldg(b + 3 * L);
      a0 = fma(__ldg(p + i), v0, a0);
      a0 = fma(__ldg(p + i + 1), v1, a0);
      a0 = fma(__ldg(p + i + 2), v2, a0);
      a0 = fma(__ldg(p + i + 3), v3, a0);
    }
    for (; i < i1; ++i) a0 = fma(__ldg(p + i), STREAM ? ld_stream_d(A + (int64_t)i * L + c, pol) : __ldg(A + (int64_t)i * L + c), a0);
    part[(int64_t)g * L + c] = a0;
  }
}

__global__ void sumsq_kernel(const double* __restrict__ A, int64_t total, double* __restrict__ scratch) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    double v = A[q];
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[blockIdx.x] = acc;
}

__global__ void sum_in_order_kernel(const double* __restrict__ scratch, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) acc += scratch[q];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

bool is_vec_ok(const double* A, int64_t L) {
  return (L % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
}

}  // namespace

int rows_gemv_slabs(int64_t L) { return (int)((L + GV_SLAB - 1) / GV_SLAB); }

void rows_gemv(cudaStream_t st, const double* A, int m, int64_t L, const double* x, double* part,
               const int32_t* done, int64_t* launches) {
  dim3 grid(rows_gemv_slabs(L), (m + GV_ROWS - 1) / GV_ROWS);
  const bool stream = (int64_t)m * L * 8 > (int64_t)64 << 20;   // stream only what cannot stay in L2
  if (is_vec_ok(A, L)) {
    if (stream) rows_gemv_kernel<true, true><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
    else rows_gemv_kernel<true, false><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
  } else {
    if (stream) rows_gemv_kernel<false, true><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
    else rows_gemv_kernel<false, false><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
  }
  if (launches) ++*launches;
}

int rows_gemvT_groups(int m, int64_t L) {
  int64_t cols_per_cta = GT_THREADS * 2;
  int64_t ctas = (L + cols_per_cta - 1) / cols_per_cta;
  int64_t want = (4 * (int64_t)g_num_sms + ctas - 1) / ctas;
  int64_t maxg = (m + 31) / 32;
  int64_t g = want < maxg ? want : maxg;
  return (int)(g < 1 ? 1 : g);
}

void rows_gemvT(cudaStream_t st, const double* A, int m, int64_t L, const double* p, double* part,
                int groups, const int32_t* done, int64_t* launches) {
  const int rpg = (m + groups - 1) / groups;
  const bool stream = (int64_t)m * L * 8 > (int64_t)64 << 20;
  if (is_vec_ok(A, L)) {
    dim3 grid((unsigned)((L + 2 * GT_THREADS - 1) / (2 * GT_THREADS)), groups);
    if (stream) rows_gemvT_kernel<true, true><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
    else rows_gemvT_kernel<true, false><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
  } else {
    dim3 grid((unsigned)((L + GT_THREADS - 1) / GT_THREADS), groups);
    if (stream) rows_gemvT_kernel<false, true><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
    else rows_gemvT_kernel<false, false><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
  }
  if (launches) ++*launches;
}

void rows_sumsq(cudaStream_t st, const double* A, int m, int64_t L, double* out, double* scratch,
                int64_t* launches) {
  const int nb = 4 * g_num_sms;
  sumsq_kernel<<<nb, 256, 0, st>>>(A, (int64_t)m * L, scratch);
  sum_in_order_kernel<<<1, 256, 0, st>>>(scratch, nb, out);
  if (launches) *launches += 2;
}

}  // namespace wc

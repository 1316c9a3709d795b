// Products with a row-major matrix streamed from memory: y = A x and y = A^T p, in FP64 or FP32.
//
// These carry the dense constraint operator A (rows svec(A_i), eq. sdp-pd / A3):
// A(Z) = [<svec A_i, svec Z>]_i and svec(A^T(y)) = sum_i y_i svec(A_i); and the
// preconditioner's B = A Q, B^T and complement-inverse products.  Each kernel streams every
// element exactly once with 16-byte loads where the row alignment allows, keeps the small
// vector operand in shared memory or L1, and writes per-slab / per-row-group partial sums
// that the consumer kernel reduces in a fixed order.  A matrix larger than L2 is loaded with
// an evict-first L2 policy so that the L2-resident operands (B, the inverse, the n x n work
// matrices) survive the stream.  In FP64 these kernels are limited by the FP64 FMA rate of
// GB300 (about 1 TFLOP/s: one FMA per 8-byte element caps them near 4 TB/s); in FP32 they
// are limited by HBM.
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int GV_SLAB = 2048;           // elements of x per CTA
constexpr int GV_WARPS = 8;

template <typename T> struct V16;
template <> struct V16<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static type ld(const type* p, uint64_t pol, bool stream) { return stream ? ld_stream_d2(p, pol) : __ldg(p); }
  __device__ static double get(const type& v, int k) { return k == 0 ? v.x : v.y; }
};
template <> struct V16<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static type ld(const type* p, uint64_t pol, bool stream) { return stream ? ld_stream_f4(p, pol) : __ldg(p); }
  __device__ static float get(const type& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }
};

template <typename T>
__device__ __forceinline__ T ld1(const T* p, uint64_t pol, bool stream);
template <>
__device__ __forceinline__ double ld1<double>(const double* p, uint64_t pol, bool stream) {
  return stream ? ld_stream_d(p, pol) : __ldg(p);
}
template <>
__device__ __forceinline__ float ld1<float>(const float* p, uint64_t pol, bool stream) {
  return stream ? ld_stream_f(p, pol) : __ldg(p);
}

// STREAM (a matrix larger than L2): 4 rows per warp, evict-first loads.  Otherwise one row per
// warp, so that the small L2-resident matrices still spread over the whole GPU.
template <typename T, bool VEC, bool STREAM>
__global__ void __launch_bounds__(GV_WARPS * 32)
rows_gemv_kernel(const T* __restrict__ A, int m, int64_t L, const T* __restrict__ x,
                 T* __restrict__ part, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  using VT = V16<T>;
  constexpr int W = VT::W;
  __shared__ __align__(16) T xs[GV_SLAB];
  const int s = blockIdx.x;
  const int64_t k0 = (int64_t)s * GV_SLAB;
  const int len = (int)((L - k0) < (int64_t)GV_SLAB ? (L - k0) : (int64_t)GV_SLAB);
  for (int q = threadIdx.x; q < len; q += blockDim.x) xs[q] = x[k0 + q];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int RPW = STREAM ? 4 : 1;
  for (int rr = 0; rr < RPW; ++rr) {
    const int i = blockIdx.y * (RPW * GV_WARPS) + rr * GV_WARPS + warp;
    if (i >= m) break;
    const T* row = A + (int64_t)i * L + k0;
    T acc = 0;
    if (VEC) {
      // row start is 16-byte aligned (L a multiple of W, base aligned); tail handled below
      const typename VT::type* rv = reinterpret_cast<const typename VT::type*>(row);
      const typename VT::type* xv = reinterpret_cast<const typename VT::type*>(xs);
      const int np = len / W;
      int q = lane;
      for (; q + 96 < np; q += 128) {
        typename VT::type v0 = VT::ld(rv + q, pol, STREAM), v1 = VT::ld(rv + q + 32, pol, STREAM);
        typename VT::type v2 = VT::ld(rv + q + 64, pol, STREAM), v3 = VT::ld(rv + q + 96, pol, STREAM);
        typename VT::type w0 = xv[q], w1 = xv[q + 32], w2 = xv[q + 64], w3 = xv[q + 96];
#pragma unroll
        for (int k = 0; k < W; ++k) {
          acc = fma(VT::get(v0, k), VT::get(w0, k), acc);
          acc = fma(VT::get(v1, k), VT::get(w1, k), acc);
          acc = fma(VT::get(v2, k), VT::get(w2, k), acc);
          acc = fma(VT::get(v3, k), VT::get(w3, k), acc);
        }
      }
      for (; q < np; q += 32) {
        typename VT::type v = VT::ld(rv + q, pol, STREAM), w = xv[q];
#pragma unroll
        for (int k = 0; k < W; ++k) acc = fma(VT::get(v, k), VT::get(w, k), acc);
      }
      for (int t = np * W + lane; t < len; t += 32) acc = fma(row[t], xs[t], acc);
    } else {
      int q = lane;
      for (; q + 96 < len; q += 128) {
        T v0 = ld1<T>(row + q, pol, STREAM), v1 = ld1<T>(row + q + 32, pol, STREAM);
        T v2 = ld1<T>(row + q + 64, pol, STREAM), v3 = ld1<T>(row + q + 96, pol, STREAM);
        acc = fma(v0, xs[q], acc); acc = fma(v1, xs[q + 32], acc);
        acc = fma(v2, xs[q + 64], acc); acc = fma(v3, xs[q + 96], acc);
      }
      for (; q < len; q += 32) acc = fma(ld1<T>(row + q, pol, STREAM), xs[q], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(int64_t)s * m + i] = acc;
  }
}

constexpr int GT_THREADS = 256;

template <typename T, bool VEC, bool STREAM>
__global__ void __launch_bounds__(GT_THREADS)
rows_gemvT_kernel(const T* __restrict__ A, int m, int64_t L, const T* __restrict__ p,
                  T* __restrict__ part, int rows_per_group, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  using VT = V16<T>;
  constexpr int W = VT::W;
  const int g = blockIdx.y;
  const int i0 = g * rows_per_group;
  const int i1 = min(m, i0 + rows_per_group);
  if (VEC) {
    const int64_t c = ((int64_t)blockIdx.x * GT_THREADS + threadIdx.x) * W;
    if (c >= L) return;
    T a[W];
#pragma unroll
    for (int k = 0; k < W; ++k) a[k] = 0;
    const int64_t stv = L / W;   // rows apart, in vector units (L a multiple of W)
    int i = i0;
    for (; i + 3 < i1; i += 4) {
      const typename VT::type* b = reinterpret_cast<const typename VT::type*>(A + (int64_t)i * L + c);
      typename VT::type v0 = VT::ld(b, pol, STREAM), v1 = VT::ld(b + stv, pol, STREAM);
      typename VT::type v2 = VT::ld(b + 2 * stv, pol, STREAM), v3 = VT::ld(b + 3 * stv, pol, STREAM);
      const T p0 = __ldg(p + i), p1 = __ldg(p + i + 1), p2 = __ldg(p + i + 2), p3 = __ldg(p + i + 3);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        a[k] = fma(p0, VT::get(v0, k), a[k]);
        a[k] = fma(p1, VT::get(v1, k), a[k]);
        a[k] = fma(p2, VT::get(v2, k), a[k]);
        a[k] = fma(p3, VT::get(v3, k), a[k]);
      }
    }
    for (; i < i1; ++i) {
      const typename VT::type* b = reinterpret_cast<const typename VT::type*>(A + (int64_t)i * L + c);
      typename VT::type v = VT::ld(b, pol, STREAM);
      const T pi = __ldg(p + i);
#pragma unroll
      for (int k = 0; k < W; ++k) a[k] = fma(pi, VT::get(v, k), a[k]);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) part[(int64_t)g * L + c + k] = a[k];
  } else {
    const int64_t c = (int64_t)blockIdx.x * GT_THREADS + threadIdx.x;
    if (c >= L) return;
    T a0 = 0;
    int i = i0;
    for (; i + 3 < i1; i += 4) {
      const T* b = A + (int64_t)i * L + c;
      T v0 = ld1<T>(b, pol, STREAM), v1 = ld1<T>(b + L, pol, STREAM);
      T v2 = ld1<T>(b + 2 * L, pol, STREAM), v3 = ld1<T>(b + 3 * L, pol, STREAM);
      a0 = fma(__ldg(p + i), v0, a0);
      a0 = fma(__ldg(p + i + 1), v1, a0);
      a0 = fma(__ldg(p + i + 2), v2, a0);
      a0 = fma(__ldg(p + i + 3), v3, a0);
    }
    for (; i < i1; ++i) a0 = fma(__ldg(p + i), ld1<T>(A + (int64_t)i * L + c, pol, STREAM), a0);
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

template <typename T>
bool is_vec_ok(const T* A, int64_t L) {
  return (L % V16<T>::W == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
}

}  // namespace

int rows_gemv_slabs(int64_t L) { return (int)((L + GV_SLAB - 1) / GV_SLAB); }

template <typename T>
void rows_gemv(cudaStream_t st, const T* A, int m, int64_t L, const T* x, T* part, const int32_t* done,
               int64_t* launches) {
  const bool stream = (int64_t)m * L * (int64_t)sizeof(T) > (int64_t)64 << 20;   // stream what cannot stay in L2
  const int rows = (stream ? 4 : 1) * GV_WARPS;
  dim3 grid(rows_gemv_slabs(L), (m + rows - 1) / rows);
  if (is_vec_ok(A, L)) {
    if (stream) rows_gemv_kernel<T, true, true><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
    else rows_gemv_kernel<T, true, false><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
  } else {
    if (stream) rows_gemv_kernel<T, false, true><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
    else rows_gemv_kernel<T, false, false><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, done);
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

template <typename T>
void rows_gemvT(cudaStream_t st, const T* A, int m, int64_t L, const T* p, T* part, int groups,
                const int32_t* done, int64_t* launches) {
  const int rpg = (m + groups - 1) / groups;
  const bool stream = (int64_t)m * L * (int64_t)sizeof(T) > (int64_t)64 << 20;
  if (is_vec_ok(A, L)) {
    constexpr int W = V16<T>::W;
    dim3 grid((unsigned)((L + W * GT_THREADS - 1) / (W * GT_THREADS)), groups);
    if (stream) rows_gemvT_kernel<T, true, true><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
    else rows_gemvT_kernel<T, true, false><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
  } else {
    dim3 grid((unsigned)((L + GT_THREADS - 1) / GT_THREADS), groups);
    if (stream) rows_gemvT_kernel<T, false, true><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
    else rows_gemvT_kernel<T, false, false><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done);
  }
  if (launches) ++*launches;
}

template void rows_gemv<double>(cudaStream_t, const double*, int, int64_t, const double*, double*, const int32_t*,
                                int64_t*);
template void rows_gemv<float>(cudaStream_t, const float*, int, int64_t, const float*, float*, const int32_t*,
                               int64_t*);
template void rows_gemvT<double>(cudaStream_t, const double*, int, int64_t, const double*, double*, int,
                                 const int32_t*, int64_t*);
template void rows_gemvT<float>(cudaStream_t, const float*, int, int64_t, const float*, float*, int, const int32_t*,
                                int64_t*);

void rows_sumsq(cudaStream_t st, const double* A, int m, int64_t L, double* out, double* scratch,
                int64_t* launches) {
  const int nb = 4 * g_num_sms;
  sumsq_kernel<<<nb, 256, 0, st>>>(A, (int64_t)m * L, scratch);
  sum_in_order_kernel<<<1, 256, 0, st>>>(scratch, nb, out);
  if (launches) *launches += 2;
}

}  // namespace wc

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
// GB300 (1.26 TFLOP/s: one FMA per 8-byte element caps them near 5 TB/s); in FP32 they are
// limited by HBM.  Launch shapes are chosen so that the CTAs spread evenly over the SMs.
#include "common.cuh"
#include "fx.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int GV_SWMAX = 4096;          // largest slab of x per CTA (elements)
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

// One CTA: R rows (warp w takes rows w, w + 8, ...; two at a time for memory-level
// parallelism) times one slab of SW columns, whose x segment it stages in shared memory.
// STREAM (a matrix larger than L2) loads A with the evict-first policy.
// Optional prologue of the GEMV: the vector is formed while it is staged,
//   x_k = base_k + c * sum_{g < G} xpart[g * L + k],  c = c0 / *cdiv (or c0 when cdiv is NULL),
// and the CTAs of the first row block also store it to xout (may be NULL).
template <typename T>
struct XForm {
  const T* base;
  const T* xpart;
  int G;
  double c0;
  const double* cdiv;
  T* xout;
};

template <typename T, bool VEC, bool STREAM>
__global__ void __launch_bounds__(GV_WARPS * 32)
rows_gemv_kernel(const T* __restrict__ A, int m, int64_t L, const T* __restrict__ x, T* __restrict__ part,
                 int SW, int R, const int32_t* __restrict__ done, XForm<T> xf) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  using VT = V16<T>;
  using V = typename VT::type;
  constexpr int W = VT::W;
  __shared__ __align__(16) T xs[GV_SWMAX];
  const int s = blockIdx.x;
  const int64_t k0 = (int64_t)s * SW;
  const int len = (int)((L - k0) < (int64_t)SW ? (L - k0) : (int64_t)SW);
  if (xf.xpart) {
    const double cc = xf.cdiv ? xf.c0 / *xf.cdiv : xf.c0;
    for (int q = threadIdx.x; q < len; q += blockDim.x) {
      double t = 0.0;
      for (int gg = 0; gg < xf.G; ++gg) t += (double)xf.xpart[(int64_t)gg * L + k0 + q];
      const T v = (T)((xf.base ? (double)xf.base[k0 + q] : 0.0) + cc * t);
      xs[q] = v;
      if (xf.xout && blockIdx.y == 0) xf.xout[k0 + q] = v;
    }
  } else {
    for (int q = threadIdx.x; q < len; q += blockDim.x) xs[q] = x[k0 + q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = blockIdx.y * R;
  for (int t = warp; t < R; t += 2 * GV_WARPS) {
    const int ia = rbase + t;
    if (ia >= m) break;
    const int ib = rbase + t + GV_WARPS;
    const bool hb = (t + GV_WARPS < R) && (ib < m);
    const T* ra = A + (int64_t)ia * L + k0;
    const T* rb = A + (int64_t)(hb ? ib : ia) * L + k0;
    T acc_a = 0, acc_b = 0;
    if (hb) {   // two rows in flight (warp-uniform branch)
      if (VEC) {
        // row starts are 16-byte aligned (L and SW multiples of W, base aligned); tail below
        const V* va = reinterpret_cast<const V*>(ra);
        const V* vb = reinterpret_cast<const V*>(rb);
        const V* xv = reinterpret_cast<const V*>(xs);
        const int np = len / W;
        int q = lane;
        for (; q + 32 < np; q += 64) {
          V a0 = VT::ld(va + q, pol, STREAM), a1 = VT::ld(va + q + 32, pol, STREAM);
          V b0 = VT::ld(vb + q, pol, STREAM), b1 = VT::ld(vb + q + 32, pol, STREAM);
          V w0 = xv[q], w1 = xv[q + 32];
#pragma unroll
          for (int k = 0; k < W; ++k) {
            acc_a = fma(VT::get(a0, k), VT::get(w0, k), acc_a);
            acc_b = fma(VT::get(b0, k), VT::get(w0, k), acc_b);
            acc_a = fma(VT::get(a1, k), VT::get(w1, k), acc_a);
            acc_b = fma(VT::get(b1, k), VT::get(w1, k), acc_b);
          }
        }
        for (; q < np; q += 32) {
          V a0 = VT::ld(va + q, pol, STREAM), b0 = VT::ld(vb + q, pol, STREAM), w0 = xv[q];
#pragma unroll
          for (int k = 0; k < W; ++k) {
            acc_a = fma(VT::get(a0, k), VT::get(w0, k), acc_a);
            acc_b = fma(VT::get(b0, k), VT::get(w0, k), acc_b);
          }
        }
        for (int c = np * W + lane; c < len; c += 32) {
          acc_a = fma(ra[c], xs[c], acc_a);
          acc_b = fma(rb[c], xs[c], acc_b);
        }
      } else {
        int q = lane;
        for (; q + 32 < len; q += 64) {
          T a0 = ld1<T>(ra + q, pol, STREAM), a1 = ld1<T>(ra + q + 32, pol, STREAM);
          T b0 = ld1<T>(rb + q, pol, STREAM), b1 = ld1<T>(rb + q + 32, pol, STREAM);
          acc_a = fma(a0, xs[q], acc_a); acc_b = fma(b0, xs[q], acc_b);
          acc_a = fma(a1, xs[q + 32], acc_a); acc_b = fma(b1, xs[q + 32], acc_b);
        }
        for (; q < len; q += 32) {
          acc_a = fma(ld1<T>(ra + q, pol, STREAM), xs[q], acc_a);
          acc_b = fma(ld1<T>(rb + q, pol, STREAM), xs[q], acc_b);
        }
      }
    } else {    // a single row: four loads in flight
      if (VEC) {
        const V* va = reinterpret_cast<const V*>(ra);
        const V* xv = reinterpret_cast<const V*>(xs);
        const int np = len / W;
        int q = lane;
        for (; q + 96 < np; q += 128) {
          V a0 = VT::ld(va + q, pol, STREAM), a1 = VT::ld(va + q + 32, pol, STREAM);
          V a2 = VT::ld(va + q + 64, pol, STREAM), a3 = VT::ld(va + q + 96, pol, STREAM);
          V w0 = xv[q], w1 = xv[q + 32], w2 = xv[q + 64], w3 = xv[q + 96];
#pragma unroll
          for (int k = 0; k < W; ++k) {
            acc_a = fma(VT::get(a0, k), VT::get(w0, k), acc_a);
            acc_b = fma(VT::get(a1, k), VT::get(w1, k), acc_b);
            acc_a = fma(VT::get(a2, k), VT::get(w2, k), acc_a);
            acc_b = fma(VT::get(a3, k), VT::get(w3, k), acc_b);
          }
        }
        for (; q < np; q += 32) {
          V a0 = VT::ld(va + q, pol, STREAM), w0 = xv[q];
#pragma unroll
          for (int k = 0; k < W; ++k) acc_a = fma(VT::get(a0, k), VT::get(w0, k), acc_a);
        }
        for (int c = np * W + lane; c < len; c += 32) acc_a = fma(ra[c], xs[c], acc_a);
      } else {
        int q = lane;
        for (; q + 96 < len; q += 128) {
          T a0 = ld1<T>(ra + q, pol, STREAM), a1 = ld1<T>(ra + q + 32, pol, STREAM);
          T a2 = ld1<T>(ra + q + 64, pol, STREAM), a3 = ld1<T>(ra + q + 96, pol, STREAM);
          acc_a = fma(a0, xs[q], acc_a); acc_b = fma(a1, xs[q + 32], acc_b);
          acc_a = fma(a2, xs[q + 64], acc_a); acc_b = fma(a3, xs[q + 96], acc_b);
        }
        for (; q < len; q += 32) acc_a = fma(ld1<T>(ra + q, pol, STREAM), xs[q], acc_a);
      }
      acc_a += acc_b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_a += __shfl_xor_sync(0xffffffffu, acc_a, o);
    if (hb) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc_b += __shfl_xor_sync(0xffffffffu, acc_b, o);
    }
    if (lane == 0) {
      part[(int64_t)s * m + ia] = acc_a;
      if (hb) part[(int64_t)s * m + ib] = acc_b;
    }
  }
}

constexpr int GT_THREADS = 256;

// svec position c -> (a, b), a >= b, of the column-major lower triangle of an n x n matrix
__device__ __forceinline__ void svec_pos(int n, int64_t c, int& a, int& b) {
  const double t = 2.0 * n + 1.0;
  int bb = (int)((t - sqrtf((float)(t * t - 8.0 * (double)c))) * 0.5f);
  if (bb < 0) bb = 0;
  if (bb > n - 1) bb = n - 1;
  while (bb > 0 && (int64_t)bb * n - (int64_t)bb * (bb - 1) / 2 > c) --bb;
  while (bb + 1 < n && (int64_t)(bb + 1) * n - (int64_t)(bb + 1) * bb / 2 <= c) ++bb;
  b = bb;
  a = bb + (int)(c - ((int64_t)bb * n - (int64_t)bb * (bb - 1) / 2));
}

// A^T p over row groups (partial sums part[g * L + c]).  With Y != NULL (UNPACK), the last CTA
// of each column block to finish (atomic ticket) adds the groups' partials in group order and
// writes them as the symmetric n x n matrix smat(.) scaled by `scale` (both triangles), so no
// separate unpack pass is needed.
template <typename T, bool VEC, bool STREAM>
__global__ void __launch_bounds__(GT_THREADS)
rows_gemvT_kernel(const T* __restrict__ A, int m, int64_t L, const T* __restrict__ p,
                  T* __restrict__ part, int rows_per_group, const int32_t* __restrict__ done,
                  int n, double scale, T* __restrict__ Y, unsigned int* __restrict__ tickets) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  using VT = V16<T>;
  constexpr int W = VT::W;
  const int g = blockIdx.y;
  const int i0 = g * rows_per_group;
  const int i1 = min(m, i0 + rows_per_group);
  if (VEC) {
    const int64_t c = ((int64_t)blockIdx.x * GT_THREADS + threadIdx.x) * W;
    if (c < L) {
    T a[W];
#pragma unroll
    for (int k = 0; k < W; ++k) a[k] = 0;
    const int64_t stv = L / W;   // rows apart, in vector units (L a multiple of W)
    int i = i0;
    for (; i + 7 < i1; i += 8) {
      const typename VT::type* b = reinterpret_cast<const typename VT::type*>(A + (int64_t)i * L + c);
      typename VT::type v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = VT::ld(b + u * stv, pol, STREAM);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T pu = __ldg(p + i + u);
#pragma unroll
        for (int k = 0; k < W; ++k) a[k] = fma(pu, VT::get(v[u], k), a[k]);
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
    }
  } else {
    const int64_t c = (int64_t)blockIdx.x * GT_THREADS + threadIdx.x;
    if (c < L) {
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
  if (!Y) return;
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(tickets + blockIdx.x, 1u) == gridDim.y - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the group partials of this CTA's columns (up to four per thread), summed in group order with
  // sixteen loads in flight
  const int per = VEC ? V16<T>::W : 1;
  const int64_t c0 = (int64_t)blockIdx.x * GT_THREADS * per;
  const int G = (int)gridDim.y;
  int64_t cols[4];
  bool has[4];
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    cols[k] = c0 + (int64_t)k * GT_THREADS + threadIdx.x;
    has[k] = (k < per) && (cols[k] < L);
  }
  int gg = 0;
  for (; gg + 3 < G; gg += 4) {
    double v[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[j][k] = has[k] ? (double)__ldcg(part + (int64_t)(gg + j) * L + cols[k]) : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) sum[k] += v[j][k];
  }
  for (; gg < G; ++gg)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (has[k]) sum[k] += (double)__ldcg(part + (int64_t)gg * L + cols[k]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!has[k]) continue;
    int a, b;
    svec_pos(n, cols[k], a, b);
    const T v = (T)((a == b ? sum[k] : sum[k] * WC_RSQRT2) * scale);
    Y[a + (int64_t)b * n] = v;
    Y[b + (int64_t)a * n] = v;
  }
  if (threadIdx.x == 0) tickets[blockIdx.x] = 0u;
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

struct GvPlan {
  int slabs, SW, R;
  bool stream;
};

// Fraction of the busiest SM's share that the average SM does, for `units` equal CTAs.
double balance(int64_t units) {
  const int64_t S = g_num_sms;
  const int64_t per = (units + S - 1) / S;
  return (double)units / (double)(per * S);
}

// Launch shape of y = A x (A m x L of `esize`-byte elements): the slab width and rows per CTA.
// A streamed matrix gets wide slabs and the rows per CTA whose CTA count spreads evenly over
// the SMs; a small one gets one row per warp and enough slabs to cover the GPU.
GvPlan gv_plan(int m, int64_t L, int esize) {
  GvPlan P;
  P.stream = (int64_t)m * L * esize > ((int64_t)64 << 20);
  const int64_t S = g_num_sms;
  if (P.stream) {
    double best = -1.0;
    P.SW = 0; P.R = 0; P.slabs = 0;
    for (int sw : {GV_SWMAX, GV_SWMAX / 2}) {
      const int64_t slabs = (L + sw - 1) / sw;
      for (int R = 16; R <= 64; ++R) {
        const int64_t units = slabs * ((m + R - 1) / R);
        if (units < 4 * S) continue;
        double b = balance(units);
        if (b > best + 1e-9) { best = b; P.SW = sw; P.R = R; P.slabs = (int)slabs; }
      }
    }
    if (P.SW == 0) { P.SW = GV_SWMAX / 2; P.R = 16; P.slabs = (int)((L + P.SW - 1) / P.SW); }
    return P;
  }
  P.R = GV_WARPS;
  const int64_t rb = (m + P.R - 1) / P.R;
  int64_t slabs = (L + 2047) / 2048;
  const int64_t want = 4 * S;
  if (slabs * rb < want) {
    int64_t need = (want + rb - 1) / rb;
    int64_t cap = (L + 127) / 128;
    slabs = need < cap ? need : cap;
    if (slabs < 1) slabs = 1;
  }
  int64_t sw = (L + slabs - 1) / slabs;
  sw = (sw + 3) / 4 * 4;
  P.SW = (int)sw;
  P.slabs = (int)((L + sw - 1) / sw);
  return P;
}

// ---- exact fixed-point passes -------------------------------------------------------------
//
// GB300 issues one FP64 FMA per element at 1.26 TFLOP/s, which caps an FP64 pass over A near
// 5 TB/s; its integer pipe has several times that rate.  So the FP64 operator can stream an
// integer copy of A instead: row i of A is scaled by 2^-e_i (2^e_i > max_k |A_ik|) and every
// entry written as N = rint(2^52 A_ik 2^-e_i) = hi 2^26 + lo (|hi| <= 2^26, -2^25 <= lo < 2^25),
// once at setup, 8 bytes per entry as in FP64.  A vector x of the pass gets one exponent f
// (2^f > max_k |x_k|, for the A^T pass after folding 2^e_i into x_i) and the same two digits.
// Then x . a = 2^(f + e) 2^-104 sum_k (hi 2^26 + lo)(xh 2^26 + xl), whose two leading parts
//   T1 = sum hi xh,  T2 = sum (hi xl + lo xh)      (every product below 2^52 in magnitude)
// are accumulated exactly in int64 (at most FX_FLUSH terms per accumulator), converted once
// to FP64 and scaled by 2^(f + e - 52) and 2^(f + e - 78).  Dropped: lo xl 2^-104 per term and
// the two roundings to 53 bits, so each output is within about 3 K 2^-53 2^(f+e) of the exact
// product with the unrounded A and x: the FP64 error bound of a K-term dot product measured
// against the largest entry of the row and of the vector.
__device__ __forceinline__ void fx_acc2(long long& t1, long long& t2, const int4& a, const int4& w) {
  t1 += (long long)a.x * w.x;
  t2 += (long long)a.x * w.y + (long long)a.y * w.x;
  t1 += (long long)a.z * w.z;
  t2 += (long long)a.z * w.w + (long long)a.w * w.z;
}

__device__ __forceinline__ int block_max_int(int v, int* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = __reduce_max_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int t = (threadIdx.x < nw) ? sh[threadIdx.x] : INT_MIN;
  if (wid == 0) t = __reduce_max_sync(0xffffffffu, t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  const int r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double fx_out(double d, int F, int e) {
  return F == FX_BAD ? __longlong_as_double(0x7ff8000000000000ll) : (fx_none(F) ? 0.0 : ldexp(d, F + e));
}

// setup: row i of A (m x L, row-major) -> digits (row length Lp = L rounded up to even, the pad
// entry zero) and its exponent e_i (0 for a zero row)
__global__ void __launch_bounds__(256) fx_split_rows_kernel(int64_t L, int64_t Lp, const double* __restrict__ A,
                                                            int2* __restrict__ Ai, int* __restrict__ ea) {
  __shared__ int sh[32];
  const int i = blockIdx.x;
  const double* row = A + (int64_t)i * L;
  int e = INT_MIN;
  for (int64_t c = threadIdx.x; c < L; c += blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(row[c]) & 0x7FFFFFFFFFFFFFFFull;
    if (b) e = max(e, fx_expo_bits(b));
  }
  e = block_max_int(e, sh);
  if (e == INT_MIN) e = 0;
  if (threadIdx.x == 0) ea[i] = e;
  int2* out = Ai + (int64_t)i * Lp;
  for (int64_t c = threadIdx.x; c < Lp; c += blockDim.x) out[c] = fx_split(c < L ? fx_fixed(row[c], 0, e) : 0);
}

// one block, integer operations only: *fout = F with |x_k| 2^(ex_k) < 2^F for every k (ex may be
// NULL), FX_NONE when x is zero, FX_BAD when x has a non-finite entry
__global__ void __launch_bounds__(1024) fx_exponent_kernel(int64_t len, const double* __restrict__ x,
                                                           const int* __restrict__ ex, int* __restrict__ fout,
                                                           const int32_t* __restrict__ done) {
  if (done && *done) return;
  __shared__ int sh[32];
  int f = INT_MIN, bad = 0;
  constexpr int U = 8;                      // loads in flight per thread
  for (int64_t j0 = 0; j0 < len; j0 += (int64_t)U * blockDim.x) {
    unsigned long long b[U];
    int e[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = j0 + (int64_t)u * blockDim.x + threadIdx.x;
      b[u] = j < len ? (unsigned long long)__double_as_longlong(x[j]) & 0x7FFFFFFFFFFFFFFFull : 0ull;
      e[u] = (ex && j < len) ? ex[j] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (b[u] >= 0x7FF0000000000000ull) bad = 1;
      else if (b[u]) f = max(f, fx_expo_bits(b[u]) + e[u]);
    }
  }
  f = block_max_int(f, sh);
  bad = block_max_int(bad, sh);
  if (threadIdx.x == 0) *fout = bad ? FX_BAD : f;
}

// A x from the digits: the slab / row-block layout of rows_gemv_kernel (partial sums
// part[s * m + i] for slab s), two rows in flight per warp
template <bool STREAM>
__global__ void __launch_bounds__(GV_WARPS * 32)
fx_rows_gemv_kernel(const int2* __restrict__ Ai, const int* __restrict__ ea, int m, int64_t L, int64_t Lp,
                    const double* __restrict__ x, const int* __restrict__ fptr, double* __restrict__ part, int SW,
                    int R, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  __shared__ __align__(16) int2 xs[GV_SWMAX];
  const int s = blockIdx.x;
  const int64_t k0 = (int64_t)s * SW;
  const int lenp = (int)((Lp - k0) < (int64_t)SW ? (Lp - k0) : (int64_t)SW);   // even
  const int f = *fptr;
  const int F = (f == FX_BAD || fx_none(f)) ? 0 : f;
  for (int q = threadIdx.x; q < lenp; q += blockDim.x)    // the digits of x 2^-F for this slab
    xs[q] = fx_split(k0 + q < L ? fx_fixed(x[k0 + q], 0, F) : 0);
  __syncthreads();
  const int np = lenp >> 1;
  const int4* xv = reinterpret_cast<const int4*>(xs);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = blockIdx.y * R;
  for (int t = warp; t < R; t += 2 * GV_WARPS) {
    const int ia = rbase + t;
    if (ia >= m) break;
    const int ib = rbase + t + GV_WARPS;
    const bool hb = (t + GV_WARPS < R) && (ib < m);
    const int4* va = reinterpret_cast<const int4*>(Ai + (int64_t)ia * Lp + k0);
    long long a1 = 0, a2 = 0, b1 = 0, b2 = 0;
    if (hb) {   // warp-uniform
      const int4* vb = reinterpret_cast<const int4*>(Ai + (int64_t)ib * Lp + k0);
      int q = lane;
      for (; q + 32 < np; q += 64) {
        const int4 u0 = STREAM ? ld_stream_i4(va + q, pol) : __ldg(va + q);
        const int4 u1 = STREAM ? ld_stream_i4(va + q + 32, pol) : __ldg(va + q + 32);
        const int4 v0 = STREAM ? ld_stream_i4(vb + q, pol) : __ldg(vb + q);
        const int4 v1 = STREAM ? ld_stream_i4(vb + q + 32, pol) : __ldg(vb + q + 32);
        const int4 w0 = xv[q], w1 = xv[q + 32];
        fx_acc2(a1, a2, u0, w0);
        fx_acc2(b1, b2, v0, w0);
        fx_acc2(a1, a2, u1, w1);
        fx_acc2(b1, b2, v1, w1);
      }
      for (; q < np; q += 32) {
        const int4 u0 = STREAM ? ld_stream_i4(va + q, pol) : __ldg(va + q);
        const int4 v0 = STREAM ? ld_stream_i4(vb + q, pol) : __ldg(vb + q);
        fx_acc2(a1, a2, u0, xv[q]);
        fx_acc2(b1, b2, v0, xv[q]);
      }
    } else {
      int q = lane;
      for (; q + 96 < np; q += 128) {
        const int4 u0 = STREAM ? ld_stream_i4(va + q, pol) : __ldg(va + q);
        const int4 u1 = STREAM ? ld_stream_i4(va + q + 32, pol) : __ldg(va + q + 32);
        const int4 u2 = STREAM ? ld_stream_i4(va + q + 64, pol) : __ldg(va + q + 64);
        const int4 u3 = STREAM ? ld_stream_i4(va + q + 96, pol) : __ldg(va + q + 96);
        fx_acc2(a1, a2, u0, xv[q]);
        fx_acc2(b1, b2, u1, xv[q + 32]);
        fx_acc2(a1, a2, u2, xv[q + 64]);
        fx_acc2(b1, b2, u3, xv[q + 96]);
      }
      for (; q < np; q += 32) fx_acc2(a1, a2, STREAM ? ld_stream_i4(va + q, pol) : __ldg(va + q), xv[q]);
    }
    // per lane at most 2 * ceil(np / 32) <= 128 terms per accumulator (SW <= 4096)
    double da = fx_value(a1, a2), db = fx_value(b1, b2);
    if (!hb) {
      da += db;
      db = 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      da += __shfl_xor_sync(0xffffffffu, da, o);
      db += __shfl_xor_sync(0xffffffffu, db, o);
    }
    if (lane == 0) {
      part[(int64_t)s * m + ia] = fx_out(da, f, ea[ia]);
      if (hb) part[(int64_t)s * m + ib] = fx_out(db, f, ea[ib]);
    }
  }
}

// A^T y from the digits (y's digits carry the row exponents): the row-group layout of
// rows_gemvT_kernel (partials part[g * L + c]), two columns per thread.  With fptr == NULL every
// CTA finds the exponent of y itself (one scan of the m entries of y and of the row exponents,
// from L2), which saves a launch for the small m of the dense kind.
template <bool STREAM>
__global__ void __launch_bounds__(GT_THREADS)
fx_rows_gemvT_kernel(const int2* __restrict__ Ai, const int* __restrict__ ea, int m, int64_t L, int64_t Lp,
                     const double* __restrict__ y, const int* __restrict__ fptr, double* __restrict__ part,
                     int rows_per_group, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const uint64_t pol = STREAM ? evict_first_policy() : 0;
  __shared__ int2 ys[FX_FLUSH];
  __shared__ int shf[32];
  const int g = blockIdx.y;
  const int i0 = g * rows_per_group;
  const int i1 = min(m, i0 + rows_per_group);
  const int64_t c = ((int64_t)blockIdx.x * GT_THREADS + threadIdx.x) * 2;   // c < Lp: c < L
  int f;
  if (fptr) {
    f = *fptr;
  } else {
    int e = INT_MIN, bad = 0;
    constexpr int U = 8;
    for (int j0 = 0; j0 < m; j0 += U * GT_THREADS) {
      unsigned long long b[U];
      int ex[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + u * GT_THREADS + threadIdx.x;
        b[u] = j < m ? (unsigned long long)__double_as_longlong(y[j]) & 0x7FFFFFFFFFFFFFFFull : 0ull;
        ex[u] = j < m ? ea[j] : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (b[u] >= 0x7FF0000000000000ull) bad = 1;
        else if (b[u]) e = max(e, fx_expo_bits(b[u]) + ex[u]);
      }
    }
    e = block_max_int(e, shf);
    bad = block_max_int(bad, shf);
    f = bad ? FX_BAD : e;
  }
  const int F = (f == FX_BAD || fx_none(f)) ? 0 : f;
  const int4* base = reinterpret_cast<const int4*>(Ai + c);
  const int64_t stv = Lp / 2;
  double d0 = 0.0, d1 = 0.0;
  for (int ic = i0; ic < i1; ic += FX_FLUSH) {
    const int ie = min(i1, ic + FX_FLUSH);
    __syncthreads();
    for (int q = threadIdx.x; q < ie - ic; q += blockDim.x)   // digits of y_i 2^(e_i - F)
      ys[q] = fx_split(fx_fixed(y[ic + q], ea[ic + q], F));
    __syncthreads();
    if (c < Lp) {
      long long p1 = 0, p2 = 0, q1 = 0, q2 = 0;
      int i = ic;
      for (; i + 7 < ie; i += 8) {
        int4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int4* ptr = base + (int64_t)(i + u) * stv;
          v[u] = STREAM ? ld_stream_i4(ptr, pol) : __ldg(ptr);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int2 w = ys[i + u - ic];
          p1 += (long long)v[u].x * w.x;
          p2 += (long long)v[u].x * w.y + (long long)v[u].y * w.x;
          q1 += (long long)v[u].z * w.x;
          q2 += (long long)v[u].z * w.y + (long long)v[u].w * w.x;
        }
      }
      for (; i < ie; ++i) {
        const int4* ptr = base + (int64_t)i * stv;
        const int4 v = STREAM ? ld_stream_i4(ptr, pol) : __ldg(ptr);
        const int2 w = ys[i - ic];
        p1 += (long long)v.x * w.x;
        p2 += (long long)v.x * w.y + (long long)v.y * w.x;
        q1 += (long long)v.z * w.x;
        q2 += (long long)v.z * w.y + (long long)v.w * w.x;
      }
      d0 += fx_value(p1, p2);
      d1 += fx_value(q1, q2);
    }
  }
  if (c < Lp) {
    part[(int64_t)g * L + c] = fx_out(d0, f, 0);
    if (c + 1 < L) part[(int64_t)g * L + c + 1] = fx_out(d1, f, 0);
  }
}

// Y = smat(scale * sum_g part[g * L + .]) (both triangles), one thread per svec position, the
// groups summed in order with eight loads in flight
__global__ void __launch_bounds__(GT_THREADS)
svec_groups_unpack_kernel(int n, int64_t L, const double* __restrict__ part, int G, double scale,
                          double* __restrict__ Y, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int64_t c = (int64_t)blockIdx.x * GT_THREADS + threadIdx.x;
  if (c >= L) return;
  double s = 0.0;
  int gg = 0;
  for (; gg + 7 < G; gg += 8) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldcg(part + (int64_t)(gg + k) * L + c);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; gg < G; ++gg) s += __ldcg(part + (int64_t)gg * L + c);
  int a, b;
  svec_pos(n, c, a, b);
  const double v = (a == b ? s : s * WC_RSQRT2) * scale;
  Y[a + (int64_t)b * n] = v;
  Y[b + (int64_t)a * n] = v;
}

}  // namespace

int rows_gemv_slabs(int m, int64_t L, int esize) { return gv_plan(m, L, esize).slabs; }

size_t rows_gemv_part_elems(int64_t rows_max, int64_t L) {
  return (size_t)(rows_max < 1 ? 1 : rows_max) * (size_t)((L + 127) / 128 + 1);
}

template <typename T>
void rows_gemv_impl(cudaStream_t st, const T* A, int m, int64_t L, const T* x, T* part, const int32_t* done,
                    int64_t* launches, XForm<T> xf) {
  const GvPlan P = gv_plan(m, L, (int)sizeof(T));
  dim3 grid(P.slabs, (m + P.R - 1) / P.R);
  const bool vec = is_vec_ok(A, L);
  if (vec) {
    if (P.stream)
      rows_gemv_kernel<T, true, true><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, P.SW, P.R, done, xf);
    else
      rows_gemv_kernel<T, true, false><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, P.SW, P.R, done, xf);
  } else {
    if (P.stream)
      rows_gemv_kernel<T, false, true><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, P.SW, P.R, done, xf);
    else
      rows_gemv_kernel<T, false, false><<<grid, GV_WARPS * 32, 0, st>>>(A, m, L, x, part, P.SW, P.R, done, xf);
  }
  if (launches) ++*launches;
}

template <typename T>
void rows_gemv(cudaStream_t st, const T* A, int m, int64_t L, const T* x, T* part, const int32_t* done,
               int64_t* launches) {
  rows_gemv_impl<T>(st, A, m, L, x, part, done, launches, XForm<T>{nullptr, nullptr, 0, 0.0, nullptr, nullptr});
}

void rows_gemv_formed(cudaStream_t st, const double* A, int m, int64_t L, const double* base, const double* xpart,
                      int G, double c0, const double* cdiv, double* xout, double* part, const int32_t* done,
                      int64_t* launches) {
  rows_gemv_impl<double>(st, A, m, L, nullptr, part, done, launches, XForm<double>{base, xpart, G, c0, cdiv, xout});
}

int rows_gemvT_groups(int m, int64_t L, int esize) {
  const int64_t W = 16 / esize;
  const int64_t cb = (L + W * GT_THREADS - 1) / (W * GT_THREADS);
  const int64_t maxg = (m + 31) / 32;
  int64_t bestg = 1;
  double best = -1.0;
  for (int64_t g = 1; g <= maxg; ++g) {
    const int64_t units = cb * g;
    double b = balance(units);
    if (units < 2 * g_num_sms) b -= 1.0;   // too few CTAs to cover the GPU
    if (b > best + 1e-9) { best = b; bestg = g; }
  }
  return (int)bestg;
}

template <typename T>
void rows_gemvT_impl(cudaStream_t st, const T* A, int m, int64_t L, const T* p, T* part, int groups,
                     const int32_t* done, int64_t* launches, int n, double scale, T* Y, unsigned int* tickets) {
  const int rpg = (m + groups - 1) / groups;
  const bool stream = (int64_t)m * L * (int64_t)sizeof(T) > (int64_t)64 << 20;
  if (is_vec_ok(A, L)) {
    constexpr int W = V16<T>::W;
    dim3 grid((unsigned)((L + W * GT_THREADS - 1) / (W * GT_THREADS)), groups);
    if (stream)
      rows_gemvT_kernel<T, true, true><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done, n, scale, Y, tickets);
    else
      rows_gemvT_kernel<T, true, false><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done, n, scale, Y, tickets);
  } else {
    dim3 grid((unsigned)((L + GT_THREADS - 1) / GT_THREADS), groups);
    if (stream)
      rows_gemvT_kernel<T, false, true><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done, n, scale, Y, tickets);
    else
      rows_gemvT_kernel<T, false, false><<<grid, GT_THREADS, 0, st>>>(A, m, L, p, part, rpg, done, n, scale, Y,
                                                                     tickets);
  }
  if (launches) ++*launches;
}

template <typename T>
void rows_gemvT(cudaStream_t st, const T* A, int m, int64_t L, const T* p, T* part, int groups,
                const int32_t* done, int64_t* launches) {
  rows_gemvT_impl<T>(st, A, m, L, p, part, groups, done, launches, 0, 1.0, nullptr, nullptr);
}

template <typename T>
void rows_gemvT_unpack(cudaStream_t st, const T* A, int m, int64_t L, const T* p, T* part, int groups, int n,
                       double scale, T* Y, unsigned int* tickets, const int32_t* done, int64_t* launches) {
  rows_gemvT_impl<T>(st, A, m, L, p, part, groups, done, launches, n, scale, Y, tickets);
}

int64_t fx_row_len(int64_t L) { return (L + 1) & ~(int64_t)1; }

static GvPlan fx_plan(int m, int64_t L);
int fx_rows_gemv_slabs(int m, int64_t L) { return fx_plan(m, L).slabs; }

void fx_split_rows(cudaStream_t st, const double* A, int m, int64_t L, int2* Ai, int* ea, int64_t* launches) {
  fx_split_rows_kernel<<<m, 256, 0, st>>>(L, fx_row_len(L), A, Ai, ea);
  if (launches) ++*launches;
}

void fx_exponent(cudaStream_t st, const double* x, const int* ex, int64_t len, int* f, const int32_t* done,
                 int64_t* launches) {
  fx_exponent_kernel<<<1, 1024, 0, st>>>(len, x, ex, f, done);
  if (launches) ++*launches;
}

// Launch shape of fx_rows_gemv: the CTAs of one launch are all resident at once (CTAs per SM
// from the occupancy of the kernel), so the (slab width, rows per CTA) pair is chosen to fill
// whole waves of resident CTAs: a partial last wave leaves most SMs idle while it runs.
static GvPlan fx_plan(int m, int64_t L) {
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fx_rows_gemv_kernel<true>, GV_WARPS * 32, 0) != cudaSuccess ||
        o < 1) {
      cudaGetLastError();
      o = 1;
    }
    occ = o;
  }
  GvPlan P = gv_plan(m, L, 8);
  if (!P.stream) return P;            // L2-resident: the plan of rows_gemv<double>
  // the widest slab (fewest partial sums) whose best row split fills >= 95% of its waves, else
  // the best-filling split
  const int64_t cap = (int64_t)occ * g_num_sms;
  double best = -1.0;
  bool good = false;
  for (int sw = GV_SWMAX; sw >= 1024; sw /= 2) {
    const int64_t slabs = (L + sw - 1) / sw;
    for (int R = 8; R <= 64; ++R) {
      const int64_t units = slabs * ((m + R - 1) / R);
      const int64_t waves = (units + cap - 1) / cap;
      const double eff = (double)units / (double)(waves * cap);
      if (!good && eff > best + 1e-9) { best = eff; P.SW = sw; P.R = R; P.slabs = (int)slabs; }
    }
    if (best >= 0.95) good = true;
  }
  return P;
}

void fx_rows_gemv(cudaStream_t st, const int2* Ai, const int* ea, int m, int64_t L, const double* x, const int* f,
                  double* part, const int32_t* done, int64_t* launches) {
  const GvPlan P = fx_plan(m, L);
  dim3 grid(P.slabs, (m + P.R - 1) / P.R);
  const int64_t Lp = fx_row_len(L);
  if (P.stream)
    fx_rows_gemv_kernel<true><<<grid, GV_WARPS * 32, 0, st>>>(Ai, ea, m, L, Lp, x, f, part, P.SW, P.R, done);
  else
    fx_rows_gemv_kernel<false><<<grid, GV_WARPS * 32, 0, st>>>(Ai, ea, m, L, Lp, x, f, part, P.SW, P.R, done);
  if (launches) ++*launches;
}

void fx_rows_gemvT_unpack(cudaStream_t st, const int2* Ai, const int* ea, int m, int64_t L, const double* y,
                          int* f, double* part, int groups, int n, double scale, double* Y, const int32_t* done,
                          int64_t* launches) {
  const int rpg = (m + groups - 1) / groups;
  const int64_t Lp = fx_row_len(L);
  const bool stream = (int64_t)m * L * 8 > (int64_t)64 << 20;
  // each CTA scans y for its exponent when y is short; else one exponent launch first
  const int* fp = nullptr;
  if (m > 8192) {
    fx_exponent(st, y, ea, m, f, done, launches);
    fp = f;
  }
  dim3 grid((unsigned)((Lp / 2 + GT_THREADS - 1) / GT_THREADS), groups);
  if (stream)
    fx_rows_gemvT_kernel<true><<<grid, GT_THREADS, 0, st>>>(Ai, ea, m, L, Lp, y, fp, part, rpg, done);
  else
    fx_rows_gemvT_kernel<false><<<grid, GT_THREADS, 0, st>>>(Ai, ea, m, L, Lp, y, fp, part, rpg, done);
  svec_groups_unpack_kernel<<<(unsigned)((L + GT_THREADS - 1) / GT_THREADS), GT_THREADS, 0, st>>>(n, L, part, groups,
                                                                                                scale, Y, done);
  if (launches) *launches += 2;
}

int rows_gemvT_blocks(int64_t L, int esize) {
  const int64_t W = 16 / esize;
  return (int)((L + W * GT_THREADS - 1) / (W * GT_THREADS));
}

template void rows_gemv<double>(cudaStream_t, const double*, int, int64_t, const double*, double*, const int32_t*,
                                int64_t*);
template void rows_gemv<float>(cudaStream_t, const float*, int, int64_t, const float*, float*, const int32_t*,
                               int64_t*);
template void rows_gemvT<double>(cudaStream_t, const double*, int, int64_t, const double*, double*, int,
                                 const int32_t*, int64_t*);
template void rows_gemvT<float>(cudaStream_t, const float*, int, int64_t, const float*, float*, int, const int32_t*,
                                int64_t*);
template void rows_gemvT_unpack<double>(cudaStream_t, const double*, int, int64_t, const double*, double*, int, int,
                                        double, double*, unsigned int*, const int32_t*, int64_t*);
template void rows_gemvT_unpack<float>(cudaStream_t, const float*, int, int64_t, const float*, float*, int, int,
                                       double, float*, unsigned int*, const int32_t*, int64_t*);

void rows_sumsq(cudaStream_t st, const double* A, int m, int64_t L, double* out, double* scratch,
                int64_t* launches) {
  const int nb = 4 * g_num_sms;
  sumsq_kernel<<<nb, 256, 0, st>>>(A, (int64_t)m * L, scratch);
  sum_in_order_kernel<<<1, 256, 0, st>>>(scratch, nb, out);
  if (launches) *launches += 2;
}

}  // namespace wc

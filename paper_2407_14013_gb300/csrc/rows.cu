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
  const int per = VEC ? V16<T>::W : 1;
  const int64_t c0 = (int64_t)blockIdx.x * GT_THREADS * per;
  for (int u = threadIdx.x; u < GT_THREADS * per; u += GT_THREADS) {
    const int64_t c = c0 + u;
    if (c >= L) break;
    double sum = 0.0;
    for (int gg = 0; gg < (int)gridDim.y; ++gg) sum += (double)__ldcg(part + (int64_t)gg * L + c);
    int a, b;
    svec_pos(n, c, a, b);
    const T v = (T)((a == b ? sum : sum * WC_RSQRT2) * scale);
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

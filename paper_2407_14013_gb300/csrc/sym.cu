// Layout conversions between full symmetric n x n matrices and svec vectors (Notations:
// svec stacks the lower triangle column by column, off-diagonal entries times sqrt(2);
// svec of a non-symmetric matrix is svec of its symmetric part).
#include "common.cuh"
#include "fx.cuh"
#include "kernels.h"

namespace wc {

namespace {

template <typename T>
__global__ void svec_unpack_sum_kernel(int n, const T* __restrict__ part, int groups, int64_t N,
                                       double scale, T* __restrict__ Y,
                                       const int32_t* __restrict__ done) {
  if (done && *done) return;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int a = (int)(q % n), b = (int)(q / n);
  int i = a > b ? a : b, j = a > b ? b : a;
  int64_t idx = svec_index(n, i, j);
  double s = 0.0;
  int g = 0;
  for (; g + 7 < groups; g += 8) {   // the groups in order, eight loads in flight
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (double)part[(int64_t)(g + k) * N + idx];
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; g < groups; ++g) s += (double)part[(int64_t)g * N + idx];
  Y[q] = (T)((a == b ? s : s * WC_RSQRT2) * scale);
}

template <typename T>
__global__ void svec_pack_plus_kernel(int n, int r, const T* __restrict__ Z, const T* __restrict__ U,
                                      const T* __restrict__ Q, T* __restrict__ out,
                                      const int32_t* __restrict__ done, int* __restrict__ expo) {
  if (done && *done) return;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int e = INT_MIN;
  if (q < (int64_t)n * n) {
    const int a = (int)(q % n), b = (int)(q / n);
    if (a >= b) {
      double v = (double)Z[a + (int64_t)b * n];   // lower triangle (a >= b) of the symmetric Z
      if (U) {
        double t = 0.0;
        for (int k = 0; k < r; ++k)
          t += (double)U[a + (int64_t)k * n] * (double)Q[b + (int64_t)k * n] +
               (double)Q[a + (int64_t)k * n] * (double)U[b + (int64_t)k * n];
        v += 0.5 * t;
      }
      const T o = (T)((a == b) ? v : v * WC_SQRT2);
      out[svec_index(n, a, b)] = o;
      if (expo) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong((double)o) & 0x7FFFFFFFFFFFFFFFull;
        e = bits >= 0x7FF0000000000000ull ? INT_MAX : (bits ? fx_expo_bits(bits) : INT_MIN);
      }
    }
  }
  if (expo) {   // one atomic per warp (no thread has returned)
    e = __reduce_max_sync(0xffffffffu, e);
    if ((threadIdx.x & 31) == 0 && e != INT_MIN) atomicMax(expo, e);
  }
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

template <typename T>
void svec_unpack_sum(cudaStream_t st, int n, const T* part, int groups, double scale, T* Y,
                     const int32_t* done, int64_t* launches) {
  int64_t N = (int64_t)n * (n + 1) / 2;
  svec_unpack_sum_kernel<T><<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, part, groups, N, scale, Y, done);
  if (launches) ++*launches;
}

template <typename T>
void svec_pack_plus(cudaStream_t st, int n, int r, const T* Z, const T* U, const T* Q, T* out,
                    const int32_t* done, int64_t* launches, int* expo) {
  svec_pack_plus_kernel<T><<<nblk((int64_t)n * n, 256), 256, 0, st>>>(n, r, Z, U, Q, out, done, expo);
  if (launches) ++*launches;
}

template void svec_unpack_sum<double>(cudaStream_t, int, const double*, int, double, double*, const int32_t*,
                                      int64_t*);
template void svec_unpack_sum<float>(cudaStream_t, int, const float*, int, double, float*, const int32_t*, int64_t*);
template void svec_pack_plus<double>(cudaStream_t, int, int, const double*, const double*, const double*, double*,
                                     const int32_t*, int64_t*, int*);
template void svec_pack_plus<float>(cudaStream_t, int, int, const float*, const float*, const float*, float*,
                                    const int32_t*, int64_t*, int*);

namespace {
template <typename To, typename From>
__global__ void convert_kernel(int64_t count, const From* __restrict__ src, To* __restrict__ dst) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = (To)src[q];
}
}  // namespace

template <typename To, typename From>
void convert(cudaStream_t st, int64_t count, const From* src, To* dst, int64_t* launches) {
  if (count <= 0) return;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 8 * g_num_sms) blocks = 8 * g_num_sms;
  convert_kernel<To, From><<<(unsigned)blocks, 256, 0, st>>>(count, src, dst);
  if (launches) ++*launches;
}

template void convert<float, double>(cudaStream_t, int64_t, const double*, float*, int64_t*);
template void convert<double, float>(cudaStream_t, int64_t, const float*, double*, int64_t*);

void svec_rows_unpack(cudaStream_t st, const double* A, int n, int i0, int mb, double* out,
                      int64_t* launches) {
  int64_t N = (int64_t)n * (n + 1) / 2;
  svec_rows_unpack_kernel<<<nblk((int64_t)n * n * mb, 256), 256, 0, st>>>(A, n, N, i0, mb, out);
  if (launches) ++*launches;
}

}  // namespace wc

namespace wc {

namespace {

constexpr int AQ_THREADS = 256;

// One CTA per constraint i: G_i = A_i Q.  The svec row of A_i is staged in shared memory,
// then thread a forms row a of G_i in registers,
//   G_i[a, :] = sum_b A_i[a, b] Q[b, :],
// reading A_i[a, b] below the diagonal from column b of the svec row (entry a - b: lanes with
// consecutive a read consecutive words) and above it from column a (entry b - a).  Every
// thread does n multiply-add rows of width r, so the work is balanced, and no partial sums
// are shared: FP64 work is the n^2 r multiply-adds of the product and nothing else.
template <int r>
__global__ void __launch_bounds__(AQ_THREADS)
dense_AiQ_kernel(const double* __restrict__ A, int n, int64_t N, int i0, int mb, const double* __restrict__ Q,
                 double* __restrict__ G) {
  extern __shared__ __align__(16) double sm[];
  double* As = sm;                                  // svec row, N entries (+ pad to 2)
  double* Qs = sm + ((N + 1) & ~int64_t(1));        // n x r, row-major
  const int il = blockIdx.x, i = i0 + il;
  const double* row = A + (int64_t)i * N;
  if ((N & 1) == 0) {                               // 16-byte rows: vector loads
    const double2* src = reinterpret_cast<const double2*>(row);
    double2* dst = reinterpret_cast<double2*>(As);
    for (int64_t q = threadIdx.x; q < N / 2; q += blockDim.x) dst[q] = __ldg(src + q);
  } else {
    for (int64_t q = threadIdx.x; q < N; q += blockDim.x) As[q] = __ldg(row + q);
  }
  for (int q = threadIdx.x; q < n * r; q += blockDim.x) {
    const int b = q / r, j = q % r;
    Qs[q] = Q[b + (int64_t)j * n];
  }
  __syncthreads();
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    double off[r], dg[r];
#pragma unroll
    for (int j = 0; j < r; ++j) off[j] = 0.0;
    int64_t idx = a;                                // (a, b = 0) in column 0
    for (int b = 0; b < a; ++b) {
      const double s = As[idx];
#pragma unroll
      for (int j = 0; j < r; ++j) off[j] = fma(s, Qs[b * r + j], off[j]);
      idx += n - b - 1;                             // (a, b + 1) in column b + 1
    }
    const double sd = As[idx];                      // diagonal (a, a)
#pragma unroll
    for (int j = 0; j < r; ++j) dg[j] = sd * Qs[a * r + j];
    for (int b = a + 1; b < n; ++b) {               // (b, a) in column a
      const double s = As[idx + (b - a)];
#pragma unroll
      for (int j = 0; j < r; ++j) off[j] = fma(s, Qs[b * r + j], off[j]);
    }
#pragma unroll
    for (int j = 0; j < r; ++j) G[a + ((int64_t)j * mb + il) * n] = fma(off[j], WC_RSQRT2, dg[j]);
  }
}

// The same product from the integer digits of the svec row (the copy the FP64 passes stream:
// N_ab = rint(a_ab 2^(52 - e_i)) = hi 2^26 + lo, row exponent e_i) and of the columns of Q
// (exponent f_j per column), summed exactly in int64 as the passes do (hi hi' and hi lo' + lo hi',
// at most n <= 1024 terms per accumulator), so the n^2 r multiply-adds run on the integer pipe.
// Off-diagonal (sqrt2-scaled) and diagonal entries keep separate sums, combined in FP64 at the end
// as G = off / sqrt2 + diag.
template <int r>
__global__ void __launch_bounds__(AQ_THREADS)
fx_AiQ_kernel(const int2* __restrict__ Ad, const int* __restrict__ ea, int n, int64_t Lp, int i0, int mb,
              const double* __restrict__ Q, double* __restrict__ G) {
  extern __shared__ __align__(16) int2 smi[];
  int2* As = smi;                                   // digits of the svec row, Lp entries
  int2* Qd = smi + Lp;                              // digits of Q, n x r row-major
  __shared__ int fq[r];
  const int il = blockIdx.x, i = i0 + il;
  // the row (Lp even: 16-byte aligned rows) by asynchronous 16-byte copies, all issued before
  // any is waited for, while the digits of Q are made
  {
    const char* src = reinterpret_cast<const char*>(Ad + (int64_t)i * Lp);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(As);
    for (int64_t q = threadIdx.x; q < Lp / 2; q += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (uint32_t)(q * 16)), "l"(src + q * 16)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  if (threadIdx.x < r) fq[threadIdx.x] = INT_MIN;
  __syncthreads();
  for (int q = threadIdx.x; q < n * r; q += blockDim.x) {   // exponents of the columns of Q
    const int b = q / r, j = q % r;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(Q[b + (int64_t)j * n]) &
                                    0x7FFFFFFFFFFFFFFFull;
    if (bits) atomicMax(&fq[j], fx_expo_bits(bits));
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n * r; q += blockDim.x) {
    const int b = q / r, j = q % r;
    const int f = fq[j] == INT_MIN ? 0 : fq[j];
    Qd[q] = fx_split(fx_fixed(Q[b + (int64_t)j * n], 0, f));
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int e = ea[i];
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    long long o1[r], o2[r], d1[r], d2[r];
#pragma unroll
    for (int j = 0; j < r; ++j) o1[j] = o2[j] = 0;
    int64_t idx = a;                                // (a, b = 0) in column 0
    for (int b = 0; b < a; ++b) {
      const int2 s = As[idx];
#pragma unroll
      for (int j = 0; j < r; ++j) {
        const int2 q = Qd[b * r + j];
        o1[j] += (long long)s.x * q.x;
        o2[j] += (long long)s.x * q.y + (long long)s.y * q.x;
      }
      idx += n - b - 1;                             // (a, b + 1) in column b + 1
    }
    {
      const int2 s = As[idx];                       // diagonal (a, a)
#pragma unroll
      for (int j = 0; j < r; ++j) {
        const int2 q = Qd[a * r + j];
        d1[j] = (long long)s.x * q.x;
        d2[j] = (long long)s.x * q.y + (long long)s.y * q.x;
      }
    }
    for (int b = a + 1; b < n; ++b) {               // (b, a) in column a
      const int2 s = As[idx + (b - a)];
#pragma unroll
      for (int j = 0; j < r; ++j) {
        const int2 q = Qd[b * r + j];
        o1[j] += (long long)s.x * q.x;
        o2[j] += (long long)s.x * q.y + (long long)s.y * q.x;
      }
    }
#pragma unroll
    for (int j = 0; j < r; ++j) {
      const int sc = e + (fq[j] == INT_MIN ? 0 : fq[j]);
      const double off = ldexp(fx_value(o1[j], o2[j]), sc), dg = ldexp(fx_value(d1[j], d2[j]), sc);
      G[a + ((int64_t)j * mb + il) * n] = fma(off, WC_RSQRT2, dg);
    }
  }
}

}  // namespace

static size_t dense_AiQ_smem(int n, int r) {
  const int64_t N = (int64_t)n * (n + 1) / 2;
  return (size_t)(((N + 1) & ~int64_t(1)) + (int64_t)n * r) * sizeof(double);
}

bool dense_AiQ(cudaStream_t st, const double* A, int n, int i0, int mb, int r, const double* Q, double* G,
               int64_t* launches) {
  const size_t smem = dense_AiQ_smem(n, r);
  if (r < 1 || r > 16 || smem > 220 * 1024) return false;
  const int64_t N = (int64_t)n * (n + 1) / 2;
  switch (r) {
#define WC_AIQ_CASE(R)                                                                              \
    case R:                                                                                         \
      raise_dyn_smem((const void*)dense_AiQ_kernel<R>, (int)smem);                                 \
      dense_AiQ_kernel<R><<<mb, AQ_THREADS, smem, st>>>(A, n, N, i0, mb, Q, G);                      \
      break;
    WC_AIQ_CASE(1) WC_AIQ_CASE(2) WC_AIQ_CASE(3) WC_AIQ_CASE(4) WC_AIQ_CASE(5) WC_AIQ_CASE(6)
    WC_AIQ_CASE(7) WC_AIQ_CASE(8) WC_AIQ_CASE(9) WC_AIQ_CASE(10) WC_AIQ_CASE(11) WC_AIQ_CASE(12)
    WC_AIQ_CASE(13) WC_AIQ_CASE(14) WC_AIQ_CASE(15) WC_AIQ_CASE(16)
#undef WC_AIQ_CASE
    default: return false;
  }
  if (launches) ++*launches;
  return true;
}

}  // namespace wc

namespace wc {

bool fx_AiQ(cudaStream_t st, const int2* Ad, const int* ea, int n, int64_t Lp, int i0, int mb, int r, const double* Q,
            double* G, int64_t* launches) {
  const size_t smem = (size_t)(Lp + (int64_t)n * r) * sizeof(int2);
  if (r < 1 || r > 16 || n > FX_FLUSH || (Lp & 1) || smem > 220 * 1024) return false;
  switch (r) {
#define WC_FXAIQ_CASE(R)                                                                            \
    case R:                                                                                         \
      raise_dyn_smem((const void*)fx_AiQ_kernel<R>, (int)smem);                                 \
      fx_AiQ_kernel<R><<<mb, AQ_THREADS, smem, st>>>(Ad, ea, n, Lp, i0, mb, Q, G);                    \
      break;
    WC_FXAIQ_CASE(1) WC_FXAIQ_CASE(2) WC_FXAIQ_CASE(3) WC_FXAIQ_CASE(4) WC_FXAIQ_CASE(5) WC_FXAIQ_CASE(6)
    WC_FXAIQ_CASE(7) WC_FXAIQ_CASE(8) WC_FXAIQ_CASE(9) WC_FXAIQ_CASE(10) WC_FXAIQ_CASE(11) WC_FXAIQ_CASE(12)
    WC_FXAIQ_CASE(13) WC_FXAIQ_CASE(14) WC_FXAIQ_CASE(15) WC_FXAIQ_CASE(16)
#undef WC_FXAIQ_CASE
    default: return false;
  }
  if (launches) ++*launches;
  return true;
}

}  // namespace wc

// Shared device helpers for the GB300 Newton-solve library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define WC_SQRT2 1.41421356237309504880
#define WC_RSQRT2 0.70710678118654752440

namespace wc {

// Index of svec position (i, j), i >= j, in the column-by-column lower triangle of an n x n matrix.
__host__ __device__ __forceinline__ int64_t svec_index(int64_t n, int64_t i, int64_t j) {
  return j * n - (j * (j - 1)) / 2 + (i - j);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 doubles */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// FP64 tensor-core MMA: D(8x8) += A(8x4, row) * B(4x8, col).
// Fragment layout (lane = threadIdx % 32, g = lane >> 2, t = lane & 3):
//   a = A[g][t], b = B[t][g], c0 = C[g][2t], c1 = C[g][2t+1].
__device__ __forceinline__ void dmma_8x8x4(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
}

// L2 policy that marks lines first for eviction: a matrix streamed once per pass is loaded
// with it so that the small operands that should stay resident in L2 are not pushed out.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double2 ld_stream_d2(const double2* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream_d(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

// 16-byte streaming load of four int32 (evict-first L2 policy, no L1 allocation).
__device__ __forceinline__ int4 ld_stream_i4(const int4* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  return v;
}

// 16-byte streaming load of four floats (evict-first L2 policy, no L1 allocation).
__device__ __forceinline__ float4 ld_stream_f4(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream_f(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

// pack(H)[h] for H n x r with leading dimension ldH.
template <typename T>
__device__ __forceinline__ double pack_at(const T* __restrict__ H, int64_t ldH, int n, int r, int h) {
  const int nb = r * (r + 1) / 2;
  if (h < nb) {
    int j = 0, base = 0;
    while (h >= base + (r - j)) { base += r - j; ++j; }
    int i = j + (h - base);
    if (i == j) return (double)H[i + (int64_t)j * ldH];
    return WC_SQRT2 * 0.5 * ((double)H[i + (int64_t)j * ldH] + (double)H[j + (int64_t)i * ldH]);
  }
  int q = h - nb;
  int k = q % (n - r), j = q / (n - r);
  return WC_SQRT2 * (double)H[r + k + (int64_t)j * ldH];
}

// Device-resident PCG control block (one per handle).
// Scalars of the MINRES recurrence (Paige-Saunders form of Def. MINRES with P = I).
struct MinresCtl {
  double beta, oldb, alfa;       // Lanczos: beta_k, beta_{k-1}, alpha_k
  double dbar, epsln, oldeps;    // entries of the rotated tridiagonal
  double delta, gamma;
  double cs, sn;                 // the last Givens rotation
  double phi, phibar;            // phibar = ||r_k|| in exact arithmetic
  int32_t itn;                   // iterations begun
  int32_t stop;                  // 1 once the stop test held: the next iteration raises done
};

struct PcgCtl {
  double rz;        // <r_k, z_k>
  double rz_new;    // <r_{k+1}, z_{k+1}>
  double pAp;       // <p_k, A p_k>
  double alpha, beta;
  double rr;        // ||r||^2 after the update
  double g_norm2;   // ||g||^2
  double rr0;       // ||r_0||^2
  double newt_rhs2; // ||[svec C~; b~]||^2, the right side of (Newt-eps)
  double tol2;      // (rtol ||[svec C~; b~]||)^2
  int32_t done;     // 1 once the stop test held (or a breakdown occurred)
  int32_t iters;    // completed iterations
  int32_t max_iters;
  int32_t status;   // 0 ok, 5 numeric breakdown
  // split / setup scalars
  double tau, beta_pc, s_A;
  int32_t r, d;
  int32_t m_free;   // linear block: rows whose slack does not dominate (precond_space 3)
  int32_t pad1;
};

// Bounds-checked gathers and scatters (the debug build: the translation units that address
// arrays through index tables compiled with -DSDP_CHECK_BOUNDS).  WC_IN(site, i, bound) is true
// when 0 <= i < bound.  Otherwise it keeps (site, i) as the first violation seen by this
// translation unit, counts it, and is false: the caller skips the access.  Without the flag it
// is the constant true and the checks compile away.  Each checked translation unit registers a
// reader of its record with the library (oob_register); sdp_bounds_report calls the readers.
typedef int (*OobReader)(unsigned long long* first, unsigned long long* count);
void oob_register(OobReader rd);

#ifdef SDP_CHECK_BOUNDS
namespace {
__device__ unsigned long long oob_rec[2];   // first violation (site << 48 | index mod 2^48), count

__device__ __noinline__ bool oob_fail(int site, int64_t i) {
  const unsigned long long code = ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull);
  atomicCAS(&oob_rec[0], 0ull, code);
  atomicAdd(&oob_rec[1], 1ull);
  return false;
}

// Reads and clears this translation unit's record; returns the cudaError_t of the copies.
int oob_read(unsigned long long* first, unsigned long long* count) {
  unsigned long long v[2] = {0ull, 0ull};
  cudaError_t e = cudaMemcpyFromSymbol(v, oob_rec, sizeof v);
  if (e == cudaSuccess) {
    const unsigned long long z[2] = {0ull, 0ull};
    e = cudaMemcpyToSymbol(oob_rec, z, sizeof z);
  }
  *first = v[0];
  *count = v[1];
  return (int)e;
}

struct OobRegistration {
  OobRegistration() { oob_register(&oob_read); }
};
OobRegistration oob_registration;
}  // namespace

#define WC_IN(site, i, bound) \
  ((uint64_t)(int64_t)(i) < (uint64_t)(int64_t)(bound) ? true : ::wc::oob_fail((site), (int64_t)(i)))
#else
#define WC_IN(site, i, bound) true
#endif

}  // namespace wc

// The low-precision products of the mixed form: BF16 and TF32 matrix products on the tensor cores
// (tcgen05, FP32 accumulators in TMEM, operands staged by TMA) and the passes over a BF16 copy of
// the dense constraint rows (BF16 products summed in FP32).
//
// In the mixed form's correction solves the block A E A^T p_u of eq. augsys is formed as
//   Y = A^T(p_u)  (BF16 rows of A, FP32 sums)      -> Y in BF16 (or FP32 for TF32)
//   G = Y E, Z = E G  (two tensor-core products)   -> Z in FP32
//   A(Z)           (BF16 rows of A, FP32 sums)
// while the FP64 refinement around it (the true residual g - M x, Section 3 eq. augsys) keeps the
// accuracy of the Newton direction.
//
// Product kernel.  One CTA per 128 x 128 output tile, 5 warps: warp 4 (one lane) issues the TMA
// loads of 128-row x 128-byte K-slices of both operands (128-byte swizzle) into a 4-stage ring and
// the 128 x 128 x (16 BF16 | 8 TF32) MMA steps into one TMEM accumulator (128 FP32 columns);
// warps 0-3 then read their 32 TMEM lanes (= 32 output rows) and store the tile column by column
// (coalesced along the rows of the column-major output).  Every wait is bounded (2 s by default,
// %globaltimer): on expiry the kernel sets an error word, stops issuing, waits with the full bound
// for its own copies and products in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "handle.h"
#include "tc_ptx.cuh"

namespace wc {

namespace {

using namespace tcx;

constexpr int LBM = 128, LBN = 128;
constexpr int LTHREADS = 160;                      // warps 0-3: epilogue; warp 4: loads and MMA
constexpr int LTILE = 128 * 128;                   // bytes of one operand tile: 128 rows x 128 bytes
constexpr int LTMEM_COLS = 128;

// MODE 0: BF16 operands (kind::f16); 1: FP32 operands read as TF32 (kind::tf32); 2: the same with
// each FP32 operand given as hi + lo, both TF32-exact, and the product taken as
// hi_A hi_B + hi_A lo_B + lo_A hi_B (three TF32 MMAs per step; the dropped lo_A lo_B is below
// 2^-22 relative), which gives about FP32 accuracy on the tensor cores.
template <int MODE>
struct LpKind {
  static constexpr uint32_t fmt = MODE == 0 ? 1u : 2u;
  // instruction descriptor: K-major A and B, FP32 D, M = 128, N = 128, operand format fmt
  static constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(LBN >> 3) << 17) |
                                    ((uint32_t)(LBM >> 4) << 24);
  static constexpr int BK = MODE == 0 ? 64 : 32;   // elements per 128-byte K-slice
  static constexpr int TILES = MODE == 2 ? 4 : 2;  // operand tiles per stage (A [, A lo], B [, B lo])
  static constexpr int STAGES = MODE == 2 ? 3 : 4;
  static constexpr int STAGE = TILES * LTILE;
  static constexpr int SMEM = STAGES * STAGE + 1024;   // + alignment slack
};

template <int MODE>
__device__ __forceinline__ void lp_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  if constexpr (MODE != 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(LpKind<MODE>::idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(LpKind<MODE>::idesc), "r"(accumulate)
        : "memory");
  }
}

// TF32-exact part of an FP32 value (10 fraction bits, rounded to nearest)
__device__ __forceinline__ float tf32_hi(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// Output modes of the epilogue: 0 FP32, 1 BF16, 2 FP32 as the pair (hi, lo) with hi TF32-exact
template <int MODE>
__global__ void __launch_bounds__(LTHREADS, 1)
lp_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapA2,
               const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapB2, int M, int N,
               int K, float alpha, void* __restrict__ C, void* __restrict__ C2, int64_t ldc, int out_mode,
               int* __restrict__ err, const int32_t* __restrict__ done, unsigned long long wait_ns) {
  using KD = LpKind<MODE>;
  constexpr int STAGES = KD::STAGES, STAGE = KD::STAGE, BK = KD::BK;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  if (done && *done) return;
  const int m0 = blockIdx.x * LBM, n0 = blockIdx.y * LBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), 1);
    }
    mbar_init(smem_u32(&acc_bar), 1);
    abort_flag = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(LTMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      // stage layout: A, B (MODE 0, 1) or A hi, B hi, A lo, B lo (MODE 2)
      int g_load = 0, g_mma = 0;
      bool ok = true;
      for (int kt = 0; kt < nk && ok; ++kt) {
        while (g_load < nk && g_load < g_mma + STAGES) {
          const int st = g_load % STAGES;
          if (g_load >= STAGES &&
              !mbar_wait(smem_u32(&empty_bar[st]), ((g_load / STAGES) - 1) & 1, &abort_flag, err, wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[st]);
          const uint32_t sb = base + st * STAGE;
          mbar_expect_tx(fb, STAGE);
          tma_load_2d(sb, &mapA, g_load * BK, m0, fb);
          tma_load_2d(sb + LTILE, &mapB, g_load * BK, n0, fb);
          if constexpr (MODE == 2) {
            tma_load_2d(sb + 2 * LTILE, &mapA2, g_load * BK, m0, fb);
            tma_load_2d(sb + 3 * LTILE, &mapB2, g_load * BK, n0, fb);
          }
          ++g_load;
        }
        if (!ok) break;
        const int st = g_mma % STAGES;
        if (!mbar_wait(smem_u32(&full_bar[st]), (g_mma / STAGES) & 1, &abort_flag, err, wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = base + st * STAGE, b0 = a0 + LTILE;
#pragma unroll
        for (int sub = 0; sub < 4; ++sub) {          // 32 bytes of K per MMA step
          lp_mma<MODE>(tmem, smem_desc(a0 + sub * 32), smem_desc(b0 + sub * 32), (kt > 0 || sub > 0) ? 1u : 0u);
          if constexpr (MODE == 2) {
            lp_mma<MODE>(tmem, smem_desc(a0 + sub * 32), smem_desc(b0 + 2 * LTILE + sub * 32), 1u);   // hi lo
            lp_mma<MODE>(tmem, smem_desc(a0 + 2 * LTILE + sub * 32), smem_desc(b0 + sub * 32), 1u);   // lo hi
          }
        }
        mma_commit(smem_u32(&empty_bar[st]));        // the stage is free once these products finish
        ++g_mma;
      }
      if (ok) {
        mma_commit(smem_u32(&acc_bar));              // the accumulator is complete
      } else {
        abort_flag = 1;
        // bounded waits (full bound) for this CTA's own products and copies still in flight
        volatile int keep_waiting = 0;
        if (g_mma > 0) {
          const int st = (g_mma - 1) % STAGES;
          mbar_wait(smem_u32(&empty_bar[st]), ((g_mma - 1) / STAGES) & 1, &keep_waiting, err);
        }
        for (int g = g_mma; g < g_load; ++g)
          mbar_wait(smem_u32(&full_bar[g % STAGES]), (g / STAGES) & 1, &keep_waiting, err);
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (tile rows) ----
    // one decision per warp: the TMEM loads below are warp-collective
    const bool got = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_bar), 0, &abort_flag, err, wait_ns));
    if (got) {
      tc_fence_after();
      const int row = m0 + 32 * warp + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < LBN; c0 += 32) {
        uint32_t r[32];
        WC_TMEM_LD32(tmem + (uint32_t)c0 + ((uint32_t)(32 * warp) << 16), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            if (col >= N) continue;
            const float v = alpha * __uint_as_float(r[j]);
            const int64_t at = (int64_t)row + (int64_t)col * ldc;
            if (out_mode == 1) {
              static_cast<__nv_bfloat16*>(C)[at] = __float2bfloat16_rn(v);
            } else if (out_mode == 2) {
              const float hi = tf32_hi(v);
              static_cast<float*>(C)[at] = hi;
              static_cast<float*>(C2)[at] = v - hi;
            } else {
              static_cast<float*>(C)[at] = v;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 4)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LTMEM_COLS) : "memory");
}

// ---- passes over the BF16 rows ----------------------------------------------------------------

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__device__ __forceinline__ void fma8(float* acc, const uint4& v, float s) {
  acc[0] = fmaf(s, bf_lo(v.x), acc[0]);
  acc[1] = fmaf(s, bf_hi(v.x), acc[1]);
  acc[2] = fmaf(s, bf_lo(v.y), acc[2]);
  acc[3] = fmaf(s, bf_hi(v.y), acc[3]);
  acc[4] = fmaf(s, bf_lo(v.z), acc[4]);
  acc[5] = fmaf(s, bf_hi(v.z), acc[5]);
  acc[6] = fmaf(s, bf_lo(v.w), acc[6]);
  acc[7] = fmaf(s, bf_hi(v.w), acc[7]);
}

__device__ __forceinline__ float dot8(const uint4& v, const float4& z0, const float4& z1, float acc) {
  acc = fmaf(bf_lo(v.x), z0.x, acc);
  acc = fmaf(bf_hi(v.x), z0.y, acc);
  acc = fmaf(bf_lo(v.y), z0.z, acc);
  acc = fmaf(bf_hi(v.y), z0.w, acc);
  acc = fmaf(bf_lo(v.z), z1.x, acc);
  acc = fmaf(bf_hi(v.z), z1.y, acc);
  acc = fmaf(bf_lo(v.w), z1.z, acc);
  acc = fmaf(bf_hi(v.w), z1.w, acc);
  return acc;
}

constexpr int GT_T = 256;

// part[g * Lp + c .. c + 7] = sum over the rows i of group g of p_i a[i, c .. c + 7]; eight
// columns (one 16-byte load) per thread and row, four rows in flight
__global__ void __launch_bounds__(GT_T) bf16_gemvT_kernel(const uint4* __restrict__ A, int m, int64_t Lp,
                                                          const float* __restrict__ p, float* __restrict__ part,
                                                          int rpg, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int64_t cv = (int64_t)blockIdx.x * GT_T + threadIdx.x;   // in units of 8 columns
  const int64_t nv = Lp / 8;
  if (cv >= nv) return;
  const int g = blockIdx.y;
  const int i0 = g * rpg, i1 = min(m, i0 + rpg);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int i = i0;
  for (; i + 7 < i1; i += 8) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(A + (int64_t)(i + u) * nv + cv);
#pragma unroll
    for (int u = 0; u < 8; ++u) fma8(acc, v[u], __ldg(p + i + u));
  }
  for (; i < i1; ++i) fma8(acc, __ldg(A + (int64_t)i * nv + cv), __ldg(p + i));
  float4* o = reinterpret_cast<float4*>(part + (int64_t)g * Lp + cv * 8);
  o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

// out[s m + i] = <a[i, slab s], z[slab s]>: one warp per row and column slab (blockIdx.y), four
// 16-byte loads in flight per lane; the slabs' partial sums are added by the consumer
__global__ void __launch_bounds__(256) bf16_gemv_kernel(const uint4* __restrict__ A, int m, int64_t Lp,
                                                        const float4* __restrict__ z, float* __restrict__ out,
                                                        const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int row = (int)(((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const int64_t nvall = Lp / 8;
  const int64_t per = (nvall + gridDim.y - 1) / gridDim.y;
  const int64_t q0 = (int64_t)blockIdx.y * per;
  const int64_t nv = min(nvall, q0 + per);
  const uint4* a = A + (int64_t)row * nvall;
  float acc0 = 0.f, acc1 = 0.f;
  int64_t q = q0 + lane;
  for (; q + 96 < nv; q += 128) {
    const uint4 v0 = __ldg(a + q), v1 = __ldg(a + q + 32), v2 = __ldg(a + q + 64), v3 = __ldg(a + q + 96);
    acc0 = dot8(v0, __ldg(z + 2 * q), __ldg(z + 2 * q + 1), acc0);
    acc1 = dot8(v1, __ldg(z + 2 * (q + 32)), __ldg(z + 2 * (q + 32) + 1), acc1);
    acc0 = dot8(v2, __ldg(z + 2 * (q + 64)), __ldg(z + 2 * (q + 64) + 1), acc0);
    acc1 = dot8(v3, __ldg(z + 2 * (q + 96)), __ldg(z + 2 * (q + 96) + 1), acc1);
  }
  for (; q < nv; q += 32) acc0 = dot8(__ldg(a + q), __ldg(z + 2 * q), __ldg(z + 2 * q + 1), acc0);
  float acc = acc0 + acc1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[(int64_t)blockIdx.y * m + row] = acc;
}

// Y[a + b ldk] = smat(sum_g part[g Lp + .]) in BF16 or FP32 (group partials summed in order)
template <typename T>
__global__ void lp_unpack_kernel(int n, const float* __restrict__ part, int groups, int64_t Lp, T* __restrict__ Y,
                                 int ldk, float* __restrict__ Ylo, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int a = (int)(q % n), b = (int)(q / n);
  const int i = a > b ? a : b, j = a > b ? b : a;
  const int64_t idx = svec_index(n, i, j);
  float s = 0.f;
  for (int g = 0; g < groups; ++g) s += __ldg(part + (int64_t)g * Lp + idx);
  const float v = (a == b) ? s : s * (float)WC_RSQRT2;
  if constexpr (sizeof(T) == 2) {
    Y[a + (int64_t)b * ldk] = __float2bfloat16_rn(v);
  } else if (Ylo) {                                 // (hi, lo) pair for the split TF32 products
    const float hi = tf32_hi(v);
    Y[a + (int64_t)b * ldk] = hi;
    Ylo[a + (int64_t)b * ldk] = v - hi;
  } else {
    Y[a + (int64_t)b * ldk] = v;
  }
}

template <typename T>
__global__ void lp_convert_kernel(int rows, int cols, const double* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                  int64_t ldy, float* __restrict__ Ylo) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)rows * ldy) return;
  const int64_t r = q / ldy, c = q % ldy;
  const double v = c < cols ? X[r * ldx + c] : 0.0;
  if constexpr (sizeof(T) == 2) {
    Y[q] = __double2bfloat16(v);
  } else if (Ylo) {                                 // (hi, lo): hi TF32-exact, lo the FP32 remainder
    const float f = (float)v;
    const float hi = tf32_hi(f);
    Y[q] = hi;
    Ylo[q] = f - hi;
  } else {
    Y[q] = (float)v;
  }
}

}  // namespace

std::atomic<unsigned long long> g_main_wait_ns_lp{tcx::kWaitNs};

cudaError_t lp_prepare() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(lp_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, LpKind<0>::SMEM);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(lp_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, LpKind<1>::SMEM);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(lp_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, LpKind<2>::SMEM);
  });
  return err;
}

cudaError_t lp_gemm(cudaStream_t st, int mode, int M, int N, int K, float alpha, const void* A, const void* Alo,
                    int64_t lda, const void* B, const void* Blo, int64_t ldb, void* C, void* Clo, int64_t ldc,
                    int out_mode, int* err, int64_t* launches, const int32_t* done) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 1 || !A || !B || !C || !err || mode < 0 || mode > 2 || out_mode < 0 || out_mode > 2) return cudaErrorInvalidValue;
  if (mode == 2 && (!Alo || !Blo)) return cudaErrorInvalidValue;
  if (out_mode == 2 && !Clo) return cudaErrorInvalidValue;
  const int esz = mode == 0 ? 2 : 4;
  if (((lda * esz) & 15) || ((ldb * esz) & 15) || (reinterpret_cast<uintptr_t>(A) & 15) ||
      (reinterpret_cast<uintptr_t>(B) & 15) || (reinterpret_cast<uintptr_t>(Alo) & 15) ||
      (reinterpret_cast<uintptr_t>(Blo) & 15) || lda < K || ldb < K)
    return cudaErrorInvalidValue;
  cudaError_t e = lp_prepare();
  if (e != cudaSuccess) return e;
  const bool f32 = mode != 0;
  const uint32_t bk = f32 ? 32u : 64u;
  CUtensorMap mapA, mapB, mapA2, mapB2;
  e = tmap_2d(&mapA, f32, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda * esz, bk, LBM);
  if (e == cudaSuccess) e = tmap_2d(&mapB, f32, B, (uint64_t)K, (uint64_t)N, (uint64_t)ldb * esz, bk, LBN);
  if (e == cudaSuccess && mode == 2) {
    e = tmap_2d(&mapA2, true, Alo, (uint64_t)K, (uint64_t)M, (uint64_t)lda * esz, bk, LBM);
    if (e == cudaSuccess) e = tmap_2d(&mapB2, true, Blo, (uint64_t)K, (uint64_t)N, (uint64_t)ldb * esz, bk, LBN);
  } else {
    mapA2 = mapA;
    mapB2 = mapB;
  }
  if (e != cudaSuccess) return e;
  const dim3 grid((M + LBM - 1) / LBM, (N + LBN - 1) / LBN);
  const unsigned long long wns = g_main_wait_ns_lp.load();
  if (mode == 0)
    lp_gemm_kernel<0><<<grid, LTHREADS, LpKind<0>::SMEM, st>>>(mapA, mapA2, mapB, mapB2, M, N, K, alpha, C, Clo, ldc,
                                                               out_mode, err, done, wns);
  else if (mode == 1)
    lp_gemm_kernel<1><<<grid, LTHREADS, LpKind<1>::SMEM, st>>>(mapA, mapA2, mapB, mapB2, M, N, K, alpha, C, Clo, ldc,
                                                               out_mode, err, done, wns);
  else
    lp_gemm_kernel<2><<<grid, LTHREADS, LpKind<2>::SMEM, st>>>(mapA, mapA2, mapB, mapB2, M, N, K, alpha, C, Clo, ldc,
                                                               out_mode, err, done, wns);
  if (launches) ++*launches;
  return cudaGetLastError();
}

int bf16_gemvT_groups(int m, int64_t Lp) {
  // enough CTAs for about four per SM: column blocks x row groups, at least 8 rows per group
  const int64_t cblocks = (Lp / 8 + GT_T - 1) / GT_T;
  int64_t groups = (4LL * g_num_sms + cblocks - 1) / cblocks;
  groups = std::max<int64_t>(1, std::min<int64_t>(groups, (m + 7) / 8));
  return (int)groups;
}

void bf16_gemvT(cudaStream_t st, const void* A16, int m, int64_t Lp, const float* p, float* part, int groups,
                const int32_t* done, int64_t* launches) {
  const int rpg = (m + groups - 1) / groups;
  const int64_t nv = Lp / 8;
  const dim3 grid((unsigned)((nv + GT_T - 1) / GT_T), (unsigned)groups);
  bf16_gemvT_kernel<<<grid, GT_T, 0, st>>>(static_cast<const uint4*>(A16), m, Lp, p, part, rpg, done);
  if (launches) ++*launches;
}

int bf16_gemv_slabs(int m, int64_t Lp) {
  // about 48 warps per SM in flight: m rows x slabs warps, each slab at least 2048 columns
  int64_t slabs = (48LL * g_num_sms + m - 1) / m;
  slabs = std::max<int64_t>(1, std::min<int64_t>(slabs, Lp / 2048));
  return (int)std::min<int64_t>(slabs, 16);
}

void bf16_gemv(cudaStream_t st, const void* A16, int m, int64_t Lp, const float* z, float* out, int slabs,
               const int32_t* done, int64_t* launches) {
  const dim3 grid((unsigned)(((int64_t)m * 32 + 255) / 256), (unsigned)slabs);
  bf16_gemv_kernel<<<grid, 256, 0, st>>>(static_cast<const uint4*>(A16), m, Lp, reinterpret_cast<const float4*>(z),
                                         out, done);
  if (launches) ++*launches;
}

void lp_unpack(cudaStream_t st, int n, const float* part, int groups, int64_t Lp, void* Y, int ldk, bool bf16,
               float* Ylo, const int32_t* done, int64_t* launches) {
  const int64_t nn = (int64_t)n * n;
  const unsigned blocks = (unsigned)((nn + 255) / 256);
  if (bf16)
    lp_unpack_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(n, part, groups, Lp, static_cast<__nv_bfloat16*>(Y), ldk,
                                                            nullptr, done);
  else
    lp_unpack_kernel<float><<<blocks, 256, 0, st>>>(n, part, groups, Lp, static_cast<float*>(Y), ldk, Ylo, done);
  if (launches) ++*launches;
}

void lp_convert(cudaStream_t st, int rows, int cols, const double* X, int64_t ldx, void* Y, int64_t ldy, bool bf16,
                float* Ylo, int64_t* launches) {
  const int64_t tot = (int64_t)rows * ldy;
  const unsigned blocks = (unsigned)((tot + 255) / 256);
  if (bf16)
    lp_convert_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(rows, cols, X, ldx, static_cast<__nv_bfloat16*>(Y), ldy,
                                                             nullptr);
  else
    lp_convert_kernel<float><<<blocks, 256, 0, st>>>(rows, cols, X, ldx, static_cast<float*>(Y), ldy, Ylo);
  if (launches) ++*launches;
}

}  // namespace wc

// Test access to the low-precision product through the C ABI (declared in wcipm.h).
extern "C" sdp_status sdp_gemm_tn_lp(void* stream, int32_t tf32, int32_t M, int32_t N, int32_t K, float alpha,
                                     const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                                     int32_t* err_word) {
  using namespace wc;
  if (M < 1 || N < 1 || K < 1) return wc_fail(nullptr, SDP_EINVAL, "sizes must be >= 1");
  if (!A || !B || !C || !err_word) return wc_fail(nullptr, SDP_EINVAL, "NULL array argument");
  const int esz = tf32 ? 4 : 2;
  if (lda < K || ldb < K || ldc < M || ((lda * esz) & 15) || ((ldb * esz) & 15) ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return wc_fail(nullptr, SDP_EINVAL, "operands need lda, ldb >= K with 16-byte rows and 16-byte aligned bases");
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
    return wc_fail(nullptr, SDP_ECUDA, "no CUDA device");
  if (major != 10) return wc_fail(nullptr, SDP_EUNSUPPORTED, "tcgen05 products need a Blackwell (sm_10x) device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(err_word, 0, sizeof(int32_t), st) != cudaSuccess)
    return wc_fail(nullptr, SDP_ECUDA, "clearing the error word");
  cudaError_t e = lp_gemm(st, tf32 ? 1 : 0, M, N, K, alpha, A, nullptr, lda, B, nullptr, ldb, C, nullptr, ldc, 0,
                          err_word, nullptr);
  if (e != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, std::string("low-precision product: ") + cudaGetErrorString(e));
  int32_t h_err = 0;
  e = cudaMemcpyAsync(&h_err, err_word, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, std::string("low-precision product: ") + cudaGetErrorString(e));
  if (h_err) return wc_fail(nullptr, SDP_ETIMEOUT, "a bounded wait of the low-precision product gave up");
  return SDP_OK;
}

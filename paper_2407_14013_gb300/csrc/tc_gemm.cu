// FP64 matrix products on the BF16 tensor cores: tcgen05 MMA with TMEM accumulators, operands
// staged by TMA, FP64 accuracy from exact integer slices (the Ozaki splitting).
//
//   C (M x N) = alpha * op(A) * op(B) + beta * C     (column-major, as gemm_f64)
//
// Splitting.  Row i of op(A) is scaled by 2^-e_i with 2^e_i > max_k |op(A)[i, k]|, so that its
// entries a lie in (-1, 1), and written as a = sum_{s=1..8} a_s 2^-(7s-1) with integers
// |a_s| <= 64: a_1 = rint(2^6 a), then each residual (|r| <= 1/2) times 2^7 rounded again.
// Every a_s is exact in BF16 (8 significand bits).  Columns of op(B) likewise (exponents f_j).
// Then op(A) op(B) = 2^(e_i + f_j) sum_{s,t} 2^-(7(s+t)-2) (A_s B_t), and each integer product
// A_s B_t over a K-chunk of at most 4096 has |sum| <= 4096 * 64 * 64 = 2^24: exact in the FP32
// accumulator of the tensor core.  The chunk results are scaled by the power of two and summed
// in FP64.  Pairs with s + t <= 9 are kept (36 BF16 products): a dropped term is below
// 2^-68 max_k|op(A)[i,k]| max_k|op(B)[k,j]| per element of K, and the splitting error of one
// entry is at most 2^-56 of its row maximum, so the product is accurate to about K 2^-55
// max_k|op(A)[i,k]| max_k|op(B)[k,j]| -- the FP64 bound when the rows and columns have no
// large internal dynamic range (use gemm_f64 where they do).
//
// Kernel (tc_gemm_cls_kernel below).  One CTA per 128 x 64 output tile: the eight slices of op(B)
// for a K-step are loaded once and each slice of op(A) meets all the B slices its pairs need, into
// one TMEM accumulator per weight class s + t; the class sums are exact in FP32 over K-chunks of
// 512 and are folded into exact int64 sums by the epilogue warps, so FP64 arithmetic is needed only
// once per output.  Every wait is bounded (about 2 s, %globaltimer): on expiry the kernel sets an
// error word, stops issuing, waits (bounded) for its own copies and products in flight, frees its
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include <string>

#include "handle.h"
#include "tc_ptx.cuh"

namespace wc {

namespace {

constexpr int S = 8;                  // slices per operand
constexpr int KC = 4096;              // host K-chunks are whole multiples of this where possible
constexpr int BK = 64;                // K-slice of one TMA box (128 bytes of BF16)
constexpr unsigned long long WAIT_NS = tcx::kWaitNs;

// ---- PTX wrappers: tc_ptx.cuh; the MMA of this kernel ----------------------------------------

using namespace tcx;

// ---- splitting ------------------------------------------------------------------------------
// Two passes over X(r, k) = X[r * rs + k * ks] (R x K): the largest magnitude of every row
// (bit patterns of non-negative doubles order like the doubles), then the slices.  The
// slices of x in row r with exponent e (2^e > max |row|) are the signed base-128 digits of the
// integer N = round(x 2^(55 - e)), |N| < 2^55: N = sum_{s=1..8} a_s 128^(8-s) with a_2..a_8 the
// centred remainders in [-64, 63] and a_1 in [-64, 64]; then x 2^-e = sum_s a_s 2^-(7s-1) up to
// the rounding of N (at most 2^-56).  Integer arithmetic only (no FP64 pipe); the BF16 bits of
// -64..64 come from a shared-memory table.

// max_k |op(X)[r, k]| as IEEE bits (monotone for non-negative doubles), over blocks of 32 rows x
// 256 entries of K: lanes run along whichever axis is contiguous, and one atomic per row and warp
// merges the blocks.
__global__ void __launch_bounds__(256) rowmax_kernel(int R, int K, const double* __restrict__ X, int64_t rs,
                                                     int64_t ks, unsigned long long* __restrict__ rmax,
                                                     const int32_t* __restrict__ done) {
  if (done && *done) return;
  __shared__ unsigned long long sm[8][32];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 256, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
  if (rs == 1) {                           // rows contiguous: lane <-> row, the warps split K
    const int gr = r0 + lane;
    unsigned long long mx = 0ull;
    if (gr < R)
      for (int k = warp; k < 256; k += 8) {
        const int gk = k0 + k;
        if (gk >= K) break;
        const unsigned long long b = (unsigned long long)__double_as_longlong(X[gr + (int64_t)gk * ks]) & ABS;
        mx = b > mx ? b : mx;
      }
    sm[warp][lane] = mx;
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int w = 1; w < 8; ++w) mx = sm[w][lane] > mx ? sm[w][lane] : mx;
      if (gr < R && mx) atomicMax(&rmax[gr], mx);
    }
  } else {                                 // K contiguous: warp <-> row, lanes along K
    for (int r = warp; r < 32; r += 8) {
      const int gr = r0 + r;
      if (gr >= R) break;
      unsigned long long mx = 0ull;
      for (int k = lane; k < 256; k += 32) {
        const int gk = k0 + k;
        if (gk >= K) break;
        const unsigned long long b = (unsigned long long)__double_as_longlong(X[(int64_t)gr * rs + (int64_t)gk * ks]) & ABS;
        mx = b > mx ? b : mx;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
      }
      if (lane == 0 && mx) atomicMax(&rmax[gr], mx);
    }
  }
}

__device__ __forceinline__ int row_exponent(unsigned long long mbits) {
  if (mbits == 0ull) return 0;
  return ilogb(__longlong_as_double((long long)mbits)) + 1;
}

// N = round(x 2^(55 - e)) from the IEEE fields of x: |x| = m 2^(ex - 1075), m < 2^53
__device__ __forceinline__ long long fixed_point(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ex) m |= 1ull << 52;
  const int sh = (ex ? ex : 1) - 1075 + 55 - e;
  long long Nv;
  if (m == 0ull || sh <= -64) Nv = 0;
  else if (sh >= 0) Nv = (long long)(m << sh);                         // sh <= 2: |N| < 2^55
  else Nv = (long long)((m + (1ull << (-sh - 1))) >> (-sh));          // rounded
  return (b >> 63) ? -Nv : Nv;
}

// One block per 32 rows x BK entries of op(X): the tile is staged in shared memory (coalesced
// whichever of rows or K is contiguous), then each thread turns 8 consecutive entries of one
// row into their 8 slices and writes each slice plane with one 16-byte store.
__global__ void __launch_bounds__(256) slice_kernel(int R, int K, int Kpad, const double* __restrict__ X,
                                                    int64_t rs, int64_t ks,
                                                    const unsigned long long* __restrict__ rmax,
                                                    __nv_bfloat16* __restrict__ out, int* __restrict__ expo,
                                                    const int32_t* __restrict__ done) {
  if (done && *done) return;
  __shared__ double tile[32][BK + 1];
  __shared__ unsigned short bf[129];
  __shared__ int rexp[32];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * BK, tid = threadIdx.x;
  if (tid < 129) bf[tid] = __bfloat16_as_ushort(__float2bfloat16((float)(tid - 64)));   // exact
  if (tid < 32) {
    const int e = (r0 + tid < R) ? row_exponent(rmax[r0 + tid]) : 0;
    rexp[tid] = e;
    if (blockIdx.y == 0 && r0 + tid < R) expo[r0 + tid] = e;
  }
  const bool rows_contig = (rs == 1);
  for (int q = tid; q < 32 * BK; q += 256) {
    int r, k;
    if (rows_contig) { r = q % 32; k = q / 32; } else { k = q % BK; r = q / BK; }
    const int gr = r0 + r, gk = k0 + k;
    tile[r][k] = (gr < R && gk < K) ? X[(int64_t)gr * rs + (int64_t)gk * ks] : 0.0;
  }
  __syncthreads();
  static_assert(BK == 64, "8 threads x 8 entries per row");
  const int r = tid >> 3, g = tid & 7;
  const int gr = r0 + r;
  if (gr >= R) return;
  // N = hi 2^28 + lo with 0 <= lo < 2^28: the four low digits come from lo and carry into hi
  // (at most 1), the four high ones from hi; the same centred digits as the 64-bit recursion,
  // in 32-bit integer arithmetic
  int hi[8], lo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long Nv = fixed_point(tile[r][g * 8 + j], rexp[r]);
    hi[j] = (int)(Nv >> 28);
    lo[j] = (int)(Nv & 0xFFFFFFFll);
  }
  // Kpad is a multiple of BK, so every row, plane and group of 8 starts on 16 bytes
  const int64_t plane16 = (int64_t)R * Kpad / 8;
  uint4* o = reinterpret_cast<uint4*>(out + (int64_t)gr * Kpad + k0 + g * 8);
#pragma unroll
  for (int sidx = S - 1; sidx >= 0; --sidx) {                           // a_8 .. a_1
    uint32_t wv[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      int a[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        int& x = sidx >= 4 ? lo[j + u] : hi[j + u];
        if (sidx > 0) {
          a[u] = ((x + 64) & 127) - 64;
          x = (x - a[u]) >> 7;                                         // exact
        } else {
          a[u] = x;                                                     // a_1, |a_1| <= 64
        }
      }
      if (sidx == 4) {                                                  // lo is spent: its carry goes up
        hi[j] += lo[j];
        hi[j + 1] += lo[j + 1];
      }
      wv[j / 2] = (uint32_t)bf[a[0] + 64] | ((uint32_t)bf[a[1] + 64] << 16);
    }
    o[sidx * plane16] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// ---- the product, class-accumulator form -------------------------------------------------------
// One CTA per 128 x 64 output tile.  Per K-step of 64 the eight slices of op(B) (64 x 64 tiles)
// are loaded once into a 2-stage buffer and the eight slices of op(A) (128 x 64 tiles) stream
// through a 4-stage ring; slice s of A meets slices t = 1 .. 9 - s of B, and each pair's product
// goes to the TMEM accumulator of its weight class g = s + t (8 classes x 64 FP32 columns: all
// 512 columns).  So each loaded tile serves up to eight MMAs instead of one, which is what the
// pairwise form lacked (it re-streamed both tiles for every pair and waited on L2).  A class sum
// over a K-chunk of 512 is an integer of at most 8 x 512 x 64 x 64 = 2^24: exact in FP32.  After
// each chunk the eight epilogue warps read the classes and fold them exactly into two int64
// sums per element, T_hi = sum_{g=2..5} S_g 2^(7(5-g)) and T_lo = sum_{g=6..9} S_g 2^(7(9-g))
// (each below 2^43 per chunk), so the only FP64 work is the final
// 2^(e_i + f_j) (T_hi 2^-33 + T_lo 2^-61).  Warp 8 (one lane) issues the TMA loads, warp 9 (one
// lane) the MMAs; every wait is bounded as in the pairwise form.

constexpr int CBM = 128, CBN = 64, CKC = 512;               // tile, exact K-chunk
constexpr int CRA = 4, CRB = 2;                              // A ring, B stages
constexpr int CA_TILE = CBM * BK * 2;                        // 16 KB
constexpr int CB_TILE = CBN * BK * 2;                        // 8 KB
constexpr int CB_STAGE = S * CB_TILE;                        // 64 KB: the eight slices of B
constexpr int CSMEM = CRA * CA_TILE + CRB * CB_STAGE + 1024;
constexpr int CEPI = 8;                                      // epilogue warps
constexpr int CTHREADS = (CEPI + 2) * 32;
constexpr uint32_t CIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CBN >> 3) << 17) |
                            ((uint32_t)(CBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16_c(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(CIDESC), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(CTHREADS, 1)
tc_gemm_cls_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                   int N, int K, int ksplit, const int* __restrict__ ea, const int* __restrict__ eb, double alpha,
                   double beta, double* __restrict__ C, int64_t ldc, double* __restrict__ part, int lower,
                   int* __restrict__ err, const int32_t* __restrict__ done, unsigned long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t fullA[CRA], emptyA[CRA], fullB[CRB], emptyB[CRB], accF, accE;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * CBN;
  if (lower && m0 + CBM <= n0) return;               // tile entirely above the diagonal
  if (done && *done) return;
  const int kz0 = blockIdx.z * ksplit;
  const int Kz = min(K, kz0 + ksplit) - kz0;
  const int nks = Kz > 0 ? (Kz + BK - 1) / BK : 0;   // K-steps of this CTA
  constexpr int KCS = CKC / BK;                      // K-steps per exact chunk
  const int nch = (nks + KCS - 1) / KCS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t abase = base, bbase = base + CRA * CA_TILE;

  if (threadIdx.x == 0) {
    for (int i = 0; i < CRA; ++i) {
      mbar_init(smem_u32(&fullA[i]), 1);
      mbar_init(smem_u32(&emptyA[i]), 1);
    }
    for (int i = 0; i < CRB; ++i) {
      mbar_init(smem_u32(&fullB[i]), 1);
      mbar_init(smem_u32(&emptyB[i]), 1);
    }
    mbar_init(smem_u32(&accF), 1);
    mbar_init(smem_u32(&accE), CEPI);
    abort_flag = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == CEPI + 1) {                            // TMEM: eight 64-column class accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == CEPI) {
    // ---- TMA loads (one thread): per K-step the eight B slices, then the eight A slices ----
    if (lane == 0) {
      int ga = 0, gb = 0;
      bool ok = true;
      for (int ks = 0; ks < nks && ok; ++ks) {
        const int k0 = kz0 + ks * BK;
        const int sb = gb % CRB;
        if (gb >= CRB && !mbar_wait(smem_u32(&emptyB[sb]), ((gb / CRB) - 1) & 1, &abort_flag, err, wait_ns)) {
          ok = false;
          break;
        }
        const uint32_t fb = smem_u32(&fullB[sb]);
        mbar_expect_tx(fb, CB_STAGE);
        for (int t = 0; t < S; ++t) tma_load_3d(bbase + sb * CB_STAGE + t * CB_TILE, &mapB, k0, n0, t, fb);
        ++gb;
        for (int sidx = 0; sidx < S; ++sidx) {
          const int sa = ga % CRA;
          if (ga >= CRA && !mbar_wait(smem_u32(&emptyA[sa]), ((ga / CRA) - 1) & 1, &abort_flag, err, wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t fa = smem_u32(&fullA[sa]);
          mbar_expect_tx(fa, CA_TILE);
          tma_load_3d(abase + sa * CA_TILE, &mapA, k0, m0, sidx, fa);
          ++ga;
        }
      }
      if (!ok) {
        abort_flag = 1;
        // bounded waits (full bound) for this CTA's own copies in flight: the last loads of each
        // ring (older ones were consumed, so they completed)
        volatile int keep_waiting = 0;
        for (int g = max(0, ga - CRA); g < ga; ++g)
          mbar_wait(smem_u32(&fullA[g % CRA]), (g / CRA) & 1, &keep_waiting, err);
        for (int g = max(0, gb - CRB); g < gb; ++g)
          mbar_wait(smem_u32(&fullB[g % CRB]), (g / CRB) & 1, &keep_waiting, err);
      }
    }
  } else if (warp == CEPI + 1) {
    // ---- MMAs (one thread) ----
    if (lane == 0) {
      int ga = 0, gb = 0;
      bool ok = true, issued = false;
      uint32_t init = 0;                             // classes already written in this chunk
      for (int ks = 0; ks < nks && ok; ++ks) {
        if (ks % KCS == 0) {
          if (ks > 0 && !mbar_wait(smem_u32(&accE), ((ks / KCS) - 1) & 1, &abort_flag, err, wait_ns)) {
            ok = false;                              // the previous chunk is not drained yet
            break;
          }
          tc_fence_after();
          init = 0;
        }
        const int sb = gb % CRB;
        if (!mbar_wait(smem_u32(&fullB[sb]), (gb / CRB) & 1, &abort_flag, err, wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t b0 = bbase + sb * CB_STAGE;
        for (int sidx = 0; sidx < S && ok; ++sidx) {
          const int sa = ga % CRA;
          if (!mbar_wait(smem_u32(&fullA[sa]), (ga / CRA) & 1, &abort_flag, err, wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = abase + sa * CA_TILE;
          for (int t = 0; sidx + t < S; ++t) {       // (s + 1) + (t + 1) <= S + 1
            const int cls = sidx + t;
            const uint32_t dcol = tmem + (uint32_t)(cls * CBN);
            const uint32_t bt = b0 + t * CB_TILE;
#pragma unroll
            for (int sub = 0; sub < BK / 16; ++sub)
              mma_bf16_c(dcol, smem_desc(a0 + sub * 32), smem_desc(bt + sub * 32),
                         ((init >> cls) & 1u) || sub > 0 ? 1u : 0u);
            init |= 1u << cls;
          }
          mma_commit(smem_u32(&emptyA[sa]));         // the A slot is free once these products finish
          issued = true;
          ++ga;
        }
        if (!ok) break;
        mma_commit(smem_u32(&emptyB[sb]));
        ++gb;
        if (ks % KCS == KCS - 1 || ks == nks - 1) mma_commit(smem_u32(&accF));   // chunk complete
      }
      if (!ok) {
        abort_flag = 1;
        volatile int keep_waiting = 0;
        if (issued) {                                // the last commit covers every product issued
          const int g = ga - 1;
          mbar_wait(smem_u32(&emptyA[g % CRA]), (g / CRA) & 1, &keep_waiting, err);
        }
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows), columns 32 (w / 4) .. + 31
    // of every class; exact int64 sums across the chunks ----
    const int q4 = warp & 3, hc = warp >> 2;
    long long thi[32], tlo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) thi[j] = tlo[j] = 0;
    bool got = true;
    for (int ch = 0; ch < nch; ++ch) {
      got = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accF), ch & 1, &abort_flag, err, wait_ns));
      if (!got) break;
      tc_fence_after();
#pragma unroll 1
      for (int cls = 0; cls < S; ++cls) {
        uint32_t r[32];
        WC_TMEM_LD32(tmem + (uint32_t)(cls * CBN + hc * 32) + ((uint32_t)(32 * q4) << 16), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int g = cls + 2;
        if (g <= 5) {
          const int sh = 7 * (5 - g);
#pragma unroll
          for (int j = 0; j < 32; ++j) thi[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
        } else {
          const int sh = 7 * (9 - g);
#pragma unroll
          for (int j = 0; j < 32; ++j) tlo[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&accE));
    }
    if (got && !abort_flag) {
      const int row = m0 + 32 * q4 + lane;
      if (row < M) {
        const int er = ea[row];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + hc * 32 + j;
          if (col >= N) continue;
          const double a = fma((double)thi[j], 0x1p-33, (double)tlo[j] * 0x1p-61);
          if (part) {                                // partial tile of this K range
            part[(int64_t)blockIdx.z * M * N + row + (int64_t)col * M] = scalbn(a, er + eb[col]);
          } else {
            const double v = alpha * scalbn(a, er + eb[col]);
            double* cp = C + (int64_t)row + (int64_t)col * ldc;
            *cp = (beta == 0.0) ? v : v + beta * *cp;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == CEPI + 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// C = alpha sum_z part[z] + beta C over the split K ranges, in z order (deterministic); tiles
// above the diagonal are skipped when `lower` is set, as in the product.
__global__ void tc_reduce_kernel(int M, int N, int nz, const double* __restrict__ part, double alpha, double beta,
                                 double* __restrict__ C, int64_t ldc, int lower, const int32_t* __restrict__ done,
                                 const int* __restrict__ err) {
  if (done && *done) return;
  if (*err) return;                          // a product tile gave up: its partials are not written
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)M * N) return;
  const int row = (int)(q % M), col = (int)(q / M);
  if (lower && (row / CBM) * CBM + CBM <= (col / CBN) * CBN) return;
  double sum = 0.0;
  for (int z = 0; z < nz; ++z) sum += part[(int64_t)z * M * N + q];
  double* cp = C + (int64_t)row + (int64_t)col * ldc;
  *cp = (beta == 0.0) ? alpha * sum : alpha * sum + beta * *cp;
}

// ---- host side ------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

cudaError_t encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      g_encode_err = (e != cudaSuccess) ? e : cudaErrorNotSupported;
      return;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode ? cudaSuccess : g_encode_err;
}

cudaError_t make_map(CUtensorMap* map, const void* slices, int rows, int Kpad, int box_rows) {
  const cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)S};
  const cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)rows * Kpad * 2};
  const cuuint32_t box[3] = {BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(slices), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// 2-D tiled tensor map (128-byte swizzle) over a row-pitched matrix: `rows` rows of `inner`
// elements (BF16 or FP32), `pitch_bytes` apart; boxes of box_inner x box_rows.  Reads outside the
// matrix return zeros.
cudaError_t tmap_2d(CUtensorMap* map, bool f32, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch_bytes,
                    uint32_t box_inner, uint32_t box_rows) {
  cudaError_t e = encode_fn();
  if (e != cudaSuccess) return e;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

// limit of the main-loop waits of the product (sdp_set_tc_wait_limit_ns); the drain after an
// expiry always keeps WAIT_NS
std::atomic<unsigned long long> g_main_wait_ns{WAIT_NS};
inline int kpad_of(int K) { return (K + BK - 1) / BK * BK; }

}  // namespace

// split-K partial tiles: at most this many doubles (the split is used only when the tiles are
// fewer than the SMs, so nz M N stays within a few SMs' worth of 128 x 64 tiles)
constexpr size_t kPartElems = (size_t)320 * 128 * 128;

size_t tc_gemm_work_bytes(int M, int N, int K) {
  const size_t kp = (size_t)kpad_of(K > 0 ? K : 1);
  return 256 + align256((size_t)S * M * kp * 2) + align256((size_t)S * N * kp * 2) + align256((size_t)M * 4) +
         align256((size_t)N * 4) + align256((size_t)M * 8) + align256((size_t)N * 8) + align256(kPartElems * 8);
}

cudaError_t tc_prepare() {
  cudaError_t e = encode_fn();
  if (e != cudaSuccess) return e;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm_cls_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CSMEM);
  });
  return attr_err;
}

namespace {

cudaError_t gemm_f64_tc_one(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                            int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                            void* work, int* err, int flags, int64_t* launches, const int32_t* done,
                            const TcSlices* cA = nullptr, const TcSlices* cB = nullptr);

}  // namespace

size_t tc_slices_bytes(int R, int K) {
  const size_t kp = (size_t)kpad_of(K > 0 ? K : 1);
  return align256((size_t)S * R * kp * 2) + align256((size_t)R * 4) + align256((size_t)R * 8);
}

// The slices of op(X) (R rows of K entries, X(r, k) = X[r rs + k ks]) made once into `mem`
// (tc_slices_bytes(R, K) bytes, 256-byte aligned), for products that reuse the operand.
cudaError_t tc_make_slices(cudaStream_t st, int R, int K, const double* X, int64_t rs, int64_t ks, void* mem,
                           TcSlices* out, int64_t* launches) {
  if (R < 1 || K < 1 || !X || !mem || !out) return cudaErrorInvalidValue;
  const int Kp = kpad_of(K);
  char* w = static_cast<char*>(mem);
  __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)S * R * Kp * 2);
  int* ex = reinterpret_cast<int*>(w);
  w += align256((size_t)R * 4);
  unsigned long long* rm = reinterpret_cast<unsigned long long*>(w);
  cudaError_t e = cudaMemsetAsync(rm, 0, (size_t)R * 8, st);
  if (e != cudaSuccess) return e;
  const unsigned kb = (unsigned)((K + 255) / 256), kp64 = (unsigned)(Kp / BK);
  rowmax_kernel<<<dim3((R + 31) / 32, kb), 256, 0, st>>>(R, K, X, rs, ks, rm, nullptr);
  slice_kernel<<<dim3((R + 31) / 32, kp64), 256, 0, st>>>(R, K, Kp, X, rs, ks, rm, sl, ex, nullptr);
  if (launches) *launches += 2;
  out->s = sl;
  out->e = ex;
  out->rows = R;
  out->K = K;
  out->valid = true;
  return cudaGetLastError();
}

// K is processed in host chunks small enough for `work` (each chunk's FP64 result is added to C).
cudaError_t gemm_f64_tc(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work,
                        size_t work_bytes, int* err, int flags, int64_t* launches, const int32_t* done,
                        const TcSlices* cA, const TcSlices* cB) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 0 || !work || !err) return cudaErrorInvalidValue;
  // slices made earlier serve only a product over their whole K in one piece
  if (cA && !(cA->valid && cA->rows == M && cA->K == K)) cA = nullptr;
  if (cB && !(cB->valid && cB->rows == N && cB->K == K)) cB = nullptr;
  if (work_bytes >= tc_gemm_work_bytes(M, N, K))
    return gemm_f64_tc_one(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work, err, flags, launches,
                           done, cA, cB);
  const size_t per_k = (size_t)S * (M + N) * 2;           // slice bytes per unit of K
  const size_t fixed = 256 + align256((size_t)M * 4) + align256((size_t)N * 4) + align256((size_t)M * 8) +
                       align256((size_t)N * 8) + align256(kPartElems * 8) + 512;
  if (work_bytes <= fixed + per_k * BK) return cudaErrorInvalidValue;
  int64_t kc64 = (int64_t)((work_bytes - fixed) / per_k) / BK * BK;
  int kc = (int)std::min<int64_t>(kc64, K);
  if (kc >= KC) kc = kc / KC * KC;                          // whole exact chunks where possible
  while (kc >= BK && tc_gemm_work_bytes(M, N, kc) > work_bytes) kc -= BK;
  if (kc < BK) return cudaErrorInvalidValue;
  for (int k0 = 0; k0 < K; k0 += kc) {
    const int kk = std::min(kc, K - k0);
    const double* Ak = A + (tA ? (int64_t)k0 : (int64_t)k0 * lda);
    const double* Bk = B + (tB ? (int64_t)k0 * ldb : (int64_t)k0);
    cudaError_t e = gemm_f64_tc_one(st, tA, tB, M, N, kk, alpha, Ak, lda, Bk, ldb, k0 == 0 ? beta : 1.0, C, ldc, work,
                                    err, flags, launches, done);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {

cudaError_t gemm_f64_tc_one(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                            int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                            void* work, int* err, int flags, int64_t* launches, const int32_t* done,
                            const TcSlices* cA, const TcSlices* cB) {
  cudaError_t e = tc_prepare();
  if (e != cudaSuccess) return e;
  const int Kp = kpad_of(K > 0 ? K : 1);
  char* w = static_cast<char*>(work) + 256;
  __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)S * M * Kp * 2);
  __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)S * N * Kp * 2);
  int* ea = reinterpret_cast<int*>(w);
  w += align256((size_t)M * 4);
  int* eb = reinterpret_cast<int*>(w);
  w += align256((size_t)N * 4);
  unsigned long long* rmA = reinterpret_cast<unsigned long long*>(w);
  w += align256((size_t)M * 8);
  unsigned long long* rmB = reinterpret_cast<unsigned long long*>(w);
  w += align256((size_t)N * 8);
  double* part = reinterpret_cast<double*>(w);
  // row i of op(A): A[i + k lda] (or A[k + i lda] transposed); row j of op(B)^T: B[k + j ldb]
  // (or B[j + k ldb] transposed)
  e = cudaMemsetAsync(rmA, 0, (size_t)M * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(rmB, 0, (size_t)N * 8, st);
  if (e != cudaSuccess) return e;
  const int64_t ars = tA ? lda : 1, aks = tA ? 1 : lda, brs = tB ? 1 : ldb, bks = tB ? ldb : 1;
  const unsigned kb = (unsigned)((std::max(K, 1) + 255) / 256), kp64 = (unsigned)(Kp / BK);
  // op(A) = op(B)^T (C = X^T X or X X^T): one operand, sliced once; operands sliced earlier
  // (cA, cB) are used as they are
  const bool same = (A == B && M == N && ars == brs && aks == bks);
  if (cA) {
    sa = static_cast<__nv_bfloat16*>(cA->s);
    ea = cA->e;
  } else {
    rowmax_kernel<<<dim3((M + 31) / 32, kb), 256, 0, st>>>(M, K, A, ars, aks, rmA, done);
    slice_kernel<<<dim3((M + 31) / 32, kp64), 256, 0, st>>>(M, K, Kp, A, ars, aks, rmA, sa, ea, done);
    if (launches) *launches += 2;
  }
  if (cB) {
    sb = static_cast<__nv_bfloat16*>(cB->s);
    eb = cB->e;
  } else if (same) {
    sb = sa;
    eb = ea;
  } else {
    rowmax_kernel<<<dim3((N + 31) / 32, kb), 256, 0, st>>>(N, K, B, brs, bks, rmB, done);
    slice_kernel<<<dim3((N + 31) / 32, kp64), 256, 0, st>>>(N, K, Kp, B, brs, bks, rmB, sb, eb, done);
    if (launches) *launches += 2;
  }
  CUtensorMap mapA, mapB;
  e = make_map(&mapA, sa, M, Kp, CBM);
  if (e == cudaSuccess) e = make_map(&mapB, sb, N, Kp, CBN);
  if (e != cudaSuccess) return e;
  const int gm = (M + CBM - 1) / CBM, gn = (N + CBN - 1) / CBN;
  int tiles = gm * gn;
  if (flags & GEMM_LOWER) tiles = (tiles + gm) / 2;
  // split K when the tiles leave SMs idle: about one CTA per SM, K ranges of >= 256
  int nz = 1;
  if (tiles < g_num_sms && K >= 2 * 256) {
    nz = std::min((g_num_sms + tiles - 1) / tiles, K / 256);
    while (nz > 1 && (size_t)nz * M * N > kPartElems) --nz;
  }
  int ksplit = K > 0 ? ((K + nz - 1) / nz + BK - 1) / BK * BK : 0;
  if (ksplit > 0) nz = (K + ksplit - 1) / ksplit;
  else nz = 1;
  dim3 grid(gm, gn, nz);
  tc_gemm_cls_kernel<<<grid, CTHREADS, CSMEM, st>>>(mapA, mapB, M, N, K, ksplit, ea, eb, alpha, beta, C, ldc,
                                                    nz > 1 ? part : nullptr, (flags & GEMM_LOWER) ? 1 : 0, err, done,
                                                    g_main_wait_ns.load());
  if (launches) ++*launches;
  if (nz > 1) {
    const int64_t tot = (int64_t)M * N;
    tc_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, nz, part, alpha, beta, C, ldc,
                                                                    (flags & GEMM_LOWER) ? 1 : 0, done, err);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace

}  // namespace wc

extern "C" size_t sdp_gemm_f64_tc_work_bytes(int32_t M, int32_t N, int32_t K) {
  if (M < 0 || N < 0 || K < 0) return 0;
  return wc::tc_gemm_work_bytes(M, N, K);
}

extern "C" sdp_status sdp_gemm_f64_tc(void* stream, int32_t tA, int32_t tB, int32_t M, int32_t N, int32_t K,
                                      double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                                      double beta, double* C, int64_t ldc, void* work, size_t work_bytes) {
  using namespace wc;
  if (M < 0 || N < 0 || K < 0) return wc_fail(nullptr, SDP_EINVAL, "negative size");
  if (M == 0 || N == 0) return SDP_OK;
  if (!C || !work || (K > 0 && (!A || !B))) return wc_fail(nullptr, SDP_EINVAL, "NULL array argument");
  if (ldc < M || lda < (tA ? K : M) || ldb < (tB ? N : K) || lda < 1 || ldb < 1)
    return wc_fail(nullptr, SDP_EINVAL, "leading dimension too small");
  if (work_bytes < tc_gemm_work_bytes(M, N, K)) return wc_fail(nullptr, SDP_EINVAL, "work too small");
  if ((reinterpret_cast<uintptr_t>(work) & 255u) != 0) return wc_fail(nullptr, SDP_EINVAL, "work not 256-byte aligned");
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) !=
                                                  cudaSuccess)
    return wc_fail(nullptr, SDP_ECUDA, "no CUDA device");
  if (major != 10) return wc_fail(nullptr, SDP_EUNSUPPORTED, "tcgen05 products need a Blackwell (sm_10x) device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = static_cast<int*>(work);
  if (cudaMemsetAsync(work, 0, 256, st) != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, "clearing the error word");
  cudaError_t e = gemm_f64_tc(st, tA != 0, tB != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work, work_bytes,
                              err, 0, nullptr, nullptr);
  if (e != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, std::string("tensor-core product: ") + cudaGetErrorString(e));
  int h_err = 0;
  e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, std::string("tensor-core product: ") + cudaGetErrorString(e));
  if (h_err) return wc_fail(nullptr, SDP_ETIMEOUT, "a bounded wait of the tensor-core product gave up");
  return SDP_OK;
}

namespace wc {
extern std::atomic<unsigned long long> g_main_wait_ns_lp;   // lp_gemm.cu
}

extern "C" void sdp_set_tc_wait_limit_ns(uint64_t ns) {
  const unsigned long long v = ns == 0 ? wc::WAIT_NS : (unsigned long long)ns;
  wc::g_main_wait_ns.store(v);
  wc::g_main_wait_ns_lp.store(v);
}

// Exact fixed-point digits of FP64 values, for products summed in integers (rows.cu: the passes
// over the dense constraint rows; gemm_fx.cu: the small dense products of the FP64 operator).
//
// A value x with |x| 2^adj < 2^F becomes N = rint(x 2^(52 + adj - F)) (|N| <= 2^52), computed by
// integer shifts of its IEEE fields, and N = hi 2^26 + lo with |hi| <= 2^26, -2^25 <= lo < 2^25.
// For two such values, x y 2^(104 - F - G) = hi hi' 2^52 + (hi lo' + lo hi') 2^26 + lo lo'; the
// first two parts are summed exactly in int64 (each product below 2^52, at most FX_FLUSH terms
// per accumulator), the third (below 2^50 per term, weight 2^-104) is dropped.
#pragma once

#include <climits>

namespace wc {

constexpr int FX_FLUSH = 1024;
constexpr int FX_BAD = 0x7fffffff;          // the vector had a non-finite entry: outputs are NaN
constexpr int FX_NONE = INT_MIN;            // no nonzero entry
constexpr int FX_NONE_MAX = -8192;          // any exponent at or below this also means "no nonzero entry"
                                            // (a 4-byte memset to 0x80 gives one)

__device__ __forceinline__ bool fx_none(int f) { return f <= FX_NONE_MAX; }

// e with |x| < 2^e from the IEEE fields (x finite and nonzero)
__device__ __forceinline__ int fx_expo_bits(unsigned long long b) {
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex) return ex - 1022;
  const unsigned long long mnt = b & 0xFFFFFFFFFFFFFull;   // subnormal: mnt 2^-1074
  return (63 - __clzll((long long)mnt)) - 1073;
}

// N = rint(x 2^(52 + adj - F)) by integer shifts of the IEEE fields, for |x| 2^adj < 2^F
// (so |N| <= 2^52); halves round away from zero
__device__ __forceinline__ long long fx_fixed(double x, int adj, int F) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long mnt = b & 0xFFFFFFFFFFFFFull;
  if (ex) mnt |= 1ull << 52;
  if (mnt == 0ull) return 0;
  const int sh = (ex ? ex : 1) - 1023 + adj - F;          // x 2^(52+adj-F) = mnt 2^sh
  long long N;
  if (sh >= 0) N = sh < 64 ? (long long)(mnt << sh) : 0;      // sh >= 0 only for subnormal x
  else if (sh <= -64) N = 0;
  else N = (long long)((mnt + (1ull << (-sh - 1))) >> (-sh));
  return (b >> 63) ? -N : N;
}

__device__ __forceinline__ int2 fx_split(long long N) {   // |N| <= 2^52
  const long long hi = (N + (1ll << 25)) >> 26;
  return make_int2((int)hi, (int)(N - (hi << 26)));
}

__device__ __forceinline__ double fx_value(long long t1, long long t2) {
  return fma((double)t1, 0x1p-52, (double)t2 * 0x1p-78);
}


}  // namespace wc

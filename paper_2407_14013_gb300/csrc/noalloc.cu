// sdp_adjoint_dense_noalloc: Y = A^T(y) = sum_i y_i A_i for dense svec rows, with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs where an allocation may not happen
// (inside a custom allocator or a memory-pool callback, in a process whose device memory
// is fully reserved up front by another framework, or on a path that must never fail with
// an out-of-memory error once it has started).  They still provide the input and output
// arrays; this entry point takes the only scratch it needs, the per-row-group partial sums
// of A^T(y), from a fixed array in the library's own device data.
//
// The array below is part of the module image: every GPU that loads the library holds its
// 4 MiB until the process exits.  Host code cannot use the symbol as a pointer (on the
// host it names a stand-in, not device memory), so every call looks up its device address
// with cudaGetSymbolAddress for the device current at the call (a lookup, no allocation).
// Looking it up per call, rather than caching it, keeps the address right when the device's
// context is torn down and made again between calls (cudaDeviceReset), which reloads the
// module at a new address.  The first call on a device loads the module, so it should come
// before any stream capture.  All calls share the array: calls that overlap on the GPU
// (different streams, or host threads) race on it.  Every partial sum the second kernel
// reads is written by the first kernel of the same call, so nothing has to be cleared
// between calls.
#include <cuda_runtime.h>

#include "../../include/wcipm.h"
#include "common.cuh"

namespace {

constexpr int64_t kScratchDoubles = 524288;          // 4 MiB of partial sums
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// partial[g * N + k] = sum_{i in group g} y_i a[i, k]
__global__ void __launch_bounds__(kThreads)
noalloc_partials_kernel(const double* __restrict__ a, int m, int64_t N, const double* __restrict__ y,
                        int rows_per_group, double* __restrict__ part) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= N) return;
  const int g = blockIdx.y;
  const int i0 = g * rows_per_group;
  const int i1 = min(m, i0 + rows_per_group);
  double acc = 0.0;
  for (int i = i0; i < i1; ++i) acc = fma(__ldg(y + i), __ldg(a + (int64_t)i * N + k), acc);
  part[(int64_t)g * N + k] = acc;
}

// Y (n x n, full) = smat(sum_g partial[g, :])
__global__ void noalloc_unpack_kernel(int n, int64_t N, int groups, const double* __restrict__ part,
                                      double* __restrict__ Y) {
  const int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int r = (int)(q % n), c = (int)(q / n);
  const int i = r > c ? r : c, j = r > c ? c : r;
  const int64_t idx = wc::svec_index(n, i, j);
  double s = 0.0;
  for (int g = 0; g < groups; ++g) s += part[(int64_t)g * N + idx];
  Y[q] = (r == c) ? s : s * WC_RSQRT2;
}

// The status code is the whole error report of this entry point (it has no handle to hold
// a message); the cases are listed with its declaration in wcipm.h.
sdp_status fail(sdp_status s, const char*) { return s; }

}  // namespace

extern "C" sdp_status sdp_adjoint_dense_noalloc(const double* a_dense, int32_t n, int32_t m, const double* y,
                                                double* Y, void* stream) {
  if (!a_dense || !y || !Y) return fail(SDP_EINVAL, "NULL array argument");
  if (n < 1 || m < 1) return fail(SDP_EINVAL, "need n >= 1 and m >= 1");
  const int64_t N = (int64_t)n * (n + 1) / 2;
  if (N > kScratchDoubles)
    return fail(SDP_EINVAL, "n too large for the fixed scratch: n(n+1)/2 must be <= 524288 (n <= 1023)");
  // the device address of the array in the current device's context
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return fail(SDP_ECUDA, "cudaGetSymbolAddress failed");
  double* scratch = static_cast<double*>(p);
  // as many row groups as the scratch holds (at most 16), each a contiguous block of rows
  int groups = (int)(kScratchDoubles / N);
  if (groups > 16) groups = 16;
  if (groups > m) groups = m;
  const int rpg = (m + groups - 1) / groups;
  groups = (m + rpg - 1) / rpg;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)((N + kThreads - 1) / kThreads), groups);
  noalloc_partials_kernel<<<grid, kThreads, 0, st>>>(a_dense, m, N, y, rpg, scratch);
  const int64_t nn = (int64_t)n * n;
  noalloc_unpack_kernel<<<(unsigned)((nn + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, N, groups, scratch, Y);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SDP_ECUDA, "kernel launch failed");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SDP_ECUDA, "stream synchronisation failed");
  return SDP_OK;
}

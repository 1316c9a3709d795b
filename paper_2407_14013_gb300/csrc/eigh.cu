// Symmetric eigen-decomposition A = V diag(lam) V^T in FP64 by the parallel cyclic Jacobi
// method (two-sided rotations, round-robin pairing of the indices).
//
// The outer interior-point loop needs eigen-decompositions of n x n scaling matrices (the NT
// scaling point W of eq. newt and its eigenpairs for the split of eq. EQSigdef, and minimum
// eigenvalues for step lengths).  Jacobi suits the GPU: one step applies n/2 disjoint plane
// rotations, all of which are independent, so a step is two kernels over O(n^2) entries; a
// sweep is n - 1 steps (every pair of indices meets once), and sweeps repeat until the
// off-diagonal mass ||A - diag A||_F falls below tol ||A||_F.  Convergence is quadratic, and
// the method is accurate in the relative sense on graded matrices, which the scaling points
// near the end of the interior-point path are.
//
// Step k pairs the indices by the circle method: position 0 is fixed, the others rotate by
// k, position P meets position npad - 1 - P (npad = n rounded up to even; the extra index
// is a dummy that no rotation touches).  The rotation (c, s) of a pair p < q makes the 2 x 2
// block [[a_pp, a_pq], [a_pq, a_qq]] diagonal: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c, and the update
// is A <- R^T A R, V <- V R with R = [[c, s], [-s, c]] on the rows / columns (p, q).
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int ET = 256;

__device__ __forceinline__ void pair_of(int k, int P, int npad, int& p, int& q) {
  const int a = (P == 0) ? 0 : ((P - 1 + k) % (npad - 1)) + 1;
  const int Pb = npad - 1 - P;
  const int b = (Pb == 0) ? 0 : ((Pb - 1 + k) % (npad - 1)) + 1;
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// rotation parameters of step k for every pair
__global__ void jacobi_params_kernel(int n, int npad, int k, const double* __restrict__ A, int2* __restrict__ pq,
                                     double2* __restrict__ cs) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= npad / 2) return;
  int p, q;
  pair_of(k, P, npad, p, q);
  double c = 1.0, s = 0.0;
  if (q < n) {
    const double apq = A[p + (int64_t)q * n];
    if (apq != 0.0) {
      const double tau = (A[q + (int64_t)q * n] - A[p + (int64_t)p * n]) / (2.0 * apq);
      double t;
      if (fabs(tau) > 1e100) t = 0.5 / tau;
      else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + t * t);
      s = t * c;
    }
  }
  pq[P] = make_int2(p, q);
  cs[P] = make_double2(c, s);
}

// A <- R^T A R on every block (I, J), I <= J, of the pairing (the (J, I) block is written as
// the transpose, so A stays exactly symmetric), and V <- V R.
__global__ void jacobi_apply_kernel(int n, int np, const int2* __restrict__ pq, const double2* __restrict__ cs,
                                    double* __restrict__ A, double* __restrict__ V) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nblk = (int64_t)np * np;
  if (t < nblk) {
    // t -> (I, J) on the full np x np grid; the blocks with I > J are written by (J, I)
    const int I = (int)(t % np), J = (int)(t / np);
    if (I > J) return;
    const int2 a = pq[I], b = pq[J];
    const double2 ra = cs[I], rb = cs[J];
    const int ri[2] = {a.x, a.y}, cj[2] = {b.x, b.y};
    double X[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v)
        X[u][v] = (ri[u] < n && cj[v] < n) ? A[ri[u] + (int64_t)cj[v] * n] : 0.0;
    // T = R_I^T X, Y = T R_J
    double T[2][2], Y[2][2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      T[0][v] = ra.x * X[0][v] - ra.y * X[1][v];
      T[1][v] = ra.y * X[0][v] + ra.x * X[1][v];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      Y[u][0] = rb.x * T[u][0] - rb.y * T[u][1];
      Y[u][1] = rb.y * T[u][0] + rb.x * T[u][1];
    }
    if (I == J) {
      Y[0][1] = 0.0;
      Y[1][0] = 0.0;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (ri[u] >= n || cj[v] >= n) continue;
        A[ri[u] + (int64_t)cj[v] * n] = Y[u][v];
        if (I != J) A[cj[v] + (int64_t)ri[u] * n] = Y[u][v];
      }
    return;
  }
  const int64_t tv = t - nblk;
  if (tv >= (int64_t)n * np) return;
  const int i = (int)(tv % n), J = (int)(tv / n);
  const int2 b = pq[J];
  if (b.y >= n) return;
  const double2 r = cs[J];
  const double vp = V[i + (int64_t)b.x * n], vq = V[i + (int64_t)b.y * n];
  V[i + (int64_t)b.x * n] = r.x * vp - r.y * vq;
  V[i + (int64_t)b.y * n] = r.y * vp + r.x * vq;
}

// sums of squares: [off-diagonal, all] of A into out (last block adds the block partials)
__global__ void jacobi_norms_kernel(int n, const double* __restrict__ A, double* __restrict__ part,
                                    unsigned int* __restrict__ counter, double* __restrict__ out) {
  __shared__ double sh[32];
  __shared__ bool last;
  double off = 0.0, all = 0.0;
  const int64_t nn = (int64_t)n * n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
    const double v = A[q];
    const int i = (int)(q % n), j = (int)(q / n);
    all = fma(v, v, all);
    if (i != j) off = fma(v, v, off);
  }
  off = block_sum(off, sh);
  all = block_sum(all, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = off;
    part[2 * blockIdx.x + 1] = all;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  double so = 0.0, sa = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    so += __ldcg(part + 2 * b);
    sa += __ldcg(part + 2 * b + 1);
  }
  so = block_sum(so, sh);
  sa = block_sum(sa, sh);
  if (threadIdx.x == 0) {
    out[0] = so;
    out[1] = sa;
    *counter = 0u;
  }
}

__global__ void identity_kernel(int n, double* __restrict__ V) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (int64_t)n * n) V[q] = ((q % n) == (q / n)) ? 1.0 : 0.0;
}

__global__ void diag_kernel(int n, const double* __restrict__ A, double* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lam[i] = A[i + (int64_t)i * n];
}

inline unsigned nb(int64_t total) { return (unsigned)((total + ET - 1) / ET); }

constexpr int kNormBlocks = 64;

}  // namespace

size_t eigh_work_elems(int n) {
  const int np = (n + 1) / 2;
  // pq (int2 = 1 double each), cs (2 doubles each), norm partials, result, counter
  return (size_t)np * 3 + 2 * kNormBlocks + 2 + 2 + 16;
}

void eigh_graph_release(EighGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->cap) cudaStreamDestroy(g->cap);
  g->exec = nullptr;
  g->cap = nullptr;
  g->n = 0;
}

cudaError_t eigh_jacobi(cudaStream_t st, int n, double* A, double* V, double* lam, double tol, int max_sweeps,
                        double* work, size_t work_elems, int* sweeps_out, double* off_out, int64_t* launches,
                        EighGraph* graph) {
  if (n < 1 || work_elems < eigh_work_elems(n)) return cudaErrorInvalidValue;
  const int npad = n + (n & 1);
  const int np = npad / 2;
  int2* pq = reinterpret_cast<int2*>(work);
  double2* cs = reinterpret_cast<double2*>(work + ((np + 1) & ~1));          // 16-byte aligned
  double* part = work + ((np + 1) & ~1) + 2 * (size_t)np;
  double* res = part + 2 * kNormBlocks;
  unsigned int* counter = reinterpret_cast<unsigned int*>(res + 2);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  identity_kernel<<<nb((int64_t)n * n), ET, 0, st>>>(n, V);
  if (launches) ++*launches;
  double h[2] = {0.0, 0.0};
  int sweep = 0;
  const int64_t apply_threads = (int64_t)np * np + (int64_t)n * np;
  auto sweep_kernels = [&](cudaStream_t s_) {
    for (int k = 0; k < npad - 1; ++k) {
      jacobi_params_kernel<<<nb(np), ET, 0, s_>>>(n, npad, k, A, pq, cs);
      jacobi_apply_kernel<<<nb(apply_threads), ET, 0, s_>>>(n, np, pq, cs, A, V);
    }
  };
  // one sweep (2 (npad - 1) kernels) as a CUDA graph, captured once per (n, A, V, work)
  if (graph && !(graph->exec && graph->n == n && graph->A == A && graph->V == V && graph->work == work)) {
    if (graph->exec) {
      cudaGraphExecDestroy(graph->exec);
      graph->exec = nullptr;
    }
    if (!graph->cap) {
      e = cudaStreamCreateWithFlags(&graph->cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    e = cudaStreamBeginCapture(graph->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    sweep_kernels(graph->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(graph->cap, &g);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&graph->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    graph->n = n;
    graph->A = A;
    graph->V = V;
    graph->work = work;
  }
  for (;; ++sweep) {
    jacobi_norms_kernel<<<kNormBlocks, ET, 0, st>>>(n, A, part, counter, res);
    if (launches) ++*launches;
    e = cudaMemcpyAsync(h, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (!(h[0] > tol * tol * h[1]) || sweep >= max_sweeps) break;
    if (graph) {
      e = cudaGraphLaunch(graph->exec, st);
      if (e != cudaSuccess) return e;
    } else {
      sweep_kernels(st);
    }
    if (launches) *launches += 2 * (npad - 1);
  }
  diag_kernel<<<nb(n), ET, 0, st>>>(n, A, lam);
  if (launches) ++*launches;
  if (sweeps_out) *sweeps_out = sweep;
  if (off_out) *off_out = (h[1] > 0.0) ? sqrt(h[0] / h[1]) : 0.0;
  return cudaGetLastError();
}

}  // namespace wc

// Symmetric eigen-decomposition A = V diag(lam) V^T in FP64 by the parallel cyclic Jacobi
// method (two-sided rotations, round-robin pairing of the indices).
//
// The outer interior-point loop needs eigen-decompositions of n x n scaling matrices (the NT
// scaling point W of eq. newt and its eigenpairs for the split of eq. EQSigdef, and minimum
// eigenvalues for step lengths).  Jacobi suits the GPU: one step applies n/2 disjoint plane
// rotations, all of which are independent, so a step is two kernels over O(n^2) entries; a
// sweep is n - 1 steps (every pair of indices meets once), and sweeps repeat until the
// off-diagonal mass ||A - diag A||_F falls below tol ||A||_F.  Convergence is quadratic.  The
// scaling points near the end of the interior-point path are graded in their spectrum but not
// in their entries (their eigenbasis is a general rotation), so the result is accurate to
// about eps ||A|| in absolute terms plus what the stop leaves: tol ||A||_F, which a stop at
// 1e-14 leaves up to about 100 eps ||A||.
//
// Step k pairs the indices by the circle method: position 0 is fixed, the others rotate by
// k, position P meets position npad - 1 - P (npad = n rounded up to even; the extra index
// is a dummy that no rotation touches).  The rotation (c, s) of a pair p < q makes the 2 x 2
// block [[a_pp, a_pq], [a_pq, a_qq]] diagonal: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c, and the update
// is A <- R^T A R, V <- V R with R = [[c, s], [-s, c]] on the rows / columns (p, q).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

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
constexpr int TI = 16;   // pairs per A tile side
constexpr int TR = 32;   // rows per V tile
constexpr int TV = 8;    // pairs per V tile

__device__ __forceinline__ double2 rotation(int n, int p, int q, const double* __restrict__ A) {
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
  return make_double2(c, s);
}

// The whole Jacobi iteration in one cooperative launch: every step reads A from one buffer and
// writes the rotated matrix to the other (so each block can compute the rotations it needs
// from the old matrix without waiting for anyone), then one grid-wide barrier; the stopping
// test after each sweep is evaluated identically by every block.  Replaces 2 (n - 1) launches
// per sweep and the host read per sweep of the graph path.
__global__ void __launch_bounds__(ET)
jacobi_coop_kernel(int n, int npad, double* __restrict__ A0, double* __restrict__ A1, double* __restrict__ V,
                   double* __restrict__ lam, double tol2, int max_sweeps, double* __restrict__ red,
                   int* __restrict__ sweeps_out, double* __restrict__ off_out) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double2 cs_s[2 * TI];
  __shared__ int2 pq_s[2 * TI];
  __shared__ double sh[32];
  const int np = npad / 2;
  const int nT = (np + TI - 1) / TI;
  const int nA = nT * (nT + 1) / 2;                          // A tiles (ti <= tj)
  const int nRT = (n + TR - 1) / TR, nV = nRT * ((np + TV - 1) / TV);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  const int64_t nn = (int64_t)n * n;
  for (int64_t q = gtid; q < nn; q += gsz) V[q] = ((q % n) == (q / n)) ? 1.0 : 0.0;
  double* Ain = A0;
  double* Aout = A1;
  int sweep = 0;
  double so = 0.0, sa = 0.0;
  for (;; ++sweep) {
    double o = 0.0, a = 0.0;
    for (int64_t q = gtid; q < nn; q += gsz) {
      const double v = Ain[q];
      a = fma(v, v, a);
      if ((q % n) != (q / n)) o = fma(v, v, o);
    }
    o = block_sum(o, sh);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) {
      red[2 * blockIdx.x] = o;
      red[2 * blockIdx.x + 1] = a;
    }
    grid.sync();
    so = 0.0;
    sa = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      so += red[2 * b];
      sa += red[2 * b + 1];
    }
    so = block_sum(so, sh);
    sa = block_sum(sa, sh);
    grid.sync();                               // every block has read red before it is reused
    if (!(so > tol2 * sa) || sweep >= max_sweeps) break;
    for (int k = 0; k < npad - 1; ++k) {
      // tiles: A blocks (TI pairs x TJ pairs, tile row <= tile column), then V (TR rows x TV pairs);
      // a block computes only the rotations its tile needs (FP64 arithmetic is the scarce unit)
      for (int tile = blockIdx.x; tile < nA + nV; tile += gridDim.x) {
        int I0 = 0, J0 = 0, R0 = 0, nI = 0, nJ = 0;
        if (tile < nA) {
          // tile = tj (tj + 1) / 2 + ti with ti <= tj
          int tj = 0;
          while ((tj + 1) * (tj + 2) / 2 <= tile) ++tj;
          const int ti = tile - tj * (tj + 1) / 2;
          I0 = ti * TI;
          J0 = tj * TI;
          nI = min(TI, np - I0);
          nJ = min(TI, np - J0);
        } else {
          const int tv = tile - nA;
          R0 = (tv % nRT) * TR;
          J0 = (tv / nRT) * TV;
          nJ = min(TV, np - J0);
        }
        // rotations of pairs I0 .. I0+nI-1 into slots [0, nI), of J0 .. into [TI, TI + nJ)
        for (int u = threadIdx.x; u < nI + nJ; u += blockDim.x) {
          const int P = (u < nI) ? I0 + u : J0 + (u - nI);
          const int slot = (u < nI) ? u : TI + (u - nI);   // J rotations at slots TI ..
          int p, q;
          pair_of(k, P, npad, p, q);
          pq_s[slot] = make_int2(p, q);
          cs_s[slot] = rotation(n, p, q, Ain);
        }
        __syncthreads();
        if (tile < nA) {
          for (int e = threadIdx.x; e < nI * nJ; e += blockDim.x) {
            const int iu = e % nI, ju = e / nI;
            const int I = I0 + iu, J = J0 + ju;
            if (I > J) continue;
            const int2 pa = pq_s[iu], pb = pq_s[TI + ju];
            const double2 ra = cs_s[iu], rb = cs_s[TI + ju];
            const int ri[2] = {pa.x, pa.y}, cj[2] = {pb.x, pb.y};
            double X[2][2], T[2][2], Y[2][2];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
              for (int v = 0; v < 2; ++v)
                X[u][v] = (ri[u] < n && cj[v] < n) ? Ain[ri[u] + (int64_t)cj[v] * n] : 0.0;
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
                Aout[ri[u] + (int64_t)cj[v] * n] = Y[u][v];
                Aout[cj[v] + (int64_t)ri[u] * n] = Y[u][v];
              }
          }
        } else {
          const int nR = min(TR, n - R0);
          for (int e = threadIdx.x; e < nR * nJ; e += blockDim.x) {
            const int i = R0 + e % nR, ju = e / nR;
            const int2 pb = pq_s[TI + ju];
            if (pb.y >= n) continue;
            const double2 r = cs_s[TI + ju];
            const double vp = V[i + (int64_t)pb.x * n], vq = V[i + (int64_t)pb.y * n];
            V[i + (int64_t)pb.x * n] = r.x * vp - r.y * vq;
            V[i + (int64_t)pb.y * n] = r.y * vp + r.x * vq;
          }
        }
        __syncthreads();
      }
      grid.sync();
      double* tmp = Ain;
      Ain = Aout;
      Aout = tmp;
    }
  }
  for (int64_t i = gtid; i < n; i += gsz) lam[i] = Ain[i + i * n];
  if (gtid == 0) {
    *sweeps_out = sweep;
    *off_out = (sa > 0.0) ? sqrt(so / sa) : 0.0;
  }
}

}  // namespace

constexpr int kCoopMaxBlocks = 1024;

size_t eigh_work_elems(int n) {
  const int np = (n + 1) / 2;
  // pq (int2 = 1 double each), cs (2 doubles each), norm partials, result, counter; the second
  // copy of A and the block partials of the cooperative path
  return (size_t)np * 3 + 2 * kNormBlocks + 2 + 2 + 16 + (size_t)n * n + 2 * kCoopMaxBlocks + 64;
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
                        EighGraph* graph, bool allow_coop) {
  if (n < 1 || work_elems < eigh_work_elems(n)) return cudaErrorInvalidValue;
  const int npad = n + (n & 1);
  const int np = npad / 2;
  if (allow_coop) {
    // cooperative path: one launch for the whole iteration
    double* A1 = work + ((size_t)np * 3 + 2 * kNormBlocks + 2 + 2 + 16 + 7) / 8 * 8;
    double* red = A1 + (size_t)n * n;
    int* out_i = reinterpret_cast<int*>(red + 2 * kCoopMaxBlocks);
    double* out_d = red + 2 * kCoopMaxBlocks + 2;
    int dev = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    const size_t smem = 0;
    if (coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel, ET, smem) == cudaSuccess &&
        per_sm > 0) {
      const int64_t nT = (np + TI - 1) / TI;
      const int64_t want = nT * (nT + 1) / 2 + ((n + TR - 1) / TR) * (int64_t)((np + TV - 1) / TV);
      int blocks = (int)std::min<int64_t>({want, (int64_t)per_sm * g_num_sms, (int64_t)kCoopMaxBlocks});
      if (blocks < 1) blocks = 1;
      double tol2 = tol * tol;
      void* args[] = {&n, (void*)&npad, &A, &A1, &V, &lam, &tol2, &max_sweeps, &red, &out_i, &out_d};
      cudaError_t e = cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel, dim3(blocks), dim3(ET), args,
                                                  smem, st);
      if (e == cudaSuccess) {
        if (launches) ++*launches;
        int sw = 0;
        double off = 0.0;
        e = cudaMemcpyAsync(&sw, out_i, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&off, out_d, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (sweeps_out) *sweeps_out = sw;
        if (off_out) *off_out = off;
        return cudaSuccess;
      }
      cudaGetLastError();   // not launchable cooperatively here: take the graph path
    }
  }
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

// ---- smallest eigenvalue by Lanczos -----------------------------------------------------------
//
// lambda_min(M) for a symmetric M (n x n): Lanczos on the Krylov space of a fixed start vector,
// with full re-orthogonalisation (classical Gram-Schmidt applied twice), run in chunks of
// iterations by one cooperative launch each; after each chunk the host finds the smallest
// eigenvalue of the tridiagonal T_k (bisection on Sturm counts).  It stops when that value moved by
// at most 1e-12 of its size over the last 8 steps, when the basis spans R^n (k = n, then T_n is
// similar to M), or on breakdown (beta_k = 0: an invariant subspace).  Ritz values of a
// symmetric matrix decrease monotonically to lambda_min as k grows, so the value returned is
// never below lambda_min; the step-length rule that uses it takes 0.98 of the bound and checks the
// shortened step by a Cholesky factorisation.

namespace wc {

namespace {

__global__ void __launch_bounds__(ET)
lanczos_coop_kernel(int n, const double* __restrict__ M, double* __restrict__ Vb, double* __restrict__ alpha,
                    double* __restrict__ beta, double* __restrict__ w, double* __restrict__ hbuf,
                    double* __restrict__ red, int k0, int k1) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  const int64_t gwarp = gtid >> 5, nwarps = gsz >> 5;
  auto grid_sum = [&](double v) -> double {   // identical result in every block
    v = block_sum(v, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = v;
    grid.sync();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += red[b];
    s = block_sum(s, sh);
    grid.sync();
    return s;
  };
  if (k0 == 0) {   // v_0 = fixed start vector, normalised
    double loc = 0.0;
    for (int64_t i = gtid; i < n; i += gsz) {
      const double v = 1.0 + 0.5 * sin(0.7 * (double)i + 0.3);
      Vb[i] = v;
      loc = fma(v, v, loc);
    }
    const double nrm = sqrt(grid_sum(loc));
    for (int64_t i = gtid; i < n; i += gsz) Vb[i] /= nrm;
    grid.sync();
  }
  for (int k = k0; k < k1; ++k) {
    const double* vk = Vb + (int64_t)k * n;
    // w = M v_k (M symmetric: row i = column i, contiguous), one warp per row
    for (int64_t i = gwarp; i < n; i += nwarps) {
      const double* col = M + i * n;
      double acc = 0.0;
      for (int j = lane; j < n; j += 32) acc = fma(col[j], vk[j], acc);
      acc = warp_sum(acc);
      if (lane == 0) w[i] = acc;
    }
    grid.sync();
    double loc = 0.0;
    for (int64_t i = gtid; i < n; i += gsz) loc = fma(vk[i], w[i], loc);
    const double a = grid_sum(loc);
    const double bprev = (k > 0) ? beta[k - 1] : 0.0;
    for (int64_t i = gtid; i < n; i += gsz) {
      double v = w[i] - a * vk[i];
      if (k > 0) v -= bprev * Vb[(int64_t)(k - 1) * n + i];
      w[i] = v;
    }
    if (gtid == 0) alpha[k] = a;
    grid.sync();
    // full re-orthogonalisation against v_0 .. v_k, twice
    for (int pass = 0; pass < 2; ++pass) {
      for (int64_t j = gwarp; j <= k; j += nwarps) {
        const double* vj = Vb + j * n;
        double acc = 0.0;
        for (int i = lane; i < n; i += 32) acc = fma(vj[i], w[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) hbuf[j] = acc;
      }
      grid.sync();
      for (int64_t i = gtid; i < n; i += gsz) {
        double v = w[i];
        for (int j = 0; j <= k; ++j) v = fma(-hbuf[j], Vb[(int64_t)j * n + i], v);
        w[i] = v;
      }
      grid.sync();
    }
    loc = 0.0;
    for (int64_t i = gtid; i < n; i += gsz) loc = fma(w[i], w[i], loc);
    const double b = sqrt(grid_sum(loc));
    if (gtid == 0) beta[k] = b;
    double* vn = Vb + (int64_t)(k + 1) * n;
    for (int64_t i = gtid; i < n; i += gsz) vn[i] = (b > 0.0) ? w[i] / b : 0.0;
    grid.sync();
  }
}

// number of eigenvalues of the tridiagonal (a, b) below x (Sturm sequence)
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    const double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

double tridiag_min(const std::vector<double>& a, const std::vector<double>& b, int k) {
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, k, mid) >= 1) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// The same Lanczos steps k0 .. k1 - 1 in ONE block (block barriers instead of grid barriers):
// for problems run side by side on their own streams, where no launch may wait for the whole
// GPU.  Same start vector, recurrence and re-orthogonalisation as the cooperative kernel.
constexpr int LT = 1024;
__global__ void __launch_bounds__(LT)
lanczos_block_kernel(int n, const double* __restrict__ M, double* __restrict__ Vb, double* __restrict__ alpha,
                     double* __restrict__ beta, double* __restrict__ w, double* __restrict__ hbuf, int k0, int k1) {
  __shared__ double sh[32];
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, wid = t >> 5, nw = T >> 5;
  if (k0 == 0) {
    double loc = 0.0;
    for (int i = t; i < n; i += T) {
      const double v = 1.0 + 0.5 * sin(0.7 * (double)i + 0.3);
      Vb[i] = v;
      loc = fma(v, v, loc);
    }
    const double nrm = sqrt(block_sum(loc, sh));
    for (int i = t; i < n; i += T) Vb[i] /= nrm;
    __syncthreads();
  }
  for (int k = k0; k < k1; ++k) {
    const double* vk = Vb + (int64_t)k * n;
    for (int i = wid; i < n; i += nw) {   // w = M v_k, one warp per row (M symmetric)
      const double* row = M + (int64_t)i * n;
      double acc = 0.0;
      for (int j = lane; j < n; j += 32) acc = fma(row[j], vk[j], acc);
      acc = warp_sum(acc);
      if (lane == 0) w[i] = acc;
    }
    __syncthreads();
    double loc = 0.0;
    for (int i = t; i < n; i += T) loc = fma(vk[i], w[i], loc);
    const double a = block_sum(loc, sh);
    const double bprev = (k > 0) ? beta[k - 1] : 0.0;
    for (int i = t; i < n; i += T) {
      double v = w[i] - a * vk[i];
      if (k > 0) v -= bprev * Vb[(int64_t)(k - 1) * n + i];
      w[i] = v;
    }
    if (t == 0) alpha[k] = a;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {   // full re-orthogonalisation against v_0 .. v_k, twice
      for (int j = wid; j <= k; j += nw) {
        const double* vj = Vb + (int64_t)j * n;
        double acc = 0.0;
        for (int i = lane; i < n; i += 32) acc = fma(vj[i], w[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) hbuf[j] = acc;
      }
      __syncthreads();
      for (int i = t; i < n; i += T) {
        double v = w[i];
        for (int j = 0; j <= k; ++j) v = fma(-hbuf[j], Vb[(int64_t)j * n + i], v);
        w[i] = v;
      }
      __syncthreads();
    }
    loc = 0.0;
    for (int i = t; i < n; i += T) loc = fma(w[i], w[i], loc);
    const double b = sqrt(block_sum(loc, sh));
    if (t == 0) beta[k] = b;
    double* vn = Vb + (int64_t)(k + 1) * n;
    for (int i = t; i < n; i += T) vn[i] = (b > 0.0) ? w[i] / b : 0.0;
    __syncthreads();
  }
}

}  // namespace

constexpr int kLanczosBlockMax = 128;

size_t lanczos_work_elems(int n) {
  const size_t K = (size_t)n + 1;
  return (size_t)n * (K + 1) + 3 * K + (size_t)n + 2 * kCoopMaxBlocks + 64;
}

cudaError_t lanczos_min(cudaStream_t st, int n, const double* M, double* work, size_t work_elems, double* lmin,
                        int* iters, int64_t* launches, bool allow_coop) {
  if (n < 1 || work_elems < lanczos_work_elems(n)) return cudaErrorInvalidValue;
  const int K = n;   // at most n vectors span R^n
  double* Vb = work;
  double* alpha = Vb + (size_t)n * (K + 2);
  double* beta = alpha + K + 1;
  double* hbuf = beta + K + 1;
  double* w = hbuf + K + 1;
  double* red = w + n;
  int dev = 0, coop = 0, per_sm = 0;
  cudaError_t e = cudaSuccess;
  // small n: one block per launch (block barriers) beats grid barriers across the GPU
  if (allow_coop && n > kLanczosBlockMax) {
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lanczos_coop_kernel, ET, 0);
      if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        coop = 0;
      }
    }
  }
  const int want = (int)std::max<int64_t>(1, ((int64_t)n * 32 + ET - 1) / ET);   // one warp per row
  const int blocks = coop ? std::min({want, per_sm * g_num_sms, kCoopMaxBlocks}) : 1;
  std::vector<double> ah(K + 1), bh(K + 1);
  double theta = 0.0;
  int k = 0;
  const int chunk = 16;
  while (k < K) {
    int k0 = k, k1 = std::min(K, k + chunk);
    if (coop) {
      void* args[] = {&n, (void*)&M, &Vb, &alpha, &beta, &w, &hbuf, &red, &k0, &k1};
      e = cudaLaunchCooperativeKernel((const void*)lanczos_coop_kernel, dim3(blocks), dim3(ET), args, 0, st);
    } else {
      lanczos_block_kernel<<<1, LT, 0, st>>>(n, M, Vb, alpha, beta, w, hbuf, k0, k1);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
    e = cudaMemcpyAsync(ah.data(), alpha, k1 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bh.data(), beta, k1 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    // breakdown: the Krylov space is invariant; T_j holds its eigenvalues
    int kk = k1;
    for (int j = k0; j < k1; ++j)
      if (!(bh[j] > 1e-300)) {
        kk = j + 1;
        break;
      }
    theta = tridiag_min(ah, bh, kk);
    k = k1;
    if (kk < k1) break;
    // converged when the smallest Ritz value (which decreases towards lambda_min) moved by at
    // most 1e-12 of its size over the last half chunk
    if (kk >= 24) {
      const double earlier = tridiag_min(ah, bh, kk - chunk / 2);
      if (std::fabs(theta - earlier) <= 1e-12 * std::max(std::fabs(theta), 1e-300)) break;
    }
  }
  *lmin = theta;
  if (iters) *iters = k;
  return cudaSuccess;
}

}  // namespace wc

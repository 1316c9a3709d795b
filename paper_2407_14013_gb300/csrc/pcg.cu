// Vector kernels of the indefinite PCG (Def. pcg with the coefficient
// beta_j = <r_{j+1}, z_{j+1}> / <r_j, z_j>, Cor. pcg) on the augmented system (eq. augsys),
// and the finishing steps of the operator, preconditioner, right-hand side and recovery.
//
// Vectors have length m + d: the u-block (m) followed by the v-block (d, h-coordinates).
// Scalars (alpha, beta, <r,z>, ||r||^2, tau, ...) live in the device control block, so a
// PCG iteration needs no host round trip; every kernel returns at once when ctl->done is set.
// Dot products are reduced deterministically: per-block partial sums, then the last block
// to finish (atomic ticket) adds them in block order.
#include "common.cuh"
#include "pcg.h"

namespace wc {

namespace {

constexpr int VT = 256;

__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return am_last;
}

__device__ __forceinline__ double sum_partials(const double* part, int nb, double* sh) {
  double s = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) s += __ldcg(part + q);   // L2: written by other blocks
  return block_sum(s, sh);
}

// out = [u_src; pack(H) - D p_v] (optionally g - that), and in mode 1 the dot <p, out> -> alpha.
__global__ void __launch_bounds__(VT)
ap_finish_kernel(int m, int d, int n, int r, const double* __restrict__ partA, int S,
                 const double* __restrict__ Up, const double* __restrict__ Vs,
                 const double* __restrict__ H, const double* __restrict__ Dv,
                 const double* __restrict__ p, const double* __restrict__ g, double* __restrict__ out,
                 int mode, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                 unsigned int* __restrict__ counter) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const int nt = m + d;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double v;
    if (q < m) {
      v = 0.0;
      for (int s = 0; s < S; ++s) v += partA[(int64_t)s * m + q];
      if (Up) {   // DIAG: A(sym(U Q^T)) = diag(U Q^T)
        for (int k = 0; k < r; ++k) v += Up[q + (int64_t)k * n] * Vs[q + (int64_t)k * n];
      }
    } else {
      const int h = q - m;
      v = pack_at(H, n, n, r, h) - Dv[h] * p[q];
    }
    if (g) v = g[q] - v;
    out[q] = v;
    if (mode == 1) acc = fma(p[q], v, acc);
  }
  if (mode != 1) return;
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    double pAp = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      ctl->pAp = pAp;
      // Def. pcg has no sign condition: with the indefinite preconditioner <p, A p> is positive
      // in exact arithmetic but may change sign at the rounding floor, which is harmless
      if (pAp == 0.0 || !isfinite(pAp) || !isfinite(ctl->rz)) {
        ctl->status = 5;
        ctl->done = 1;
      } else {
        ctl->alpha = ctl->rz / pAp;
      }
    }
  }
}

// x += alpha p; r -= alpha Ap; ||r||^2 -> stop test.
__global__ void __launch_bounds__(VT)
update_kernel(int nt, double* __restrict__ x, double* __restrict__ rv, const double* __restrict__ p,
              const double* __restrict__ Ap, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
              unsigned int* __restrict__ counter) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const double alpha = ctl->alpha;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    x[q] = fma(alpha, p[q], x[q]);
    double rr = fma(-alpha, Ap[q], rv[q]);
    rv[q] = rr;
    acc = fma(rr, rr, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    double rr = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      ctl->rr = rr;
      ctl->iters += 1;
      if (!isfinite(rr)) { ctl->status = 5; ctl->done = 1; }
      else if (rr <= ctl->tol2) { ctl->status = 0; ctl->done = 1; }
      else if (ctl->iters >= ctl->max_iters) { ctl->status = 4; ctl->done = 1; }
    }
  }
}

// d-space: s = r_v - beta^{-1} (B^T r_u)
__global__ void pc_d_s_kernel(int m, int d, int G, const double* __restrict__ partB, const double* __restrict__ rv,
                              double* __restrict__ s, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double t = 0.0;
  for (int gg = 0; gg < G; ++gg) t += partB[(int64_t)gg * d + h];
  s[h] = rv[m + h] - t / ctl->beta_pc;
}

// d-space: z_v = -(C^{-1} s)
__global__ void pc_d_zv_kernel(int m, int d, int S, const double* __restrict__ partC, double* __restrict__ z,
                               const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double t = 0.0;
  for (int s = 0; s < S; ++s) t += partC[(int64_t)s * d + h];
  z[m + h] = -t;
}

// z_u (d-space: beta^{-1}(r_u - B z_v); m-space: K^{-1} w) then <r, z> -> beta_pcg.
// mode 0 (start): rz = <r0, z0>;  mode 1 (iteration): beta = <r_{k+1}, z_{k+1}> / <r_k, z_k>.
__global__ void __launch_bounds__(VT)
pc_zu_dot_kernel(int m, int d, int S, const double* __restrict__ partU, int space,
                 const double* __restrict__ rv, double* __restrict__ z, int mode, PcgCtl* __restrict__ ctl,
                 double* __restrict__ dotbuf, unsigned int* __restrict__ counter) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const int nt = m + d;
  const double ib = 1.0 / ctl->beta_pc;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double zq;
    if (q < m && partU) {
      double t = 0.0;
      for (int s = 0; s < S; ++s) t += partU[(int64_t)s * m + q];
      zq = (space == 1) ? (rv[q] - t) * ib : t;
      z[q] = zq;
    } else {
      zq = z[q];
    }
    acc = fma(rv[q], zq, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    double rz = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      if (!isfinite(rz)) { ctl->status = 5; ctl->done = 1; }
      if (mode == 0) { ctl->rz = rz; ctl->beta = 0.0; }
      else { ctl->rz_new = rz; ctl->beta = rz / ctl->rz; ctl->rz = rz; }
    }
  }
}

// m-space helpers: t_v = r_v / D;  w = r_u + B t_v;  z_v = (B^T z_u - r_v) / D
__global__ void pc_m_tv_kernel(int m, int d, const double* __restrict__ rv, const double* __restrict__ Dv,
                               double* __restrict__ t, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  t[h] = rv[m + h] / Dv[h];
}

__global__ void pc_m_w_kernel(int m, int S, const double* __restrict__ partB, const double* __restrict__ rv,
                              double* __restrict__ w, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double t = 0.0;
  for (int s = 0; s < S; ++s) t += partB[(int64_t)s * m + i];
  w[i] = (rv ? rv[i] : 0.0) + t;
}

__global__ void pc_m_zv_kernel(int m, int d, int G, const double* __restrict__ partBt, const double* __restrict__ rv,
                               const double* __restrict__ Dv, double* __restrict__ z, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double t = 0.0;
  for (int gg = 0; gg < G; ++gg) t += partBt[(int64_t)gg * d + h];
  z[m + h] = (t - rv[m + h]) / Dv[h];
}

// p = z + beta p  (start: p = z)
__global__ void p_update_kernel(int nt, const double* __restrict__ z, double* __restrict__ p, int start,
                                const PcgCtl* __restrict__ ctl) {
  if (ctl->done && !start) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  p[q] = start ? z[q] : fma(ctl->beta, p[q], z[q]);
}

// Right side of eq. augsys: g = [b~ + tau^2 A(E C~ E); tau^2 pack(H)], x0 = [0; -g_v / D]
// (v0 = -Sigma^{-1} Q^T c of Cor. pcg), ||g||^2 and the stop threshold.
__global__ void __launch_bounds__(VT)
rhs_finish_kernel(int m, int d, int n, int r, const double* __restrict__ partA, int S,
                  const double* __restrict__ F, const double* __restrict__ E, const double* __restrict__ bt,
                  const double* __restrict__ Ct,
                  const double* __restrict__ H, const double* __restrict__ Dv, double* __restrict__ g,
                  double* __restrict__ x, double rtol, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                  unsigned int* __restrict__ counter) {
  __shared__ double sh[32];
  const int nt = m + d;
  const double tau = ctl->tau, t2 = tau * tau;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double v;
    if (q < m) {
      double a = 0.0;
      if (partA) {
        for (int s = 0; s < S; ++s) a += partA[(int64_t)s * m + q];
      } else {   // DIAG: diag(F E) with F = E C~
        for (int k = 0; k < n; ++k) a += F[q + (int64_t)k * n] * E[k + (int64_t)q * n];
      }
      v = bt[q] + t2 * a;
      x[q] = 0.0;
    } else {
      const int h = q - m;
      v = t2 * pack_at(H, n, n, r, h);
      x[q] = -v / Dv[h];
    }
    g[q] = v;
    acc = fma(v, v, acc);
  }
  // ||[svec C~; b~]||^2 = ||C~||_F^2 + ||b~||^2, the right side of (Newt-eps)
  double nrm = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * n + m;
       q += (int64_t)gridDim.x * blockDim.x) {
    double v = (q < (int64_t)n * n) ? Ct[q] : bt[q - (int64_t)n * n];
    nrm = fma(v, v, nrm);
  }
  acc = block_sum(acc, sh);
  nrm = block_sum(nrm, sh);
  if (threadIdx.x == 0) { dotbuf[blockIdx.x] = acc; dotbuf[512 + blockIdx.x] = nrm; }
  if (last_block(counter)) {
    double gg = sum_partials(dotbuf, gridDim.x, sh);
    double cb = sum_partials(dotbuf + 512, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      ctl->g_norm2 = gg;
      ctl->newt_rhs2 = cb;
      // stop when ||r_k|| <= rtol ||[svec C~; b~]||: with the second-block residual at rounding
      // level, ||r_k|| is the (Newt-eps) residual of the recovered direction (Lemma smallres)
      ctl->tol2 = rtol * rtol * cb;
      ctl->iters = 0;
      if (!isfinite(gg)) ctl->status = 5;
      ctl->done = (ctl->status != 0) ? 1 : 0;   // a non-positive pivot in the setup ends the solve
    }
  }
}

// ||r0||^2 and the stop test before the first iteration.
__global__ void __launch_bounds__(VT)
norm_check_kernel(int nt, const double* __restrict__ rv, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                  unsigned int* __restrict__ counter) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) acc = fma(rv[q], rv[q], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    double rr = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      ctl->rr = rr;
      ctl->rr0 = rr;
      if (!isfinite(rr)) { ctl->status = 5; ctl->done = 1; }
      else if (rr <= ctl->tol2) ctl->done = 1;
    }
  }
}

// T = diag(p_u) Q  (DIAG kind: A^T(p_u) Q)
__global__ void diag_scale_rows_kernel(int n, int r, const double* __restrict__ pu, const double* __restrict__ Vs,
                                       double* __restrict__ T, const int32_t* __restrict__ done) {
  if (done && *done) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * r) return;
  T[q] = pu[q % n] * Vs[q];
}

// Y = diag(u) (DIAG kind: A^T(u))
__global__ void diag_matrix_kernel(int n, const double* __restrict__ u, double* __restrict__ Y) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int a = (int)(q % n), b = (int)(q / n);
  Y[q] = (a == b) ? u[a] : 0.0;
}

// EE = E o E (Hadamard square; DIAG kind: diag(E diag(p) E) = (E o E) p)
__global__ void hadamard_sq_kernel(int64_t nn, const double* __restrict__ E, double* __restrict__ EE) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nn) return;
  EE[q] = E[q] * E[q];
}

// Recovery (eq. recover): Cw = Y_u - tau^2 C~ ;  dy = u / tau^2 ;  dS = C~ - Y_u / tau^2
__global__ void recover_pre_kernel(int n, int m, const double* __restrict__ Yu, const double* __restrict__ Ct,
                                   const double* __restrict__ u, double* __restrict__ Cw, double* __restrict__ dy,
                                   double* __restrict__ dS, const PcgCtl* __restrict__ ctl) {
  const double t2 = ctl->tau * ctl->tau;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (int64_t)n * n) {
    double y = Yu[q], c = Ct[q];
    Cw[q] = y - t2 * c;
    dS[q] = c - y / t2;
  }
  if (q < m) dy[q] = u[q] / t2;
}

// dX = sym(Z) + sym(U Q^T)
__global__ void sym_plus_full_kernel(int n, int r, const double* __restrict__ Z, const double* __restrict__ U,
                                     const double* __restrict__ Q, double* __restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int a = (int)(q % n), b = (int)(q / n);
  double v = 0.5 * (Z[a + (int64_t)b * n] + Z[b + (int64_t)a * n]);
  double t = 0.0;
  for (int k = 0; k < r; ++k)
    t += U[a + (int64_t)k * n] * Q[b + (int64_t)k * n] + Q[a + (int64_t)k * n] * U[b + (int64_t)k * n];
  out[q] = v + 0.5 * t;
}

// C += diag(Dv) * c_d + c_i * I  on an n x n matrix
__global__ void add_diag_kernel(int n, double* __restrict__ C, const double* __restrict__ Dv, double c_i) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  C[i + (int64_t)i * n] += (Dv ? Dv[i] : 0.0) + c_i;
}

// Bs (d x m, col-major view of B row-major) scaled rows: Bs[h, i] = B[i, h] / sqrt(D[h])
__global__ void scale_B_kernel(int m, int d, const double* __restrict__ B, const double* __restrict__ Dv,
                               double* __restrict__ Bs) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)m * d) return;
  int h = (int)(q % d);
  Bs[q] = B[q] / sqrt(Dv[h]);
}

inline unsigned nblk(int64_t total, int t) { return (unsigned)((total + t - 1) / t); }
inline int vec_blocks(int nt) {
  int b = (nt + VT - 1) / VT;
  return b > 256 ? 256 : b;
}

}  // namespace

void launch_ap_finish(cudaStream_t st, int m, int d, int n, int r, const double* partA, int S, const double* Up,
                      const double* Vs, const double* H, const double* Dv, const double* p, const double* g,
                      double* out, int mode, PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches) {
  ap_finish_kernel<<<vec_blocks(m + d), VT, 0, st>>>(m, d, n, r, partA, S, Up, Vs, H, Dv, p, g, out, mode, ctl,
                                                    dotbuf, counter);
  ++*launches;
}

void launch_update(cudaStream_t st, int nt, double* x, double* rv, const double* p, const double* Ap, PcgCtl* ctl,
                   double* dotbuf, unsigned int* counter, int64_t* launches) {
  update_kernel<<<vec_blocks(nt), VT, 0, st>>>(nt, x, rv, p, Ap, ctl, dotbuf, counter);
  ++*launches;
}

void launch_pc_d_s(cudaStream_t st, int m, int d, int G, const double* partB, const double* rv, double* s,
                   const PcgCtl* ctl, int64_t* launches) {
  pc_d_s_kernel<<<nblk(d, VT), VT, 0, st>>>(m, d, G, partB, rv, s, ctl);
  ++*launches;
}

void launch_pc_d_zv(cudaStream_t st, int m, int d, int S, const double* partC, double* z, const PcgCtl* ctl,
                    int64_t* launches) {
  pc_d_zv_kernel<<<nblk(d, VT), VT, 0, st>>>(m, d, S, partC, z, ctl);
  ++*launches;
}

void launch_pc_zu_dot(cudaStream_t st, int m, int d, int S, const double* partU, int space, const double* rv,
                      double* z, int mode, PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches) {
  pc_zu_dot_kernel<<<vec_blocks(m + d), VT, 0, st>>>(m, d, S, partU, space, rv, z, mode, ctl, dotbuf, counter);
  ++*launches;
}

void launch_pc_m_tv(cudaStream_t st, int m, int d, const double* rv, const double* Dv, double* t, const PcgCtl* ctl,
                    int64_t* launches) {
  pc_m_tv_kernel<<<nblk(d, VT), VT, 0, st>>>(m, d, rv, Dv, t, ctl);
  ++*launches;
}

void launch_pc_m_w(cudaStream_t st, int m, int S, const double* partB, const double* rv, double* w,
                   const PcgCtl* ctl, int64_t* launches) {
  pc_m_w_kernel<<<nblk(m, VT), VT, 0, st>>>(m, S, partB, rv, w, ctl);
  ++*launches;
}

void launch_pc_m_zv(cudaStream_t st, int m, int d, int G, const double* partBt, const double* rv, const double* Dv,
                    double* z, const PcgCtl* ctl, int64_t* launches) {
  pc_m_zv_kernel<<<nblk(d, VT), VT, 0, st>>>(m, d, G, partBt, rv, Dv, z, ctl);
  ++*launches;
}

void launch_p_update(cudaStream_t st, int nt, const double* z, double* p, int start, const PcgCtl* ctl,
                     int64_t* launches) {
  p_update_kernel<<<nblk(nt, VT), VT, 0, st>>>(nt, z, p, start, ctl);
  ++*launches;
}

void launch_rhs_finish(cudaStream_t st, int m, int d, int n, int r, const double* partA, int S, const double* F,
                       const double* E, const double* bt, const double* Ct, const double* H, const double* Dv,
                       double* g, double* x, double rtol, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                       int64_t* launches) {
  rhs_finish_kernel<<<vec_blocks(m + d), VT, 0, st>>>(m, d, n, r, partA, S, F, E, bt, Ct, H, Dv, g, x, rtol, ctl,
                                                     dotbuf, counter);
  ++*launches;
}

void launch_norm_check(cudaStream_t st, int nt, const double* rv, PcgCtl* ctl, double* dotbuf,
                       unsigned int* counter, int64_t* launches) {
  norm_check_kernel<<<vec_blocks(nt), VT, 0, st>>>(nt, rv, ctl, dotbuf, counter);
  ++*launches;
}

void launch_diag_scale_rows(cudaStream_t st, int n, int r, const double* pu, const double* Vs, double* T,
                            const int32_t* done, int64_t* launches) {
  diag_scale_rows_kernel<<<nblk((int64_t)n * r, VT), VT, 0, st>>>(n, r, pu, Vs, T, done);
  ++*launches;
}

void launch_diag_matrix(cudaStream_t st, int n, const double* u, double* Y, int64_t* launches) {
  diag_matrix_kernel<<<nblk((int64_t)n * n, VT), VT, 0, st>>>(n, u, Y);
  ++*launches;
}

void launch_hadamard_sq(cudaStream_t st, int64_t nn, const double* E, double* EE, int64_t* launches) {
  hadamard_sq_kernel<<<nblk(nn, VT), VT, 0, st>>>(nn, E, EE);
  ++*launches;
}

void launch_recover_pre(cudaStream_t st, int n, int m, const double* Yu, const double* Ct, const double* u,
                        double* Cw, double* dy, double* dS, const PcgCtl* ctl, int64_t* launches) {
  int64_t tot = (int64_t)n * n > m ? (int64_t)n * n : m;
  recover_pre_kernel<<<nblk(tot, VT), VT, 0, st>>>(n, m, Yu, Ct, u, Cw, dy, dS, ctl);
  ++*launches;
}

void launch_sym_plus_full(cudaStream_t st, int n, int r, const double* Z, const double* U, const double* Q,
                          double* out, int64_t* launches) {
  sym_plus_full_kernel<<<nblk((int64_t)n * n, VT), VT, 0, st>>>(n, r, Z, U, Q, out);
  ++*launches;
}

void launch_add_diag(cudaStream_t st, int n, double* C, const double* Dv, double c_i, int64_t* launches) {
  add_diag_kernel<<<nblk(n, VT), VT, 0, st>>>(n, C, Dv, c_i);
  ++*launches;
}

void launch_scale_B(cudaStream_t st, int m, int d, const double* B, const double* Dv, double* Bs, int64_t* launches) {
  scale_B_kernel<<<nblk((int64_t)m * d, VT), VT, 0, st>>>(m, d, B, Dv, Bs);
  ++*launches;
}

}  // namespace wc

// Vector kernels of the indefinite PCG (Def. pcg with the coefficient
// beta_j = <r_{j+1}, z_{j+1}> / <r_j, z_j>, Cor. pcg) on the augmented system (eq. augsys),
// and the finishing steps of the operator, preconditioner, right-hand side and recovery.
//
// Vectors have length m + d: the u-block (m) followed by the v-block (d, h-coordinates).
// Vectors and scalars (alpha, beta, <r,z>, ||r||^2, tau, ...) are FP64; the scalars live in a
// device control block, so an iteration needs no host round trip; every kernel returns
// at once when ctl->done is set.  Dot products are accumulated in FP64 and reduced
// deterministically: per-block partial sums, then the last block to finish (atomic ticket)
// adds them in block order.
#include <algorithm>
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
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

// The PCG update x += alpha p, r -= alpha Ap, ||r||^2 and the stop test (update_kernel's work),
// done by the one block that finished a reduction last, when the vectors are short enough for
// one block (saves a launch per iteration).  Every thread of the block calls it.
__device__ void update_tail(int nt, double* __restrict__ x, double* __restrict__ rv, const double* __restrict__ p,
                            const double* __restrict__ Ap, PcgCtl* __restrict__ ctl, double* sh) {
  __syncthreads();
  if (ctl->done) return;                   // uniform: written before the barrier
  const double alpha = ctl->alpha;
  double acc = 0.0;
  for (int q = threadIdx.x; q < nt; q += blockDim.x) {
    x[q] = fma(alpha, p[q], x[q]);
    const double rr = fma(-alpha, __ldcg(Ap + q), rv[q]);   // Ap: written by the other blocks
    rv[q] = rr;
    acc = fma(rr, rr, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    ctl->rr = acc;
    ctl->iters += 1;
    if (!isfinite(acc)) { ctl->status = 5; ctl->done = 1; }
    else if (acc <= ctl->tol2) { ctl->status = 0; ctl->done = 1; }
    else if (ctl->iters >= ctl->max_iters) { ctl->status = 4; ctl->done = 1; }
  }
}

// out = [u_src; pack(H) - D p_v] (optionally g - that), and in mode 1 the dot <p, out> -> alpha.
template <typename T>
__global__ void __launch_bounds__(VT)
ap_finish_kernel(int m, int d, int n, int r, const T* __restrict__ partA, int S, const T* __restrict__ Up,
                 const T* __restrict__ Vs, const T* __restrict__ H, const T* __restrict__ Dv,
                 const T* __restrict__ p, const T* __restrict__ g, T* __restrict__ out, int mode,
                 PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf, unsigned int* __restrict__ counter,
                 const float* __restrict__ partA32, int S32, const double* __restrict__ lin,
                 double* __restrict__ ux, double* __restrict__ ur) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const int nt = m + d;
  const double itau2 = lin ? 1.0 / (ctl->tau * ctl->tau) : 0.0;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double v;
    if (q < m) {
      v = 0.0;
      for (int s = 0; s < S; ++s) v += (double)partA[(int64_t)s * m + q];
      for (int s = 0; s < S32; ++s) v += (double)partA32[(int64_t)s * m + q];
      if (lin) v += lin[q] * itau2 * (double)p[q];   // linear block: tau^-2 diag(delta) p_u
      if (Up) {   // DIAG: A(sym(U Q^T)) = diag(U Q^T)
        for (int k = 0; k < r; ++k) v += (double)Up[q + (int64_t)k * n] * (double)Vs[q + (int64_t)k * n];
      }
    } else {
      const int h = q - m;
      v = pack_at(H, n, n, r, h) - (double)Dv[h] * (double)p[q];
    }
    if (g) v = (double)g[q] - v;
    out[q] = (T)v;
    if (mode == 1) acc = fma((double)p[q], v, acc);
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
    if (ux) update_tail(nt, ux, ur, reinterpret_cast<const double*>(p), reinterpret_cast<const double*>(out), ctl, sh);
  }
}

// x += alpha p; r -= alpha Ap; ||r||^2 -> stop test.
template <typename T>
__global__ void __launch_bounds__(VT)
update_kernel(int nt, T* __restrict__ x, T* __restrict__ rv, const T* __restrict__ p, const T* __restrict__ Ap,
              PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf, unsigned int* __restrict__ counter) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const double alpha = ctl->alpha;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    x[q] = (T)fma(alpha, (double)p[q], (double)x[q]);
    const T rr = (T)fma(-alpha, (double)Ap[q], (double)rv[q]);
    rv[q] = rr;
    acc = fma((double)rr, (double)rr, acc);
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
template <typename T>
__global__ void pc_d_s_kernel(int m, int d, int G, const T* __restrict__ partB, const T* __restrict__ rv,
                              T* __restrict__ s, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double t = 0.0;
  for (int gg = 0; gg < G; ++gg) t += (double)partB[(int64_t)gg * d + h];
  s[h] = (T)((double)rv[m + h] - t / ctl->beta_pc);
}

// d-space: z_v = -(C^{-1} s)
template <typename T>
__global__ void pc_d_zv_kernel(int m, int d, int S, const T* __restrict__ partC, T* __restrict__ z,
                               const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double t = 0.0;
  for (int s = 0; s < S; ++s) t += (double)partC[(int64_t)s * d + h];
  z[m + h] = (T)(-t);
}

// z_u (d-space: beta^{-1}(r_u - B z_v), or Lam^{-1}(r_u - B z_v) with a linear block; m-space:
// already formed) then <r, z> -> beta_pcg.
// mode 0 (start): rz = <r0, z0>;  mode 1 (iteration): beta = <r_{k+1}, z_{k+1}> / <r_k, z_k>.
template <typename T>
__global__ void __launch_bounds__(VT)
pc_zu_dot_kernel(int m, int d, int S, const T* __restrict__ partU, int space, const T* __restrict__ rv,
                 T* __restrict__ z, int mode, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                 unsigned int* __restrict__ counter, const double* __restrict__ lam, T* __restrict__ pf) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const int nt = m + d;
  const double ib = 1.0 / ctl->beta_pc;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double zq;
    if (q < m && partU) {
      double t = 0.0;
      for (int s = 0; s < S; ++s) t += (double)partU[(int64_t)s * m + q];
      zq = (space == 1) ? ((double)rv[q] - t) * (lam ? 1.0 / lam[q] : ib) : t;
      z[q] = (T)zq;
    } else {
      zq = (double)z[q];
    }
    acc = fma((double)rv[q], zq, acc);
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
    if (pf && mode == 1) {   // p = z + beta p in this block (p_update_kernel's work, one launch fewer)
      __syncthreads();
      if (ctl->done) return;
      const double beta = ctl->beta;
      for (int q = threadIdx.x; q < nt; q += blockDim.x) pf[q] = (T)fma(beta, (double)pf[q], (double)__ldcg(z + q));
    }
  }
}

// m-space helpers: t_v = r_v / D;  w = r_u + B t_v;  z_v = (B^T z_u - r_v) / D
template <typename T>
__global__ void pc_m_tv_kernel(int m, int d, const T* __restrict__ rv, const T* __restrict__ Dv, T* __restrict__ t,
                               const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  t[h] = (T)((double)rv[m + h] / (double)Dv[h]);
}

template <typename T>
__global__ void pc_m_w_kernel(int m, int S, const T* __restrict__ partB, const T* __restrict__ rv, T* __restrict__ w,
                              const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double t = 0.0;
  for (int s = 0; s < S; ++s) t += (double)partB[(int64_t)s * m + i];
  w[i] = (T)((rv ? (double)rv[i] : 0.0) + t);
}

template <typename T>
__global__ void pc_m_zv_kernel(int m, int d, int G, const T* __restrict__ partBt, const T* __restrict__ rv,
                               const T* __restrict__ Dv, T* __restrict__ z, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double t = 0.0;
  for (int gg = 0; gg < G; ++gg) t += (double)partBt[(int64_t)gg * d + h];
  z[m + h] = (T)((t - (double)rv[m + h]) / (double)Dv[h]);
}

// DIAG kind, m-space core with the products with B formed from Vs (no explicit B):
//   B t   = A(Q t) = diag(sym(U Q^T)) = rowdot(U, Q) with U = Vs unpack(t)
//   B^T u = Q^T svec(Diag(u)) = pack(Vs^T diag(u) Q)
// w = r_u + rowdot(U, Q)
__global__ void diag_w_kernel(int n, int r, const double* __restrict__ U, const double* __restrict__ Vs,
                              const double* __restrict__ rv, double* __restrict__ w, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = rv[i];
  for (int k = 0; k < r; ++k) t = fma(U[i + (int64_t)k * n], Vs[i + (int64_t)k * n], t);
  w[i] = t;
}

// z_v = (pack(H) - r_v) / D with H = Vs^T diag(z_u) Q
__global__ void diag_zv_kernel(int m, int d, int n, int r, const double* __restrict__ H,
                               const double* __restrict__ rv, const double* __restrict__ Dv, double* __restrict__ z,
                               const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  z[m + h] = (pack_at(H, n, n, r, h) - rv[m + h]) / Dv[h];
}

// d-space with B^T r_u = pack(H): s = r_v - beta^{-1} pack(H)
__global__ void pc_d_s_H_kernel(int m, int d, int n, int r, const double* __restrict__ H,
                                const double* __restrict__ rv, double* __restrict__ s,
                                const PcgCtl* __restrict__ ctl, int scaled) {
  if (ctl->done) return;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  // scaled: H came from Lam^{-1} r_u (linear block), so no division by beta
  s[h] = rv[m + h] - (scaled ? pack_at(H, n, n, r, h) : pack_at(H, n, n, r, h) / ctl->beta_pc);
}

// Tm = Q (Lam - tau I): the first r columns of Vs scaled by lam_j - tau
__global__ void shift_cols_kernel(int n, int r, const double* __restrict__ Vs, const double* __restrict__ lam_s,
                                  const PcgCtl* __restrict__ ctl, double* __restrict__ Tm) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * r) return;
  Tm[q] = Vs[q] * (lam_s[q / n] - ctl->tau);
}

// DIAG kind, m-space core in closed form (lower triangle and diagonal):
//   K = beta I + B D^{-1} B^T = beta I + tau^-2 G o (G + 2 tau E),  G = Q (Lam - tau I) Q^T.
// Row i of B is [svec(q_i q_i^T); sqrt2 vec(p_i q_i^T)] (q_i, p_i: row i of Q, Qp), and
// D^{-1} = diag(Lam (x)s Lam - tau^2 I, (Lam - tau I) (x) Lamp) / tau^2 (eq. EQSigdef), so
//   (B D^{-1} B^T)_il = tau^-2 [ (Q Lam Q^T)_il^2 - tau^2 (Q Q^T)_il^2
//                                + 2 (Q (Lam - tau I) Q^T)_il (Qp Lamp Qp^T)_il ];
// with Qp Lamp Qp^T = tau (E - Q Q^T) the bracket factors as G_il (G_il + 2 tau E_il).
__global__ void diag_K_kernel(int n, const double* __restrict__ G, const double* __restrict__ E,
                              const PcgCtl* __restrict__ ctl, double* __restrict__ K) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int i = (int)(q % n), l = (int)(q / n);
  if (i < l) return;
  const double tau = ctl->tau;
  const double g = G[q];
  double v = g * fma(2.0 * tau, E[q], g) / (tau * tau);
  if (i == l) v += ctl->beta_pc;
  K[q] = v;
}

// ---- MINRES (Def. MINRES with P = I; the recurrence of Paige and Saunders) ----------------
// r1, r2: the last two Lanczos residuals (r2 = beta v_{k+1}); v: the Lanczos vector; y = M v;
// w, w1, w2: the search directions; x: the iterate.  Scalars in MinresCtl, the stop test and
// the iteration count in PcgCtl (rr = phibar^2 against tol2).

// start: r1 = r2 = g, x = w = w2 = 0; beta = ||g|| (last block), phibar = beta, cs = -1
__global__ void __launch_bounds__(VT)
minres_init_kernel(int nt, const double* __restrict__ g, double* __restrict__ r1, double* __restrict__ r2,
                   double* __restrict__ x, double* __restrict__ w, double* __restrict__ w2,
                   MinresCtl* __restrict__ mc, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                   unsigned int* __restrict__ counter) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    const double v = g[q];
    r1[q] = v;
    r2[q] = v;
    x[q] = 0.0;
    w[q] = 0.0;
    w2[q] = 0.0;
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    const double gg = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      const double b1 = sqrt(gg);
      mc->beta = b1;
      mc->oldb = 0.0;
      mc->alfa = 0.0;
      mc->dbar = 0.0;
      mc->epsln = 0.0;
      mc->oldeps = 0.0;
      mc->delta = 0.0;
      mc->gamma = 1.0;
      mc->cs = -1.0;
      mc->sn = 0.0;
      mc->phi = 0.0;
      mc->phibar = b1;
      mc->itn = 0;
      mc->stop = 0;
      ctl->rr = gg;
      ctl->rr0 = gg;
      ctl->iters = 0;
      ctl->status = 0;
      ctl->done = (gg <= ctl->tol2 || !(b1 > 0.0)) ? 1 : 0;
    }
  }
}

// v = r2 / beta; a stop recorded by the previous iteration raises done here (after that
// iteration's update of x)
__global__ void minres_v_kernel(int nt, const double* __restrict__ r2, double* __restrict__ v,
                                MinresCtl* __restrict__ mc, PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  if (mc->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->done = 1;
    return;
  }
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  v[q] = r2[q] / mc->beta;
}

// y -= (beta / oldb) r1 (from the second iteration on); alfa = <v, y>
__global__ void __launch_bounds__(VT)
minres_alfa_kernel(int nt, const double* __restrict__ v, double* __restrict__ y, const double* __restrict__ r1,
                   MinresCtl* __restrict__ mc, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                   unsigned int* __restrict__ counter) {
  if (ctl->done || mc->stop) return;
  __shared__ double sh[32];
  const double c = (mc->itn >= 1) ? mc->beta / mc->oldb : 0.0;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double t = y[q];
    if (c != 0.0) t = fma(-c, r1[q], t);
    y[q] = t;
    acc = fma(v[q], t, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    const double a = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      mc->alfa = a;
    }
  }
}

// t = y - (alfa / beta) r2; r1 = r2; r2 = t; beta_{k+1} = ||t||; then the Givens rotation that
// eliminates beta_{k+1} from the tridiagonal, phi, phibar = ||r_k||, and the stop test
__global__ void __launch_bounds__(VT)
minres_beta_kernel(int nt, const double* __restrict__ y, double* __restrict__ r1, double* __restrict__ r2,
                   MinresCtl* __restrict__ mc, PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf,
                   unsigned int* __restrict__ counter) {
  if (ctl->done || mc->stop) return;
  __shared__ double sh[32];
  const double c = mc->alfa / mc->beta;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    const double old2 = r2[q];
    const double t = fma(-c, old2, y[q]);
    r1[q] = old2;
    r2[q] = t;
    acc = fma(t, t, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    const double bb = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      const double alfa = mc->alfa;
      mc->oldb = mc->beta;
      const double beta = sqrt(bb);
      mc->beta = beta;
      mc->oldeps = mc->epsln;
      const double delta = mc->cs * mc->dbar + mc->sn * alfa;
      const double gbar = mc->sn * mc->dbar - mc->cs * alfa;
      mc->epsln = mc->sn * beta;
      mc->dbar = -mc->cs * beta;
      double gamma = hypot(gbar, beta);
      if (!(gamma > 0.0)) gamma = 1e-300;
      mc->delta = delta;
      mc->gamma = gamma;
      mc->cs = gbar / gamma;
      mc->sn = beta / gamma;
      mc->phi = mc->cs * mc->phibar;
      mc->phibar = mc->sn * mc->phibar;
      mc->itn += 1;
      const double rr = mc->phibar * mc->phibar;
      ctl->rr = rr;
      ctl->iters += 1;
      if (!isfinite(rr) || !isfinite(mc->phi)) { ctl->status = 5; ctl->done = 1; }
      else if (rr <= ctl->tol2 || beta == 0.0) { ctl->status = 0; mc->stop = 1; }
      else if (ctl->iters >= ctl->max_iters) { ctl->status = 4; mc->stop = 1; }
    }
  }
}

// w1 = w2; w2 = w; w = (v - oldeps w1 - delta w2) / gamma; x += phi w
__global__ void minres_update_kernel(int nt, const double* __restrict__ v, double* __restrict__ w,
                                     double* __restrict__ w1, double* __restrict__ w2, double* __restrict__ x,
                                     const MinresCtl* __restrict__ mc, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  const double a = w2[q], b = w[q];
  const double nw = (v[q] - mc->oldeps * a - mc->delta * b) / mc->gamma;
  w1[q] = a;
  w2[q] = b;
  w[q] = nw;
  x[q] = fma(mc->phi, nw, x[q]);
}

// p = z + beta p  (start: p = z)
template <typename T>
__global__ void p_update_kernel(int nt, const T* __restrict__ z, T* __restrict__ p, int start,
                                const PcgCtl* __restrict__ ctl) {
  if (ctl->done && !start) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  p[q] = start ? z[q] : (T)fma(ctl->beta, (double)p[q], (double)z[q]);
}

// DIAG kind: the slab partial sums of diag(F E) = diag(E C~ E) with F = E C~, E symmetric (stored
// in full), so that (F E)_qq = sum_k F[q, k] E[q, k]: thread q of slab s sums k in
// [s KS, (s + 1) KS) with coalesced loads of both operands and four independent chains.
__global__ void __launch_bounds__(VT)
diag_FE_kernel(int n, int KS, const double* __restrict__ F, const double* __restrict__ E, double* __restrict__ part) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int k0 = blockIdx.y * KS, k1 = min(n, k0 + KS);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = k0;
  for (; k + 3 < k1; k += 4) {
    const int64_t o = q + (int64_t)k * n;
    a0 = fma(F[o], E[o], a0);
    a1 = fma(F[o + n], E[o + n], a1);
    a2 = fma(F[o + 2 * n], E[o + 2 * n], a2);
    a3 = fma(F[o + 3 * n], E[o + 3 * n], a3);
  }
  for (; k < k1; ++k) a0 = fma(F[q + (int64_t)k * n], E[q + (int64_t)k * n], a0);
  part[(int64_t)blockIdx.y * n + q] = (a0 + a1) + (a2 + a3);
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

// ||r||^2 and the stop test (rel_rtol2 > 0: the threshold becomes rel_rtol2 ||r||^2).
template <typename T>
__global__ void __launch_bounds__(VT)
norm_check_kernel(int nt, const T* __restrict__ rv, double rel_rtol2, PcgCtl* __restrict__ ctl,
                  double* __restrict__ dotbuf, unsigned int* __restrict__ counter) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x)
    acc = fma((double)rv[q], (double)rv[q], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) dotbuf[blockIdx.x] = acc;
  if (last_block(counter)) {
    double rr = sum_partials(dotbuf, gridDim.x, sh);
    if (threadIdx.x == 0) {
      *counter = 0;
      ctl->rr = rr;
      if (ctl->iters == 0) ctl->rr0 = rr;
      if (rel_rtol2 > 0.0) ctl->tol2 = rel_rtol2 * rr;
      if (!isfinite(rr)) { ctl->status = 5; ctl->done = 1; }
      else if (rr <= ctl->tol2) ctl->done = 1;
    }
  }
}

// T = diag(p_u) Q  (DIAG kind: A^T(p_u) Q)
template <typename T>
__global__ void diag_scale_rows_kernel(int n, int r, const T* __restrict__ pu, const T* __restrict__ Vs,
                                       T* __restrict__ Tm, const int32_t* __restrict__ done) {
  if (done && *done) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * r) return;
  Tm[q] = pu[q % n] * Vs[q];
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
  const double it2 = 1.0 / t2;   // one division per thread, not per entry (FP64 division is a long chain)
  const int64_t nn = (int64_t)n * n, tot = nn > m ? nn : m;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    if (q < nn) {
      const double y = Yu[q], c = Ct[q];
      if (Cw) Cw[q] = y - t2 * c;
      dS[q] = c - y * it2;
    }
    if (q < m) dy[q] = u[q] * it2;
  }
}

// E Cw with Cw = A^T(u) - tau^2 C~, from F = E C~ of the right side (overwritten):
// F = E A^T(u) - tau^2 F, with E A^T(u) given (EYu) or, for the DIAG kind, E diag(u)
__global__ void recover_F_kernel(int n, const double* __restrict__ EYu, const double* __restrict__ E,
                                 const double* __restrict__ u, double* __restrict__ F,
                                 const PcgCtl* __restrict__ ctl) {
  const double t2 = ctl->tau * ctl->tau;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const double ey = EYu ? EYu[q] : E[q] * u[q / n];
  F[q] = ey - t2 * F[q];
}

// C += diag(Dv) * c_d + c_i * I  on an n x n matrix
// linear block of the Newton system: Lam = beta + tau^-2 delta (the (1,1) block of the preconditioner)
__global__ void lin_lam_kernel(int m, const double* __restrict__ delta, const PcgCtl* __restrict__ ctl,
                               double* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) lam[i] = ctl->beta_pc + delta[i] / (ctl->tau * ctl->tau);
}

// m_free = #{i : tau^-2 delta_i <= dominance beta}: the rows of the linear block not fixed by their
// slack (one block; deterministic integer count)
__global__ void lin_free_count_kernel(int m, const double* __restrict__ delta, double dominance,
                                      PcgCtl* __restrict__ ctl) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const double lim = dominance * ctl->beta_pc * ctl->tau * ctl->tau;
  int c = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) c += (delta[i] <= lim) ? 1 : 0;
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) ctl->m_free = cnt;
}

// out = r_u / Lam (the first block of r only)
__global__ void lin_div_kernel(int m, const double* __restrict__ r, const double* __restrict__ lam,
                               double* __restrict__ out, const PcgCtl* __restrict__ ctl) {
  if (ctl->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = r[i] / lam[i];
}

// Bw (d x m, col-major view of B row-major) = B with row i scaled by Lam_i^-1/2
__global__ void lin_scale_rows_kernel(int m, int d, const double* __restrict__ B, const double* __restrict__ lam,
                                      double* __restrict__ Bw) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)m * d) return;
  Bw[q] = B[q] / sqrt(lam[q / d]);
}

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

// Mixed form: [0; rho_v], whose image under the preconditioner starts the correction solve
// (P delta0 = [0; rho_v] leaves the second block of rho - M delta0 at zero, as Cor. pcg asks,
// while delta0 stays of the size of rho_v, with no division by the small entries of D).
__global__ void correction_rhs_kernel(int m, int d, const double* __restrict__ rho, double* __restrict__ out) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m + d) return;
  out[q] = (q < m) ? 0.0 : rho[q];
}

// out = (g + g^T) / 2 (n x n)
__global__ void sym_copy_kernel(int n, const double* __restrict__ g, double* __restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  int a = (int)(q % n), b = (int)(q / n);
  out[q] = 0.5 * (g[q] + g[b + (int64_t)a * n]);
}

// x += delta
__global__ void add_correction_kernel(int nt, const double* __restrict__ delta, double* __restrict__ x) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  x[q] += delta[q];
}

// Mixed-form operator: the well-conditioned block A E A^T p_u from FP32 partial sums, the
// blocks with B = A Q (which meet D^{-1} through the iterates) in FP64:
//   out = [sum_s partA32 + sum_s partBv; sum_g partBu - D p_v]  (optionally g - that);
// mode 1 also forms <p, out> and alpha.
__global__ void __launch_bounds__(VT)
mixed_finish_kernel(int m, int d, const float* __restrict__ partA32, int SA, const double* __restrict__ partBv,
                    int SB, const double* __restrict__ partBu, int SBu, const double* __restrict__ Dv,
                    const double* __restrict__ p, const double* __restrict__ g, double* __restrict__ out, int mode,
                    PcgCtl* __restrict__ ctl, double* __restrict__ dotbuf, unsigned int* __restrict__ counter,
                    double* __restrict__ ux, double* __restrict__ ur) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const int nt = m + d;
  double acc = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (q < m) {
      for (int s = 0; s < SA; ++s) v += (double)partA32[(int64_t)s * m + q];
      for (int s = 0; s < SB; ++s) v += partBv[(int64_t)s * m + q];
    } else {
      const int h = q - m;
      for (int s = 0; s < SBu; ++s) v += partBu[(int64_t)s * d + h];
      v -= Dv[h] * p[q];
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
      if (pAp == 0.0 || !isfinite(pAp) || !isfinite(ctl->rz)) {
        ctl->status = 5;
        ctl->done = 1;
      } else {
        ctl->alpha = ctl->rz / pAp;
      }
    }
    if (ux) update_tail(nt, ux, ur, p, out, ctl, sh);
  }
}

// p_u32 = (float) p_u
__global__ void to_float_kernel(int cnt, const double* __restrict__ src, float* __restrict__ dst,
                                const int32_t* __restrict__ done) {
  if (done && *done) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < cnt) dst[q] = (float)src[q];
}

// inner control block: the split scalars of src, counters reset
__global__ void ctl_reset_kernel(PcgCtl* __restrict__ dst, const PcgCtl* __restrict__ src, int max_iters) {
  if (threadIdx.x != 0) return;
  *dst = *src;
  dst->done = 0;
  dst->iters = 0;
  dst->status = 0;
  dst->max_iters = max_iters;
  dst->tol2 = 0.0;
}

inline unsigned nblk(int64_t total, int t) { return (unsigned)((total + t - 1) / t); }
inline int vec_blocks(int nt) {
  int b = (nt + VT - 1) / VT;
  return b > 256 ? 256 : b;
}

// The adjoint with the slacks of eq. rmc-sdp (G = [I, -I], D = diag(d_v, d_w)): delta = d_v + d_w,
// b~ = g_y + G D c~ with c~ = (g_v, g_w); afterwards dx = D(G^T dy - c~).
__global__ void slack_grad_rhs_kernel(int m, const double* __restrict__ dv, const double* __restrict__ dw,
                                      const double* __restrict__ gy, const double* __restrict__ gv,
                                      const double* __restrict__ gw, double* __restrict__ delta,
                                      double* __restrict__ bt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  delta[i] = dv[i] + dw[i];
  bt[i] = gy[i] + dv[i] * gv[i] - dw[i] * gw[i];
}

__global__ void slack_grad_out_kernel(int m, const double* __restrict__ dv, const double* __restrict__ dw,
                                      const double* __restrict__ dy, const double* __restrict__ gv,
                                      const double* __restrict__ gw, double* __restrict__ ov,
                                      double* __restrict__ ow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  ov[i] = dv[i] * (dy[i] - gv[i]);
  ow[i] = dw[i] * (-dy[i] - gw[i]);
}

// y_i = <row i of M, v> for i < rows (M row-major, leading dimension ld), this CTA's share, with
// every output passed to out(i, y_i) by one thread.  The rows spread over the whole grid: the
// CTA's 8 warps form groups of g warps (g = the grid's warps per row, a power of two <= 8), group
// q of CTA b takes rows (t G + b) (8 / g) + q, and the 32 g lanes of a group stride over the row
// with four independent accumulators (on GB300 a dependent FP64 FMA waits about 140 clocks and an
// L2 load several hundred, so one warp walking a long row alone would set the time).  v (written
// by other blocks of the launch) is read through L2, once per CTA into shared memory when it fits.
// The partial sums are combined in a fixed order.
constexpr int kStageMax = 4096;   // vectors up to this length are staged in shared memory

template <typename Out>
__device__ void cta_rows_dot(int rows, int len, const double* __restrict__ M, int64_t ld,
                             const double* __restrict__ vg, Out out, double* sh /* >= 8 doubles */,
                             double* vs /* kStageMax doubles of shared memory */) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = (int)gridDim.x;
  int g = (G * 8) / max(rows, 1);
  g = g >= 8 ? 8 : g >= 4 ? 4 : g >= 2 ? 2 : 1;
  const int gpc = 8 / g, q = warp / g, wi = warp % g, step = 32 * g;
  const int slots = (rows + gpc - 1) / gpc;
  // v is read by every row: once per CTA into shared memory (all loads issued before the stores)
  const double* v = vg;
  if (len <= kStageMax && (int)blockIdx.x < slots) {
    for (int k0 = threadIdx.x; k0 < len; k0 += 8 * blockDim.x) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u * blockDim.x;
        t[u] = k < len ? __ldcg(vg + k) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u * blockDim.x;
        if (k < len) vs[k] = t[u];
      }
    }
    __syncthreads();
    v = vs;
  }
  for (int t = blockIdx.x; t < slots; t += G) {       // the same trip count in every thread of the CTA
    const int i = t * gpc + q;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (i < rows) {
      const double* row = M + (int64_t)i * ld;
      int k = wi * 32 + lane;
      for (; k + 3 * step < len; k += 4 * step) {
        a0 = fma(row[k], v[k], a0);
        a1 = fma(row[k + step], v[k + step], a1);
        a2 = fma(row[k + 2 * step], v[k + 2 * step], a2);
        a3 = fma(row[k + 3 * step], v[k + 3 * step], a3);
      }
      for (; k < len; k += step) a0 = fma(row[k], v[k], a0);
    }
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (wi == 0 && lane == 0 && i < rows) {
      double y = 0.0;
      for (int w = 0; w < g; ++w) y += sh[q * g + w];
      out(i, y);
    }
    __syncthreads();
  }
}

// The d-space preconditioner apply of the dense kind in one cooperative launch (Section 6: the
// block LDL^T inverse of P = [beta I, B; B^T, -D]):
//   s = r_v - beta^{-1} B^T r_u,  z_v = -C^{-1} s,  z_u = beta^{-1} (r_u - B z_v),
// then <r, z> (mode 0: rz; mode 1: beta_pcg = <r_new, z_new> / <r, z>) and, with pf, p = z + beta p.
// With ux (mode 1 inside the PCG loop) the launch first does the PCG update x += alpha p,
// r -= alpha Ap with ||r||^2 and the stop test, so that no single block of the operator's
// finishing kernel walks the whole vectors.  Three products that depend on each other, on
// L2-resident matrices (B^T, C^{-1}, B): one warp per output row, grid-wide barriers between the
// steps.  Every block reduces the per-block partial sums itself, in block order, so all blocks
// take the same decisions from bit-identical scalars; only block 0 writes the control block.
__global__ void __launch_bounds__(256)
pc_dense_d_coop_kernel(int m, int d, const double* __restrict__ Bt, const double* __restrict__ Pinv,
                       const double* __restrict__ B, double* __restrict__ rv, double* __restrict__ z,
                       double* __restrict__ sd, double* __restrict__ part, int mode, PcgCtl* __restrict__ ctl,
                       double* __restrict__ pf, double* __restrict__ ux, const double* __restrict__ Ap) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  if (ctl->done) return;                     // uniform: set only by earlier launches
  __shared__ double sh[32];
  const int G = (int)gridDim.x, bid = (int)blockIdx.x;
  const int gt = (int)(blockIdx.x * blockDim.x + threadIdx.x), nthr = (int)(gridDim.x * blockDim.x);
  const int nt = m + d;
  // the scalars this launch needs, read before block 0 writes any of them
  const double ib = 1.0 / ctl->beta_pc;
  const double rz_old = ctl->rz;
  if (ux) {
    const double alpha = ctl->alpha, tol2 = ctl->tol2;
    const int iters = ctl->iters, max_iters = ctl->max_iters;
    double acc = 0.0;
    for (int q = gt; q < nt; q += nthr) {
      ux[q] = fma(alpha, pf[q], ux[q]);
      const double rr = fma(-alpha, Ap[q], rv[q]);
      rv[q] = rr;
      acc = fma(rr, rr, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[G + bid] = acc;
    grid.sync();
    double rr = 0.0;
    for (int q = threadIdx.x; q < G; q += blockDim.x) rr += __ldcg(part + G + q);
    rr = block_sum(rr, sh);
    int stop = -1;
    if (!isfinite(rr)) stop = 5;
    else if (rr <= tol2) stop = 0;
    else if (iters + 1 >= max_iters) stop = 4;
    if (bid == 0 && threadIdx.x == 0) {
      ctl->rr = rr;
      ctl->iters = iters + 1;
      if (stop >= 0) { ctl->status = stop; ctl->done = 1; }
    }
    if (stop >= 0) return;                   // uniform: every block reduced the same partials
  }
  const double* ru = rv;
  const double* rvv = rv + m;
  __shared__ double shw[8];
  __shared__ double vstage[kStageMax];
  // s = r_v - beta^{-1} B^T r_u
  cta_rows_dot(d, m, Bt, m, ru, [&](int i, double y) { sd[i] = __ldcg(rvv + i) - ib * y; }, shw, vstage);
  grid.sync();
  // z_v = -C^{-1} s, and its part of <r, z>
  double dot = 0.0;
  cta_rows_dot(d, d, Pinv, d, sd, [&](int i, double y) {
    z[m + i] = -y;
    dot = fma(__ldcg(rvv + i), -y, dot);
  }, shw, vstage);
  grid.sync();
  // z_u = beta^{-1} (r_u - B z_v), and its part of <r, z>
  cta_rows_dot(m, d, B, d, z + m, [&](int j, double y) {
    const double u = __ldcg(ru + j);
    const double zu = ib * (u - y);
    z[j] = zu;
    dot = fma(u, zu, dot);
  }, shw, vstage);
  dot = block_sum(dot, sh);
  if (threadIdx.x == 0) part[bid] = dot;
  grid.sync();
  double rz = 0.0;
  for (int q = threadIdx.x; q < G; q += blockDim.x) rz += __ldcg(part + q);
  rz = block_sum(rz, sh);
  const bool ok = isfinite(rz);
  const double beta = mode == 0 ? 0.0 : rz / rz_old;
  if (bid == 0 && threadIdx.x == 0) {
    if (!ok) { ctl->status = 5; ctl->done = 1; }
    if (mode == 0) { ctl->rz = rz; ctl->beta = 0.0; }
    else { ctl->rz_new = rz; ctl->beta = beta; ctl->rz = rz; }
  }
  if (pf && mode == 1 && ok)                 // p = z + beta p, every block its slice
    for (int q = gt; q < nt; q += nthr) pf[q] = fma(beta, pf[q], __ldcg(z + q));
}

// The condition of the device-side PCG loop (a WHILE graph node around one iteration): go on
// while the stop flag is clear, and in any case for at most max_iters + 2 passes, counted here
// independently of the other kernels, so that the loop ends even if no kernel ever set the flag.
__global__ void loop_cond_kernel(cudaGraphConditionalHandle hc, const PcgCtl* __restrict__ ctl,
                                 int* __restrict__ guard) {
  const int passes = ++*guard;
  cudaGraphSetConditional(hc, (!ctl->done && passes <= ctl->max_iters + 2) ? 1u : 0u);
}

}  // namespace

void launch_loop_cond(cudaStream_t st, cudaGraphConditionalHandle hc, const PcgCtl* ctl, int* guard,
                      int64_t* launches) {
  loop_cond_kernel<<<1, 1, 0, st>>>(hc, ctl, guard);
  if (launches) ++*launches;
}

template <typename T>
void launch_ap_finish(cudaStream_t st, int m, int d, int n, int r, const T* partA, int S, const T* Up, const T* Vs,
                      const T* H, const T* Dv, const T* p, const T* g, T* out, int mode, PcgCtl* ctl,
                      double* dotbuf, unsigned int* counter, int64_t* launches, const float* partA32, int S32,
                      const double* lin, double* ux, double* ur) {
  ap_finish_kernel<T><<<vec_blocks(m + d), VT, 0, st>>>(m, d, n, r, partA, S, Up, Vs, H, Dv, p, g, out, mode, ctl,
                                                       dotbuf, counter, partA32, S32, lin, mode == 1 ? ux : nullptr,
                                                       ur);
  ++*launches;
}

template <typename T>
void launch_update(cudaStream_t st, int nt, T* x, T* rv, const T* p, const T* Ap, PcgCtl* ctl, double* dotbuf,
                   unsigned int* counter, int64_t* launches) {
  update_kernel<T><<<vec_blocks(nt), VT, 0, st>>>(nt, x, rv, p, Ap, ctl, dotbuf, counter);
  ++*launches;
}

template <typename T>
void launch_pc_d_s(cudaStream_t st, int m, int d, int G, const T* partB, const T* rv, T* s, const PcgCtl* ctl,
                   int64_t* launches) {
  pc_d_s_kernel<T><<<nblk(d, VT), VT, 0, st>>>(m, d, G, partB, rv, s, ctl);
  ++*launches;
}

template <typename T>
void launch_pc_d_zv(cudaStream_t st, int m, int d, int S, const T* partC, T* z, const PcgCtl* ctl,
                    int64_t* launches) {
  pc_d_zv_kernel<T><<<nblk(d, VT), VT, 0, st>>>(m, d, S, partC, z, ctl);
  ++*launches;
}

template <typename T>
void launch_pc_zu_dot(cudaStream_t st, int m, int d, int S, const T* partU, int space, const T* rv, T* z, int mode,
                      PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches, const double* lam,
                      T* pf) {
  pc_zu_dot_kernel<T><<<vec_blocks(m + d), VT, 0, st>>>(m, d, S, partU, space, rv, z, mode, ctl, dotbuf, counter,
                                                       lam, pf);
  ++*launches;
}

template <typename T>
void launch_pc_m_tv(cudaStream_t st, int m, int d, const T* rv, const T* Dv, T* t, const PcgCtl* ctl,
                    int64_t* launches) {
  pc_m_tv_kernel<T><<<nblk(d, VT), VT, 0, st>>>(m, d, rv, Dv, t, ctl);
  ++*launches;
}

template <typename T>
void launch_pc_m_w(cudaStream_t st, int m, int S, const T* partB, const T* rv, T* w, const PcgCtl* ctl,
                   int64_t* launches) {
  pc_m_w_kernel<T><<<nblk(m, VT), VT, 0, st>>>(m, S, partB, rv, w, ctl);
  ++*launches;
}

template <typename T>
void launch_pc_m_zv(cudaStream_t st, int m, int d, int G, const T* partBt, const T* rv, const T* Dv, T* z,
                    const PcgCtl* ctl, int64_t* launches) {
  pc_m_zv_kernel<T><<<nblk(d, VT), VT, 0, st>>>(m, d, G, partBt, rv, Dv, z, ctl);
  ++*launches;
}

template <typename T>
void launch_p_update(cudaStream_t st, int nt, const T* z, T* p, int start, const PcgCtl* ctl, int64_t* launches) {
  p_update_kernel<T><<<nblk(nt, VT), VT, 0, st>>>(nt, z, p, start, ctl);
  ++*launches;
}

template <typename T>
void launch_norm_check(cudaStream_t st, int nt, const T* rv, double rel_rtol2, PcgCtl* ctl, double* dotbuf,
                       unsigned int* counter, int64_t* launches) {
  norm_check_kernel<T><<<vec_blocks(nt), VT, 0, st>>>(nt, rv, rel_rtol2, ctl, dotbuf, counter);
  ++*launches;
}

template <typename T>
void launch_diag_scale_rows(cudaStream_t st, int n, int r, const T* pu, const T* Vs, T* Tm, const int32_t* done,
                            int64_t* launches) {
  diag_scale_rows_kernel<T><<<nblk((int64_t)n * r, VT), VT, 0, st>>>(n, r, pu, Vs, Tm, done);
  ++*launches;
}

#define WC_INSTANTIATE(T)                                                                                          \
  template void launch_ap_finish<T>(cudaStream_t, int, int, int, int, const T*, int, const T*, const T*, const T*,  \
                                    const T*, const T*, const T*, T*, int, PcgCtl*, double*, unsigned int*,          \
                                    int64_t*, const float*, int, const double*, double*, double*);                  \
  template void launch_update<T>(cudaStream_t, int, T*, T*, const T*, const T*, PcgCtl*, double*, unsigned int*,   \
                                 int64_t*);                                                                         \
  template void launch_pc_d_s<T>(cudaStream_t, int, int, int, const T*, const T*, T*, const PcgCtl*, int64_t*);      \
  template void launch_pc_d_zv<T>(cudaStream_t, int, int, int, const T*, T*, const PcgCtl*, int64_t*);              \
  template void launch_pc_zu_dot<T>(cudaStream_t, int, int, int, const T*, int, const T*, T*, int, PcgCtl*, double*, \
                                    unsigned int*, int64_t*, const double*, T*);                                    \
  template void launch_pc_m_tv<T>(cudaStream_t, int, int, const T*, const T*, T*, const PcgCtl*, int64_t*);         \
  template void launch_pc_m_w<T>(cudaStream_t, int, int, const T*, const T*, T*, const PcgCtl*, int64_t*);          \
  template void launch_pc_m_zv<T>(cudaStream_t, int, int, int, const T*, const T*, const T*, T*, const PcgCtl*,     \
                                  int64_t*);                                                                        \
  template void launch_p_update<T>(cudaStream_t, int, const T*, T*, int, const PcgCtl*, int64_t*);                  \
  template void launch_norm_check<T>(cudaStream_t, int, const T*, double, PcgCtl*, double*, unsigned int*,          \
                                     int64_t*);                                                                     \
  template void launch_diag_scale_rows<T>(cudaStream_t, int, int, const T*, const T*, T*, const int32_t*, int64_t*);
WC_INSTANTIATE(double)
#undef WC_INSTANTIATE

void launch_rhs_finish(cudaStream_t st, int m, int d, int n, int r, const double* partA, int S, const double* F,
                       const double* E, const double* bt, const double* Ct, const double* H, const double* Dv,
                       double* g, double* x, double rtol, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                       int64_t* launches) {
  rhs_finish_kernel<<<vec_blocks(m + d), VT, 0, st>>>(m, d, n, r, partA, S, F, E, bt, Ct, H, Dv, g, x, rtol, ctl,
                                                     dotbuf, counter);
  ++*launches;
}

int launch_diag_FE(cudaStream_t st, int n, const double* F, const double* E, double* part, int max_slabs,
                   int64_t* launches) {
  int S = std::min(std::min(32, (n + 31) / 32), std::max(1, max_slabs));
  const int KS = (n + S - 1) / S;
  S = (n + KS - 1) / KS;
  diag_FE_kernel<<<dim3((unsigned)((n + VT - 1) / VT), (unsigned)S), VT, 0, st>>>(n, KS, F, E, part);
  ++*launches;
  return S;
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
  recover_pre_kernel<<<(unsigned)std::min<int64_t>(nblk(tot, VT), 8 * (int64_t)g_num_sms), VT, 0, st>>>(n, m, Yu, Ct, u,
                                                                                                 Cw, dy, dS, ctl);
  ++*launches;
}

void launch_recover_F(cudaStream_t st, int n, const double* EYu, const double* E, const double* u, double* F,
                      const PcgCtl* ctl, int64_t* launches) {
  recover_F_kernel<<<nblk((int64_t)n * n, VT), VT, 0, st>>>(n, EYu, E, u, F, ctl);
  ++*launches;
}

void launch_lin_lam(cudaStream_t st, int m, const double* delta, const PcgCtl* ctl, double* lam, int64_t* launches) {
  lin_lam_kernel<<<nblk(m, VT), VT, 0, st>>>(m, delta, ctl, lam);
  ++*launches;
}

void launch_lin_free_count(cudaStream_t st, int m, const double* delta, double dominance, PcgCtl* ctl,
                           int64_t* launches) {
  lin_free_count_kernel<<<1, 1024, 0, st>>>(m, delta, dominance, ctl);
  ++*launches;
}

void launch_lin_div(cudaStream_t st, int m, const double* r, const double* lam, double* out, const PcgCtl* ctl,
                    int64_t* launches) {
  lin_div_kernel<<<nblk(m, VT), VT, 0, st>>>(m, r, lam, out, ctl);
  ++*launches;
}

void launch_lin_scale_rows(cudaStream_t st, int m, int d, const double* B, const double* lam, double* Bw,
                           int64_t* launches) {
  lin_scale_rows_kernel<<<nblk((int64_t)m * d, VT), VT, 0, st>>>(m, d, B, lam, Bw);
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

void launch_correction_rhs(cudaStream_t st, int m, int d, const double* rho, double* out, int64_t* launches) {
  correction_rhs_kernel<<<nblk(m + d, VT), VT, 0, st>>>(m, d, rho, out);
  ++*launches;
}

void launch_mixed_finish(cudaStream_t st, int m, int d, const float* partA32, int SA, const double* partBv, int SB,
                         const double* partBu, int SBu, const double* Dv, const double* p, const double* g,
                         double* out, int mode, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                         int64_t* launches, double* ux, double* ur) {
  mixed_finish_kernel<<<vec_blocks(m + d), VT, 0, st>>>(m, d, partA32, SA, partBv, SB, partBu, SBu, Dv, p, g, out,
                                                       mode, ctl, dotbuf, counter, mode == 1 ? ux : nullptr, ur);
  ++*launches;
}

void launch_to_float(cudaStream_t st, int cnt, const double* src, float* dst, const int32_t* done, int64_t* launches) {
  to_float_kernel<<<nblk(cnt, VT), VT, 0, st>>>(cnt, src, dst, done);
  ++*launches;
}

void launch_sym_copy(cudaStream_t st, int n, const double* g, double* out, int64_t* launches) {
  sym_copy_kernel<<<nblk((int64_t)n * n, VT), VT, 0, st>>>(n, g, out);
  ++*launches;
}

void launch_add_correction(cudaStream_t st, int nt, const double* delta, double* x, int64_t* launches) {
  add_correction_kernel<<<nblk(nt, VT), VT, 0, st>>>(nt, delta, x);
  ++*launches;
}

void launch_diag_w(cudaStream_t st, int n, int r, const double* U, const double* Vs, const double* rv, double* w,
                   const PcgCtl* ctl, int64_t* launches) {
  diag_w_kernel<<<nblk(n, VT), VT, 0, st>>>(n, r, U, Vs, rv, w, ctl);
  ++*launches;
}

void launch_diag_zv(cudaStream_t st, int m, int d, int n, int r, const double* H, const double* rv, const double* Dv,
                    double* z, const PcgCtl* ctl, int64_t* launches) {
  diag_zv_kernel<<<nblk(d, VT), VT, 0, st>>>(m, d, n, r, H, rv, Dv, z, ctl);
  ++*launches;
}

void launch_pc_d_s_H(cudaStream_t st, int m, int d, int n, int r, const double* H, const double* rv, double* s,
                     const PcgCtl* ctl, int64_t* launches, bool scaled) {
  pc_d_s_H_kernel<<<nblk(d, VT), VT, 0, st>>>(m, d, n, r, H, rv, s, ctl, scaled ? 1 : 0);
  ++*launches;
}

void launch_shift_cols(cudaStream_t st, int n, int r, const double* Vs, const double* lam_s, const PcgCtl* ctl,
                       double* Tm, int64_t* launches) {
  shift_cols_kernel<<<nblk((int64_t)n * r, VT), VT, 0, st>>>(n, r, Vs, lam_s, ctl, Tm);
  ++*launches;
}

void launch_diag_K(cudaStream_t st, int n, const double* G, const double* E, const PcgCtl* ctl, double* K,
                   int64_t* launches) {
  diag_K_kernel<<<nblk((int64_t)n * n, VT), VT, 0, st>>>(n, G, E, ctl, K);
  ++*launches;
}

void launch_minres_init(cudaStream_t st, int nt, const double* g, double* r1, double* r2, double* x, double* w,
                        double* w2, MinresCtl* mc, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                        int64_t* launches) {
  minres_init_kernel<<<vec_blocks(nt), VT, 0, st>>>(nt, g, r1, r2, x, w, w2, mc, ctl, dotbuf, counter);
  ++*launches;
}

void launch_minres_v(cudaStream_t st, int nt, const double* r2, double* v, MinresCtl* mc, PcgCtl* ctl,
                     int64_t* launches) {
  minres_v_kernel<<<nblk(nt, VT), VT, 0, st>>>(nt, r2, v, mc, ctl);
  ++*launches;
}

void launch_minres_alfa(cudaStream_t st, int nt, const double* v, double* y, const double* r1, MinresCtl* mc,
                        PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches) {
  minres_alfa_kernel<<<vec_blocks(nt), VT, 0, st>>>(nt, v, y, r1, mc, ctl, dotbuf, counter);
  ++*launches;
}

void launch_minres_beta(cudaStream_t st, int nt, const double* y, double* r1, double* r2, MinresCtl* mc, PcgCtl* ctl,
                        double* dotbuf, unsigned int* counter, int64_t* launches) {
  minres_beta_kernel<<<vec_blocks(nt), VT, 0, st>>>(nt, y, r1, r2, mc, ctl, dotbuf, counter);
  ++*launches;
}

void launch_minres_update(cudaStream_t st, int nt, const double* v, double* w, double* w1, double* w2, double* x,
                          const MinresCtl* mc, const PcgCtl* ctl, int64_t* launches) {
  minres_update_kernel<<<nblk(nt, VT), VT, 0, st>>>(nt, v, w, w1, w2, x, mc, ctl);
  ++*launches;
}

void launch_ctl_reset(cudaStream_t st, PcgCtl* dst, const PcgCtl* src, int max_iters, int64_t* launches) {
  ctl_reset_kernel<<<1, 32, 0, st>>>(dst, src, max_iters);
  ++*launches;
}

void launch_slack_grad_rhs(cudaStream_t st, int m, const double* dv, const double* dw, const double* gy,
                           const double* gv, const double* gw, double* delta, double* bt, int64_t* launches) {
  slack_grad_rhs_kernel<<<(m + VT - 1) / VT, VT, 0, st>>>(m, dv, dw, gy, gv, gw, delta, bt);
  if (launches) ++*launches;
}

void launch_slack_grad_out(cudaStream_t st, int m, const double* dv, const double* dw, const double* dy,
                           const double* gv, const double* gw, double* ov, double* ow, int64_t* launches) {
  slack_grad_out_kernel<<<(m + VT - 1) / VT, VT, 0, st>>>(m, dv, dw, dy, gv, gw, ov, ow);
  if (launches) ++*launches;
}

int pc_dense_coop_blocks() {
  static int blocks = -1;
  if (blocks < 0) {
    int dev = 0, coop = 0, per = 0;
    blocks = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pc_dense_d_coop_kernel, 256, 0) == cudaSuccess && per > 0)
      blocks = std::min(g_num_sms * std::min(per, 2), 512);   // the partial sums take 2 x blocks of dotbuf
    cudaGetLastError();
  }
  return blocks;
}

cudaError_t launch_pc_dense_d_coop(cudaStream_t st, int m, int d, const double* Bt, const double* Pinv,
                                   const double* B, double* rv, double* z, double* sd, double* part, int mode,
                                   PcgCtl* ctl, double* pf, double* ux, const double* Ap, int64_t* launches) {
  const int blocks = pc_dense_coop_blocks();
  if (blocks <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e =
      cudaLaunchKernelEx(&cfg, pc_dense_d_coop_kernel, m, d, Bt, Pinv, B, rv, z, sd, part, mode, ctl, pf, ux, Ap);
  if (e == cudaSuccess && launches) ++*launches;
  return e;
}

}  // namespace wc

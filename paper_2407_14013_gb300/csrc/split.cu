// The low-rank plus well-conditioned split of the scaling point (eq. EQSigdef, Section 3):
//   W = Q Lam Q^T + Qp Lamp Qp^T (top r eigenvalues in Lam), tau = lambda_{r+1}(W) / 2,
//   E = Q Q^T + tau^{-1} Qp Lamp Qp^T = Vs diag(e) Vs^T with e = [1 (r times), lamp / tau],
//   Sigma = diag(Lam (x)s Lam - tau^2 I, (Lam - tau I) (x) Lamp)^{-1},
// the rank rule r = argmax_{i <= r_hat} lambda_i / lambda_{i+1} and
// beta = (median eigenvalue of E)^2 of Section 7 (optionally times s_A = ||A||_F^2 / m).
// The eigenvalues of E are exactly the entries of e, so the median needs no eigensolve.
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

// One block per eigenpair i: its descending rank (ties broken by index), then the column move.
__global__ void split_sort_kernel(int n, const double* __restrict__ V, const double* __restrict__ lam,
                                  double* __restrict__ Vs, double* __restrict__ lam_s) {
  __shared__ double sh[32];
  __shared__ int rank_sh;
  const int i = blockIdx.x;
  const double li = lam[i];
  double cnt = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double lj = lam[j];
    cnt += (lj > li || (lj == li && j < i)) ? 1.0 : 0.0;
  }
  cnt = block_sum(cnt, sh);
  if (threadIdx.x == 0) rank_sh = (int)(cnt + 0.5);
  __syncthreads();
  const int rk = rank_sh;
  if (threadIdx.x == 0) lam_s[rk] = li;
  for (int a = threadIdx.x; a < n; a += blockDim.x) Vs[a + (int64_t)rk * n] = V[a + (int64_t)i * n];
}

__device__ double kth_largest_e(int n, int r, int c, const double* lam_s, double tau, int k) {
  // descending order of {1 (r times)} U {lam_s[r + q] / tau}: the c tail values > 1 come first
  if (k < c) return lam_s[r + k] / tau;
  if (k < c + r) return 1.0;
  return lam_s[k] / tau;   // tail index k - r, i.e. lam_s[r + (k - r)]
}

__global__ void split_params_kernel(int n, int r_fixed, int r_hat, int beta_rule,
                                    const double* __restrict__ lam_s, double* __restrict__ e,
                                    PcgCtl* __restrict__ ctl) {
  __shared__ double sh[32];
  __shared__ int r_sh;
  __shared__ int bad_sh;
  if (threadIdx.x == 0) {
    int bad = 0;
    int r = r_fixed;
    if (r <= 0) {
      int rh = r_hat < n - 1 ? r_hat : n - 1;
      double best = -1.0;
      r = 1;
      for (int i = 1; i <= rh; ++i) {
        double ratio = lam_s[i - 1] / lam_s[i];
        if (ratio > best) { best = ratio; r = i; }
      }
    }
    if (r < 1 || r >= n) bad = 1;
    r_sh = r;
    bad_sh = bad;
  }
  __syncthreads();
  // every eigenvalue must be positive and finite (W is positive definite)
  double nonpos = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double l = lam_s[k];
    nonpos += (l > 0.0 && l < INFINITY) ? 0.0 : 1.0;
  }
  nonpos = block_sum(nonpos, sh);
  if (bad_sh || nonpos > 0.0) {
    if (threadIdx.x == 0) { ctl->status = 1; ctl->r = 0; ctl->d = 0; }
    return;
  }
  const int r = r_sh;
  const double tau = 0.5 * lam_s[r];
  for (int k = threadIdx.x; k < n; k += blockDim.x) e[k] = (k < r) ? 1.0 : lam_s[k] / tau;
  double cgt = 0.0;
  for (int k = r + threadIdx.x; k < n; k += blockDim.x) cgt += (lam_s[k] / tau > 1.0) ? 1.0 : 0.0;
  cgt = block_sum(cgt, sh);
  if (threadIdx.x == 0) {
    const int c = (int)(cgt + 0.5);
    double med;
    if (n & 1) med = kth_largest_e(n, r, c, lam_s, tau, n / 2);
    else med = 0.5 * (kth_largest_e(n, r, c, lam_s, tau, n / 2 - 1) + kth_largest_e(n, r, c, lam_s, tau, n / 2));
    double beta = med * med;
    if (beta_rule == 0) beta *= ctl->s_A;
    ctl->r = r;
    ctl->d = n * r - r * (r - 1) / 2;
    ctl->tau = tau;
    ctl->beta_pc = beta;
    ctl->status = 0;
  }
}

__global__ void split_scale_cols_kernel(int n, const double* __restrict__ Vs, const double* __restrict__ e,
                                        double* __restrict__ Ve) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  Ve[q] = Vs[q] * e[q / n];
}

// D[h] = tau^2 Sigma[h] in h = [svec B; vec N] coordinates.
__global__ void split_sigma_kernel(int n, int r, const double* __restrict__ lam_s,
                                   const PcgCtl* __restrict__ ctl, double* __restrict__ Dv) {
  const int d = n * r - r * (r - 1) / 2;
  const int nb = r * (r + 1) / 2;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  const double tau = ctl->tau, t2 = tau * tau;
  if (h < nb) {
    int j = 0, base = 0;
    while (h >= base + (r - j)) { base += r - j; ++j; }
    int i = j + (h - base);
    Dv[h] = t2 / (lam_s[i] * lam_s[j] - t2);
  } else {
    int q = h - nb;
    int k = q % (n - r), j = q / (n - r);
    Dv[h] = t2 / ((lam_s[j] - tau) * lam_s[r + k]);
  }
}

}  // namespace

void split_sort(cudaStream_t st, int n, const double* V, const double* lam, double* Vs, double* lam_s,
                int64_t* launches) {
  split_sort_kernel<<<n, 256, 0, st>>>(n, V, lam, Vs, lam_s);
  if (launches) ++*launches;
}

void split_params(cudaStream_t st, int n, int r_fixed, int r_hat, int beta_rule, const double* lam_s,
                  double* e, PcgCtl* ctl, int64_t* launches) {
  split_params_kernel<<<1, 256, 0, st>>>(n, r_fixed, r_hat, beta_rule, lam_s, e, ctl);
  if (launches) ++*launches;
}

void split_scale_cols(cudaStream_t st, int n, const double* Vs, const double* e, double* Ve,
                      int64_t* launches) {
  int64_t tot = (int64_t)n * n;
  split_scale_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, Vs, e, Ve);
  if (launches) ++*launches;
}

void split_sigma(cudaStream_t st, int n, int r, const double* lam_s, const PcgCtl* ctl, double* Dv,
                 int64_t* launches) {
  int d = n * r - r * (r - 1) / 2;
  split_sigma_kernel<<<(d + 255) / 256, 256, 0, st>>>(n, r, lam_s, ctl, Dv);
  if (launches) ++*launches;
}

}  // namespace wc

// The outer primal-dual interior-point loop on the device: NT scaling, the Mehrotra
// predictor-corrector around two Newton solves on the well-conditioned reformulation, step
// lengths, and the stopping test.  The paper keeps an existing solver's outer loop unchanged
// (Section 7) and specifies it only through the log-barrier path and eq. newt; this file is
// the textbook method that the oracle also writes down (same definitions, same order):
//
//   measures   pobj = <C,X>, dobj = b^T y, rel_gap, pinf = ||b - A(X)||/(1+||b||),
//              dinf = ||C - A^T y - S||_F/(1+||C||_F), mu = <X,S>/n
//   NT scaling X = L L^T, L^T S L = U Gamma U^T, G = L U Gamma^{-1/4}, W = G G^T
//              (= L (L^T S L)^{-1/2} L^T of eq. newt); Lam = G^{-1} X G^{-T} = Gamma^{1/2}
//   predictor  (Newt-eps) with b~ = r_p, C~ = R_d + S  (R_c = -X);  dS = R_d - A^T(dy)
//   sigma      = min(1, (mu_aff / mu)^3), mu_aff from full predictor steps
//   corrector  Lam R + R Lam = 2 sigma mu I - 2 Lam^2 - (Dx Ds + Ds Dx), Dx = G^{-1} dX_a G^{-T},
//              Ds = G^T dS_a G;  C~ = R_d - G^{-T} R G^{-1}  (= R_d - W^{-1} R_c W^{-1})
//   steps      a = min(1, f * sup{a : Lam + a D PSD}) from the smallest eigenvalue of
//              Lam^{-1/2} D Lam^{-1/2}  (f = 1 for the predictor, 0.98 for the step)
//
// Every Newton direction is one sdp_newton_solve (the hot path); eig(W) for its split, eig of
// L^T S L and the smallest eigenvalues come from the Jacobi eigensolver (eigh.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <exception>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "kernels.h"
#include "pcg.h"

using namespace wc;

namespace wc {

struct IpmWork {
  int n = 0, m = 0;
  char* pool = nullptr;
  double *L = nullptr, *Linv = nullptr, *T = nullptr, *U = nullptr, *G = nullptr, *Ginv = nullptr, *Wm = nullptr;
  double *V = nullptr, *Rd = nullptr, *Ct = nullptr, *Y = nullptr, *dX = nullptr, *dS = nullptr, *dSs = nullptr;
  double *dXa = nullptr, *dSa = nullptr, *Dx = nullptr, *Ds = nullptr, *R = nullptr, *M1 = nullptr, *M2 = nullptr;
  double *Eg = nullptr, *EV = nullptr, *Vprev = nullptr, *Uprev = nullptr;
  bool have_prev = false;   // Vprev, Uprev hold the eigenvectors of the previous W and L^T S L
  double *lam = nullptr, *gam = nullptr, *g = nullptr, *q = nullptr, *qi = nullptr, *elam = nullptr;
  double *rp = nullptr, *dy = nullptr, *dya = nullptr, *Ax = nullptr, *rownrm = nullptr;
  double *zsvec = nullptr, *partY = nullptr, *partA = nullptr;
  double *eigw = nullptr, *chw = nullptr, *dots = nullptr, *dpart = nullptr, *lzw = nullptr;
  size_t eigw_elems = 0, chw_elems = 0, lzw_elems = 0;
  int32_t* status = nullptr;
  double xi = 0.0;
  EighGraph eg[2];   // Jacobi sweeps for L^T S L, and for W and the step-length matrices
  // slack variables of the robust form (sdp_solve_slack), allocated on first use
  double* lp_pool = nullptr;
  double *delta = nullptr, *rlv = nullptr, *rlw = nullptr, *ctv = nullptr, *ctw = nullptr, *btl = nullptr;
  double *dv = nullptr, *dw = nullptr, *dzv = nullptr, *dzw = nullptr;
  double *dva = nullptr, *dwa = nullptr, *dzva = nullptr, *dzwa = nullptr;
};

}  // namespace wc

namespace {

constexpr int IT = 256;
constexpr int kDotBlocks = 128;
constexpr int kDots = 32;

inline unsigned nb(int64_t total) { return (unsigned)((total + IT - 1) / IT); }

#define CUI(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return wc_fail(h, SDP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

__global__ void scaled_identity_kernel(int n, double xi, double* __restrict__ X) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < (int64_t)n * n) X[q] = ((q % n) == (q / n)) ? xi : 0.0;
}

// out = a * A + b * B (+ c * Cm), elementwise over `count`
__global__ void lincomb_kernel(int64_t count, double a, const double* __restrict__ A, double b,
                               const double* __restrict__ B, double c, const double* __restrict__ Cm,
                               double* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double v = a * A[q] + b * B[q];
  if (Cm) v += c * Cm[q];
  out[q] = v;
}

// X += alpha sym(D) (n x n), keeping X exactly symmetric
__global__ void sym_axpy_kernel(int n, double alpha, const double* __restrict__ D, double* __restrict__ X) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int i = (int)(q % n), j = (int)(q / n);
  if (i < j) return;
  const double d = 0.5 * (D[q] + D[j + (int64_t)i * n]);
  const double v = 0.5 * (X[q] + X[j + (int64_t)i * n]) + alpha * d;
  X[q] = v;
  X[j + (int64_t)i * n] = v;
}

__global__ void axpy_kernel(int count, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count) y[q] += alpha * x[q];
}

// rp = b - sum_s part[s * m + i]  (A(X) from the slab partials), or b - X_ii (DIAG: part = X, nslab < 0)
__global__ void rp_kernel(int m, int n, const double* __restrict__ b, const double* __restrict__ part, int nslab,
                          double* __restrict__ Ax, double* __restrict__ rp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double v = 0.0;
  if (nslab < 0) v = part[i + (int64_t)i * n];
  else
    for (int s = 0; s < nslab; ++s) v += part[(int64_t)s * m + i];
  Ax[i] = v;
  rp[i] = b[i] - v;
}

// gamma -> g = gamma^{1/2}, q = gamma^{-1/4}, qi = gamma^{1/4}
__global__ void gamma_kernel(int n, const double* __restrict__ gam, double* __restrict__ g, double* __restrict__ q,
                             double* __restrict__ qi, int32_t* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = gam[i];
  if (!(v > 0.0) || !isfinite(v)) {
    *status = 5;
    v = 1.0;
  }
  const double s = sqrt(v);
  g[i] = s;
  qi[i] = sqrt(s);
  q[i] = 1.0 / sqrt(s);
}

// out[i, j] = dl[i] * M[i, j] * dr[j]  (dl, dr may be NULL)
__global__ void scale_kernel(int n, const double* __restrict__ M, const double* __restrict__ dl,
                             const double* __restrict__ dr, double* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int i = (int)(q % n), j = (int)(q / n);
  double v = M[q];
  if (dl) v *= dl[i];
  if (dr) v *= dr[j];
  out[q] = v;
}

// out = I + s M
__global__ void shift_identity_kernel(int n, double s, const double* __restrict__ M, double* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  out[q] = s * M[q] + (((q % n) == (q / n)) ? 1.0 : 0.0);
}

// R_ij = rhs_ij / (g_i + g_j), rhs = 2 sigma mu I - 2 diag(g)^2 - (P + P^T)
__global__ void lyap_kernel(int n, double smu2, const double* __restrict__ g, const double* __restrict__ P,
                            double* __restrict__ R) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int i = (int)(q % n), j = (int)(q / n);
  double rhs = -(P[q] + P[j + (int64_t)i * n]);
  if (i == j) rhs += smu2 - 2.0 * g[i] * g[i];
  R[q] = rhs / (g[i] + g[j]);
}

// sum of a[k] * b[k] (b NULL: sum of a[k]^2) into per-block partials
__global__ void dot_partial_kernel(int64_t count, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[q], b ? b[q] : a[q], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void dot_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc += part[q];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

// squared norms of the svec rows (||A_i||_F^2), one warp per row
__global__ void row_sumsq_kernel(const double* __restrict__ A, int m, int64_t N, double* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= m) return;
  const double* row = A + (int64_t)w * N;
  double acc = 0.0;
  for (int64_t k = lane; k < N; k += 32) acc = fma(row[k], row[k], acc);
  acc = warp_sum(acc);
  if (lane == 0) out[w] = acc;
}

// ---- slack variables of the robust form: A(X) + v - w = b, v, w >= 0 (eq. rmc-sdp) ----

// rp -= v - w;  rlv = cv - y - zv;  rlw = cw + y - zw  (the dual constraints of v and w)
__global__ void slack_resid_kernel(int m, const double* __restrict__ v, const double* __restrict__ w,
                                   const double* __restrict__ y, const double* __restrict__ zv,
                                   const double* __restrict__ zw, const double* __restrict__ cv,
                                   const double* __restrict__ cw, double* __restrict__ rp, double* __restrict__ rlv,
                                   double* __restrict__ rlw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  rp[i] -= v[i] - w[i];
  rlv[i] = cv[i] - y[i] - zv[i];
  rlw[i] = cw[i] + y[i] - zw[i];
}

// delta = v / zv + w / zw  (diag(G D G^T) with G = [I, -I], D = diag(x / z))
__global__ void slack_delta_kernel(int m, const double* __restrict__ v, const double* __restrict__ w,
                                   const double* __restrict__ zv, const double* __restrict__ zw,
                                   double* __restrict__ delta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) delta[i] = v[i] / zv[i] + w[i] / zw[i];
}

// right side of the Newton system: r_x = smu - x z (- dx_a dz_a in the corrector),
// c~ = r_l - r_x / x, and b~ = r_p + G D c~ = r_p + d_v c~_v - d_w c~_w
__global__ void slack_rhs_kernel(int m, double smu, int corr, const double* __restrict__ v,
                                 const double* __restrict__ w, const double* __restrict__ zv,
                                 const double* __restrict__ zw, const double* __restrict__ dva,
                                 const double* __restrict__ dwa, const double* __restrict__ dzva,
                                 const double* __restrict__ dzwa, const double* __restrict__ rlv,
                                 const double* __restrict__ rlw, const double* __restrict__ rp,
                                 double* __restrict__ ctv, double* __restrict__ ctw, double* __restrict__ btl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double rxv = smu - v[i] * zv[i] - (corr ? dva[i] * dzva[i] : 0.0);
  const double rxw = smu - w[i] * zw[i] - (corr ? dwa[i] * dzwa[i] : 0.0);
  const double cv_ = rlv[i] - rxv / v[i], cw_ = rlw[i] - rxw / w[i];
  ctv[i] = cv_;
  ctw[i] = cw_;
  btl[i] = rp[i] + (v[i] / zv[i]) * cv_ - (w[i] / zw[i]) * cw_;
}

// dx = D (G^T dy - c~):  dv = d_v (dy - c~_v), dw = d_w (-dy - c~_w);  dz = r_l - G^T dy
__global__ void slack_dir_kernel(int m, const double* __restrict__ v, const double* __restrict__ w,
                                 const double* __restrict__ zv, const double* __restrict__ zw,
                                 const double* __restrict__ ctv, const double* __restrict__ ctw,
                                 const double* __restrict__ rlv, const double* __restrict__ rlw,
                                 const double* __restrict__ dy, double* __restrict__ dv, double* __restrict__ dw,
                                 double* __restrict__ dzv, double* __restrict__ dzw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  dv[i] = (v[i] / zv[i]) * (dy[i] - ctv[i]);
  dw[i] = (w[i] / zw[i]) * (-dy[i] - ctw[i]);
  dzv[i] = rlv[i] - dy[i];
  dzw[i] = rlw[i] + dy[i];
}

__device__ __forceinline__ double block_min(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : INFINITY;
  if (wid == 0)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// ratio test: min over i of -a_i / da_i (da_i < 0) and -b_i / db_i (db_i < 0), per block
__global__ void ratio_partial_kernel(int m, const double* __restrict__ a, const double* __restrict__ da,
                                     const double* __restrict__ b, const double* __restrict__ db,
                                     double* __restrict__ part) {
  __shared__ double sh[32];
  double r = INFINITY;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (da[i] < 0.0) r = fmin(r, -a[i] / da[i]);
    if (db[i] < 0.0) r = fmin(r, -b[i] / db[i]);
  }
  r = block_min(r, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void min_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double sh[32];
  double r = INFINITY;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) r = fmin(r, part[q]);
  r = block_min(r, sh);
  if (threadIdx.x == 0) *out = r;
}

// sum of (v + ap dv)(zv + ad dzv) + (w + ap dw)(zw + ad dzw), per block
__global__ void slack_muaff_kernel(int m, double ap, double ad, const double* __restrict__ v,
                                   const double* __restrict__ dv, const double* __restrict__ zv,
                                   const double* __restrict__ dzv, const double* __restrict__ w,
                                   const double* __restrict__ dw, const double* __restrict__ zw,
                                   const double* __restrict__ dzw, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    acc += (v[i] + ap * dv[i]) * (zv[i] + ad * dzv[i]) + (w[i] + ap * dw[i]) * (zw[i] + ad * dzw[i]);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void fill_kernel(int m, double val, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) x[i] = val;
}

struct Ctx {
  sdp_handle* h;
  IpmWork* w;
  int n, m;
  cudaStream_t st;
  int64_t* L;
  double gap_tol = 1e-8;   // the stop test of the loop; also bounds the residual of a usable direction
};

cudaError_t gemm(Ctx& c, bool tA, bool tB, const double* A, const double* B, double* C, double alpha = 1.0,
                 double beta = 0.0) {
  const int n = c.n;
  return gemm_f64(c.st, tA, tB, n, n, n, alpha, A, n, B, n, beta, C, n, c.h->s64.ws, c.h->s64.ws_elems, c.L);
}

void dot(Ctx& c, int64_t count, const double* a, const double* b, int slot) {
  dot_partial_kernel<<<kDotBlocks, IT, 0, c.st>>>(count, a, b, c.w->dpart + slot * kDotBlocks);
  dot_final_kernel<<<1, IT, 0, c.st>>>(c.w->dpart + slot * kDotBlocks, kDotBlocks, c.w->dots + slot);
  *c.L += 2;
}

// Y = A^T(y) as a full matrix
void adjoint(Ctx& c, const double* y, double* Y) {
  sdp_handle* h = c.h;
  if (h->kind == SDP_A_DENSE_SVEC) {
    rows_gemvT<double>(c.st, h->a_dense, c.m, h->N, y, c.w->partY, h->GY, nullptr, c.L);
    svec_unpack_sum<double>(c.st, c.n, c.w->partY, h->GY, 1.0, Y, nullptr, c.L);
  } else if (h->kind == SDP_A_SPARSE_COO) {
    sparse_adjoint(c.st, h->sp, c.n, y, 1.0, Y, nullptr, c.L);   // Y is zero off the pattern
  } else {
    launch_diag_matrix(c.st, c.n, y, Y, c.L);
  }
}

// Ax = A(X) (X symmetric, lower triangle read) and rp = b - Ax
void residual_p(Ctx& c, const double* b, const double* X) {
  sdp_handle* h = c.h;
  if (h->kind == SDP_A_DENSE_SVEC) {
    svec_pack_plus<double>(c.st, c.n, 0, X, nullptr, nullptr, c.w->zsvec, nullptr, c.L);
    rows_gemv<double>(c.st, h->a_dense, c.m, h->N, c.w->zsvec, c.w->partA, nullptr, c.L);
    rp_kernel<<<nb(c.m), IT, 0, c.st>>>(c.m, c.n, b, c.w->partA, rows_gemv_slabs(c.m, h->N), c.w->Ax, c.w->rp);
  } else if (h->kind == SDP_A_SPARSE_COO) {
    sparse_apply(c.st, h->sp, c.n, c.m, 0, X, nullptr, nullptr, c.w->partA, nullptr, c.L);
    rp_kernel<<<nb(c.m), IT, 0, c.st>>>(c.m, c.n, b, c.w->partA, 1, c.w->Ax, c.w->rp);
  } else {
    rp_kernel<<<nb(c.m), IT, 0, c.st>>>(c.m, c.n, b, X, -1, c.w->Ax, c.w->rp);
  }
  ++*c.L;
}

// smallest eigenvalue of the symmetric M (copied; M is kept)
// smallest eigenvalue of the symmetric M by the Jacobi eigensolver (all eigenvalues)
sdp_status lam_min_jacobi(Ctx& c, const double* M, double* out, int* sweeps) {
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const size_t nn = (size_t)c.n * c.n;
  CUI(cudaMemcpyAsync(w->Eg, M, nn * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  int sw = 0;
  double off = 0.0;
  CUI(eigh_jacobi(c.st, c.n, w->Eg, w->EV, w->elam, 1e-12, 40, w->eigw, w->eigw_elems, &sw, &off, c.L, &w->eg[1], !h->no_coop));
  *sweeps += sw;
  std::vector<double> lh(c.n);
  CUI(cudaMemcpyAsync(lh.data(), w->elam, c.n * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  *out = *std::min_element(lh.begin(), lh.end());
  return SDP_OK;
}

// smallest eigenvalue of M by Lanczos (one block per launch in batched solves)
sdp_status lam_min(Ctx& c, const double* M, double* out, int* sweeps) {
  (void)sweeps;
  sdp_handle* h = c.h;
  int it = 0;
  CUI(lanczos_min(c.st, c.n, M, c.w->lzw, c.w->lzw_elems, out, &it, c.L, !h->no_coop));
  return SDP_OK;
}

// sup{a : Lam + a D PSD} for D = Dx or Ds, through Lam^{-1/2} D Lam^{-1/2} (Lam^{-1/2} = diag(q)).
// The caller uses min(1, f sup); when I + M / f is positive definite (a Cholesky factorisation
// succeeds) that is 1 and the eigenvalue is not needed, so +inf is returned.
sdp_status max_step(Ctx& c, const double* D, double f, double* a, int* sweeps) {
  NvtxRange nvtx_range("ipm step length");
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int64_t nn = (int64_t)c.n * c.n;
  scale_kernel<<<nb(nn), IT, 0, c.st>>>(c.n, D, w->q, w->q, w->M2);
  shift_identity_kernel<<<nb(nn), IT, 0, c.st>>>(c.n, 1.0 / f, w->M2, w->Eg);   // Eg = I + M / f
  *c.L += 2;
  CUI(cudaMemsetAsync(w->status, 0, sizeof(int32_t), c.st));
  CUI(spd_cholesky(c.st, c.n, w->Eg, nullptr, w->chw, w->chw_elems, h->s64.ws, h->s64.ws_elems, w->status, c.L,
                   !h->no_coop));
  int32_t st_h = 0;
  CUI(cudaMemcpyAsync(&st_h, w->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  if (st_h == 0) {
    *a = INFINITY;
    return SDP_OK;
  }
  double lmin = 0.0;
  sdp_status s = lam_min(c, w->M2, &lmin, sweeps);
  if (s != SDP_OK) return s;
  *a = (lmin >= 0.0) ? INFINITY : -1.0 / lmin;
  if (f < 1.0 && std::isfinite(*a) && f * *a < 1.0) {
    // the step taken is f a: check that I + f a M is positive definite, else recompute lambda_min
    // with the Jacobi eigensolver
    shift_identity_kernel<<<nb(nn), IT, 0, c.st>>>(c.n, f * *a, w->M2, w->Eg);
    ++*c.L;
    CUI(cudaMemsetAsync(w->status, 0, sizeof(int32_t), c.st));
    CUI(spd_cholesky(c.st, c.n, w->Eg, nullptr, w->chw, w->chw_elems, h->s64.ws, h->s64.ws_elems, w->status, c.L,
                   !h->no_coop));
    int32_t ok = 0;
    CUI(cudaMemcpyAsync(&ok, w->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    CUI(cudaStreamSynchronize(c.st));
    if (ok != 0) {
      s = lam_min_jacobi(c, w->M2, &lmin, sweeps);
      if (s != SDP_OK) return s;
      *a = (lmin >= 0.0) ? INFINITY : -1.0 / lmin;
    }
  }
  return SDP_OK;
}

// Newton direction at the current scaling point; `again` reuses the split and preconditioner of
// the previous call (the corrector has the predictor's scaling point)
sdp_status newton(Ctx& c, const double* Ct, const double* bt, double* dX, double* dy, double* dSs, sdp_ipm_info* info,
                  bool again = false) {
  sdp_newton_info ni;
  std::memset(&ni, 0, sizeof(ni));
  sdp_status s = again ? sdp_newton_resolve(c.h, Ct, bt, dX, dy, dSs, &ni)
                       : sdp_newton_solve(c.h, c.w->V, c.w->lam, Ct, bt, dX, dy, dSs, &ni);
  info->pcg_iters += ni.pcg_iters;
  info->newton_ms += ni.setup_ms + ni.pcg_ms + ni.recover_ms;
  if (s == SDP_ENOTCONV) {
    // PCG stopped at max_pcg.  The direction is used only when its (Newt-eps) residual is already
    // below a tenth of the loop's tolerance relative to the right side (Lemma smallres: ||r_k||
    // is that residual), so that stepping on it cannot move the iterate's residuals past the
    // stop test; otherwise the loop stops here and the caller keeps the last iterate.
    if (ni.res_norm <= 0.1 * c.gap_tol * ni.rhs_norm) {
      info->newton_inexact += 1;
      return SDP_OK;
    }
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "Newton direction not converged (PCG at max_pcg, residual %.3g of the right side): stopped at "
                  "the last iterate", ni.rhs_norm > 0.0 ? ni.res_norm / ni.rhs_norm : ni.res_norm);
    return wc_fail(c.h, SDP_ENOTCONV, msg);
  }
  return s;
}

sdp_status ensure_workspace(sdp_handle* h) {
  if (h->ipm) return SDP_OK;
  IpmWork* w = new (std::nothrow) IpmWork();
  if (!w) return wc_fail(h, SDP_ENOMEM, "host allocation failed");
  const int n = h->n, m = h->m;
  const size_t nn = (size_t)n * n;
  w->n = n;
  w->m = m;
  w->eigw_elems = eigh_work_elems(n);
  w->chw_elems = spd_inverse_work(n);
  w->lzw_elems = lanczos_work_elems(n);
  size_t off = 0;
  auto take = [&](size_t count) {
    off = (off + 31) & ~size_t(31);
    size_t at = off;
    off += count;
    return at;
  };
  std::vector<std::pair<double**, size_t>> plan = {
      {&w->L, nn}, {&w->Linv, nn}, {&w->T, nn}, {&w->U, nn}, {&w->G, nn}, {&w->Ginv, nn}, {&w->Wm, nn},
      {&w->V, nn}, {&w->Rd, nn}, {&w->Ct, nn}, {&w->Y, nn}, {&w->dX, nn}, {&w->dS, nn}, {&w->dSs, nn},
      {&w->dXa, nn}, {&w->dSa, nn}, {&w->Dx, nn}, {&w->Ds, nn}, {&w->R, nn}, {&w->M1, nn}, {&w->M2, nn},
      {&w->Eg, nn}, {&w->EV, nn}, {&w->Vprev, nn}, {&w->Uprev, nn}, {&w->lam, (size_t)n}, {&w->gam, (size_t)n}, {&w->g, (size_t)n},
      {&w->q, (size_t)n}, {&w->qi, (size_t)n}, {&w->elam, (size_t)n}, {&w->rp, (size_t)m}, {&w->dy, (size_t)m},
      {&w->dya, (size_t)m}, {&w->Ax, (size_t)m}, {&w->rownrm, (size_t)m}, {&w->eigw, w->eigw_elems},
      {&w->chw, w->chw_elems}, {&w->lzw, w->lzw_elems}, {&w->dots, (size_t)kDots}, {&w->dpart, (size_t)kDots * kDotBlocks}};
  if (h->kind == SDP_A_DENSE_SVEC) {
    plan.push_back({&w->zsvec, (size_t)h->N});
    plan.push_back({&w->partY, (size_t)h->GY * h->N});
    plan.push_back({&w->partA, rows_gemv_part_elems(m, h->N)});
  } else if (h->kind == SDP_A_SPARSE_COO) {
    plan.push_back({&w->partA, (size_t)m});
  }
  std::vector<size_t> at;
  for (auto& p : plan) at.push_back(take(p.second));
  const size_t status_at = take(1);
  const size_t total = off * sizeof(double) + 256;
  cudaError_t e = cudaMalloc(&w->pool, total);
  if (e != cudaSuccess) {
    delete w;
    return wc_fail(h, SDP_ENOMEM, std::string("cudaMalloc of the interior-point workspace failed: ") +
                                      cudaGetErrorString(e));
  }
  double* base = reinterpret_cast<double*>(w->pool);
  for (size_t k = 0; k < plan.size(); ++k) *plan[k].first = base + at[k];
  w->status = reinterpret_cast<int32_t*>(base + status_at);
  // A^T(y) of the SPARSE_COO kind writes only the pattern: the rest of Y stays zero
  e = cudaMemsetAsync(w->Y, 0, nn * sizeof(double), h->st);
  if (e != cudaSuccess) {
    cudaFree(w->pool);
    delete w;
    return wc_fail(h, SDP_ECUDA, std::string("clearing the interior-point workspace failed: ") +
                                     cudaGetErrorString(e));
  }
  h->ipm = w;
  return SDP_OK;
}

struct Measures {
  double pobj, dobj, gap, pinf, dinf, mu, nb, nc;
};

// R_d = C - A^T(y) - S, r_p = b - A(X), and the measures (one host read)
sdp_status residuals(Ctx& c, const double* b, const double* C, const double* X, const double* y, const double* S,
                     Measures* M) {
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int64_t nn = (int64_t)c.n * c.n;
  adjoint(c, y, w->Y);
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, C, -1.0, w->Y, -1.0, S, w->Rd);
  ++*c.L;
  residual_p(c, b, X);
  dot(c, nn, C, X, 0);
  dot(c, c.m, b, y, 1);
  dot(c, c.m, w->rp, nullptr, 2);
  dot(c, nn, w->Rd, nullptr, 3);
  dot(c, nn, X, S, 4);
  dot(c, c.m, b, nullptr, 5);
  dot(c, nn, C, nullptr, 6);
  double d[7];
  CUI(cudaMemcpyAsync(d, w->dots, 7 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  M->pobj = d[0];
  M->dobj = d[1];
  M->gap = std::fabs(d[0] - d[1]) / (1.0 + std::fabs(d[0]) + std::fabs(d[1]));
  M->nb = std::sqrt(d[5]);
  M->nc = std::sqrt(d[6]);
  M->pinf = std::sqrt(d[2]) / (1.0 + M->nb);
  M->dinf = std::sqrt(d[3]) / (1.0 + M->nc);
  M->mu = d[4] / c.n;
  return SDP_OK;
}

void fill_info(sdp_ipm_info* info, const Measures& M) {
  info->pobj = M.pobj;
  info->dobj = M.dobj;
  info->rel_gap = M.gap;
  info->pinf = M.pinf;
  info->dinf = M.dinf;
  info->mu = M.mu;
}

// one predictor-corrector step from (X, y, S) whose residuals w->Rd, w->rp and measures M
// are current
// NT scaling of (X, S) (Section 3, eq. newt): X = L L^T, L^T S L = U Gamma U^T,
// G = L U Gamma^{-1/4}, W = G G^T, and eig(W) = (V, lam).  Both eigen-decompositions start from
// the previous call's eigenvectors when there are any (the iterates move little along the path).
sdp_status scaling(Ctx& c, const double* X, const double* S, int* sweeps) {
  NvtxRange nvtx_range("ipm scaling point (eigen-decompositions)");
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int n = c.n;
  const int64_t nn = (int64_t)n * n;
  const size_t bytes = (size_t)nn * sizeof(double);
  double off = 0.0;
  // ---- NT scaling: X = L L^T, L^T S L = U Gamma U^T, G = L U Gamma^{-1/4}, W = G G^T
  CUI(cudaMemsetAsync(w->status, 0, sizeof(int32_t), c.st));
  CUI(cudaMemcpyAsync(w->L, X, bytes, cudaMemcpyDeviceToDevice, c.st));
  CUI(spd_cholesky(c.st, n, w->L, w->Linv, w->chw, w->chw_elems, h->s64.ws, h->s64.ws_elems, w->status, c.L,
                   !h->no_coop));
  CUI(gemm(c, false, false, S, w->L, w->M1));
  CUI(gemm(c, true, false, w->L, w->M1, w->T));
  int sw = 0;
  // eig(L^T S L), started like eig(W) below from the previous iteration's eigenvectors
  if (w->have_prev) {
    CUI(gemm(c, false, false, w->T, w->Uprev, w->M1));
    CUI(gemm(c, true, false, w->Uprev, w->M1, w->T));
  }
  CUI(eigh_jacobi(c.st, n, w->T, w->U, w->gam, 1e-14, 40, w->eigw, w->eigw_elems, &sw, &off, c.L, &w->eg[0], !h->no_coop));
  *sweeps += sw;
  if (w->have_prev) {
    CUI(gemm(c, false, false, w->Uprev, w->U, w->M1));
    CUI(cudaMemcpyAsync(w->U, w->M1, bytes, cudaMemcpyDeviceToDevice, c.st));
  }
  CUI(cudaMemcpyAsync(w->Uprev, w->U, bytes, cudaMemcpyDeviceToDevice, c.st));
  gamma_kernel<<<nb(n), IT, 0, c.st>>>(n, w->gam, w->g, w->q, w->qi, w->status);
  ++*c.L;
  CUI(gemm(c, false, false, w->L, w->U, w->M1));
  scale_kernel<<<nb(nn), IT, 0, c.st>>>(n, w->M1, nullptr, w->q, w->G);          // G = L U Gamma^{-1/4}
  CUI(gemm(c, true, false, w->U, w->Linv, w->M1));
  scale_kernel<<<nb(nn), IT, 0, c.st>>>(n, w->M1, w->qi, nullptr, w->Ginv);      // G^{-1} = Gamma^{1/4} U^T L^{-1}
  *c.L += 2;
  CUI(gemm(c, false, true, w->G, w->G, w->Wm));                                  // W = G G^T
  // eig(W), started from the previous iteration's eigenvectors when there are any: Jacobi on
  // Vprev^T W Vprev (nearly diagonal along the path), then V = Vprev V'
  if (w->have_prev) {
    CUI(gemm(c, false, false, w->Wm, w->Vprev, w->M1));
    CUI(gemm(c, true, false, w->Vprev, w->M1, w->Eg));
  } else {
    CUI(cudaMemcpyAsync(w->Eg, w->Wm, bytes, cudaMemcpyDeviceToDevice, c.st));
  }
  CUI(eigh_jacobi(c.st, n, w->Eg, w->EV, w->lam, 1e-14, 40, w->eigw, w->eigw_elems, &sw, &off, c.L, &w->eg[1], !h->no_coop));
  *sweeps += sw;
  if (w->have_prev) CUI(gemm(c, false, false, w->Vprev, w->EV, w->V));
  else CUI(cudaMemcpyAsync(w->V, w->EV, bytes, cudaMemcpyDeviceToDevice, c.st));
  CUI(cudaMemcpyAsync(w->Vprev, w->V, bytes, cudaMemcpyDeviceToDevice, c.st));
  w->have_prev = true;
  int32_t st_h = 0;
  CUI(cudaMemcpyAsync(&st_h, w->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  if (st_h != 0) return wc_fail(h, SDP_ENUMERIC, "X is not positive definite or L^T S L is singular");
  return SDP_OK;
}

sdp_status step(Ctx& c, double* X, double* y, double* S, const Measures& Mz, sdp_ipm_info* info) {
  NvtxRange nvtx_range("ipm predictor-corrector step");
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int n = c.n;
  const int64_t nn = (int64_t)n * n;
  const size_t bytes = (size_t)nn * sizeof(double);
  const double mu = Mz.mu;
  int sweeps = 0;
  double off = 0.0;
  sdp_status s0 = scaling(c, X, S, &sweeps);
  if (s0 != SDP_OK) return s0;

  // ---- predictor: C~ = R_d + S, b~ = r_p
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->Rd, 1.0, S, 0.0, nullptr, w->Ct);
  ++*c.L;
  sdp_status s = newton(c, w->Ct, w->rp, w->dXa, w->dya, w->dSs, info);
  if (s != SDP_OK) return s;
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->dSs, -1.0, S, 0.0, nullptr, w->dSa);   // R_d - A^T dy
  ++*c.L;
  CUI(gemm(c, false, false, w->Ginv, w->dXa, w->M1));
  CUI(gemm(c, false, true, w->M1, w->Ginv, w->Dx));                              // Dx = G^{-1} dX G^{-T}
  CUI(gemm(c, true, false, w->G, w->dSa, w->M1));
  CUI(gemm(c, false, false, w->M1, w->G, w->Ds));                                // Ds = G^T dS G
  double ap = 0.0, ad = 0.0;
  s = max_step(c, w->Dx, 1.0, &ap, &sweeps);
  if (s != SDP_OK) return s;
  s = max_step(c, w->Ds, 1.0, &ad, &sweeps);
  if (s != SDP_OK) return s;
  ap = std::min(1.0, ap);
  ad = std::min(1.0, ad);
  // mu_aff = <X + ap dX, S + ad dS> / n
  dot(c, nn, X, w->dSa, 7);
  dot(c, nn, w->dXa, S, 8);
  dot(c, nn, w->dXa, w->dSa, 9);
  double d3[3];
  CUI(cudaMemcpyAsync(d3, w->dots + 7, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  const double mu_aff = (mu * n + ad * d3[0] + ap * d3[1] + ap * ad * d3[2]) / n;
  const double sigma = std::min(1.0, std::pow(mu_aff / mu, 3.0));

  // ---- corrector: Lam R + R Lam = 2 sigma mu I - 2 Lam^2 - (Dx Ds + Ds Dx)
  CUI(gemm(c, false, false, w->Dx, w->Ds, w->M1));
  lyap_kernel<<<nb(nn), IT, 0, c.st>>>(n, 2.0 * sigma * mu, w->g, w->M1, w->R);
  ++*c.L;
  CUI(gemm(c, false, false, w->R, w->Ginv, w->M1));
  CUI(gemm(c, true, false, w->Ginv, w->M1, w->M2));                             // G^{-T} R G^{-1}
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->Rd, -1.0, w->M2, 0.0, nullptr, w->Ct);
  ++*c.L;
  CUI(cudaMemcpyAsync(w->T, w->M2, bytes, cudaMemcpyDeviceToDevice, c.st));    // keep G^{-T} R G^{-1}
  s = newton(c, w->Ct, w->rp, w->dX, w->dy, w->dSs, info, true);
  if (s != SDP_OK) return s;
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->dSs, 1.0, w->T, 0.0, nullptr, w->dS);  // R_d - A^T dy
  ++*c.L;
  CUI(gemm(c, false, false, w->Ginv, w->dX, w->M1));
  CUI(gemm(c, false, true, w->M1, w->Ginv, w->Dx));
  CUI(gemm(c, true, false, w->G, w->dS, w->M1));
  CUI(gemm(c, false, false, w->M1, w->G, w->Ds));
  s = max_step(c, w->Dx, 0.98, &ap, &sweeps);
  if (s != SDP_OK) return s;
  s = max_step(c, w->Ds, 0.98, &ad, &sweeps);
  if (s != SDP_OK) return s;
  ap = std::min(1.0, 0.98 * ap);
  ad = std::min(1.0, 0.98 * ad);
  sym_axpy_kernel<<<nb(nn), IT, 0, c.st>>>(n, ap, w->dX, X);
  sym_axpy_kernel<<<nb(nn), IT, 0, c.st>>>(n, ad, w->dS, S);
  axpy_kernel<<<nb(c.m), IT, 0, c.st>>>(c.m, ad, w->dy, y);
  *c.L += 3;
  CUI(cudaGetLastError());
  info->alpha_p = ap;
  info->alpha_d = ad;
  info->sigma = sigma;
  info->eig_sweeps += sweeps;
  return SDP_OK;
}

// start X = S = xi I, y = 0, xi = max(10, sqrt n, max_i (1+|b_i|)/(1+||A_i||_F), (1+||C||_F)/sqrt n)
sdp_status start(Ctx& c, const double* b, const double* C, double* X, double* y, double* S) {
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int n = c.n, m = c.m;
  std::vector<double> bh(m), rn(m, 1.0);
  CUI(cudaMemcpyAsync(bh.data(), b, m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (h->kind == SDP_A_DENSE_SVEC) {
    row_sumsq_kernel<<<(unsigned)((m * 32 + IT - 1) / IT), IT, 0, h->st>>>(h->a_dense, m, h->N, w->rownrm);
    CUI(cudaMemcpyAsync(rn.data(), w->rownrm, m * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  }
  dot(c, (int64_t)n * n, C, nullptr, 6);
  double cc = 0.0;
  CUI(cudaMemcpyAsync(&cc, w->dots + 6, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CUI(cudaStreamSynchronize(h->st));
  double xi = std::max(10.0, std::sqrt((double)n));
  for (int i = 0; i < m; ++i) {
    const double an = (h->kind == SDP_A_DENSE_SVEC) ? std::sqrt(rn[i])
                      : (h->kind == SDP_A_SPARSE_COO) ? std::sqrt(h->sp_rownorm2[i]) : 1.0;
    xi = std::max(xi, (1.0 + std::fabs(bh[i])) / (1.0 + an));
  }
  xi = std::max(xi, (1.0 + std::sqrt(cc)) / std::sqrt((double)n));
  w->xi = xi;
  w->have_prev = false;
  scaled_identity_kernel<<<nb((int64_t)n * n), IT, 0, h->st>>>(n, xi, X);
  scaled_identity_kernel<<<nb((int64_t)n * n), IT, 0, h->st>>>(n, xi, S);
  *c.L += 2;
  CUI(cudaMemsetAsync(y, 0, m * sizeof(double), h->st));
  return SDP_OK;
}

// ---- the robust form with slacks: A(X) + v - w = b, v, w >= 0, costs cv, cw (eq. rmc-sdp) ----

struct Slack {
  double *v, *w, *zv, *zw;
  const double *cv, *cw;
  double xz;   // v^T zv + w^T zw
  double xs;   // <X, S>
};

sdp_status ensure_slack_workspace(sdp_handle* h) {
  IpmWork* w = h->ipm;
  if (w->lp_pool) return SDP_OK;
  const size_t m = (size_t)h->m, mp = (m + 31) & ~size_t(31);
  double* pool = nullptr;
  cudaError_t e = cudaMalloc(&pool, 14 * mp * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return wc_fail(h, SDP_ENOMEM, std::string("slack workspace: ") + cudaGetErrorString(e));
  }
  w->lp_pool = pool;
  double** bufs[14] = {&w->delta, &w->rlv, &w->rlw, &w->ctv, &w->ctw, &w->btl, &w->dv,
                       &w->dw,    &w->dzv, &w->dzw, &w->dva, &w->dwa, &w->dzva, &w->dzwa};
  for (int k = 0; k < 14; ++k) *bufs[k] = pool + k * mp;
  return SDP_OK;
}

// the slack terms of the residuals and measures (after residuals(): w->rp = b - A(X), w->Rd)
sdp_status slack_measures(Ctx& c, const double* y, Slack& sl, Measures* M) {
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int m = c.m;
  const double rd2 = std::pow(M->dinf * (1.0 + M->nc), 2.0);
  const double xs = M->mu * c.n;
  slack_resid_kernel<<<nb(m), IT, 0, c.st>>>(m, sl.v, sl.w, y, sl.zv, sl.zw, sl.cv, sl.cw, w->rp, w->rlv, w->rlw);
  ++*c.L;
  dot(c, m, w->rp, nullptr, 16);
  dot(c, m, sl.cv, sl.v, 17);
  dot(c, m, sl.cw, sl.w, 18);
  dot(c, m, w->rlv, nullptr, 19);
  dot(c, m, w->rlw, nullptr, 20);
  dot(c, m, sl.v, sl.zv, 21);
  dot(c, m, sl.w, sl.zw, 22);
  dot(c, m, sl.cv, nullptr, 23);
  dot(c, m, sl.cw, nullptr, 24);
  double d[9];
  CUI(cudaMemcpyAsync(d, w->dots + 16, 9 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  M->pobj += d[1] + d[2];
  M->gap = std::fabs(M->pobj - M->dobj) / (1.0 + std::fabs(M->pobj) + std::fabs(M->dobj));
  M->pinf = std::sqrt(d[0]) / (1.0 + M->nb);
  M->dinf = std::sqrt(rd2 + d[3] + d[4]) / (1.0 + M->nc + std::sqrt(d[7] + d[8]));
  sl.xs = xs;
  sl.xz = d[5] + d[6];
  M->mu = (xs + sl.xz) / (c.n + 2.0 * m);
  return SDP_OK;
}

// sup{a : x + a dx >= 0} over two vector pairs
sdp_status ratio_step(Ctx& c, const double* a, const double* da, const double* b, const double* db, double* out) {
  sdp_handle* h = c.h;
  ratio_partial_kernel<<<kDotBlocks, IT, 0, c.st>>>(c.m, a, da, b, db, c.w->dpart + 25 * kDotBlocks);
  min_final_kernel<<<1, IT, 0, c.st>>>(c.w->dpart + 25 * kDotBlocks, kDotBlocks, c.w->dots + 25);
  *c.L += 2;
  CUI(cudaMemcpyAsync(out, c.w->dots + 25, sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  return SDP_OK;
}

// one predictor-corrector step of the robust form (the method of step() with the orthant)
sdp_status step_slack(Ctx& c, double* X, double* y, double* S, Slack& sl, const Measures& Mz, sdp_ipm_info* info) {
  sdp_handle* h = c.h;
  IpmWork* w = c.w;
  const int n = c.n, m = c.m;
  const int64_t nn = (int64_t)n * n;
  const size_t bytes = (size_t)nn * sizeof(double);
  const double mu = Mz.mu;
  int sweeps = 0;
  sdp_status s0 = scaling(c, X, S, &sweeps);
  if (s0 != SDP_OK) return s0;
  slack_delta_kernel<<<nb(m), IT, 0, c.st>>>(m, sl.v, sl.w, sl.zv, sl.zw, w->delta);   // the linear block
  ++*c.L;

  // ---- predictor: C~ = R_d + S (R_c = -X), r_x = -x z
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->Rd, 1.0, S, 0.0, nullptr, w->Ct);
  slack_rhs_kernel<<<nb(m), IT, 0, c.st>>>(m, 0.0, 0, sl.v, sl.w, sl.zv, sl.zw, nullptr, nullptr, nullptr, nullptr,
                                           w->rlv, w->rlw, w->rp, w->ctv, w->ctw, w->btl);
  *c.L += 2;
  sdp_status s = newton(c, w->Ct, w->btl, w->dXa, w->dya, w->dSs, info);
  if (s != SDP_OK) return s;
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->dSs, -1.0, S, 0.0, nullptr, w->dSa);   // R_d - A^T dy
  slack_dir_kernel<<<nb(m), IT, 0, c.st>>>(m, sl.v, sl.w, sl.zv, sl.zw, w->ctv, w->ctw, w->rlv, w->rlw, w->dya,
                                           w->dva, w->dwa, w->dzva, w->dzwa);
  *c.L += 2;
  CUI(gemm(c, false, false, w->Ginv, w->dXa, w->M1));
  CUI(gemm(c, false, true, w->M1, w->Ginv, w->Dx));                              // Dx = G^{-1} dX G^{-T}
  CUI(gemm(c, true, false, w->G, w->dSa, w->M1));
  CUI(gemm(c, false, false, w->M1, w->G, w->Ds));                                // Ds = G^T dS G
  double ap = 0.0, ad = 0.0, rp_ = 0.0, rd_ = 0.0;
  s = max_step(c, w->Dx, 1.0, &ap, &sweeps);
  if (s != SDP_OK) return s;
  s = max_step(c, w->Ds, 1.0, &ad, &sweeps);
  if (s != SDP_OK) return s;
  s = ratio_step(c, sl.v, w->dva, sl.w, w->dwa, &rp_);
  if (s != SDP_OK) return s;
  s = ratio_step(c, sl.zv, w->dzva, sl.zw, w->dzwa, &rd_);
  if (s != SDP_OK) return s;
  ap = std::min({1.0, ap, rp_});
  ad = std::min({1.0, ad, rd_});
  // mu_aff = (<X + ap dX, S + ad dS> + (x + ap dx)^T (z + ad dz)) / (n + 2m)
  dot(c, nn, X, w->dSa, 7);
  dot(c, nn, w->dXa, S, 8);
  dot(c, nn, w->dXa, w->dSa, 9);
  slack_muaff_kernel<<<kDotBlocks, IT, 0, c.st>>>(m, ap, ad, sl.v, w->dva, sl.zv, w->dzva, sl.w, w->dwa, sl.zw,
                                                  w->dzwa, w->dpart + 10 * kDotBlocks);
  dot_final_kernel<<<1, IT, 0, c.st>>>(w->dpart + 10 * kDotBlocks, kDotBlocks, w->dots + 10);
  *c.L += 2;
  double d4[4];
  CUI(cudaMemcpyAsync(d4, w->dots + 7, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CUI(cudaStreamSynchronize(c.st));
  const double mu_aff = (sl.xs + ad * d4[0] + ap * d4[1] + ap * ad * d4[2] + d4[3]) / (n + 2.0 * m);
  const double sigma = std::min(1.0, std::pow(mu_aff / mu, 3.0));

  // ---- corrector: Lam R + R Lam = 2 sigma mu I - 2 Lam^2 - (Dx Ds + Ds Dx);
  //      r_x = sigma mu - x z - dx_a dz_a
  CUI(gemm(c, false, false, w->Dx, w->Ds, w->M1));
  lyap_kernel<<<nb(nn), IT, 0, c.st>>>(n, 2.0 * sigma * mu, w->g, w->M1, w->R);
  ++*c.L;
  CUI(gemm(c, false, false, w->R, w->Ginv, w->M1));
  CUI(gemm(c, true, false, w->Ginv, w->M1, w->M2));                             // G^{-T} R G^{-1}
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->Rd, -1.0, w->M2, 0.0, nullptr, w->Ct);
  slack_rhs_kernel<<<nb(m), IT, 0, c.st>>>(m, sigma * mu, 1, sl.v, sl.w, sl.zv, sl.zw, w->dva, w->dwa, w->dzva,
                                           w->dzwa, w->rlv, w->rlw, w->rp, w->ctv, w->ctw, w->btl);
  *c.L += 2;
  CUI(cudaMemcpyAsync(w->T, w->M2, bytes, cudaMemcpyDeviceToDevice, c.st));    // keep G^{-T} R G^{-1}
  s = newton(c, w->Ct, w->btl, w->dX, w->dy, w->dSs, info, true);
  if (s != SDP_OK) return s;
  lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->dSs, 1.0, w->T, 0.0, nullptr, w->dS);  // R_d - A^T dy
  slack_dir_kernel<<<nb(m), IT, 0, c.st>>>(m, sl.v, sl.w, sl.zv, sl.zw, w->ctv, w->ctw, w->rlv, w->rlw, w->dy,
                                           w->dv, w->dw, w->dzv, w->dzw);
  *c.L += 2;
  CUI(gemm(c, false, false, w->Ginv, w->dX, w->M1));
  CUI(gemm(c, false, true, w->M1, w->Ginv, w->Dx));
  CUI(gemm(c, true, false, w->G, w->dS, w->M1));
  CUI(gemm(c, false, false, w->M1, w->G, w->Ds));
  s = max_step(c, w->Dx, 0.98, &ap, &sweeps);
  if (s != SDP_OK) return s;
  s = max_step(c, w->Ds, 0.98, &ad, &sweeps);
  if (s != SDP_OK) return s;
  s = ratio_step(c, sl.v, w->dv, sl.w, w->dw, &rp_);
  if (s != SDP_OK) return s;
  s = ratio_step(c, sl.zv, w->dzv, sl.zw, w->dzw, &rd_);
  if (s != SDP_OK) return s;
  ap = std::min(1.0, 0.98 * std::min(ap, rp_));
  ad = std::min(1.0, 0.98 * std::min(ad, rd_));
  sym_axpy_kernel<<<nb(nn), IT, 0, c.st>>>(n, ap, w->dX, X);
  sym_axpy_kernel<<<nb(nn), IT, 0, c.st>>>(n, ad, w->dS, S);
  axpy_kernel<<<nb(m), IT, 0, c.st>>>(m, ad, w->dy, y);
  axpy_kernel<<<nb(m), IT, 0, c.st>>>(m, ap, w->dv, sl.v);
  axpy_kernel<<<nb(m), IT, 0, c.st>>>(m, ap, w->dw, sl.w);
  axpy_kernel<<<nb(m), IT, 0, c.st>>>(m, ad, w->dzv, sl.zv);
  axpy_kernel<<<nb(m), IT, 0, c.st>>>(m, ad, w->dzw, sl.zw);
  *c.L += 7;
  CUI(cudaGetLastError());
  info->alpha_p = ap;
  info->alpha_d = ad;
  info->sigma = sigma;
  info->eig_sweeps += sweeps;
  return SDP_OK;
}

sdp_status check_args(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S) {
  if (!h) return wc_fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!b || !C || !X || !y || !S) return wc_fail(h, SDP_EINVAL, "NULL array argument");
  if (h->kind != SDP_A_DENSE_SVEC && h->kind != SDP_A_DIAG && h->kind != SDP_A_SPARSE_COO)
    return wc_fail(h, SDP_EUNSUPPORTED, "constraint kind not built");
  if (h->lin)
    return wc_fail(h, SDP_EUNSUPPORTED,
                   "the outer loop has no nonnegative variables: remove the linear block first");
  return ensure_workspace(h);
}

}  // namespace

void wc_ipm_free(sdp_handle* h) {
  if (!h || !h->ipm) return;
  for (auto& g : h->ipm->eg) eigh_graph_release(&g);
  if (h->ipm->pool) cudaFree(h->ipm->pool);
  if (h->ipm->lp_pool) cudaFree(h->ipm->lp_pool);
  delete h->ipm;
  h->ipm = nullptr;
}

extern "C" int64_t sdp_eigh_work_elems(int32_t n) { return n < 1 ? 0 : (int64_t)eigh_work_elems(n); }

extern "C" sdp_status sdp_eigh(void* stream, int32_t n, double* A, double* V, double* lam, double tol,
                               int32_t max_sweeps, double* work, int64_t work_elems, int32_t* sweeps) {
  sdp_handle* h = nullptr;
  if (n < 1 || !A || !V || !lam || !work) return wc_fail(nullptr, SDP_EINVAL, "bad eigh argument");
  if (work_elems < (int64_t)eigh_work_elems(n)) return wc_fail(nullptr, SDP_EINVAL, "eigh workspace too small");
  if (!(tol > 0.0) || max_sweeps < 1) return wc_fail(nullptr, SDP_EINVAL, "bad eigh tolerance or sweep cap");
  int sw = 0;
  double off = 0.0;
  cudaError_t e = eigh_jacobi(static_cast<cudaStream_t>(stream), n, A, V, lam, tol, max_sweeps, work,
                              (size_t)work_elems, &sw, &off, nullptr);
  if (e != cudaSuccess) return wc_fail(h, SDP_ECUDA, std::string("eigh: ") + cudaGetErrorString(e));
  if (sweeps) *sweeps = sw;
  return (off <= tol) ? SDP_OK : SDP_ENOTCONV;
}

extern "C" sdp_status ipm_step(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S,
                               sdp_ipm_info* info) {
  NvtxRange nvtx_range("ipm_step");
  sdp_status s = check_args(h, b, C, X, y, S);
  if (s != SDP_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  int64_t L = 0;
  Ctx c{h, h->ipm, h->n, h->m, h->st, &L};
  sdp_ipm_info loc;
  std::memset(&loc, 0, sizeof(loc));
  Measures M;
  s = residuals(c, b, C, X, y, S, &M);
  if (s != SDP_OK) return s;
  fill_info(&loc, M);
  s = step(c, X, y, S, M, &loc);
  loc.iters = 1;
  loc.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  return s;
}

extern "C" sdp_status sdp_solve(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S,
                                double gap_tol, int32_t max_iter, sdp_ipm_info* info) {
  NvtxRange nvtx_range("sdp_solve");
  sdp_status s = check_args(h, b, C, X, y, S);
  if (s != SDP_OK) return s;
  if (!(gap_tol > 0.0) || max_iter < 0) return wc_fail(h, SDP_EINVAL, "bad gap_tol or max_iter");
  const auto t0 = std::chrono::steady_clock::now();
  int64_t L = 0;
  IpmWork* w = h->ipm;
  Ctx c{h, w, h->n, h->m, h->st, &L};
  c.gap_tol = gap_tol;
  s = start(c, b, C, X, y, S);
  if (s != SDP_OK) return s;
  sdp_ipm_info loc;
  std::memset(&loc, 0, sizeof(loc));
  Measures M;
  int it = 0;
  for (;; ++it) {
    s = residuals(c, b, C, X, y, S, &M);
    if (s != SDP_OK) return s;
    fill_info(&loc, M);
    if (M.gap <= gap_tol && M.pinf <= gap_tol && M.dinf <= gap_tol) {
      loc.converged = 1;
      break;
    }
    if (it >= max_iter) break;
    s = step(c, X, y, S, M, &loc);
    if (s != SDP_OK) {
      loc.iters = it;
      if (info) *info = loc;
      return s;
    }
  }
  loc.iters = it;
  loc.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  return loc.converged ? SDP_OK : SDP_ENOTCONV;
}

extern "C" sdp_status sdp_solve_slack(sdp_handle* h, const double* b, const double* C, const double* cv,
                                      const double* cw, double* X, double* y, double* S, double* v, double* wv,
                                      double* zv, double* zw, double gap_tol, int32_t max_iter, sdp_ipm_info* info) {
  if (!h) return wc_fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!cv || !cw || !v || !wv || !zv || !zw) return wc_fail(h, SDP_EINVAL, "NULL array argument");
  // what the linear block supports, checked before X, y, S are written
  if (h->kind == SDP_A_DIAG || h->mixed || h->opt.krylov != 0)
    return wc_fail(h, SDP_EUNSUPPORTED,
                   "nonnegative variables are built for the DENSE_SVEC and SPARSE_COO kinds, the FP64 form and PCG");
  sdp_status s = check_args(h, b, C, X, y, S);   // also refuses a linear block set by the caller
  if (s != SDP_OK) return s;
  if (!(gap_tol > 0.0) || max_iter < 0) return wc_fail(h, SDP_EINVAL, "bad gap_tol or max_iter");
  s = ensure_slack_workspace(h);
  if (s != SDP_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  int64_t L = 0;
  IpmWork* w = h->ipm;
  Ctx c{h, w, h->n, h->m, h->st, &L};
  c.gap_tol = gap_tol;
  const int m = h->m;
  s = start(c, b, C, X, y, S);
  if (s != SDP_OK) return s;
  for (double* x : {v, wv, zv, zw}) fill_kernel<<<nb(m), IT, 0, h->st>>>(m, w->xi, x);   // x = z = xi 1
  L += 4;
  // the Newton solves of this loop carry the linear block delta = v/zv + w/zw (updated in place)
  s = sdp_set_linear_diag(h, w->delta);
  if (s != SDP_OK) return s;
  Slack sl{v, wv, zv, zw, cv, cw, 0.0, 0.0};
  sdp_ipm_info loc;
  std::memset(&loc, 0, sizeof(loc));
  Measures M;
  int it = 0;
  for (;; ++it) {
    s = residuals(c, b, C, X, y, S, &M);
    if (s == SDP_OK) s = slack_measures(c, y, sl, &M);
    if (s != SDP_OK) break;
    fill_info(&loc, M);
    if (M.gap <= gap_tol && M.pinf <= gap_tol && M.dinf <= gap_tol) {
      loc.converged = 1;
      break;
    }
    if (it >= max_iter) break;
    s = step_slack(c, X, y, S, sl, M, &loc);
    if (s != SDP_OK) break;
  }
  const std::string err = h->err;
  sdp_set_linear_diag(h, nullptr);   // the handle is left as the caller set it up
  h->err = err;
  loc.iters = it;
  loc.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  if (s != SDP_OK) return s;
  return loc.converged ? SDP_OK : SDP_ENOTCONV;
}

// Newton steps towards the central-path point of parameter mu (X S = mu I with A(X) = b and
// A^T(y) + S = C): the NT direction of R_c = mu S^{-1} - X, i.e. Lam R + R Lam = 2 mu I - 2 Lam^2
// in the scaled frame (sigma mu = mu, no second-order term), one step length for both sides.
extern "C" sdp_status sdp_center(sdp_handle* h, const double* b, const double* C, double* X, double* y, double* S,
                                 double mu, double tol, int32_t max_iter, sdp_ipm_info* info) {
  sdp_status s = check_args(h, b, C, X, y, S);
  if (s != SDP_OK) return s;
  if (!(mu > 0.0) || !std::isfinite(mu) || !(tol > 0.0) || max_iter < 0)
    return wc_fail(h, SDP_EINVAL, "bad mu, tol or max_iter");
  const auto t0 = std::chrono::steady_clock::now();
  int64_t L = 0;
  IpmWork* w = h->ipm;
  Ctx c{h, w, h->n, h->m, h->st, &L};
  c.gap_tol = tol;
  const int n = h->n;
  const int64_t nn = (int64_t)n * n;
  const size_t bytes = (size_t)nn * sizeof(double);
  sdp_ipm_info loc;
  std::memset(&loc, 0, sizeof(loc));
  std::vector<double> gh(n);
  Measures M;
  int it = 0;
  for (;; ++it) {
    s = residuals(c, b, C, X, y, S, &M);
    if (s != SDP_OK) break;
    fill_info(&loc, M);
    int sweeps = 0;
    s = scaling(c, X, S, &sweeps);
    if (s != SDP_OK) break;
    loc.eig_sweeps += sweeps;
    // centrality ||Lam^2 - mu I||_F / mu with Lam = G^{-1} X G^{-T} = G^T S G = diag(g)
    if (cudaMemcpyAsync(gh.data(), w->g, n * sizeof(double), cudaMemcpyDeviceToHost, c.st) != cudaSuccess ||
        cudaStreamSynchronize(c.st) != cudaSuccess) {
      s = wc_fail(h, SDP_ECUDA, "reading the scaled iterate failed");
      break;
    }
    double cen = 0.0;
    for (int i = 0; i < n; ++i) cen += (gh[i] * gh[i] - mu) * (gh[i] * gh[i] - mu);
    cen = std::sqrt(cen) / mu;
    loc.sigma = cen;   // reported: the centrality of the last iterate
    if (cen <= tol && M.pinf <= tol && M.dinf <= tol) {
      loc.converged = 1;
      break;
    }
    if (it >= max_iter) break;
    // R with Lam R + R Lam = 2 mu I - 2 Lam^2 (P = 0), C~ = R_d - G^{-T} R G^{-1}
    if (cudaMemsetAsync(w->M1, 0, bytes, c.st) != cudaSuccess) {
      s = wc_fail(h, SDP_ECUDA, "clearing a work matrix failed");
      break;
    }
    lyap_kernel<<<nb(nn), IT, 0, c.st>>>(n, 2.0 * mu, w->g, w->M1, w->R);
    ++L;
    if (gemm(c, false, false, w->R, w->Ginv, w->M1) != cudaSuccess ||
        gemm(c, true, false, w->Ginv, w->M1, w->M2) != cudaSuccess) {
      s = wc_fail(h, SDP_ECUDA, "centring products failed");
      break;
    }
    lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->Rd, -1.0, w->M2, 0.0, nullptr, w->Ct);
    ++L;
    s = newton(c, w->Ct, w->rp, w->dX, w->dy, w->dSs, &loc);
    if (s != SDP_OK) break;
    lincomb_kernel<<<nb(nn), IT, 0, c.st>>>(nn, 1.0, w->dSs, 1.0, w->M2, 0.0, nullptr, w->dS);  // R_d - A^T dy
    ++L;
    if (gemm(c, false, false, w->Ginv, w->dX, w->M1) != cudaSuccess ||
        gemm(c, false, true, w->M1, w->Ginv, w->Dx) != cudaSuccess ||
        gemm(c, true, false, w->G, w->dS, w->M1) != cudaSuccess ||
        gemm(c, false, false, w->M1, w->G, w->Ds) != cudaSuccess) {
      s = wc_fail(h, SDP_ECUDA, "centring products failed");
      break;
    }
    double ap = 0.0, ad = 0.0;
    s = max_step(c, w->Dx, 0.95, &ap, &sweeps);
    if (s == SDP_OK) s = max_step(c, w->Ds, 0.95, &ad, &sweeps);
    if (s != SDP_OK) break;
    const double a = std::min(1.0, 0.95 * std::min(ap, ad));
    sym_axpy_kernel<<<nb(nn), IT, 0, c.st>>>(n, a, w->dX, X);
    sym_axpy_kernel<<<nb(nn), IT, 0, c.st>>>(n, a, w->dS, S);
    axpy_kernel<<<nb(c.m), IT, 0, c.st>>>(c.m, a, w->dy, y);
    L += 3;
    loc.alpha_p = loc.alpha_d = a;
  }
  loc.iters = it;
  loc.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  if (s != SDP_OK) return s;
  if (cudaGetLastError() != cudaSuccess) return wc_fail(h, SDP_ECUDA, "centring kernels failed");
  return loc.converged ? SDP_OK : SDP_ENOTCONV;
}

extern "C" sdp_status sdp_scaling_point(sdp_handle* h, const double* X, const double* S, double* V, double* lam) {
  if (!h) return wc_fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!X || !S || !V || !lam) return wc_fail(h, SDP_EINVAL, "NULL array argument");
  sdp_status s = ensure_workspace(h);
  if (s != SDP_OK) return s;
  int64_t L = 0;
  IpmWork* w = h->ipm;
  Ctx c{h, w, h->n, h->m, h->st, &L};
  int sweeps = 0;
  s = scaling(c, X, S, &sweeps);
  if (s != SDP_OK) return s;
  const size_t nn = (size_t)h->n * h->n;
  if (cudaMemcpyAsync(V, w->V, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->st) != cudaSuccess ||
      cudaMemcpyAsync(lam, w->lam, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return wc_fail(h, SDP_ECUDA, "copying the scaling point failed");
  return SDP_OK;
}

extern "C" sdp_status sdp_solve_batch(int32_t count, sdp_handle* const* hs, const double* const* b,
                                      const double* const* C, double* const* X, double* const* y, double* const* S,
                                      double gap_tol, int32_t max_iter, int32_t workers, sdp_ipm_info* infos,
                                      int32_t* statuses) {
  using namespace wc;
  if (count < 0) return wc_fail(nullptr, SDP_EINVAL, "count < 0");
  if (count == 0) return SDP_OK;
  if (!hs || !b || !C || !X || !y || !S || !statuses) return wc_fail(nullptr, SDP_EINVAL, "NULL array argument");
  for (int32_t i = 0; i < count; ++i) statuses[i] = SDP_EINVAL;   // until instance i is solved
  if (!(gap_tol > 0.0) || max_iter < 0) return wc_fail(nullptr, SDP_EINVAL, "bad gap_tol or max_iter");
  std::vector<sdp_handle*> seen(hs, hs + count);
  for (auto* h : seen)
    if (!h) return wc_fail(nullptr, SDP_EINVAL, "NULL handle");
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return wc_fail(nullptr, SDP_EINVAL, "a handle appears twice in the batch");
  // the interior-point workspaces first (allocation is not left to the concurrent solves)
  for (int32_t i = 0; i < count; ++i) {
    sdp_handle* h = hs[i];
    if (h->lin)
      return wc_fail(nullptr, SDP_EUNSUPPORTED, "the outer loop has no nonnegative variables: remove the linear block");
    if (cudaSetDevice(h->dev) != cudaSuccess) return wc_fail(nullptr, SDP_ECUDA, "cudaSetDevice failed");
    sdp_status s = ensure_workspace(h);
    if (s != SDP_OK) {
      statuses[i] = s;
      return s;
    }
  }
  // largest first: about n^3 per outer iteration (eigensolver, dense products) plus m N for
  // the dense passes over A
  std::vector<int32_t> order(count);
  std::vector<double> cost(count);
  for (int32_t i = 0; i < count; ++i) {
    const sdp_handle* h = hs[i];
    order[i] = i;
    cost[i] = (double)h->n * h->n * h->n + (h->kind == SDP_A_DENSE_SVEC ? 64.0 * h->m * (double)h->N : 0.0);
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return cost[a] > cost[c]; });
  for (int32_t i = 0; i < count; ++i) {
    hs[i]->no_coop = true;
    if (hs[i]->coop_pc) wc_drop_graphs(hs[i]);   // recaptured without the cooperative launch
  }
  std::atomic<int32_t> next{0};
  auto work = [&]() {
    for (;;) {
      const int32_t k = next.fetch_add(1);
      if (k >= count) return;
      const int32_t i = order[k];
      sdp_handle* h = hs[i];
      if (cudaSetDevice(h->dev) != cudaSuccess) {
        statuses[i] = SDP_ECUDA;
        continue;
      }
      statuses[i] = sdp_solve(h, b[i], C[i], X[i], y[i], S[i], gap_tol, max_iter, infos ? &infos[i] : nullptr);
    }
  };
  int32_t nw = workers > 0 ? workers : std::min<int32_t>(count, 16);
  nw = std::max<int32_t>(1, std::min<int32_t>({nw, count, 64}));
  std::vector<std::thread> pool;
  for (int32_t t = 1; t < nw; ++t) {
    try {
      pool.emplace_back(work);
    } catch (const std::exception&) {
      break;   // fewer threads: the remaining instances go to the ones that started
    }
  }
  work();
  for (auto& t : pool) t.join();
  for (int32_t i = 0; i < count; ++i) {
    hs[i]->no_coop = false;
    if (hs[i]->coop_pc) wc_drop_graphs(hs[i]);
  }
  for (int32_t i = 0; i < count; ++i)
    if (statuses[i] != SDP_OK) return (sdp_status)statuses[i];
  return SDP_OK;
}

// C ABI and orchestration of one Newton solve on the well-conditioned reformulation
// (Section 3 eq. augsys / eq. recover, Section 6 preconditioner, Cor. pcg).
//
// Per call (all on the handle's stream; one host read after the split for r, then one
// read every `check_every` PCG iterations for the stop flag):
//   a1  split (eq. EQSigdef): sort eig(W), choose r, tau, E = Vs diag(e) Vs^T, Sigma, beta
//   a2  B = A Q (m x d) and the inverse of the preconditioner's Schur complement
//       (d-space C = tau^2 Sigma + beta^{-1} B^T B, or m-space K = beta I + B D^{-1} B^T)
//   a3  g = [b~ + tau^2 A(E C~ E); tau^2 Q^T c], x0 = [0; -Sigma^{-1} Q^T c], r0, z0, p0
//   a4  operator (matrix-free, Section 5): [A(E A^T(p_u) E + sym(U_p Q^T)); Q^T A^T(p_u) - D p_v]
//   a5  preconditioner (block-triangular inverse, Section 6)
//   a6  PCG scalars / updates (Def. pcg)
//   a8  recovery (eq. recover): dy = u / tau^2, dX = E(A^T u - tau^2 C~)E + sym(U_v Q^T),
//       dS = C~ - A^T(dy)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/wcipm.h"
#include "common.cuh"
#include "kernels.h"
#include "pcg.h"

using namespace wc;

struct sdp_handle {
  // problem (device pointers owned by the caller)
  int n = 0, m = 0, kind = 0;
  int64_t nnz = 0, N = 0;
  const int32_t *a_con = nullptr, *a_row = nullptr, *a_col = nullptr;
  const double *a_val = nullptr, *a_dense = nullptr;
  sdp_options opt{};
  cudaStream_t st = nullptr;
  int r_max = 0, d_max = 0, mb = 0;
  double s_A = 1.0;
  // workspace
  char* pool = nullptr;
  size_t pool_bytes = 0;
  PcgCtl* ctl = nullptr;
  PcgCtl* ctl_host = nullptr;      // pinned mirror
  unsigned int* counter = nullptr;
  double *Vs = nullptr, *lam_s = nullptr, *e = nullptr, *Ve = nullptr, *E = nullptr, *EE = nullptr;
  double *Dv = nullptr, *B = nullptr, *Bs = nullptr, *Pinv = nullptr;
  double *Y = nullptr, *F = nullptr, *Z = nullptr, *Cw = nullptr;
  double *T = nullptr, *H = nullptr, *Hp = nullptr, *Up = nullptr;
  double *zsvec = nullptr, *partY = nullptr, *partA = nullptr;
  double *x = nullptr, *rv = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *g = nullptr;
  double *sd = nullptr, *wm = nullptr, *partB = nullptr, *partBt = nullptr, *partC = nullptr;
  double *dotbuf = nullptr, *scratch = nullptr;
  double *gemm_ws = nullptr;
  size_t gemm_ws_elems = 0;
  double *gj_work = nullptr;
  size_t gj_work_elems = 0;
  double *ubatch = nullptr, *Gb = nullptr, *Hb = nullptr;
  // device staging for the host-pointer entry point
  double *hV = nullptr, *hlam = nullptr, *hCt = nullptr, *hbt = nullptr, *hdX = nullptr, *hdy = nullptr, *hdS = nullptr;
  int GY = 1, SA = 1;   // row groups of A^T products, column slabs of A products
  int64_t launches = 0;
  int space = 1, r = 0, d = 0;
  std::string err;
  // optional CUDA-event timing of the constraint-operator passes (sdp_set_profiling)
  struct ProfEntry { int kind; int iter; };
  bool prof = false;
  int cur_iter = -1;
  std::vector<cudaEvent_t> ev;
  std::vector<ProfEntry> prof_entries;
  cudaEvent_t ev_phase[4] = {nullptr, nullptr, nullptr, nullptr};
  double prof_ms[2] = {0.0, 0.0};
  int64_t prof_n[2] = {0, 0};
  double phase_ms[3] = {0.0, 0.0, 0.0};
};

static std::string g_setup_err;

static sdp_status fail(sdp_handle* h, sdp_status s, const std::string& msg) {
  if (h) h->err = msg; else g_setup_err = msg;
  return s;
}

#define CU(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(h, SDP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

extern "C" void sdp_default_options(sdp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->r_fixed = 0;
  o->r_hat = 10;
  o->precision = SDP_FP64;
  o->precond_space = 0;
  o->max_pcg = 2000;
  o->check_every = 8;
  o->beta_rule = 0;
  o->newton_rtol = 1e-12;
}

namespace {

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

inline int dof(int n, int r) { return n * r - r * (r - 1) / 2; }

// Lay out every buffer; with base == nullptr only the size is computed.
size_t carve(sdp_handle* h, char* base) {
  Carver c(base);
  const size_t n = h->n, m = h->m, nn = n * n, rm = h->r_max, dm = h->d_max;
  const size_t vt = m + dm;
  const size_t pdim = std::max(dm, m);
  h->ctl = c.take<PcgCtl>(1);
  h->counter = c.take<unsigned int>(4);
  h->Vs = c.take<double>(nn);
  h->lam_s = c.take<double>(n);
  h->e = c.take<double>(n);
  h->Ve = c.take<double>(nn);
  h->E = c.take<double>(nn);
  h->EE = (h->kind == SDP_A_DIAG) ? c.take<double>(nn) : nullptr;
  h->Dv = c.take<double>(dm);
  h->B = c.take<double>(m * dm);
  h->Bs = c.take<double>(m * dm);
  h->Pinv = c.take<double>(pdim * pdim);
  h->Y = c.take<double>(nn);
  h->F = c.take<double>(nn);
  h->Z = c.take<double>(nn);
  h->Cw = c.take<double>(nn);
  h->T = c.take<double>(n * rm);
  h->H = c.take<double>(n * rm);
  h->Hp = c.take<double>(n * rm);
  h->Up = c.take<double>(n * rm);
  if (h->kind == SDP_A_DENSE_SVEC) {
    h->zsvec = c.take<double>(h->N);
    h->partY = c.take<double>((size_t)h->GY * h->N);
  }
  const size_t sa = std::max<size_t>(h->SA, (size_t)rows_gemv_slabs(std::max<int64_t>(n, pdim)));
  h->partA = c.take<double>(sa * std::max(m, pdim));
  h->x = c.take<double>(vt);
  h->rv = c.take<double>(vt);
  h->z = c.take<double>(vt);
  h->p = c.take<double>(vt);
  h->Ap = c.take<double>(vt);
  h->g = c.take<double>(vt);
  h->sd = c.take<double>(dm);
  h->wm = c.take<double>(m);
  // upper bound of rows_gemvT_groups(m, d) over every d <= d_max
  const size_t gb = std::min<size_t>((m + 31) / 32, 4 * (size_t)g_num_sms) + 1;
  h->partB = c.take<double>(gb * dm);
  h->partBt = c.take<double>(gb * dm);
  h->partC = c.take<double>((size_t)rows_gemv_slabs(pdim) * pdim);
  h->dotbuf = c.take<double>(1024);
  h->scratch = c.take<double>(8192);
  h->gemm_ws_elems = 4 * std::max({nn, dm * dm, pdim * pdim, (size_t)h->mb * n * rm * 2});
  h->gemm_ws = c.take<double>(h->gemm_ws_elems);
  h->gj_work_elems = 64 * 64 + 2 * pdim * 64;
  h->gj_work = c.take<double>(h->gj_work_elems);
  if (h->kind == SDP_A_DENSE_SVEC) {
    h->ubatch = c.take<double>((size_t)h->mb * nn);
    h->Gb = c.take<double>((size_t)h->mb * n * rm);
    h->Hb = c.take<double>((size_t)h->mb * n * rm);
  }
  h->hV = c.take<double>(nn);
  h->hlam = c.take<double>(n);
  h->hCt = c.take<double>(nn);
  h->hbt = c.take<double>(m);
  h->hdX = c.take<double>(nn);
  h->hdy = c.take<double>(m);
  h->hdS = c.take<double>(nn);
  return c.off + 256;
}

}  // namespace

extern "C" sdp_status sdp_setup(const sdp_problem* prob, const sdp_options* opt_in, void* stream,
                                sdp_handle** out) {
  sdp_handle* h = nullptr;
  if (!prob || !out) return fail(nullptr, SDP_EINVAL, "NULL argument");
  *out = nullptr;
  sdp_options opt;
  if (opt_in) opt = *opt_in; else sdp_default_options(&opt);
  const int n = prob->n, m = prob->m;
  if (n < 2 || m < 1) return fail(nullptr, SDP_EINVAL, "need n >= 2 and m >= 1");
  if (prob->kind != SDP_A_DIAG && prob->kind != SDP_A_DENSE_SVEC)
    return fail(nullptr, SDP_EUNSUPPORTED, "constraint kind not built");
  if (prob->kind == SDP_A_DIAG && m != n) return fail(nullptr, SDP_EINVAL, "DIAG kind needs m == n");
  if (prob->kind == SDP_A_DENSE_SVEC && !prob->a_dense) return fail(nullptr, SDP_EINVAL, "a_dense is NULL");
  if (opt.precision != SDP_FP64) return fail(nullptr, SDP_EUNSUPPORTED, "precision not built");
  if (opt.max_pcg < 1 || opt.check_every < 1 || !(opt.newton_rtol >= 0.0))
    return fail(nullptr, SDP_EINVAL, "bad PCG options");
  const int r_max = opt.r_fixed > 0 ? opt.r_fixed : std::min(opt.r_hat, n - 1);
  if (r_max < 1 || r_max >= n) return fail(nullptr, SDP_EINVAL, "rank parameter out of range [1, n)");
  if (opt.precond_space < 0 || opt.precond_space > 2) return fail(nullptr, SDP_EINVAL, "bad precond_space");

  h = new (std::nothrow) sdp_handle();
  if (!h) return fail(nullptr, SDP_ENOMEM, "host allocation failed");
  h->n = n; h->m = m; h->kind = prob->kind; h->nnz = prob->nnz;
  h->a_con = prob->a_con; h->a_row = prob->a_row; h->a_col = prob->a_col; h->a_val = prob->a_val;
  h->a_dense = prob->a_dense;
  h->opt = opt;
  h->st = static_cast<cudaStream_t>(stream);
  h->N = (int64_t)n * (n + 1) / 2;
  h->r_max = r_max;
  h->d_max = dof(n, r_max);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->kind == SDP_A_DENSE_SVEC) {
    h->GY = rows_gemvT_groups(m, h->N);
    h->SA = rows_gemv_slabs(h->N);
    // batch of constraints unpacked to full matrices while forming B (at most ~64 MB)
    int64_t per = (int64_t)n * n * 8;
    h->mb = (int)std::max<int64_t>(1, std::min<int64_t>(m, ((int64_t)64 << 20) / per));
  }
  h->pool_bytes = carve(h, nullptr);
  cudaError_t e = cudaMalloc(&h->pool, h->pool_bytes);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, SDP_ENOMEM, std::string("cudaMalloc of workspace failed: ") + cudaGetErrorString(e));
  }
  carve(h, h->pool);
  e = cudaMallocHost(&h->ctl_host, sizeof(PcgCtl));
  if (e != cudaSuccess) {
    cudaFree(h->pool);
    delete h;
    return fail(nullptr, SDP_ENOMEM, "pinned allocation failed");
  }
  std::memset(h->ctl_host, 0, sizeof(PcgCtl));
  CU(cudaMemsetAsync(h->counter, 0, 4 * sizeof(unsigned int), h->st));
  // s_A = ||A||_F^2 / m (beta rule 0)
  if (h->kind == SDP_A_DENSE_SVEC) {
    rows_sumsq(h->st, h->a_dense, m, h->N, h->dotbuf, h->scratch, &h->launches);
    double tot = 0.0;
    CU(cudaMemcpyAsync(&tot, h->dotbuf, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(cudaStreamSynchronize(h->st));
    h->s_A = tot / m;
    if (!(h->s_A > 0.0) || !std::isfinite(h->s_A)) {
      sdp_destroy(h);
      return fail(nullptr, SDP_EINVAL, "A has a zero or non-finite Frobenius norm");
    }
  } else {
    h->s_A = 1.0;
  }
  *out = h;
  return SDP_OK;
}

namespace {

constexpr size_t kProfCap = 8192;

// Bracket one launch with events when profiling (kind 0: A^T pass, 1: A pass).
void prof_begin(sdp_handle* h, int kind) {
  if (!h->prof || h->prof_entries.size() >= kProfCap) return;
  size_t k = h->prof_entries.size();
  cudaEventRecord(h->ev[2 * k], h->st);
  h->prof_entries.push_back({kind, h->cur_iter});
}
void prof_end(sdp_handle* h) {
  if (!h->prof || h->prof_entries.empty()) return;
  size_t k = h->prof_entries.size() - 1;
  cudaEventRecord(h->ev[2 * k + 1], h->st);
}

// Y = A^T(u) as a full n x n matrix.
void adjoint_full(sdp_handle* h, const double* u, double* Y, const int32_t* done) {
  if (h->kind == SDP_A_DENSE_SVEC) {
    prof_begin(h, 0);
    rows_gemvT(h->st, h->a_dense, h->m, h->N, u, h->partY, h->GY, done, &h->launches);
    prof_end(h);
    svec_unpack_sum(h->st, h->n, h->partY, h->GY, 1.0, Y, done, &h->launches);
  } else {
    launch_diag_matrix(h->st, h->n, u, Y, &h->launches);
  }
}

// out = M pin (mode 1 also computes alpha) or out = g - M pin (mode 0, g != NULL).
sdp_status apply_operator(sdp_handle* h, const double* pin, double* out, const double* gsub, int mode) {
  const int n = h->n, m = h->m, r = h->r, d = h->d;
  const int32_t* done = &h->ctl->done;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  const double* Q = h->Vs;   // first r columns
  const size_t ws = h->gemm_ws_elems;
  const double* pu = pin;
  const double* pv = pin + m;
  // Up = Vs Hp with Hp = [B_p; sqrt2 N_p]: Q p_v as an n x r factor (Section 5)
  h_unpack(st, n, r, pv, h->Hp, done, L);
  CU(gemm_f64(st, false, false, n, r, n, 1.0, h->Vs, n, h->Hp, n, 0.0, h->Up, n, h->gemm_ws, ws, L, done));
  if (h->kind == SDP_A_DENSE_SVEC) {
    adjoint_full(h, pu, h->Y, done);                                   // Y = A^T(p_u)
    CU(gemm_f64(st, false, false, n, r, n, 1.0, h->Y, n, Q, n, 0.0, h->T, n, h->gemm_ws, ws, L, done));
    CU(gemm_f64(st, true, false, n, r, n, 1.0, h->Vs, n, h->T, n, 0.0, h->H, n, h->gemm_ws, ws, L, done));
    CU(gemm_f64(st, false, false, n, n, n, 1.0, h->E, n, h->Y, n, 0.0, h->F, n, h->gemm_ws, ws, L, done));
    CU(gemm_f64(st, false, false, n, n, n, 1.0, h->F, n, h->E, n, 0.0, h->Z, n, h->gemm_ws, ws, L, done));
    svec_pack_plus(st, n, r, h->Z, h->Up, Q, h->zsvec, done, L);      // svec(E Y E + sym(Up Q^T))
    prof_begin(h, 1);
    rows_gemv(st, h->a_dense, m, h->N, h->zsvec, h->partA, done, L);
    prof_end(h);
    launch_ap_finish(st, m, d, n, r, h->partA, h->SA, nullptr, h->Vs, h->H, h->Dv, pin, gsub, out, mode,
                     h->ctl, h->dotbuf, h->counter, L);
  } else {
    launch_diag_scale_rows(st, n, r, pu, h->Vs, h->T, done, L);       // A^T(p_u) Q = diag(p_u) Q
    CU(gemm_f64(st, true, false, n, r, n, 1.0, h->Vs, n, h->T, n, 0.0, h->H, n, h->gemm_ws, ws, L, done));
    rows_gemv(st, h->EE, n, n, pu, h->partA, done, L);                 // diag(E diag(p_u) E) = (E o E) p_u
    launch_ap_finish(st, m, d, n, r, h->partA, rows_gemv_slabs(n), h->Up, h->Vs, h->H, h->Dv, pin, gsub, out,
                     mode, h->ctl, h->dotbuf, h->counter, L);
  }
  return SDP_OK;
}

// z = P^{-1} rin (Section 6), then <r, z>; mode 0 sets rz, mode 1 computes the PCG beta.
void apply_precond(sdp_handle* h, const double* rin, double* zout, int mode) {
  const int m = h->m, d = h->d;
  const int32_t* done = &h->ctl->done;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  const int Gb = rows_gemvT_groups(m, d);
  if (h->space == 1) {
    rows_gemvT(st, h->B, m, d, rin, h->partB, Gb, done, L);           // B^T r_u
    launch_pc_d_s(st, m, d, Gb, h->partB, rin, h->sd, h->ctl, L);      // s = r_v - beta^{-1} B^T r_u
    rows_gemv(st, h->Pinv, d, d, h->sd, h->partC, done, L);            // C^{-1} s
    launch_pc_d_zv(st, m, d, rows_gemv_slabs(d), h->partC, zout, h->ctl, L);
    rows_gemv(st, h->B, m, d, zout + m, h->partA, done, L);            // B z_v
    launch_pc_zu_dot(st, m, d, rows_gemv_slabs(d), h->partA, 1, rin, zout, mode, h->ctl, h->dotbuf, h->counter, L);
  } else {
    launch_pc_m_tv(st, m, d, rin, h->Dv, h->sd, h->ctl, L);            // t = D^{-1} r_v
    rows_gemv(st, h->B, m, d, h->sd, h->partA, done, L);               // B t
    launch_pc_m_w(st, m, rows_gemv_slabs(d), h->partA, rin, h->wm, h->ctl, L);   // w = r_u + B D^{-1} r_v
    rows_gemv(st, h->Pinv, m, m, h->wm, h->partC, done, L);            // K^{-1} w
    launch_pc_m_w(st, m, rows_gemv_slabs(m), h->partC, nullptr, zout, h->ctl, L);  // z_u
    rows_gemvT(st, h->B, m, d, zout, h->partBt, Gb, done, L);          // B^T z_u
    launch_pc_m_zv(st, m, d, Gb, h->partBt, rin, h->Dv, zout, h->ctl, L);          // z_v = D^{-1}(B^T z_u - r_v)
    launch_pc_zu_dot(st, m, d, 0, nullptr, 2, rin, zout, mode, h->ctl, h->dotbuf, h->counter, L);
  }
}

}  // namespace

extern "C" sdp_status sdp_newton_solve(sdp_handle* h, const double* V, const double* lam, const double* Ct,
                                       const double* bt, double* dX, double* dy, double* dS,
                                       sdp_newton_info* info) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!V || !lam || !Ct || !bt || !dX || !dy || !dS) return fail(h, SDP_EINVAL, "NULL array argument");
  h->launches = 0;
  const int n = h->n, m = h->m;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  const size_t ws = h->gemm_ws_elems;
  h->prof_entries.clear();
  h->cur_iter = -1;
  if (!h->ev_phase[0])
    for (auto& e : h->ev_phase) CU(cudaEventCreate(&e));
  CU(cudaEventRecord(h->ev_phase[0], st));

  // ---- a1: split ----
  PcgCtl init{};
  init.s_A = h->s_A;
  init.max_iters = h->opt.max_pcg;
  init.done = 0;
  CU(cudaMemcpyAsync(h->ctl, &init, sizeof(PcgCtl), cudaMemcpyHostToDevice, st));
  split_sort(st, n, V, lam, h->Vs, h->lam_s, L);
  split_params(st, n, h->opt.r_fixed, h->opt.r_hat, h->opt.beta_rule, h->lam_s, h->e, h->ctl, L);
  CU(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (h->ctl_host->status != 0) return fail(h, SDP_EINVAL, "eigenvalues must be positive and finite, 1 <= r < n");
  const int r = h->ctl_host->r, d = h->ctl_host->d;
  if (r > h->r_max) return fail(h, SDP_EINVAL, "rank above the setup maximum");
  h->r = r;
  h->d = d;
  h->space = h->opt.precond_space == 0 ? (d <= m ? 1 : 2) : h->opt.precond_space;
  const int nt = m + d;
  split_scale_cols(st, n, h->Vs, h->e, h->Ve, L);
  CU(gemm_f64(st, false, true, n, n, n, 1.0, h->Ve, n, h->Vs, n, 0.0, h->E, n, h->gemm_ws, ws, L));
  split_sigma(st, n, r, h->lam_s, h->ctl, h->Dv, L);

  // ---- a2: B = A Q and the preconditioner core ----
  if (h->kind == SDP_A_DENSE_SVEC) {
    for (int i0 = 0; i0 < m; i0 += h->mb) {
      const int mb = std::min(h->mb, m - i0);
      svec_rows_unpack(st, h->a_dense, n, i0, mb, h->ubatch, L);
      // Gb (mb n x r) = [A_i] Q ; Hb (n x mb r) = Vs^T Gb viewed n x (mb r)
      CU(gemm_f64(st, false, false, mb * n, r, n, 1.0, h->ubatch, (int64_t)mb * n, h->Vs, n, 0.0, h->Gb,
                  (int64_t)mb * n, h->gemm_ws, ws, L));
      CU(gemm_f64(st, true, false, n, mb * r, n, 1.0, h->Vs, n, h->Gb, n, 0.0, h->Hb, n, h->gemm_ws, ws, L));
      h_pack_rows(st, n, r, mb, i0, h->Hb, h->B, d, L);
    }
  } else {
    launch_hadamard_sq(st, (int64_t)n * n, h->E, h->EE, L);
    h_pack_rows_diag(st, n, r, h->Vs, h->B, d, L);
  }
  int32_t* pstatus = &h->ctl->status;
  if (h->space == 1) {
    // C = beta^{-1} B^T B + tau^2 Sigma  (B row-major m x d == column-major d x m)
    const double beta = h->ctl_host->beta_pc;
    CU(gemm_f64(st, false, true, d, d, m, 1.0 / beta, h->B, d, h->B, d, 0.0, h->Pinv, d, h->gemm_ws, ws, L));
    launch_add_diag(st, d, h->Pinv, h->Dv, 0.0, L);
    CU(spd_inverse(st, d, h->Pinv, h->gj_work, h->gj_work_elems, h->gemm_ws, ws, pstatus, L));
  } else {
    // K = beta I + B D^{-1} B^T = Bs^T Bs + beta I with Bs = D^{-1/2} B^T (d x m)
    launch_scale_B(st, m, d, h->B, h->Dv, h->Bs, L);
    CU(gemm_f64(st, true, false, m, m, d, 1.0, h->Bs, d, h->Bs, d, 0.0, h->Pinv, m, h->gemm_ws, ws, L));
    launch_add_diag(st, m, h->Pinv, nullptr, h->ctl_host->beta_pc, L);
    CU(spd_inverse(st, m, h->Pinv, h->gj_work, h->gj_work_elems, h->gemm_ws, ws, pstatus, L));
  }

  CU(cudaEventRecord(h->ev_phase[1], st));

  // ---- a3: right-hand side and start ----
  const double* Q = h->Vs;
  CU(gemm_f64(st, false, false, n, n, n, 1.0, h->E, n, Ct, n, 0.0, h->F, n, h->gemm_ws, ws, L));
  CU(gemm_f64(st, false, false, n, r, n, 1.0, Ct, n, Q, n, 0.0, h->T, n, h->gemm_ws, ws, L));
  CU(gemm_f64(st, true, false, n, r, n, 1.0, h->Vs, n, h->T, n, 0.0, h->H, n, h->gemm_ws, ws, L));
  if (h->kind == SDP_A_DENSE_SVEC) {
    CU(gemm_f64(st, false, false, n, n, n, 1.0, h->F, n, h->E, n, 0.0, h->Z, n, h->gemm_ws, ws, L));
    svec_pack_plus(st, n, r, h->Z, nullptr, nullptr, h->zsvec, nullptr, L);
    prof_begin(h, 1);
    rows_gemv(st, h->a_dense, m, h->N, h->zsvec, h->partA, nullptr, L);
    prof_end(h);
    launch_rhs_finish(st, m, d, n, r, h->partA, h->SA, nullptr, nullptr, bt, Ct, h->H, h->Dv, h->g, h->x,
                      h->opt.newton_rtol, h->ctl, h->dotbuf, h->counter, L);
  } else {
    launch_rhs_finish(st, m, d, n, r, nullptr, 0, h->F, h->E, bt, Ct, h->H, h->Dv, h->g, h->x,
                      h->opt.newton_rtol, h->ctl, h->dotbuf, h->counter, L);
  }
  // the inverse above may have flagged a non-positive pivot: keep it
  // r0 = g - M x0 ; stop test ; z0 = P^{-1} r0 ; p0 = z0
  {
    sdp_status s = apply_operator(h, h->x, h->rv, h->g, 0);
    if (s != SDP_OK) return s;
  }
  launch_norm_check(st, nt, h->rv, h->ctl, h->dotbuf, h->counter, L);
  apply_precond(h, h->rv, h->z, 0);
  launch_p_update(st, nt, h->z, h->p, 1, h->ctl, L);

  // ---- a4-a6: PCG loop ----
  const int every = h->opt.check_every;
  int host_iter = 0;
  for (;;) {
    CU(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h->ctl_host->done) break;
    for (int k = 0; k < every; ++k, ++host_iter) {
      h->cur_iter = host_iter;
      sdp_status s = apply_operator(h, h->p, h->Ap, nullptr, 1);
      if (s != SDP_OK) return s;
      launch_update(st, nt, h->x, h->rv, h->p, h->Ap, h->ctl, h->dotbuf, h->counter, L);
      apply_precond(h, h->rv, h->z, 1);
      launch_p_update(st, nt, h->z, h->p, 0, h->ctl, L);
    }
  }

  h->cur_iter = -1;
  CU(cudaEventRecord(h->ev_phase[2], st));

  // ---- a8: recovery ----
  const double* u = h->x;
  const double* v = h->x + m;
  adjoint_full(h, u, h->Y, nullptr);
  launch_recover_pre(st, n, m, h->Y, Ct, u, h->Cw, dy, dS, h->ctl, L);
  CU(gemm_f64(st, false, false, n, n, n, 1.0, h->E, n, h->Cw, n, 0.0, h->F, n, h->gemm_ws, ws, L));
  CU(gemm_f64(st, false, false, n, n, n, 1.0, h->F, n, h->E, n, 0.0, h->Z, n, h->gemm_ws, ws, L));
  h_unpack(st, n, r, v, h->Hp, nullptr, L);
  CU(gemm_f64(st, false, false, n, r, n, 1.0, h->Vs, n, h->Hp, n, 0.0, h->Up, n, h->gemm_ws, ws, L));
  launch_sym_plus_full(st, n, r, h->Z, h->Up, Q, dX, L);
  CU(cudaEventRecord(h->ev_phase[3], st));
  CU(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());

  const PcgCtl& c = *h->ctl_host;
  for (int q = 0; q < 3; ++q) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, h->ev_phase[q], h->ev_phase[q + 1]));
    h->phase_ms[q] = ms;
  }
  h->prof_ms[0] = h->prof_ms[1] = 0.0;
  h->prof_n[0] = h->prof_n[1] = 0;
  for (size_t k = 0; k < h->prof_entries.size(); ++k) {
    const auto& pe = h->prof_entries[k];
    if (pe.iter >= c.iters) continue;          // launches after the stop returned at once
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]));
    h->prof_ms[pe.kind] += ms;
    h->prof_n[pe.kind] += 1;
  }
  if (info) {
    info->r = r;
    info->d = d;
    info->pcg_iters = c.iters;
    info->space = h->space;
    info->converged = (c.status == 0 && c.rr <= c.tol2) ? 1 : 0;
    info->tau = c.tau;
    info->beta = c.beta_pc;
    info->res_norm = std::sqrt(c.rr);
    info->rhs_norm = std::sqrt(c.newt_rhs2);
    info->res0_norm = std::sqrt(c.rr0);
    info->setup_ms = h->phase_ms[0];
    info->pcg_ms = h->phase_ms[1];
    info->recover_ms = h->phase_ms[2];
    info->prof_At_ms = h->prof_ms[0];
    info->prof_At_launches = (int32_t)h->prof_n[0];
    info->prof_A_ms = h->prof_ms[1];
    info->prof_A_launches = (int32_t)h->prof_n[1];
    info->s_A = h->s_A;
  }
  if (c.status == 5) return fail(h, SDP_ENUMERIC, "PCG breakdown or non-positive pivot");
  if (c.status == 4 || !(c.rr <= c.tol2)) return fail(h, SDP_ENOTCONV, "PCG did not reach the stopping test");
  return SDP_OK;
}

extern "C" sdp_status sdp_newton_solve_host(sdp_handle* h, const double* V, const double* lam, const double* Ct,
                                            const double* bt, double* dX, double* dy, double* dS,
                                            sdp_newton_info* info) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!V || !lam || !Ct || !bt || !dX || !dy || !dS) return fail(h, SDP_EINVAL, "NULL array argument");
  const size_t nn = (size_t)h->n * h->n * sizeof(double);
  cudaStream_t st = h->st;
  CU(cudaMemcpyAsync(h->hV, V, nn, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(h->hlam, lam, h->n * sizeof(double), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(h->hCt, Ct, nn, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(h->hbt, bt, h->m * sizeof(double), cudaMemcpyHostToDevice, st));
  sdp_status s = sdp_newton_solve(h, h->hV, h->hlam, h->hCt, h->hbt, h->hdX, h->hdy, h->hdS, info);
  if (s != SDP_OK && s != SDP_ENOTCONV) return s;
  CU(cudaMemcpyAsync(dX, h->hdX, nn, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(dy, h->hdy, h->m * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(dS, h->hdS, nn, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return s;
}

extern "C" sdp_status sdp_debug_copy(sdp_handle* h, int32_t which, double* dst, int64_t count) {
  if (!h || !dst || count < 0) return fail(h, SDP_EINVAL, "bad debug copy argument");
  const int64_t n = h->n, m = h->m, d = h->d;
  const int64_t pd = h->space == 1 ? d : m;
  const double* src = nullptr;
  int64_t avail = 0;
  switch (which) {
    case 0: src = h->E; avail = n * n; break;
    case 1: src = h->Dv; avail = d; break;
    case 2: src = h->B; avail = m * d; break;
    case 3: src = h->Pinv; avail = pd * pd; break;
    case 4: src = h->Vs; avail = n * n; break;
    case 5: src = h->x; avail = m + d; break;
    case 6: src = h->g; avail = m + d; break;
    case 7: src = reinterpret_cast<const double*>(h->ctl); avail = sizeof(PcgCtl) / sizeof(double); break;
    case 8: src = h->rv; avail = m + d; break;
    case 9: src = h->z; avail = m + d; break;
    case 10: src = h->p; avail = m + d; break;
    case 11: src = h->Ap; avail = m + d; break;
    default: return fail(h, SDP_EINVAL, "unknown buffer");
  }
  if (count > avail) return fail(h, SDP_EINVAL, "count exceeds the buffer");
  CU(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CU(cudaStreamSynchronize(h->st));
  return SDP_OK;
}

extern "C" sdp_status sdp_set_profiling(sdp_handle* h, int32_t on) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (on && h->ev.empty()) {
    h->ev.resize(2 * kProfCap);
    for (auto& e : h->ev) CU(cudaEventCreate(&e));
  }
  h->prof = on != 0;
  return SDP_OK;
}

extern "C" size_t sdp_workspace_bytes(const sdp_handle* h) { return h ? h->pool_bytes : 0; }

extern "C" int64_t sdp_last_launch_count(const sdp_handle* h) { return h ? h->launches : 0; }

extern "C" const char* sdp_last_error(const sdp_handle* h) {
  return h ? h->err.c_str() : g_setup_err.c_str();
}

extern "C" void sdp_destroy(sdp_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->pool) cudaFree(h->pool);
  for (auto& e : h->ev) cudaEventDestroy(e);
  for (auto& e : h->ev_phase)
    if (e) cudaEventDestroy(e);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  delete h;
}

// C ABI and orchestration of one Newton solve on the well-conditioned reformulation
// (Section 3 eq. augsys / eq. recover, Section 6 preconditioner, Cor. pcg).
//
// Per call (all on the handle's stream; one host read after the split for r; the PCG loop is
// one graph launch with a WHILE node conditioned on the device stop flag, or, where that
// graph is refused, replays of `check_every` iterations with a host read of the flag between):
//   a1  split (eq. EQSigdef): sort eig(W), choose r, tau, E = Vs diag(e) Vs^T, Sigma, beta
//   a2  B = A Q (m x d) and the inverse of the preconditioner's Schur complement
//       (d-space C = tau^2 Sigma + beta^{-1} B^T B, or m-space K = beta I + B D^{-1} B^T)
//   a3  g = [b~ + tau^2 A(E C~ E); tau^2 Q^T c], x0 = [0; -Sigma^{-1} Q^T c], r0, z0, p0
//   a4  operator (matrix-free, Section 5): [A(E A^T(p_u) E + sym(U_p Q^T)); Q^T A^T(p_u) - D p_v]
//   a5  preconditioner (block-triangular inverse, Section 6)
//   a6  PCG scalars / updates (Def. pcg)
//   a7  (mixed form) FP64 refinement: rho = g - M x in FP64, then M~ delta = rho by the same
//       PCG, where M~ forms the A E A^T block from an FP32 copy of A (the two A passes and the
//       n^3 products in FP32) and keeps the rows with B = A Q, the vectors, the scalars and the
//       preconditioner in FP64; x += delta, until the FP64 residual passes the stop test
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

#include "handle.h"

static std::string g_setup_err;

// products go to the tensor cores for n >= kTcMin and M N K >= kTcMinWork (all three >= 64)
constexpr int kTcMin = 512;
// a slack "fixes" its row of the linear block when tau^-2 delta_i exceeds this multiple of beta
constexpr double kLinDominance = 1e8;
constexpr double kTcMinWork = 134217728.0;   // 512^3
constexpr int kFuseMax = 65536;              // PCG vectors short enough for one block's update

static sdp_status fail(sdp_handle* h, sdp_status s, const std::string& msg) {
  if (h) h->err = msg; else g_setup_err = msg;
  return s;
}

sdp_status wc_fail(sdp_handle* h, sdp_status s, const std::string& msg) { return fail(h, s, msg); }

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
  o->use_graph = 1;
  o->newton_rtol = 1e-12;
  o->max_refine = 10;
  o->max_inner = 500;
  o->inner_rtol = 1e-6;
  o->pcg_start = 0;
  o->tc_products = 1;
  o->krylov = 0;
  o->int_passes = 1;
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

void carve_space(sdp_handle* h, Carver& c, Space& S) {
  const size_t n = h->n, m = h->m, nn = n * n, rm = h->r_max, dm = h->d_max;
  const size_t vt = m + dm;
  const size_t pc = h->pinv_dim;
  S.Vs = c.take<double>(nn);
  S.E = c.take<double>(nn);
  S.EE = (h->kind == SDP_A_DIAG) ? c.take<double>(nn) : nullptr;
  S.Dv = c.take<double>(dm);
  S.B = h->b_elems ? c.take<double>(h->b_elems) : nullptr;
  S.Bt = h->bt_elems ? c.take<double>(h->bt_elems) : nullptr;
  S.Pinv = c.take<double>(pc * pc);
  S.Y = c.take<double>(nn);
  S.F = c.take<double>(nn);
  S.Z = c.take<double>(nn);
  S.Tm = c.take<double>(n * rm);
  S.H = c.take<double>(n * rm);
  S.Hp = c.take<double>(n * rm);
  S.Up = c.take<double>(n * rm);
  if (h->kind == SDP_A_DENSE_SVEC) {
    S.zsvec = c.take<double>(h->N);
    S.partY = c.take<double>((size_t)h->GY * h->N);
  }
  if (h->fx) S.fxe = c.take<int>(2);
  if (h->fx && n <= 512) {   // digits of E for the integer-digit E Y E
    S.Ed = c.take<int2>(nn);
    S.eE = c.take<int>(n);
  }
  if (h->kind == SDP_A_SPARSE_COO) {
    S.ypos = c.take<double>(h->sp.npos);
    S.zpos = c.take<double>(h->sp.npos);
  }
  if (h->opt.krylov == 1) {
    S.mw = c.take<double>(vt);
    S.mw1 = c.take<double>(vt);
    S.mw2 = c.take<double>(vt);
  }
  size_t pa = std::max(rows_gemv_part_elems(m, dm), rows_gemv_part_elems(pc, pc));
  if (h->kind == SDP_A_DENSE_SVEC) pa = std::max(pa, rows_gemv_part_elems(m, h->N));
  else pa = std::max(pa, rows_gemv_part_elems(n, n));
  S.partA = c.take<double>(pa);
  S.x = c.take<double>(vt);
  S.rv = c.take<double>(vt);
  S.z = c.take<double>(vt);
  S.p = c.take<double>(vt);
  S.Ap = c.take<double>(vt);
  S.sd = c.take<double>(dm);
  S.wm = c.take<double>(m);
  S.partB = c.take<double>(rows_gemv_part_elems(dm, m));
  S.partBt = c.take<double>(rows_gemv_part_elems(dm, m));
  S.partC = c.take<double>(rows_gemv_part_elems(pc, pc));
  S.ws_elems = 4 * std::max({nn, pc * pc, (size_t)h->mb2 * n * rm * 2});
  S.ws = c.take<double>(S.ws_elems);
}

void carve_mixed(sdp_handle* h, Carver& c, Mixed32& M) {
  const size_t n = h->n, m = h->m, nn = n * n, dm = h->d_max;
  const bool bf = h->lp == SDP_MIXED_BF16, tc = h->lp == SDP_MIXED_TF32 || bf;
  M.ldk = (int)((n + 7) / 8 * 8);                  // pitch of the tensor-core operands (16-byte rows)
  M.Lp = (h->N + 7) / 8 * 8;                       // pitch of the BF16 rows of A
  const size_t esz = bf ? 2 : 4;
  if (h->kind == SDP_A_DENSE_SVEC) {
    if (bf) {
      M.A16 = c.take<char>((size_t)m * M.Lp * 2);
      M.G16 = bf16_gemvT_groups(h->m, M.Lp);
      M.partY = c.take<float>((size_t)M.G16 * M.Lp);
    } else {
      M.A = c.take<float>((size_t)m * h->N);
      M.partY = c.take<float>((size_t)h->GY32 * h->N);
    }
    if (!tc) {
      M.E = c.take<float>(nn);
      M.Y = c.take<float>(nn);
      M.F = c.take<float>(nn);
    } else {
      M.Elp = c.take<char>(n * M.ldk * esz);
      M.Ylp = c.take<char>(n * M.ldk * esz);
      M.Glp = c.take<char>(n * M.ldk * esz);
      if (!bf) {                                   // TF32: the FP32 remainders of (hi, lo) pairs
        M.Elo = c.take<float>(n * M.ldk);
        M.Ylo = c.take<float>(n * M.ldk);
        M.Glo = c.take<float>(n * M.ldk);
      }
    }
    M.Z = c.take<float>(nn);
    M.zsvec = c.take<float>(M.Lp);                 // the tail beyond n(n+1)/2 stays zero
    M.partA = c.take<float>(std::max(rows_gemv_part_elems(m, h->N), (size_t)16 * m));
  } else {
    if (bf) M.EE16 = c.take<char>(n * M.ldk * 2);
    else M.EE = c.take<float>(nn);
    M.partA = c.take<float>(std::max(rows_gemv_part_elems(n, n), (size_t)16 * n));
  }
  M.pu = c.take<float>(std::max(m, (size_t)M.ldk));   // zero tail: the BF16 GEMV over E o E reads ldk
  M.ws_elems = 4 * nn;
  M.ws = c.take<float>(M.ws_elems);
  M.partBv = c.take<double>(rows_gemv_part_elems(m, dm));
  M.partBu = c.take<double>(rows_gemv_part_elems(dm, m));
  M.err = c.take<int>(4);
}

// Lay out every buffer; with base == nullptr only the size is computed.
size_t carve(sdp_handle* h, char* base) {
  Carver c(base);
  const size_t n = h->n, m = h->m, nn = n * n, rm = h->r_max, dm = h->d_max;
  const size_t vt = m + dm;
  h->ctl = c.take<PcgCtl>(1);
  h->ctl_in = c.take<PcgCtl>(1);
  h->mctl = c.take<MinresCtl>(1);
  h->counter = c.take<unsigned int>(4);
  h->loop_guard = c.take<int>(1);
  // one ticket per column block of the A^T pass (at most one block per 256 columns)
  h->gt_tickets = c.take<unsigned int>(h->kind == SDP_A_DENSE_SVEC ? (size_t)(h->N + 255) / 256 + 1 : 1);
  h->lam_s = c.take<double>(n);
  h->e = c.take<double>(n);
  h->Ve = c.take<double>(nn);
  h->Bs = h->bs_elems ? c.take<double>(h->bs_elems) : nullptr;
  h->Cw = c.take<double>(nn);
  h->g = c.take<double>(vt);
  h->dotbuf = c.take<double>(1024);
  h->scratch = c.take<double>(8192);
  h->gj_work_elems = spd_inverse_work(h->pinv_dim);
  if (h->tcw_bytes) h->gj_work_elems = std::max(h->gj_work_elems, spd_inverse_tc_work(h->pinv_dim));
  if (h->kind == SDP_A_SPARSE_COO) {
    h->sp.con_ptr = c.take<int32_t>(m + 1);
    h->sp.pos_r = c.take<int32_t>(h->sp.npos);
    h->sp.pos_c = c.take<int32_t>(h->sp.npos);
    h->sp.pos_ptr = c.take<int32_t>(h->sp.npos + 1);
    h->sp.perm = c.take<int32_t>(h->sp.nnz);
    h->sp.epos = c.take<int32_t>(h->sp.nnz);
    h->sp.cptr = c.take<int32_t>(n + 1);
    h->sp.yptr = c.take<int32_t>(n + 1);
    h->sp.ycol = c.take<int32_t>(h->sp.nnzY);
    h->sp.ypidx = c.take<int32_t>(h->sp.nnzY);
    if (h->sp.npairs > 0) {
      h->sp.pptr = c.take<int32_t>(n + 1);
      h->sp.pxp = c.take<int32_t>(h->sp.npairs);
      h->sp.py = c.take<int32_t>(h->sp.npairs);
      h->sp.pyp = c.take<int32_t>(h->sp.npairs);
      h->sp.pcon = c.take<int32_t>(h->sp.npairs);
      h->sp.pw = c.take<double>(h->sp.npairs);
      h->sp.pcf = c.take<double>(h->sp.npairs);
    }
  }
  h->gj_work = c.take<double>(h->gj_work_elems);
  if (h->fx) {
    h->a_fx = c.take<int2>((size_t)m * fx_row_len(h->N));
    h->a_fx_e = c.take<int>(m);
  }
  if (h->kind == SDP_A_DENSE_SVEC) {
    h->ubatch = c.take<double>((size_t)h->mb * nn);
    h->Gb = c.take<double>((size_t)h->mb2 * n * rm);
    h->Hb = c.take<double>((size_t)h->mb2 * n * rm);
  }
  carve_space(h, c, h->s64);
  h->s64.ctl = h->ctl;
  h->ws_b_elems = 64 * n * rm + 4096;
  h->ws_b[0] = c.take<double>(h->ws_b_elems);
  h->ws_b[1] = c.take<double>(h->ws_b_elems);
  if (h->mixed) {
    h->sin = h->s64;
    h->sin.x = c.take<double>(vt);
    h->sin.rv = c.take<double>(vt);
    h->sin.z = c.take<double>(vt);
    h->sin.p = c.take<double>(vt);
    h->sin.Ap = c.take<double>(vt);
    h->sin.ctl = h->ctl_in;
    carve_mixed(h, c, h->m32);
  }
  if (h->tcw_bytes) {
    h->tc_err = c.take<int>(64);
    h->tcw = c.take<char>(h->tcw_bytes);
    if (h->tcw_b_bytes) h->tcw_b = c.take<char>(h->tcw_b_bytes);
    if (n >= (size_t)kTcMin) {
      h->vs_mem[0] = c.take<char>(tc_slices_bytes(h->n, h->n));
      h->vs_mem[1] = c.take<char>(tc_slices_bytes(h->n, h->n));
    }
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
  if (prob->kind != SDP_A_DIAG && prob->kind != SDP_A_DENSE_SVEC && prob->kind != SDP_A_SPARSE_COO)
    return fail(nullptr, SDP_EINVAL, "unknown constraint kind");
  if (prob->kind == SDP_A_SPARSE_COO) {
    if (prob->nnz < 1 || prob->nnz > INT32_MAX || !prob->a_con || !prob->a_row || !prob->a_col || !prob->a_val)
      return fail(nullptr, SDP_EINVAL, "SPARSE_COO needs 1 <= nnz < 2^31 and all four entry arrays");
    if (opt_in && opt_in->precision != SDP_FP64)
      return fail(nullptr, SDP_EUNSUPPORTED, "the mixed forms are built for the DIAG and DENSE_SVEC kinds");
  }
  if (prob->kind == SDP_A_DIAG && m != n) return fail(nullptr, SDP_EINVAL, "DIAG kind needs m == n");
  if (prob->kind == SDP_A_DENSE_SVEC && !prob->a_dense) return fail(nullptr, SDP_EINVAL, "a_dense is NULL");
  if (opt.precision != SDP_FP64 && opt.precision != SDP_MIXED_FP32 && opt.precision != SDP_MIXED_TF32 &&
      opt.precision != SDP_MIXED_BF16)
    return fail(nullptr, SDP_EUNSUPPORTED, "precision not built");
  if (opt.max_pcg < 1 || opt.check_every < 1 || !(opt.newton_rtol >= 0.0))
    return fail(nullptr, SDP_EINVAL, "bad PCG options");
  if (opt.precision != SDP_FP64 && (opt.max_refine < 1 || opt.max_inner < 1 || !(opt.inner_rtol > 0.0)))
    return fail(nullptr, SDP_EINVAL, "bad refinement options");
  const int r_max = opt.r_fixed > 0 ? opt.r_fixed : std::min(opt.r_hat, n - 1);
  if (r_max < 1 || r_max >= n) return fail(nullptr, SDP_EINVAL, "rank parameter out of range [1, n)");
  if (opt.precond_space < 0 || opt.precond_space > 3) return fail(nullptr, SDP_EINVAL, "bad precond_space");
  if (opt.precond_space == 3 && prob->kind == SDP_A_DIAG)
    return fail(nullptr, SDP_EINVAL, "precond_space 3 (the linear-block rule) needs a kind with a linear block");
  if (opt.pcg_start < 0 || opt.pcg_start > 1) return fail(nullptr, SDP_EINVAL, "bad pcg_start");
  if (opt.tc_products < 0 || opt.tc_products > 1) return fail(nullptr, SDP_EINVAL, "bad tc_products");
  if (opt.krylov < 0 || opt.krylov > 1) return fail(nullptr, SDP_EINVAL, "bad krylov");
  if (opt.int_passes < 0 || opt.int_passes > 1) return fail(nullptr, SDP_EINVAL, "bad int_passes");
  if (opt.krylov == 1 && opt.precision != SDP_FP64)
    return fail(nullptr, SDP_EUNSUPPORTED, "MINRES is built for the FP64 form only");

  // SPARSE_COO: validate the entries and build the index tables on the host (once per problem)
  std::vector<int32_t> sp_con_ptr, sp_pos_r, sp_pos_c, sp_pos_ptr, sp_perm, sp_epos, sp_yptr, sp_ycol, sp_ypidx,
      sp_cptr, sp_pptr, sp_pxp, sp_py, sp_pyp, sp_pcon;
  std::vector<double> sp_pw;
  std::vector<double> sp_rownorm2;
  if (prob->kind == SDP_A_SPARSE_COO) {
    const int64_t nnz = prob->nnz;
    std::vector<int32_t> con(nnz), row(nnz), col(nnz);
    std::vector<double> val(nnz);
    if (cudaMemcpy(con.data(), prob->a_con, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(row.data(), prob->a_row, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(col.data(), prob->a_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(val.data(), prob->a_val, nnz * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(nullptr, SDP_ECUDA, "reading the sparse entries failed");
    sp_con_ptr.assign(m + 1, 0);
    sp_rownorm2.assign(m, 0.0);
    for (int64_t e = 0; e < nnz; ++e) {
      if (con[e] < 0 || con[e] >= m || (e > 0 && con[e] < con[e - 1]))
        return fail(nullptr, SDP_EINVAL, "a_con must be nondecreasing and in [0, m)");
      if (col[e] < 0 || row[e] < col[e] || row[e] >= n)
        return fail(nullptr, SDP_EINVAL, "entries need 0 <= a_col <= a_row < n");
      if (!std::isfinite(val[e])) return fail(nullptr, SDP_EINVAL, "non-finite a_val");
      sp_con_ptr[con[e] + 1] += 1;
      sp_rownorm2[con[e]] += val[e] * val[e] * (row[e] == col[e] ? 1.0 : 2.0);
    }
    for (int i = 0; i < m; ++i) {
      if (sp_con_ptr[i + 1] == 0) return fail(nullptr, SDP_EINVAL, "every constraint needs at least one entry");
      sp_con_ptr[i + 1] += sp_con_ptr[i];
    }
    sp_perm.resize(nnz);
    for (int64_t e = 0; e < nnz; ++e) sp_perm[e] = (int32_t)e;
    auto key = [&](int32_t e) { return (int64_t)col[e] * n + row[e]; };
    std::stable_sort(sp_perm.begin(), sp_perm.end(), [&](int32_t a, int32_t b) { return key(a) < key(b); });
    for (int64_t k = 0; k < nnz; ++k) {
      if (k == 0 || key(sp_perm[k]) != key(sp_perm[k - 1])) {
        sp_pos_r.push_back(row[sp_perm[k]]);
        sp_pos_c.push_back(col[sp_perm[k]]);
        sp_pos_ptr.push_back((int32_t)k);
      }
    }
    sp_pos_ptr.push_back((int32_t)nnz);
    // entry -> position, and the CSR of the symmetric pattern of A^T(y): row i holds (c, p) for
    // every position p = (i, c) and, off the diagonal, (c, p) for p = (c, i)
    const int npos = (int)sp_pos_r.size();
    sp_epos.resize(nnz);
    for (int p = 0; p < npos; ++p)
      for (int k = sp_pos_ptr[p]; k < sp_pos_ptr[p + 1]; ++k) sp_epos[sp_perm[k]] = p;
    // positions are sorted by column: cptr[b] .. cptr[b+1]-1 are those of column b
    sp_cptr.assign(n + 1, 0);
    for (int p = 0; p < npos; ++p) sp_cptr[sp_pos_c[p] + 1] += 1;
    for (int b = 0; b < n; ++b) sp_cptr[b + 1] += sp_cptr[b];
    sp_yptr.assign(n + 1, 0);
    for (int p = 0; p < npos; ++p) {
      sp_yptr[sp_pos_r[p] + 1] += 1;
      if (sp_pos_r[p] != sp_pos_c[p]) sp_yptr[sp_pos_c[p] + 1] += 1;
    }
    for (int i = 0; i < n; ++i) sp_yptr[i + 1] += sp_yptr[i];
    sp_ycol.resize(sp_yptr[n]);
    sp_ypidx.resize(sp_yptr[n]);
    std::vector<int32_t> fill(sp_yptr.begin(), sp_yptr.end() - 1);
    for (int p = 0; p < npos; ++p) {
      const int a = sp_pos_r[p], b = sp_pos_c[p];
      sp_ycol[fill[a]] = b;
      sp_ypidx[fill[a]++] = p;
      if (a != b) {
        sp_ycol[fill[b]] = a;
        sp_ypidx[fill[b]++] = p;
      }
    }
    // term pairs for the Gram form of the d-space complement: A_i = sum_t w_t e_{x_t} e_{y_t}^T
    // (an off-diagonal entry (r, c) gives the terms (r, c) and (c, r)), every pair of terms of one
    // constraint, grouped by x_t; built when the table stays moderate (else the complement is formed
    // from the explicit B)
    int64_t np = 0;
    for (int i = 0; i < m; ++i) {
      int64_t t = 0;
      for (int e = sp_con_ptr[i]; e < sp_con_ptr[i + 1]; ++e) t += (row[e] == col[e]) ? 1 : 2;
      np += t * t;
    }
    if (np <= (int64_t)1 << 26) {
      sp_pptr.assign(n + 1, 0);
      std::vector<int32_t> tx, ty;
      std::vector<double> tw;
      for (int pass = 0; pass < 2; ++pass) {   // counts per row x, then the fill
        std::vector<int32_t> pos;
        if (pass == 1) {
          for (int x = 0; x < n; ++x) sp_pptr[x + 1] += sp_pptr[x];
          pos.assign(sp_pptr.begin(), sp_pptr.end() - 1);
          sp_pxp.resize(np);
          sp_py.resize(np);
          sp_pyp.resize(np);
          sp_pcon.resize(np);
          sp_pw.resize(np);
        }
        for (int i = 0; i < m; ++i) {
          tx.clear();
          ty.clear();
          tw.clear();
          for (int e = sp_con_ptr[i]; e < sp_con_ptr[i + 1]; ++e) {
            tx.push_back(row[e]);
            ty.push_back(col[e]);
            tw.push_back(val[e]);
            if (row[e] != col[e]) {
              tx.push_back(col[e]);
              ty.push_back(row[e]);
              tw.push_back(val[e]);
            }
          }
          for (size_t t = 0; t < tx.size(); ++t) {
            if (pass == 0) {
              sp_pptr[tx[t] + 1] += (int32_t)tx.size();
              continue;
            }
            for (size_t u = 0; u < tx.size(); ++u) {
              const int32_t q = pos[tx[t]]++;
              sp_pxp[q] = tx[u];
              sp_py[q] = ty[t];
              sp_pyp[q] = ty[u];
              sp_pcon[q] = i;
              sp_pw[q] = tw[t] * tw[u];
            }
          }
        }
      }
    }
  }

  h = new (std::nothrow) sdp_handle();
  if (!h) return fail(nullptr, SDP_ENOMEM, "host allocation failed");
  if (prob->kind == SDP_A_SPARSE_COO) {
    h->sp.nnz = prob->nnz;
    h->sp.npos = (int)sp_pos_r.size();
    h->sp.nnzY = (int64_t)sp_ycol.size();
    h->sp.npairs = (int64_t)sp_pxp.size();
    h->sp.m = m;
    h->sp.con = prob->a_con;
    h->sp.row = prob->a_row;
    h->sp.col = prob->a_col;
    h->sp.val = prob->a_val;
    h->sp_rownorm2 = sp_rownorm2;
  }
  h->n = n; h->m = m; h->kind = prob->kind; h->nnz = prob->nnz;
  h->a_con = prob->a_con; h->a_row = prob->a_row; h->a_col = prob->a_col; h->a_val = prob->a_val;
  h->a_dense = prob->a_dense;
  h->opt = opt;
  h->mixed = (opt.precision != SDP_FP64);
  h->lp = opt.precision;
  h->st = static_cast<cudaStream_t>(stream);
  h->N = (int64_t)n * (n + 1) / 2;
  h->fx = (h->kind == SDP_A_DENSE_SVEC && opt.int_passes == 1);
  h->r_max = r_max;
  h->d_max = dof(n, r_max);
  // d-space core (d x d) when d <= m, m-space core (m x m) otherwise, unless forced
  h->pinv_dim = opt.precond_space == 1 ? h->d_max : opt.precond_space == 2 ? m
              : opt.precond_space == 3 ? std::max(h->d_max, m) : std::min(h->d_max, m);
  if (opt.krylov == 1) h->pinv_dim = 0;   // MINRES: no preconditioner core
  // explicit B = A Q: DIAG forms its m-space core in closed form and its products with B from
  // Vs, so it needs B only for the d-space core (auto selects that only at r = 1, d = n)
  // SPARSE_COO reads B only to form the core (its products with B go through the pattern);
  // DENSE_SVEC streams B and B^T in every preconditioner application
  const bool m_space_possible = opt.precond_space == 2 || opt.precond_space == 3 ||
                                (opt.precond_space == 0 && h->d_max > m);
  if (h->kind == SDP_A_DIAG) {
    h->b_elems = opt.precond_space == 2 ? 0 : (int64_t)m * (opt.precond_space == 1 ? h->d_max : dof(n, 1));
    h->bt_elems = h->b_elems;
    h->bs_elems = 0;
  } else {
    h->b_elems = (int64_t)m * h->d_max;
    h->bt_elems = (h->kind == SDP_A_SPARSE_COO && !h->mixed) ? 0 : h->b_elems;
    h->bs_elems = m_space_possible ? (int64_t)m * h->d_max : 0;
  }
  if (opt.krylov == 1) h->b_elems = h->bt_elems = h->bs_elems = 0;   // MINRES: no B = A Q
  int dev = 0;
  cudaGetDevice(&dev);
  h->dev = dev;
  cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->kind == SDP_A_DENSE_SVEC) {
    h->GY = rows_gemvT_groups(m, h->N, 8);
    h->SA = h->fx ? fx_rows_gemv_slabs(m, h->N) : rows_gemv_slabs(m, h->N, 8);
    h->GY32 = rows_gemvT_groups(m, h->N, 4);
    h->SA32 = rows_gemv_slabs(m, h->N, 4);
    // batch of constraints unpacked to full matrices while forming B (at most ~64 MB)
    int64_t per = (int64_t)n * n * 8;
    h->mb = (int)std::max<int64_t>(1, std::min<int64_t>(m, ((int64_t)64 << 20) / per));
    // batch of constraints whose A_i Q factors are formed at once (at most ~32 MB per factor)
    h->mb2 = (int)std::max<int64_t>(h->mb, std::min<int64_t>(m, ((int64_t)32 << 20) / ((int64_t)n * r_max * 8)));
  }
  // slices of the tensor-core products: the n^3 products, and the complement B^T B or
  // B D^{-1} B^T (processed in K-chunks when the whole K does not fit in 4 GiB)
  const bool big_core = h->kind != SDP_A_DIAG && h->pinv_dim >= kTcMin;
  if (opt.tc_products && (n >= kTcMin || big_core)) {
    size_t need = n >= kTcMin ? tc_gemm_work_bytes(n, n, n) : 0;
    if (big_core) {
      need = std::max(need, tc_gemm_work_bytes(h->pinv_dim, h->pinv_dim, std::max(h->d_max, m)));
      need = std::max(need, tc_gemm_work_bytes(h->pinv_dim, h->pinv_dim, h->pinv_dim));
    }
    if (h->kind == SDP_A_DENSE_SVEC)   // H = Vs^T [A_i Q] for a batch of constraints
      need = std::max(need, tc_gemm_work_bytes(n, h->mb2 * r_max, n));
    h->tcw_bytes = std::min(need, std::max(n >= kTcMin ? tc_gemm_work_bytes(n, n, n) : need, (size_t)4 << 30));
    if (r_max >= 64) h->tcw_b_bytes = tc_gemm_work_bytes(n, r_max, n);
    if (tc_prepare() != cudaSuccess) {   // no tensor-map encoder: every product on the FP64 MMA path
      cudaGetLastError();
      h->tcw_bytes = h->tcw_b_bytes = 0;
    }
  }
  if (h->lp == SDP_MIXED_TF32 || h->lp == SDP_MIXED_BF16) {
    if (prob->kind == SDP_A_DENSE_SVEC && (tc_prepare() != cudaSuccess || lp_prepare() != cudaSuccess)) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, SDP_EUNSUPPORTED, "the TF32 / BF16 forms need tcgen05 (a Blackwell GPU)");
    }
  }
  h->pool_bytes = carve(h, nullptr);
  cudaError_t e = cudaMalloc(&h->pool, h->pool_bytes);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, SDP_ENOMEM, std::string("cudaMalloc of workspace failed: ") + cudaGetErrorString(e));
  }
  carve(h, h->pool);
  // zero workspace: the split-K tickets of the GEMMs must start at zero (and, for SPARSE_COO,
  // the n x n matrices that A^T(y) fills only on the pattern)
  e = cudaMemsetAsync(h->pool, 0, h->pool_bytes, h->st);
  if (e != cudaSuccess) {
    cudaFree(h->pool);
    delete h;
    return fail(nullptr, SDP_ECUDA, std::string("workspace clear failed: ") + cudaGetErrorString(e));
  }
  if (h->kind == SDP_A_SPARSE_COO) {
    if (sparse_prepare(n) != cudaSuccess) {
      cudaGetLastError();
      sdp_destroy(h);
      return fail(nullptr, SDP_EUNSUPPORTED, "SPARSE_COO is built for n <= 29000 (one row of E Y in shared memory)");
    }
    const size_t b32 = sizeof(int32_t);
    CU(cudaMemcpyAsync(h->sp.con_ptr, sp_con_ptr.data(), sp_con_ptr.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.pos_r, sp_pos_r.data(), sp_pos_r.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.pos_c, sp_pos_c.data(), sp_pos_c.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.pos_ptr, sp_pos_ptr.data(), sp_pos_ptr.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.perm, sp_perm.data(), sp_perm.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.epos, sp_epos.data(), sp_epos.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.cptr, sp_cptr.data(), sp_cptr.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.yptr, sp_yptr.data(), sp_yptr.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.ycol, sp_ycol.data(), sp_ycol.size() * b32, cudaMemcpyHostToDevice, h->st));
    CU(cudaMemcpyAsync(h->sp.ypidx, sp_ypidx.data(), sp_ypidx.size() * b32, cudaMemcpyHostToDevice, h->st));
    if (h->sp.npairs > 0) {
      const size_t np = (size_t)h->sp.npairs;
      CU(cudaMemcpyAsync(h->sp.pptr, sp_pptr.data(), sp_pptr.size() * b32, cudaMemcpyHostToDevice, h->st));
      CU(cudaMemcpyAsync(h->sp.pxp, sp_pxp.data(), np * b32, cudaMemcpyHostToDevice, h->st));
      CU(cudaMemcpyAsync(h->sp.py, sp_py.data(), np * b32, cudaMemcpyHostToDevice, h->st));
      CU(cudaMemcpyAsync(h->sp.pyp, sp_pyp.data(), np * b32, cudaMemcpyHostToDevice, h->st));
      CU(cudaMemcpyAsync(h->sp.pcon, sp_pcon.data(), np * b32, cudaMemcpyHostToDevice, h->st));
      CU(cudaMemcpyAsync(h->sp.pw, sp_pw.data(), np * sizeof(double), cudaMemcpyHostToDevice, h->st));
    }
  }
  e = cudaMallocHost(&h->ctl_host, sizeof(PcgCtl));
  if (e != cudaSuccess) {
    cudaFree(h->pool);
    delete h;
    return fail(nullptr, SDP_ENOMEM, "pinned allocation failed");
  }
  std::memset(h->ctl_host, 0, sizeof(PcgCtl));
  for (auto& a : h->aux) CU(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
  // the cooperative preconditioner apply (dense kind, d-space) where the device launches it;
  // batched solves turn it off with the other grid barriers
  h->coop_pc = (h->kind == SDP_A_DENSE_SVEC) && pc_dense_coop_blocks() > 0 && pc_dense_coop_blocks() <= 1024;
  for (auto& ev : h->br_ev) CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CU(cudaMemsetAsync(h->counter, 0, 4 * sizeof(unsigned int), h->st));
  // s_A = ||A||_F^2 / m (beta rule 0); FP32 copy of A for the mixed form
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
    if (h->mixed && h->lp == SDP_MIXED_BF16)   // BF16 rows, zero padded to a 16-byte pitch
      lp_convert(h->st, m, (int)h->N, h->a_dense, h->N, h->m32.A16, h->m32.Lp, true, nullptr, &h->launches);
    else if (h->mixed)
      convert<float, double>(h->st, (int64_t)m * h->N, h->a_dense, h->m32.A, &h->launches);
    if (h->fx) fx_split_rows(h->st, h->a_dense, m, h->N, h->a_fx, h->a_fx_e, &h->launches);
  } else if (h->kind == SDP_A_SPARSE_COO) {
    sparse_sumsq(h->st, h->sp, h->dotbuf, h->scratch, &h->launches);
    double tot = 0.0;
    CU(cudaMemcpyAsync(&tot, h->dotbuf, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(cudaStreamSynchronize(h->st));
    h->s_A = tot / m;
  } else {
    h->s_A = 1.0;
  }
  CU(cudaStreamSynchronize(h->st));
  *out = h;
  return SDP_OK;
}

namespace {

constexpr size_t kProfCap = 8192;

// Bracket one launch with events when profiling.
void prof_begin(sdp_handle* h, int kind) {
  if (!h->prof || h->prof_entries.size() >= kProfCap) return;
  size_t k = h->prof_entries.size();
  if (h->capturing) cudaEventRecordWithFlags(h->ev[2 * k], h->st, cudaEventRecordExternal);
  else cudaEventRecord(h->ev[2 * k], h->st);
  h->prof_entries.push_back({kind, h->cur_iter});
}

void prof_end(sdp_handle* h) {
  if (!h->prof || h->prof_entries.empty()) return;
  size_t k = h->prof_entries.size() - 1;
  if (h->capturing) cudaEventRecordWithFlags(h->ev[2 * k + 1], h->st, cudaEventRecordExternal);
  else cudaEventRecord(h->ev[2 * k + 1], h->st);
}

// Time of the profiled launches whose iteration (relative to `base`) ran, given `iters` done.
// Events first..last-1 belong to entries meta[0..]; meta defaults to prof_entries[first..].
sdp_status prof_collect(sdp_handle* h, size_t first, size_t last, int base, int iters,
                        const std::vector<ProfEntry>* meta = nullptr) {
  for (size_t k = first; k < last; ++k) {
    const auto& pe = meta ? (*meta)[k - first] : h->prof_entries[k];
    if (pe.iter >= 0 && base + pe.iter >= iters) continue;   // launches after the stop returned at once
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]) != cudaSuccess) {
      cudaGetLastError();
      return SDP_ECUDA;
    }
    h->prof_ms[pe.kind] += ms;
    h->prof_n[pe.kind] += 1;
  }
  return SDP_OK;
}

// Side branch: a stream that starts after everything issued so far on h->st (event fork; inside
// stream capture the side stream joins the capture), and the join back into h->st.
cudaStream_t fork(sdp_handle* h, int which, int ev) {
  cudaEventRecord(h->br_ev[ev], h->st);
  cudaStreamWaitEvent(h->aux[which], h->br_ev[ev], 0);
  return h->aux[which];
}

void join(sdp_handle* h, int which, int ev) {
  cudaEventRecord(h->br_ev[ev], h->aux[which]);
  cudaStreamWaitEvent(h->st, h->br_ev[ev], 0);
}

// Dense FP64 product: on the tensor cores (exact slices) when the handle holds their workspace
// and the product is large, else on the FP64 MMA path.
// slot 0: products on the handle's stream; slot 1: on the first side stream (its own slices).
cudaError_t gemm_big(sdp_handle* h, cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                     double* ws, size_t ws_elems, int64_t* L, int flags = 0, const int32_t* done = nullptr,
                     int slot = 0) {
  char* w = slot == 0 ? h->tcw : h->tcw_b;
  const size_t wb = slot == 0 ? h->tcw_bytes : h->tcw_b_bytes;
  if (w && M >= 64 && N >= 64 && K >= 64 && (double)M * N * K >= kTcMinWork &&
      !(flags & (GEMM_KSTART_ROW | GEMM_KSTART_COL)) && tc_gemm_work_bytes(M, N, std::min(K, 4096)) <= wb) {
    // the eigenvectors Vs of this solve enter many products: their slices are made once per split
    const double* Vs = h->s64.Vs;
    const TcSlices* cA = (A == Vs && lda == h->n) ? &h->vs_sl[tA ? 1 : 0] : nullptr;
    const TcSlices* cB = (B == Vs && ldb == h->n) ? &h->vs_sl[tB ? 0 : 1] : nullptr;
    return gemm_f64_tc(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, w, wb, h->tc_err, flags, L, done,
                       cA, cB);
  }
  return gemm_f64(st, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_elems, L, done, flags);
}

// Inverse of the SPD preconditioner core: two-level with tensor-core products when the handle
// holds their workspace, else the one-level FP64 form.
cudaError_t spd_inverse_any(sdp_handle* h, cudaStream_t st, int dim, double* P, double* ws, size_t ws_elems,
                            int32_t* status, int64_t* L) {
  if (h->tcw) {
    TcCtx tc;
    tc.work = h->tcw;
    tc.bytes = h->tcw_bytes;
    tc.err = h->tc_err;
    return spd_inverse_tc(st, dim, P, h->gj_work, h->gj_work_elems, ws, ws_elems, &tc, status, L, !h->no_coop);
  }
  return spd_inverse(st, dim, P, h->gj_work, h->gj_work_elems, ws, ws_elems, status, L, !h->no_coop);
}

// Y = A^T(u) as a full n x n matrix (DENSE kind).
void adjoint_dense(sdp_handle* h, Space& S, const double* u, double* Y, const int32_t* done) {
  if (h->fx) {
    prof_begin(h, 0);
    fx_rows_gemvT_unpack(h->st, h->a_fx, h->a_fx_e, h->m, h->N, u, S.fxe, S.partY, h->GY, h->n, 1.0, Y, done,
                         &h->launches);
    prof_end(h);
    return;
  }
  prof_begin(h, 0);
  rows_gemvT_unpack<double>(h->st, h->a_dense, h->m, h->N, u, S.partY, h->GY, h->n, 1.0, Y, h->gt_tickets, done,
                            &h->launches);
  prof_end(h);
}

// z = svec(Z + sym(U Q^T)) (U may be NULL), then partA = the slab partial sums of A(z) (DENSE
// kind); on the integer path the packing kernel also gives the exponent of z
cudaError_t pack_apply_dense(sdp_handle* h, Space& S, cudaStream_t st, int r, const double* U, const double* Q,
                             const int32_t* done, int64_t* L, bool packed = false) {
  const int n = h->n;
  const double* z = S.zsvec;
  if (h->fx) {
    if (!packed) {   // else the E Y E product packed z and found its exponent
      cudaError_t e = cudaMemsetAsync(S.fxe + 1, 0x80, sizeof(int), st);   // below FX_NONE_MAX: no entry yet
      if (e != cudaSuccess) return e;
      svec_pack_plus<double>(st, n, r, S.Z, U, Q, S.zsvec, done, L, S.fxe + 1);
    }
    prof_begin(h, 1);
    fx_rows_gemv(st, h->a_fx, h->a_fx_e, h->m, h->N, z, S.fxe + 1, S.partA, done, L);
    prof_end(h);
    return cudaGetLastError();
  }
  svec_pack_plus<double>(st, n, r, S.Z, U, Q, S.zsvec, done, L);
  prof_begin(h, 1);
  rows_gemv<double>(st, h->a_dense, h->m, h->N, z, S.partA, done, L);
  prof_end(h);
  return cudaGetLastError();
}

// The dense d-space preconditioner apply runs as one cooperative launch.
bool pc_coop_on(const sdp_handle* h) {
  return h->space == 1 && !h->lin && h->kind == SDP_A_DENSE_SVEC && h->coop_pc && !h->no_coop;
}

// The SPARSE kind's d-space complement in its Gram form (no explicit B) where that is cheaper:
// r (r + 1) / 2 column pairs, each a sparse product over the term pairs and one n^3 product,
// against the m d^2 / 2 of B^T B.
bool gram_on(const sdp_handle* h) {
  if (h->kind != SDP_A_SPARSE_COO || h->space != 1 || h->mixed || h->opt.krylov == 1 || h->sp.npairs == 0)
    return false;
  const double n = h->n, r = h->r, d = h->d, m = h->m;
  return 0.5 * r * (r + 1) * ((double)h->sp.npairs * n + n * n * n) < 0.5 * m * d * d;
}

// Small DIAG problems in the m-space form run their whole FP64 PCG solve as one cluster launch
// (with use_graph: the device-resident form of the loop; use_graph = 0 keeps the launch chain).
bool small_pcg_on(const sdp_handle* h) {
  if (h->kind != SDP_A_DIAG || h->mixed || h->opt.krylov != 0 || h->space != 2 || h->lin || h->prof) return false;
  if (!h->opt.use_graph || !h->small_ok) return false;
  return small_pcg_plan(h->n, h->r, h->d, nullptr) > 0;
}

// Inside the PCG loop the update x += alpha p, r -= alpha Ap runs in the last block of the
// operator's finishing kernel, or, with the cooperative preconditioner apply, inside that launch.
double* fuse_x(const sdp_handle* h, Space& S) { return h->fuse && !pc_coop_on(h) ? S.x : nullptr; }

// out = M pin (mode 1 also computes alpha) or out = g - M pin (mode 0, g != NULL), in FP64.
sdp_status apply_operator(sdp_handle* h, Space& S, const double* pin, double* out, const double* gsub, int mode) {
  const int n = h->n, m = h->m, r = h->r, d = h->d;
  const int32_t* done = &S.ctl->done;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  const double* Q = S.Vs;   // first r columns
  const double* pu = pin;
  const double* pv = pin + m;
  // side branch 0: Up = Vs Hp with Hp = [B_p; sqrt2 N_p], Q p_v as an n x r factor (Section 5),
  // independent of A^T(p_u)
  cudaStream_t s0 = fork(h, 0, 0);
  h_unpack<double>(s0, n, r, pv, S.Hp, done, L);
  CU(gemm_big(h, s0, false, false, n, r, n, 1.0, S.Vs, n, S.Hp, n, 0.0, S.Up, n, h->ws_b[0], h->ws_b_elems, L, 0, done,
              1));
  if (h->kind == SDP_A_DENSE_SVEC) {
    adjoint_dense(h, S, pu, S.Y, done);                                // Y = A^T(p_u)
    // side branch 1: H = Vs^T (Y Q), beside E Y E on the main stream
    cudaStream_t s1 = fork(h, 1, 1);
    CU(gemm_f64(s1, false, false, n, r, n, 1.0, S.Y, n, Q, n, 0.0, S.Tm, n, h->ws_b[1], h->ws_b_elems, L, done));
    CU(gemm_f64(s1, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, h->ws_b[1], h->ws_b_elems, L, done));
    bool packed = false;
    if (h->fx && n < kTcMin) {   // E Y E from exact integer sums (the integer pipe outruns the FP64 one)
      const int pa = S.ed_valid ? 1 : 0, pb = S.ed_valid ? 2 : 0;   // E's digits made at setup
      CU(fx_gemm(st, n, n, n, S.E, n, S.Y, n, S.F, n, false, done, L, pa, S.Ed, S.eE));
      // the second product writes svec(E Y E + sym(Up Q^T)) and its exponent directly (no Z)
      join(h, 0, 2);
      CU(cudaMemsetAsync(S.fxe + 1, 0x80, sizeof(int), st));   // below FX_NONE_MAX: no entry yet
      FxPack pk;
      pk.U = S.Up;
      pk.Q = Q;
      pk.r = r;
      pk.out = S.zsvec;
      pk.expo = S.fxe + 1;
      CU(fx_gemm(st, n, n, n, S.F, n, S.E, n, S.Z, n, true, done, L, pb, S.Ed, S.eE, &pk));
      packed = true;
    } else {
      CU(gemm_f64(st, false, false, n, n, n, 1.0, S.E, n, S.Y, n, 0.0, S.F, n, S.ws, S.ws_elems, L, done));
      CU(gemm_f64(st, false, false, n, n, n, 1.0, S.F, n, S.E, n, 0.0, S.Z, n, S.ws, S.ws_elems, L, done,
                  GEMM_LOWER));                                        // E Y E is symmetric: lower triangle
    }
    if (!packed) join(h, 0, 2);
    join(h, 1, 3);
    CU(pack_apply_dense(h, S, st, r, S.Up, Q, done, L, packed));       // A(svec(E Y E + sym(Up Q^T)))
    launch_ap_finish<double>(st, m, d, n, r, S.partA, h->SA, nullptr, S.Vs, S.H, S.Dv, pin, gsub, out, mode, S.ctl,
                             h->dotbuf, h->counter, L, nullptr, 0, h->lin,   // + tau^-2 delta p_u
                             fuse_x(h, S), S.rv);
  } else if (h->kind == SDP_A_SPARSE_COO) {
    // Y = A^T(p_u) kept as its pattern values; E Y E only at the pattern positions
    sparse_posval(st, h->sp, pu, S.ypos, done, L);
    cudaStream_t s1 = fork(h, 1, 1);                                   // H = Vs^T (Y Q)
    sparse_sym_spmm(s1, h->sp, n, r, S.ypos, Q, n, S.Tm, n, done, L);
    CU(gemm_f64(s1, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, h->ws_b[1], h->ws_b_elems, L, done));
    // (S.F keeps E C~ of the right side for the recovery)
    sparse_EY(st, h->sp, n, S.ypos, S.E, S.Z, done, L);                   // E Y
    CU(sparse_pos_dots_col(st, h->sp, n, S.E, S.Z, S.zpos, done, L));     // (E Y E)_ab at the positions
    join(h, 0, 2);
    join(h, 1, 3);
    sparse_apply_pos(st, h->sp, n, m, r, S.zpos, S.Up, Q, S.partA, done, L);   // A(E Y E + sym(Up Q^T))
    launch_ap_finish<double>(st, m, d, n, r, S.partA, 1, nullptr, S.Vs, S.H, S.Dv, pin, gsub, out, mode, S.ctl,
                             h->dotbuf, h->counter, L, nullptr, 0, h->lin,   // + tau^-2 delta p_u
                             fuse_x(h, S), S.rv);
  } else {
    launch_diag_scale_rows<double>(st, n, r, pu, S.Vs, S.Tm, done, L);  // A^T(p_u) Q = diag(p_u) Q
    CU(gemm_big(h, st, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, S.ws, S.ws_elems, L, 0, done));
    rows_gemv<double>(st, S.EE, n, n, pu, S.partA, done, L);              // diag(E diag(p_u) E) = (E o E) p_u
    join(h, 0, 2);
    launch_ap_finish<double>(st, m, d, n, r, S.partA, rows_gemv_slabs(n, n), S.Up, S.Vs, S.H, S.Dv, pin, gsub, out,
                             mode, S.ctl, h->dotbuf, h->counter, L, nullptr, 0, nullptr,
                             fuse_x(h, S), S.rv);
  }
  return SDP_OK;
}

// The mixed form's operator M~: [A E A^T p_u + B p_v; B^T p_u - D p_v] with A E A^T p_u from the
// FP32 copies (FP32 products, FP32 accumulation inside each slab, FP64 sum of the slabs) and the
// B rows in FP64 from the explicit B, so that M~ and the preconditioner share their second block
// row exactly and the Prop. indefpcg invariant r_v = 0 survives (in the rounding of FP64).
sdp_status apply_operator_mixed(sdp_handle* h, Space& S, const double* pin, double* out, const double* gsub,
                                int mode) {
  const int n = h->n, m = h->m, d = h->d;
  const int32_t* done = &S.ctl->done;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  Mixed32& M = h->m32;
  const double* pu = pin;
  const double* pv = pin + m;
  if (h->kind == SDP_A_DIAG) {
    // the FP64 products with B from Vs, as in the FP64 operator, beside the FP32 (E o E) p_u
    const int n = h->n, r = h->r;
    cudaStream_t s0 = fork(h, 0, 0);
    h_unpack<double>(s0, n, r, pv, S.Hp, done, L);
    CU(gemm_big(h, s0, false, false, n, r, n, 1.0, S.Vs, n, S.Hp, n, 0.0, S.Up, n, h->ws_b[0], h->ws_b_elems, L, 0,
                done, 1));
    launch_to_float(st, m, pu, M.pu, done, L);
    int S32;
    if (M.EE16) {                                                            // (E o E) p_u, BF16 copy
      S32 = bf16_gemv_slabs(n, M.ldk);
      bf16_gemv(st, M.EE16, n, M.ldk, M.pu, M.partA, S32, done, L);
    } else {                                                                 // (E o E) p_u, FP32 copy
      rows_gemv<float>(st, M.EE, n, n, M.pu, M.partA, done, L);
      S32 = rows_gemv_slabs(n, n, 4);
    }
    launch_diag_scale_rows<double>(st, n, r, pu, S.Vs, S.Tm, done, L);
    CU(gemm_big(h, st, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, S.ws, S.ws_elems, L, 0, done));
    join(h, 0, 2);
    launch_ap_finish<double>(st, m, d, n, r, nullptr, 0, S.Up, S.Vs, S.H, S.Dv, pin, gsub, out, mode, S.ctl,
                             h->dotbuf, h->counter, L, M.partA, S32, nullptr,
                             fuse_x(h, S), S.rv);
    return SDP_OK;
  }
  // side branch: the FP64 rows with B, beside the FP32 A E A^T chain on the main stream
  cudaStream_t s0 = fork(h, 0, 0);
  rows_gemv<double>(s0, S.B, m, d, pv, M.partBv, done, L);                  // B p_v
  rows_gemv<double>(s0, S.Bt, d, m, pu, M.partBu, done, L);                 // B^T p_u
  launch_to_float(st, m, pu, M.pu, done, L);
  int SA;
  if (h->kind == SDP_A_DENSE_SVEC && h->lp == SDP_MIXED_FP32) {
    prof_begin(h, 2);
    // A^T(p_u); the FP32 pass has twice the row groups of the FP64 one, and a separate unpack
    // (all SMs) reduces them faster than the last CTA of each column block would
    rows_gemvT<float>(st, M.A, m, h->N, M.pu, M.partY, h->GY32, done, L);
    prof_end(h);
    svec_unpack_sum<float>(st, n, M.partY, h->GY32, 1.0, M.Y, done, L);
    CU(gemm_f32(st, false, false, n, n, n, 1.f, M.E, n, M.Y, n, 0.f, M.F, n, M.ws, M.ws_elems, L, done));
    CU(gemm_f32(st, false, false, n, n, n, 1.f, M.F, n, M.E, n, 0.f, M.Z, n, M.ws, M.ws_elems, L, done));
    svec_pack_plus<float>(st, n, 0, M.Z, nullptr, nullptr, M.zsvec, done, L);
    prof_begin(h, 3);
    rows_gemv<float>(st, M.A, m, h->N, M.zsvec, M.partA, done, L);          // A(E Y E)
    prof_end(h);
    SA = h->SA32;
  } else if (h->kind == SDP_A_DENSE_SVEC) {
    // TF32 / BF16 forms: Y = A^T(p_u) in the operand layout of the tensor cores, G = Y E and
    // Z = E G as tcgen05 products with FP32 accumulation, then A(Z)
    const bool bf = h->lp == SDP_MIXED_BF16;
    prof_begin(h, 2);
    if (bf) bf16_gemvT(st, M.A16, m, M.Lp, M.pu, M.partY, M.G16, done, L);
    else rows_gemvT<float>(st, M.A, m, h->N, M.pu, M.partY, h->GY32, done, L);
    prof_end(h);
    lp_unpack(st, n, M.partY, bf ? M.G16 : h->GY32, bf ? M.Lp : h->N, M.Ylp, M.ldk, bf, M.Ylo, done, L);
    // K runs over the whole pitch: the entries n .. ldk - 1 of every operand column are zero.
    // BF16: one kind::f16 product each; TF32: (hi, lo) operand pairs, three kind::tf32 MMAs a step
    const int mode = bf ? 0 : 2;
    CU(lp_gemm(st, mode, n, n, M.ldk, 1.f, M.Ylp, M.Ylo, M.ldk, M.Elp, M.Elo, M.ldk, M.Glp, M.Glo, M.ldk,
               bf ? 1 : 2, M.err, L, done));                                                          // G = Y E
    CU(lp_gemm(st, mode, n, n, M.ldk, 1.f, M.Elp, M.Elo, M.ldk, M.Glp, M.Glo, M.ldk, M.Z, nullptr, n, 0, M.err,
               L, done));                                                                              // Z = E G
    svec_pack_plus<float>(st, n, 0, M.Z, nullptr, nullptr, M.zsvec, done, L);
    prof_begin(h, 3);
    if (bf) {
      SA = bf16_gemv_slabs(m, M.Lp);
      bf16_gemv(st, M.A16, m, M.Lp, M.zsvec, M.partA, SA, done, L);          // A(E Y E)
    } else {
      rows_gemv<float>(st, M.A, m, h->N, M.zsvec, M.partA, done, L);
      SA = h->SA32;
    }
    prof_end(h);
  } else {
    rows_gemv<float>(st, M.EE, n, n, M.pu, M.partA, done, L);               // (E o E) p_u
    SA = rows_gemv_slabs(n, n, 4);
  }
  join(h, 0, 2);
  launch_mixed_finish(st, m, d, M.partA, SA, M.partBv, rows_gemv_slabs(m, d), M.partBu, rows_gemv_slabs(d, m), S.Dv, pin,
                      gsub, out, mode, S.ctl, h->dotbuf, h->counter, L, fuse_x(h, S), S.rv);
  return SDP_OK;
}

sdp_status apply_op(sdp_handle* h, Space& S, bool mixed, const double* pin, double* out, const double* gsub,
                    int mode) {
  return mixed ? apply_operator_mixed(h, S, pin, out, gsub, mode) : apply_operator(h, S, pin, out, gsub, mode);
}

// z = P^{-1} rin (Section 6), then <r, z>; mode 0 sets rz, mode 1 computes the PCG beta.
sdp_status apply_precond(sdp_handle* h, Space& S, const double* rin, double* zout, int mode) {
  const int m = h->m, d = h->d;
  const int32_t* done = &S.ctl->done;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  const int Sm = rows_gemv_slabs(d, m);   // slabs of the products with the rows of B^T
  if (h->kind == SDP_A_SPARSE_COO) {
    // the products with B through the pattern: B t = A(sym(Vs unpack(t) Q^T)) and
    // B^T u = pack(Vs^T (A^T(u) Q)), A^T(u) kept as its pattern values
    const int n = h->n, r = h->r;
    const double* Q = S.Vs;
    if (h->space == 1) {
      if (h->lin) launch_lin_div(st, m, rin, h->lin_lam, S.wm, S.ctl, L);   // Lam^{-1} r_u (linear block)
      sparse_posval(st, h->sp, h->lin ? S.wm : rin, S.ypos, done, L);
      sparse_sym_spmm(st, h->sp, n, r, S.ypos, Q, n, S.Tm, n, done, L);
      CU(gemm_big(h, st, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, S.ws, S.ws_elems, L, 0, done));
      launch_pc_d_s_H(st, m, d, n, r, S.H, rin, S.sd, S.ctl, L, h->lin != nullptr);   // s = r_v - B^T Lam^{-1} r_u
      rows_gemv<double>(st, S.Pinv, d, d, S.sd, S.partC, done, L);          // C^{-1} s
      launch_pc_d_zv<double>(st, m, d, rows_gemv_slabs(d, d), S.partC, zout, S.ctl, L);   // z_v = -C^{-1} s
      h_unpack<double>(st, n, r, zout + m, S.Hp, done, L);
      CU(gemm_big(h, st, false, false, n, r, n, 1.0, S.Vs, n, S.Hp, n, 0.0, S.Up, n, S.ws, S.ws_elems, L, 0, done));
      sparse_apply_pos(st, h->sp, n, m, r, nullptr, S.Up, Q, S.partA, done, L);  // B z_v
      launch_pc_zu_dot<double>(st, m, d, 1, S.partA, 1, rin, zout, mode, S.ctl, h->dotbuf, h->counter, L,
                               h->lin ? h->lin_lam : nullptr, h->fuse ? S.p : nullptr);
    } else {
      h_unpack<double>(st, n, r, rin + m, S.Hp, done, L, S.Dv);            // unpack(D^{-1} r_v)
      CU(gemm_big(h, st, false, false, n, r, n, 1.0, S.Vs, n, S.Hp, n, 0.0, S.Up, n, S.ws, S.ws_elems, L, 0, done));
      sparse_apply_pos(st, h->sp, n, m, r, nullptr, S.Up, Q, S.partA, done, L);
      launch_pc_m_w<double>(st, m, 1, S.partA, rin, S.wm, S.ctl, L);      // w = r_u + B D^{-1} r_v
      rows_gemv<double>(st, S.Pinv, m, m, S.wm, S.partC, done, L);         // K^{-1} w
      launch_pc_m_w<double>(st, m, rows_gemv_slabs(m, m), S.partC, nullptr, zout, S.ctl, L);  // z_u
      sparse_posval(st, h->sp, zout, S.ypos, done, L);
      sparse_sym_spmm(st, h->sp, n, r, S.ypos, Q, n, S.Tm, n, done, L);
      CU(gemm_big(h, st, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, S.ws, S.ws_elems, L, 0, done));
      launch_diag_zv(st, m, d, n, r, S.H, rin, S.Dv, zout, S.ctl, L);      // z_v = D^{-1}(B^T z_u - r_v)
      launch_pc_zu_dot<double>(st, m, d, 0, nullptr, 2, rin, zout, mode, S.ctl, h->dotbuf, h->counter, L, nullptr, h->fuse ? S.p : nullptr);
    }
  } else if (pc_coop_on(h)) {
    // the three products and the dot in one cooperative launch (grid barriers between them); in
    // the PCG loop it also takes the update of x and r (the operator's finishing kernel skips it)
    const bool upd = h->fuse && mode == 1 && rin == S.rv;
    CU(launch_pc_dense_d_coop(st, m, d, S.Bt, S.Pinv, S.B, upd ? S.rv : const_cast<double*>(rin), zout, S.sd,
                              h->dotbuf, mode, S.ctl, h->fuse ? S.p : nullptr, upd ? S.x : nullptr,
                              upd ? S.Ap : nullptr, L));
  } else if (h->space == 1) {
    if (h->lin) {   // linear block: s = r_v - B^T (Lam^{-1} r_u), z_u = Lam^{-1}(r_u - B z_v)
      launch_lin_div(st, m, rin, h->lin_lam, S.wm, S.ctl, L);
      rows_gemv<double>(st, S.Bt, d, m, S.wm, S.partB, done, L);
      rows_gemv_formed(st, S.Pinv, d, d, rin + m, S.partB, Sm, -1.0, nullptr, nullptr, S.partC, done, L);
    } else {
      rows_gemv<double>(st, S.Bt, d, m, rin, S.partB, done, L);            // B^T r_u (rows of B^T)
      // C^{-1} s with s = r_v - beta^{-1} B^T r_u formed while staged
      rows_gemv_formed(st, S.Pinv, d, d, rin + m, S.partB, Sm, -1.0, &S.ctl->beta_pc, nullptr, S.partC, done, L);
    }
    // B z_v with z_v = -(C^{-1} s) formed while staged and stored
    rows_gemv_formed(st, S.B, m, d, nullptr, S.partC, rows_gemv_slabs(d, d), -1.0, nullptr, zout + m, S.partA, done,
                     L);
    launch_pc_zu_dot<double>(st, m, d, rows_gemv_slabs(m, d), S.partA, 1, rin, zout, mode, S.ctl, h->dotbuf,
                             h->counter, L, h->lin ? h->lin_lam : nullptr, h->fuse ? S.p : nullptr);
  } else if (h->kind == SDP_A_DIAG) {
    // the products with B from Vs: B t = rowdot(Vs unpack(t), Q), B^T u = pack(Vs^T diag(u) Q)
    const int n = h->n, r = h->r;
    const double* Q = S.Vs;
    h_unpack<double>(st, n, r, rin + m, S.Hp, done, L, S.Dv);              // unpack(D^{-1} r_v)
    CU(gemm_big(h, st, false, false, n, r, n, 1.0, S.Vs, n, S.Hp, n, 0.0, S.Up, n, S.ws, S.ws_elems, L, 0, done));
    launch_diag_w(st, n, r, S.Up, Q, rin, S.wm, S.ctl, L);                 // w = r_u + B D^{-1} r_v
    rows_gemv<double>(st, S.Pinv, m, m, S.wm, S.partC, done, L);           // K^{-1} w
    launch_pc_m_w<double>(st, m, rows_gemv_slabs(m, m), S.partC, nullptr, zout, S.ctl, L);  // z_u
    launch_diag_scale_rows<double>(st, n, r, zout, S.Vs, S.Tm, done, L);  // diag(z_u) Q
    CU(gemm_big(h, st, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, S.ws, S.ws_elems, L, 0, done));
    launch_diag_zv(st, m, d, n, r, S.H, rin, S.Dv, zout, S.ctl, L);        // z_v = D^{-1}(B^T z_u - r_v)
    launch_pc_zu_dot<double>(st, m, d, 0, nullptr, 2, rin, zout, mode, S.ctl, h->dotbuf, h->counter, L, nullptr, h->fuse ? S.p : nullptr);
  } else {
    launch_pc_m_tv<double>(st, m, d, rin, S.Dv, S.sd, S.ctl, L);           // t = D^{-1} r_v
    rows_gemv<double>(st, S.B, m, d, S.sd, S.partA, done, L);              // B t
    launch_pc_m_w<double>(st, m, rows_gemv_slabs(m, d), S.partA, rin, S.wm, S.ctl, L);   // w = r_u + B D^{-1} r_v
    rows_gemv<double>(st, S.Pinv, m, m, S.wm, S.partC, done, L);           // K^{-1} w
    launch_pc_m_w<double>(st, m, rows_gemv_slabs(m, m), S.partC, nullptr, zout, S.ctl, L);  // z_u
    rows_gemv<double>(st, S.Bt, d, m, zout, S.partBt, done, L);            // B^T z_u (rows of B^T)
    launch_pc_m_zv<double>(st, m, d, Sm, S.partBt, rin, S.Dv, zout, S.ctl, L);  // z_v = D^{-1}(B^T z_u - r_v)
    launch_pc_zu_dot<double>(st, m, d, 0, nullptr, 2, rin, zout, mode, S.ctl, h->dotbuf, h->counter, L, nullptr, h->fuse ? S.p : nullptr);
  }
  return SDP_OK;
}

// r0 = g - M x (given), stop test, z0 = P^{-1} r0, p0 = z0.  rel_rtol2 > 0 sets a relative threshold.
sdp_status pcg_start(sdp_handle* h, Space& S, bool mixed, const double* gsub, double rel_rtol2) {
  sdp_status s = apply_op(h, S, mixed, S.x, S.rv, gsub, 0);
  if (s != SDP_OK) return s;
  launch_norm_check<double>(h->st, h->m + h->d, S.rv, rel_rtol2, S.ctl, h->dotbuf, h->counter, &h->launches);
  s = apply_precond(h, S, S.rv, S.z, 0);
  if (s != SDP_OK) return s;
  launch_p_update<double>(h->st, h->m + h->d, S.z, S.p, 1, S.ctl, &h->launches);
  return SDP_OK;
}

// PCG iterations until the device stop flag is set: one launch of a graph whose WHILE node
// repeats one iteration while the flag is clear or, where that graph is refused, replays of a
// captured graph of `check_every` iterations (every kernel returns at once after the stop),
// with one host read of the control block between replays.
sdp_status krylov_loop(sdp_handle* h, Space& S, bool mixed, bool minres) {
  const int every = h->opt.check_every;
  const int nt = h->m + h->d;
  Graph& G = h->graph[minres ? 2 : mixed ? 1 : 0];
  // short vectors: the PCG update and p = z + beta p run in the last block of the operator's and
  // the preconditioner's finishing kernels (two launches fewer per iteration)
  h->fuse = !minres && nt <= kFuseMax;
  int64_t* L = &h->launches;
  cudaStream_t st = h->st;
  CU(cudaMemcpyAsync(h->ctl_host, S.ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (h->prof) {   // launches recorded so far (outside any graph) are complete: collect them
    sdp_status ps = prof_collect(h, h->prof_base, h->prof_entries.size(), 0, 1);
    if (ps != SDP_OK) return fail(h, ps, "event timing failed");
  }
  h->prof_entries.clear();
  h->prof_base = 0;
  auto chunk = [&](cudaStream_t s_, int iters) -> sdp_status {
    cudaStream_t saved = h->st;
    h->st = s_;
    for (int k = 0; k < iters; ++k) {
      h->cur_iter = k;
      if (minres) {
        // v = r2 / beta; y = M v; alfa; beta, rotation, stop; w and x (r1 = rv, r2 = z, v = p, y = Ap)
        launch_minres_v(s_, nt, S.z, S.p, h->mctl, S.ctl, L);
        sdp_status s = apply_operator(h, S, S.p, S.Ap, nullptr, 0);
        if (s != SDP_OK) { h->st = saved; return s; }
        launch_minres_alfa(s_, nt, S.p, S.Ap, S.rv, h->mctl, S.ctl, h->dotbuf, h->counter, L);
        launch_minres_beta(s_, nt, S.Ap, S.rv, S.z, h->mctl, S.ctl, h->dotbuf, h->counter, L);
        launch_minres_update(s_, nt, S.p, S.mw, S.mw1, S.mw2, S.x, h->mctl, S.ctl, L);
        continue;
      }
      sdp_status s = apply_op(h, S, mixed, S.p, S.Ap, nullptr, 1);
      if (s != SDP_OK) { h->st = saved; return s; }
      if (!h->fuse) launch_update<double>(s_, nt, S.x, S.rv, S.p, S.Ap, S.ctl, h->dotbuf, h->counter, L);
      s = apply_precond(h, S, S.rv, S.z, 1);
      if (s != SDP_OK) { h->st = saved; return s; }
      if (!h->fuse) launch_p_update<double>(s_, nt, S.z, S.p, 0, S.ctl, L);
    }
    h->st = saved;
    h->cur_iter = -1;
    return SDP_OK;
  };
  const int key[4] = {h->r, h->d, h->space, every * 2 + (h->prof ? 1 : 0)};
  // The whole loop as one graph: a WHILE conditional node around one iteration, its condition set
  // on the device from the stop flag, so no host read between iterations and no iteration past the
  // stop.  Built once per shape; where the device or the driver refuses it (capture or
  // instantiation fails), the handle keeps the replays of `check_every` iterations below.
  if (!h->ctl_host->done && h->opt.use_graph && !h->prof && !minres && h->while_ok) {
    if (G.wexec && std::memcmp(key, G.wkey, sizeof(key)) != 0) {
      cudaGraphExecDestroy(G.wexec);
      G.wexec = nullptr;
    }
    if (!G.wexec) {
      if (!h->cap_stream) CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      const int64_t before = h->launches;
      cudaGraph_t g = nullptr;
      bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
      cudaGraphConditionalHandle hc{};
      cudaGraph_t body = nullptr;
      if (ok) ok = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
      if (ok) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        ok = cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
        if (ok) body = cp.conditional.phGraph_out[0];
      }
      if (ok) ok = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        h->capturing = true;
        sdp_status cs = chunk(h->cap_stream, 1);
        if (cs == SDP_OK) launch_loop_cond(h->cap_stream, hc, S.ctl, h->loop_guard, L);
        h->capturing = false;
        cudaGraph_t out = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &out);
        ok = cs == SDP_OK && ce == cudaSuccess;
      }
      if (ok) ok = cudaGraphInstantiate(&G.wexec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      G.wlaunches = h->launches - before;
      h->launches = before;
      if (!ok) {
        cudaGetLastError();
        if (G.wexec) cudaGraphExecDestroy(G.wexec);
        G.wexec = nullptr;
        h->while_ok = false;
      } else {
        std::memcpy(G.wkey, key, sizeof(key));
      }
    }
    if (G.wexec) {
      const int it0 = h->ctl_host->iters;
      CU(cudaMemsetAsync(h->loop_guard, 0, sizeof(int), st));
      CU(cudaGraphLaunch(G.wexec, st));
      CU(cudaMemcpyAsync(h->ctl_host, S.ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      h->launches += 1 + G.wlaunches * std::max(1, h->ctl_host->iters - it0);
      // a loop the guard ended without the stop flag continues below, replay by replay
    }
  }
  if (!h->ctl_host->done && h->opt.use_graph) {
    if (!G.exec || std::memcmp(key, G.key, sizeof(key)) != 0) {
      if (G.exec) { cudaGraphExecDestroy(G.exec); G.exec = nullptr; }
      if (!h->cap_stream) CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      const int64_t before = h->launches;
      const size_t prof_before = h->prof_entries.size();
      CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      h->capturing = true;
      sdp_status s = chunk(h->cap_stream, every);
      h->capturing = false;
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
      if ((s != SDP_OK || ce != cudaSuccess) && h->coop_pc) {
        // a cooperative launch that stream capture does not take: capture again without it
        if (graph) cudaGraphDestroy(graph);
        graph = nullptr;
        cudaGetLastError();
        h->coop_pc = false;
        h->launches = before;
        h->prof_entries.resize(prof_before);
        CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        s = chunk(h->cap_stream, every);
        h->capturing = false;
        ce = cudaStreamEndCapture(h->cap_stream, &graph);
      }
      if (s != SDP_OK) { if (graph) cudaGraphDestroy(graph); return s; }
      if (ce != cudaSuccess) return fail(h, SDP_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&G.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return fail(h, SDP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
      std::memcpy(G.key, key, sizeof(key));
      G.launches = h->launches - before;
      h->launches = before;
      G.prof_first = 0;
      G.prof_last = h->prof_entries.size();
      G.entries = h->prof_entries;
    }
  }
  int base = 0;
  while (!h->ctl_host->done) {
    size_t first = 0, last = 0;
    if (h->opt.use_graph) {
      CU(cudaGraphLaunch(G.exec, st));
      h->launches += G.launches;
      first = G.prof_first;
      last = G.prof_last;
    } else {
      h->prof_entries.clear();
      sdp_status s = chunk(st, every);
      if (s != SDP_OK) return s;
      last = h->prof_entries.size();
    }
    CU(cudaMemcpyAsync(h->ctl_host, S.ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h->prof) {
      sdp_status ps = h->opt.use_graph ? prof_collect(h, first, last, base, h->ctl_host->iters, &G.entries)
                                       : prof_collect(h, first, last, base, h->ctl_host->iters);
      if (ps != SDP_OK) return fail(h, ps, "event timing failed");
    }
    base += every;
  }
  h->fuse = false;
  // later profiled launches take events after the ones the graph records into
  h->prof_entries.assign(h->opt.use_graph ? G.prof_last : 0, ProfEntry{0, 0});
  h->prof_base = h->prof_entries.size();
  return SDP_OK;
}

}  // namespace

namespace {

// One Newton solve; with `reuse` the split and the preconditioner core (a1, a2) of the previous
// solve on this handle are kept (a second right side at the same scaling point).
sdp_status newton_solve_impl(sdp_handle* h, const double* V, const double* lam, const double* Ct, const double* bt,
                             double* dX, double* dy, double* dS, sdp_newton_info* info, bool reuse) {
  h->launches = 0;
  NvtxRange range_solve("sdp newton solve");
  NvtxPhase phase(reuse ? "a1-a2 setup (reused)" : "a1-a2 split and preconditioner core");
  const int n = h->n, m = h->m;
  cudaStream_t st = h->st;
  int64_t* L = &h->launches;
  Space& S = h->s64;
  const size_t ws = S.ws_elems;
  h->prof_entries.clear();
  h->prof_base = 0;
  h->cur_iter = -1;
  for (int k = 0; k < 4; ++k) { h->prof_ms[k] = 0.0; h->prof_n[k] = 0; }
  h->refine_steps = 0;
  h->inner_iters = 0;
  h->refine_rate = 0.0;
  h->refine_rr0 = 0.0;
  if (!h->ev_phase[0])
    for (auto& e : h->ev_phase) CU(cudaEventCreate(&e));
  CU(cudaEventRecord(h->ev_phase[0], st));

  if (reuse) {
    // the control block keeps r, d, tau, beta and s_A of the last setup; its counters restart
    PcgCtl c = h->setup_ctl;
    c.done = 0;
    c.iters = 0;
    c.status = 0;
    c.max_iters = h->opt.max_pcg;
    CU(cudaMemcpyAsync(h->ctl, &c, sizeof(PcgCtl), cudaMemcpyHostToDevice, st));
    CU(cudaEventRecord(h->ev_phase[1], st));
  }
  int r = h->r, d = h->d;
  bool rhs_side = false;   // the right side's products run beside the preconditioner setup
  int rhs_slabs = 0;       // DIAG: slabs of diag(F E) left in S.Y by the side stream
  if (!reuse) {
  h->setup_valid = false;
  // ---- a1: split ----
  PcgCtl init{};
  init.s_A = h->s_A;
  init.max_iters = h->opt.max_pcg;
  init.done = 0;
  CU(cudaMemcpyAsync(h->ctl, &init, sizeof(PcgCtl), cudaMemcpyHostToDevice, st));
  split_sort(st, n, V, lam, S.Vs, h->lam_s, L);
  split_params(st, n, h->opt.r_fixed, h->opt.r_hat, h->opt.beta_rule, h->lam_s, h->e, h->ctl, L);
  if (h->opt.precond_space == 3 && h->lin) launch_lin_free_count(st, m, h->lin, kLinDominance, h->ctl, L);
  CU(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (h->ctl_host->status != 0) return fail(h, SDP_EINVAL, "eigenvalues must be positive and finite, 1 <= r < n");
  r = h->ctl_host->r;
  d = h->ctl_host->d;
  if (r > h->r_max) return fail(h, SDP_EINVAL, "rank above the setup maximum");
  h->r = r;
  h->d = d;
  if (h->opt.precond_space == 3) {
    // with the linear block: the m-space complement when fewer than d rows are free of their
    // slack (the d-space elimination rests on those rows and loses the direction to rounding at
    // small mu, where the m-space complement is nearly diagonal on the fixed rows); else the
    // smaller space
    h->space = h->lin ? (h->ctl_host->m_free < d ? 2 : 1) : (d <= m ? 1 : 2);
  } else {
    h->space = h->opt.precond_space == 0 ? (d <= m ? 1 : 2) : h->opt.precond_space;
  }
  h->vs_sl[0].valid = h->vs_sl[1].valid = false;
  if (h->vs_mem[0]) {   // slices of Vs (rows of Vs and of Vs^T) for every tensor-core product with it
    CU(tc_make_slices(st, n, n, S.Vs, 1, n, h->vs_mem[0], &h->vs_sl[0], L));
    CU(tc_make_slices(st, n, n, S.Vs, n, 1, h->vs_mem[1], &h->vs_sl[1], L));
  }
  split_scale_cols(st, n, S.Vs, h->e, h->Ve, L);
  // E = Ve Vs^T is symmetric: the lower triangle by the product, the upper by a mirror
  CU(gemm_big(h, st, false, true, n, n, n, 1.0, h->Ve, n, S.Vs, n, 0.0, S.E, n, S.ws, ws, L, GEMM_LOWER));
  lower_to_full(st, n, S.E, L);
  // digits of E's columns (E is symmetric: its rows too) for every E Y E of this solve
  S.ed_valid = S.Ed && h->fx && n < kTcMin && fx_col_digits(st, n, S.E, S.Ed, S.eE, L);
  if (h->mixed) h->sin.ed_valid = S.ed_valid;
  split_sigma(st, n, r, h->lam_s, h->ctl, S.Dv, L);

  // ---- a3 products on a side stream, beside a2 (DENSE kind, FP64 MMA products): the right side
  // needs E, Q and D only, and the factorisation of a2 is a chain of small launches that leaves
  // most of the GPU idle.  The finishing kernel (which reads the factorisation's status) stays on
  // the handle's stream after the join.
  rhs_side = !h->prof && (h->kind == SDP_A_DENSE_SVEC || h->kind == SDP_A_DIAG) && n < kTcMin &&
             h->opt.krylov != 1;
  if (rhs_side) {
    cudaStream_t s0 = fork(h, 0, 4);
    CU(gemm_big(h, s0, false, false, n, n, n, 1.0, S.E, n, Ct, n, 0.0, S.F, n, h->ws_b[0], h->ws_b_elems, L));
    CU(gemm_big(h, s0, false, false, n, r, n, 1.0, Ct, n, S.Vs, n, 0.0, S.Tm, n, h->ws_b[0], h->ws_b_elems, L));
    CU(gemm_big(h, s0, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, h->ws_b[0], h->ws_b_elems, L));
    if (h->kind == SDP_A_DIAG) {   // A(E C~ E) = diag(F E) in slabs, into S.Y (free until the recovery)
      rhs_slabs = launch_diag_FE(s0, n, S.F, S.E, S.Y, n, L);
    } else {
      CU(gemm_big(h, s0, false, false, n, n, n, 1.0, S.F, n, S.E, n, 0.0, S.Z, n, h->ws_b[0], h->ws_b_elems, L,
                  GEMM_LOWER));
      CU(pack_apply_dense(h, S, s0, r, nullptr, nullptr, nullptr, L));
    }
  }

  // ---- a2: B = A Q and the preconditioner core (MINRES: only E o E of the DIAG operator) ----
  if (h->opt.krylov == 1) {
    if (h->kind == SDP_A_DIAG) launch_hadamard_sq(st, (int64_t)n * n, S.E, S.EE, L);
  } else if (h->kind == SDP_A_DENSE_SVEC) {
    // row i of B is Q^T svec(A_i) = pack(Vs^T A_i Q): G = [A_i Q] straight from the svec rows,
    // then one GEMM H = Vs^T G for a whole batch of constraints
    bool direct = true;
    for (int i0 = 0; i0 < m && direct; i0 += h->mb2) {
      const int mb = std::min(h->mb2, m - i0);
      direct = (h->fx && fx_AiQ(st, h->a_fx, h->a_fx_e, n, fx_row_len(h->N), i0, mb, r, S.Vs, h->Gb, L)) ||
               dense_AiQ(st, h->a_dense, n, i0, mb, r, S.Vs, h->Gb, L);
      if (!direct) break;
      CU(gemm_big(h, st, true, false, n, mb * r, n, 1.0, S.Vs, n, h->Gb, n, 0.0, h->Hb, n, S.ws, ws, L));
      h_pack_rows(st, n, r, mb, i0, h->Hb, S.B, d, S.Bt, m, L);
    }
    if (!direct) {   // n r too large for the shared-memory accumulators: unpack, then GEMM
      for (int i0 = 0; i0 < m; i0 += h->mb) {
        const int mb = std::min(h->mb, m - i0);
        svec_rows_unpack(st, h->a_dense, n, i0, mb, h->ubatch, L);
        // Gb (mb n x r) = [A_i] Q ; Hb (n x mb r) = Vs^T Gb viewed n x (mb r)
        CU(gemm_f64(st, false, false, mb * n, r, n, 1.0, h->ubatch, (int64_t)mb * n, S.Vs, n, 0.0, h->Gb,
                    (int64_t)mb * n, S.ws, ws, L));
        CU(gemm_f64(st, true, false, n, mb * r, n, 1.0, S.Vs, n, h->Gb, n, 0.0, h->Hb, n, S.ws, ws, L));
        h_pack_rows(st, n, r, mb, i0, h->Hb, S.B, d, S.Bt, m, L);
      }
    }
  } else if (h->kind == SDP_A_SPARSE_COO) {
    if (!gram_on(h)) sparse_B(st, h->sp, n, m, r, S.Vs, S.B, d, S.Bt, m, L);   // else C needs no B
  } else {
    launch_hadamard_sq(st, (int64_t)n * n, S.E, S.EE, L);
    if (h->space == 1) {
      if ((int64_t)m * d > h->b_elems) return fail(h, SDP_EINVAL, "d-space core larger than the setup allows");
      h_pack_rows_diag(st, n, r, S.Vs, S.B, d, S.Bt, m, L);
    }
  }
  int32_t* pstatus = &h->ctl->status;
  const int pd = (h->space == 1) ? d : m;
  if (h->lin) launch_lin_lam(st, m, h->lin, h->ctl, h->lin_lam, L);   // Lam = beta + tau^-2 delta
  if (h->opt.krylov == 1) {
    // MINRES (Cor. minres): no preconditioner core
  } else if (pd > h->pinv_dim) {
    return fail(h, SDP_EINVAL, "preconditioner core larger than the setup allows");
  } else if (h->kind == SDP_A_DIAG && h->space == 2) {
    // K = beta I + tau^-2 G o (G + 2 tau E) with G = Q (Lam - tau I) Q^T (lower triangle), in
    // buffers the right side's products (perhaps running beside) do not use
    launch_shift_cols(st, n, r, S.Vs, h->lam_s, h->ctl, S.Hp, L);
    CU(gemm_big(h, st, false, true, n, n, r, 1.0, S.Hp, n, S.Vs, n, 0.0, S.Z, n, S.ws, ws, L, GEMM_LOWER));
    launch_diag_K(st, n, S.Z, S.E, h->ctl, S.Pinv, L);
    CU(spd_inverse_any(h, st, m, S.Pinv, S.ws, ws, pstatus, L));
  } else if (h->space == 1) {
    // C = beta^{-1} B^T B + tau^2 Sigma  (B row-major m x d == column-major d x m); with a linear
    // block, C = B^T Lam^{-1} B + tau^2 Sigma
    if (gram_on(h)) {
      // Gram form: C = sum_i s_i pack(H_i) pack(H_i)^T with H_i = Vs^T A_i Q, by column pairs
      // (j1, j2) of the H_i: G = Vs^T W_{j1 j2} Vs over the sparse W of the constraints' term
      // pairs, scattered into C through the h-coordinate map
      CU(cudaMemsetAsync(S.Pinv, 0, (size_t)d * d * sizeof(double), st));
      const double ib = 1.0 / h->ctl_host->beta_pc;
      for (int j1 = 0; j1 < r; ++j1)
        for (int j2 = j1; j2 < r; ++j2) {   // G_{j2 j1} = G_{j1 j2}^T: the scatter mirrors it
          // (S.F and S.Z as scratch: S.Y must stay zero off the pattern for the sparse A^T(.))
          sparse_gram_spmm(st, h->sp, n, j1, j2, S.Vs, ib, h->lin ? h->lin_lam : nullptr, S.F, L);
          CU(gemm_big(h, st, true, false, n, n, n, 1.0, S.Vs, n, S.F, n, 0.0, S.Z, n, S.ws, ws, L));
          sparse_gram_scatter(st, n, r, j1, j2, j2 != j1, S.Z, S.Pinv, d, L);
        }
    } else if (h->lin) {
      launch_lin_scale_rows(st, m, d, S.B, h->lin_lam, h->lin_Bw, L);
      CU(gemm_big(h, st, false, true, d, d, m, 1.0, h->lin_Bw, d, h->lin_Bw, d, 0.0, S.Pinv, d, S.ws, ws, L,
                  GEMM_LOWER));
    } else {
      const double beta = h->ctl_host->beta_pc;
      CU(gemm_big(h, st, false, true, d, d, m, 1.0 / beta, S.B, d, S.B, d, 0.0, S.Pinv, d, S.ws, ws, L,
                  GEMM_LOWER));   // the Cholesky reads the lower triangle only
    }
    launch_add_diag(st, d, S.Pinv, S.Dv, 0.0, L);
    CU(spd_inverse_any(h, st, d, S.Pinv, S.ws, ws, pstatus, L));
  } else {
    // K = beta I + B D^{-1} B^T = Bs^T Bs + beta I with Bs = D^{-1/2} B^T (d x m)
    if ((int64_t)m * d > h->bs_elems) return fail(h, SDP_EINVAL, "m-space core larger than the setup allows");
    launch_scale_B(st, m, d, S.B, S.Dv, h->Bs, L);
    CU(gemm_big(h, st, true, false, m, m, d, 1.0, h->Bs, d, h->Bs, d, 0.0, S.Pinv, m, S.ws, ws, L, GEMM_LOWER));
    launch_add_diag(st, m, S.Pinv, h->lin ? h->lin_lam : nullptr, h->lin ? 0.0 : h->ctl_host->beta_pc, L);  // + Lam
    CU(spd_inverse_any(h, st, m, S.Pinv, S.ws, ws, pstatus, L));
  }
  if (h->mixed) {   // low-precision copies for the A E A^T block of the mixed operator
    Mixed32& M = h->m32;
    if (S.EE && M.EE16) lp_convert(st, n, n, S.EE, n, M.EE16, M.ldk, true, nullptr, L);
    else if (S.EE) convert<float, double>(st, (int64_t)n * n, S.EE, M.EE, L);
    else if (M.Elp) lp_convert(st, n, n, S.E, n, M.Elp, M.ldk, h->lp == SDP_MIXED_BF16, M.Elo, L);
    else convert<float, double>(st, (int64_t)n * n, S.E, M.E, L);
  }
  CU(cudaEventRecord(h->ev_phase[1], st));
  CU(cudaMemcpyAsync(&h->setup_ctl, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  }   // !reuse
  const int nt = m + d;

  // ---- a3: right-hand side and start ----
  phase.next("a3 right side");
  const double* Q = S.Vs;
  if (rhs_side) {
    join(h, 0, 5);
  } else {
    CU(gemm_big(h, st, false, false, n, n, n, 1.0, S.E, n, Ct, n, 0.0, S.F, n, S.ws, ws, L));
    CU(gemm_big(h, st, false, false, n, r, n, 1.0, Ct, n, Q, n, 0.0, S.Tm, n, S.ws, ws, L));
    CU(gemm_big(h, st, true, false, n, r, n, 1.0, S.Vs, n, S.Tm, n, 0.0, S.H, n, S.ws, ws, L));
  }
  if (h->kind == SDP_A_DENSE_SVEC) {
    if (!rhs_side) {
      CU(gemm_big(h, st, false, false, n, n, n, 1.0, S.F, n, S.E, n, 0.0, S.Z, n, S.ws, ws, L, GEMM_LOWER));
      CU(pack_apply_dense(h, S, st, r, nullptr, nullptr, nullptr, L));
    }
    launch_rhs_finish(st, m, d, n, r, S.partA, h->SA, nullptr, nullptr, bt, Ct, S.H, S.Dv, h->g, S.x,
                      h->opt.newton_rtol, h->ctl, h->dotbuf, h->counter, L);
  } else if (h->kind == SDP_A_SPARSE_COO) {
    CU(sparse_pos_dots_col(st, h->sp, n, S.E, S.F, S.zpos, nullptr, L));  // E C~ E at the positions
    sparse_apply_pos(st, h->sp, n, m, r, S.zpos, nullptr, nullptr, S.partA, nullptr, L);   // A(E C~ E)
    launch_rhs_finish(st, m, d, n, r, S.partA, 1, nullptr, nullptr, bt, Ct, S.H, S.Dv, h->g, S.x,
                      h->opt.newton_rtol, h->ctl, h->dotbuf, h->counter, L);
  } else {   // DIAG: A(E C~ E) = diag(F E), summed in slabs over the whole GPU
    if (!rhs_side) rhs_slabs = launch_diag_FE(st, n, S.F, S.E, S.Y, n, L);
    if (!small_pcg_on(h))   // else the cluster solve finishes the right side itself
      launch_rhs_finish(st, m, d, n, r, S.Y, rhs_slabs, nullptr, nullptr, bt, Ct, S.H, S.Dv, h->g, S.x,
                        h->opt.newton_rtol, h->ctl, h->dotbuf, h->counter, L);
  }

  phase.next("a4-a7 Krylov solve");
  if (h->opt.krylov == 1) {
    // ---- Cor. minres: MINRES_k(augsys, g, I, 0) ----
    launch_minres_init(st, nt, h->g, S.rv, S.z, S.x, S.mw, S.mw2, h->mctl, h->ctl, h->dotbuf, h->counter, L);
    sdp_status s = krylov_loop(h, S, false, true);
    if (s != SDP_OK) return s;
  } else if (!h->mixed) {
    // ---- a4-a6: FP64 PCG from x0 ----
    bool small = small_pcg_on(h);
    if (small) {   // the whole solve in one cluster launch
      const cudaError_t e = launch_small_pcg(st, n, r, d, h->opt.pcg_start == 0 ? 1 : 0, S.Vs, S.EE, S.Pinv, S.Dv,
                                             S.Y, rhs_slabs, bt, Ct, S.H, h->opt.newton_rtol, h->g, S.x, S.rv,
                                             S.z, S.p, S.Ap, S.ctl, L);
      if (e != cudaSuccess) {   // refused on this device (launch configuration): the launch chain
        cudaGetLastError();
        h->small_ok = false;
        small = false;
        launch_rhs_finish(st, m, d, n, r, S.Y, rhs_slabs, nullptr, nullptr, bt, Ct, S.H, S.Dv, h->g, S.x,
                          h->opt.newton_rtol, h->ctl, h->dotbuf, h->counter, L);
      }   // no host read here: the recovery reads the scalars on the device, the host at the end
    }
    if (!small) {
      if (h->opt.pcg_start == 0) {   // x0 = P^{-1}[0; g_v]: P x0 = [0; g_v], so r0_v = 0 with r0_u ~ g
        launch_correction_rhs(st, m, d, h->g, S.z, L);
        sdp_status s0 = apply_precond(h, S, S.z, S.x, 0);
        if (s0 != SDP_OK) return s0;
      }
      sdp_status s = pcg_start(h, S, false, h->g, 0.0);
      if (s != SDP_OK) return s;
      s = krylov_loop(h, S, false, false);
      if (s != SDP_OK) return s;
    }
  } else {
    // ---- a7: FP64 refinement around solves with the mixed operator ----
    // x starts at 0, so that rho_0 = g and the first correction starts at P^{-1}[0; g_v]: the
    // second block of the residual vanishes as Cor. pcg asks, without the large first block
    // that x0 = [0; -Sigma^{-1} Q^T c] leaves (it sets the floor of the true residual).
    Space& Si = h->sin;
    CU(cudaMemsetAsync(S.x, 0, nt * sizeof(double), st));
    bool fallback = false;
    for (;;) {
      // rho = g - M x in FP64, and the stop test on ||rho|| (the true residual)
      if (h->refine_steps == 0) {
        CU(cudaMemcpyAsync(S.rv, h->g, nt * sizeof(double), cudaMemcpyDeviceToDevice, st));
      } else {
        sdp_status s = apply_operator(h, S, S.x, S.rv, h->g, 0);
        if (s != SDP_OK) return s;
      }
      launch_norm_check<double>(st, nt, S.rv, 0.0, h->ctl, h->dotbuf, h->counter, L);
      CU(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      if (h->refine_steps == 0) h->refine_rr0 = h->ctl_host->rr;
      else h->refine_rate = std::pow(std::sqrt(h->ctl_host->rr / h->refine_rr0), 1.0 / h->refine_steps);
      if (h->ctl_host->done) break;
      if (h->refine_steps >= h->opt.max_refine) {
        fallback = true;
        break;
      }
      // M~ delta = rho by PCG from delta0 = P^{-1}[0; rho_v], to inner_rtol relative reduction
      launch_ctl_reset(st, h->ctl_in, h->ctl, h->opt.max_inner, L);
      launch_correction_rhs(st, m, d, S.rv, Si.z, L);
      sdp_status s = apply_precond(h, Si, Si.z, Si.x, 0);
      if (s != SDP_OK) return s;
      s = pcg_start(h, Si, true, S.rv, h->opt.inner_rtol * h->opt.inner_rtol);
      if (s != SDP_OK) return s;
      s = krylov_loop(h, Si, true, false);
      if (s != SDP_OK) return s;
      h->inner_iters += h->ctl_host->iters;
      if (h->ctl_host->status == 5) {   // breakdown of the correction solve: its correction is dropped
        fallback = true;
        break;
      }
      launch_add_correction(st, nt, Si.x, S.x, L);
      h->refine_steps += 1;
    }
    if (fallback) {
      // a correction solve broke down, or max_refine corrections did not reach the stop test:
      // the FP64 PCG continues from the refined iterate
      sdp_status s = pcg_start(h, S, false, h->g, 0.0);
      if (s != SDP_OK) return s;
      s = krylov_loop(h, S, false, false);
      if (s != SDP_OK) return s;
      h->inner_iters += h->ctl_host->iters;
    }
  }

  h->cur_iter = -1;
  CU(cudaEventRecord(h->ev_phase[2], st));

  // ---- a8: recovery ----
  phase.next("a8 recovery");
  const double* u = S.x;
  const double* v = S.x + m;
  // dX = E Cw E + sym(Up Q^T) with Cw = A^T(u) - tau^2 C~ and Up = Vs unpack(v): E Cw from
  // F = E C~ of the right side where A^T(u) is sparse or diagonal (one product instead of two)
  if (h->kind == SDP_A_DENSE_SVEC) {
    adjoint_dense(h, S, u, S.Y, nullptr);
    launch_recover_pre(st, n, m, S.Y, Ct, u, h->Cw, dy, dS, h->ctl, L);
    CU(gemm_big(h, st, false, false, n, n, n, 1.0, S.E, n, h->Cw, n, 0.0, S.F, n, S.ws, ws, L));
  } else if (h->kind == SDP_A_SPARSE_COO) {
    sparse_adjoint(st, h->sp, n, u, 1.0, S.Y, nullptr, L);
    launch_recover_pre(st, n, m, S.Y, Ct, u, nullptr, dy, dS, h->ctl, L);
    sparse_posval(st, h->sp, u, S.ypos, nullptr, L);
    sparse_EY(st, h->sp, n, S.ypos, S.E, S.Z, nullptr, L);
    launch_recover_F(st, n, S.Z, S.E, nullptr, S.F, h->ctl, L);
  } else {
    launch_diag_matrix(st, n, u, S.Y, L);
    launch_recover_pre(st, n, m, S.Y, Ct, u, nullptr, dy, dS, h->ctl, L);
    launch_recover_F(st, n, nullptr, S.E, u, S.F, h->ctl, L);
  }
  CU(gemm_big(h, st, false, false, n, n, n, 1.0, S.F, n, S.E, n, 0.0, dX, n, S.ws, ws, L, GEMM_LOWER));
  h_unpack<double>(st, n, r, v, S.Hp, nullptr, L);
  CU(gemm_big(h, st, false, false, n, r, n, 1.0, S.Vs, n, S.Hp, n, 0.0, S.Up, n, S.ws, ws, L));
  CU(gemm_big(h, st, false, true, n, n, r, 0.5, S.Up, n, Q, n, 1.0, dX, n, S.ws, ws, L, GEMM_LOWER));
  CU(gemm_big(h, st, false, true, n, n, r, 0.5, Q, n, S.Up, n, 1.0, dX, n, S.ws, ws, L, GEMM_LOWER));
  lower_to_full(st, n, dX, L);
  CU(cudaEventRecord(h->ev_phase[3], st));
  CU(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  int tc_err = 0, lp_err = 0;
  if (h->tc_err) CU(cudaMemcpyAsync(&tc_err, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (h->m32.err) CU(cudaMemcpyAsync(&lp_err, h->m32.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());

  if (tc_err || lp_err) return fail(h, SDP_ETIMEOUT, "a bounded wait inside a tensor-core product gave up");
  const PcgCtl& c = *h->ctl_host;
  for (int q = 0; q < 3; ++q) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, h->ev_phase[q], h->ev_phase[q + 1]));
    h->phase_ms[q] = ms;
  }
  if (h->prof) {
    sdp_status ps = prof_collect(h, h->prof_base, h->prof_entries.size(), 0, 1);
    if (ps != SDP_OK) return fail(h, ps, "event timing failed");
  }
  if (info) {
    info->r = r;
    info->d = d;
    info->pcg_iters = h->mixed ? h->inner_iters : c.iters;
    info->space = h->space;
    info->converged = (c.status == 0 && c.rr <= c.tol2) ? 1 : 0;
    info->refine_steps = h->refine_steps;
    info->tau = c.tau;
    info->beta = c.beta_pc;
    info->res_norm = std::sqrt(c.rr);
    info->rhs_norm = std::sqrt(c.newt_rhs2);
    info->res0_norm = std::sqrt(c.rr0);
    info->s_A = h->s_A;
    info->setup_ms = h->phase_ms[0];
    info->pcg_ms = h->phase_ms[1];
    info->recover_ms = h->phase_ms[2];
    info->prof_At_ms = h->prof_ms[0];
    info->prof_A_ms = h->prof_ms[1];
    info->prof_At_launches = (int32_t)h->prof_n[0];
    info->prof_A_launches = (int32_t)h->prof_n[1];
    info->prof_At32_ms = h->prof_ms[2];
    info->prof_A32_ms = h->prof_ms[3];
    info->prof_At32_launches = (int32_t)h->prof_n[2];
    info->prof_A32_launches = (int32_t)h->prof_n[3];
    info->refine_rate = h->refine_rate;
  }
  // the split and the preconditioner core stay usable for another right side (sdp_newton_resolve)
  // unless the factorisation failed
  h->setup_valid = (c.status != 5);
  if (c.status == 5) return fail(h, SDP_ENUMERIC, "PCG breakdown or non-positive pivot");
  if (c.status == 4 || !(c.rr <= c.tol2)) return fail(h, SDP_ENOTCONV, "PCG did not reach the stopping test");
  return SDP_OK;
}

}  // namespace

extern "C" sdp_status sdp_newton_solve(sdp_handle* h, const double* V, const double* lam, const double* Ct,
                                       const double* bt, double* dX, double* dy, double* dS,
                                       sdp_newton_info* info) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!V || !lam || !Ct || !bt || !dX || !dy || !dS) return fail(h, SDP_EINVAL, "NULL array argument");
  return newton_solve_impl(h, V, lam, Ct, bt, dX, dy, dS, info, false);
}

extern "C" sdp_status sdp_newton_resolve(sdp_handle* h, const double* Ct, const double* bt, double* dX, double* dy,
                                         double* dS, sdp_newton_info* info) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!Ct || !bt || !dX || !dy || !dS) return fail(h, SDP_EINVAL, "NULL array argument");
  if (!h->setup_valid) return fail(h, SDP_EINVAL, "no previous Newton solve to reuse on this handle");
  return newton_solve_impl(h, nullptr, nullptr, Ct, bt, dX, dy, dS, info, true);
}

extern "C" sdp_status sdp_apply_augsys(sdp_handle* h, const double* pin, double* out, int32_t which) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!pin || !out) return fail(h, SDP_EINVAL, "NULL array argument");
  if (which != 0 && which != 1) return fail(h, SDP_EINVAL, "which must be 0 (operator) or 1 (preconditioner)");
  if (!h->setup_valid) return fail(h, SDP_EINVAL, "no previous Newton solve on this handle");
  if (which == 1 && h->opt.krylov == 1) return fail(h, SDP_EUNSUPPORTED, "a MINRES handle has no preconditioner");
  Space& S = h->s64;
  cudaStream_t st = h->st;
  h->launches = 0;
  h->fuse = false;
  // every kernel of the applies returns at once while the control block's stop flag is set (it
  // is, after the solve): clear it for this call
  CU(cudaMemsetAsync(&S.ctl->done, 0, sizeof(int32_t), st));
  const sdp_status s = which == 0 ? apply_operator(h, S, pin, out, nullptr, 0) : apply_precond(h, S, pin, out, 0);
  if (s != SDP_OK) return s;
  CU(cudaGetLastError());   // enqueued on the handle's stream; the caller orders its reads after it
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

extern "C" sdp_status sdp_grad(sdp_handle* h, const double* V, const double* lam, const double* gX,
                               const double* gy, double* gC, double* gb, sdp_newton_info* info) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!V || !lam || !gX || !gy || !gC || !gb) return fail(h, SDP_EINVAL, "NULL array argument");
  if (h->lin) return fail(h, SDP_EUNSUPPORTED, "the adjoint has no nonnegative variables: remove the linear block");
  // (C~, b~) = (sym gX, gy); the handle's host-staging buffers hold sym gX and the unused dS
  launch_sym_copy(h->st, h->n, gX, h->hCt, &h->launches);
  CU(cudaGetLastError());
  return sdp_newton_solve(h, V, lam, h->hCt, gy, gC, gb, h->hdS, info);
}

extern "C" sdp_status sdp_grad_slack(sdp_handle* h, const double* V, const double* lam, const double* dv,
                                     const double* dw, const double* gX, const double* gy, const double* gv,
                                     const double* gw, double* gC, double* gb, double* gcv, double* gcw,
                                     sdp_newton_info* info) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (!V || !lam || !dv || !dw || !gX || !gy || !gv || !gw || !gC || !gb || !gcv || !gcw)
    return fail(h, SDP_EINVAL, "NULL array argument");
  if (h->lin) return fail(h, SDP_EUNSUPPORTED, "remove the caller's linear block first");
  // staging buffers of the host entry point: hdy = delta, hbt = b~, hCt = sym gX, hdS = the unused dS
  launch_slack_grad_rhs(h->st, h->m, dv, dw, gy, gv, gw, h->hdy, h->hbt, &h->launches);
  launch_sym_copy(h->st, h->n, gX, h->hCt, &h->launches);
  CU(cudaGetLastError());
  sdp_status s = sdp_set_linear_diag(h, h->hdy);
  if (s != SDP_OK) return s;
  s = newton_solve_impl(h, V, lam, h->hCt, h->hbt, gC, gb, h->hdS, info, false);
  const std::string err = h->err;
  sdp_set_linear_diag(h, nullptr);   // the handle is left as the caller set it up
  h->err = err;
  if (s != SDP_OK && s != SDP_ENOTCONV) return s;
  launch_slack_grad_out(h->st, h->m, dv, dw, gb, gv, gw, gcv, gcw, &h->launches);   // dx = D(G^T dy - c~)
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(h->st));
  return s;
}

extern "C" sdp_status sdp_debug_copy(sdp_handle* h, int32_t which, double* dst, int64_t count) {
  if (!h || !dst || count < 0) return fail(h, SDP_EINVAL, "bad debug copy argument");
  const int64_t n = h->n, m = h->m, d = h->d;
  const int64_t pd = h->space == 1 ? d : m;
  const Space& S = h->s64;
  const double* src = nullptr;
  int64_t avail = 0;
  if (h->opt.krylov == 1 && (which == 2 || which == 3))
    return fail(h, SDP_EINVAL, "MINRES forms neither B nor the preconditioner core");
  switch (which) {
    case 0: src = S.E; avail = n * n; break;
    case 1: src = S.Dv; avail = d; break;
    case 2:
      if (h->kind == SDP_A_DIAG && h->space == 2) return fail(h, SDP_EINVAL, "B is not formed for this kind and space");
      src = S.B; avail = m * d; break;
    case 3: src = S.Pinv; avail = pd * pd; break;
    case 4: src = S.Vs; avail = n * n; break;
    case 5: src = S.x; avail = m + d; break;
    case 6: src = h->g; avail = m + d; break;
    case 7: src = reinterpret_cast<const double*>(h->ctl); avail = sizeof(PcgCtl) / sizeof(double); break;
    case 8: src = S.rv; avail = m + d; break;
    case 9: src = S.z; avail = m + d; break;
    case 10: src = S.p; avail = m + d; break;
    case 11: src = S.Ap; avail = m + d; break;
    case 12: src = reinterpret_cast<const double*>(h->ctl_in); avail = sizeof(PcgCtl) / sizeof(double); break;
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

namespace wc {
// Readers of the bounds records of the checked translation units (registered while the library
// loads; none in the default build).
static std::vector<OobReader>& oob_readers() {
  static std::vector<OobReader> v;
  return v;
}
void oob_register(OobReader rd) { oob_readers().push_back(rd); }
}  // namespace wc

extern "C" sdp_status sdp_bounds_report(uint64_t* first, uint64_t* count) {
  if (!first || !count) return SDP_EINVAL;
  *first = 0;
  *count = 0;
  if (wc::oob_readers().empty()) return SDP_EUNSUPPORTED;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return SDP_ECUDA;
  }
  bool ok = true;
  for (wc::OobReader rd : wc::oob_readers()) {
    unsigned long long f = 0, c = 0;
    if (rd(&f, &c) != (int)cudaSuccess) ok = false;
    if (!*first) *first = f;
    *count += c;
  }
  if (!ok) {
    cudaGetLastError();
    return SDP_ECUDA;
  }
  return *count ? SDP_EINVAL : SDP_OK;
}

extern "C" sdp_status sdp_bounds_selftest(void* stream, int64_t index, int64_t bound) {
  if (bound < 0) return SDP_EINVAL;
  if (wc::oob_readers().empty()) return SDP_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  if (wc::sparse_bounds_selftest(st, index, bound) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SDP_ECUDA;
  }
  return SDP_OK;
}

extern "C" size_t sdp_workspace_bytes(const sdp_handle* h) { return h ? h->pool_bytes : 0; }

extern "C" int64_t sdp_last_launch_count(const sdp_handle* h) { return h ? h->launches : 0; }

extern "C" const char* sdp_last_error(const sdp_handle* h) {
  return h ? h->err.c_str() : g_setup_err.c_str();
}

extern "C" sdp_status sdp_set_linear_diag(sdp_handle* h, const double* delta) {
  if (!h) return fail(nullptr, SDP_EINVAL, "NULL handle");
  if (delta) {
    if (h->kind == SDP_A_DIAG || h->mixed || h->opt.krylov != 0)
      return fail(h, SDP_EUNSUPPORTED,
                  "a linear block is built for the DENSE_SVEC and SPARSE_COO kinds, the FP64 form and PCG");
    if (!h->lin_lam) {
      cudaError_t e = cudaMalloc(&h->lin_lam, (size_t)h->m * sizeof(double));
      if (e == cudaSuccess && h->b_elems > 0) e = cudaMalloc(&h->lin_Bw, (size_t)h->b_elems * sizeof(double));
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, SDP_ENOMEM, std::string("linear block workspace: ") + cudaGetErrorString(e));
      }
    }
  }
  h->lin = delta;
  h->setup_valid = false;           // the preconditioner core depends on delta
  wc_drop_graphs(h);                // captured graphs hold the old pointer
  return SDP_OK;
}

extern "C" void sdp_destroy(sdp_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->pool) cudaFree(h->pool);
  if (h->lin_lam) cudaFree(h->lin_lam);
  if (h->lin_Bw) cudaFree(h->lin_Bw);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  for (auto& e : h->ev) cudaEventDestroy(e);
  for (auto& e : h->ev_phase)
    if (e) cudaEventDestroy(e);
  wc_drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto& a : h->aux)
    if (a) cudaStreamDestroy(a);
  for (auto& ev : h->br_ev)
    if (ev) cudaEventDestroy(ev);
  wc_ipm_free(h);
  delete h;
}

// Captured PCG graphs hold the launch forms chosen when they were captured (the cooperative
// preconditioner apply or not): drop them when that choice changes.
void wc_drop_graphs(sdp_handle* h) {
  for (auto& G : h->graph) {
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
    if (G.wexec) {
      cudaGraphExecDestroy(G.wexec);
      G.wexec = nullptr;
    }
  }
}

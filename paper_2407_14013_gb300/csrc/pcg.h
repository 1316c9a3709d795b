// Launch wrappers of pcg.cu (internal).  The finishing kernels of the operator (ap_finish,
// mixed_finish) take optional x, r to do the PCG update in their last block, and pc_zu_dot an
// optional p to do p = z + beta p there (mode 1), when the vectors are short.  The PCG vectors and scalars are FP64 in both forms;
// the mixed form computes only the A E A^T block of its inner operator in FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace wc {

template <typename T>
void launch_ap_finish(cudaStream_t st, int m, int d, int n, int r, const T* partA, int S, const T* Up, const T* Vs,
                      const T* H, const T* Dv, const T* p, const T* g, T* out, int mode, PcgCtl* ctl,
                      double* dotbuf, unsigned int* counter, int64_t* launches, const float* partA32 = nullptr,
                      int S32 = 0, const double* lin = nullptr, double* ux = nullptr, double* ur = nullptr);
template <typename T>
void launch_update(cudaStream_t st, int nt, T* x, T* rv, const T* p, const T* Ap, PcgCtl* ctl, double* dotbuf,
                   unsigned int* counter, int64_t* launches);
template <typename T>
void launch_pc_d_s(cudaStream_t st, int m, int d, int G, const T* partB, const T* rv, T* s, const PcgCtl* ctl,
                   int64_t* launches);
template <typename T>
void launch_pc_d_zv(cudaStream_t st, int m, int d, int S, const T* partC, T* z, const PcgCtl* ctl, int64_t* launches);
template <typename T>
void launch_pc_zu_dot(cudaStream_t st, int m, int d, int S, const T* partU, int space, const T* rv, T* z, int mode,
                      PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches,
                      const double* lam = nullptr, T* pf = nullptr);
template <typename T>
void launch_pc_m_tv(cudaStream_t st, int m, int d, const T* rv, const T* Dv, T* t, const PcgCtl* ctl,
                    int64_t* launches);
template <typename T>
void launch_pc_m_w(cudaStream_t st, int m, int S, const T* partB, const T* rv, T* w, const PcgCtl* ctl,
                   int64_t* launches);
template <typename T>
void launch_pc_m_zv(cudaStream_t st, int m, int d, int G, const T* partBt, const T* rv, const T* Dv, T* z,
                    const PcgCtl* ctl, int64_t* launches);
template <typename T>
void launch_p_update(cudaStream_t st, int nt, const T* z, T* p, int start, const PcgCtl* ctl, int64_t* launches);
template <typename T>
void launch_norm_check(cudaStream_t st, int nt, const T* rv, double rel_rtol2, PcgCtl* ctl, double* dotbuf,
                       unsigned int* counter, int64_t* launches);
template <typename T>
void launch_diag_scale_rows(cudaStream_t st, int n, int r, const T* pu, const T* Vs, T* Tm, const int32_t* done,
                            int64_t* launches);

void launch_rhs_finish(cudaStream_t st, int m, int d, int n, int r, const double* partA, int S, const double* F,
                       const double* E, const double* bt, const double* Ct, const double* H, const double* Dv,
                       double* g, double* x, double rtol, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                       int64_t* launches);
void launch_diag_matrix(cudaStream_t st, int n, const double* u, double* Y, int64_t* launches);
void launch_hadamard_sq(cudaStream_t st, int64_t nn, const double* E, double* EE, int64_t* launches);
void launch_recover_pre(cudaStream_t st, int n, int m, const double* Yu, const double* Ct, const double* u,
                        double* Cw, double* dy, double* dS, const PcgCtl* ctl, int64_t* launches);
// F = E A^T(u) - tau^2 F (EYu = E A^T(u), or NULL for the DIAG kind: E diag(u))
void launch_recover_F(cudaStream_t st, int n, const double* EYu, const double* E, const double* u, double* F,
                      const PcgCtl* ctl, int64_t* launches);
// Linear block of the Newton system (the nonnegative variables of Section 7's robust problems):
// Lam = beta + tau^-2 delta; out = r_u / Lam; Bw = B with row i scaled by Lam_i^-1/2.
void launch_lin_lam(cudaStream_t st, int m, const double* delta, const PcgCtl* ctl, double* lam, int64_t* launches);
// ctl->m_free = #{i : tau^-2 delta_i <= dominance beta} (after the split has set tau and beta)
void launch_lin_free_count(cudaStream_t st, int m, const double* delta, double dominance, PcgCtl* ctl,
                           int64_t* launches);
void launch_lin_div(cudaStream_t st, int m, const double* r, const double* lam, double* out, const PcgCtl* ctl,
                    int64_t* launches);
void launch_lin_scale_rows(cudaStream_t st, int m, int d, const double* B, const double* lam, double* Bw,
                           int64_t* launches);
void launch_add_diag(cudaStream_t st, int n, double* C, const double* Dv, double c_i, int64_t* launches);
void launch_scale_B(cudaStream_t st, int m, int d, const double* B, const double* Dv, double* Bs, int64_t* launches);
void launch_correction_rhs(cudaStream_t st, int m, int d, const double* rho, double* out, int64_t* launches);
void launch_add_correction(cudaStream_t st, int nt, const double* delta, double* x, int64_t* launches);
void launch_mixed_finish(cudaStream_t st, int m, int d, const float* partA32, int SA, const double* partBv, int SB,
                         const double* partBu, int SBu, const double* Dv, const double* p, const double* g,
                         double* out, int mode, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                         int64_t* launches, double* ux = nullptr, double* ur = nullptr);
// The adjoint with the slacks of eq. rmc-sdp (G = [I, -I]): delta = d_v + d_w and
// b~ = g_y + d_v g_v - d_w g_w; then the cotangents of the slack costs dx = D(G^T dy - c~)
void launch_slack_grad_rhs(cudaStream_t st, int m, const double* dv, const double* dw, const double* gy,
                           const double* gv, const double* gw, double* delta, double* bt, int64_t* launches);
void launch_slack_grad_out(cudaStream_t st, int m, const double* dv, const double* dw, const double* dy,
                           const double* gv, const double* gw, double* ov, double* ow, int64_t* launches);
// The dense kind's d-space preconditioner apply in one cooperative launch (B^T r_u, C^{-1} s, B z_v,
// <r, z>, and with pf the p update); with ux (mode 1) it first does the PCG update x += alpha p,
// rv -= alpha Ap and the stop test (rv is written only then).  part: at least
// 2 pc_dense_coop_blocks() doubles.  Returns cudaErrorNotSupported where the device has no
// cooperative launch.
// Last kernel of the body of the device-side PCG loop: sets the WHILE condition from the stop flag
// (guard: a device counter of passes, zeroed before each launch of the loop).
void launch_loop_cond(cudaStream_t st, cudaGraphConditionalHandle hc, const PcgCtl* ctl, int* guard,
                      int64_t* launches);
int pc_dense_coop_blocks();
cudaError_t launch_pc_dense_d_coop(cudaStream_t st, int m, int d, const double* Bt, const double* Pinv,
                                   const double* B, double* rv, double* z, double* sd, double* part, int mode,
                                   PcgCtl* ctl, double* pf, double* ux, const double* Ap, int64_t* launches);
void launch_to_float(cudaStream_t st, int cnt, const double* src, float* dst, const int32_t* done, int64_t* launches);
void launch_sym_copy(cudaStream_t st, int n, const double* g, double* out, int64_t* launches);
void launch_ctl_reset(cudaStream_t st, PcgCtl* dst, const PcgCtl* src, int max_iters, int64_t* launches);
// DIAG kind: part[s n + q] = the slab-s partial sums of diag(F E) (F = E C~, E symmetric), at most
// max_slabs slabs of n entries; returns the number of slabs written.
int launch_diag_FE(cudaStream_t st, int n, const double* F, const double* E, double* part, int max_slabs,
                   int64_t* launches);

// Small DIAG problems (n <= 128, r <= 16, shared memory <= 227 KB per CTA), m-space form, FP64
// PCG: the whole solve in one launch of one thread-block cluster (small_pcg.cu), from the right
// side's finishing step (rhs_finish's work: g from the slabs of diag(F E), b~ and H = Vs^T C~ Q,
// x0, ||[svec C~; b~]|| and the stop threshold rtol^2 ||.||^2) through the stop test.  Reads Vs,
// E o E, K^{-1} (m x m), D and the control block (tau, max_iters, the setup's status);
// leaves x, r, z, p, Ap and the PCG scalars as the launch chain of the loop does.
// small_pcg_plan: the cluster size it launches with for (n, r, d) (16 where that cluster can be
// resident and n > 32, else 8) and its shared memory per CTA; 0 when the shape is outside its range.
int small_pcg_plan(int n, int r, int d, size_t* bytes);
cudaError_t launch_small_pcg(cudaStream_t st, int n, int r, int d, int start0, const double* Vs, const double* EE,
                             const double* Pinv, const double* Dv, const double* part, int slabs, const double* bt,
                             const double* Ct, const double* H, double rtol, double* g, double* x, double* rv,
                             double* z, double* p, double* Ap, PcgCtl* ctl, int64_t* launches);

// DIAG kind, m-space core without an explicit B: w = r_u + rowdot(U, Q); z_v = (pack(H) - r_v) / D;
// Tm = Q (Lam - tau I); K = beta I + tau^-2 G o (G + 2 tau E) (lower triangle)
void launch_diag_w(cudaStream_t st, int n, int r, const double* U, const double* Vs, const double* rv, double* w,
                   const PcgCtl* ctl, int64_t* launches);
void launch_diag_zv(cudaStream_t st, int m, int d, int n, int r, const double* H, const double* rv, const double* Dv,
                    double* z, const PcgCtl* ctl, int64_t* launches);
// MINRES (Def. MINRES, P = I): start, v = r2 / beta, alfa, beta and the rotation, w / x update
void launch_minres_init(cudaStream_t st, int nt, const double* g, double* r1, double* r2, double* x, double* w,
                        double* w2, MinresCtl* mc, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                        int64_t* launches);
void launch_minres_v(cudaStream_t st, int nt, const double* r2, double* v, MinresCtl* mc, PcgCtl* ctl,
                     int64_t* launches);
void launch_minres_alfa(cudaStream_t st, int nt, const double* v, double* y, const double* r1, MinresCtl* mc,
                        PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches);
void launch_minres_beta(cudaStream_t st, int nt, const double* y, double* r1, double* r2, MinresCtl* mc, PcgCtl* ctl,
                        double* dotbuf, unsigned int* counter, int64_t* launches);
void launch_minres_update(cudaStream_t st, int nt, const double* v, double* w, double* w1, double* w2, double* x,
                          const MinresCtl* mc, const PcgCtl* ctl, int64_t* launches);
void launch_pc_d_s_H(cudaStream_t st, int m, int d, int n, int r, const double* H, const double* rv, double* s,
                     const PcgCtl* ctl, int64_t* launches, bool scaled = false);
void launch_shift_cols(cudaStream_t st, int n, int r, const double* Vs, const double* lam_s, const PcgCtl* ctl,
                       double* Tm, int64_t* launches);
void launch_diag_K(cudaStream_t st, int n, const double* G, const double* E, const PcgCtl* ctl, double* K,
                   int64_t* launches);

}  // namespace wc

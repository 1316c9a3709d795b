// Launch wrappers of pcg.cu (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace wc {

void launch_ap_finish(cudaStream_t st, int m, int d, int n, int r, const double* partA, int S, const double* Up,
                      const double* Vs, const double* H, const double* Dv, const double* p, const double* g,
                      double* out, int mode, PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches);
void launch_update(cudaStream_t st, int nt, double* x, double* rv, const double* p, const double* Ap, PcgCtl* ctl,
                   double* dotbuf, unsigned int* counter, int64_t* launches);
void launch_pc_d_s(cudaStream_t st, int m, int d, int G, const double* partB, const double* rv, double* s,
                   const PcgCtl* ctl, int64_t* launches);
void launch_pc_d_zv(cudaStream_t st, int m, int d, int S, const double* partC, double* z, const PcgCtl* ctl,
                    int64_t* launches);
void launch_pc_zu_dot(cudaStream_t st, int m, int d, int S, const double* partU, int space, const double* rv,
                      double* z, int mode, PcgCtl* ctl, double* dotbuf, unsigned int* counter, int64_t* launches);
void launch_pc_m_tv(cudaStream_t st, int m, int d, const double* rv, const double* Dv, double* t, const PcgCtl* ctl,
                    int64_t* launches);
void launch_pc_m_w(cudaStream_t st, int m, int S, const double* partB, const double* rv, double* w,
                   const PcgCtl* ctl, int64_t* launches);
void launch_pc_m_zv(cudaStream_t st, int m, int d, int G, const double* partBt, const double* rv, const double* Dv,
                    double* z, const PcgCtl* ctl, int64_t* launches);
void launch_p_update(cudaStream_t st, int nt, const double* z, double* p, int start, const PcgCtl* ctl,
                     int64_t* launches);
void launch_rhs_finish(cudaStream_t st, int m, int d, int n, int r, const double* partA, int S, const double* F,
                       const double* E, const double* bt, const double* Ct, const double* H, const double* Dv,
                       double* g, double* x, double rtol, PcgCtl* ctl, double* dotbuf, unsigned int* counter,
                       int64_t* launches);
void launch_norm_check(cudaStream_t st, int nt, const double* rv, PcgCtl* ctl, double* dotbuf,
                       unsigned int* counter, int64_t* launches);
void launch_diag_scale_rows(cudaStream_t st, int n, int r, const double* pu, const double* Vs, double* T,
                            const int32_t* done, int64_t* launches);
void launch_diag_matrix(cudaStream_t st, int n, const double* u, double* Y, int64_t* launches);
void launch_hadamard_sq(cudaStream_t st, int64_t nn, const double* E, double* EE, int64_t* launches);
void launch_recover_pre(cudaStream_t st, int n, int m, const double* Yu, const double* Ct, const double* u,
                        double* Cw, double* dy, double* dS, const PcgCtl* ctl, int64_t* launches);
void launch_sym_plus_full(cudaStream_t st, int n, int r, const double* Z, const double* U, const double* Q,
                          double* out, int64_t* launches);
void launch_add_diag(cudaStream_t st, int n, double* C, const double* Dv, double c_i, int64_t* launches);
void launch_scale_B(cudaStream_t st, int m, int d, const double* B, const double* Dv, double* Bs, int64_t* launches);

}  // namespace wc

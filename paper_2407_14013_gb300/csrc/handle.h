// Internal layout of the library handle, shared by the translation units that drive it
// (newton.cu: setup and the Newton solve; ipm.cu: the outer interior-point loop).
#pragma once

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/wcipm.h"
#include "common.cuh"
#include "kernels.h"

namespace wc {

// The FP64 buffers of one PCG solve.  The inner solve of the mixed form shares everything
// with the outer one except its vectors and its control block.
struct Space {
  double *Vs = nullptr, *E = nullptr, *EE = nullptr, *Dv = nullptr, *B = nullptr, *Bt = nullptr, *Pinv = nullptr;
  double *Y = nullptr, *F = nullptr, *Z = nullptr, *Tm = nullptr, *H = nullptr, *Hp = nullptr, *Up = nullptr;
  double *zsvec = nullptr, *partY = nullptr, *partA = nullptr, *sd = nullptr, *wm = nullptr;
  double *partB = nullptr, *partBt = nullptr, *partC = nullptr;
  double *ypos = nullptr, *zpos = nullptr;     // SPARSE_COO: A^T(y) and E Y E at the pattern positions
  double *mw = nullptr, *mw1 = nullptr, *mw2 = nullptr;   // MINRES search directions
  int* fxe = nullptr;                          // exponents of the vectors of the integer passes over A
  int2* Ed = nullptr;                          // digits of E's columns (made once per Newton solve)
  int* eE = nullptr;                           // their exponents
  bool ed_valid = false;                       // Ed, eE hold this solve's E
  double *x = nullptr, *rv = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;
  double* ws = nullptr;                        // split-K GEMM scratch
  size_t ws_elems = 0;
  PcgCtl* ctl = nullptr;
};

// Low-precision data of the mixed forms' A E A^T block, plus their FP64 partial sums of B p_v,
// B^T p_u.  FP32 form: FP32 copies and FFMA products; TF32 form: the same FP32 copy of A with the
// n^3 products on the tensor cores (each FP32 operand as a TF32 pair hi + lo, three MMAs per step);
// BF16 form: a BF16 copy of A (or of E o E) and
// BF16 tensor-core products.  Every low-precision sum is accumulated in FP32.
struct Mixed32 {
  float* A = nullptr;                          // FP32 copy of the svec rows (DENSE kind; FP32, TF32)
  void* A16 = nullptr;                         // BF16 copy of the svec rows, pitch Lp (BF16)
  void* EE16 = nullptr;                        // BF16 copy of E o E, pitch ldk (DIAG kind, BF16)
  void *Elp = nullptr, *Ylp = nullptr, *Glp = nullptr;   // tensor-core operands, n x n, pitch ldk
  float *Elo = nullptr, *Ylo = nullptr, *Glo = nullptr;  // TF32 form: their FP32 remainders (hi + lo)
  float *E = nullptr, *EE = nullptr, *Y = nullptr, *F = nullptr, *Z = nullptr;
  float *zsvec = nullptr, *partY = nullptr, *partA = nullptr, *pu = nullptr;
  float* ws = nullptr;
  size_t ws_elems = 0;
  int64_t Lp = 0;                              // row pitch of the BF16 rows (elements, multiple of 8)
  int ldk = 0;                                 // pitch of the tensor-core operands (multiple of 8)
  int G16 = 1;                                 // row groups of the BF16 A^T pass
  int* err = nullptr;                          // set by a tensor-core product whose bounded wait gave up
  double *partBv = nullptr, *partBu = nullptr;
};

struct ProfEntry {
  int kind;   // 0: A^T pass FP64, 1: A pass FP64, 2: A^T pass FP32, 3: A pass FP32
  int iter;   // chunk-local PCG iteration, or -1 outside the loop
};

struct Graph {
  cudaGraphExec_t exec = nullptr;
  int key[4] = {-1, -1, -1, -1};
  int64_t launches = 0;
  // the whole PCG loop as one graph: a WHILE conditional node whose body is one iteration and
  // whose condition a last kernel sets from the device stop flag (no host read between iterations)
  cudaGraphExec_t wexec = nullptr;
  int wkey[4] = {-1, -1, -1, -1};
  int64_t wlaunches = 0;                // launches of one pass of the body
  size_t prof_first = 0, prof_last = 0;
  std::vector<ProfEntry> entries;
};


struct IpmWork;

// One NVTX range for the life of the object.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// NVTX ranges around the phases of a solve (header-only NVTX v3: nothing happens unless a tool
// such as Nsight Systems is attached).  next() closes the current range and opens another; the
// destructor closes the last one, also on an early return.
struct NvtxPhase {
  explicit NvtxPhase(const char* name) { nvtxRangePushA(name); }
  void next(const char* name) {
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  ~NvtxPhase() { nvtxRangePop(); }
  NvtxPhase(const NvtxPhase&) = delete;
  NvtxPhase& operator=(const NvtxPhase&) = delete;
};

}  // namespace wc


struct sdp_handle {
  // problem (device pointers owned by the caller)
  int n = 0, m = 0, kind = 0;
  int64_t nnz = 0, N = 0;
  const int32_t *a_con = nullptr, *a_row = nullptr, *a_col = nullptr;
  const double *a_val = nullptr, *a_dense = nullptr;
  wc::SparseA sp;                   // SPARSE_COO: the entries and the index tables built at setup
  std::vector<double> sp_rownorm2;  // SPARSE_COO: ||A_i||_F^2 (start point of the outer loop)
  sdp_options opt{};
  bool mixed = false;
  int lp = 0;                       // sdp_precision of the handle
  cudaStream_t st = nullptr;
  int r_max = 0, d_max = 0, mb = 0, mb2 = 0;
  double s_A = 1.0;
  // workspace
  char* pool = nullptr;
  size_t pool_bytes = 0;
  wc::PcgCtl* ctl = nullptr;            // FP64 solve / outer refinement
  wc::PcgCtl* ctl_in = nullptr;         // inner solve of the mixed form
  wc::PcgCtl* ctl_host = nullptr;       // pinned mirror
  unsigned int* counter = nullptr;
  unsigned int* gt_tickets = nullptr;   // per column block of the fused A^T(y) pass
  double *lam_s = nullptr, *e = nullptr, *Ve = nullptr, *Bs = nullptr, *Cw = nullptr, *g = nullptr;
  double *dotbuf = nullptr, *scratch = nullptr;
  double* gj_work = nullptr;
  size_t gj_work_elems = 0;
  double *ubatch = nullptr, *Gb = nullptr, *Hb = nullptr;
  int pinv_dim = 0;                 // order of the largest preconditioner core the options allow
  int dev = 0;                      // device of the handle (current at setup)
  wc::MinresCtl* mctl = nullptr;    // MINRES scalars (device)
  char* tcw = nullptr;              // slices of the tensor-core FP64 products (NULL: not used)
  size_t tcw_bytes = 0;
  char* tcw_b = nullptr;            // the same for the n x r products on the first side stream
  size_t tcw_b_bytes = 0;
  int* tc_err = nullptr;            // set by a tensor-core product whose bounded wait gave up
  char* vs_mem[2] = {nullptr, nullptr};   // slices of the sorted eigenvectors Vs, made once per split:
  wc::TcSlices vs_sl[2];                  // [0] rows of Vs (op = Vs), [1] rows of Vs^T (op = Vs^T)
  bool no_coop = false;             // batched solves: no cooperative (grid-barrier) launches
  bool while_ok = true;             // the device-side PCG loop graph can be built on this device
  bool small_ok = true;             // the one-cluster PCG solve of small DIAG problems launches here
  int* loop_guard = nullptr;        // passes of that loop (a bound independent of the stop flag)
  bool coop_pc = false;             // dense d-space preconditioner apply as one cooperative launch
  int64_t b_elems = 0;              // capacity of the explicit B = A Q (m x d)
  int64_t bt_elems = 0;             // capacity of B^T (d x m)
  int64_t bs_elems = 0;             // capacity of D^{-1/2} B^T (m-space core by a product)
  const double* lin = nullptr;      // linear block delta (m, caller-owned device memory) or NULL
  double* lin_lam = nullptr;        // Lam = beta + tau^-2 delta (m)
  double* lin_Bw = nullptr;         // B with row i scaled by Lam_i^-1/2 (d-space complement)
  bool fx = false;                  // DENSE_SVEC: the FP64 passes over A run on its integer copy
  int2* a_fx = nullptr;             // digits of A (m rows of fx_row_len(N) entries)
  int* a_fx_e = nullptr;            // row exponents
  wc::Space s64;                        // FP64 solve, outer refinement of the mixed form
  wc::Space sin;                        // inner solve of the mixed form (own vectors and control block)
  wc::Mixed32 m32;
  // device staging for the host-pointer entry point
  double *hV = nullptr, *hlam = nullptr, *hCt = nullptr, *hbt = nullptr, *hdX = nullptr, *hdy = nullptr, *hdS = nullptr;
  int GY = 1, SA = 1;       // row groups of the FP64 A^T products, column slabs of the FP64 A products
  int GY32 = 1, SA32 = 1;   // the same for the FP32 copy of A (mixed form)
  int64_t launches = 0;
  int space = 1, r = 0, d = 0;
  int refine_steps = 0, inner_iters = 0;
  bool fuse = false;                // inside the PCG loop: update and p-update in the finishing kernels
  double refine_rate = 0.0, refine_rr0 = 0.0;   // mixed forms: contraction of the FP64 residual
  std::string err;
  // optional CUDA-event timing of the constraint-operator passes (sdp_set_profiling)
  bool prof = false;
  bool capturing = false;           // inside stream capture: event records become graph nodes
  int cur_iter = -1;
  std::vector<cudaEvent_t> ev;
  std::vector<wc::ProfEntry> prof_entries;
  size_t prof_base = 0;             // first entry not yet collected
  cudaEvent_t ev_phase[4] = {nullptr, nullptr, nullptr, nullptr};
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_n[4] = {0, 0, 0, 0};
  double phase_ms[3] = {0.0, 0.0, 0.0};
  // CUDA graphs of `check_every` PCG iterations (FP64 operator, mixed operator), captured once per shape
  cudaStream_t cap_stream = nullptr;
  // side streams and events for the independent branches of the operator (also inside capture)
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t br_ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *ws_b[2] = {nullptr, nullptr};   // split-K scratch of the GEMMs on the side streams
  size_t ws_b_elems = 0;
  wc::Graph graph[3];              // PCG FP64, PCG of the mixed corrections, MINRES
  // the split and preconditioner core of the last solve can serve another right side
  bool setup_valid = false;
  wc::PcgCtl setup_ctl{};           // the control block as a2 left it (r, d, tau, beta, s_A)
  // outer interior-point loop (ipm.cu): workspace allocated on first use
  wc::IpmWork* ipm = nullptr;
};


// Record an error message on the handle (or the setup slot when h is NULL) and return s.
sdp_status wc_fail(sdp_handle* h, sdp_status s, const std::string& msg);
// Release the interior-point workspace (ipm.cu).
void wc_ipm_free(sdp_handle* h);
// Drop the captured PCG graphs of the handle (newton.cu).
void wc_drop_graphs(sdp_handle* h);

// Internal launch wrappers shared by the translation units of the library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace wc {

extern int g_num_sms;
// Raise a kernel's limit of dynamic shared memory to at least `bytes`, never lowering it, under a
// lock: handles of different sizes set it from several host threads, and a limit lowered by one
// of them between another's set and launch would fail that launch.
cudaError_t raise_dyn_smem(const void* func, int bytes);

// ---- gemm_f64.cu -----------------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C (column-major).  ws: split-K partial tiles, its last 16 KB the
// per-tile tickets of the in-kernel reduction; it must be zero when first used (the tickets
// return to zero after every product).  flags:
enum : int {
  GEMM_LOWER = 1,        // only output tiles that meet the lower triangle (i >= j) are written
  GEMM_KSTART_ROW = 2,   // op(A)[i, k] = 0 for k < i (skip those K steps)
  GEMM_KSTART_COL = 4    // op(B)[k, j] = 0 for k < j
};
cudaError_t gemm_f64(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                     double* C, int64_t ldc, double* ws, size_t ws_elems, int64_t* launches,
                     const int32_t* done = nullptr, int flags = 0);

// ---- tc_gemm.cu: FP64 products on the BF16 tensor cores (exact slices) -------------------------
// Same convention as gemm_f64 (flags: GEMM_LOWER only).  work: tc_gemm_work_bytes(M, N, K)
// bytes, 256-byte aligned (its first 256 bytes are not used by the product); err: a device
// word set to 1 when a bounded wait gave up (the caller clears and reads it).
// Products with few output tiles split K over the SMs (FP64 partial tiles, reduced in a fixed
// order).  done: device stop flag (may be NULL): every kernel returns at once when it is set.
// tc_prepare(): the one-time setup (driver entry point, shared-memory attribute); call it
// before any stream capture.
// Slices of an operand made once and reused by later products over the same K (rows of op(X)).
struct TcSlices {
  void* s = nullptr;      // 8 planes of rows x kpad(K) BF16 digits
  int* e = nullptr;       // per-row power-of-two exponents
  int rows = 0, K = 0;
  bool valid = false;
};
size_t tc_slices_bytes(int R, int K);
cudaError_t tc_make_slices(cudaStream_t st, int R, int K, const double* X, int64_t rs, int64_t ks, void* mem,
                           TcSlices* out, int64_t* launches);
size_t tc_gemm_work_bytes(int M, int N, int K);
cudaError_t tc_prepare();
// 2-D TMA tensor map (128-byte swizzle, zero fill outside) over `rows` rows of `inner` BF16 or FP32
// elements, `pitch_bytes` apart (a multiple of 16), boxes of box_inner x box_rows
cudaError_t tmap_2d(CUtensorMap* map, bool f32, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch_bytes,
                    uint32_t box_inner, uint32_t box_rows);

// ---- lp_gemm.cu: BF16 / TF32 tensor-core products with FP32 accumulation (mixed forms) -----------
// C (M x N, column-major, pitch ldc) = alpha op(A) op(B), op(A) given by its rows and op(B) by its
// columns, both K-contiguous with pitches lda, ldb (elements; 16-byte rows): C = A_s^T B_s for
// A_s (K x M) and B_s (K x N) column-major.  mode 0: BF16 operands (kind::f16); 1: FP32 operands
// read as TF32 (kind::tf32); 2: FP32 operands given as TF32-exact (hi, lo) pairs (A, Alo), (B, Blo),
// product hi hi + hi lo + lo hi (about FP32 accuracy).  out_mode 0: FP32 C; 1: BF16 C; 2: FP32 as
// the pair (C, Clo) with C TF32-exact.  K >= 1; err as for gemm_f64_tc.
cudaError_t lp_prepare();
cudaError_t lp_gemm(cudaStream_t st, int mode, int M, int N, int K, float alpha, const void* A, const void* Alo,
                    int64_t lda, const void* B, const void* Blo, int64_t ldb, void* C, void* Clo, int64_t ldc,
                    int out_mode, int* err, int64_t* launches, const int32_t* done = nullptr);
// Passes over a BF16 copy of the svec rows (m rows, pitch Lp, a multiple of 8, zero padded):
// part[g * Lp + c] = sum_{i in group g} p_i a[i, c] (FP32), and out[i] = <a[i, :], z> (z FP32 of
// length Lp, zero padded), in column slabs
int bf16_gemvT_groups(int m, int64_t Lp);
void bf16_gemvT(cudaStream_t st, const void* A16, int m, int64_t Lp, const float* p, float* part, int groups,
                const int32_t* done, int64_t* launches);
int bf16_gemv_slabs(int m, int64_t Lp);   // column slabs of the A pass: out holds slabs x m partial sums
void bf16_gemv(cudaStream_t st, const void* A16, int m, int64_t Lp, const float* z, float* out, int slabs,
               const int32_t* done, int64_t* launches);
// Y (n x n, pitch ldk, BF16 or FP32, both triangles) = smat(sum_g part[g * Lp + .]); with Ylo (FP32)
// Y is written as the pair (TF32-exact hi, FP32 remainder)
void lp_unpack(cudaStream_t st, int n, const float* part, int groups, int64_t Lp, void* Y, int ldk, bool bf16,
               float* Ylo, const int32_t* done, int64_t* launches);
// X (rows x cols FP64, pitch ldx) -> Y (BF16 or FP32, pitch ldy); columns cols .. ldy-1 of Y are zeroed;
// with Ylo (FP32) as the pair (TF32-exact hi, FP32 remainder)
void lp_convert(cudaStream_t st, int rows, int cols, const double* X, int64_t ldx, void* Y, int64_t ldy, bool bf16,
                float* Ylo, int64_t* launches);
cudaError_t gemm_f64_tc(cudaStream_t st, bool tA, bool tB, int M, int N, int K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work,
                        size_t work_bytes, int* err, int flags, int64_t* launches, const int32_t* done = nullptr,
                        const TcSlices* cA = nullptr, const TcSlices* cB = nullptr);

// ---- rows.cu: products with row-major matrices streamed from memory ---------------------------
// Partial sums of y_i = <row_i(A), x>: part[s * m + i] over column slabs s.  The slab count
// depends on the shape and the element size (8: double, 4: float); a partial-sum buffer of
// rows_gemv_part_elems(rows_max, L) elements serves every m <= rows_max.
int rows_gemv_slabs(int m, int64_t L, int esize = 8);
size_t rows_gemv_part_elems(int64_t rows_max, int64_t L);
template <typename T>
void rows_gemv(cudaStream_t st, const T* A, int m, int64_t L, const T* x, T* part, const int32_t* done,
               int64_t* launches);
// rows_gemv with the vector formed while it is staged: x = base + c * sum_{g < G} xpart[g L + k]
// with c = c0 / *cdiv (cdiv device pointer, may be NULL: c = c0); x is also stored to xout
// (may be NULL).  Fuses an elementwise step that would otherwise be its own launch.
void rows_gemv_formed(cudaStream_t st, const double* A, int m, int64_t L, const double* base, const double* xpart,
                      int G, double c0, const double* cdiv, double* xout, double* part, const int32_t* done,
                      int64_t* launches);
// Partial sums of y = sum_i p_i row_i(A): part[g * L + k] over row groups g; the group count
// for an m x L matrix of `esize`-byte elements spreads the CTAs evenly over the SMs.
int rows_gemvT_groups(int m, int64_t L, int esize = 8);
template <typename T>
void rows_gemvT(cudaStream_t st, const T* A, int m, int64_t L, const T* p, T* part, int groups,
                const int32_t* done, int64_t* launches);
// The same with the partial sums reduced in-kernel (last CTA per column block) and written as
// the full symmetric n x n matrix Y = scale * smat(sum_g part_g) (L = n(n+1)/2).  tickets: at
// least rows_gemvT_blocks(L, sizeof(T)) zeroed words (left zero after the call).
template <typename T>
void rows_gemvT_unpack(cudaStream_t st, const T* A, int m, int64_t L, const T* p, T* part, int groups, int n,
                       double scale, T* Y, unsigned int* tickets, const int32_t* done, int64_t* launches);
int rows_gemvT_blocks(int64_t L, int esize);
// Exact fixed-point forms of the FP64 passes over dense rows (rows.cu): A (m x L) split once into
// two int32 digits per entry (rows of fx_row_len(L) entries) with a power-of-two exponent per
// row; a pass takes its vector's exponent (the device int *f) from fx_exponent, from the kernel
// that produced the vector, or finds it itself, splits the vector as it stages it, and sums
// exact int64 digit products.  Same outputs and partial-sum layouts as
// rows_gemv<double> and rows_gemvT_unpack<double>, with an error within the FP64 dot-product bound.
// C = A B (column-major, M x N x K, no transposes) from exact int64 sums of two-digit products
// (gemm_fx.cu); `lower` writes only the entries i >= j.  Error within the FP64 dot-product bound
// measured against the largest entry of each row of A and column of B.  pre = 1: A is given by
// its row digits (Dd[i K + k], exponents De[i]); pre = 2: B by its column digits (Dd[j K + k],
// De[j]), as fx_col_digits makes them (the same bits as without them).
// With pack (M == N, lower), C is not written: out gets svec(C + sym(U Q^T)) (U, Q: n x r, U may be
// NULL) and *expo the largest exponent of it, as svec_pack_plus does from C (the same bits).
struct FxPack {
  const double* U = nullptr;
  const double* Q = nullptr;
  int r = 0;
  double* out = nullptr;
  int* expo = nullptr;
};
cudaError_t fx_gemm(cudaStream_t st, int M, int N, int K, const double* A, int64_t lda, const double* B, int64_t ldb,
                    double* C, int64_t ldc, bool lower, const int32_t* done, int64_t* launches, int pre = 0,
                    const int2* Dd = nullptr, const int* De = nullptr, const FxPack* pack = nullptr);
// Digits of the columns of M (n x n, column-major, n <= 512; false otherwise): exponents e[j]
// (2^e[j] > max_k |M_kj|) and int32 digit pairs D[j n + k], those fx_gemm forms for M's columns.
bool fx_col_digits(cudaStream_t st, int n, const double* M, int2* D, int* e, int64_t* launches);
int64_t fx_row_len(int64_t L);
int fx_rows_gemv_slabs(int m, int64_t L);   // slab partial sums written by fx_rows_gemv
void fx_split_rows(cudaStream_t st, const double* A, int m, int64_t L, int2* Ai, int* ea, int64_t* launches);
void fx_exponent(cudaStream_t st, const double* x, const int* ex, int64_t len, int* f, const int32_t* done,
                 int64_t* launches);
void fx_rows_gemv(cudaStream_t st, const int2* Ai, const int* ea, int m, int64_t L, const double* x, const int* f,
                  double* part, const int32_t* done, int64_t* launches);
void fx_rows_gemvT_unpack(cudaStream_t st, const int2* Ai, const int* ea, int m, int64_t L, const double* y,
                          int* f, double* part, int groups, int n, double scale, double* Y, const int32_t* done,
                          int64_t* launches);
// sum_i ||row_i||^2
void rows_sumsq(cudaStream_t st, const double* A, int m, int64_t L, double* out, double* scratch,
                int64_t* launches);

// ---- sym.cu: symmetric-matrix layouts ----------------------------------------------------------
// Y (n x n full) = smat(sum_g part[g * N + idx]) ; scale multiplies the result.
template <typename T>
void svec_unpack_sum(cudaStream_t st, int n, const T* part, int groups, double scale, T* Y,
                     const int32_t* done, int64_t* launches);
// out(svec, N) = svec(Z + sym(U Q^T)) with U, Q n x r (U may be NULL); Z is symmetric and only
// its lower triangle is read.  With expo (FP64 only), atomically raises *expo to the exponent e
// (|out_k| < 2^e) of every nonzero output, or to INT_MAX for a non-finite one: the caller sets
// *expo below FX_NONE_MAX first (the exponent of the integer A pass).
template <typename T>
void svec_pack_plus(cudaStream_t st, int n, int r, const T* Z, const T* U, const T* Q, T* out,
                    const int32_t* done, int64_t* launches, int* expo = nullptr);
// Stack of full matrices from svec rows i0 .. i0+mb-1: out[b * (mb n) + il * n + a] = A_{i0+il}[a, b].
void svec_rows_unpack(cudaStream_t st, const double* A, int n, int i0, int mb, double* out,
                      int64_t* launches);

// ---- split.cu: eq. EQSigdef ------------------------------------------------------------------
// Sort lam descending (ties by index), permute V's columns, choose r, tau, beta and write them to ctl;
// e[k] = diagonal of V^T E V (1 for k < r, lam_k / tau after); Ve = Vs diag(e).
void split_sort(cudaStream_t st, int n, const double* V, const double* lam, double* Vs, double* lam_s,
                int64_t* launches);
void split_params(cudaStream_t st, int n, int r_fixed, int r_hat, int beta_rule, const double* lam_s,
                  double* e, PcgCtl* ctl, int64_t* launches);
void split_scale_cols(cudaStream_t st, int n, const double* Vs, const double* e, double* Ve,
                      int64_t* launches);
// D (d) = tau^2 Sigma in h-coordinates.
void split_sigma(cudaStream_t st, int n, int r, const double* lam_s, const PcgCtl* ctl, double* Dv,
                 int64_t* launches);

// ---- hcoord.cu: coordinates h = [svec B; vec N] of range(Q) (Section 5) ---------------------
// out[h] = c_out * pack(H)[h] + c_in * in[h] - Dv[h] * pv[h] (any of in / Dv may be NULL)
void h_pack(cudaStream_t st, int n, int r, const double* H, int64_t ldH, double c_out, const double* in,
            double c_in, const double* Dv, const double* pv, double* out, const int32_t* done,
            int64_t* launches);
// Hp (n x r) with Vs Hp = Q B + sqrt2 Qp N for h = [svec B; vec N] (of h / Dv when Dv is given)
template <typename T>
void h_unpack(cudaStream_t st, int n, int r, const T* h, T* Hp, const int32_t* done, int64_t* launches,
              const T* Dv = nullptr);
// B rows of A Q from a batch H = Vs^T [A_i Q] (n x mb r, column j * mb + il): B[(i0+il) * d + h]
void h_pack_rows(cudaStream_t st, int n, int r, int mb, int i0, const double* H, double* B,
                 int64_t ldB, double* Bt, int64_t ldBt, int64_t* launches);
// DIAG kind: B[i, :] = pack(Vs[i, :]^T Q[i, :])
void h_pack_rows_diag(cudaStream_t st, int n, int r, const double* Vs, double* B, int64_t ldB,
                      double* Bt, int64_t ldBt, int64_t* launches);
// DENSE kind: G (n x mb r, column j * mb + il) = A_{i0+il} Q for a batch of constraints, straight
// from the svec rows (one CTA per constraint, per-warp accumulators in shared memory).  Returns
// false when n r is too large for the shared-memory accumulators.
bool dense_AiQ(cudaStream_t st, const double* A, int n, int i0, int mb, int r, const double* Q, double* G,
               int64_t* launches);
// The same from the integer digits of the rows (fx_split_rows) on the integer pipe; false when
// the row does not fit in shared memory or n > 1024 (then use dense_AiQ).
bool fx_AiQ(cudaStream_t st, const int2* Ad, const int* ea, int n, int64_t Lp, int i0, int mb, int r, const double* Q,
            double* G, int64_t* launches);

// ---- gemm_f32.cu: FP32 GEMM (FFMA tiles, FP32 accumulation), same conventions as gemm_f64 ----
cudaError_t gemm_f32(cudaStream_t st, bool tA, bool tB, int M, int N, int K, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                     float* C, int64_t ldc, float* ws, size_t ws_elems, int64_t* launches,
                     const int32_t* done = nullptr);
// element-wise conversion dst = (To) src
template <typename To, typename From>
void convert(cudaStream_t st, int64_t count, const From* src, To* dst, int64_t* launches);

// ---- sparse.cu: SDP_A_SPARSE_COO operators ------------------------------------------------------
// The caller's entries (con, row, col, val; sorted by con, row >= col) plus the index tables
// sdp_setup builds: con_ptr (m + 1) and the entries grouped by position (pos_r, pos_c,
// pos_ptr (npos + 1), perm (nnz): entry indices in position order).
struct SparseA {
  int64_t nnz = 0;
  int npos = 0;
  int64_t nnzY = 0;      // nonzeros of the symmetric pattern of A^T(y) (off-diagonal positions twice)
  int m = 0;             // constraints
  const int32_t *con = nullptr, *row = nullptr, *col = nullptr;
  const double* val = nullptr;
  int32_t *con_ptr = nullptr, *pos_r = nullptr, *pos_c = nullptr, *pos_ptr = nullptr, *perm = nullptr;
  int32_t* epos = nullptr;                                  // position index of each entry (nnz)
  int32_t* cptr = nullptr;                                  // positions of column b: cptr[b] .. cptr[b+1]-1
  int32_t *yptr = nullptr, *ycol = nullptr, *ypidx = nullptr;   // CSR of the pattern: row i holds
                                                            // (column, position index) pairs
  // Term pairs of the constraints for the Gram form of the d-space complement: A_i = sum_t w_t
  // e_{x_t} e_{y_t}^T over its terms (an off-diagonal entry gives two), and every pair (t, t') of
  // terms of one constraint, grouped by x_t (CSR over the n rows): x' = x_t', y = y_t, y' = y_t',
  // w = w_t w_t', con = i.  npairs = 0 when the table was not built (too large).
  int64_t npairs = 0;
  int32_t *pptr = nullptr, *pxp = nullptr, *py = nullptr, *pyp = nullptr, *pcon = nullptr;
  double* pw = nullptr;
  double* pcf = nullptr;   // scratch: the pairs' coefficients of one column pair (j1, j2)
};
// Y = scale * A^T(y) on the pattern positions (both triangles); Y is zero elsewhere already.
void sparse_adjoint(cudaStream_t st, const SparseA& S, int n, const double* y, double scale, double* Y,
                    const int32_t* done, int64_t* launches);
// out[i] = <A_i, Z + sym(U Q^T)>, Z symmetric with its lower triangle read, U may be NULL.
void sparse_apply(cudaStream_t st, const SparseA& S, int n, int m, int r, const double* Z, const double* U,
                  const double* Q, double* out, const int32_t* done, int64_t* launches);
// B = A Q (m x d row-major, ld ldB) and B^T (d x m, ld ldBt) in h-coordinates.
void sparse_B(cudaStream_t st, const SparseA& S, int n, int m, int r, const double* Vs, double* B, int64_t ldB,
              double* Bt, int64_t ldBt, int64_t* launches);
// One bounds check of index against bound in the sparse translation unit (no access is made);
// recorded as a violation in the bounds-checked build when index is outside [0, bound).
cudaError_t sparse_bounds_selftest(cudaStream_t st, int64_t index, int64_t bound);
// Gram form of C = sum_i s_i b_i b_i^T (b_i = row i of B = A Q in h-coordinates, s_i = 1 / beta
// or 1 / Lam_i): for one column pair (j1, j2) of the n x r matrices H_i = Vs^T A_i Q,
//   Y = W Vs with W = sum over term pairs p of s_{con_p} w_p Q[y_p, j1] Q[y'_p, j2] e_{x_p} e_{x'_p}^T
// (sparse_gram_spmm), G = Vs^T Y = sum_i s_i H_i[:, j1] H_i[:, j2]^T (a dense product by the caller),
// then C[h(a1, j1), h(a2, j2)] += c(a1, j1) c(a2, j2) G[a1, a2] through the h-coordinate map
// (sparse_gram_scatter; C d x d column-major, zeroed by the caller before the first block; with
// mirror also at the transposed entries, the (j2, j1) pair's share, so j1 <= j2 suffices).
void sparse_gram_spmm(cudaStream_t st, const SparseA& S, int n, int j1, int j2, const double* Vs, double inv_beta,
                      const double* lam, double* Y, int64_t* launches);
void sparse_gram_scatter(cudaStream_t st, int n, int r, int j1, int j2, bool mirror, const double* G, double* C,
                         int64_t ldc, int64_t* launches);
// Position values of Y = A^T(y): ypos[p] = sum over the entries e at position p of y[con_e] val_e.
void sparse_posval(cudaStream_t st, const SparseA& S, const double* y, double* ypos, const int32_t* done,
                   int64_t* launches);
// Out (n x ncols, ld ldo) = Y Bm (Bm n x ncols, ld ldb) with Y = A^T(y) given by its position values.
void sparse_sym_spmm(cudaStream_t st, const SparseA& S, int n, int ncols, const double* ypos, const double* Bm,
                     int64_t ldb, double* Out, int64_t ldo, const int32_t* done, int64_t* launches);
// F = E Y (n x n) for E (n x n) and Y = A^T(y) given by its position values.
void sparse_EY(cudaStream_t st, const SparseA& S, int n, const double* ypos, const double* E, double* F,
               const int32_t* done, int64_t* launches);
// zpos[p] = (F E)[a_p, b_p] = <F[b_p, :], E[:, a_p]> for symmetric E and F E (E Y E with F = E Y);
// needs n doubles of shared memory per CTA: sparse_prepare(n) once per process and n (before any
// capture; cudaErrorInvalidValue when n * 8 bytes exceed 227 KB).
cudaError_t sparse_prepare(int n);
cudaError_t sparse_pos_dots_col(cudaStream_t st, const SparseA& S, int n, const double* E, const double* F,
                                double* zpos, const int32_t* done, int64_t* launches);
// out[i] = <A_i, Z + sym(U Q^T)> with Z given by its values at the pattern positions (zpos, may be
// NULL: Z = 0) and U, Q n x r (U may be NULL).
void sparse_apply_pos(cudaStream_t st, const SparseA& S, int n, int m, int r, const double* zpos, const double* U,
                      const double* Q, double* out, const int32_t* done, int64_t* launches);
// *out = sum_i ||A_i||_F^2; scratch holds 2 * g_num_sms doubles.
void sparse_sumsq(cudaStream_t st, const SparseA& S, double* out, double* scratch, int64_t* launches);

// ---- spd_inverse.cu ----------------------------------------------------------------------------
// In-place inverse of an SPD matrix (n x n, column-major, ld = n) through its Cholesky factor;
// work must hold spd_inverse_work(n) doubles.
size_t spd_inverse_work(int n);
// n <= 1024 with allow_coop: one cooperative launch (falls back to the launch chain when the
// cooperative launch is not possible).
cudaError_t spd_inverse(cudaStream_t st, int n, double* A, double* work, size_t work_elems,
                        double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches,
                        bool allow_coop = true);
// A[j, i] = A[i, j] for i > j (n x n, column-major): the upper triangle from the lower.
void lower_to_full(cudaStream_t st, int n, double* A, int64_t* launches);
// The same for large n with 512-wide outer panels: the panel solves, trailing updates, the
// block rows of L^{-1} and L^{-T} L^{-1} go through the tensor-core product when `tc` allows
// (NULL: FP64 MMA); the 512 x 512 diagonal blocks use the one-CTA 32 x 32 factorisation.
struct TcCtx {
  void* work = nullptr;
  size_t bytes = 0;
  int* err = nullptr;
};
size_t spd_inverse_tc_work(int n);
cudaError_t spd_inverse_tc(cudaStream_t st, int n, double* A, double* work, size_t work_elems, double* gemm_ws,
                           size_t gemm_ws_elems, const TcCtx* tc, int32_t* status, int64_t* launches,
                           bool allow_coop = true);
// Cholesky A = L L^T (L into A, upper zeroed) and Linv = L^{-1} (NULL: factor only); same workspace.
cudaError_t spd_cholesky(cudaStream_t st, int n, double* A, double* Linv, double* work, size_t work_elems,
                         double* gemm_ws, size_t gemm_ws_elems, int32_t* status, int64_t* launches,
                         bool allow_coop = true);

// ---- eigh.cu: symmetric eigen-decomposition (parallel cyclic Jacobi, FP64) ------------------
// A (n x n, symmetric, destroyed) = V diag(lam) V^T; stops when ||offdiag A||_F <= tol ||A||_F
// or after max_sweeps sweeps (sweeps and the final relative off-diagonal norm are returned).
// With `graph` non-NULL a sweep runs as one replay of a CUDA graph captured (on the graph's own
// stream) for these pointers; the graph is recaptured when n or a pointer changes.
struct EighGraph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  int n = 0;
  const void *A = nullptr, *V = nullptr, *work = nullptr;
};
void eigh_graph_release(EighGraph* g);
// Smallest eigenvalue of the symmetric M (n x n) by Lanczos with full re-orthogonalisation:
// cooperative launches over the GPU when allowed and supported, else one block per launch.
size_t lanczos_work_elems(int n);
cudaError_t lanczos_min(cudaStream_t st, int n, const double* M, double* work, size_t work_elems, double* lmin,
                        int* iters, int64_t* launches, bool allow_coop = true);
size_t eigh_work_elems(int n);
cudaError_t eigh_jacobi(cudaStream_t st, int n, double* A, double* V, double* lam, double tol, int max_sweeps,
                        double* work, size_t work_elems, int* sweeps_out, double* off_out, int64_t* launches,
                        EighGraph* graph = nullptr, bool allow_coop = true);

}  // namespace wc

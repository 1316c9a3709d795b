// Sparse constraint operators (SDP_A_SPARSE_COO): A_i = sum over its entries e of
// val_e (e_r e_c^T + e_c e_r^T) for r > c, val_e e_r e_r^T for r = c, so that
// <A_i, X> = sum_e val_e X[r, c] (2 if r != c) (eq. sdp-pd with A given by its entries; matrix
// completion samples one off-diagonal entry per constraint).
//
// The entries arrive sorted by constraint; sdp_setup adds two index tables (built once per
// problem): con_ptr (the entries of constraint i are con_ptr[i] .. con_ptr[i+1]-1) and the
// entries grouped by matrix position (pos_r, pos_c, pos_ptr, perm), so that
//   A(Z):     one thread per constraint sums its entries          (a gather, no atomics)
//   A^T(y):   one thread per distinct position sums its entries   (fixed order, no atomics)
// both deterministic.  A^T(y) writes only the positions of the pattern; every other entry of
// the output matrix must already be zero (the callers zero it once).
//
// Inside the PCG loop Y = A^T(y) is never formed as a matrix: it is kept as its values at the
// pattern positions, with a CSR table of the symmetric pattern (row i: the columns c with
// Y[i, c] a pattern entry, and their position index), so that
//   Y Bm        one thread per (row, column of Bm) sums its row's pattern entries (SpMM)
//   (E Y E)_ab  only at the pattern positions: <E[:, a], (Y E)[:, b]>, one warp each
// which replaces the two dense n^3 products E Y and (E Y) E by O(nnz(Y) n + npos n) work.
//
// The d-space complement C = tau^2 Sigma + sum_i s_i b_i b_i^T (b_i = row i of B = A Q) is formed
// without B where that is cheaper: for each column pair (j1 <= j2) of the H_i = Vs^T A_i Q, the
// block sum_i s_i H_i[:, j1] H_i[:, j2]^T equals Vs^T W Vs with W sparse over the constraints'
// term pairs (gram_*), and its entries go to C through the h-coordinate map of pack(.).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

constexpr int ST = 256;

inline unsigned nb(int64_t total) { return (unsigned)((total + ST - 1) / ST); }

// Lengths of the arrays that the index tables address (used by the bounds-checked build only).
struct SpLen {
  int64_t nnz;    // entries: con, row, col, val, perm, epos
  int64_t nnzY;   // symmetric pattern: ycol, ypidx
  int npos;       // distinct positions: pos_r, pos_c, position values
  int m;          // constraints: y
};

inline SpLen lens(const SparseA& S) { return SpLen{S.nnz, S.nnzY, S.npos, S.m}; }

// Sites of the checks in the bounds-checked build (the site number kept with a violation)
enum : int {
  kAdjPtr = 1, kAdjPerm, kAdjCon, kAdjPos,              // sparse_adjoint_kernel
  kAppPtr, kAppRC,                                      // sparse_apply_kernel
  kBPtr, kBRC,                                          // sparse_B_kernel
  kValPtr, kValPerm, kValCon,                           // sparse_posval_kernel
  kMmPtr, kMmPidx, kMmCol,                              // sym_spmm_kernel
  kEyPtr, kEyPidx, kEyCol,                              // sparse_EY_kernel
  kDotPtr, kDotRow,                                     // pos_dots_col_kernel
  kApPtr, kApPos, kApRC,                                // sparse_apply_pos_kernel
  kSelfTest,                                            // oob_selftest_kernel
  kGramPtr, kGramIdx                                    // gram_spmm_kernel, gram_coef_kernel
};

// Y[r, c] = Y[c, r] = sum over the entries e at position (r, c) of y[con_e] val_e (times scale)
__global__ void sparse_adjoint_kernel(int n, int npos, const int32_t* __restrict__ pos_r,
                                      const int32_t* __restrict__ pos_c, const int32_t* __restrict__ pos_ptr,
                                      const int32_t* __restrict__ perm, const int32_t* __restrict__ con,
                                      const double* __restrict__ val, const double* __restrict__ y, double scale,
                                      double* __restrict__ Y, SpLen L, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  double s = 0.0;
  for (int k = pos_ptr[p]; k < pos_ptr[p + 1]; ++k) {
    if (!WC_IN(kAdjPtr, k, L.nnz)) break;
    const int e = perm[k];
    if (!WC_IN(kAdjPerm, e, L.nnz)) continue;
    const int i = con[e];
    if (!WC_IN(kAdjCon, i, L.m)) continue;
    s = fma(y[i], val[e], s);
  }
  s *= scale;
  const int r = pos_r[p], c = pos_c[p];
  if (!WC_IN(kAdjPos, r, n) || !WC_IN(kAdjPos, c, n)) return;
  Y[r + (int64_t)c * n] = s;
  Y[c + (int64_t)r * n] = s;
}

// out[i] = <A_i, Z + sym(U Q^T)> for the symmetric Z (lower triangle read) and U, Q n x r
// (U may be NULL)
__global__ void sparse_apply_kernel(int n, int m, int r, const int32_t* __restrict__ con_ptr,
                                    const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, const double* __restrict__ Z,
                                    const double* __restrict__ U, const double* __restrict__ Q,
                                    double* __restrict__ out, SpLen L, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int e = con_ptr[i]; e < con_ptr[i + 1]; ++e) {
    if (!WC_IN(kAppPtr, e, L.nnz)) break;
    const int a = row[e], b = col[e];   // a >= b
    if (!WC_IN(kAppRC, a, n) || !WC_IN(kAppRC, b, n)) continue;
    double z = Z[a + (int64_t)b * n];
    if (U) {
      double t = 0.0;
      for (int k = 0; k < r; ++k)
        t += U[a + (int64_t)k * n] * Q[b + (int64_t)k * n] + Q[a + (int64_t)k * n] * U[b + (int64_t)k * n];
      z += 0.5 * t;
    }
    s = fma(val[e] * (a == b ? 1.0 : 2.0), z, s);
  }
  out[i] = s;
}

// Row i of B = A Q in h-coordinates: B[i, h] = pack(Vs^T A_i Q)[h] with
// (Vs^T A_i Q)[k, j] = sum_e val_e (Vs[r,k] Q[c,j] + Vs[c,k] Q[r,j])  (one term when r = c)
__device__ __forceinline__ double sparse_H(int n, int k, int j, int e0, int e1, const int32_t* __restrict__ row,
                                           const int32_t* __restrict__ col, const double* __restrict__ val,
                                           const double* __restrict__ Vs, int64_t nnz) {
  double s = 0.0;
  for (int e = e0; e < e1; ++e) {
    if (!WC_IN(kBPtr, e, nnz)) break;
    const int a = row[e], b = col[e];
    if (!WC_IN(kBRC, a, n) || !WC_IN(kBRC, b, n)) continue;
    double t = Vs[a + (int64_t)k * n] * Vs[b + (int64_t)j * n];
    if (a != b) t += Vs[b + (int64_t)k * n] * Vs[a + (int64_t)j * n];
    s = fma(val[e], t, s);
  }
  return s;
}

__global__ void sparse_B_kernel(int n, int m, int r, const int32_t* __restrict__ con_ptr,
                                const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ Vs, double* __restrict__ B,
                                int64_t ldB, double* __restrict__ Bt, int64_t ldBt, SpLen L) {
  const int d = n * r - r * (r - 1) / 2;
  const int nb_ = r * (r + 1) / 2;
  const int64_t total = (int64_t)m * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / d), h = (int)(q % d);
    const int e0 = con_ptr[i], e1 = con_ptr[i + 1];
    double v;
    if (h < nb_) {
      int j = 0, base = 0;
      while (h >= base + (r - j)) { base += r - j; ++j; }
      const int a = j + (h - base);
      if (a == j) v = sparse_H(n, a, a, e0, e1, row, col, val, Vs, L.nnz);
      else
        v = WC_SQRT2 * 0.5 *
            (sparse_H(n, a, j, e0, e1, row, col, val, Vs, L.nnz) + sparse_H(n, j, a, e0, e1, row, col, val, Vs, L.nnz));
    } else {
      const int qq = h - nb_;
      const int k = qq % (n - r), j = qq / (n - r);
      v = WC_SQRT2 * sparse_H(n, r + k, j, e0, e1, row, col, val, Vs, L.nnz);
    }
    B[(int64_t)i * ldB + h] = v;
    if (Bt) Bt[(int64_t)h * ldBt + i] = v;
  }
}

__global__ void sparse_posval_kernel(int npos, const int32_t* __restrict__ pos_ptr, const int32_t* __restrict__ perm,
                                     const int32_t* __restrict__ con, const double* __restrict__ val,
                                     const double* __restrict__ y, double* __restrict__ ypos, SpLen L,
                                     const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  double s = 0.0;
  for (int k = pos_ptr[p]; k < pos_ptr[p + 1]; ++k) {
    if (!WC_IN(kValPtr, k, L.nnz)) break;
    const int e = perm[k];
    if (!WC_IN(kValPerm, e, L.nnz)) continue;
    const int i = con[e];
    if (!WC_IN(kValCon, i, L.m)) continue;
    s = fma(y[i], val[e], s);
  }
  ypos[p] = s;
}

// Out[i, j] = sum over the pattern entries (i, c) of row i of Y[i, c] Bm[c, j]; grid (row blocks, ncols)
__global__ void sym_spmm_kernel(int n, const int32_t* __restrict__ yptr, const int32_t* __restrict__ ycol,
                                const int32_t* __restrict__ ypidx, const double* __restrict__ ypos,
                                const double* __restrict__ Bm, int64_t ldb, double* __restrict__ Out, int64_t ldo,
                                SpLen L, const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = blockIdx.y;
  const double* b = Bm + (int64_t)j * ldb;
  double s = 0.0;
  for (int k = yptr[i]; k < yptr[i + 1]; ++k) {
    if (!WC_IN(kMmPtr, k, L.nnzY)) break;
    const int p = ypidx[k], c = ycol[k];
    if (!WC_IN(kMmPidx, p, L.npos) || !WC_IN(kMmCol, c, n)) continue;
    s = fma(ypos[p], b[c], s);
  }
  Out[i + (int64_t)j * ldo] = s;
}

// F = E Y, column c of F = sum over the pattern entries (r, c) of Y[r, c] E[:, r]: one CTA per
// (column, block of 1024 rows); the entry loop is uniform over the CTA and every load of E is a
// coalesced column segment.
constexpr int EY_ROWS = 4;   // rows per thread
__global__ void sparse_EY_kernel(int n, const int32_t* __restrict__ yptr, const int32_t* __restrict__ ycol,
                                 const int32_t* __restrict__ ypidx, const double* __restrict__ ypos,
                                 const double* __restrict__ E, double* __restrict__ F, SpLen L,
                                 const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int c = blockIdx.x;
  const int i0 = blockIdx.y * (ST * EY_ROWS) + threadIdx.x;
  double acc[EY_ROWS];
#pragma unroll
  for (int q = 0; q < EY_ROWS; ++q) acc[q] = 0.0;
  for (int k = yptr[c]; k < yptr[c + 1]; ++k) {
    if (!WC_IN(kEyPtr, k, L.nnzY)) break;
    const int p = ypidx[k], col = ycol[k];
    if (!WC_IN(kEyPidx, p, L.npos) || !WC_IN(kEyCol, col, n)) continue;
    const double w = ypos[p];
    const double* ec = E + (int64_t)col * n;
#pragma unroll
    for (int q = 0; q < EY_ROWS; ++q) {
      const int i = i0 + q * ST;
      if (i < n) acc[q] = fma(w, ec[i], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < EY_ROWS; ++q) {
    const int i = i0 + q * ST;
    if (i < n) F[i + (int64_t)c * n] = acc[q];
  }
}

// (E Y E)[a, b] = <F[b, :], E[:, a]> with F = E Y, for the positions (a, b) of column b: one CTA
// per column b stages row b of F in shared memory, one warp per position reads a column of E.
__global__ void pos_dots_col_kernel(int n, const int32_t* __restrict__ cptr, const int32_t* __restrict__ pos_r,
                                    const double* __restrict__ E, const double* __restrict__ F,
                                    double* __restrict__ zpos, SpLen L, const int32_t* __restrict__ done) {
  if (done && *done) return;
  extern __shared__ double frow[];
  const int b = blockIdx.x;
  const int p0 = cptr[b], p1 = cptr[b + 1];
  if (p0 == p1) return;
  for (int c = threadIdx.x; c < n; c += blockDim.x) frow[c] = F[b + (int64_t)c * n];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = p0 + warp; p < p1; p += nw) {
    if (!WC_IN(kDotPtr, p, L.npos)) break;
    const int a = pos_r[p];
    if (!WC_IN(kDotRow, a, n)) continue;
    const double* ea = E + (int64_t)a * n;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s = fma(ea[c], frow[c], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) zpos[p] = s;
  }
}

__global__ void sparse_apply_pos_kernel(int n, int m, int r, const int32_t* __restrict__ con_ptr,
                                        const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                        const double* __restrict__ val, const int32_t* __restrict__ epos,
                                        const double* __restrict__ zpos, const double* __restrict__ U,
                                        const double* __restrict__ Q, double* __restrict__ out, SpLen L,
                                        const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int e = con_ptr[i]; e < con_ptr[i + 1]; ++e) {
    if (!WC_IN(kApPtr, e, L.nnz)) break;
    const int a = row[e], b = col[e];
    if (!WC_IN(kApRC, a, n) || !WC_IN(kApRC, b, n)) continue;
    const int p = zpos ? epos[e] : 0;
    if (zpos && !WC_IN(kApPos, p, L.npos)) continue;
    double z = zpos ? zpos[p] : 0.0;
    if (U) {
      double t = 0.0;
      for (int k = 0; k < r; ++k)
        t += U[a + (int64_t)k * n] * Q[b + (int64_t)k * n] + Q[a + (int64_t)k * n] * U[b + (int64_t)k * n];
      z += 0.5 * t;
    }
    s = fma(val[e] * (a == b ? 1.0 : 2.0), z, s);
  }
  out[i] = s;
}

// sum_i ||A_i||_F^2 = sum_e val_e^2 (2 if off-diagonal), per-block partials then one block
__global__ void sparse_sumsq_kernel(int64_t nnz, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(val[e] * val[e], row[e] == col[e] ? 1.0 : 2.0, acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Gram form of the d-space complement, one column pair (j1, j2) of the H_i = Vs^T A_i Q:
// cf_p = s_{con_p} w_p Q[y_p, j1] Q[y'_p, j2] for every term pair p (Q = Vs[:, :r]) ...
__global__ void gram_coef_kernel(int64_t np, int n, int j1, int j2, const int32_t* __restrict__ py,
                                 const int32_t* __restrict__ pyp, const int32_t* __restrict__ pcon,
                                 const double* __restrict__ pw, const double* __restrict__ Vs, double inv_beta,
                                 const double* __restrict__ lam, int m, double* __restrict__ cf) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const int y = py[p], yp = pyp[p], i = pcon[p];
    double v = 0.0;
    if (WC_IN(kGramIdx, y, n) && WC_IN(kGramIdx, yp, n) && WC_IN(kGramIdx, i, m))
      v = pw[p] * Vs[y + (int64_t)j1 * n] * Vs[yp + (int64_t)j2 * n] * (lam ? 1.0 / lam[i] : inv_beta);
    cf[p] = v;
  }
}

// ... then Y = W Vs: Y[x, k] = sum over the pairs p of row x of cf_p Vs[x'_p, k]; grid (rows, columns)
__global__ void gram_spmm_kernel(int n, int64_t np, const int32_t* __restrict__ pptr, const int32_t* __restrict__ pxp,
                                 const double* __restrict__ cf, const double* __restrict__ Vs, double* __restrict__ Y) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const int k = blockIdx.y;
  const double* vk = Vs + (int64_t)k * n;
  double s = 0.0;
  for (int p = pptr[x]; p < pptr[x + 1]; ++p) {
    if (!WC_IN(kGramPtr, p, np)) break;
    const int xp = pxp[p];
    if (!WC_IN(kGramIdx, xp, n)) continue;
    s = fma(cf[p], vk[xp], s);
  }
  Y[x + (int64_t)k * n] = s;
}

// h-coordinate of entry (a, j) of an n x r matrix and its weight in pack(.):  a < r: the svec
// position of (max, min) with 1 on the diagonal and sqrt2 / 2 off it; a >= r: r(r+1)/2 + (a - r) +
// j (n - r) with sqrt2
__device__ __forceinline__ int64_t hcoord(int n, int r, int a, int j, double& c) {
  if (a < r) {
    const int i = a > j ? a : j, jj = a > j ? j : a;
    c = (i == jj) ? 1.0 : 0.5 * WC_SQRT2;
    return svec_index(r, i, jj);
  }
  c = WC_SQRT2;
  return (int64_t)r * (r + 1) / 2 + (a - r) + (int64_t)j * (n - r);
}

// C[h(a1, j1), h(a2, j2)] += c(a1, j1) c(a2, j2) G[a1, a2]: within one (j1, j2) every (a1, a2) lands
// on its own entry of C, so no atomics; the column pairs run one after another (a fixed order).
// mirror (j1 != j2): the same value also at the transposed entry, which is the (j2, j1) pair's
// contribution (G_{j2 j1} = G_{j1 j2}^T): one product serves both pairs.  The two writes of one thread coincide only when h1 = h2 (then both add, as the two
// pairs do); two threads never write one entry.
__global__ void gram_scatter_kernel(int n, int r, int j1, int j2, int mirror, const double* __restrict__ G,
                                    double* __restrict__ C, int64_t ldc) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
    const int a1 = (int)(q % n), a2 = (int)(q / n);
    double c1, c2;
    const int64_t h1 = hcoord(n, r, a1, j1, c1), h2 = hcoord(n, r, a2, j2, c2);
    const double v = c1 * c2 * G[q];
    C[h1 + h2 * ldc] += v;
    if (mirror) C[h2 + h1 * ldc] += v;
  }
}

// One check of index i against bound and nothing else (no memory is addressed): lets a test see
// a violation recorded and reported without an out-of-range index ever reaching an access.
__global__ void oob_selftest_kernel(int64_t i, int64_t bound) { (void)WC_IN(kSelfTest, i, bound); }

__global__ void sum_parts_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) acc += part[q];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace

void sparse_adjoint(cudaStream_t st, const SparseA& S, int n, const double* y, double scale, double* Y,
                    const int32_t* done, int64_t* launches) {
  if (S.npos > 0)
    sparse_adjoint_kernel<<<nb(S.npos), ST, 0, st>>>(n, S.npos, S.pos_r, S.pos_c, S.pos_ptr, S.perm, S.con, S.val, y,
                                                     scale, Y, lens(S), done);
  if (launches) ++*launches;
}

void sparse_apply(cudaStream_t st, const SparseA& S, int n, int m, int r, const double* Z, const double* U,
                  const double* Q, double* out, const int32_t* done, int64_t* launches) {
  sparse_apply_kernel<<<nb(m), ST, 0, st>>>(n, m, r, S.con_ptr, S.row, S.col, S.val, Z, U, Q, out, lens(S), done);
  if (launches) ++*launches;
}

void sparse_B(cudaStream_t st, const SparseA& S, int n, int m, int r, const double* Vs, double* B, int64_t ldB,
              double* Bt, int64_t ldBt, int64_t* launches) {
  const int d = n * r - r * (r - 1) / 2;
  int64_t blocks = ((int64_t)m * d + ST - 1) / ST;
  if (blocks > 16 * (int64_t)g_num_sms) blocks = 16 * (int64_t)g_num_sms;
  sparse_B_kernel<<<(unsigned)blocks, ST, 0, st>>>(n, m, r, S.con_ptr, S.row, S.col, S.val, Vs, B, ldB, Bt, ldBt,
                                                   lens(S));
  if (launches) ++*launches;
}

void sparse_posval(cudaStream_t st, const SparseA& S, const double* y, double* ypos, const int32_t* done,
                   int64_t* launches) {
  if (S.npos > 0)
    sparse_posval_kernel<<<nb(S.npos), ST, 0, st>>>(S.npos, S.pos_ptr, S.perm, S.con, S.val, y, ypos, lens(S), done);
  if (launches) ++*launches;
}

void sparse_sym_spmm(cudaStream_t st, const SparseA& S, int n, int ncols, const double* ypos, const double* Bm,
                     int64_t ldb, double* Out, int64_t ldo, const int32_t* done, int64_t* launches) {
  dim3 grid(nb(n), (unsigned)ncols);
  sym_spmm_kernel<<<grid, ST, 0, st>>>(n, S.yptr, S.ycol, S.ypidx, ypos, Bm, ldb, Out, ldo, lens(S), done);
  if (launches) ++*launches;
}

void sparse_EY(cudaStream_t st, const SparseA& S, int n, const double* ypos, const double* E, double* F,
               const int32_t* done, int64_t* launches) {
  dim3 grid((unsigned)n, (unsigned)((n + ST * EY_ROWS - 1) / (ST * EY_ROWS)));
  sparse_EY_kernel<<<grid, ST, 0, st>>>(n, S.yptr, S.ycol, S.ypidx, ypos, E, F, lens(S), done);
  if (launches) ++*launches;
}

cudaError_t sparse_prepare(int n) {
  const size_t smem = (size_t)n * sizeof(double);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  return raise_dyn_smem((const void*)pos_dots_col_kernel, (int)smem);
}

cudaError_t sparse_pos_dots_col(cudaStream_t st, const SparseA& S, int n, const double* E, const double* F,
                                double* zpos, const int32_t* done, int64_t* launches) {
  const size_t smem = (size_t)n * sizeof(double);
  pos_dots_col_kernel<<<(unsigned)n, ST, smem, st>>>(n, S.cptr, S.pos_r, E, F, zpos, lens(S), done);
  if (launches) ++*launches;
  return cudaGetLastError();
}

void sparse_apply_pos(cudaStream_t st, const SparseA& S, int n, int m, int r, const double* zpos, const double* U,
                      const double* Q, double* out, const int32_t* done, int64_t* launches) {
  sparse_apply_pos_kernel<<<nb(m), ST, 0, st>>>(n, m, r, S.con_ptr, S.row, S.col, S.val, S.epos, zpos, U, Q, out,
                                                lens(S), done);
  if (launches) ++*launches;
}

void sparse_gram_spmm(cudaStream_t st, const SparseA& S, int n, int j1, int j2, const double* Vs, double inv_beta,
                      const double* lam, double* Y, int64_t* launches) {
  double* cf = S.pcf;   // the pairs' coefficients for this (j1, j2)
  const int64_t cb = std::min<int64_t>((S.npairs + ST - 1) / ST, 16 * (int64_t)g_num_sms);
  gram_coef_kernel<<<(unsigned)std::max<int64_t>(cb, 1), ST, 0, st>>>(S.npairs, n, j1, j2, S.py, S.pyp, S.pcon, S.pw,
                                                                      Vs, inv_beta, lam, S.m, cf);
  gram_spmm_kernel<<<dim3(nb(n), (unsigned)n), ST, 0, st>>>(n, S.npairs, S.pptr, S.pxp, cf, Vs, Y);
  if (launches) *launches += 2;
}

void sparse_gram_scatter(cudaStream_t st, int n, int r, int j1, int j2, bool mirror, const double* G, double* C,
                         int64_t ldc, int64_t* launches) {
  const int64_t nn = (int64_t)n * n;
  const int64_t blocks = std::min<int64_t>((nn + ST - 1) / ST, 16 * (int64_t)g_num_sms);
  gram_scatter_kernel<<<(unsigned)blocks, ST, 0, st>>>(n, r, j1, j2, mirror ? 1 : 0, G, C, ldc);
  if (launches) ++*launches;
}

cudaError_t sparse_bounds_selftest(cudaStream_t st, int64_t index, int64_t bound) {
  oob_selftest_kernel<<<1, 1, 0, st>>>(index, bound);
  return cudaGetLastError();
}

void sparse_sumsq(cudaStream_t st, const SparseA& S, double* out, double* scratch, int64_t* launches) {
  const int np = 2 * g_num_sms;
  sparse_sumsq_kernel<<<np, ST, 0, st>>>(S.nnz, S.row, S.col, S.val, scratch);
  sum_parts_kernel<<<1, ST, 0, st>>>(scratch, np, out);
  if (launches) *launches += 2;
}

}  // namespace wc

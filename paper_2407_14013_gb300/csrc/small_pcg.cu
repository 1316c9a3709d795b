// The whole FP64 PCG solve of the augmented system (eq. augsys; Def. pcg with Cor. pcg's start)
// for small DIAG problems (A_i = e_i e_i^T, m = n <= 128) in the m-space preconditioner form, held
// by one thread-block cluster of 8 or 16 CTAs: one launch instead of about 16 per iteration.
//
// An iteration of the launch chain it replaces is a string of tiny products (n x r outputs of
// length-n sums) and vector kernels; at n = 64 each one costs its launch and a few FP64 latency
// chains, so the iteration takes about 100 us while its arithmetic is about 60 K multiply-adds.
// Here the n rows (and the n columns of Vs for H = Vs^T diag(t) Q) are split over the CTAs of the
// cluster; each CTA keeps its slices of Vs, E o E and the preconditioner core in shared memory
// for the whole solve, computes its rows of each product (a warp per row, the lanes splitting the
// length-n sum, so that no FP64 dependency chain is longer than a few operations), and writes its
// rows into every CTA's copy of the result through distributed shared memory; a cluster barrier
// then gives every CTA the whole vector.  The O(m + d) work (the h-coordinate pack and unpack, the
// dot products, the PCG updates) is done by every CTA on its own copy of the vectors, in the same
// order, so every CTA holds bit-identical vectors and scalars and takes the same stop decision.
// Four cluster barriers per iteration; no flag waits.
//
// Per iteration, with t = p_u (operator) or z_u (preconditioner), Q = Vs[:, :r]:
//   operator        Up = Vs unpack(p_v);  H = Vs^T diag(p_u) Q
//                   (M p)_u = (E o E) p_u + rowdot(Up, Q);  (M p)_v = pack(H) - D p_v
//   preconditioner  w = r_u + rowdot(Vs unpack(D^{-1} r_v), Q);  z_u = K^{-1} w
//                   z_v = D^{-1} (pack(Vs^T diag(z_u) Q) - r_v)
// which is the m-space form P^{-1} = [K^{-1}, K^{-1} B D^{-1}; D^{-1} B^T K^{-1}, D^{-1} B^T K^{-1} B D^{-1} - D^{-1}]
// applied as in the launch chain (products with B from Vs: B t = rowdot(Vs unpack(t), Q),
// B^T u = pack(Vs^T diag(u) Q)), and the PCG scalars of Def. pcg.
#include <cooperative_groups.h>

#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "kernels.h"
#include "pcg.h"

namespace wc {

namespace {

namespace cg = cooperative_groups;

constexpr int SCL = 16;            // CTAs of the cluster: 16 (non-portable) where it launches, else 8
constexpr int SNT = 256;           // threads per CTA
constexpr int SNW = SNT / 32;
constexpr int SRMAX = 16;          // largest r
constexpr int SNMAX = 128;         // largest n

struct SmallArgs {
  int n, r, d, chunk, start0, slabs;
  double rtol;
  const double *Vs, *EE, *Pinv, *Dv;
  const double *part, *bt, *Ct, *Hg;   // the right side's inputs: diag(F E) slabs, b~, C~, Vs^T C~ Q
  double *g, *x, *rv, *z, *p, *Ap;
  PcgCtl* ctl;
};

// Shared-memory layout (doubles): the CTA's slices, then the vectors and scratch.
struct SmallLayout {
  int vsr, vsc, q, eer, pir, dv, idv, X, R, Z, P, AP, hp, ha, hq, tq, wb, red, cbp, total;
  __host__ __device__ SmallLayout(int n, int r, int d, int chunk) {
    const int nt = n + d;
    int o = 0;
    vsr = o; o += chunk * n;     // rows i0.. of Vs:          vsr[il n + a] = Vs[i0 + il, a]
    vsc = o; o += chunk * n;     // columns i0.. of Vs:       vsc[al n + i] = Vs[i, i0 + al]
    q = o;   o += n * r;         // Q = Vs[:, :r], column-major
    eer = o; o += chunk * n;     // rows i0.. of E o E (symmetric: its columns)
    pir = o; o += chunk * n;     // rows i0.. of K^{-1} (symmetric)
    dv = o;  o += d;
    idv = o; o += d;             // 1 / D
    X = o;   o += nt;
    R = o;   o += nt;
    Z = o;   o += nt;
    P = o;   o += nt;
    AP = o;  o += nt;
    ha = o;  o += n * r;         // H of the operator (rows from every CTA)
    hq = o;  o += n * r;         // H of the preconditioner (rows from every CTA)
    // the unpack of a v-block (every CTA makes its own) shares hq: the unpack is written at the
    // start of an apply and read before its first cluster barrier, and hq receives the other
    // CTAs' rows only between the second and third barriers of a preconditioner apply
    hp = hq;
    tq = o;  o += n * r;         // T = diag(t) Q for H = Vs^T T (every CTA makes its own)
    wb = o;  o += n;             // w = r_u + B D^{-1} r_v (rows from every CTA)
    red = o; o += 64;            // block reductions
    cbp = o; o += 32;            // every CTA's share of ||C~||_F^2 + ||b~||^2
    total = o;
  }
};

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// What every pass needs to find its data: the shape, this CTA's rows, the shared memory.
struct SmallCtx {
  int n, r, d, chunk, i0, rows, ncta;
  double* sm;
};

// Sum over the CTA's threads, valid in every thread: a butterfly in each warp, then the SNW warp
// totals by a three-level butterfly (eight dependent additions in all); fixed order, so every CTA
// of the cluster gets the same bits from the same data.
__device__ double cta_sum(double v, double* red) {
  v = warp_allsum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();   // red may still be read by the previous sum
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = red[lane & (SNW - 1)];
#pragma unroll
  for (int o = SNW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// <a, b> over [0, len), the same bits in every CTA (fixed thread mapping and reduction order)
__device__ double cta_dot(const double* a, const double* b, int len, double* red) {
  double s = 0.0;
  for (int q = threadIdx.x; q < len; q += SNT) s = fma(a[q], b[q], s);
  return cta_sum(s, red);
}

// Hp = unpack(v) (n x r, column-major), v scaled by D^{-1} first when idv != NULL
__device__ void cta_unpack(int n, int r, const double* v, const double* idv, double* Hp) {
  for (int q = threadIdx.x; q < n * r; q += SNT) {
    const int j = q / n, a = q - j * n;
    double val;
    if (a < r) {
      const int i = a > j ? a : j, jj = a > j ? j : a;
      const int k = (int)svec_index(r, i, jj);
      const double hv = idv ? v[k] * idv[k] : v[k];
      val = (i == jj) ? hv : hv * WC_RSQRT2;
    } else {
      const int k = r * (r + 1) / 2 + (a - r) + j * (n - r);
      val = WC_SQRT2 * (idv ? v[k] * idv[k] : v[k]);
    }
    Hp[q] = val;
  }
}

// The unpack of one v-block entry k (value val, already scaled as wanted) into Hp: the thread that
// makes entry k writes its one or two places, so an update loop can leave the unpack of its vector
// ready for the next product pass (the inverse of the index map of cta_unpack).
__device__ __forceinline__ void hp_put(int n, int r, int k, double val, double* Hp) {
  const int nb = r * (r + 1) / 2;
  if (k < nb) {
    int jj = 0, base = 0;
    while (k >= base + (r - jj)) {
      base += r - jj;
      ++jj;
    }
    const int i = jj + (k - base);
    if (i == jj) {
      Hp[i + jj * n] = val;
    } else {
      Hp[i + jj * n] = val * WC_RSQRT2;
      Hp[jj + i * n] = val * WC_RSQRT2;
    }
  } else {
    const int q = k - nb;
    Hp[r + q % (n - r) + (q / (n - r)) * n] = WC_SQRT2 * val;
  }
}

// Transposed butterfly over the warp of K accumulators per lane (K a power of two, 1..32): at
// each of the first log2 K levels a lane keeps half of its live accumulators (the lower half if
// its lane bit is clear) and adds the partner's copy of that half, so K - 1 additions leave one
// accumulator per lane; plain butterfly levels finish it.  Returns the total of component
// lane >> (5 - log2 K), the same bits in every lane that holds it.  FP64 additions cost a warp
// instruction each on GB300's narrow FP64 pipe: K - 1 + 5 - log2 K of them instead of 5 K.
template <int K>
__device__ __forceinline__ double warp_treduce(double (&a)[K], int lane) {
#pragma unroll
  for (int h = K / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const double send = upper ? a[j] : a[j + h];
      const double keep = upper ? a[j + h] : a[j];
      a[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double v = a[0];
#pragma unroll
  for (int o = 16 / K; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int K>
__device__ __forceinline__ int treduce_comp(int lane) {
  return K == 1 ? 0 : lane >> (5 - (K >= 32 ? 5 : K >= 16 ? 4 : K >= 8 ? 3 : K >= 4 ? 2 : 1));
}

// Writes the total v of component comp (held by the 32 / K lanes with that component) into
// dst of every CTA of the cluster (ncta of them): each of those lanes covers ncta K / 32 ranks.
template <int K>
__device__ __forceinline__ void put_all(const cg::cluster_group& cl, int lane, int ncta, double v, double* dst) {
  constexpr int LPC = 32 / K;                       // lanes per component
  const int t = lane & (LPC - 1);
  for (int q = t; q < ncta; q += LPC) *cl.map_shared_rank(dst, q) = v;
}

// This CTA's rows i = i0 + il of U = Vs Hp (Hp in shared memory), each finished into
// w[i] = v_u[i] + sum_k U[i, k] Q[i, k] (w = r_u + B D^{-1} r_v) and written at dst[i] in every
// CTA of the cluster.  A warp per row: the lanes split the length-n sums (RB independent chains
// each), a transposed butterfly finds U[i, :], and a butterfly over the components forms the sum.
template <int RB>
__device__ __noinline__ void rows_pass(SmallCtx c, const double* vu, double* dst) {
  const cg::cluster_group cl = cg::this_cluster();
  const SmallLayout L(c.n, c.r, c.d, c.chunk);
  const int n = c.n, r = c.r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* Hp = c.sm + L.hp;
  const int comp = treduce_comp<RB>(lane);
  for (int il = warp; il < c.rows; il += SNW) {
    const double* vr = c.sm + L.vsr + il * n;
    double acc[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] = 0.0;
    for (int a = lane; a < n; a += 32) {
      const double va = vr[a];
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (j < r) acc[j] = fma(va, Hp[a + j * n], acc[j]);
    }
    const int i = c.i0 + il;
    const double u = warp_treduce<RB>(acc, lane);                  // U[i, comp]
    double t = comp < r ? u * c.sm[L.q + i + comp * n] : 0.0;      // U[i, comp] Q[i, comp]
#pragma unroll
    for (int o = 16; o >= 32 / RB; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const double v = vu[i] + t;
    if (lane < c.ncta) *cl.map_shared_rank(dst + i, lane) = v;
  }
}

// This CTA's rows a = i0 + al of H = Vs^T T with T = diag(t) Q (n x r, formed in shared memory
// beforehand): H[a, j] = sum_i Vs[i, a] T[i, j], written at dstH[a + j n] in every CTA.
template <int RB>
__device__ __noinline__ void cols_pass(SmallCtx c, double* dstH) {
  const cg::cluster_group cl = cg::this_cluster();
  const SmallLayout L(c.n, c.r, c.d, c.chunk);
  const int n = c.n, r = c.r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* T = c.sm + L.tq;
  const int comp = treduce_comp<RB>(lane);
  for (int al = warp; al < c.rows; al += SNW) {
    const double* vc = c.sm + L.vsc + al * n;
    double acc[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double w = vc[i];
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (j < r) acc[j] = fma(w, T[i + j * n], acc[j]);
    }
    const int a = c.i0 + al;
    const double h = warp_treduce<RB>(acc, lane);
    if (comp < r) put_all<RB>(cl, lane, c.ncta, h, dstH + a + comp * n);
  }
}

// The operator's two products in one pass over this CTA's rows: row i of U = Vs unpack(v_v) and
// row i of H = Vs^T T (T = diag(v_u) Q) side by side in one transposed butterfly of 2 RB
// accumulators, plus ((E o E) v_u)_i; finished into (M v)_u[i] = ((E o E) v_u)_i +
// sum_k U[i, k] Q[i, k] at dst[i] and H[i, :] at dstH, in every CTA.
template <int RB>
__device__ __noinline__ void op_pass(SmallCtx c, const double* v, double* dst, double* dstH) {
  constexpr int K = 2 * RB;
  const cg::cluster_group cl = cg::this_cluster();
  const SmallLayout L(c.n, c.r, c.d, c.chunk);
  const int n = c.n, r = c.r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* Hp = c.sm + L.hp;
  const double* T = c.sm + L.tq;
  const int comp = treduce_comp<K>(lane);                          // < RB: U[i, comp]; else H[i, comp - RB]
  for (int il = warp; il < c.rows; il += SNW) {
    const double* vr = c.sm + L.vsr + il * n;
    const double* vc = c.sm + L.vsc + il * n;
    const double* er = c.sm + L.eer + il * n;
    double acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = 0.0;
    double ee = 0.0;
    for (int x = lane; x < n; x += 32) {
      const double va = vr[x], vcx = vc[x];
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        if (j < r) {
          acc[j] = fma(va, Hp[x + j * n], acc[j]);
          acc[RB + j] = fma(vcx, T[x + j * n], acc[RB + j]);
        }
      }
      ee = fma(er[x], v[x], ee);
    }
    const int i = c.i0 + il;
    const double s = warp_treduce<K>(acc, lane);
    ee = warp_allsum(ee);
    // (M v)_u[i]: the terms U[i, k] Q[i, k] sit in the lanes of components k < RB (lanes < 16)
    double t = comp < r ? s * c.sm[L.q + i + comp * n] : 0.0;
#pragma unroll
    for (int o = 8; o >= 32 / K; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < c.ncta) *cl.map_shared_rank(dst + i, lane) = ee + t;
    if (comp >= RB && comp - RB < r) put_all<K>(cl, lane, c.ncta, s, dstH + i + (comp - RB) * n);
  }
}

// This CTA's rows of z_u = K^{-1} w (w gathered in shared memory), written at dst[i] everywhere.
__device__ void pinv_pass(SmallCtx c, double* dst) {
  const cg::cluster_group cl = cg::this_cluster();
  const SmallLayout L(c.n, c.r, c.d, c.chunk);
  const int n = c.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int il = warp; il < c.rows; il += SNW) {
    const double* pr = c.sm + L.pir + il * n;
    double s = 0.0;
    for (int l = lane; l < n; l += 32) s = fma(pr[l], c.sm[L.wb + l], s);
    s = warp_allsum(s);
    if (lane < c.ncta) *cl.map_shared_rank(dst + c.i0 + il, lane) = s;
  }
}

// T = diag(t) Q (n x r) in shared memory, every CTA its own copy
__device__ void cta_scale_q(int n, int r, const double* t, const double* Q, double* T) {
  for (int q = threadIdx.x; q < n * r; q += SNT) {
    const int j = q / n, i = q - j * n;
    T[q] = t[i] * Q[q];
  }
}

// out = M v, or g - M v when g != NULL (one cluster barrier); returns <v, out>
template <int RB>
__device__ __noinline__ double op_apply(SmallCtx c, const double* v, double* out, const double* __restrict__ g,
                                        bool ready) {
  const cg::cluster_group cl = cg::this_cluster();
  const SmallLayout L(c.n, c.r, c.d, c.chunk);
  const int n = c.n, r = c.r, d = c.d, m = n;
  if (!ready) {   // else the update loop that made v left them in place
    cta_unpack(n, r, v + m, nullptr, c.sm + L.hp);
    cta_scale_q(n, r, v, c.sm + L.q, c.sm + L.tq);
  }
  __syncthreads();
  op_pass<RB>(c, v, out, c.sm + L.ha);
  cl.sync();
  double acc = 0.0;
  for (int q = threadIdx.x; q < m + d; q += SNT) {
    double val = q < m ? out[q] : pack_at(c.sm + L.ha, n, n, r, q - m) - c.sm[L.dv + q - m] * v[q];
    if (g) val = g[q] - val;
    out[q] = val;
    acc = fma(v[q], val, acc);
  }
  return cta_sum(acc, c.sm + L.red);   // its barriers also order the writes above
}

// z = P^{-1} rin in the m-space form (three cluster barriers); returns <rin, z>
template <int RB>
__device__ __noinline__ double pc_apply(SmallCtx c, const double* rin, double* z, bool ready) {
  const cg::cluster_group cl = cg::this_cluster();
  const SmallLayout L(c.n, c.r, c.d, c.chunk);
  const int n = c.n, r = c.r, d = c.d, m = n;
  if (!ready) cta_unpack(n, r, rin + m, c.sm + L.idv, c.sm + L.hp);   // unpack(D^{-1} r_v)
  __syncthreads();
  rows_pass<RB>(c, rin, c.sm + L.wb);                    // w = r_u + B D^{-1} r_v
  cl.sync();
  pinv_pass(c, z);                                              // z_u = K^{-1} w
  cl.sync();
  cta_scale_q(n, r, z, c.sm + L.q, c.sm + L.tq);
  __syncthreads();
  cols_pass<RB>(c, c.sm + L.hq);                                // Vs^T diag(z_u) Q
  cl.sync();
  double acc = 0.0;
  for (int q = threadIdx.x; q < m + d; q += SNT) {              // z_v = D^{-1}(B^T z_u - r_v)
    double zq = z[q];
    if (q >= m) {
      zq = (pack_at(c.sm + L.hq, n, n, r, q - m) - rin[q]) * c.sm[L.idv + q - m];
      z[q] = zq;
    }
    acc = fma(rin[q], zq, acc);
  }
  return cta_sum(acc, c.sm + L.red);
}

template <int RB>
__global__ void __launch_bounds__(SNT) small_pcg_kernel(SmallArgs A) {
  const cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  PcgCtl* ctl = A.ctl;
  const int n = A.n, r = A.r, d = A.d, m = n, nt = n + d;
  const SmallLayout L(n, r, d, A.chunk);
  const int rank = (int)cl.block_rank();
  SmallCtx c;
  c.n = n;
  c.r = r;
  c.d = d;
  c.chunk = A.chunk;
  c.ncta = (int)cl.num_blocks();
  c.i0 = rank * A.chunk;
  c.rows = max(0, min(A.chunk, n - c.i0));
  c.sm = sm;
  const int i0 = c.i0, rows = c.rows;
  // this CTA's slices and the shared operands, kept for the whole solve
#pragma unroll 4
  for (int q = threadIdx.x; q < rows * n; q += SNT) {
    const int il = q % rows, a = q / rows;
    sm[L.vsr + il * n + a] = A.Vs[(i0 + il) + (int64_t)a * n];
    const int al = q / n, i = q % n;
    sm[L.vsc + al * n + i] = A.Vs[i + (int64_t)(i0 + al) * n];
    sm[L.eer + al * n + i] = A.EE[i + (int64_t)(i0 + al) * n];
    sm[L.pir + al * n + i] = A.Pinv[i + (int64_t)(i0 + al) * m];
  }
  for (int q = threadIdx.x; q < n * r; q += SNT) sm[L.q + q] = A.Vs[q];
  for (int h = threadIdx.x; h < d; h += SNT) {
    const double dh = A.Dv[h];
    sm[L.dv + h] = dh;
    sm[L.idv + h] = 1.0 / dh;   // the preconditioner multiplies by D^{-1} (one division per entry per solve)
  }
  double* X = sm + L.X;
  double* R = sm + L.R;
  double* Z = sm + L.Z;
  double* P = sm + L.P;
  double* AP = sm + L.AP;
  double* red = sm + L.red;
  // the right side of eq. augsys, g = [b~ + tau^2 diag(F E); tau^2 pack(Vs^T C~ Q)] (kept in AP
  // until the loop needs it), x0 = [0; -g_v / D] (Cor. pcg's printed start) and [0; g_v] (the
  // right side of the default start's correction)
  const double tau = ctl->tau, t2 = tau * tau;
  __syncthreads();   // D in shared memory
  for (int q = threadIdx.x; q < nt; q += SNT) {
    double v;
    if (q < m) {
      double a = 0.0;
      for (int sl = 0; sl < A.slabs; ++sl) a += A.part[(int64_t)sl * m + q];
      v = A.bt[q] + t2 * a;
    } else {
      v = t2 * pack_at(A.Hg, n, n, r, q - m);
    }
    AP[q] = v;
    X[q] = (A.start0 || q < m) ? 0.0 : -v / sm[L.dv + q - m];
    Z[q] = q < m ? 0.0 : v;
    if (rank == 0) A.g[q] = v;
  }
  // ||[svec C~; b~]||^2 (the right side of (Newt-eps)): this CTA's share now, the total after the
  // next cluster barrier
  const int64_t ncb = (int64_t)n * n + m, seg = (ncb + c.ncta - 1) / c.ncta;
  double cpart = 0.0;
  for (int64_t q = rank * seg + threadIdx.x; q < ncb && q < (rank + 1) * seg; q += SNT) {
    const double v = q < (int64_t)n * n ? A.Ct[q] : A.bt[q - (int64_t)n * n];
    cpart = fma(v, v, cpart);
  }
  cpart = cta_sum(cpart, red);
  const double gg = cta_dot(AP, AP, nt, red);
  const int max_iters = ctl->max_iters;
  int iters = 0, status = ctl->status, done = 0;   // status: a non-positive pivot in the setup
  double rr = 0.0, rr0 = 0.0, rz = 0.0, rz_new = 0.0, beta = 0.0, alpha = 0.0, pAp = 0.0, tol2 = 0.0;
  if (!isfinite(gg)) status = 5;
  if (status != 0) done = 1;
  cl.sync();   // every CTA has started and holds its operands before any writes into it
  if (threadIdx.x < c.ncta) *cl.map_shared_rank(sm + L.cbp + rank, (int)threadIdx.x) = cpart;
  auto rhs_norm2 = [&]() {   // after a cluster barrier that follows the shares' writes
    double cb = 0.0;
    for (int k = 0; k < c.ncta; ++k) cb += sm[L.cbp + k];
    return cb;
  };
  if (done) cl.sync();
  if (A.start0 && !done) {   // x0 = P^{-1} [0; g_v], so that P x0 = [0; g_v] and r0_v = 0 (Cor. pcg)
    const double t = pc_apply<RB>(c, Z, X, false);
    if (!isfinite(t)) { status = 5; done = 1; }
  }
  if (!done) {   // r0 = g - M x0, ||r0||^2 and the stop test; z0 = P^{-1} r0; p0 = z0
    op_apply<RB>(c, X, R, AP, false);
    // stop when ||r_k|| <= rtol ||[svec C~; b~]|| (the (Newt-eps) residual of the recovered direction)
    tol2 = A.rtol * A.rtol * rhs_norm2();
    rr = cta_dot(R, R, nt, red);
    if (iters == 0) rr0 = rr;
    if (!isfinite(rr)) { status = 5; done = 1; }
    else if (rr <= tol2) done = 1;
  }
  if (!done) {
    rz = pc_apply<RB>(c, R, Z, false);
    beta = 0.0;
    if (!isfinite(rz)) { status = 5; done = 1; }
    for (int q = threadIdx.x; q < nt; q += SNT) {   // p0 = z0, with its unpack and diag(p_u) Q
      const double pq = Z[q];
      P[q] = pq;
      if (q >= m) {
        hp_put(n, r, q - m, pq, sm + L.hp);
      } else {
        for (int j = 0; j < r; ++j) sm[L.tq + q + j * n] = pq * sm[L.q + q + j * n];
      }
    }
    __syncthreads();
  }
  while (!done) {
    pAp = op_apply<RB>(c, P, AP, nullptr, true);
    // Def. pcg has no sign condition: with the indefinite preconditioner <p, M p> is positive in
    // exact arithmetic but may change sign at the rounding floor
    if (pAp == 0.0 || !isfinite(pAp) || !isfinite(rz)) { status = 5; done = 1; break; }
    alpha = rz / pAp;
    double acc = 0.0;
    for (int q = threadIdx.x; q < nt; q += SNT) {
      X[q] = fma(alpha, P[q], X[q]);
      const double rq = fma(-alpha, AP[q], R[q]);
      R[q] = rq;
      if (q >= m) hp_put(n, r, q - m, rq * sm[L.idv + q - m], sm + L.hp);   // unpack(D^{-1} r_v) for the next apply
      acc = fma(rq, rq, acc);
    }
    rr = cta_sum(acc, red);
    iters += 1;
    if (!isfinite(rr)) { status = 5; done = 1; }
    else if (rr <= tol2) { status = 0; done = 1; }
    else if (iters >= max_iters) { status = 4; done = 1; }
    if (done) break;
    const double t = pc_apply<RB>(c, R, Z, true);
    if (!isfinite(t)) { status = 5; done = 1; }
    rz_new = t;
    beta = t / rz;
    rz = t;
    if (done) break;
    for (int q = threadIdx.x; q < nt; q += SNT) {   // p = z + beta p, with its unpack and diag(p_u) Q
      const double pq = fma(beta, P[q], Z[q]);
      P[q] = pq;
      if (q >= m) {
        hp_put(n, r, q - m, pq, sm + L.hp);
      } else {
        for (int j = 0; j < r; ++j) sm[L.tq + q + j * n] = pq * sm[L.q + q + j * n];
      }
    }
    __syncthreads();
  }
  // the iterate and the scalars back to global memory (every CTA holds the same: rank 0 writes)
  if (rank == 0) {
    for (int q = threadIdx.x; q < nt; q += SNT) {
      A.x[q] = X[q];
      A.rv[q] = R[q];
      A.z[q] = Z[q];
      A.p[q] = P[q];
      A.Ap[q] = AP[q];
    }
    if (threadIdx.x == 0) {
      const double cb = rhs_norm2();
      ctl->g_norm2 = gg;
      ctl->newt_rhs2 = cb;
      ctl->tol2 = A.rtol * A.rtol * cb;
      ctl->rr = rr;
      ctl->rr0 = rr0;
      ctl->rz = rz;
      ctl->rz_new = rz_new;
      ctl->beta = beta;
      ctl->alpha = alpha;
      ctl->pAp = pAp;
      ctl->iters = iters;
      ctl->status = status;
      ctl->done = 1;
    }
  }
  cl.sync();   // no CTA leaves while another may still address its shared memory
}

}  // namespace

namespace {

const void* small_pcg_fn(int r) {
  return r <= 4 ? (const void*)small_pcg_kernel<4>
                : r <= 8 ? (const void*)small_pcg_kernel<8> : (const void*)small_pcg_kernel<SRMAX>;
}

size_t layout_bytes(int n, int r, int d, int ncta) {
  return (size_t)SmallLayout(n, r, d, (n + ncta - 1) / ncta).total * sizeof(double);
}

// Whether a 16-CTA cluster of this kernel (one CTA per SM at up to 227 KB of shared memory) can
// be resident on this device: asked once per kernel, by the occupancy query.
bool cluster16_ok(const void* fn) {
  static std::mutex mu;
  static std::unordered_map<const void*, bool> known;
  std::lock_guard<std::mutex> lock(mu);
  auto it = known.find(fn);
  if (it != known.end()) return it->second;
  bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            raise_dyn_smem(fn, 227 * 1024) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SCL);
    cfg.blockDim = dim3(SNT);
    cfg.dynamicSmemBytes = 227 * 1024;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = SCL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int num = 0;
    ok = cudaOccupancyMaxActiveClusters(&num, fn, &cfg) == cudaSuccess && num >= 1;
  }
  cudaGetLastError();
  known[fn] = ok;
  return ok;
}

}  // namespace

int small_pcg_plan(int n, int r, int d, size_t* bytes) {
  if (bytes) *bytes = 0;
  if (n < 2 || n > SNMAX || r < 1 || r > SRMAX || r >= n) return 0;
  constexpr size_t kMax = 227 * 1024;
  // 16 CTAs once there are rows for them (twice the FP64 pipes for the products), else 8
  if (n > 32 && layout_bytes(n, r, d, SCL) <= kMax && cluster16_ok(small_pcg_fn(r))) {
    if (bytes) *bytes = layout_bytes(n, r, d, SCL);
    return SCL;
  }
  if (layout_bytes(n, r, d, 8) > kMax) return 0;
  if (bytes) *bytes = layout_bytes(n, r, d, 8);
  return 8;
}

cudaError_t launch_small_pcg(cudaStream_t st, int n, int r, int d, int start0, const double* Vs, const double* EE,
                             const double* Pinv, const double* Dv, const double* part, int slabs, const double* bt,
                             const double* Ct, const double* H, double rtol, double* g, double* x, double* rv,
                             double* z, double* p, double* Ap, PcgCtl* ctl, int64_t* launches) {
  size_t bytes = 0;
  const int ncta = small_pcg_plan(n, r, d, &bytes);
  if (ncta == 0) return cudaErrorInvalidValue;
  const void* fn = small_pcg_fn(r);
  cudaError_t e = raise_dyn_smem(fn, (int)bytes);
  if (e != cudaSuccess) return e;
  SmallArgs A;
  A.n = n;
  A.r = r;
  A.d = d;
  A.chunk = (n + ncta - 1) / ncta;
  A.start0 = start0;
  A.slabs = slabs;
  A.rtol = rtol;
  A.part = part;
  A.bt = bt;
  A.Ct = Ct;
  A.Hg = H;
  A.Vs = Vs;
  A.EE = EE;
  A.Pinv = Pinv;
  A.Dv = Dv;
  A.g = g;
  A.x = x;
  A.rv = rv;
  A.z = z;
  A.p = p;
  A.Ap = Ap;
  A.ctl = ctl;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ncta);
  cfg.blockDim = dim3(SNT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[] = {&A};
  e = cudaLaunchKernelExC(&cfg, fn, args);
  if (launches) ++*launches;
  return e;
}

}  // namespace wc

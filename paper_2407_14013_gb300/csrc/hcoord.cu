// Coordinates of range(Q) (Section 5 and Lemma spanQ): h = [svec B; vec N] with B r x r
// symmetric and N (n - r) x r column-major, d = r(r+1)/2 + (n-r) r = n r - r(r-1)/2, and
//   Q h     = svec( [Q Qp] [B; sqrt2 N] Q^T )            (symmetric part)
//   Q^T X   = [ svec(Q^T X Q); sqrt2 vec(Qp^T X Q) ].
// With Vs = [Q Qp] and H = Vs^T X Q (n x r), Q^T svec(X) = pack(H); with Hp = [B; sqrt2 N],
// Q h = svec(sym(Vs Hp Q^T)).
#include "common.cuh"
#include "kernels.h"

namespace wc {

namespace {

__global__ void h_pack_kernel(int n, int r, const double* __restrict__ H, int64_t ldH, double c_out,
                              const double* __restrict__ in, double c_in, const double* __restrict__ Dv,
                              const double* __restrict__ pv, double* __restrict__ out,
                              const int32_t* __restrict__ done) {
  if (done && *done) return;
  const int d = n * r - r * (r - 1) / 2;
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= d) return;
  double v = c_out * pack_at(H, ldH, n, r, h);
  if (in) v += c_in * in[h];
  if (Dv) v -= Dv[h] * pv[h];
  out[h] = v;
}

template <typename T>
__global__ void h_unpack_kernel(int n, int r, const T* __restrict__ h, const T* __restrict__ Dv, T* __restrict__ Hp,
                                const int32_t* __restrict__ done) {
  if (done && *done) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * r) return;
  const int a = q % n, j = q / n;
  double v;
  if (a < r) {
    int i = a > j ? a : j, jj = a > j ? j : a;
    const int k = svec_index(r, i, jj);
    double hv = Dv ? (double)h[k] / (double)Dv[k] : (double)h[k];
    v = (i == jj) ? hv : hv * WC_RSQRT2;
  } else {
    const int k = r * (r + 1) / 2 + (a - r) + j * (n - r);
    v = WC_SQRT2 * (Dv ? (double)h[k] / (double)Dv[k] : (double)h[k]);
  }
  Hp[q] = (T)v;
}

__global__ void h_pack_rows_kernel(int n, int r, int mb, int i0, const double* __restrict__ H,
                                   double* __restrict__ B, int64_t ldB, double* __restrict__ Bt, int64_t ldBt) {
  const int d = n * r - r * (r - 1) / 2;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)mb * d) return;
  const int il = (int)(q / d), h = (int)(q % d);
  // column j of H_il is column j * mb + il of H: H_il = H + il * n with leading dimension mb * n
  const double v = pack_at(H + (int64_t)il * n, (int64_t)mb * n, n, r, h);
  B[(int64_t)(i0 + il) * ldB + h] = v;
  if (Bt) Bt[(int64_t)h * ldBt + i0 + il] = v;
}

// DIAG: A_i = e_i e_i^T, so Vs^T A_i Q = Vs[i, :]^T Q[i, :].
__global__ void h_pack_rows_diag_kernel(int n, int r, const double* __restrict__ Vs, double* __restrict__ B,
                                        int64_t ldB, double* __restrict__ Bt, int64_t ldBt) {
  const int d = n * r - r * (r - 1) / 2;
  const int nb = r * (r + 1) / 2;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * d) return;
  const int i = (int)(q / d), h = (int)(q % d);
  double v;
  if (h < nb) {
    int j = 0, base = 0;
    while (h >= base + (r - j)) { base += r - j; ++j; }
    int a = j + (h - base);
    double x = Vs[i + (int64_t)a * n] * Vs[i + (int64_t)j * n];
    v = (a == j) ? x : WC_SQRT2 * x;    // symmetric part of the outer product is itself
  } else {
    int qq = h - nb;
    int k = qq % (n - r), j = qq / (n - r);
    v = WC_SQRT2 * Vs[i + (int64_t)(r + k) * n] * Vs[i + (int64_t)j * n];
  }
  B[(int64_t)i * ldB + h] = v;
  if (Bt) Bt[(int64_t)h * ldBt + i] = v;
}

inline unsigned nblk(int64_t total, int t) { return (unsigned)((total + t - 1) / t); }

}  // namespace

void h_pack(cudaStream_t st, int n, int r, const double* H, int64_t ldH, double c_out, const double* in,
            double c_in, const double* Dv, const double* pv, double* out, const int32_t* done,
            int64_t* launches) {
  int d = n * r - r * (r - 1) / 2;
  h_pack_kernel<<<nblk(d, 256), 256, 0, st>>>(n, r, H, ldH, c_out, in, c_in, Dv, pv, out, done);
  if (launches) ++*launches;
}

template <typename T>
void h_unpack(cudaStream_t st, int n, int r, const T* h, T* Hp, const int32_t* done, int64_t* launches,
              const T* Dv) {
  h_unpack_kernel<T><<<nblk((int64_t)n * r, 256), 256, 0, st>>>(n, r, h, Dv, Hp, done);
  if (launches) ++*launches;
}

template void h_unpack<double>(cudaStream_t, int, int, const double*, double*, const int32_t*, int64_t*,
                               const double*);

void h_pack_rows(cudaStream_t st, int n, int r, int mb, int i0, const double* H, double* B,
                 int64_t ldB, double* Bt, int64_t ldBt, int64_t* launches) {
  int d = n * r - r * (r - 1) / 2;
  h_pack_rows_kernel<<<nblk((int64_t)mb * d, 256), 256, 0, st>>>(n, r, mb, i0, H, B, ldB, Bt, ldBt);
  if (launches) ++*launches;
}

void h_pack_rows_diag(cudaStream_t st, int n, int r, const double* Vs, double* B, int64_t ldB,
                      double* Bt, int64_t ldBt, int64_t* launches) {
  int d = n * r - r * (r - 1) / 2;
  h_pack_rows_diag_kernel<<<nblk((int64_t)n * d, 256), 256, 0, st>>>(n, r, Vs, B, ldB, Bt, ldBt);
  if (launches) ++*launches;
}

}  // namespace wc

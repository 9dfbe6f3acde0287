// Expected degrees and strengths and their gradients: the O(N^2) sums that
// parameter inference has to evaluate (Sec. 2.2, Sec. 2.5, Sec. 4).
//
//   <k_i> = sum_{j != i} p_ij,   <s_i> = sum_{j != i} m_ij,   m_ij = p_ij / (1 - r_ij)
//
// with E[w | w > 0] = 1 / (1 - r) from Eq. 4.  Each thread owns one row i and
// walks all j in tiles staged through shared memory, recomputing every pair
// term (nothing of size N^2 is stored).  Sums run in FP64 in a fixed order:
// a per-tile partial, then the running total.
//
// Derivatives (A = a_i a_j, a = x y, r = y_i y_j, D = 1 - r + A, z = x_i x_j):
//   UBCM  dp/dx_i = x_j / (1 + z)^2
//   UECM  dp/dx_i = y_i a_j (1 - r) / D^2       dm/dx_i = y_i a_j / D^2
//         dp/dy_i = x_i a_j / D^2               dm/dy_i = x_i a_j / (D^2 (1 - r)) + p y_j / (1 - r)^2
// which equal p(1-p)/x_i, p/(y_i D), ... without dividing by x_i or y_i.
#include "mh_internal.cuh"

namespace mh {

namespace {

constexpr int kPairThreads = 256;

template <int kModel>
__global__ void __launch_bounds__(kPairThreads) expected_fwd_kernel(const double* __restrict__ x,
                                                                     const double* __restrict__ y, int64_t n,
                                                                     double* __restrict__ k_out,
                                                                     double* __restrict__ s_out) {
  __shared__ double sa[kPairThreads];
  __shared__ double sy[kPairThreads];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kPairThreads + threadIdx.x;
  const bool row = i < n;
  double ai = 0.0, yi = 0.0;
  if (row) {
    ai = (kModel == MH_UBCM) ? x[i] : x[i] * y[i];
    if (kModel == MH_UECM) yi = y[i];
  }
  double k_tot = 0.0, s_tot = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += kPairThreads) {
    const int64_t jl = j0 + threadIdx.x;
    if (jl < n) {
      sa[threadIdx.x] = (kModel == MH_UBCM) ? x[jl] : x[jl] * y[jl];
      if (kModel == MH_UECM) sy[threadIdx.x] = y[jl];
    }
    __syncthreads();
    const int m = (n - j0) < kPairThreads ? static_cast<int>(n - j0) : kPairThreads;
    double k_part = 0.0, s_part = 0.0;
    for (int t = 0; t < m; ++t) {
      if (j0 + t == i) continue;
      if (kModel == MH_UBCM) {
        const double z = ai * sa[t];
        k_part += z / (1.0 + z);
      } else {
        const double A = ai * sa[t];
        const double omr = 1.0 - yi * sy[t];
        const double p = A / (omr + A);
        k_part += p;
        s_part += p / omr;
      }
    }
    k_tot += k_part;
    s_tot += s_part;
    __syncthreads();
  }
  if (row) {
    k_out[i] = k_tot;
    if (kModel == MH_UECM) s_out[i] = s_tot;
  }
}

template <int kModel>
__global__ void __launch_bounds__(kPairThreads) expected_bwd_kernel(const double* __restrict__ x,
                                                                     const double* __restrict__ y, int64_t n,
                                                                     const double* __restrict__ gk,
                                                                     const double* __restrict__ gs,
                                                                     double* __restrict__ gx,
                                                                     double* __restrict__ gy) {
  __shared__ double sx[kPairThreads];
  __shared__ double sy[kPairThreads];
  __shared__ double sgk[kPairThreads];
  __shared__ double sgs[kPairThreads];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kPairThreads + threadIdx.x;
  const bool row = i < n;
  double xi = 0.0, yi = 0.0, gki = 0.0, gsi = 0.0;
  if (row) {
    xi = x[i];
    gki = gk[i];
    if (kModel == MH_UECM) {
      yi = y[i];
      gsi = gs[i];
    }
  }
  const double ai = xi * yi;
  double gx_tot = 0.0, gy_tot = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += kPairThreads) {
    const int64_t jl = j0 + threadIdx.x;
    if (jl < n) {
      sx[threadIdx.x] = x[jl];
      sgk[threadIdx.x] = gk[jl];
      if (kModel == MH_UECM) {
        sy[threadIdx.x] = y[jl];
        sgs[threadIdx.x] = gs[jl];
      }
    }
    __syncthreads();
    const int m = (n - j0) < kPairThreads ? static_cast<int>(n - j0) : kPairThreads;
    double gx_part = 0.0, gy_part = 0.0;
    for (int t = 0; t < m; ++t) {
      if (j0 + t == i) continue;
      const double gkk = gki + sgk[t];
      if (kModel == MH_UBCM) {
        const double xj = sx[t];
        const double opz = 1.0 + xi * xj;
        gx_part += gkk * (xj / (opz * opz));
      } else {
        const double yj = sy[t];
        const double aj = sx[t] * yj;
        const double A = ai * aj;
        const double r = yi * yj;
        const double omr = 1.0 - r;
        const double D = omr + A;
        const double D2 = D * D;
        const double p = A / D;
        const double gss = gsi + sgs[t];
        gx_part += gkk * (yi * aj * omr / D2) + gss * (yi * aj / D2);
        gy_part += gkk * (xi * aj / D2) + gss * (xi * aj / (D2 * omr) + p * yj / (omr * omr));
      }
    }
    gx_tot += gx_part;
    gy_tot += gy_part;
    __syncthreads();
  }
  if (row) {
    gx[i] = gx_tot;
    if (kModel == MH_UECM) gy[i] = gy_tot;
  }
}

}  // namespace

cudaError_t launch_expected_fwd(int model, const double* x, const double* y, int64_t n, double* k, double* s,
                                cudaStream_t st) {
  const unsigned blocks = grid_for(n, kPairThreads);
  if (model == MH_UBCM)
    expected_fwd_kernel<MH_UBCM><<<blocks, kPairThreads, 0, st>>>(x, y, n, k, s);
  else
    expected_fwd_kernel<MH_UECM><<<blocks, kPairThreads, 0, st>>>(x, y, n, k, s);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_expected_bwd(int model, const double* x, const double* y, int64_t n, const double* gk,
                                const double* gs, double* gx, double* gy, cudaStream_t st) {
  const unsigned blocks = grid_for(n, kPairThreads);
  if (model == MH_UBCM)
    expected_bwd_kernel<MH_UBCM><<<blocks, kPairThreads, 0, st>>>(x, y, n, gk, gs, gx, gy);
  else
    expected_bwd_kernel<MH_UECM><<<blocks, kPairThreads, 0, st>>>(x, y, n, gk, gs, gx, gy);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh

// Expected degrees and strengths and their gradients: the O(N^2) sums that
// parameter inference has to evaluate (Sec. 2.2, Sec. 2.5, Sec. 4).
//
//   <k_i> = sum_{j != i} p_ij,   <s_i> = sum_{j != i} m_ij,   m_ij = p_ij / (1 - r_ij)
//
// with E[w | w > 0] = 1 / (1 - r) from Eq. 4.  Each thread owns one row i and
// walks all j in tiles staged through shared memory, recomputing every pair
// term (nothing of size N^2 is stored).
//
// Arithmetic.  FP64 runs at 1/64 of the FP32 rate on this GPU, so each pair
// term is evaluated in double-float arithmetic (pairs of FP32 values, about
// 48 significant bits; walk_math.cuh), summed in double-float over a tile of
// kPairThreads columns, and the tile sums are accumulated in FP64.  A term is
// within a few 2^-45 of its exact value, a tile sum within 2^-38 of its
// terms' total, and the FP64 accumulation over N / 256 tiles adds less than
// N 2^-61, so the row sums are within about 1e-11 relative of exact sums.
//
// Derivatives (A = a_i a_j, a = x y, r = y_i y_j, D = 1 - r + A, z = x_i x_j):
//   UBCM  dp/dx_i = x_j / (1 + z)^2
//   UECM  dp/dx_i = y_i a_j (1 - r) / D^2       dm/dx_i = y_i a_j / D^2
//         dp/dy_i = x_i a_j / D^2               dm/dy_i = x_i a_j / (D^2 (1 - r)) + p y_j / (1 - r)^2
// which equal p(1-p)/x_i, p/(y_i D), ... without dividing by x_i or y_i.
#include "mh_internal.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

constexpr int kPairThreads = 256;

__device__ __forceinline__ double df_to_double(df2 v) {
  return static_cast<double>(v.hi) + static_cast<double>(v.lo);
}

// Operands the double-float path represents without overflow or loss of
// its low part; pairs with any other operand use the FP64 terms below.
__device__ __forceinline__ bool df_safe(double v) { return v == 0.0 || (v >= 0x1p-60 && v <= 0x1p60); }
__device__ __forceinline__ bool df_safe_grad(double g) { return fabs(g) < 0x1p100; }

// FP64 terms of one pair (the same expressions, for out-of-range operands).
__device__ __noinline__ void pair_fwd_fp64(int model, double xi, double yi, double xj, double yj, double& p,
                                           double& m) {
  if (model == MH_UBCM) {
    const double z = xi * xj;
    p = z / (1.0 + z);
    m = 0.0;
    return;
  }
  const double A = (xi * yi) * (xj * yj);
  const double omr = 1.0 - yi * yj;
  p = A / (omr + A);
  m = p / omr;
}

__device__ __noinline__ void pair_bwd_fp64(int model, double xi, double yi, double xj, double yj, double gkk,
                                           double gss, double& dx, double& dy) {
  if (model == MH_UBCM) {
    const double opz = 1.0 + xi * xj;
    dx = gkk * (xj / (opz * opz));
    dy = 0.0;
    return;
  }
  const double aj = xj * yj;
  const double A = (xi * yi) * aj;
  const double omr = 1.0 - yi * yj;
  const double D = omr + A;
  const double D2 = D * D;
  const double p = A / D;
  dx = gkk * (yi * aj * omr / D2) + gss * (yi * aj / D2);
  dy = gkk * (xi * aj / D2) + gss * (xi * aj / (D2 * omr) + p * yj / (omr * omr));
}

// 1 - y_i y_j in double-float (exact product of the high parts by FMA).
__device__ __forceinline__ df2 one_minus_prod(df2 yi, df2 yj) {
  const df2 r = df_mul(yi, yj);
  return df_add(df2{1.0f, 0.0f}, df2{-r.hi, -r.lo});
}

template <int kModel>
__global__ void __launch_bounds__(kPairThreads) expected_fwd_kernel(const double* __restrict__ x,
                                                                     const double* __restrict__ y, int64_t n,
                                                                     double* __restrict__ k_out,
                                                                     double* __restrict__ s_out) {
  __shared__ float2 sa[kPairThreads];  // x_j (UBCM) or a_j (UECM), double-float
  __shared__ float2 sy[kPairThreads];
  __shared__ bool sok[kPairThreads];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kPairThreads + threadIdx.x;
  const bool row = i < n;
  df2 ai{0.0f, 0.0f}, yi{0.0f, 0.0f};
  double xi64 = 0.0, yi64 = 0.0;
  bool iok = true;
  if (row) {
    xi64 = x[i];
    if (kModel == MH_UECM) yi64 = y[i];
    const double av = (kModel == MH_UBCM) ? xi64 : xi64 * yi64;
    ai = df_from_double(av);
    iok = df_safe(av);
    if (kModel == MH_UECM) yi = df_from_double(yi64);
  }
  double k_tot = 0.0, s_tot = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += kPairThreads) {
    const int64_t jl = j0 + threadIdx.x;
    if (jl < n) {
      const double av = (kModel == MH_UBCM) ? x[jl] : x[jl] * y[jl];
      const df2 v = df_from_double(av);
      sa[threadIdx.x] = make_float2(v.hi, v.lo);
      sok[threadIdx.x] = df_safe(av);
      if (kModel == MH_UECM) {
        const df2 w = df_from_double(y[jl]);
        sy[threadIdx.x] = make_float2(w.hi, w.lo);
      }
    }
    __syncthreads();
    const int m = (n - j0) < kPairThreads ? static_cast<int>(n - j0) : kPairThreads;
    df2 k_part{0.0f, 0.0f}, s_part{0.0f, 0.0f};
    for (int t = 0; t < m; ++t) {
      if (j0 + t == i) continue;
      if (!(iok && sok[t])) {
        double p, mm;
        pair_fwd_fp64(kModel, xi64, yi64, x[j0 + t], kModel == MH_UECM ? y[j0 + t] : 0.0, p, mm);
        k_part = df_add(k_part, df_from_double(p));
        if (kModel == MH_UECM) s_part = df_add(s_part, df_from_double(mm));
        continue;
      }
      const df2 prod = df_mul(ai, to_df(sa[t]));
      if (kModel == MH_UBCM) {
        k_part = df_add(k_part, df_div(prod, df_add_f(prod, 1.0f)));
      } else {
        const df2 omr = one_minus_prod(yi, to_df(sy[t]));
        const df2 p = df_div(prod, df_add(omr, prod));
        k_part = df_add(k_part, p);
        s_part = df_add(s_part, df_div(p, omr));
      }
    }
    k_tot += df_to_double(k_part);
    if (kModel == MH_UECM) s_tot += df_to_double(s_part);
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
  __shared__ float2 sx[kPairThreads];
  __shared__ float2 sy[kPairThreads];
  __shared__ float2 sgk[kPairThreads];
  __shared__ float2 sgs[kPairThreads];
  __shared__ bool sok[kPairThreads];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kPairThreads + threadIdx.x;
  const bool row = i < n;
  df2 xi{0.0f, 0.0f}, yi{0.0f, 0.0f}, gki{0.0f, 0.0f}, gsi{0.0f, 0.0f};
  double xi64 = 0.0, yi64 = 0.0, gki64 = 0.0, gsi64 = 0.0;
  bool iok = true;
  if (row) {
    xi64 = x[i];
    gki64 = gk[i];
    xi = df_from_double(xi64);
    gki = df_from_double(gki64);
    iok = df_safe(xi64) && df_safe_grad(gki64);
    if (kModel == MH_UECM) {
      yi64 = y[i];
      gsi64 = gs[i];
      yi = df_from_double(yi64);
      gsi = df_from_double(gsi64);
      iok = iok && df_safe(xi64 * yi64) && df_safe_grad(gsi64);
    }
  }
  const df2 ai = df_mul(xi, yi);
  double gx_tot = 0.0, gy_tot = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += kPairThreads) {
    const int64_t jl = j0 + threadIdx.x;
    if (jl < n) {
      df2 v = df_from_double(x[jl]);
      sx[threadIdx.x] = make_float2(v.hi, v.lo);
      sok[threadIdx.x] = df_safe(x[jl]) && df_safe_grad(gk[jl]) &&
                         (kModel == MH_UBCM || (df_safe(x[jl] * y[jl]) && df_safe_grad(gs[jl])));
      v = df_from_double(gk[jl]);
      sgk[threadIdx.x] = make_float2(v.hi, v.lo);
      if (kModel == MH_UECM) {
        v = df_from_double(y[jl]);
        sy[threadIdx.x] = make_float2(v.hi, v.lo);
        v = df_from_double(gs[jl]);
        sgs[threadIdx.x] = make_float2(v.hi, v.lo);
      }
    }
    __syncthreads();
    const int m = (n - j0) < kPairThreads ? static_cast<int>(n - j0) : kPairThreads;
    df2 gx_part{0.0f, 0.0f}, gy_part{0.0f, 0.0f};
    for (int t = 0; t < m; ++t) {
      if (j0 + t == i) continue;
      if (!(iok && sok[t])) {
        double dx, dy;
        const double yj64 = kModel == MH_UECM ? y[j0 + t] : 0.0;
        const double gss64 = kModel == MH_UECM ? gsi64 + gs[j0 + t] : 0.0;
        pair_bwd_fp64(kModel, xi64, yi64, x[j0 + t], yj64, gki64 + gk[j0 + t], gss64, dx, dy);
        gx_part = df_add(gx_part, df_from_double(dx));
        if (kModel == MH_UECM) gy_part = df_add(gy_part, df_from_double(dy));
        continue;
      }
      const df2 gkk = df_add(gki, to_df(sgk[t]));
      const df2 xj = to_df(sx[t]);
      if (kModel == MH_UBCM) {
        const df2 opz = df_add_f(df_mul(xi, xj), 1.0f);
        gx_part = df_add(gx_part, df_mul(gkk, df_div(xj, df_mul(opz, opz))));
      } else {
        const df2 yj = to_df(sy[t]);
        const df2 aj = df_mul(xj, yj);
        const df2 A = df_mul(ai, aj);
        const df2 omr = one_minus_prod(yi, yj);
        const df2 D = df_add(omr, A);
        const df2 D2 = df_mul(D, D);
        const df2 p = df_div(A, D);
        const df2 gss = df_add(gsi, to_df(sgs[t]));
        const df2 yaj = df_div(df_mul(yi, aj), D2);  // y_i a_j / D^2 = dm/dx_i
        const df2 xaj = df_div(df_mul(xi, aj), D2);  // x_i a_j / D^2 = dp/dy_i
        // dp/dx_i = (1 - r) dm/dx_i;  dm/dy_i = dp/dy_i / (1 - r) + p y_j / (1 - r)^2
        gx_part = df_add(gx_part, df_mul(df_add(df_mul(gkk, omr), gss), yaj));
        const df2 dmdy = df_add(df_div(xaj, omr), df_div(df_mul(p, yj), df_mul(omr, omr)));
        gy_part = df_add(gy_part, df_add(df_mul(gkk, xaj), df_mul(gss, dmdy)));
      }
    }
    gx_tot += df_to_double(gx_part);
    if (kModel == MH_UECM) gy_tot += df_to_double(gy_part);
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

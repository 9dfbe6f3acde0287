// Expected degrees and strengths and their gradients: the O(N^2) sums that
// parameter inference has to evaluate (Sec. 2.2, Sec. 2.5, Sec. 4).
//
//   <k_i> = sum_{j != i} p_ij,   <s_i> = sum_{j != i} m_ij,   m_ij = p_ij / (1 - r_ij)
//
// with E[w | w > 0] = 1 / (1 - r) from Eq. 4.  Every pair term is recomputed
// (nothing of size N^2 is stored).
//
// Work decomposition.  A persistent grid (SM count x resident blocks) walks
// groups of 64 rows of the requested range [row_begin, row_begin + rows); in
// a block of 16 warps every lane owns two rows of the group and warp w sums
// them over the w-th sixteenth of the columns, staged 32 at a time in the
// warp's own shared memory.  The 16 partial sums of a row are added in warp
// order by one thread, so a row's result depends neither on the grid, the
// timing nor the rows it shares a group with: a row range (one rank's share
// of a sharded call) gives bit for bit the values of the whole call.  Groups
// of 64 rows keep the tail of the grid at about 1/40 of the work for
// N = 2*10^5 (one row per thread in blocks of 256 left a second wave 29%
// full).
//
// Arithmetic.  FP64 runs at 1/64 of the FP32 rate on this GPU, so each pair
// term is evaluated in double-float arithmetic (pairs of FP32 values, about
// 48 significant bits; walk_math.cuh).  Terms are summed with an error-free
// two_sum of the high parts and a plain FP32 sum of the low parts and errors,
// renormalised every 8 terms and added to an FP64 total every 32: a term is
// within a few 2^-45 of its exact value, a 32-term partial within 2^-38 of
// the sum of its absolute terms, so the row sums are within about 1e-11 of
// the sum of |terms|.  Operands outside the double-float range (df_safe_*)
// take FP64 terms added straight to the FP64 totals.  A batch of 32 columns
// that is full, within range and away from the group's own rows takes a loop
// without per-pair checks.
//
// Derivatives (a = x y, A = a_i a_j, r = y_i y_j, D = 1 - r + A, Q = a_j / D^2,
// z = x_i x_j), each written without dividing by x_i or y_i:
//   UBCM  dp/dx_i = x_j / (1 + z)^2
//   UECM  dp/dx_i = y_i (1 - r) Q        dm/dx_i = y_i Q
//         dp/dy_i = x_i Q                dm/dy_i = x_i Q (1 - r + r D) / (1 - r)^2
// so that, with gk = g_k,i + g_k,j and gs = g_s,i + g_s,j,
//   dL/dx_i = y_i sum_j Q (gk (1 - r) + gs)
//   dL/dy_i = x_i sum_j Q (gk + gs (1 - r + r D) / (1 - r)^2)
// and the row factors y_i, x_i multiply the finished sums.
#include <algorithm>

#include "mh_internal.cuh"
#include "pair_math.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

constexpr int kPairWarps = 16;
constexpr int kPairThreads = 32 * kPairWarps;
constexpr int kLaneRows = 2;
constexpr int kGroupRows = 32 * kLaneRows;
constexpr int kBatch = 32;
constexpr int kNormEvery = 8;
constexpr unsigned kFull = 0xffffffffu;

// Batches [begin, end) of kBatch columns that warp w of a block covers.
struct BatchRange {
  int64_t begin, end;
};
__device__ __forceinline__ BatchRange warp_batches(int64_t n, int w) {
  const int64_t nb = (n + kBatch - 1) / kBatch;
  const int64_t per = (nb + kPairWarps - 1) / kPairWarps;
  const int64_t b0 = per * w < nb ? per * w : nb;
  return {b0, b0 + per < nb ? b0 + per : nb};
}

// ---- expected sums and the diagonal of their Jacobian ---------------------------------

// What a row-sum kernel adds up over j: the expected sums (p, and m for the
// UECM) or the diagonal of their Jacobian: UBCM x_j / (1 + z)^2 = dp/dx_i;
// UECM (1 - r) Q, Q and Q (1 - r + r D) / (1 - r)^2, which the row factors
// y_i and x_i turn into d<k_i>/dx_i, d<k_i>/dy_i (x_i Q), d<s_i>/dx_i (y_i Q)
// and d<s_i>/dy_i.
enum RowSumKind { kExpectedSums = 0, kJacobianDiag = 1 };

template <int kModel, int kKind>
struct RowSums {
  static constexpr int kCount = kModel == MH_UBCM ? 1 : (kKind == kExpectedSums ? 2 : 3);
};

// FP64 terms of one pair (the same expressions, for out-of-range operands).
template <int kModel, int kKind>
__device__ __noinline__ void row_terms_fp64(double xi, double yi, double xj, double yj, double* t) {
  if constexpr (kModel == MH_UBCM) {
    const double z = xi * xj;
    if constexpr (kKind == kExpectedSums) {
      t[0] = z / (1.0 + z);
    } else {
      const double opz = 1.0 + z;
      t[0] = xj / (opz * opz);
    }
  } else {
    const double aj = xj * yj;
    const double r = yi * yj;
    const double omr = 1.0 - r;
    const double A = (xi * yi) * aj;
    if constexpr (kKind == kExpectedSums) {
      t[0] = A / (omr + A);
      t[1] = t[0] / omr;
    } else {
      const double D = omr + A;
      const double Q = aj / (D * D);
      t[0] = omr * Q;
      t[1] = Q;
      t[2] = Q * ((omr + r * D) / (omr * omr));
    }
  }
}

// Double-float terms; c = (a_j, y_j) as staged (x_j for the UBCM).
template <int kModel, int kKind>
__device__ __forceinline__ void row_terms(df2 ai, df2 yi, float4 c, df2* t) {
  const df2 aj{c.x, c.y};
  const df2 prod = dfu_mul(ai, aj);
  if constexpr (kModel == MH_UBCM) {
    const df2 opz = df_add_f(prod, 1.0f);
    if constexpr (kKind == kExpectedSums) {
      t[0] = dfu_div(prod, opz);
    } else {
      t[0] = dfu_div(aj, dfu_mul(opz, opz));
    }
  } else {
    const df2 r = dfu_mul(yi, df2{c.z, c.w});
    const df2 omr = one_minus(r);
    const df2 D = df_add_sloppy(omr, prod);  // both >= 0
    if constexpr (kKind == kExpectedSums) {
      t[0] = dfu_div(prod, D);
      t[1] = dfu_div(t[0], omr);
    } else {
      const df2 Q = dfu_div(aj, dfu_mul(D, D));
      t[0] = dfu_mul(omr, Q);
      t[1] = Q;
      t[2] = dfu_mul(Q, dfu_div(df_add_sloppy(omr, dfu_mul(r, D)), dfu_mul(omr, omr)));  // (1 - r + r D) / (1 - r)^2
    }
  }
}

// out0..out3: <k>, <s> (expected sums); d<k>/dx, d<k>/dy, d<s>/dx, d<s>/dy
// (Jacobian diagonal; only d<k>/dx for the UBCM).  Entry r is row row_begin + r.
template <int kModel, int kKind>
__global__ void __launch_bounds__(kPairThreads, 1) row_sums_kernel(const double* __restrict__ x,
                                                                    const double* __restrict__ y, int64_t n,
                                                                    int64_t row_begin, int64_t rows,
                                                                    double* __restrict__ out0,
                                                                    double* __restrict__ out1,
                                                                    double* __restrict__ out2,
                                                                    double* __restrict__ out3) {
  constexpr bool kW = kModel == MH_UECM;
  constexpr int kQ = RowSums<kModel, kKind>::kCount;
  __shared__ float4 stage[kPairWarps][kBatch];
  __shared__ double part[kQ][kPairWarps][kGroupRows];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const BatchRange br = warp_batches(n, warp);
  const int64_t row_end = row_begin + rows;  // <= n
  const int64_t groups = (rows + kGroupRows - 1) / kGroupRows;
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t row0 = row_begin + g * kGroupRows;
    df2 ai[kLaneRows], yi[kLaneRows];
    bool rok[kLaneRows];
#pragma unroll
    for (int q = 0; q < kLaneRows; ++q) {
      const int64_t i = row0 + 32 * q + lane;
      ai[q] = df2{0.0f, 0.0f};
      yi[q] = df2{0.0f, 0.0f};
      rok[q] = true;  // rows past the range compute zero terms and are not stored
      if (i < row_end) {
        const double av = kW ? x[i] * y[i] : x[i];
        ai[q] = df_from_double(av);
        rok[q] = df_safe_a(av);
        if (kW) {
          yi[q] = df_from_double(y[i]);
          rok[q] = rok[q] && df_safe_y(y[i]);
        }
      }
    }
    bool lane_ok = true;
#pragma unroll
    for (int q = 0; q < kLaneRows; ++q) lane_ok = lane_ok && rok[q];
    const bool rows_ok = __all_sync(kFull, lane_ok);
    double tot[kQ][kLaneRows] = {};
    for (int64_t b = br.begin; b < br.end; ++b) {
      const int64_t c0 = b * kBatch;
      const int64_t jl = c0 + lane;
      bool ok = true;
      if (jl < n) {
        const double av = kW ? x[jl] * y[jl] : x[jl];
        const df2 a = df_from_double(av);
        float4 v = make_float4(a.hi, a.lo, 0.0f, 0.0f);
        ok = df_safe_a(av);
        if (kW) {
          const df2 w = df_from_double(y[jl]);
          v.z = w.hi;
          v.w = w.lo;
          ok = ok && df_safe_y(y[jl]);
        }
        stage[warp][lane] = v;
      }
      const unsigned okmask = __ballot_sync(kFull, ok);
      __syncwarp();
      const int m = n - c0 < kBatch ? static_cast<int>(n - c0) : kBatch;
      const bool own_rows = c0 < row0 + kGroupRows && c0 + kBatch > row0;  // the batch meets the group's rows
      DfAcc acc[kQ][kLaneRows];
      if (rows_ok && okmask == kFull && m == kBatch && !own_rows) {
#pragma unroll 1
        for (int t0 = 0; t0 < kBatch; t0 += kNormEvery) {
#pragma unroll 2
          for (int u = 0; u < kNormEvery; ++u) {
            const float4 c = stage[warp][t0 + u];
#pragma unroll
            for (int q = 0; q < kLaneRows; ++q) {
              df2 t[kQ];
              row_terms<kModel, kKind>(ai[q], yi[q], c, t);
#pragma unroll
              for (int e = 0; e < kQ; ++e) acc[e][q].add(t[e]);
            }
          }
#pragma unroll
          for (int e = 0; e < kQ; ++e)
#pragma unroll
            for (int q = 0; q < kLaneRows; ++q) acc[e][q].norm();
        }
      } else {
        for (int t = 0; t < m; ++t) {
          const int64_t j = c0 + t;
          const float4 c = stage[warp][t];
          const bool jok = (okmask >> t) & 1u;
#pragma unroll
          for (int q = 0; q < kLaneRows; ++q) {
            const int64_t i = row0 + 32 * q + lane;
            if (i >= row_end || i == j) continue;
            if (rok[q] && jok) {
              df2 tt[kQ];
              row_terms<kModel, kKind>(ai[q], yi[q], c, tt);
#pragma unroll
              for (int e = 0; e < kQ; ++e) acc[e][q].add(tt[e]);
            } else {
              double tf[kQ];
              row_terms_fp64<kModel, kKind>(x[i], kW ? y[i] : 0.0, x[j], kW ? y[j] : 0.0, tf);
#pragma unroll
              for (int e = 0; e < kQ; ++e) tot[e][q] += tf[e];
            }
          }
          if ((t % kNormEvery) == kNormEvery - 1) {
#pragma unroll
            for (int e = 0; e < kQ; ++e)
#pragma unroll
              for (int q = 0; q < kLaneRows; ++q) acc[e][q].norm();
          }
        }
      }
#pragma unroll
      for (int e = 0; e < kQ; ++e)
#pragma unroll
        for (int q = 0; q < kLaneRows; ++q) tot[e][q] += acc[e][q].value();
      __syncwarp();  // the next batch overwrites stage[warp]
    }
#pragma unroll
    for (int e = 0; e < kQ; ++e)
#pragma unroll
      for (int q = 0; q < kLaneRows; ++q) part[e][warp][32 * q + lane] = tot[e][q];
    __syncthreads();
    if (threadIdx.x < kGroupRows) {
      const int r = threadIdx.x;
      double S[kQ];
#pragma unroll
      for (int e = 0; e < kQ; ++e) S[e] = 0.0;
      for (int w = 0; w < kPairWarps; ++w)
#pragma unroll
        for (int e = 0; e < kQ; ++e) S[e] += part[e][w][r];
      const int64_t i = row0 + r;
      if (i < row_end) {
        const int64_t o = i - row_begin;
        if constexpr (kKind == kExpectedSums) {
          out0[o] = S[0];
          if constexpr (kW) out1[o] = S[1];
        } else if constexpr (!kW) {
          out0[o] = S[0];
        } else {
          const double xi = x[i], yv = y[i];
          out0[o] = yv * S[0];
          out1[o] = xi * S[1];
          out2[o] = yv * S[1];
          out3[o] = xi * S[2];
        }
      }
    }
    __syncthreads();  // part[] is rewritten by the next group
  }
}

// ---- backward ----------------------------------------------------------------------

// FP64 terms of one pair without the row factor (y_i for x, x_i for y).
__device__ __noinline__ void pair_bwd_fp64(int model, double xi, double yi, double xj, double yj, double gk,
                                           double gs, double& tx, double& ty) {
  if (model == MH_UBCM) {
    const double opz = 1.0 + xi * xj;
    tx = gk * (xj / (opz * opz));
    ty = 0.0;
    return;
  }
  const double aj = xj * yj;
  const double r = yi * yj;
  const double omr = 1.0 - r;
  const double D = omr + (xi * yi) * aj;
  const double Q = aj / (D * D);
  tx = Q * (gk * omr + gs);
  ty = Q * (gk + gs * ((omr + r * D) / (omr * omr)));
}

// Double-float row state: UBCM v = x_i, UECM v = a_i (and y_i); gradients g_k,i, g_s,i.
struct BwdRow {
  df2 v, y, gk, gs;
};

// Double-float terms.  Staged columns: UBCM c0 = (x_j, g_k,j); UECM c0 = (a_j, y_j),
// c1 = (g_k,j, g_s,j).  Mixed-sign sums use the sloppy addition: its error is a
// few 2^-48 of the sum of the operands' magnitudes.
template <int kModel>
__device__ __forceinline__ void bwd_term(const BwdRow& R, float4 c0, float4 c1, df2& tx, df2& ty) {
  if (kModel == MH_UBCM) {
    const df2 xj{c0.x, c0.y};
    const df2 opz = df_add_f(dfu_mul(R.v, xj), 1.0f);
    const df2 gk = df_add_sloppy(R.gk, df2{c0.z, c0.w});
    tx = dfu_mul(gk, dfu_div(xj, dfu_mul(opz, opz)));
    return;
  }
  const df2 aj{c0.x, c0.y};
  const df2 r = dfu_mul(R.y, df2{c0.z, c0.w});
  const df2 omr = one_minus(r);
  const df2 D = df_add_sloppy(omr, dfu_mul(R.v, aj));  // both >= 0
  const df2 Q = dfu_div(aj, dfu_mul(D, D));
  const df2 gk = df_add_sloppy(R.gk, df2{c1.x, c1.y});
  const df2 gs = df_add_sloppy(R.gs, df2{c1.z, c1.w});
  tx = dfu_mul(df_add_sloppy(dfu_mul(gk, omr), gs), Q);
  const df2 fr = dfu_div(df_add_sloppy(omr, dfu_mul(r, D)), dfu_mul(omr, omr));  // (1 - r + r D) / (1 - r)^2
  ty = dfu_mul(df_add_sloppy(gk, dfu_mul(gs, fr)), Q);
}

template <int kModel>
__global__ void __launch_bounds__(kPairThreads, 1) expected_bwd_kernel(const double* __restrict__ x,
                                                                        const double* __restrict__ y, int64_t n,
                                                                        int64_t row_begin, int64_t rows,
                                                                        const double* __restrict__ gk,
                                                                        const double* __restrict__ gs,
                                                                        double* __restrict__ gx,
                                                                        double* __restrict__ gy) {
  constexpr bool kW = kModel == MH_UECM;
  __shared__ float4 stage0[kPairWarps][kBatch];
  __shared__ float4 stage1[kW ? kPairWarps : 1][kBatch];
  __shared__ double part[2][kPairWarps][kGroupRows];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const BatchRange br = warp_batches(n, warp);
  const int64_t row_end = row_begin + rows;  // <= n
  const int64_t groups = (rows + kGroupRows - 1) / kGroupRows;
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t row0 = row_begin + g * kGroupRows;
    BwdRow R[kLaneRows];
    bool rok[kLaneRows];
#pragma unroll
    for (int q = 0; q < kLaneRows; ++q) {
      const int64_t i = row0 + 32 * q + lane;
      const df2 zero{0.0f, 0.0f};
      R[q] = BwdRow{zero, zero, zero, zero};
      rok[q] = true;  // rows past the range compute zero terms and are not stored
      if (i < row_end) {
        const double v = kW ? x[i] * y[i] : x[i];
        R[q].v = df_from_double(v);
        R[q].gk = df_from_double(gk[i]);
        rok[q] = df_safe_a(v) && df_safe_g(gk[i]);
        if (kW) {
          R[q].y = df_from_double(y[i]);
          R[q].gs = df_from_double(gs[i]);
          rok[q] = rok[q] && df_safe_y(y[i]) && df_safe_g(gs[i]);
        }
      }
    }
    bool lane_ok = true;
#pragma unroll
    for (int q = 0; q < kLaneRows; ++q) lane_ok = lane_ok && rok[q];
    const bool rows_ok = __all_sync(kFull, lane_ok);
    double x_tot[kLaneRows] = {}, y_tot[kLaneRows] = {};
    for (int64_t b = br.begin; b < br.end; ++b) {
      const int64_t c0 = b * kBatch;
      const int64_t jl = c0 + lane;
      bool ok = true;
      if (jl < n) {
        const double v = kW ? x[jl] * y[jl] : x[jl];
        const df2 a = df_from_double(v);
        const df2 k = df_from_double(gk[jl]);
        ok = df_safe_a(v) && df_safe_g(gk[jl]);
        if (kW) {
          const df2 w = df_from_double(y[jl]);
          const df2 s = df_from_double(gs[jl]);
          stage0[warp][lane] = make_float4(a.hi, a.lo, w.hi, w.lo);
          stage1[warp][lane] = make_float4(k.hi, k.lo, s.hi, s.lo);
          ok = ok && df_safe_y(y[jl]) && df_safe_g(gs[jl]);
        } else {
          stage0[warp][lane] = make_float4(a.hi, a.lo, k.hi, k.lo);
        }
      }
      const unsigned okmask = __ballot_sync(kFull, ok);
      __syncwarp();
      const int m = n - c0 < kBatch ? static_cast<int>(n - c0) : kBatch;
      const bool own_rows = c0 < row0 + kGroupRows && c0 + kBatch > row0;  // the batch meets the group's rows
      DfAcc ax[kLaneRows], ay[kLaneRows];
      if (rows_ok && okmask == kFull && m == kBatch && !own_rows) {
#pragma unroll 1
        for (int t0 = 0; t0 < kBatch; t0 += kNormEvery) {
#pragma unroll 1
          for (int u = 0; u < kNormEvery; ++u) {
            const float4 s0 = stage0[warp][t0 + u];
            const float4 s1 = kW ? stage1[warp][t0 + u] : s0;
#pragma unroll
            for (int q = 0; q < kLaneRows; ++q) {
              df2 tx, ty;
              bwd_term<kModel>(R[q], s0, s1, tx, ty);
              ax[q].add(tx);
              if (kW) ay[q].add(ty);
            }
          }
#pragma unroll
          for (int q = 0; q < kLaneRows; ++q) {
            ax[q].norm();
            if (kW) ay[q].norm();
          }
        }
      } else {
        for (int t = 0; t < m; ++t) {
          const int64_t j = c0 + t;
          const float4 s0 = stage0[warp][t];
          const float4 s1 = kW ? stage1[warp][t] : s0;
          const bool jok = (okmask >> t) & 1u;
#pragma unroll
          for (int q = 0; q < kLaneRows; ++q) {
            const int64_t i = row0 + 32 * q + lane;
            if (i >= row_end || i == j) continue;
            if (rok[q] && jok) {
              df2 tx, ty;
              bwd_term<kModel>(R[q], s0, s1, tx, ty);
              ax[q].add(tx);
              if (kW) ay[q].add(ty);
            } else {
              double tx, ty;
              pair_bwd_fp64(kModel, x[i], kW ? y[i] : 0.0, x[j], kW ? y[j] : 0.0, gk[i] + gk[j],
                            kW ? gs[i] + gs[j] : 0.0, tx, ty);
              x_tot[q] += tx;
              if (kW) y_tot[q] += ty;
            }
          }
          if ((t % kNormEvery) == kNormEvery - 1) {
#pragma unroll
            for (int q = 0; q < kLaneRows; ++q) {
              ax[q].norm();
              if (kW) ay[q].norm();
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kLaneRows; ++q) {
        x_tot[q] += ax[q].value();
        if (kW) y_tot[q] += ay[q].value();
      }
      __syncwarp();  // the next batch overwrites stage0/stage1[warp]
    }
#pragma unroll
    for (int q = 0; q < kLaneRows; ++q) {
      part[0][warp][32 * q + lane] = x_tot[q];
      if (kW) part[1][warp][32 * q + lane] = y_tot[q];
    }
    __syncthreads();
    if (threadIdx.x < kGroupRows) {
      const int r = threadIdx.x;
      double sx = 0.0, sy = 0.0;
      for (int w = 0; w < kPairWarps; ++w) {
        sx += part[0][w][r];
        if (kW) sy += part[1][w][r];
      }
      const int64_t i = row0 + r;
      if (i < row_end) {
        gx[i - row_begin] = kW ? y[i] * sx : sx;
        if (kW) gy[i - row_begin] = x[i] * sy;
      }
    }
    __syncthreads();  // part[] is rewritten by the next group
  }
}

// Persistent grid: resident blocks per SM (queried once per device and
// kernel) times the SM count, at most one block per row group.
template <typename Kernel>
unsigned pair_grid(Kernel kernel, int* cache, int64_t rows) {
  int dev = 0;
  int per_sm = 1;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    if (cache[dev] == 0) {
      int v = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kPairThreads, 0) != cudaSuccess || v < 1) v = 1;
      cache[dev] = v;
    }
    per_sm = cache[dev];
  }
  const int64_t groups = (rows + kGroupRows - 1) / kGroupRows;
  const int64_t cap = static_cast<int64_t>(sm_count()) * per_sm;
  return static_cast<unsigned>(std::min(groups, cap));
}

int g_occ_fwd[2][64];
int g_occ_bwd[2][64];
int g_occ_diag[2][64];

}  // namespace

cudaError_t launch_expected_fwd(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                int64_t rows, double* k, double* s, cudaStream_t st) {
  if (model == MH_UBCM) {
    auto kernel = row_sums_kernel<MH_UBCM, kExpectedSums>;
    kernel<<<pair_grid(kernel, g_occ_fwd[0], rows), kPairThreads, 0, st>>>(x, y, n, row_begin, rows, k, s, nullptr,
                                                                          nullptr);
  } else {
    auto kernel = row_sums_kernel<MH_UECM, kExpectedSums>;
    kernel<<<pair_grid(kernel, g_occ_fwd[1], rows), kPairThreads, 0, st>>>(x, y, n, row_begin, rows, k, s, nullptr,
                                                                          nullptr);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_expected_jacobian_diag(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                          int64_t rows, double* dk_dx, double* dk_dy, double* ds_dx, double* ds_dy,
                                          cudaStream_t st) {
  if (model == MH_UBCM) {
    auto kernel = row_sums_kernel<MH_UBCM, kJacobianDiag>;
    kernel<<<pair_grid(kernel, g_occ_diag[0], rows), kPairThreads, 0, st>>>(x, y, n, row_begin, rows, dk_dx,
                                                                           nullptr, nullptr, nullptr);
  } else {
    auto kernel = row_sums_kernel<MH_UECM, kJacobianDiag>;
    kernel<<<pair_grid(kernel, g_occ_diag[1], rows), kPairThreads, 0, st>>>(x, y, n, row_begin, rows, dk_dx, dk_dy,
                                                                           ds_dx, ds_dy);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_expected_bwd(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                int64_t rows, const double* gk, const double* gs, double* gx, double* gy,
                                cudaStream_t st) {
  if (model == MH_UBCM) {
    const unsigned blocks = pair_grid(expected_bwd_kernel<MH_UBCM>, g_occ_bwd[0], rows);
    expected_bwd_kernel<MH_UBCM><<<blocks, kPairThreads, 0, st>>>(x, y, n, row_begin, rows, gk, gs, gx, gy);
  } else {
    const unsigned blocks = pair_grid(expected_bwd_kernel<MH_UECM>, g_occ_bwd[1], rows);
    expected_bwd_kernel<MH_UECM><<<blocks, kPairThreads, 0, st>>>(x, y, n, row_begin, rows, gk, gs, gx, gy);
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh

// Expected sums, their Jacobian diagonal and the gradient with every
// unordered pair {i, j} evaluated once (Sec. 2.2, Sec. 2.5, Sec. 4): the same
// sums as the row kernels of pairwise.cu, for half the pair terms.
//
// Symmetry.  p_ij = p_ji and m_ij = m_ji, so the expected sums take one term
// for both rows.  Every derivative term is a factor G_ij symmetric in i and j
// times a_j for row i and a_i for row j (a = x for the UBCM, x y for the
// UECM; z = x_i x_j, A = a_i a_j, r = y_i y_j, D = 1 - r + A):
//   UBCM  dp_ij/dx_i = x_j / (1 + z)^2
//   UECM  Q_ij = a_j / D^2 in d<k_i>/dx_i (1 - r), d<k_i>/dy_i and
//         d<s_i>/dx_i (Q), d<s_i>/dy_i (Q (1 - r + r D) / (1 - r)^2)
//   gradient  UBCM (g_i + g_j) x_j / (1 + z)^2;
//         UECM Q_ij (gk (1 - r) + gs) and Q_ij (gk + gs (1 - r + r D) / (1 - r)^2)
//         with gk = g_k,i + g_k,j and gs = g_s,i + g_s,j
// and the row factors y_i, x_i multiply the finished sums, as in pairwise.cu.
//
// Work decomposition.  The nodes are cut into bands of L (a multiple of 512);
// a unit is a pair of bands I <= J (a persistent grid takes units in turn).
// A block of 16 warps sweeps the unit's columns in sub-bands of 512, warp w
// owning 32 of them; for each tile of 64 rows, lane l of warp w holds rows
// r0 + l and r0 + 32 + l and column c0 + l, and in step t pairs both rows
// with column (l + t) mod 32 of its warp's columns: the row terms go to the
// lane's own row sums, the column terms to the column's owner, lane
// (l + t) mod 32, by shuffles.  A 32-row half on the diagonal of a diagonal
// unit takes steps 1..16 (step 16 on lanes 0..15 only), so each unordered
// pair comes once.
//
// Determinism.  Sums go to a partial array P[q][B][i] = sum over the j of
// band B of row i's terms (kQ quantities, nb bands): a row's 32 terms of a
// tile and a column's terms of a whole sub-band in double-float (DfAcc,
// folded every 8 terms), the 16 warps' row partials added in warp order,
// tiles and sub-bands in loop order; a row's entry for its own
// band (diagonal unit) gets the row and column parts in that fixed order.
// A second kernel adds P over B in order.  The result therefore depends on
// neither the grid nor the timing, but the order of additions differs from
// the row kernels': both are within the error bound of pairwise.cu (about
// 1e-11 of the sum of |terms|), not bit for bit equal.
//
// Operands outside the double-float range (df_safe_* in pair_math.cuh) make
// their whole tile take FP64 terms.
#include "mh_internal.cuh"
#include "pair_math.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

constexpr int kSymWarps = 16;
constexpr int kSymThreads = 32 * kSymWarps;
constexpr int kSubBand = 32 * kSymWarps;  // columns of one sweep
constexpr int kSymRows = 64;              // rows of a tile: two per lane
constexpr unsigned kAll = 0xffffffffu;

// kSymDiagF / kSymBwdF: the Jacobian diagonal and the gradient with FP32 pair
// terms summed in FP32 over a tile (rows: 32 terms, columns: 64), the
// tiles' partials then added as the other kinds add theirs.  Each term is
// within a few units of 2^-24 and a tile's sum within about 2^-19 of its
// terms' magnitudes: the relative accuracy of a Newton direction (the fit's
// conjugate gradients stop at a relative residual of 5e-2), at a fraction
// of the double-float terms' cost.
enum SymKind { kSymFwd = 0, kSymDiag = 1, kSymBwd = 2, kSymDiagF = 3, kSymBwdF = 4 };

__host__ __device__ constexpr int base_kind(int k) { return k == kSymDiagF ? kSymDiag : (k == kSymBwdF ? kSymBwd : k); }
__host__ __device__ constexpr bool f32_kind(int k) { return k == kSymDiagF || k == kSymBwdF; }

template <int kModel, int kKind>
struct SymCount {
  static constexpr int kB = base_kind(kKind);
  static constexpr int kQ = kModel == MH_UBCM ? 1 : (kB == kSymDiag ? 3 : 2);
  static constexpr bool kTwo = kModel == MH_UECM && kB == kSymBwd;  // a second float4 per node
};

// Per-node double-float operands, written once per call:
//   d0  UBCM (x, g_k) / UECM (a, y)    d1  UECM gradient (g_k, g_s)
// (FP32 kinds: d0 UBCM (x, g_k, 0, 0) / UECM (a, y, 1 - y, g_k), d1 (g_s, 0,
// 0, 0)) and a bit per node (word i / 32) set when an operand is outside the
// double-float range.
struct SymNodes {
  const float4* d0;
  const float4* d1;
  const unsigned* unsafe;
};

template <int kModel, int kKind>
__global__ void sym_nodes_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ gk, const double* __restrict__ gs, int64_t n,
                                 float4* __restrict__ d0, float4* __restrict__ d1, unsigned* __restrict__ unsafe) {
  constexpr bool kW = kModel == MH_UECM;
  const int64_t words = (n + 31) / 32;
  for (int64_t w0 = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); w0 < words;
       w0 += static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5)) {
    const int64_t i = w0 * 32 + (threadIdx.x & 31);
    bool bad = false;
    if (f32_kind(kKind) && i < n) {
      constexpr bool kG = base_kind(kKind) == kSymBwd;
      const double a = kW ? x[i] * y[i] : x[i];
      bad = !df_safe_a(a);
      float4 v = make_float4(__double2float_rn(a), 0.0f, 0.0f, 0.0f);
      if constexpr (kW) {
        v.y = __double2float_rn(y[i]);
        v.z = __double2float_rn(1.0 - y[i]);  // 1 - y_i y_j = (1 - y_i) + y_i (1 - y_j) without cancellation
        bad = bad || !df_safe_y(y[i]);
        if constexpr (kG) {
          v.w = __double2float_rn(gk[i]);
          d1[i] = make_float4(__double2float_rn(gs[i]), 0.0f, 0.0f, 0.0f);
          bad = bad || !df_safe_g(gk[i]) || !df_safe_g(gs[i]);
        }
      } else if constexpr (kG) {
        v.y = __double2float_rn(gk[i]);
        bad = bad || !df_safe_g(gk[i]);
      }
      d0[i] = v;
    } else if (i < n) {
      const double a = kW ? x[i] * y[i] : x[i];
      const df2 av = df_from_double(a);
      bad = !df_safe_a(a);
      float4 v = make_float4(av.hi, av.lo, 0.0f, 0.0f);
      if constexpr (kW) {
        const df2 yv = df_from_double(y[i]);
        v.z = yv.hi;
        v.w = yv.lo;
        bad = bad || !df_safe_y(y[i]);
      }
      if constexpr (kKind == kSymBwd) {
        const df2 k = df_from_double(gk[i]);
        bad = bad || !df_safe_g(gk[i]);
        if constexpr (kW) {
          const df2 s = df_from_double(gs[i]);
          bad = bad || !df_safe_g(gs[i]);
          d1[i] = make_float4(k.hi, k.lo, s.hi, s.lo);
        } else {
          v.z = k.hi;
          v.w = k.lo;
        }
      }
      d0[i] = v;
    }
    const unsigned m = __ballot_sync(kAll, bad);
    if ((threadIdx.x & 31) == 0) unsafe[w0] = m;
  }
}

// Double-float terms of one pair: tr for the row (factor a_j), tc for the
// column (factor a_i).  r0/c0: d0 of the row and column node, r1/c1: d1.
template <int kModel, int kKind>
__device__ __forceinline__ void sym_terms(float4 r0, float4 r1, float4 c0, float4 c1, df2* tr, df2* tc) {
  const df2 ai{r0.x, r0.y}, aj{c0.x, c0.y};
  const df2 prod = dfu_mul(ai, aj);
  if constexpr (kModel == MH_UBCM) {
    const df2 opz = df_add_f(prod, 1.0f);
    if constexpr (kKind == kSymFwd) {
      tr[0] = tc[0] = dfu_div(prod, opz);
    } else {
      df2 num{1.0f, 0.0f};
      if constexpr (kKind == kSymBwd) num = df_add_sloppy(df2{r0.z, r0.w}, df2{c0.z, c0.w});
      const df2 F = dfu_div(num, dfu_mul(opz, opz));
      tr[0] = dfu_mul(aj, F);
      tc[0] = dfu_mul(ai, F);
    }
  } else {
    const df2 r = dfu_mul(df2{r0.z, r0.w}, df2{c0.z, c0.w});
    const df2 omr = one_minus(r);
    const df2 D = df_add_sloppy(omr, prod);  // both >= 0
    if constexpr (kKind == kSymFwd) {
      const df2 p = dfu_div(prod, D);
      tr[0] = tc[0] = p;
      tr[1] = tc[1] = dfu_div(p, omr);
    } else {
      const df2 H = dfu_div(df2{1.0f, 0.0f}, dfu_mul(D, D));
      const df2 fr = dfu_div(df_add_sloppy(omr, dfu_mul(r, D)), dfu_mul(omr, omr));  // (1 - r + r D) / (1 - r)^2
      if constexpr (kKind == kSymDiag) {
        const df2 s0 = dfu_mul(omr, H);
        const df2 s2 = dfu_mul(H, fr);
        tr[0] = dfu_mul(aj, s0);
        tr[1] = dfu_mul(aj, H);
        tr[2] = dfu_mul(aj, s2);
        tc[0] = dfu_mul(ai, s0);
        tc[1] = dfu_mul(ai, H);
        tc[2] = dfu_mul(ai, s2);
      } else {
        const df2 gk = df_add_sloppy(df2{r1.x, r1.y}, df2{c1.x, c1.y});
        const df2 gsum = df_add_sloppy(df2{r1.z, r1.w}, df2{c1.z, c1.w});
        const df2 U = dfu_mul(df_add_sloppy(dfu_mul(gk, omr), gsum), H);
        const df2 V = dfu_mul(df_add_sloppy(gk, dfu_mul(gsum, fr)), H);
        tr[0] = dfu_mul(aj, U);
        tr[1] = dfu_mul(aj, V);
        tc[0] = dfu_mul(ai, U);
        tc[1] = dfu_mul(ai, V);
      }
    }
  }
}

// FP32 terms of one pair (kinds kSymDiagF, kSymBwdF), the same expressions as
// sym_terms; with the operands in the double-float range every intermediate
// is a normal FP32 number (D^2 <= 2^120, 1 - r >= 2^-11).
template <int kModel, int kKind>
__device__ __forceinline__ void sym_terms_f32(float4 r0, float4 r1, float4 c0, float4 c1, float* tr, float* tc) {
  const float ai = r0.x, aj = c0.x;
  if constexpr (kModel == MH_UBCM) {
    const float opz = fmaf(ai, aj, 1.0f);
    const float num = kKind == kSymBwdF ? r0.y + c0.y : 1.0f;
    const float F = __fdividef(num, opz * opz);
    tr[0] = aj * F;
    tc[0] = ai * F;
  } else {
    const float r = r0.y * c0.y;
    const float omr = fmaf(r0.y, c0.z, r0.z);  // (1 - y_i) + y_i (1 - y_j)
    const float D = fmaf(ai, aj, omr);
    const float H = __fdividef(1.0f, D * D);
    const float rc = __fdividef(1.0f, omr);
    const float fr = fmaf(r, D, omr) * rc * rc;  // (1 - r + r D) / (1 - r)^2
    if constexpr (kKind == kSymDiagF) {
      const float s0 = omr * H;
      const float s2 = H * fr;
      tr[0] = aj * s0;
      tr[1] = aj * H;
      tr[2] = aj * s2;
      tc[0] = ai * s0;
      tc[1] = ai * H;
      tc[2] = ai * s2;
    } else {
      const float gk = r0.w + c0.w;
      const float gsum = r1.x + c1.x;
      const float U = fmaf(gk, omr, gsum) * H;
      const float V = fmaf(gsum, fr, gk) * H;
      tr[0] = aj * U;
      tr[1] = aj * V;
      tc[0] = ai * U;
      tc[1] = ai * V;
    }
  }
}

// FP64 terms of one pair (tiles with an operand outside the double-float range).
template <int kModel, int kKind>
__device__ __noinline__ void sym_terms_fp64(const double* x, const double* y, const double* gk, const double* gs,
                                            int64_t i, int64_t j, double* tr, double* tc) {
  const double xi = x[i], xj = x[j];
  if constexpr (kModel == MH_UBCM) {
    const double z = xi * xj;
    if constexpr (kKind == kSymFwd) {
      tr[0] = tc[0] = z / (1.0 + z);
    } else {
      const double opz = 1.0 + z;
      const double F = (kKind == kSymBwd ? gk[i] + gk[j] : 1.0) / (opz * opz);
      tr[0] = xj * F;
      tc[0] = xi * F;
    }
  } else {
    const double yi = y[i], yj = y[j];
    const double ai = xi * yi, aj = xj * yj;
    const double r = yi * yj;
    const double omr = 1.0 - r;
    const double A = ai * aj;
    const double D = omr + A;
    if constexpr (kKind == kSymFwd) {
      const double p = A / D;
      tr[0] = tc[0] = p;
      tr[1] = tc[1] = p / omr;
    } else {
      const double H = 1.0 / (D * D);
      const double fr = (omr + r * D) / (omr * omr);
      if constexpr (kKind == kSymDiag) {
        tr[0] = aj * (omr * H);
        tr[1] = aj * H;
        tr[2] = aj * (H * fr);
        tc[0] = ai * (omr * H);
        tc[1] = ai * H;
        tc[2] = ai * (H * fr);
      } else {
        const double gsk = gk[i] + gk[j], gss = gs[i] + gs[j];
        const double U = (gsk * omr + gss) * H;
        const double V = (gsk + gss * fr) * H;
        tr[0] = aj * U;
        tr[1] = aj * V;
        tc[0] = ai * U;
        tc[1] = ai * V;
      }
    }
  }
}

// Unit u of the upper triangle of nb x nb bands, row-major: (I, J), I <= J.
__device__ __forceinline__ void unit_bands(int64_t u, int64_t nb, int64_t& I, int64_t& J) {
  int64_t b = 0, first = 0;
  while (first + (nb - b) <= u) {
    first += nb - b;
    ++b;
  }
  I = b;
  J = b + (u - first);
}

__device__ __forceinline__ float4 node_or_zero(const float4* d, int64_t i, int64_t n) {
  return i < n ? d[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}
// Past the last node: a = 0 with y = 0 (1 - y = 1 for the FP32 kinds'
// third word), so the pair terms are zero and finite.
template <bool kF>
__device__ __forceinline__ float4 node_or_pad(const float4* d, int64_t i, int64_t n) {
  return i < n ? d[i] : make_float4(0.0f, 0.0f, kF ? 1.0f : 0.0f, 0.0f);
}
__device__ __forceinline__ bool node_unsafe(const unsigned* unsafe, int64_t i, int64_t n) {
  return i < n && ((unsafe[i >> 5] >> (i & 31)) & 1u);
}

// P[(q nb + B) n + i]: row i's sum of quantity q over the columns of band B.
// Row tiles are 64 rows: lane l holds rows r0 + l and r0 + 32 + l (two
// independent pair terms per step), each against the same column.
template <int kModel, int kKind>
__global__ void __launch_bounds__(kSymThreads, 1) sym_pairs_kernel(SymNodes N, const double* __restrict__ x,
                                                                   const double* __restrict__ y,
                                                                   const double* __restrict__ gk,
                                                                   const double* __restrict__ gs, int64_t n,
                                                                   int64_t L, int64_t nb, double* __restrict__ P) {
  constexpr int kQ = SymCount<kModel, kKind>::kQ;
  constexpr bool kTwo = SymCount<kModel, kKind>::kTwo;
  constexpr bool kF = f32_kind(kKind);
  __shared__ float4 cst0[kSymWarps][32];
  __shared__ float4 cst1[kTwo ? kSymWarps : 1][32];
  // a tile's row partials: double-float (hi, lo) bits, or FP64 bits where the
  // warp's tile took the FP64 terms (rslow), whose sums may lie below FP32's range
  // two buffers where they fit the static shared memory: one barrier a tile
  constexpr int kBufs = (kQ <= 2 && !kTwo) ? 2 : 1;
  __shared__ unsigned long long rpart[kBufs][kQ][kSymWarps][kSymRows];
  __shared__ int rslow[kBufs][kSymWarps];
  int buf = 0;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t units = nb * (nb + 1) / 2;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    int64_t I, J;
    unit_bands(u, nb, I, J);
    const bool dg = I == J;
    const int64_t rb = I * L, cb = J * L;
    // the row entries this unit adds into: P[q][J][rows of band I]
    for (int64_t t = threadIdx.x; t < L && rb + t < n; t += kSymThreads)
#pragma unroll
      for (int q = 0; q < kQ; ++q) P[(q * nb + J) * n + rb + t] = 0.0;
    __syncthreads();
    for (int64_t s = 0; s < L && cb + s < n; s += kSubBand) {
      const int64_t cw = cb + s + 32 * warp;  // the warp's first column
      const int64_t j = cw + lane;
      cst0[warp][lane] = node_or_pad<kF>(N.d0, j, n);
      if constexpr (kTwo) cst1[warp][lane] = node_or_zero(N.d1, j, n);
      const unsigned cbad = __ballot_sync(kAll, node_unsafe(N.unsafe, j, n));
      __syncwarp();
      // column sums: double-float over the whole sub-band (FP64 tiles add to ctot)
      DfAcc cacc[kQ];
      double ctot[kQ];
#pragma unroll
      for (int q = 0; q < kQ; ++q) ctot[q] = 0.0;
      const int64_t ct = (s >> 5) + warp;  // the warp's column tile (of 32) within the band
      const int64_t tiles = dg ? (s + kSubBand + kSymRows - 1) / kSymRows : L / kSymRows;
      for (int64_t rt = 0; rt < tiles && rb + kSymRows * rt < n; ++rt) {
        const int64_t r0 = rb + kSymRows * rt;
        float4 rd0[2], rd1[2];
        unsigned rbad = 0u;
        int mode[2];  // 0 skip (the transposed tile holds these pairs), 1 same 32 nodes, 2 all pairs
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t i = r0 + 32 * h + lane;
          rd0[h] = node_or_pad<kF>(N.d0, i, n);
          rd1[h] = kTwo ? node_or_zero(N.d1, i, n) : rd0[h];
          rbad |= __ballot_sync(kAll, node_unsafe(N.unsafe, i, n));
          const int64_t rh = 2 * rt + h;  // row sub-tile (of 32) within the band
          mode[h] = !dg || rh < ct ? 2 : (rh == ct ? 1 : 0);
        }
        df2 rsum[2][kQ];  // the tile's row sums, double-float
        double rs[2][kQ];  // or FP64 (slow)
        bool slow = false;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            rsum[h][q] = df2{0.0f, 0.0f};
            rs[h][q] = 0.0;
          }
        const bool any_full = mode[0] == 2 || mode[1] == 2;
        if (mode[0] | mode[1]) {
          const int t0 = any_full ? 0 : 1, t1 = any_full ? 32 : 17;
          if (kF && (rbad | cbad) == 0u && mode[0] == 2 && mode[1] == 2) {
            // FP32 kinds, every pair of the tile: FP32 sums over the tile
            float ra[2][kQ], cf[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) ra[0][q] = ra[1][q] = cf[q] = 0.0f;
#pragma unroll 4
            for (int t = 0; t < 32; ++t) {
              const int c = (lane + t) & 31;
              const float4 c0 = cst0[warp][c];
              const float4 c1 = kTwo ? cst1[warp][c] : c0;
              const int from = (lane - t) & 31;
              float tr0[kQ], tc0[kQ], tr1[kQ], tc1[kQ];
              sym_terms_f32<kModel, kKind>(rd0[0], rd1[0], c0, c1, tr0, tc0);
              sym_terms_f32<kModel, kKind>(rd0[1], rd1[1], c0, c1, tr1, tc1);
#pragma unroll
              for (int q = 0; q < kQ; ++q) {
                ra[0][q] += tr0[q];
                ra[1][q] += tr1[q];
                cf[q] += __shfl_sync(kAll, tc0[q] + tc1[q], from);  // both rows meet the same column
              }
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
              cacc[q].add(df2{cf[q], 0.0f});
              cacc[q].norm();
              rsum[0][q] = df2{ra[0][q], 0.0f};
              rsum[1][q] = df2{ra[1][q], 0.0f};
            }
          } else if (kF && (rbad | cbad) == 0u) {
            float ra[2][kQ], cf[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) ra[0][q] = ra[1][q] = cf[q] = 0.0f;
#pragma unroll 2
            for (int t = t0; t < t1; ++t) {
              const int c = (lane + t) & 31;
              const float4 c0 = cst0[warp][c];
              const float4 c1 = kTwo ? cst1[warp][c] : c0;
              const int from = (lane - t) & 31;
              float cs[kQ];
#pragma unroll
              for (int q = 0; q < kQ; ++q) cs[q] = 0.0f;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float tr[kQ], tc[kQ];
                sym_terms_f32<kModel, kKind>(rd0[h], rd1[h], c0, c1, tr, tc);
                // a diagonal sub-tile takes steps 1..16, step 16 on lanes 0..15 only
                const bool use = mode[h] == 2 || (mode[h] == 1 && t >= 1 && (t < 16 || (t == 16 && lane < 16)));
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                  if (use) {
                    ra[h][q] += tr[q];
                    cs[q] += tc[q];
                  }
                }
              }
#pragma unroll
              for (int q = 0; q < kQ; ++q) cf[q] += __shfl_sync(kAll, cs[q], from);
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
              cacc[q].add(df2{cf[q], 0.0f});
              cacc[q].norm();
              rsum[0][q] = df2{ra[0][q], 0.0f};
              rsum[1][q] = df2{ra[1][q], 0.0f};
            }
          } else if ((rbad | cbad) == 0u && mode[0] == 2 && mode[1] == 2) {
            // every pair of the tile, no per-step checks (all tiles of off-diagonal units)
            DfAcc ra[2][kQ];
#pragma unroll 4
            for (int t = 0; t < 32; ++t) {
              const int c = (lane + t) & 31;
              const float4 c0 = cst0[warp][c];
              const float4 c1 = kTwo ? cst1[warp][c] : c0;
              const int from = (lane - t) & 31;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                df2 tr[kQ], tc[kQ];
                sym_terms<kModel, base_kind(kKind)>(rd0[h], rd1[h], c0, c1, tr, tc);
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                  ra[h][q].add(tr[q]);
                  cacc[q].add(df2{__shfl_sync(kAll, tc[q].hi, from), __shfl_sync(kAll, tc[q].lo, from)});
                }
              }
              if ((t & 3) == 3) {  // ca takes two terms a step, ra[h] one: at most 8 terms between folds
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                  cacc[q].norm();
                  if ((t & 7) == 7) {
                    ra[0][q].norm();
                    ra[1][q].norm();
                  }
                }
              }
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
              cacc[q].norm();
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                ra[h][q].norm();
                rsum[h][q] = df2{ra[h][q].hi, ra[h][q].lo};
              }
            }
          } else if ((rbad | cbad) == 0u) {
            DfAcc ra[2][kQ];
#pragma unroll 2
            for (int t = t0; t < t1; ++t) {
              const int c = (lane + t) & 31;
              const float4 c0 = cst0[warp][c];
              const float4 c1 = kTwo ? cst1[warp][c] : c0;
              const int from = (lane - t) & 31;  // the lane whose rows meet my column in this step
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                df2 tr[kQ], tc[kQ];
                sym_terms<kModel, base_kind(kKind)>(rd0[h], rd1[h], c0, c1, tr, tc);
                // a diagonal sub-tile takes steps 1..16, step 16 on lanes 0..15 only
                const bool use = mode[h] == 2 || (mode[h] == 1 && t >= 1 && (t < 16 || (t == 16 && lane < 16)));
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                  if (use) ra[h][q].add(tr[q]);
                  const float hi = __shfl_sync(kAll, use ? tc[q].hi : 0.0f, from);
                  const float lo = __shfl_sync(kAll, use ? tc[q].lo : 0.0f, from);
                  cacc[q].add(df2{hi, lo});
                }
              }
              if ((t & 3) == 3) {  // ca takes two terms a step, ra[h] one: at most 8 terms between folds
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                  cacc[q].norm();
                  if ((t & 7) == 7) {
                    ra[0][q].norm();
                    ra[1][q].norm();
                  }
                }
              }
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
              cacc[q].norm();
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                ra[h][q].norm();
                rsum[h][q] = df2{ra[h][q].hi, ra[h][q].lo};
              }
            }
          } else {
            slow = true;
            double cs[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) cs[q] = 0.0;
            for (int t = t0; t < t1; ++t) {
              const int c = (lane + t) & 31;
              const int64_t jj = cw + c;
              const int from = (lane - t) & 31;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int64_t i = r0 + 32 * h + lane;
                double tr[kQ], tc[kQ];
#pragma unroll
                for (int q = 0; q < kQ; ++q) tr[q] = tc[q] = 0.0;
                const bool use = mode[h] == 2 || (mode[h] == 1 && t >= 1 && (t < 16 || (t == 16 && lane < 16)));
                if (use && i < n && jj < n) sym_terms_fp64<kModel, base_kind(kKind)>(x, y, gk, gs, i, jj, tr, tc);
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                  rs[h][q] += tr[q];
                  cs[q] += __shfl_sync(kAll, tc[q], from);
                }
              }
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) ctot[q] += cs[q];
          }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            rpart[buf][q][warp][32 * h + lane] =
                slow ? static_cast<unsigned long long>(__double_as_longlong(rs[h][q]))
                     : (static_cast<unsigned long long>(__float_as_uint(rsum[h][q].lo)) << 32) |
                           __float_as_uint(rsum[h][q].hi);
        if (lane == 0) rslow[buf][warp] = slow;
        __syncthreads();
        if (warp < kQ) {  // warp q adds quantity q of the 16 warps, in warp order
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            DfAcc v;
            double sv = 0.0;
#pragma unroll
            for (int w = 0; w < kSymWarps; ++w) {
              const unsigned long long e = rpart[buf][warp][w][32 * h + lane];
              if (rslow[buf][w])
                sv += __longlong_as_double(static_cast<long long>(e));
              else
                v.add(df2{__uint_as_float(static_cast<unsigned>(e)), __uint_as_float(static_cast<unsigned>(e >> 32))});
              if ((w & 7) == 7) v.norm();
            }
            const int64_t i = r0 + 32 * h + lane;
            if (i < n) P[(warp * nb + J) * n + i] += v.value() + sv;
          }
        }
        if (kBufs == 1) __syncthreads();  // rpart is rewritten by the next tile
        buf ^= kBufs - 1;
      }
      __syncthreads();  // the last tile's row entries may be these columns (diagonal unit)
      if (j < n) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          double* e = &P[(q * nb + I) * n + j];
          const double v = ctot[q] + cacc[q].value();
          if (dg)
            *e += v;  // after the row part of its own tile, before later sub-bands
          else
            *e = v;
        }
      }
    }
    __syncthreads();  // the unit's entries are complete before the next unit's zeroing
  }
}

// Sums P over the bands in order and applies the row factors.
template <int kModel, int kKind>
__global__ void sym_reduce_kernel(const double* __restrict__ P, int64_t n, int64_t nb,
                                  const double* __restrict__ x, const double* __restrict__ y,
                                  double* __restrict__ o0, double* __restrict__ o1, double* __restrict__ o2,
                                  double* __restrict__ o3) {
  constexpr int kQ = SymCount<kModel, kKind>::kQ;
  constexpr int kB = base_kind(kKind);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double S[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      double v = 0.0;
      for (int64_t b = 0; b < nb; ++b) v += P[(q * nb + b) * n + i];
      S[q] = v;
    }
    if constexpr (kModel == MH_UBCM) {
      o0[i] = S[0];
    } else if constexpr (kB == kSymFwd) {
      o0[i] = S[0];
      o1[i] = S[1];
    } else if constexpr (kB == kSymDiag) {
      const double xi = x[i], yi = y[i];
      o0[i] = yi * S[0];
      o1[i] = xi * S[1];
      o2[i] = yi * S[1];
      o3[i] = xi * S[2];
    } else {
      o0[i] = y[i] * S[0];
      o1[i] = x[i] * S[1];
    }
  }
}

// Band length: a multiple of kSubBand, at least 2048, with at most 128 bands.
int64_t sym_band(int64_t n) {
  int64_t L = (n + 127) / 128;
  L = (L + kSubBand - 1) / kSubBand * kSubBand;
  return L < 2048 ? 2048 : L;
}

struct SymLayout {
  int64_t L, nb;
  size_t d0, d1, unsafe, P, total;
};

SymLayout sym_layout(int model, int64_t n) {
  SymLayout S;
  S.L = sym_band(n);
  S.nb = (n + S.L - 1) / S.L;
  const int kq = model == MH_UBCM ? 1 : 3;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~static_cast<size_t>(255);
    return at;
  };
  const size_t N = static_cast<size_t>(n);
  S.d0 = take(16 * N);
  S.d1 = take(model == MH_UECM ? 16 * N : 0);
  S.unsafe = take(4 * ((N + 31) / 32));
  S.P = take(8 * static_cast<size_t>(kq) * static_cast<size_t>(S.nb) * N);
  S.total = off;
  return S;
}

int g_occ_sym[2][5][64];

template <int kModel, int kKind>
cudaError_t run_sym(const double* x, const double* y, const double* gk, const double* gs, int64_t n, char* ws,
                    double* o0, double* o1, double* o2, double* o3, cudaStream_t st) {
  const SymLayout S = sym_layout(kModel, n);
  float4* d0 = reinterpret_cast<float4*>(ws + S.d0);
  float4* d1 = kModel == MH_UECM ? reinterpret_cast<float4*>(ws + S.d1) : nullptr;
  unsigned* unsafe = reinterpret_cast<unsigned*>(ws + S.unsafe);
  double* P = reinterpret_cast<double*>(ws + S.P);
  const unsigned sms = static_cast<unsigned>(sm_count());
  sym_nodes_kernel<kModel, kKind><<<grid_for((n + 31) / 32, 8, sms * 4), 256, 0, st>>>(x, y, gk, gs, n, d0, d1,
                                                                                         unsafe);
  int dev = 0;
  int per_sm = 1;
  auto kernel = sym_pairs_kernel<kModel, kKind>;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    int& c = g_occ_sym[kModel == MH_UECM][kKind][dev];
    if (c == 0) {
      int v = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kSymThreads, 0) != cudaSuccess || v < 1) v = 1;
      c = v;
    }
    per_sm = c;
  }
  const int64_t units = S.nb * (S.nb + 1) / 2;
  const int64_t cap = static_cast<int64_t>(sms) * per_sm;
  const unsigned blocks = static_cast<unsigned>(units < cap ? units : cap);
  kernel<<<blocks, kSymThreads, 0, st>>>(SymNodes{d0, d1, unsafe}, x, y, gk, gs, n, S.L, S.nb, P);
  sym_reduce_kernel<kModel, kKind><<<grid_for(n, 256, sms * 8), 256, 0, st>>>(P, n, S.nb, x, y, o0, o1, o2, o3);
  note_launches(3);
  return cudaGetLastError();
}

}  // namespace

size_t expected_sym_workspace_bytes(int model, int64_t n) { return sym_layout(model, n).total; }

cudaError_t launch_expected_sym(int kind, int model, const double* x, const double* y, const double* gk,
                                const double* gs, int64_t n, void* workspace, double* o0, double* o1, double* o2,
                                double* o3, cudaStream_t st) {
  char* ws = static_cast<char*>(workspace);
  if (model == MH_UBCM) {
    if (kind == kSymFwd) return run_sym<MH_UBCM, kSymFwd>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
    if (kind == kSymDiag) return run_sym<MH_UBCM, kSymDiag>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
    if (kind == kSymDiagF) return run_sym<MH_UBCM, kSymDiagF>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
    if (kind == kSymBwdF) return run_sym<MH_UBCM, kSymBwdF>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
    return run_sym<MH_UBCM, kSymBwd>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
  }
  if (kind == kSymFwd) return run_sym<MH_UECM, kSymFwd>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
  if (kind == kSymDiag) return run_sym<MH_UECM, kSymDiag>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
  if (kind == kSymDiagF) return run_sym<MH_UECM, kSymDiagF>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
  if (kind == kSymBwdF) return run_sym<MH_UECM, kSymBwdF>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
  return run_sym<MH_UECM, kSymBwd>(x, y, gk, gs, n, ws, o0, o1, o2, o3, st);
}

}  // namespace mh

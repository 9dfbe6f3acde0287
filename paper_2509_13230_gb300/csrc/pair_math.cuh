// Double-float helpers shared by the pairwise kernels (pairwise.cu,
// pairsym.cu): the operand ranges the double-float terms accept, the
// compensated accumulator, 1 - r, and products and quotients whose results
// stay unnormalised.
#pragma once

#include "walk_math.cuh"

namespace mh {

// Operands the double-float path takes.  Every intermediate of the pair terms
// then stays a normal FP32 number, low parts included:
//   a (x for the UBCM, x y for the UECM): 0 or [2^-30, 2^30], so a product of
//     two lies in [2^-60, 2^60], D^2 below 2^121 and Q above 2^-90;
//   y: in [0, 1 - 2^-12], so 1 - y_i y_j >= 2^-11 and its double-float value
//     (absolute error about 2^-48) is good to 2^-37 relative;
//   gradients: |g| <= 2^40.
__device__ __forceinline__ bool df_safe_a(double v) { return v == 0.0 || (v >= 0x1p-30 && v <= 0x1p30); }
__device__ __forceinline__ bool df_safe_y(double v) { return v >= 0.0 && v <= 1.0 - 0x1p-12; }
__device__ __forceinline__ bool df_safe_g(double g) { return fabs(g) <= 0x1p40; }

// Sum of double-float terms: two_sum on the high parts, the low parts and the
// rounding errors summed in FP32 until norm() folds them back.
struct DfAcc {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(df2 t) {
    const df2 s = two_sum(hi, t.hi);
    hi = s.hi;
    lo += s.lo + t.lo;
  }
  __device__ __forceinline__ void norm() {
    const df2 s = two_sum(hi, lo);
    hi = s.hi;
    lo = s.lo;
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

// 1 - r for a double-float r in [0, 1 - 2^-11]: |1| >= r.hi, so fast_two_sum
// returns 1 - r.hi exactly as a pair, and the low parts add without cancellation.
__device__ __forceinline__ df2 one_minus(df2 r) {
  const df2 s = fast_two_sum(1.0f, -r.hi);
  return fast_two_sum(s.hi, s.lo - r.lo);
}

// Products and quotients of the pair terms without the final renormalising
// fast_two_sum: every consumer in the pair kernels takes a pair whose low word is up to a
// few units of 2^-24 of its high word (the quotient's residual subtracts the
// high words exactly and the low words separately, the sloppy sums and the
// accumulators add the words apart), so the value hi + lo keeps the same
// accuracy at three fewer operations each.
__device__ __forceinline__ df2 dfu_mul(df2 a, df2 b) {
  const float p = a.hi * b.hi;
  return df2{p, fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, fmaf(a.hi, b.hi, -p)))};
}
__device__ __forceinline__ df2 dfu_div(df2 a, df2 b) {
  const float rc = __fdividef(1.0f, b.hi);
  const float th = a.hi * rc;
  const float p = b.hi * th;
  const float e = fmaf(b.lo, th, fmaf(b.hi, th, -p));  // b th = p + e
  // a.hi - p is exact: th is within a few ulp of a.hi / b.hi
  return df2{th, ((a.hi - p) + (a.lo - e)) * rc};
}

}  // namespace mh

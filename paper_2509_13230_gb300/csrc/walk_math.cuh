// Decision arithmetic of the walk and of the weight draw.
//
// Edge probabilities in the canonical FP64 order (no FMA contraction; the
// library is built with --fmad=false):
//   UBCM  (Eq. 1): z = x_i x_j,          p = z / (1 + z)
//   UECM  (Eq. 3): A = a_i a_j,          p = A / ((1 - r) + A),  r = y_i y_j
//   bound (Eq. 5):                       phat = A / ((1 - c) + A)
// with a = x y.  The geometric skip and the weight need floor(ln U / ln v)
// for v = 1 - q and v = r; skip_floor / weight_floor return it exactly up to
// draws within a few ulp of an integer, where the FP64 library logarithm of
// the device and of the host may round differently.
#pragma once

#include "mh_internal.cuh"

namespace mh {

__device__ __forceinline__ double prob_ubcm(double xi, double xj) {
  const double z = xi * xj;
  return z / (1.0 + z);
}
__device__ __forceinline__ double prob_uecm(double ai, double aj, double r) {
  const double A = ai * aj;
  return A / ((1.0 - r) + A);
}
__device__ __forceinline__ double prob_hat(double ai, double aj, double c) {
  const double A = ai * aj;
  return A / ((1.0 - c) + A);
}

// floor(t), t = ln U / ln(1 - q) with U from 53 random bits, 0 < q < 1.
// Returns `room` (or more) when t >= room, i.e. the candidate falls past the
// segment end.
__device__ __forceinline__ int64_t skip_floor(uint32_t hi, uint32_t lo, double q, int64_t room, bool fp64_only,
                                              unsigned long long& fallbacks) {
  (void)fp64_only;
  (void)fallbacks;
  const double U = unit_open0(hi, lo);
  const double t = log(U) / log1p(-q);
  if (t >= static_cast<double>(room)) return room;
  return static_cast<int64_t>(floor(t));
}

// UECM weight of edge e of segment k, row i, sample s (Eq. 4):
// w = 1 + floor(ln U_w / ln r), U_w from Philox {2^31 | e/2, k, i, s},
// words (1,0) for even e and (3,2) for odd e.  Sets `overflow` and returns
// INT32_MAX above INT32_MAX - 1.
__device__ __forceinline__ int32_t draw_weight(uint32_t e, uint32_t k, uint32_t i, uint32_t sample, uint32_t key0,
                                               uint32_t key1, double r, bool& overflow) {
  if (!(r > 0.0)) return 1;
  const uint4 w = philox4x32_10(make_uint4(0x80000000u | (e >> 1), k, i, sample), key0, key1);
  const double Uw = (e & 1u) ? unit_open0(w.w, w.z) : unit_open0(w.y, w.x);
  const double tw = log(Uw) / log(r);
  if (tw >= 2147483646.0) {
    overflow = true;
    return 2147483647;
  }
  return 1 + static_cast<int32_t>(floor(tw));
}

}  // namespace mh

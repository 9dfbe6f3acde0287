// Decision arithmetic of the walk and of the weight draw.
//
// Canonical values (the definition every decision must reproduce): FP64
// expressions in one fixed order, no FMA contraction (--fmad=false):
//   UBCM  (Eq. 1): z = x_i x_j,          p = z / (1 + z)
//   UECM  (Eq. 3): A = a_i a_j,          p = A / ((1 - r) + A),  r = y_i y_j
//   bound (Eq. 5):                       phat = A / ((1 - c) + A)
//   skip  (Fig. 2): L = 1 + floor(log(U) / log1p(-q))
//   accept:        V < p / q
//   weight (Eq. 4): w = 1 + floor(log(U_w) / log(r))
// with a = x y and the FP64 library log / log1p.
//
// Fast path.  Values are unevaluated sums hi + lo of two FP32 numbers,
// built from error-free transformations (Dekker 1971; Joldes, Muller,
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", 2017).  Logarithms use Tang's table-driven method
// ("Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 1990): f = c_k (1 + r) with c_k from a
// 512-entry table, ln f = ln c_k + log1p(r), |r| < 2^-9, log1p by its
// alternating series.  With these
//   t = E / lambda,  E = -ln U,  lambda = -ln(1 - q) = log1p(z)  (UBCM)
//                                              = log1p(A / (1 - c))  (UECM)
// is estimated twice: by the first level (FP32 pairs whose low words carry
// only the leading error terms, within 2^-30.4 t of the canonical t; the skip
// is decided when t lies more than t 2^-28 + 2^-22 from every integer) and,
// for the few draws that level leaves, by full double-float arithmetic
// (about 48 significant bits, relative error far below 2^-36; decided when t
// lies more than t 2^-36 + 2^-40 from every integer).  The acceptance is
// decided when V lies more than p/q 2^-18 from the FP32 estimate of p/q.
// Anything else, and any input outside the fast path's range, takes the
// canonical FP64 path above, so decisions equal the canonical ones except
// where the device and host FP64 logarithms themselves round differently
// (draws within a few ulp of an integer boundary).
//
// Fast range.  lambda above is the exact -ln(1 - q) of the exact q, while
// the canonical t divides by log1p(-fl(q)): q = z / (1 + z) carries two
// roundings, fl(q) = q (1 + eps) with |eps| <= 2^-52, and 1 - fl(q) =
// (1 - q)(1 - z eps).  The canonical lambda is therefore off by a relative
// z 2^-52 / ln(1 + z) (z = x_i x_j, or A / fl(1 - c) for the UECM bound),
// which grows without limit in z: 2^-36 at z = 2^21.  The fast levels take
// only q with z < kFastZq = 2^16, where that term is at most 2^-39.5, below a
// ninth of the double-float margin (and far below the first level's); larger z go
// to the canonical FP64 path.  The acceptance quotient p/q and the weight's
// ln r carry no such term (p/q is a ratio of two values near 1 with relative
// errors of a few 2^-53; fl(y_i y_j) moves ln r by at most 2^-53 against
// |ln r| >= 2^-12 on the fast path).
#pragma once

#include "mh_internal.cuh"

namespace mh {

// Largest z (x_i x_j, or A / (1 - c)) whose q the fast levels decide.
constexpr float kFastZq = 0x1p16f;

// ---- canonical FP64 values ----------------------------------------------------
__device__ __forceinline__ double prob_ubcm(double xi, double xj) {
  const double z = xi * xj;
  return z / (1.0 + z);
}
// Chung-Lu (MH_CHUNG_LU): the expected multiplicity read as a probability.
__device__ __forceinline__ double prob_cl(double xi, double xj) {
  const double z = xi * xj;
  return z >= 1.0 ? 1.0 : z;
}
__device__ __forceinline__ double prob_uecm(double ai, double aj, double r) {
  const double A = ai * aj;
  return A / ((1.0 - r) + A);
}
__device__ __forceinline__ double prob_hat(double ai, double aj, double c) {
  const double A = ai * aj;
  return A / ((1.0 - c) + A);
}

// ---- double-float primitives ---------------------------------------------------
struct df2 {
  float hi, lo;
};

__device__ __forceinline__ df2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df2{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df2 fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return df2{s, b - (s - a)};
}
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df2 df_mul_f(df2 a, float b) {
  const float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const df2 s = two_sum(a.hi, b.hi);
  const df2 t = two_sum(a.lo, b.lo);
  const df2 v = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(v.hi, t.lo + v.lo);
}
// Sum without the second error-free transformation on the low parts
// (Joldes et al.'s "sloppy" addition).  Used only where the operands cannot
// cancel by more than a small factor (same signs, or a bounded ratio),
// where its error stays a few units of 2^-48 of the result.
__device__ __forceinline__ df2 df_add_sloppy(df2 a, df2 b) {
  const df2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df2 df_add_f(df2 a, float b) {
  const df2 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, a.lo + s.lo);
}
__device__ __forceinline__ df2 df_div(df2 a, df2 b) {
  const float th = __fdividef(a.hi, b.hi);
  const df2 r = df_mul_f(b, th);
  const float dh = a.hi - r.hi;  // exact: th is within a few ulp of a.hi / b.hi
  const float dl = a.lo - r.lo;
  const float tl = __fdividef(dh + dl, b.hi);
  return fast_two_sum(th, tl);
}
__device__ __forceinline__ df2 to_df(float2 v) { return df2{v.x, v.y}; }

// FP64 value -> nearest double-float (setup only; uses the FP64 pipe).
__device__ __forceinline__ df2 df_from_double(double v) {
  const float h = __double2float_rn(v);
  return df2{h, __double2float_rn(v - static_cast<double>(h))};
}

// ---- logarithm table (Tang 1990) ------------------------------------------------
// Entry k: c_k = the FP32 value f with the 14 low fraction bits cleared, for
// f in [0.75, 1.5): k < 256 covers c in [1, 1.5) (step 2^-9), k >= 256 covers
// c in [0.75, 1) (step 2^-10).  inv = 1 / c_k and ln = ln c_k as double-floats.
constexpr int kLnTable = 512;
struct LnEntry {
  float inv_hi, inv_lo, ln_hi, ln_lo;
};

__device__ __forceinline__ float ln_table_c(int k) {
  return k < 256 ? 1.0f + static_cast<float>(k) * 0x1p-9f : 0.5f * (1.0f + static_cast<float>(k) * 0x1p-9f);
}

// Fills `tab` (kLnTable entries); one thread per entry.
__device__ __forceinline__ void ln_table_entry(LnEntry* tab, int k) {
  const double c = static_cast<double>(ln_table_c(k));
  const df2 inv = df_from_double(1.0 / c);
  const df2 ln = df_from_double(log(c));
  tab[k] = LnEntry{inv.hi, inv.lo, ln.hi, ln.lo};
}

// Copies the workspace table into shared memory (whole block, then sync).
__device__ __forceinline__ void ln_table_to_shared(LnEntry* sh, const LnEntry* global) {
  for (int t = threadIdx.x; t < kLnTable; t += blockDim.x) sh[t] = global[t];
}

constexpr float kLn2Hi = 0.693147182464599609375f;    // ln 2 rounded to FP32
constexpr float kLn2Lo = -1.904654323148236017e-09f;  // ln 2 - kLn2Hi

// ln f for a double-float f in [0.75, 1.5) (|ln f| >= 2^-10 when f < 1,
// see neg_ln_u53).  Relative error below 2^-44 away from f = 1.
__device__ __forceinline__ df2 ln_mid(df2 f, const LnEntry* tab) {
  const unsigned bits = __float_as_uint(f.hi);
  const int k = static_cast<int>((bits >> 14) & 511u);
  const float c = __uint_as_float(bits & ~0x3FFFu);  // f.hi with 14 low bits cleared
  const LnEntry e = tab[k];
  const df2 d = two_sum(f.hi - c, f.lo);             // f.hi - c is exact
  const df2 r = df_mul(d, df2{e.inv_hi, e.inv_lo});  // f = c (1 + r), |r| < 2^-9
  // log1p(r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 (truncation < |r|^6/6 < 2^-56)
  const float rh = r.hi;
  const float r2h = rh * rh;
  const float r2l = fmaf(rh, rh, -r2h) + 2.0f * rh * r.lo;
  const float tail = rh * r2h * fmaf(rh, fmaf(rh, 0.2f, -0.25f), 0.333333343f);
  const df2 half_r2 = df2{-0.5f * r2h, -0.5f * r2l};
  df2 s = df_add_sloppy(r, half_r2);           // |r^2/2| < 2^-10 |r|
  s = df_add_f(s, tail);
  return df_add_sloppy(df2{e.ln_hi, e.ln_lo}, s);  // cancels at most about 2x (see neg_ln_u53)
}

// Splits a double-float v >= 2^-100 into 2^e * f with f in [0.75, 1.5).
__device__ __forceinline__ df2 split_mid(df2 v, int& e) {
  int ex = static_cast<int>((__float_as_uint(v.hi) >> 23) & 0xFF) - 127;
  if (__uint_as_float((__float_as_uint(v.hi) & 0x007FFFFFu) | 0x3F800000u) >= 1.5f) ex += 1;
  e = ex;
  const float sc = __uint_as_float(static_cast<unsigned>(127 - ex) << 23);  // 2^-ex, exact
  return df2{v.hi * sc, v.lo * sc};
}

// log1p(v) for a double-float v >= 0 (v.hi >= 2^-100).
__device__ __forceinline__ df2 log1p_df(df2 v, const LnEntry* tab) {
  if (v.hi < 0x1p-9f) {
    // v - v^2/2 + v^3/3 - v^4/4 + v^5/5 (truncation < v^6/6)
    const float vh = v.hi;
    const float v2h = vh * vh;
    const float v2l = fmaf(vh, vh, -v2h) + 2.0f * vh * v.lo;
    const float tail = vh * v2h * fmaf(vh, fmaf(vh, 0.2f, -0.25f), 0.333333343f);
    df2 s = df_add_sloppy(v, df2{-0.5f * v2h, -0.5f * v2l});
    return df_add_f(s, tail);
  }
  int e;
  const df2 f = split_mid(df_add_f(v, 1.0f), e);
  const df2 lf = ln_mid(f, tab);
  if (e == 0) return lf;
  const float ef = static_cast<float>(e);
  const df2 eln2 = df_mul_f(df2{kLn2Hi, kLn2Lo}, ef);
  return df_add_sloppy(eln2, lf);  // e >= 1: |ln f| < 0.41 < e ln 2
}

// Exact u32 -> f32 conversion for values below 2^24 (a 32-bit convert; the
// 64-bit integer converts run on the FP64 unit).
__device__ __forceinline__ float u32f(unsigned v) { return __uint2float_rn(v); }

// E = -ln U for U = N 2^-53, N = 1 .. 2^53 (exact integer input).
__device__ __forceinline__ df2 neg_ln_u53(unsigned long long N, const LnEntry* tab) {
  const unsigned long long W = (1ull << 53) - N;  // (1 - U) 2^53, exact
  if (W < (1ull << 44)) {
    // -ln(1 - w) = w + w^2/2 + w^3/3 + w^4/4 + w^5/5 (truncation < w^6/6), w < 2^-9
    const float wh0 = u32f(static_cast<unsigned>(W >> 20)) * 0x1p-33f;          // exact (24 bits)
    const float wl0 = u32f(static_cast<unsigned>(W & 0xFFFFFu)) * 0x1p-53f;    // exact (20 bits)
    const df2 w = fast_two_sum(wh0, wl0);
    const float wh = w.hi;
    const float w2h = wh * wh;
    const float w2l = fmaf(wh, wh, -w2h) + 2.0f * wh * w.lo;
    const float tail = wh * w2h * fmaf(wh, fmaf(wh, 0.2f, 0.25f), 0.333333343f);
    df2 s = df_add_sloppy(w, df2{0.5f * w2h, 0.5f * w2l});
    return df_add_f(s, tail);
  }
  // N = 2^e f, f in [0.75, 1.5); E = (53 - e) ln 2 - ln f
  const int lz = __clzll(static_cast<long long>(N));
  const unsigned long long Nn = N << lz;  // leading one at bit 63
  const unsigned top = static_cast<unsigned>(Nn >> 40);                 // 24 bits
  const unsigned mid = static_cast<unsigned>(Nn >> 16) & 0xFFFFFFu;     // next 24 bits
  const float h = u32f(top) * 0x1p-23f;                                  // in [1, 2), exact
  const float l = u32f(mid) * 0x1p-47f;                                  // exact; bits below 2^-47 dropped
  int e = 63 - lz;
  df2 f = fast_two_sum(h, l);
  if (f.hi >= 1.5f) {
    f = df2{f.hi * 0.5f, f.lo * 0.5f};
    e += 1;
  }
  const df2 lf = ln_mid(f, tab);
  const int m = 53 - e;
  if (m == 0) return df2{-lf.hi, -lf.lo};
  const df2 mln2 = df_mul_f(df2{kLn2Hi, kLn2Lo}, static_cast<float>(m));
  return df_add_sloppy(mln2, df2{-lf.hi, -lf.lo});  // m >= 1, ln f < 0.41: cancels at most 2.4x
}

// Exact decision of floor(t) for a double-float t >= 0 against `room`
// (0 <= room < 2^31): returns 1 and sets `fl` when decided, 0 when t lies
// within the error margin of an integer.  fl >= room: past the segment end.
__device__ __forceinline__ int floor_decided(df2 t, int room, unsigned& fl) {
  const float froom = static_cast<float>(room);
  if (t.hi > fmaf(froom, 0x1p-20f, froom) + 2.0f) {  // far past the end
    fl = static_cast<unsigned>(room);
    return 1;
  }
  const float margin = fmaf(t.hi, 0x1p-36f, 0x1p-40f);
  const float fh = floorf(t.hi);
  float f0, f1;
  unsigned F;
  if (fh == t.hi) {
    const float fl_lo = floorf(t.lo);
    F = __float2uint_rz(fh) + static_cast<unsigned>(__float2int_rz(fl_lo));
    f0 = t.lo - fl_lo;
    f1 = 1.0f - f0;
  } else {
    F = __float2uint_rz(fh);
    const float d = t.hi - fh;  // exact
    f0 = d + t.lo;
    f1 = (1.0f - d) - t.lo;
  }
  if (!(f0 > margin) || !(f1 > margin)) return 0;
  fl = F;
  return 1;
}

// ---- FP32 level of the weight draw ------------------------------------------------
// The same table, used in FP32: ln f = ln c_k + log1p(r) with r rounded once
// and a cubic in r.  The estimate of E below has a relative error of at most
// 6u (u = 2^-24); a weight is decided from it only when tw lies 2^-18 tw +
// 2^-22 away from an integer.

// float(v) for v < 2^23, exact, without a convert instruction.
__device__ __forceinline__ float small_u2f(unsigned v) { return __uint_as_float(0x4B000000u | v) - 8388608.0f; }

__device__ __forceinline__ float log1p_poly_f(float r) {  // r - r^2/2 + r^3/3, |r| < 2^-9
  return r * fmaf(r, fmaf(r, 0.333333343f, -0.5f), 1.0f);
}

// -ln U for U = N 2^-53.  Sets ok = false for U < 2^-8 (about 2^-8 of the
// draws), which the double-float level then handles.
__device__ __forceinline__ float neg_ln_u53_f(unsigned long long N, const LnEntry* tab, bool& ok) {
  const unsigned long long W = (1ull << 53) - N;
  ok = true;
  if (W < (1ull << 44)) {  // U > 1 - 2^-9: -ln(1 - w) = w + w^2/2 + w^3/3 + ...
    const float w = small_u2f(static_cast<unsigned>(W >> 22)) * 0x1p-31f +
                    small_u2f(static_cast<unsigned>(W & 0x3FFFFFu)) * 0x1p-53f;
    return w * fmaf(w, fmaf(w, 0.333333343f, 0.5f), 1.0f);
  }
  const unsigned nh = static_cast<unsigned>(N >> 21);  // top 32 bits of the 53-bit N
  const int lz = __clz(nh);
  if (lz > 8) {
    ok = false;
    return 0.0f;
  }
  const unsigned top = nh << lz;                // leading one at bit 31: f = top 2^-31 in [1, 2)
  const int k = static_cast<int>((top >> 22) & 511u);
  const bool half = top >= 0xC0000000u;         // f >= 1.5: use f / 2 and one more power of two
  // f - c_k: the 22 bits of top below the table index (exact) plus the 21
  // bits of N below nh, worth lo 2^(lz - 52) in f = N 2^(lz - 52), added with
  // one rounding (dropping them would cost up to 2^(lz - 31) in U)
  const float d_top = small_u2f(top & 0x3FFFFFu) * (half ? 0x1p-32f : 0x1p-31f);
  const float lo_scale = __uint_as_float(static_cast<unsigned>(127 + lz - 52 - (half ? 1 : 0)) << 23);
  const float d = fmaf(small_u2f(static_cast<unsigned>(N & 0x1FFFFFull)), lo_scale, d_top);
  const LnEntry e = tab[k];
  const float lnf = e.ln_hi + log1p_poly_f(d * e.inv_hi);
  const float m = static_cast<float>(1 + lz - static_cast<int>(half));  // U = 2^-m f
  return fmaf(m, kLn2Lo, fmaf(m, kLn2Hi, -lnf));
}

// ---- first level of the walk: FP32 pairs ---------------------------------------------
// E = -ln U and lambda = log1p(z) as unevaluated pairs hi + lo of FP32
// numbers, from the same table: the leading terms (m ln 2, ln c_k, r) are
// added with error-free transformations and everything smaller (the low
// words of ln 2, ln c_k, 1 / c_k and of the inputs, and the series beyond r)
// is summed in FP32 into lo, and the pair is normalised (|lo| <= ulp(hi) /
// 2; the pair quotient needs it: its low word divides by hi alone).  Error
// bounds (u = 2^-24), from the term sizes:
//   E, U > 1 - 2^-9 (w = 1 - U < 2^-9): the quartic w + w^2/2 + w^3/3 + w^4/4
//     (truncation below 2^-38 w) with its square term rounded three times,
//     3u w^2/2 <= 2^-32.4 w, the low word of w in the square (2^-33 w) and the
//     last rounding (2^-34 w): 2^-31.5 relative;
//   E, U <= 1 - 2^-9: absolute errors of about 2^-41 (the cubic's roundings,
//     3u r^2/2 with |r| <= 2^-9.6; the low word of r in the square; the three
//     roundings of lo) against E >= 2^-9: 2^-32;
//   lambda, z < 2^-9: as the first case, 2^-31.5 (plus 2^-44 carried by the
//     double-float z itself);
//   lambda, z >= 2^-9: absolute about 2^-40.3 against lambda >= 2^-9: 2^-31.3.
// The pair quotient adds below 2^-41 and the canonical FP64 t differs from
// E / lambda by at most 2^-39.5 relative (the fast-range note above), so the
// estimate of t lies within 2^-30.4 t (plus 2^-24 from rounding its
// fraction) of the canonical t; floor_decided_m decides a skip only when t
// lies 2^-28 t + 2^-22 away from every integer, over five times that.

// ln 2 = kLn2A + kLn2B with kLn2A of 17 significant bits (m kLn2A exact for
// integers m < 128) and kLn2B rounded to FP32 (error below 2^-44).
constexpr float kLn2A = 0x1.62e4p-1f;
constexpr float kLn2B = 0x1.7f7d1cp-20f;

// log1p(r) - r = r^2 (-1/2 + r/3 - r^2/4) + lo, for |r| < 2^-9 (truncation
// below |r|^5 / 5); `lo` is the low word of r.
__device__ __forceinline__ float log1p_rest(float r, float lo) {
  return fmaf(r * r, fmaf(r, fmaf(r, -0.25f, 0.333333343f), -0.5f), lo);
}

// E = -ln U for U = N 2^-53, N = 1 .. 2^53, as hi + lo.
__device__ __forceinline__ df2 neg_ln_u53_m(unsigned long long N, const LnEntry* tab) {
  const unsigned long long W = (1ull << 53) - N;
  if (W < (1ull << 44)) {  // U > 1 - 2^-9: -ln(1 - w) = w + w^2/2 + w^3/3 + w^4/4
    const df2 w = fast_two_sum(small_u2f(static_cast<unsigned>(W >> 21)) * 0x1p-32f,   // exact (23 bits)
                               small_u2f(static_cast<unsigned>(W & 0x1FFFFFu)) * 0x1p-53f);  // exact (21 bits)
    return fast_two_sum(w.hi, fmaf(w.hi * w.hi, fmaf(w.hi, fmaf(w.hi, 0.25f, 0.333333343f), 0.5f), w.lo));
  }
  // N = 2^(63 - lz64) f with f = top 2^-31 + low 2^-52 in [1, 2): top holds the
  // leading 32 bits, low the 21 bits below them
  unsigned nh = static_cast<unsigned>(N >> 21);
  unsigned low = static_cast<unsigned>(N) & 0x1FFFFFu;
  int lz = __clz(nh);
  float lo_scale;
  int m;  // U = 2^-m f before the halving below
  if (lz <= 8) {
    nh <<= lz;
    lo_scale = __uint_as_float(static_cast<unsigned>(127 + lz - 52) << 23);
    m = 1 + lz;
  } else {  // U < 2^-8: normalise over the whole word (about 2^-8 of the draws)
    lz = __clzll(static_cast<long long>(N));
    const unsigned long long Nn = N << lz;
    nh = static_cast<unsigned>(Nn >> 32);
    low = static_cast<unsigned>(Nn) >> 11;  // the 21 low significant bits (bits 10..0 of Nn are zero)
    lo_scale = 0x1p-52f;
    m = lz - 10;
  }
  const bool half = nh >= 0xC0000000u;  // f >= 1.5: use f / 2 and one more power of two
  const LnEntry e = tab[(nh >> 22) & 511u];
  // f - c_k = d_hi + d_lo, both exact: the 22 bits of nh below the table index and the low bits
  const float d_hi = small_u2f(nh & 0x3FFFFFu) * (half ? 0x1p-32f : 0x1p-31f);
  const float d_lo = small_u2f(low) * (half ? 0.5f * lo_scale : lo_scale);
  const float mf = static_cast<float>(m - static_cast<int>(half));  // U = 2^-m f, m >= 0
  // r = (f - c_k) / c_k = r_hi + r_lo, |r| < 2^-9.6.  d_hi + d_lo is not
  // normalised (d_lo reaches 2^-23), so r_lo can exceed an ulp of r_hi: the
  // square term takes the rounded sum r_hi + r_lo (relative error 2^-24).
  const float r_hi = d_hi * e.inv_hi;
  const float r_lo = fmaf(d_lo, e.inv_hi, fmaf(d_hi, e.inv_lo, fmaf(d_hi, e.inv_hi, -r_hi)));
  // E = m ln 2 - ln c_k - log1p(r).  m kLn2A >= |ln c_k| (m >= 1) or m = 0,
  // and |m kLn2A - ln c_k| >= 2^-9 > |r_hi| (m = 0 only for f / 2 < 1 - 2^-9).
  const df2 s = fast_two_sum(mf * kLn2A, -e.ln_hi);
  const df2 v = fast_two_sum(s.hi, -r_hi);
  return fast_two_sum(v.hi, v.lo + (s.lo + (fmaf(mf, kLn2B, -e.ln_lo) - log1p_rest(r_hi + r_lo, r_lo))));
}

// lambda = log1p(v) for a double-float v with v.hi in [2^-100, 2^40), as hi + lo.
__device__ __forceinline__ df2 log1p_m(df2 v, const LnEntry* tab) {
  if (v.hi < 0x1p-9f) return fast_two_sum(v.hi, log1p_rest(v.hi, v.lo));
  const df2 D = two_sum(1.0f, v.hi);  // 1 + v.hi exactly
  const float corr = __fdividef(D.lo + v.lo, D.hi);  // log1p(corr) = corr to 2^-47
  int ex = static_cast<int>((__float_as_uint(D.hi) >> 23) & 0xFF) - 127;
  float f = __uint_as_float((__float_as_uint(D.hi) & 0x007FFFFFu) | 0x3F800000u);
  if (f >= 1.5f) {
    f *= 0.5f;
    ex += 1;
  }
  const unsigned bits = __float_as_uint(f);
  const LnEntry e = tab[(bits >> 14) & 511u];
  const float d = f - __uint_as_float(bits & ~0x3FFFu);  // f - c_k, exact
  const float r_hi = d * e.inv_hi;
  const float r_lo = fmaf(d, e.inv_lo, fmaf(d, e.inv_hi, -r_hi));
  // lambda = ex ln 2 + ln c_k + log1p(r) + corr.  ex kLn2A >= |ln c_k| (ex >=
  // 1) or ex = 0, where c_k >= 1 and ln c_k >= r_hi or ln c_k = 0.
  const float fe = static_cast<float>(ex);
  const df2 s = fast_two_sum(fe * kLn2A, e.ln_hi);
  const df2 w = fast_two_sum(s.hi, r_hi);
  return fast_two_sum(w.hi, w.lo + (s.lo + (fmaf(fe, kLn2B, e.ln_lo) + (log1p_rest(r_hi, r_lo) + corr))));
}

// a / b for normalised pairs (|lo| <= ulp(hi) / 2): a reciprocal
// estimate corrected once by Newton-Raphson with an FMA residual (Markstein,
// "IA-64 and Elementary Functions", 2000), then the low word from the
// residual a - q b: relative error below 2^-41.
__device__ __forceinline__ df2 quot_df(df2 a, df2 b) {
  const float rc = __fdividef(1.0f, b.hi);
  const float q0 = a.hi * rc;
  const float q1 = fmaf(fmaf(-q0, b.hi, a.hi), rc, q0);
  const float rho = fmaf(-q1, b.lo, fmaf(-q1, b.hi, a.hi) + a.lo);
  return df2{q1, rho * rc};
}

// floor(t) of a first-level estimate t = hi + lo (t >= 0, hi < 2^32): 1 and
// `fl` when t lies more than t 2^-28 + 2^-22 from every integer, 0 otherwise.
__device__ __forceinline__ int floor_m(df2 t, unsigned& fl) {
  const float margin = fmaf(t.hi, 0x1p-28f, 0x1p-22f);
  const float fh = floorf(t.hi);
  const float fr0 = (t.hi - fh) + t.lo;  // t.hi - fh exact
  const float ff = floorf(fr0);          // -1, 0 or 1 below 2^23; lo's whole part above
  const float fr = fr0 - ff;             // exact, or rounded up to 1 when fr0 is a tiny negative
  if (!(fr > margin) || !(1.0f - fr > margin)) return 0;
  fl = __float2uint_rz(fh) + static_cast<unsigned>(__float2int_rz(ff));
  return 1;
}

// The skip's floor(t) against `room` (0 <= room < 2^31): fl >= room means
// past the end of the segment.
__device__ __forceinline__ int floor_decided_m(df2 t, int room, unsigned& fl) {
  const float froom = static_cast<float>(room);
  if (t.hi > fmaf(froom, 0x1p-20f, froom) + 1.0f) {  // past the end of the segment
    fl = static_cast<unsigned>(room);
    return 1;
  }
  return floor_m(t, fl);
}

// A boundary draw: t >= 0.5 lies within 8 ulp of an integer.  The device
// and host FP64 log / log1p may round differently only for such draws, so
// they are counted (MH_STAT_BOUNDARY); the same rule as the oracle's.
__device__ __forceinline__ bool near_integer(double t) {
  if (!(t >= 0.5) || !isfinite(t)) return false;
  // ulp of a positive normal t: 2^(exponent - 52), the step to the next double up
  const double ulp = __longlong_as_double(__double_as_longlong(t) & 0x7FF0000000000000ll) * 0x1p-52;
  return fabs(t - rint(t)) <= 8.0 * ulp;
}

// Double-float level of the skip: floor(t) for U = N 2^-53 and lambda =
// log1p(zq), capped at `room`, or -1 when t lies within that level's margin
// of an integer.  Out of line: the walk reaches it only for draws within the
// first level's margin (a few in 10^5 on long skips), and inlined it would
// hold registers across the whole walk loop.
static __device__ __noinline__ int skip_df(unsigned long long N, df2 zq, int room, const LnEntry* tab) {
  const df2 t = df_div(neg_ln_u53(N, tab), log1p_df(zq, tab));
  unsigned fl = 0;
  return floor_decided(t, room, fl) ? static_cast<int>(fl) : -1;
}

// Canonical FP64 skip: floor(log(U) / log1p(-q)), capped at `room`.  A draw
// near an integer m in [1, room] (one that decides the candidate) is counted
// in `boundary`.  Every such draw reaches this function: the fast levels
// decide only draws whose t lies farther than their margins from an integer.
static __device__ __noinline__ unsigned skip_fp64(unsigned long long N, double q, int room,
                                                  unsigned long long& boundary) {
  if (q >= 1.0) return 0;
  const double U = static_cast<double>(N) * 0x1p-53;
  const double t = log(U) / log1p(-q);
  if (near_integer(t) && rint(t) <= static_cast<double>(room)) boundary += 1;
  if (t >= static_cast<double>(room)) return static_cast<unsigned>(room);
  return static_cast<unsigned>(floor(t));
}

// Acceptance filter: 1 = accept, 0 = reject, -1 = undecided (use FP64).
// p_f / q_f approximates p/q to a relative error well below 2^-18.  vw is
// the high word of the draw's words (3,2): V = top53(vw, lo) 2^-53 lies in
// [vlo, vlo + 2^-24) with vlo = (vw >> 8) 2^-24 (a 32-bit convert, exact).
__device__ __forceinline__ int accept_decided(uint32_t vw, float p_f, float q_f) {
  const float R = __fdividef(p_f, q_f);
  const float vlo = __uint2float_rn(vw >> 8) * 0x1p-24f;
  const float vhi = vlo + 0x1p-24f;
  if (vhi <= R * (1.0f - 0x1p-18f)) return 1;
  if (vlo >= R * (1.0f + 0x1p-18f)) return 0;
  return -1;
}

// ---- UECM weight (Eq. 4) ---------------------------------------------------------
// w = 1 + floor(ln U_w / ln r) for edge e of segment k, row i, sample s; U_w
// from Philox {2^31 | e/2, k, i, s}, words (1,0) for even e and (3,2) for odd
// e.  lny_i + lny_j approximates ln r in double-float (per-node ln y); the
// FP64 path computes log(U_w) / log(fl(y_i y_j)).
static __device__ __noinline__ int32_t weight_fp64(unsigned long long N, double r, bool& overflow,
                                                   unsigned long long& boundary) {
  if (!(r > 0.0)) return 1;
  const double tw = log(static_cast<double>(N) * 0x1p-53) / log(r);
  if (near_integer(tw)) boundary += 1;
  if (tw >= 2147483646.0) {
    overflow = true;
    return 2147483647;
  }
  return 1 + static_cast<int32_t>(floor(tw));
}

// yj points at y_j: it is read only on the canonical FP64 path (rare), so the
// usual draw costs no load of it.
__device__ __forceinline__ int32_t draw_weight(uint32_t e, uint32_t k, uint32_t i, uint32_t sample, uint32_t key0,
                                               uint32_t key1, double yi, const double* yj, df2 lnyi, df2 lnyj,
                                               const LnEntry* tab, bool fp64_only, bool& overflow,
                                               unsigned long long& fallbacks, unsigned long long& boundary) {
  const uint4 w = philox4x32_10(make_uint4(0x80000000u | (e >> 1), k, i, sample), key0, key1);
  const unsigned long long N = (e & 1u) ? top53(w.w, w.z) + 1ull : top53(w.y, w.x) + 1ull;
  const df2 nlr = df_add(lnyi, lnyj);  // ln r (negative)
  if (!fp64_only && nlr.hi < -0x1p-12f && nlr.hi > -0x1p+100f) {
    // FP32 level: t = E / -ln r with E from the FP32 logarithm of U (within
    // 6u), the divisor the double-float ln r rounded once (0.5u) and a 2-ulp
    // quotient: about 9u in all, far inside the margin 2^-18 t + 2^-22.
    bool ok;
    const float Ef = neg_ln_u53_f(N, tab, ok);
    if (ok) {
      const float t = __fdividef(Ef, -nlr.hi);
      if (t < 0x1p22f) {
        const float margin = fmaf(t, 0x1p-18f, 0x1p-22f);
        const float fh = floorf(t);
        const float fr = t - fh;  // exact
        if (fr > margin && 1.0f - fr > margin) return 1 + static_cast<int32_t>(fh);
      }
    }
    const df2 E = neg_ln_u53(N, tab);
    const df2 t = df_div(E, df2{-nlr.hi, -nlr.lo});
    unsigned fl;
    if (t.hi < 2.0e9f && floor_decided(t, 0x7FFFFFFF, fl)) return 1 + static_cast<int32_t>(fl);
  }
  fallbacks += 1;
  return weight_fp64(N, yi * *yj, overflow, boundary);
}

}  // namespace mh

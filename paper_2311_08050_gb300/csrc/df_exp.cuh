// exp(-x) for x >= 0 in double-float on the FP32 pipes (~2^-46 relative).
//
// Method: reduction by multiples of ln 2 (Cody and Waite, "Software Manual for the
// Elementary Functions", 1980): -x = k ln 2 + r, |r| <= ln 2 / 2, with ln 2 held as a
// double-float so that r is accurate; then exp(r) = (exp(r / 4))^4, the inner factor by its
// Taylor series to degree 10 (|r / 4| <= 0.0867: the first dropped term is below 2^-64), two
// squarings (each doubles the relative error, so few of them), and the exact scaling by 2^k.
// The series' terms of degree 6 and up sum to less than 6e-10, so they are evaluated in FP32
// (error below 2^-52 of the result); the degrees 5 .. 0 run in double-float by Horner's rule,
// each step adding a coefficient to a product at most 0.1 of it, so the leading words add by
// the fast two-sum.
#pragma once
#include "df64.cuh"

namespace inla {

static __device__ __forceinline__ df df_exp_neg(df x) {
  constexpr double kLn2 = 0.69314718055994530942;
  const float ln2_hi = (float)kLn2;
  const float ln2_lo = (float)(kLn2 - (double)(float)kLn2);
  const df ln2 = df_make(ln2_hi, ln2_lo);
  // k = round(-x / ln 2) from the leading word; x >= 0 so k <= 0
  const float kf = rintf(-x.hi * 1.4426950408889634f);
  const df r = df_add(df_neg(x), df_neg(df_mul(df_make(kf, 0.f), ln2)));
  const df u = df_scale(r, 0.25f);  // r / 4, exact
  // Taylor coefficients 1/n!, n = 0..10, as double-float
  constexpr double c[11] = {1.0,           1.0,            0.5,             1.0 / 6.0,        1.0 / 24.0,        1.0 / 120.0,
                            1.0 / 720.0,   1.0 / 5040.0,   1.0 / 40320.0,   1.0 / 362880.0,   1.0 / 3628800.0};
  float tail = (float)c[10];
#pragma unroll
  for (int n = 9; n >= 6; --n) tail = __fmaf_rn(tail, u.hi, (float)c[n]);
  df p = df_mul(df_make(tail, 0.f), u);
#pragma unroll
  for (int n = 5; n >= 0; --n) {
    const df cn = df_make((float)c[n], (float)(c[n] - (double)(float)c[n]));
    if (n < 5) p = df_mul(p, u);
    // cn + p with |p| < |cn|: the leading words by the fast two-sum, then the low words
    float sh, se;
    fast_two_sum(cn.hi, p.hi, sh, se);
    se = __fadd_rn(se, __fadd_rn(cn.lo, p.lo));
    fast_two_sum(sh, se, sh, se);
    p = df{sh, se};
  }
  p = df_mul(p, p);
  p = df_mul(p, p);
  const int k = (int)kf;
  return k >= -126 ? df_scale(p, pow2f(k)) : df_make(0.f, 0.f);
}

}  // namespace inla

// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, giving ~48 significant bits.  Built from the error-free
// transformations TwoSum (Knuth) and TwoProduct via FMA (Dekker / Ogita-Rump-Oishi), so
// every operation runs on the FP32 pipes: on this GPU FP64 has 1/64 of the FP32 rate.
#pragma once
#include <cuda_runtime.h>

namespace inla {

struct df {
  float hi, lo;
};

static __device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// exact: s + e = a + b
static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// exact when |a| >= |b| (or a == 0)
static __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

static __device__ __forceinline__ df df_add(df a, df b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return df{s, e};
}
static __device__ __forceinline__ df df_add_f(df a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  fast_two_sum(s, e, s, e);
  return df{s, e};
}
static __device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
static __device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s;
  fast_two_sum(p, e, s, e);
  return df{s, e};
}
// a + b without the second error-free step on the low words: error ~2^-44 (|a| + |b|), the
// bound of a backward-stable sum, against ~2^-44 |a + b| for df_add
static __device__ __forceinline__ df df_add_fast(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  fast_two_sum(s, e, s, e);
  return df{s, e};
}
// 1 / a: FP32 reciprocal refined by one Newton step in double-float (~2^-46 relative)
static __device__ __forceinline__ df df_recip(df a) {
  const float r0 = 1.0f / a.hi;
  // residual 1 - a r0, its leading part exact through the FMA
  const float e = __fmaf_rn(-a.lo, r0, __fmaf_rn(-a.hi, r0, 1.0f));
  float s, t;
  fast_two_sum(r0, r0 * e, s, t);
  return df{s, t};
}
// sqrt(a), a > 0: FP32 square root refined by one Newton step in double-float
static __device__ __forceinline__ df df_sqrt(df a) {
  const float s0 = sqrtf(a.hi);
  const float res = __fadd_rn(__fmaf_rn(-s0, s0, a.hi), a.lo);  // a - s0^2 (leading part exact)
  float s, t;
  fast_two_sum(s0, res * (0.5f / s0), s, t);
  return df{s, t};
}
// a * b for an exact power-of-two scale b (no rounding unless under/overflow)
static __device__ __forceinline__ df df_scale(df a, float p2) { return df{a.hi * p2, a.lo * p2}; }
// acc + a * b
static __device__ __forceinline__ df df_fma(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }

static __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
static __device__ __forceinline__ df df_from_double(double v) {
  const float h = __double2float_rn(v);
  const float l = __double2float_rn(v - (double)h);
  return df{h, l};
}
static __device__ __forceinline__ df df_load(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}
static __device__ __forceinline__ void df_store(float2* p, df a) { *p = make_float2(a.hi, a.lo); }

// 2^e as a float for e in the normal range
static __device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((e + 127) << 23);
}

}  // namespace inla

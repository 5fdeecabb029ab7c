// Ozaki slicing of one lane's 8 consecutive operand values (shared by the slicing kernels and
// by the diagonal-tile kernel, which slices its inverse tile in place of a separate launch).
#pragma once
#include <cstdint>
#include "df64.cuh"

namespace inla {

// Slice the 8 values of one lane, given the exponent e of their (row, chunk): x 2^(7-e) has
// magnitude <= 128; slice s is v_s = round(h) of the running remainder h (scaled by 2^7 per
// slice), stored as the BF16 number v_s 2^(-7s) -- exact: |v_s| <= 128 has at most 8
// significant bits, so the BF16 encoding is the upper half of the FP32 one.  The remainder
// h - v_s is exact (Sterbenz), and adding the low word back is exact too: h - v_s is zero or a
// multiple of ulp(h), at least twice the low word.  Integer rounding by the 1.5 * 2^23 shift.
static __device__ __forceinline__ void slice_and_store(const df (&x)[8], int e, uint16_t* planes,
                                                       int64_t plane_stride, int S, int64_t base, bool valid) {
  constexpr float kRound = 12582912.f;  // 1.5 * 2^23
  const float sc = pow2f(7 - e);
  float h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    h[i] = x[i].hi * sc;
    l[i] = x[i].lo * sc;
  }
  float p7 = 1.f;  // 2^(-7s)
  for (int s = 0; s < S; ++s) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = __fsub_rn(__fadd_rn(h[i], kRound), kRound);
      const uint32_t bits = __float_as_uint(v * p7) >> 16;
      if (i & 1) w[i >> 1] |= bits << 16;
      else w[i >> 1] = bits;
      float a, b;
      fast_two_sum(__fsub_rn(h[i], v), l[i], a, b);
      h[i] = a * 128.f;
      l[i] = b * 128.f;
    }
    if (valid) *reinterpret_cast<uint4*>(planes + s * plane_stride + base) = make_uint4(w[0], w[1], w[2], w[3]);
    p7 *= 0.0078125f;
  }
}

static __device__ __forceinline__ int chunk_exponent(float m) {
  // smallest e with m <= 2^e  (m > 0); e = 0 for an all-zero chunk
  if (!(m > 0.f)) return 0;
  int e;
  const float f = frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  (void)f;
  return e;
}

}  // namespace inla

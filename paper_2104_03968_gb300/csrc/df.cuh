// Double-float arithmetic on the FP32 pipe: a value is an unevaluated sum hi + lo of two floats
// (about 48 significant bits).  GB300 issues FP32 FMAs ~70x faster than FP64 ones, so FP64-grade
// residual updates of the mixed solver are cheaper in this form.
//
// Building blocks (exact transformations, Dekker 1971 and Knuth, TAOCP vol. 2, 4.2.2):
//   two_prod(a, b)      p + e == a * b exactly (e from one FMA)
//   two_sum(a, b)       s + e == a + b exactly (six additions, no ordering condition)
//   quick_two_sum(a, b) s + e == a + b exactly when |a| >= |b| or a == 0
// and an integer split of an FP64 number into hi (its leading 24 significant bits) + lo (the rest
// rounded to 24 bits), relative error <= 2^-47.
#pragma once

namespace fld {

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// d = hi + lo.  hi is d truncated to 24 significant bits (so it equals d rounded toward zero);
// lo is the remainder, rounded to nearest.  Integer and FP32 instructions only when 2^-74 <=
// |d| < 2^128, where both parts are normal floats; other values take FP64 conversions.
__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const int e = (int)((h >> 20) & 0x7ffu);  // biased binary exponent
  if (e >= 1023 - 74 && e <= 1023 + 127) {
    const unsigned sign = h & 0x80000000u;
    hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
    // the low 29 significand bits have weight 2^(E - 52), E = e - 1023
    lo = __uint2float_rn(l & 0x1fffffffu) * __uint_as_float(sign | ((unsigned)(e - 1023 - 52 + 127) << 23));
  } else {
    hi = __double2float_rz(d);
    lo = __double2float_rn(d - (double)hi);
  }
}

}  // namespace fld

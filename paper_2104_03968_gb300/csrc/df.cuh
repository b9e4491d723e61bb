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
// The FP64 fallbacks are out of line: inlined, the compiler predicates them into every split and
// the FP64 pipe (~1/70 of the FP32 rate on GB300) becomes the bottleneck.
static __device__ __noinline__ void split_f64_slow(double d, int shift, float& hi, float& lo) {
  const double ds = shift ? ldexp(d, -shift) : d;
  hi = __double2float_rz(ds);
  lo = __double2float_rn(ds - (double)hi);
}

__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const int e = (int)((h >> 20) & 0x7ffu);  // biased binary exponent
  if (e >= 1023 - 74 && e <= 1023 + 127) {
    const unsigned sign = h & 0x80000000u;
    hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
    // the low 29 significand bits have weight 2^(E - 52), E = e - 1023
    lo = __uint2float_rn(l & 0x1fffffffu) * __uint_as_float(sign | ((unsigned)(e - 1023 - 52 + 127) << 23));
  } else {
    split_f64_slow(d, 0, hi, lo);
  }
}

// d * 2^-shift split as above (shift is an integer power of two, so the scaling is exact); ok is
// false -- and hi, lo hold an FP64-computed fallback -- when the scaled value leaves the range
// of the integer path.
__device__ __forceinline__ void split_f64_scaled(double d, int shift, float& hi, float& lo, bool& ok) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const int e = (int)((h >> 20) & 0x7ffu) - shift;
  ok = e >= 1023 - 74 && e <= 1023 + 127 && ((h >> 20) & 0x7ffu) != 0u;
  if (ok) {
    const unsigned sign = h & 0x80000000u;
    hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
    lo = __uint2float_rn(l & 0x1fffffffu) * __uint_as_float(sign | ((unsigned)(e - 1023 - 52 + 127) << 23));
  } else {
    split_f64_slow(d, shift, hi, lo);
  }
}

// unbiased binary exponent of a positive normal double (integer instructions only)
__device__ __forceinline__ int exponent_f64(double d) {
  return (int)(((unsigned)__double2hiint(d) >> 20) & 0x7ffu) - 1023;
}

// x * 2^k for a float whose result stays a normal float (exponent-field arithmetic)
__device__ __forceinline__ float scale_pow2(float x, int k) {
  return x == 0.0f ? 0.0f : __int_as_float(__float_as_int(x) + (k << 23));
}

// double-float values and their arithmetic (~2^-47 relative per operation)
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_norm(float s, float e) {
  dfl r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e += t;
  quick_two_sum(s, e, s, e);
  e += f;
  return df_norm(s, e);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_norm(p, e);
}

// a / b: a first FP32 quotient, its remainder a - q1 b in double-float, one correction
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = a.hi * rb;
  const dfl r = df_add(a, df_neg(df_mul(b, {q1, 0.0f})));
  const float q2 = r.hi * rb;
  return df_norm(q1, q2);
}

}  // namespace fld

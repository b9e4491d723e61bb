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

// a + b for operands of the same sign (no cancellation, so the low parts are summed plainly)
__device__ __forceinline__ dfl df_add_pos(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return df_norm(s, e);
}

// a * b for a float b
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
  float p, e;
  two_prod(a.hi, b, p, e);
  e = fmaf(a.lo, b, e);
  return df_norm(p, e);
}

__device__ __forceinline__ dfl df_sqr(dfl a) {
  float p, e;
  two_prod(a.hi, a.hi, p, e);
  e = fmaf(a.hi + a.hi, a.lo, e);
  return df_norm(p, e);
}

// a * 2^k exactly for a power-of-two float s = 2^k (no overflow or underflow)
__device__ __forceinline__ dfl df_scale(dfl a, float s) { return {a.hi * s, a.lo * s}; }

// hardware approximations (SFU), about one ulp; flush-to-zero is harmless inside the window
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// a / b: an FP32 quotient q1 = a.hi r (r: the hardware reciprocal after one FP32 Newton step,
// ~2^-24), its remainder a - b q1 in double-float (a.hi - p is exact by Sterbenz's lemma since p is
// within a factor 2 of a.hi), and one correction q2 = remainder * r.  Relative error ~2^-47.
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  float r = rcp_approx(b.hi);
  r = fmaf(r, fmaf(-b.hi, r, 1.0f), r);
  const float q1 = a.hi * r;
  float p, pe;
  two_prod(b.hi, q1, p, pe);
  float rem = (a.hi - p) - pe;
  rem += a.lo;
  rem = fmaf(-b.lo, q1, rem);
  return df_norm(q1, rem * r);
}

// sqrt(a) for a > 0 by Karp and Markstein's method (ACM TOMS 23(4), 1997): s0 = a.hi y with
// y ~ 1/sqrt(a.hi) from the hardware, and one correction s0 + (a - s0^2) y / 2 whose remainder
// a - s0^2 is formed in double-float (a.hi - p exact by Sterbenz's lemma).  Relative error ~2^-46.
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  const float y = rsqrt_approx(a.hi);
  const float s0 = a.hi * y;
  float p, pe;
  two_prod(s0, s0, p, pe);
  const float rem = ((a.hi - p) - pe) + a.lo;
  return df_norm(s0, rem * (0.5f * y));
}

// Window of the fast double-float paths: |hi| in [2^-100, 2^126), so that lo (~2^-24 |hi|) is a
// normal float and products of two in-window values stay finite or leave the window visibly.
// Zero, subnormal, infinite and NaN values are outside.
__device__ __forceinline__ bool df_in(dfl x) {
  const unsigned e = (__float_as_uint(x.hi) >> 23) & 0xffu;
  return e >= 27u && e <= 252u;
}

// split_f64 without the FP64 fallback: ok is false (hi, lo undefined) outside 2^-74 <= |d| < 2^128
// unless d is +-0, which splits to (0, 0)
__device__ __forceinline__ void split_f64_try(double d, float& hi, float& lo, bool& ok) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const int e = (int)((h >> 20) & 0x7ffu);
  const unsigned sign = h & 0x80000000u;
  const bool zero = ((h & 0x7fffffffu) | l) == 0u;
  ok = (e >= 1023 - 74 && e <= 1023 + 127) || zero;
  hi = zero ? 0.0f : __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
  lo = zero ? 0.0f
            : __uint2float_rn(l & 0x1fffffffu) * __uint_as_float(sign | ((unsigned)(e - 1023 - 52 + 127) << 23));
}

// exact float -> double for zero and normal floats, with integer instructions only
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned m = b & 0x7fffffffu;
  const unsigned hi = (b & 0x80000000u) | (m ? (m >> 3) + (896u << 20) : 0u);
  return __hiloint2double((int)hi, (int)(m << 29));
}

// hi + lo rounded to FP64 (one FP64 addition)
__device__ __forceinline__ double df_to_f64(dfl x) { return f32_to_f64(x.hi) + f32_to_f64(x.lo); }

// 2^e as a float, -126 <= e <= 127
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

// binary exponent of a nonzero normal float
__device__ __forceinline__ int exponent_f32(float x) { return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127; }

// d = m 2^ex with m in [1, 2) as a double-float (hi: the leading 24 bits, lo: the other 29 rounded
// to 24), integer instructions only.  ok is false for zero, subnormal, infinite and NaN d;
// xsplit0 also accepts +-0 (m = 0, ex = 0).
__device__ __forceinline__ void xsplit(double d, dfl& m, int& ex, bool& ok) {
  const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
  const unsigned ef = (h >> 20) & 0x7ffu, sign = h & 0x80000000u;
  ok = ef != 0u && ef != 0x7ffu;
  ex = (int)ef - 1023;
  m.hi = __uint_as_float(sign | (127u << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
  m.lo = __uint2float_rn(l & 0x1fffffffu) * __uint_as_float(sign | (75u << 23));  // weight 2^-52
}
__device__ __forceinline__ void xsplit0(double d, dfl& m, int& ex, bool& ok) {
  xsplit(d, m, ex, ok);
  if (((unsigned)__double2hiint(d) & 0x7fffffffu) == 0u && __double2loint(d) == 0) {
    m = {0.0f, 0.0f};
    ex = 0;
    ok = true;
  }
}

// The double-float m 2^e: exact when the result lies in the window; 0 below 2^-150 (negligible
// beside any in-window sum it is added to); ok is cleared above 2^125.
__device__ __forceinline__ dfl xval(dfl m, int e, bool& ok) {
  const int te = e + exponent_f32(m.hi);
  if (m.hi == 0.0f || te < -150) return {0.0f, 0.0f};
  if (te > 125) ok = false;
  const int e1 = min(max(e, -126), 127);
  const float s = pow2f(e1), s2 = pow2f(min(max(e - e1, -126), 127));
  return {m.hi * s * s2, m.lo * s * s2};
}

// v 2^k for a normal double v by exponent-field arithmetic; ok is cleared unless the result is a
// normal double
__device__ __forceinline__ double ldexp_f64(double v, int k, bool& ok) {
  const int h = __double2hiint(v);
  const int ef = (h >> 20) & 0x7ff;
  ok = ok && ef != 0 && ef + k >= 1 && ef + k <= 2046;
  return __hiloint2double(h + k * (1 << 20), __double2loint(v));
}

}  // namespace fld

// Natural logarithm and exponential of FP64 arguments with their work in double-float arithmetic
// on the FP32 pipe (df.cuh), for the tabulated opacity of the mixed precision (bilinear in
// log10 rho and log10 T on log10 kappa, Sect. 5.1's tables).  GB300 runs FP64 instructions at
// ~1/64 of the FP32 rate, and the FP64 logarithms and power of ten of a table lookup were the
// larger part of the wind-column step's FP64 work.
//
// Both follow the textbook construction: reduce the argument by a power of two, then sum a
// series whose leading terms are evaluated in double-float and whose small tail is evaluated in
// FP32 (the tail is below 2^-30 of the result, so its FP32 rounding stays below 2^-53).
//   ln x   = e ln 2 + ln m,  x = m 2^e with m in [1/sqrt 2, sqrt 2),
//            ln m = 2 atanh s = 2 s (1 + s^2/3 + s^4/5 + ...),  s = (m - 1)/(m + 1), |s| <= 0.172;
//   exp y  = 2^n exp r,  n = round(y / ln 2), |r| <= ln 2 / 2,  exp r = sum r^k / k!.
// Absolute error of ln x below ~1e-15 plus the rounding of e ln 2; relative error of exp y below
// ~1e-15 plus 2^-53 |y|.  Arguments: ln_df takes a positive normal double, exp_df |y| < 700.
#pragma once

#include "df.cuh"
#include "fld_common.cuh"

namespace fld {

// a double constant as a double-float (hi its float rounding, lo the rounded remainder)
struct dfc {
  float hi, lo;
};
constexpr dfc make_dfc(double v) { return {(float)v, (float)(v - (double)(float)v)}; }

__device__ __forceinline__ dfl df_add_c(dfl a, dfc c) { return df_add(a, dfl{c.hi, c.lo}); }

constexpr double kLn2 = 0.69314718055994530942;
// ln 2 = kLn2Hi + kLn2Lo with kLn2Hi = 22713 / 32768 (15 significant bits: n kLn2Hi is exact)
constexpr double kLn2Hi = 0.693145751953125;
constexpr double kLn2Lo = kLn2 - kLn2Hi;

__device__ __forceinline__ double ln_df(double x) {
  dfl m;
  int e;
  bool ok;
  xsplit(x, m, e, ok);  // m in [1, 2)
  if (m.hi > 1.41421356f) {
    m.hi *= 0.5f;
    m.lo *= 0.5f;
    e += 1;
  }
  // s = (m - 1) / (m + 1); m.hi - 1 is exact (Sterbenz: m.hi in [1/2, 2])
  const dfl s = df_div(df_norm(m.hi - 1.0f, m.lo), df_add(m, dfl{1.0f, 0.0f}));
  const dfl s2 = df_sqr(s);
  // 1/13 + s^2/15 + s^4/17 + s^6/19 in FP32 (s^12 <= 7e-10: its rounding is negligible)
  const float z = s2.hi;
  float t = fmaf(z, 1.0f / 19.0f, 1.0f / 17.0f);
  t = fmaf(z, t, 1.0f / 15.0f);
  t = fmaf(z, t, 1.0f / 13.0f);
  constexpr dfc c11 = make_dfc(1.0 / 11.0), c9 = make_dfc(1.0 / 9.0), c7 = make_dfc(1.0 / 7.0),
                c5 = make_dfc(1.0 / 5.0), c3 = make_dfc(1.0 / 3.0);
  dfl q = df_add_c(df_mul_f(s2, t), c11);
  q = df_add_c(df_mul(s2, q), c9);
  q = df_add_c(df_mul(s2, q), c7);
  q = df_add_c(df_mul(s2, q), c5);
  q = df_add_c(df_mul(s2, q), c3);
  q = df_add(df_mul(s2, q), dfl{1.0f, 0.0f});
  const dfl lnm = df_scale(df_mul(s, q), 2.0f);
  return (double)e * kLn2Hi + fma((double)e, kLn2Lo, df_to_f64(lnm));
}

__device__ __forceinline__ double exp_df(double y) {
  const double n = rint(y * (1.0 / kLn2));
  double r = fma(-n, kLn2Hi, y);
  r = fma(-n, kLn2Lo, r);  // |r| <= ln 2 / 2 (plus rounding)
  dfl rd;
  split_f64(r, rd.hi, rd.lo);
  // 1/8! + r/9! + ... + r^5/13! in FP32 (r^8/8! <= 5.3e-9 of the result)
  const float z = rd.hi;
  float t = fmaf(z, 1.0f / 6227020800.0f, 1.0f / 479001600.0f);
  t = fmaf(z, t, 1.0f / 39916800.0f);
  t = fmaf(z, t, 1.0f / 3628800.0f);
  t = fmaf(z, t, 1.0f / 362880.0f);
  t = fmaf(z, t, 1.0f / 40320.0f);
  constexpr dfc c7 = make_dfc(1.0 / 5040.0), c6 = make_dfc(1.0 / 720.0), c5 = make_dfc(1.0 / 120.0),
                c4 = make_dfc(1.0 / 24.0), c3 = make_dfc(1.0 / 6.0);
  dfl q = df_add_c(df_mul_f(rd, t), c7);
  q = df_add_c(df_mul(rd, q), c6);
  q = df_add_c(df_mul(rd, q), c5);
  q = df_add_c(df_mul(rd, q), c4);
  q = df_add_c(df_mul(rd, q), c3);
  q = df_add(df_mul(rd, q), dfl{0.5f, 0.0f});
  q = df_add(df_mul(rd, q), dfl{1.0f, 0.0f});
  q = df_add(df_mul(rd, q), dfl{1.0f, 0.0f});
  bool in = true;
  return ldexp_f64(df_to_f64(q), (int)n, in);
}

// The bilinear table opacity of opacity() (fld_common.cuh) with the two logarithms and the power
// of ten in double-float: the same lookup and interpolation, in FP64, between them.
__device__ __forceinline__ double opacity_table_df(const Opacity& o, double rho, double T) {
  constexpr double kInvLn10 = 0.43429448190325182765, kLn10 = 2.30258509299404568402;
  double u = (ln_df(rho) * kInvLn10 - o.tlo0) * o.su0;
  double v = (ln_df(T) * kInvLn10 - o.tlo1) * o.su1;
  u = fmin(fmax(u, 0.0), (double)(o.tn0 - 1));
  v = fmin(fmax(v, 0.0), (double)(o.tn1 - 1));
  int i = min((int)u, o.tn0 - 2), j = min((int)v, o.tn1 - 2);
  double fu = u - i, fv = v - j;
  const double* t = o.table + (long long)i * o.tn1 + j;
  double l = (1 - fu) * ((1 - fv) * __ldg(t) + fv * __ldg(t + 1)) +
             fu * ((1 - fv) * __ldg(t + o.tn1) + fv * __ldg(t + o.tn1 + 1));
  return exp_df(l * kLn10);
}

}  // namespace fld

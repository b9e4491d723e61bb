// Per-cell point-implicit gas-radiation energy exchange (arXiv 2104.03968, Sect. 3.3).
//
// Backward Euler on the heating/cooling terms gives the quartic
//     a1 x^4 + (1 + a2) x - (1 + a2) eps^n - a2 E^n = 0,   x = eps^{n+1} in ]0, eps^n + E^n[,
// with a2 = c kappa rho dt and a1 = 4 kappa rho sigma dt ((gamma-1)/(rho gas_R))^4 (the gas law
// turns T^4 into a multiple of eps^4), then E^{n+1} = (a1 x^4 + E^n) / (1 + a2).
//
// FP64 is scarce on GB300, so the root is found in two phases: the quartic, rescaled to
// coefficients in (0, 1], is solved by safeguarded Halley iterations in FP32; FP64 Newton steps
// (FP64 residual, FP32 reciprocal of the derivative) then polish it to FP64 accuracy.
// Coefficients outside the FP32-safe range take the paper's FP64 Halley iteration, which falls
// back to bisection after `maxit` iterations.
#pragma once

#include "df.cuh"
#include "fld_common.cuh"

namespace fld {

// FP64 safeguarded Halley on a y^4 + y - cc = 0 over ]0, 1], bisection after maxit iterations.
__device__ inline double halley64(double a, double cc, int maxit, int* iters, int* bisected) {
  double lo = 0.0, hi = 1.0, y = cc;
  int it = 0;
  const double tol = 4.0 * 2.220446049250313e-16;
  while (it < maxit) {
    double y2 = y * y;
    double f = fma(a * y2, y2, y - cc);
    if (f == 0.0) {
      *iters = it;
      return y;
    }
    if (f < 0) lo = y;
    else hi = y;
    double f1 = fma(4.0 * a * y2, y, 1.0);
    double f2 = 12.0 * a * y2;
    double yn = y - 2.0 * f * f1 / (2.0 * f1 * f1 - f * f2);
    ++it;
    // a converged step may land on the bracket end just set from y: accept it first
    if (fabs(yn - y) <= tol * yn) {
      *iters = it;
      return yn;
    }
    if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
    y = yn;
  }
  *bisected = 1;
  for (int k = 0; k < 200 && hi - lo > tol * hi; ++k) {
    double m = 0.5 * (lo + hi);
    double m2 = m * m;
    if (fma(a * m2, m2, m - cc) < 0) lo = m;
    else hi = m;
  }
  *iters = it;
  return 0.5 * (lo + hi);
}

// two FP64 Newton steps from the FP32 root (tiny or huge coefficients); d: the last step
static __device__ __noinline__ double polish64(double a, double cc, float y32, float r1f, float* d) {
  const double r1 = (double)r1f;
  double y = (double)y32, dd = 0.0;
  for (int it = 0; it < 2; ++it) {
    const double y2 = y * y;
    dd = fma(a * y2, y2, y - cc) * r1;
    y -= dd;
  }
  *d = (float)dd;
  return y;
}

// FP32 root of a y^4 + y - cc = 0 for af in [1e-30, 1e30], cf in [1e-30, 1]: y = ys z with
// ys = min(cc, (cc/a)^(1/4)) >= root, so that alpha z^4 + beta z = 1 with max(alpha, beta) = 1 and
// the root z lies in [0.72, 1]; safeguarded Halley on z.  Also returns r1 = 1/f'(y) for the polish.
// The divisions and roots take the hardware approximations (about one ulp): they only shift the
// FP32 root by a few ulps, which the polish removes.
__device__ __forceinline__ float halley32(float af, float cf, int& iters, float& r1) {
  const float icf = rcp_approx(cf);
  const float ys = fminf(cf, rsqrt_approx(sqrt_approx(af * icf)));
  const float ys2 = ys * ys;
  const float alpha = af * ys2 * ys2 * icf, beta = ys * icf;
  float z = 1.0f, lo = 0.0f, hi = 1.0f;
  for (int it = 0; it < 12; ++it) {
    const float z2 = z * z;
    const float f = fmaf(alpha * z2, z2, fmaf(beta, z, -1.0f));
    ++iters;
    if (f < 0.0f) lo = z;
    else hi = z;
    const float f1 = fmaf(4.0f * alpha * z2, z, beta);
    const float f2 = 12.0f * alpha * z2;
    float zn = z - 2.0f * f * f1 * rcp_approx(2.0f * f1 * f1 - f * f2);
    // a converged step may land on the bracket end just set from z: accept it before the
    // safeguard would replace it by a bisection
    if (fabsf(zn - z) <= 4e-7f * zn) {
      z = zn;
      break;
    }
    if (!(zn > lo && zn < hi)) zn = 0.5f * (lo + hi);
    z = zn;
  }
  const float y32 = ys * z;
  r1 = rcp_approx(fmaf(4.0f * af * y32 * y32, y32, 1.0f));
  return y32;
}

// Newton polish of the FP32 root in double-float arithmetic, two steps with the FP32 root's
// reciprocal slope r1 = 1/(4 a y^3 + 1) as the step factor (each step multiplies the error by
// ~1e-7, so two take the FP32 root to the rounding of the arithmetic).  d: the last step.
__device__ __forceinline__ dfl polish_df(dfl A, dfl C, float y32, float r1, float& d) {
  dfl Y{y32, 0.0f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const dfl Y2 = df_sqr(Y);
    const dfl F = df_add(df_add(df_mul(A, df_sqr(Y2)), Y), df_neg(C));
    d = F.hi * r1;
    Y = df_add(Y, {-d, 0.0f});
  }
  return Y;
}

// Updates (e, E) of one cell in place with FP64 coefficients.  Returns false (and leaves them) on
// invalid input.
__device__ inline bool exchange_cell(const ExchangeParams& p, double r, double k, double& e, double& E, int& iters,
                                     int& bis) {
  const double e0 = e, E0 = E;
  if (!(gt_zero(r) && gt_zero(k) && ge_zero(e0) && ge_zero(E0))) return false;
  const double S = e0 + E0;
  if (!pos_finite(S)) return true;  // eps = E = 0: nothing to exchange
  const double a2 = p.cdt * k * r;  // c kappa rho dt
  const double B = 1.0 + a2;
  const double r3 = r * r * r;
  const double P = r3 * B;
  // one reciprocal gives 1/rho^3, 1/(1+a2) and 1/S
  const double inv = rcp_nr(P * S);
  double ir3, u, invS;
  if (pos_finite(inv)) {
    ir3 = B * S * inv;
    u = r3 * S * inv;
    invS = P * inv;
  } else {
    ir3 = 1.0 / r3;
    u = 1.0 / B;
    invS = 1.0 / S;
  }
  // a1 = 4 sigma dt kappa rho ((gamma-1)/(rho gas_R))^4 = k4 kappa / rho^3
  const double a1 = p.k4 * k * ir3;
  // y = x / S solves  a y^4 + y - cc = 0,  a = a1 S^3/(1+a2) >= 0,  cc in (0, 1]
  const double a = a1 * (S * S) * S * u;
  const double cc = fma(a2 * u, E0, e0) * invS;
  const float af = (float)a, cf = (float)cc;
  double y;
  if (!p.plain64 && af >= 1e-30f && af <= 1e30f && cf >= 1e-30f) {
    float r1;
    const float y32 = halley32(af, cf, iters, r1);
    // polish in double-float while a, cc and y keep their low parts normal floats, else in FP64
    // (out of line)
    float d = 0.0f, yh = 0.0f;
    if (cf >= 0x1p-60f && af <= 0x1p60f) {
      float ah, al, ch, cl;
      split_f64(a, ah, al);
      split_f64(cc, ch, cl);
      const dfl Y = polish_df({ah, al}, {ch, cl}, y32, r1, d);
      y = (double)Y.hi + (double)Y.lo;
      yh = Y.hi;
    } else {
      y = polish64(a, cc, y32, r1, &d);
      yh = (float)y;
    }
    iters += 2;
    if (!(fabsf(d) <= 1e-12f * yh) || !(yh > 0.0f)) {
      int it2 = 0;
      y = halley64(a, cc, p.maxit, &it2, &bis);
      iters += it2;
    }
  } else {
    y = halley64(a, cc, p.maxit, &iters, &bis);
  }
  const double x = S * y;
  const double x2 = x * x;
  e = x;
  E = fma(a1 * x2, x2, E0) * u;
  return true;
}

static __device__ __noinline__ bool exchange_cell_f64(const ExchangeParams& p, double r, double k, double& e,
                                                      double& E, int& iters, int& bis) {
  return exchange_cell(p, r, k, e, E, iters, bis);
}

// The exchange of one valid cell (S = eps + E > 0) in double-float arithmetic, with no FP64
// arithmetic but the sum S and the two final roundings.  Each FP64 input is split into a mantissa
// in [1, 2) and a power of two; the products and quotients that form the dimensionless quartic
// coefficients
//     a2 = c dt kappa rho,   a = k4 kappa S^3 / (rho^3 (1 + a2)),   cc = a2 v + eps/S,
//     v = E / ((1 + a2) S)
// and the new energies
//     x = S y,   E^{n+1} = S (a y^4 + v)      (from E^{n+1} = (a1 x^4 + E^n)/(1 + a2))
// multiply mantissas and add the exponents as integers, so the path holds in any unit system in
// which a, cc and E^{n+1}/S lie in the double-float window (cgs included), not only near 1.
// Returns false (outputs unset) where the cell needs the FP64 path: a value outside the window or
// the FP32 root's range, or a polish that did not converge.
__device__ __forceinline__ bool exchange_cell_df(const ExchangeParams& p, double r, double k, double e0, double E0,
                                                 double S, double& e_out, double& E_out, int& iters) {
  bool ok, o1, o2, o5, o6;
  dfl rm, km, Sm, em, Em;
  int re, ke, Se, ee, Ee;
  xsplit(r, rm, re, ok);
  xsplit(k, km, ke, o1);
  xsplit(S, Sm, Se, o2);
  xsplit0(e0, em, ee, o5);
  xsplit0(E0, Em, Ee, o6);
  ok = ok && o1 && o2 && o5 && o6 && p.df_ok;
  const dfl cm{p.cdt_hi, p.cdt_lo}, qm{p.k4_hi, p.k4_lo};
  const int ce = p.cdt_e, qx = p.k4_e;
  // a2 = c dt kappa rho; B = 1 + a2 as mantissa and exponent (1 is negligible beside a2 > 2^100)
  const dfl a2m = df_mul(df_mul(cm, km), rm);
  const int a2e = ce + ke + re;
  dfl Bm = a2m;
  int Be = a2e;
  if (a2e <= 100) {
    const dfl B = df_add_pos({1.0f, 0.0f}, xval(a2m, a2e, ok));
    Be = exponent_f32(B.hi);
    Bm = df_scale(B, pow2f(-Be));
  }
  // v = E / (B S), cc = a2 v + eps / S, a = k4 kappa S^3 / (rho^3 B)
  const dfl vm = df_div(Em, df_mul(Bm, Sm));
  const int ve = Ee - Be - Se;
  const dfl C = df_add_pos(xval(df_mul(a2m, vm), a2e + ve, ok), xval(df_div(em, Sm), ee - Se, ok));
  const dfl am = df_div(df_mul(df_mul(qm, km), df_mul(df_sqr(Sm), Sm)), df_mul(df_mul(df_sqr(rm), rm), Bm));
  const int ae = qx + ke + 3 * Se - 3 * re - Be;
  const dfl A = xval(am, ae, ok);
  const float af = A.hi, cf = C.hi;
  // the FP32 root's range and the double-float polish's window
  if (!(ok && df_in(A) && df_in(C) && af >= 1e-30f && af <= 0x1p60f && cf >= 0x1p-60f)) return false;
  float r1, d = 0.0f;
  const float y32 = halley32(af, cf, iters, r1);
  const dfl Y = polish_df(A, C, y32, r1, d);
  iters += 2;
  if (!(fabsf(d) <= 1e-12f * Y.hi) || !(Y.hi > 0.0f)) return false;
  // x = S y and E^{n+1} / S = a y^4 + v (y = Ym 2^Ye)
  const int Ye = exponent_f32(Y.hi);
  const dfl Ym = df_scale(Y, pow2f(-Ye));
  const dfl ES = df_add_pos(xval(df_mul(am, df_sqr(df_sqr(Ym))), ae + 4 * Ye, ok), xval(vm, ve, ok));
  ok = ok && df_in(ES);
  e_out = ldexp_f64(df_to_f64(df_mul(Sm, Y)), Se, ok);
  E_out = ldexp_f64(df_to_f64(df_mul(ES, Sm)), Se, ok);
  return ok;
}

// Either path for one cell: double-float, else FP64 (out of line).  Same contract as exchange_cell.
__device__ __forceinline__ bool exchange_cell_fast(const ExchangeParams& p, double r, double k, double& e, double& E,
                                                   int& iters, int& bis) {
  const double e0 = e, E0 = E;
  if (!(gt_zero(r) && gt_zero(k) && ge_zero(e0) && ge_zero(E0))) return false;
  const double S = e0 + E0;
  if (!pos_finite(S)) return true;  // eps = E = 0: nothing to exchange
  double eo, Eo;
  int it = 0;
  if (exchange_cell_df(p, r, k, e0, E0, S, eo, Eo, it)) {
    e = eo;
    E = Eo;
    iters += it;
    return true;
  }
  return exchange_cell_f64(p, r, k, e, E, iters, bis);
}

// warp-aggregated diagnostics: max iterations and bisection count
__device__ inline void exchange_report(int iters, int bis, int* info_iters, int* info_bisect) {
  for (int o = 16; o > 0; o >>= 1) {
    iters = max(iters, __shfl_down_sync(0xffffffffu, iters, o));
    bis += __shfl_down_sync(0xffffffffu, bis, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (iters) atomicMax(info_iters, iters);
    if (bis) atomicAdd(info_bisect, bis);
  }
}

}  // namespace fld

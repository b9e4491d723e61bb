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

// Updates (e, E) of one cell in place.  Returns false (and leaves them) on invalid input.
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
  if (af >= 1e-30f && af <= 1e30f && cf >= 1e-30f) {
    // y = ys z with ys = min(cc, (cc/a)^(1/4)) >= root: alpha z^4 + beta z = 1 with
    // max(alpha, beta) = 1, so the root z lies in [0.72, 1]
    float ys = fminf(cf, sqrtf(sqrtf(cf / af)));
    float ys2 = ys * ys;
    float alpha = af * ys2 * ys2 / cf, beta = ys / cf;
    float z = 1.0f, lo = 0.0f, hi = 1.0f;
    for (int it = 0; it < 12; ++it) {
      float z2 = z * z;
      float f = fmaf(alpha * z2, z2, fmaf(beta, z, -1.0f));
      ++iters;
      if (f < 0.0f) lo = z;
      else hi = z;
      float f1 = fmaf(4.0f * alpha * z2, z, beta);
      float f2 = 12.0f * alpha * z2;
      float zn = z - 2.0f * f * f1 / (2.0f * f1 * f1 - f * f2);
      // a converged step may land on the bracket end just set from z: accept it before the
      // safeguard would replace it by a bisection
      if (fabsf(zn - z) <= 4e-7f * zn) {
        z = zn;
        break;
      }
      if (!(zn > lo && zn < hi)) zn = 0.5f * (lo + hi);
      z = zn;
    }
    // Newton polish of the FP32 root, two steps with the FP32 root's reciprocal slope
    // 1/f'(y) = 1/(4 a y^3 + 1) as the step factor (each step multiplies the error by ~1e-7, so two
    // take the FP32 root to the rounding of the arithmetic): in double-float arithmetic (df.cuh)
    // while a, cc and y keep their low parts normal floats, else in FP64 (out of line).
    const float y32 = ys * z;
    const float r1 = __frcp_rn(fmaf(4.0f * af * y32 * y32, y32, 1.0f));
    float d = 0.0f, yh = 0.0f;
    if (cf >= 0x1p-60f && af <= 0x1p60f) {
      float ah, al, ch, cl;
      split_f64(a, ah, al);
      split_f64(cc, ch, cl);
      const dfl A{ah, al}, C{-ch, -cl};
      dfl Y{y32, 0.0f};
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const dfl Y2 = df_mul(Y, Y);
        const dfl F = df_add(df_add(df_mul(A, df_mul(Y2, Y2)), Y), C);
        d = F.hi * r1;
        Y = df_add(Y, {-d, 0.0f});
      }
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

// Shared device-side definitions of the GB300 FLD library (sm_103a).
//
// Grid convention: cell (i,j,k) is element i + n0*(j + n1*k) (x fastest).  Face arrays of
// axis a hold the n_a + 1 faces along a for every cross-section cell: the x-face f of row
// (j,k) is element f + (n0+1)*(j + n1*k), the y-face f of column (i,k) is i + n0*(f + (n1+1)*k),
// the z-face f is i + n0*(j + n1*f).  Face f of axis a lies between cells f-1 and f.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "../../include/fld.h"

namespace fld {

constexpr int kBlock = 256;

// Kernels this library has launched in the process, for fld_launch_count: every launch site calls
// note_launch; a captured CUDA graph counts its kernels at capture (its first launch follows) and
// again at each later replay.
extern std::atomic<unsigned long long> g_kernel_launches;
__host__ inline void note_launch(unsigned long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }
__host__ inline void unnote_launches(unsigned long long n) {
  g_kernel_launches.fetch_sub(n, std::memory_order_relaxed);
}
__host__ inline unsigned long long launch_count() { return g_kernel_launches.load(std::memory_order_relaxed); }

// Grid size for kernels that walk rows block-cyclically: at most cap blocks, and no more than the
// device keeps resident at once (blocks of kBlock threads of kernel fn), so that all of them
// advance through the rows in one front and the neighbouring rows and planes a block re-reads are
// the ones its neighbours fetched just before (a grid twice the resident size splits the rows in
// two fronts far apart, and the re-reads then miss in L2).
__host__ inline int front_grid(const void* fn, int cap, size_t smem = 0) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, smem) != cudaSuccess || per_sm <= 0)
    return cap;
  return per_sm * sms < cap ? per_sm * sms : cap;
}

struct GridDev {
  int n[3];
  int ndim;
  int bc[6];
  double bc_val[6];
  double dx[3];
  double inv_dx2[3];  // 1/dx^2 per axis
  long long ncell;
};

struct ExchangeParams {
  double c, sigma, gamma, gas_R, dt;
  int maxit;
  double cdt;  // c dt
  double k4;   // 4 sigma dt ((gamma-1)/gas_R)^4: a1 = k4 kappa / rho^3
  // cdt and k4 as m 2^e, m in [1, 2) split into two floats (the double-float exchange path);
  // df_ok is 0 unless both are positive and finite
  float cdt_hi, cdt_lo, k4_hi, k4_lo;
  int cdt_e, k4_e, df_ok;
  // 1: plain FP64 throughout (the FP64 solver's exchange): the FP64 safeguarded Halley iteration
  // from its first step, no double-float path and no FP32 start
  int plain64;
};

__host__ __device__ inline void mant_split(double v, float& hi, float& lo, int& e) {
  int ee = 0;
  const double m = 2.0 * frexp(v, &ee);
  e = ee - 1;
  hi = (float)m;
  lo = (float)(m - (double)hi);
}

__host__ __device__ inline ExchangeParams make_exchange(double c, double a_rad, double gamma, double gas_R, double dt,
                                                        int maxit) {
  ExchangeParams p;
  p.c = c;
  p.sigma = a_rad * c / 4.0;  // a_r = 4 sigma / c
  p.gamma = gamma;
  p.gas_R = gas_R;
  p.dt = dt;
  p.maxit = maxit;
  p.cdt = c * dt;
  double t = (gamma - 1.0) / gas_R;
  p.k4 = 4.0 * p.sigma * dt * t * t * t * t;
  mant_split(p.cdt, p.cdt_hi, p.cdt_lo, p.cdt_e);
  mant_split(p.k4, p.k4_hi, p.k4_lo, p.k4_e);
  p.df_ok = p.cdt > 0.0 && p.cdt <= 1.7e308 && p.k4 > 0.0 && p.k4 <= 1.7e308 && p.cdt >= 2.3e-308 && p.k4 >= 2.3e-308;
  p.plain64 = 0;
  return p;
}

// The exchange constants of one call; plain64 selects the FP64 arithmetic of the FP64 solver.
__host__ __device__ inline ExchangeParams make_exchange(double c, double a_rad, double gamma, double gas_R, double dt,
                                                        int maxit, bool plain64) {
  ExchangeParams p = make_exchange(c, a_rad, gamma, gas_R, dt, maxit);
  if (plain64) {
    p.plain64 = 1;
    p.df_ok = 0;
  }
  return p;
}

struct Opacity {
  int model;
  double kappa0, kr_a, kr_b;
  const double* table;
  int tn0, tn1;
  double tlo0, tlo1, thi0, thi1;
  double su0, su1;  // (tn - 1) / (thi - tlo) per axis: table cells per decade
};

// the Opacity of a parameter set (every path builds it here, so that the derived table scales
// are always set)
__host__ inline Opacity make_opacity(const fld_params& p) {
  Opacity o{};
  o.model = p.opacity;
  o.kappa0 = p.kappa0;
  o.kr_a = p.kr_a;
  o.kr_b = p.kr_b;
  o.table = p.table;
  o.tn0 = p.tn[0];
  o.tn1 = p.tn[1];
  o.tlo0 = p.tlo[0];
  o.tlo1 = p.tlo[1];
  o.thi0 = p.thi[0];
  o.thi1 = p.thi[1];
  o.su0 = o.thi0 > o.tlo0 ? (o.tn0 - 1) / (o.thi0 - o.tlo0) : 0.0;
  o.su1 = o.thi1 > o.tlo1 ? (o.tn1 - 1) / (o.thi1 - o.tlo1) : 0.0;
  return o;
}

// device status word: bit flags OR-ed by kernels, read back by the host
enum : unsigned { kStatNonpositive = 1u, kStatNonfinite = 2u };

// Range tests on the bit pattern (integer pipe); FP64 compares would occupy the scarce FP64 pipe.
// gt_zero(x) == (x > 0.0) and ge_zero(x) == (x >= 0.0), NaN giving false, +inf allowed.
__device__ __forceinline__ bool gt_zero(double x) {
  long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool ge_zero(double x) {
  long long b = __double_as_longlong(x);
  return (b >= 0 && b <= 0x7FF0000000000000LL) || b == (long long)0x8000000000000000ULL;
}
// x > 0 and finite
__device__ __forceinline__ bool pos_finite(double x) {
  long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000LL;
}

__host__ __device__ inline long long face_count(const int n[3], int a) {
  long long c = 1;
  for (int b = 0; b < 3; ++b) c *= (b == a) ? (long long)(n[b] + 1) : (long long)n[b];
  return c;
}

// index of face f along axis a for the cross-section coordinates of cell (i,j,k)
__device__ __forceinline__ long long face_index(const int n[3], int a, int i, int j, int k, int f) {
  if (a == 0) return (long long)f + (long long)(n[0] + 1) * ((long long)j + (long long)n[1] * k);
  if (a == 1) return (long long)i + (long long)n[0] * ((long long)f + (long long)(n[1] + 1) * k);
  return (long long)i + (long long)n[0] * ((long long)j + (long long)n[1] * f);
}

// Division of 32-bit unsigned numerators by a run-time invariant divisor d >= 1 with a multiply
// and shifts (Granlund and Montgomery, "Division by invariant integers using multiplication",
// PLDI 1994, Sect. 4): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) where t = umulhi(m, n).
struct FastDiv {
  unsigned d, m;
  int s1, s2;
};

__host__ inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ unsigned fast_div(unsigned n, const FastDiv& f) {
  const unsigned t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

__device__ __forceinline__ long long cell_index(const int n[3], int i, int j, int k) {
  return (long long)i + (long long)n[0] * ((long long)j + (long long)n[1] * k);
}

// Reciprocal and reciprocal square root for positive FP64 values, by Newton-Raphson refinement of
// an FP32 seed: x = m 2^k with m in [1, 2) (or [2, 4) for the square root, k even), the FP32
// intrinsic on m, one Newton step in FP64, and the power of two put back through the exponent
// field.  Relative error ~2^-47 (one step squares the seed's ~2^-24); about half the FP64
// instructions of the correctly rounded operations, which GB300 builds from the same pieces.
// Zero, subnormal, infinite or NaN input takes the IEEE operation (out of line, so that the
// compiler does not predicate it into every call).
static __device__ __noinline__ double rcp_ieee(double x) { return 1.0 / x; }
static __device__ __noinline__ double rsqrt_ieee(double x) { return 1.0 / sqrt(x); }

__device__ __forceinline__ double rcp_nr(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int ef = (hi >> 20) & 0x7ff;
  if (ef == 0 || ef == 0x7ff) return rcp_ieee(x);
  const double m = __hiloint2double((hi & 0x800fffff) | 0x3ff00000, lo);
  const double r0 = (double)__frcp_rn((float)m);
  const double r = fma(r0, fma(-m, r0, 1.0), r0);  // 1/m, in (0.5, 1]
  return __hiloint2double(__double2hiint(r) - ((ef - 1023) << 20), __double2loint(r));
}

__device__ __forceinline__ double rsqrt_nr(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int ef = (hi >> 20) & 0x7ff;
  if (ef == 0 || ef == 0x7ff || hi < 0) return rsqrt_ieee(x);
  const int k = ef - 1023, kk = k & ~1;  // x = m 2^kk, m in [1, 4)
  const double m = __hiloint2double((hi & 0x000fffff) | ((1023 + (k - kk)) << 20), lo);
  const double y0 = (double)__frsqrt_rn((float)m);
  const double y = y0 * fma(-0.5 * m * y0, y0, 1.5);  // 1/sqrt(m), in (0.5, 1]
  return __hiloint2double(__double2hiint(y) - ((kk / 2) << 20), __double2loint(y));
}

// sqrt(x) = x / sqrt(x) for x > 0, 0 for x == 0
__device__ __forceinline__ double sqrt_nr(double x) { return x > 0.0 ? x * rsqrt_nr(x) : 0.0; }

__device__ __forceinline__ double temperature(double gamma, double gas_R, double rho, double eps) {
  return (gamma - 1.0) * eps * rcp_nr(rho * gas_R);
}

// Opacity per cell: constant, Kramers-like power law, or bilinear table in (log10 rho,
// log10 T) on log10 kappa, clamped to the table edges.
__device__ inline double opacity(const Opacity& o, double rho, double T) {
  if (o.model == FLD_OPACITY_CONST) return o.kappa0;
  if (o.model == FLD_OPACITY_KRAMERS) {
    if (o.kr_a == 1.0 && o.kr_b == -3.5) {
      const double it = rcp_nr(T);
      return o.kappa0 * rho * (it * it * it) * sqrt_nr(it);  // rho T^-3.5
    }
    return o.kappa0 * pow(rho, o.kr_a) * pow(T, o.kr_b);
  }
  double u = (log10(rho) - o.tlo0) / (o.thi0 - o.tlo0) * (o.tn0 - 1);
  double v = (log10(T) - o.tlo1) / (o.thi1 - o.tlo1) * (o.tn1 - 1);
  u = fmin(fmax(u, 0.0), (double)(o.tn0 - 1));
  v = fmin(fmax(v, 0.0), (double)(o.tn1 - 1));
  int i = min((int)u, o.tn0 - 2), j = min((int)v, o.tn1 - 2);
  double fu = u - i, fv = v - j;
  const double* t = o.table + (long long)i * o.tn1 + j;
  double l = (1 - fu) * ((1 - fv) * __ldg(t) + fv * __ldg(t + 1)) +
             fu * ((1 - fv) * __ldg(t + o.tn1) + fv * __ldg(t + o.tn1 + 1));
  return exp10(l);
}

// Cell diffusion coefficient D = c lambda(R) / (kappa rho) with R = |grad E| / (kappa rho E)
// (Sect. 2.2, Eqs. fld_lambda and fld_F).  q = kappa rho, g2 = |grad E|^2, gm = |grad E|.  Each
// limiter is multiplied through by powers of q E so that one reciprocal and at most one square
// root remain:
//   LP       lambda = (2+R)/(6+3R+R^2)                 D = c E (2qE + g) / (qE (6qE + 3g) + g^2)
//   Minerbo  lambda = 2/(3+sqrt(9+12R^2)), R <= 3/2     D = 2 c E / (3qE + sqrt(9 (qE)^2 + 12 g^2))
//            lambda = 1/(1+R+sqrt(1+2R)),  R > 3/2      D = c E / (qE + g + sqrt(qE (qE + 2g)))
//   third    lambda = 1/3                              D = c / (3q)
__device__ __forceinline__ double limited_D(int limiter, double c, double q, double e, double g2, double gm) {
  const double qe = q * e;
  if (limiter == FLD_LIMITER_THIRD) return c * rcp_nr(3.0 * q);
  if (limiter == FLD_LIMITER_MINERBO) {
    if (gm <= 1.5 * qe) return 2.0 * c * e * rcp_nr(3.0 * qe + sqrt_nr(fma(9.0 * qe, qe, 12.0 * g2)));
    return c * e * rcp_nr(qe + gm + sqrt_nr(qe * (qe + 2.0 * gm)));
  }
  return c * e * (2.0 * qe + gm) * rcp_nr(qe * (6.0 * qe + 3.0 * gm) + g2);
}

}  // namespace fld

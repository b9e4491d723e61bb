// Per-cell FLD coefficient math shared by the single-grid and batched kernels (arXiv
// 2104.03968: Sect. 2.2 Eqs. fld_lambda and fld_F; Sect. 3.2 Eq. ileyk_flux; Sect. 3.4 faces).
#pragma once

#include <cmath>

#include "df.cuh"
#include "fld_common.cuh"

namespace fld {

struct CoeffPhys {
  Opacity op;
  double c, gamma, gas_R;
  int limiter;
};

// E at integer position p along axis a of cell (q0,q1,q2), with ghost cells outside [0, n_a):
// periodic wrap, Dirichlet ghost value, Neumann gradient across the boundary face, or linear
// extrapolation from the two interior cells ("continuous").
__device__ __forceinline__ double sample_E(const double* __restrict__ E, const GridDev& g, int q0, int q1,
                                           int q2, int a, int p) {
  int n = g.n[a];
  int q[3] = {q0, q1, q2};
  if (p >= 0 && p < n) {
    q[a] = p;
    return __ldg(E + cell_index(g.n, q[0], q[1], q[2]));
  }
  int side = p < 0 ? 0 : 1;
  int bc = g.bc[2 * a + side];
  double v = g.bc_val[2 * a + side];
  if (bc == FLD_BC_PERIODIC) {
    q[a] = ((p % n) + n) % n;
    return __ldg(E + cell_index(g.n, q[0], q[1], q[2]));
  }
  if (bc == FLD_BC_DIRICHLET) return v;
  if (bc == FLD_BC_NEUMANN) {
    int m = side ? p - n : -1 - p;
    q[a] = side ? n - 1 - m : m;
    double e = __ldg(E + cell_index(g.n, q[0], q[1], q[2]));
    return side ? e + (2 * m + 1) * v * g.dx[a] : e - (2 * m + 1) * v * g.dx[a];
  }
  // continuous
  q[a] = side ? n - 1 : 0;
  double e0 = __ldg(E + cell_index(g.n, q[0], q[1], q[2]));
  q[a] = side ? n - 2 : 1;
  double e1 = __ldg(E + cell_index(g.n, q[0], q[1], q[2]));
  int d = side ? p - (n - 1) : -p;
  return e0 + d * (e0 - e1);
}

// The two FP64 differences of the 5-point stencil of Eq. ileyk_flux along axis a at cell (i,j,k):
// d1 = E[p-2] - E[p+2] and d2 = E[p+1] - E[p-1], so that dE/dx = (d1 + 8 d2) / (12 dx).
__device__ __forceinline__ void grad_diffs(const GridDev& g, const double* __restrict__ E, long long idx, int i, int j,
                                           int k, int a, double& d1, double& d2) {
  const int p = a == 0 ? i : (a == 1 ? j : k);
  double em2, em1, ep1, ep2;
  if (p >= 2 && p < g.n[a] - 2) {
    const long long s = a == 0 ? 1 : (a == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
    em2 = __ldg(E + idx - 2 * s);
    em1 = __ldg(E + idx - s);
    ep1 = __ldg(E + idx + s);
    ep2 = __ldg(E + idx + 2 * s);
  } else {
    em2 = sample_E(E, g, i, j, k, a, p - 2);
    em1 = sample_E(E, g, i, j, k, a, p - 1);
    ep1 = sample_E(E, g, i, j, k, a, p + 1);
    ep2 = sample_E(E, g, i, j, k, a, p + 2);
  }
  d1 = em2 - ep2;
  d2 = ep1 - em1;
}

// Opacity and cell-centred D of one cell in FP64: kappa(rho, T), the 5-point gradient of E, R,
// lambda(R) and D = c lambda/(kappa rho).  Returns false (D = 0) for rho, kappa, E <= 0 or eps < 0.
__device__ __forceinline__ bool coeffs_cell(const GridDev& g, const CoeffPhys& ph, const double* __restrict__ E,
                                            const double* __restrict__ rho, const double* __restrict__ eps,
                                            long long idx, double& kap_out, double& D_out) {
  int i = (int)(idx % g.n[0]);
  long long r = idx / g.n[0];
  int j = (int)(r % g.n[1]);
  int k = (int)(r / g.n[1]);
  double e = __ldg(E + idx), rh = __ldg(rho + idx), ep = __ldg(eps + idx);
  double kap;
  if (ph.op.model == FLD_OPACITY_KRAMERS && ph.op.kr_a == 1.0 && ph.op.kr_b == -3.5) {
    // kappa = kappa0 rho T^-3.5 with 1/T = rho gas_R / ((gamma-1) eps): one reciprocal, one sqrt
    double it = rh * ph.gas_R * rcp_nr((ph.gamma - 1.0) * ep);
    double it2 = it * it;
    kap = ph.op.kappa0 * rh * it2 * it * sqrt_nr(it);
  } else {
    kap = opacity(ph.op, rh, temperature(ph.gamma, ph.gas_R, rh, ep));
  }
  kap_out = kap;
  if (!(gt_zero(e) && gt_zero(rh) && gt_zero(kap) && ge_zero(ep))) {
    D_out = 0.0;
    return false;
  }
  double g2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) break;
    double d1, d2;
    grad_diffs(g, E, idx, i, j, k, a, d1, d2);
    // 5-point 4th-order central difference (the 1/dx factor is applied with g2 below)
    double d = d1 * (1.0 / 12.0) + d2 * (2.0 / 3.0);
    g2 = fma(d * d, g.inv_dx2[a], g2);
  }
  const double q_ = kap * rh;  // kappa rho, the inverse mean free path
  const double D = limited_D(ph.limiter, ph.c, q_, e, g2, ph.limiter == FLD_LIMITER_THIRD ? 0.0 : sqrt_nr(g2));
  D_out = D;
  return true;
}

static __device__ __noinline__ bool coeffs_cell_f64(const GridDev& g, const CoeffPhys& ph, const double* E,
                                                   const double* rho, const double* eps, long long idx, double& kap,
                                                   double& D) {
  return coeffs_cell(g, ph, E, rho, eps, idx, kap, D);
}

// Constants of the double-float coefficient path, split on the host.
struct CoeffDf {
  dfl c, gm1, gas_R, kappa0;  // c, gamma - 1, gas_R, kappa0
  dfl ig[3];                  // 1 / (144 dx_a^2): |grad E|^2 = sum_a (d1 + 8 d2)^2 ig_a
  int kramers;                // 1: kappa0 rho T^-3.5; 0: constant kappa0
  int ok;                     // the opacity model is one of the two and every constant is in the window
};

__host__ inline CoeffDf make_coeff_df(const CoeffPhys& ph, const GridDev& g) {
  auto split = [](double v) {
    dfl x;
    x.hi = (float)v;
    x.lo = (float)(v - (double)x.hi);
    return x;
  };
  auto in = [](double v) { return v == 0.0 || (std::fabs(v) >= 0x1p-100 && std::fabs(v) < 0x1p125); };
  CoeffDf K{};
  K.c = split(ph.c);
  K.gm1 = split(ph.gamma - 1.0);
  K.gas_R = split(ph.gas_R);
  K.kappa0 = split(ph.op.kappa0);
  K.kramers = ph.op.model == FLD_OPACITY_KRAMERS;
  bool ok = (ph.op.model == FLD_OPACITY_CONST ||
             (ph.op.model == FLD_OPACITY_KRAMERS && ph.op.kr_a == 1.0 && ph.op.kr_b == -3.5)) &&
            ph.c > 0.0 && in(ph.c) && ph.op.kappa0 > 0.0 && in(ph.op.kappa0) &&
            (ph.op.model == FLD_OPACITY_CONST ||
             (ph.gamma > 1.0 && in(ph.gamma - 1.0) && ph.gas_R > 0.0 && in(ph.gas_R)));
  for (int a = 0; a < 3; ++a) {
    const double v = a < g.ndim ? g.inv_dx2[a] / 144.0 : 0.0;
    K.ig[a] = split(v);
    ok = ok && in(v);
  }
  K.ok = ok;
  return K;
}

// The same cell in double-float arithmetic (df.cuh) on the FP32 pipe, for constant or Kramers
// (a = 1, b = -3.5) opacity: the FP64 stencil differences d1 + 8 d2 are the only FP64 arithmetic
// besides the two final roundings.  Inputs must already be valid (E, rho, eps > 0).  Every product whose low
// part could leave the normal floats is checked against the double-float window (df_in); sums of
// positive terms need no check, since an underflowed term is negligible beside an in-window sum.
// Returns false, with the outputs unset, when a value leaves the window; the caller then takes the
// FP64 path.  Relative error a few 2^-47.
__device__ __forceinline__ bool coeffs_cell_df(const GridDev& g, const CoeffPhys& ph, const CoeffDf& K,
                                               const double* __restrict__ E, long long idx, int i, int j, int k,
                                               double e, double rh, double ep, double& kap_out, double& D_out) {
  bool ok, o2, o3;
  dfl Ed, R, EP;
  split_f64_try(e, Ed.hi, Ed.lo, ok);
  split_f64_try(rh, R.hi, R.lo, o2);
  split_f64_try(ep, EP.hi, EP.lo, o3);
  ok = ok && o2 && o3 && df_in(Ed) && df_in(R);
  dfl kap = K.kappa0;
  if (K.kramers) {
    // 1/T = rho gas_R / ((gamma-1) eps); kappa = kappa0 rho (1/T)^3 sqrt(1/T)
    const dfl den = df_mul(EP, K.gm1);
    ok = ok && df_in(den);
    const dfl rg = df_mul(R, K.gas_R);
    const dfl it = df_div(rg, den);
    const dfl it3 = df_mul(df_sqr(it), it);  // it^2 lies between it and it^3
    const dfl kr = df_mul(K.kappa0, R);
    const dfl krt = df_mul(kr, it3);
    kap = df_mul(krt, df_sqrt(it));
    ok = ok && df_in(rg) && df_in(it) && df_in(it3) && df_in(kr) && df_in(krt);
  }
  const dfl q = df_mul(kap, R);  // kappa rho
  ok = ok && df_in(kap) && df_in(q);
  dfl g2{0.0f, 0.0f};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) break;
    double d1, d2;
    grad_diffs(g, E, idx, i, j, k, a, d1, d2);
    dfl d;
    split_f64_try(fma(8.0, d2, d1), d.hi, d.lo, o2);  // 12 dx dE/dx
    ok = ok && o2 && (d.hi == 0.0f || df_in(d));
    g2 = df_add_pos(g2, df_mul(df_sqr(d), K.ig[a]));
  }
  ok = ok && (g2.hi == 0.0f || df_in(g2));
  const dfl qe = df_mul(q, Ed);
  ok = ok && df_in(qe);
  dfl D;
  if (ph.limiter == FLD_LIMITER_THIRD) {
    D = df_div(K.c, df_mul_f(q, 3.0f));
  } else {
    const dfl gm = g2.hi == 0.0f ? dfl{0.0f, 0.0f} : df_sqrt(g2);
    const dfl ce = df_mul(K.c, Ed);
    ok = ok && df_in(ce);
    if (ph.limiter == FLD_LIMITER_MINERBO) {
      if (gm.hi <= 1.5f * qe.hi) {
        // 2 c E / (3 qE + sqrt(9 (qE)^2 + 12 g^2))
        const dfl t = df_add_pos(df_mul_f(df_sqr(qe), 9.0f), df_mul_f(g2, 12.0f));
        ok = ok && df_in(t);
        const dfl s = df_sqrt(t);
        D = df_div(df_scale(ce, 2.0f), df_add_pos(df_mul_f(qe, 3.0f), s));
      } else {
        // c E / (qE + g + sqrt(qE (qE + 2 g)))
        const dfl t = df_mul(qe, df_add_pos(qe, df_scale(gm, 2.0f)));
        ok = ok && df_in(t);
        const dfl s = df_sqrt(t);
        D = df_div(ce, df_add_pos(df_add_pos(qe, gm), s));
      }
    } else {
      // Levermore-Pomraning: c E (2 qE + g) / (qE (6 qE + 3 g) + g^2)
      const dfl num = df_mul(ce, df_add_pos(df_scale(qe, 2.0f), gm));
      const dfl den = df_add_pos(df_mul(qe, df_add_pos(df_mul_f(qe, 6.0f), df_mul_f(gm, 3.0f))), g2);
      ok = ok && df_in(num) && df_in(den);
      D = df_div(num, den);
    }
  }
  ok = ok && df_in(D);
  if (!ok) return false;
  kap_out = df_to_f64(kap);
  D_out = df_to_f64(D);
  return true;
}

// Either path for one cell: the double-float one when its constants allow, else (or when a value
// leaves its window) FP64.  Returns false (D = 0) for invalid input, as coeffs_cell.
// (i, j, k) are the cell's coordinates, idx its index.
__device__ __forceinline__ bool coeffs_cell_fast(const GridDev& g, const CoeffPhys& ph, const CoeffDf& K,
                                                 const double* __restrict__ E, const double* __restrict__ rho,
                                                 const double* __restrict__ eps, long long idx, int i, int j, int k,
                                                 double& kap, double& D) {
  if (K.ok) {
    const double e = __ldg(E + idx), rh = __ldg(rho + idx), ep = __ldg(eps + idx);
    if (gt_zero(e) && gt_zero(rh) && gt_zero(ep) && coeffs_cell_df(g, ph, K, E, idx, i, j, k, e, rh, ep, kap, D))
      return true;
  }
  return coeffs_cell_f64(g, ph, E, rho, eps, idx, kap, D);
}

// One thread per cell writes the lower face of each axis (face q_a), and the face n_a when it
// owns it: the cell at q_a = 0 on a periodic axis (face n_a is face 0 again), the cell at
// q_a = n_a - 1 otherwise (boundary face: ghost D = interior D).  The three harmonic means
// 2 D_c D_nb / (D_c + D_nb) share one reciprocal: 1/(s0 s1 s2), then 1/s_a is the product of the
// other two sums times it.
// With lo arrays (l0..l2 non-null, TW = float) the FP32 copy is the truncated leading part of the
// FP64 weight and lo receives the remainder, so that t + l carries the weight to ~2^-47.
// D[a] is the cell-centred diffusion coefficient of axis a: the same array three times for the
// scalar D of the paper, three arrays for a diagonal-tensor D.
template <class TW>
__device__ __forceinline__ void faces_cell_at(const GridDev& g, double dt, const double* const (&D)[3], const int (&q)[3],
                                              long long idx, double* __restrict__ w0, double* __restrict__ w1,
                                              double* __restrict__ w2, TW* __restrict__ t0, TW* __restrict__ t1,
                                              TW* __restrict__ t2, float* __restrict__ l0 = nullptr,
                                              float* __restrict__ l1 = nullptr, float* __restrict__ l2 = nullptr) {
  double Dc[3] = {0.0, 0.0, 0.0};
  double num[3] = {0, 0, 0}, den[3] = {1, 1, 1};
  bool pair[3] = {false, false, false};
  long long stride = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < g.ndim) {
      int p = q[a];
      Dc[a] = (a == 0 || D[a] != D[0]) ? __ldg(D[a] + idx) : Dc[0];
      if (p > 0 || g.bc[2 * a] == FLD_BC_PERIODIC) {
        double Dn = __ldg(D[a] + (p > 0 ? idx - stride : idx + (long long)(g.n[a] - 1) * stride));
        num[a] = 2.0 * Dc[a] * Dn;
        den[a] = Dc[a] + Dn;
        pair[a] = true;
      } else {
        num[a] = Dc[a];
      }
    }
    stride *= g.n[a];
  }
  const double inv = rcp_nr(den[0] * den[1] * den[2]);
  const double rd[3] = {den[1] * den[2] * inv, den[0] * den[2] * inv, den[0] * den[1] * inv};
  double* W[3] = {w0, w1, w2};
  TW* Tt[3] = {t0, t1, t2};
  float* Lo[3] = {l0, l1, l2};
  auto put = [&](int a, long long f, double w) {
    W[a][f] = w;
    if (Lo[a]) {
      float h, l;
      split_f64(w, h, l);
      Tt[a][f] = (TW)h;
      Lo[a][f] = l;
    } else if (Tt[a]) {
      Tt[a][f] = (TW)w;
    }
  };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) break;
    const double s = dt * g.inv_dx2[a];
    const double w = s * (pair[a] ? num[a] * rd[a] : num[a]);
    put(a, face_index(g.n, a, q[0], q[1], q[2], q[a]), w);
    const bool periodic = g.bc[2 * a + 1] == FLD_BC_PERIODIC;
    if ((periodic && q[a] == 0) || (!periodic && q[a] == g.n[a] - 1)) {
      const double wu = periodic ? w : s * Dc[a];
      put(a, face_index(g.n, a, q[0], q[1], q[2], g.n[a]), wu);
    }
  }
}

template <class TW>
__device__ __forceinline__ void faces_cell(const GridDev& g, double dt, const double* const (&D)[3], long long idx,
                                           double* __restrict__ w0, double* __restrict__ w1, double* __restrict__ w2,
                                           TW* __restrict__ t0, TW* __restrict__ t1, TW* __restrict__ t2,
                                           float* __restrict__ l0 = nullptr, float* __restrict__ l1 = nullptr,
                                           float* __restrict__ l2 = nullptr) {
  int q[3];
  q[0] = (int)(idx % g.n[0]);
  long long r = idx / g.n[0];
  q[1] = (int)(r % g.n[1]);
  q[2] = (int)(r / g.n[1]);
  faces_cell_at<TW>(g, dt, D, q, idx, w0, w1, w2, t0, t1, t2, l0, l1, l2);
}

}  // namespace fld

// Per-cell FLD coefficient math shared by the single-grid and batched kernels (arXiv
// 2104.03968: Sect. 2.2 Eqs. fld_lambda and fld_F; Sect. 3.2 Eq. ileyk_flux; Sect. 3.4 faces).
#pragma once

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

// Opacity and cell-centred D of one cell: kappa(rho, T), the 5-point gradient of E, R,
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
  int q[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) break;
    int p = q[a];
    double em2, em1, ep1, ep2;
    if (p >= 2 && p < g.n[a] - 2) {
      long long s = a == 0 ? 1 : (a == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
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
    // 5-point 4th-order central difference (the 1/dx factor is applied with g2 below)
    double d = (em2 - ep2) * (1.0 / 12.0) + (ep1 - em1) * (2.0 / 3.0);
    g2 = fma(d * d, g.inv_dx2[a], g2);
  }
  const double q_ = kap * rh;  // kappa rho, the inverse mean free path
  const double D = limited_D(ph.limiter, ph.c, q_, e, g2, ph.limiter == FLD_LIMITER_THIRD ? 0.0 : sqrt_nr(g2));
  D_out = D;
  return true;
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

}  // namespace fld

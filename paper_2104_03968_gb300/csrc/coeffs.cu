// FLD coefficients on the device: opacity, 4th-order gradient of E, ratio R, Levermore-
// Pomraning limiter and the cell-centred diffusion coefficient D (arXiv 2104.03968,
// Sect. 2.2 Eqs. fld_lambda and fld_F; Sect. 3.2 Eq. ileyk_flux), and the dt-scaled
// harmonic-mean face weights of the implicit operator (Sect. 3.4).
//
// FP64 throughout: D enters the operator whose residual is checked in FP64.
#include "fld_common.cuh"
#include "kernels.h"
#include "trace.h"

namespace fld {

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

__global__ void k_coeffs(GridDev g, Opacity op, double c, double gamma, double gas_R, int limiter,
                         const double* __restrict__ E, const double* __restrict__ rho,
                         const double* __restrict__ eps, double* __restrict__ kappa_out,
                         double* __restrict__ D_out, unsigned* __restrict__ status) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  int i = (int)(idx % g.n[0]);
  long long r = idx / g.n[0];
  int j = (int)(r % g.n[1]);
  int k = (int)(r / g.n[1]);
  double e = __ldg(E + idx), rh = __ldg(rho + idx), ep = __ldg(eps + idx);
  double T = temperature(gamma, gas_R, rh, ep);
  double kap = opacity(op, rh, T);
  if (!(e > 0.0) || !(rh > 0.0) || !(kap > 0.0) || !(ep >= 0.0)) {
    atomicOr(status, kStatNonpositive);
    if (kappa_out) kappa_out[idx] = kap;
    D_out[idx] = 0.0;
    return;
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
    // 5-point 4th-order central difference
    double d = ((em2 - ep2) * (1.0 / 12.0) + (ep1 - em1) * (2.0 / 3.0)) / g.dx[a];
    g2 += d * d;
  }
  double gm = sqrt(g2);
  double q_ = kap * rh;  // kappa rho, the inverse mean free path
  double D;
  if (limiter == FLD_LIMITER_THIRD) {
    D = c / (3.0 * q_);
  } else {
    // c lambda/(kappa rho) with lambda = (2+R)/(6+3R+R^2), R = |grad E|/(kappa rho E),
    // multiplied through by (kappa rho E)^2 so that one division remains
    double qe = q_ * e;
    D = c * e * (2.0 * qe + gm) / (qe * (6.0 * qe + 3.0 * gm) + gm * gm);
  }
  if (kappa_out) kappa_out[idx] = kap;
  D_out[idx] = D;
}

// dt-scaled face weights w = dt * Dface / dx^2 along axis a; Dface is the harmonic mean of the
// two cells (periodic faces wrap), a non-periodic boundary face takes its interior cell's D.
template <class TW>
__global__ void k_faces(GridDev g, int a, double dt, const double* __restrict__ D, double* __restrict__ w64,
                        TW* __restrict__ wT) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[a] += 1;
  long long total = (long long)m[0] * m[1] * m[2];
  if (idx >= total) return;
  int q[3];
  q[0] = (int)(idx % m[0]);
  long long r = idx / m[0];
  q[1] = (int)(r % m[1]);
  q[2] = (int)(r / m[1]);
  int f = q[a];
  int n = g.n[a];
  double s = dt / (g.dx[a] * g.dx[a]);
  double w;
  int lo[3] = {q[0], q[1], q[2]}, hi[3] = {q[0], q[1], q[2]};
  if (f > 0 && f < n) {
    lo[a] = f - 1;
    hi[a] = f;
    double d0 = __ldg(D + cell_index(g.n, lo[0], lo[1], lo[2]));
    double d1 = __ldg(D + cell_index(g.n, hi[0], hi[1], hi[2]));
    w = s * 2.0 * d0 * d1 / (d0 + d1);
  } else if (g.bc[2 * a + (f == n)] == FLD_BC_PERIODIC) {
    lo[a] = n - 1;
    hi[a] = 0;
    double d0 = __ldg(D + cell_index(g.n, lo[0], lo[1], lo[2]));
    double d1 = __ldg(D + cell_index(g.n, hi[0], hi[1], hi[2]));
    w = s * 2.0 * d0 * d1 / (d0 + d1);
  } else {
    lo[a] = f == n ? n - 1 : 0;
    w = s * __ldg(D + cell_index(g.n, lo[0], lo[1], lo[2]));
  }
  w64[idx] = w;
  if (wT) wT[idx] = (TW)w;
}

static inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

cudaError_t launch_coeffs(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                          int limiter, const double* E, const double* rho, const double* eps,
                          double* kappa_out, double* D_out, unsigned* status, cudaStream_t s) {
  if (g.ncell == 0) return cudaSuccess;
  TraceScope ts("coeffs", s);
  k_coeffs<<<blocks_for(g.ncell), kBlock, 0, s>>>(g, op, c, gamma, gas_R, limiter, E, rho, eps, kappa_out,
                                                  D_out, status);
  return cudaGetLastError();
}

cudaError_t launch_faces(const GridDev& g, double dt, const double* D, double* const w64[3], float* const w32[3],
                         cudaStream_t s) {
  TraceScope ts("faces", s);
  for (int a = 0; a < g.ndim; ++a) {
    long long total = face_count(g.n, a);
    if (w32 && w32[a])
      k_faces<float><<<blocks_for(total), kBlock, 0, s>>>(g, a, dt, D, w64[a], w32[a]);
    else
      k_faces<double><<<blocks_for(total), kBlock, 0, s>>>(g, a, dt, D, w64[a], nullptr);
  }
  return cudaGetLastError();
}

}  // namespace fld

// Explicit radiation terms of the FLD closure (arXiv 2104.03968, Sect. 2.1-2.2 and 3.2): the
// flux F = -D grad E (Eq. fld_F), the radiation force density f_r = rho kappa F / c (Eq.
// rhd_force) and its work v . f_r, the Eddington factor f = lambda + lambda^2 R^2 (Eq.
// fld_Edd_fac), the pressure tensor P = E [(1-f)/2 I + (3f-1)/2 n n] (Eq. fld_Edd, n = grad E /
// |grad E|) and the photon-tiring term P : grad v, with every gradient by the 5-point stencil of
// Eq. ileyk_flux.  Velocity ghosts on non-periodic faces: linear extrapolation.  Optionally the
// pseudo-planar geometric source of E (Appendix A) on a grid whose x axis stands for the radius:
// -2 (E v_x + F_x) / x + 2 v_x P_xx / x at the cell centre's radius x.  FP64; one thread per cell
// (these terms are evaluated once per step and are FP64-pipe bound like k_coeffs).
#include "coeffs.cuh"
#include "kernels.h"
#include "trace.h"

namespace fld {

struct SourceOut {
  double* F[3];
  double* fr[3];
  double* work;
  double* fedd;
  double* P[6];  // xx yy zz xy xz yz
  double* tiring;
  double* sg;  // pseudo-planar source of E
  double x0;   // radius of the grid's lower x face (for sg)
};

struct VelIn {
  const double* v[3];
};

// velocity component at position p along axis a: periodic wrap, else linear extrapolation
__device__ __forceinline__ double sample_v(const double* __restrict__ f, const GridDev& g, int q0, int q1, int q2, int a,
                                           int p) {
  const int n = g.n[a];
  int q[3] = {q0, q1, q2};
  if (p >= 0 && p < n) {
    q[a] = p;
    return __ldg(f + cell_index(g.n, q[0], q[1], q[2]));
  }
  const int side = p < 0 ? 0 : 1;
  if (g.bc[2 * a + side] == FLD_BC_PERIODIC) {
    q[a] = ((p % n) + n) % n;
    return __ldg(f + cell_index(g.n, q[0], q[1], q[2]));
  }
  q[a] = side ? n - 1 : 0;
  const double f0 = __ldg(f + cell_index(g.n, q[0], q[1], q[2]));
  q[a] = side ? n - 2 : 1;
  const double f1 = __ldg(f + cell_index(g.n, q[0], q[1], q[2]));
  const int d = side ? p - (n - 1) : -p;
  return f0 + d * (f0 - f1);
}

__device__ __forceinline__ double five_point(double fm2, double fm1, double fp1, double fp2, double inv_dx) {
  return ((fm2 - fp2) * (1.0 / 12.0) + (fp1 - fm1) * (2.0 / 3.0)) * inv_dx;
}

__global__ void k_radiation_terms(GridDev g, CoeffPhys ph, const double* __restrict__ E, const double* __restrict__ rho,
                                  const double* __restrict__ eps, VelIn V, SourceOut O, unsigned* __restrict__ status) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  const int i = (int)(idx % g.n[0]);
  const long long r = idx / g.n[0];
  const int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
  const int q[3] = {i, j, k};
  const double e = E[idx], rh = rho[idx];
  const double kap = opacity(ph.op, rh, temperature(ph.gamma, ph.gas_R, rh, eps[idx]));
  if (!(gt_zero(e) && gt_zero(rh) && gt_zero(kap) && ge_zero(eps[idx]))) {
    atomicOr(status, kStatNonpositive);
    return;
  }
  double gE[3] = {0.0, 0.0, 0.0}, g2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) break;
    const int p = q[a];
    gE[a] = five_point(sample_E(E, g, i, j, k, a, p - 2), sample_E(E, g, i, j, k, a, p - 1),
                       sample_E(E, g, i, j, k, a, p + 1), sample_E(E, g, i, j, k, a, p + 2), 1.0 / g.dx[a]);
    g2 = fma(gE[a], gE[a], g2);
  }
  const double gm = sqrt(g2);
  const double qk = kap * rh;
  const double D = limited_D(ph.limiter, ph.c, qk, e, g2, gm);
  const double lam = D * qk / ph.c;
  const double R = gm / (qk * e);
  const double f = lam + lam * lam * R * R;
  const double inv_gm = gm > 0.0 ? 1.0 / gm : 0.0;
  double w = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) break;
    const double Fa = -D * gE[a];
    const double fa = qk * Fa / ph.c;
    if (O.F[a]) O.F[a][idx] = Fa;
    if (O.fr[a]) O.fr[a][idx] = fa;
    if (V.v[0]) w = fma(V.v[a][idx], fa, w);
  }
  if (O.work) O.work[idx] = w;
  if (O.fedd) O.fedd[idx] = f;
  const double iso = 0.5 * (1.0 - f) * e, ani = 0.5 * (3.0 * f - 1.0) * e;
  const double n[3] = {gE[0] * inv_gm, gE[1] * inv_gm, gE[2] * inv_gm};
  double P[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) P[a][b] = (a == b ? iso : 0.0) + ani * n[a] * n[b];
  if (O.P[0]) {
    O.P[0][idx] = P[0][0];
    O.P[1][idx] = P[1][1];
    O.P[2][idx] = P[2][2];
    O.P[3][idx] = P[0][1];
    O.P[4][idx] = P[0][2];
    O.P[5][idx] = P[1][2];
  }
  if (O.sg) {
    const double x = O.x0 + (i + 0.5) * g.dx[0];
    const double vx = V.v[0] ? V.v[0][idx] : 0.0;
    O.sg[idx] = (-2.0 * fma(e, vx, -D * gE[0]) + 2.0 * vx * P[0][0]) / x;
  }
  if (O.tiring) {
    double t = 0.0;
    if (V.v[0]) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.ndim) break;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (b >= g.ndim) break;
          const int p = q[b];
          const double dv = five_point(sample_v(V.v[a], g, i, j, k, b, p - 2), sample_v(V.v[a], g, i, j, k, b, p - 1),
                                       sample_v(V.v[a], g, i, j, k, b, p + 1), sample_v(V.v[a], g, i, j, k, b, p + 2),
                                       1.0 / g.dx[b]);
          t = fma(P[a][b], dv, t);
        }
      }
    }
    O.tiring[idx] = t;
  }
}

// E <- E + a * S: the explicit addition of a source over a step (Sect. 3.2: a = -dt with
// S = P : grad v; Appendix A: a = dt with the pseudo-planar source)
__global__ void k_explicit_update(long long n, double a, const double* __restrict__ S, double* __restrict__ E,
                                  unsigned* __restrict__ status) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const double v = fma(a, S[idx], E[idx]);
  if (!(v > 0.0)) atomicOr(status, kStatNonpositive);
  E[idx] = v;
}

cudaError_t launch_radiation_terms(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                                   int limiter, const double* E, const double* rho, const double* eps,
                                   const double* const v[3], double* const F[3], double* const fr[3], double* work,
                                   double* fedd, double* const P[6], double* tiring, double* sg, double x0,
                                   unsigned* status, cudaStream_t s) {
  if (g.ncell == 0) return cudaSuccess;
  TraceScope ts("radiation_terms", s);
  CoeffPhys ph{op, c, gamma, gas_R, limiter};
  VelIn V{};
  SourceOut O{};
  for (int a = 0; a < 3; ++a) {
    V.v[a] = v ? v[a] : nullptr;
    O.F[a] = F ? F[a] : nullptr;
    O.fr[a] = fr ? fr[a] : nullptr;
  }
  for (int m = 0; m < 6; ++m) O.P[m] = P ? P[m] : nullptr;
  O.work = work;
  O.fedd = fedd;
  O.tiring = tiring;
  O.sg = sg;
  O.x0 = x0;
  note_launch(),
      k_radiation_terms<<<(unsigned)((g.ncell + kBlock - 1) / kBlock), kBlock, 0, s>>>(g, ph, E, rho, eps, V, O, status);
  return cudaGetLastError();
}

cudaError_t launch_explicit_update(long long n, double a, const double* S, double* E, unsigned* status,
                                   cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  TraceScope ts("explicit_update", s);
  note_launch(), k_explicit_update<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, a, S, E, status);
  return cudaGetLastError();
}

}  // namespace fld

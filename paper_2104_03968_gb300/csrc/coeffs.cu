// FLD coefficients on the device: opacity, 4th-order gradient of E, ratio R, Levermore-
// Pomraning limiter and the cell-centred diffusion coefficient D (arXiv 2104.03968,
// Sect. 2.2 Eqs. fld_lambda and fld_F; Sect. 3.2 Eq. ileyk_flux), and the dt-scaled
// harmonic-mean face weights of the implicit operator (Sect. 3.4).  The per-cell math is in
// coeffs.cuh.
//
// FP64 throughout: D enters the operator whose residual is checked in FP64.
#include "coeffs.cuh"
#include "dfmath.cuh"
#include "kernels.h"
#include "trace.h"

namespace fld {

// One thread per cell; the coordinates come from 32-bit divisions by invariant divisors (the
// launcher takes the 64-bit kernel beyond 2^32 cells).
// The structures are __grid_constant__ so that the out-of-line FP64 fallback can take their
// address without a per-thread local copy; six blocks of 256 per SM (40 registers), as the
// double-float chains are latency-bound (measured 7 % faster than five).
__global__ void __launch_bounds__(kBlock, 6)
    k_coeffs(const __grid_constant__ GridDev g, const __grid_constant__ CoeffPhys ph, CoeffDf K, FastDiv f0,
             FastDiv f1, unsigned first, unsigned end, const double* __restrict__ E, const double* __restrict__ rho,
             const double* __restrict__ eps, double* __restrict__ kappa_out, double* __restrict__ D_out,
             unsigned* __restrict__ status) {
  const unsigned idx = first + blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= end) return;
  const unsigned r = fast_div(idx, f0), k = fast_div(r, f1);
  const int i = (int)(idx - r * f0.d), j = (int)(r - k * f1.d);
  double kap, D;
  if (!coeffs_cell_fast(g, ph, K, E, rho, eps, idx, i, j, (int)k, kap, D)) atomicOr(status, kStatNonpositive);
  if (kappa_out) kappa_out[idx] = kap;
  D_out[idx] = D;
}

__global__ void k_coeffs64(const __grid_constant__ GridDev g, const __grid_constant__ CoeffPhys ph, CoeffDf K,
                           long long first, long long end, const double* __restrict__ E,
                           const double* __restrict__ rho, const double* __restrict__ eps,
                           double* __restrict__ kappa_out, double* __restrict__ D_out, unsigned* __restrict__ status) {
  const long long idx = first + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= end) return;
  const long long r = idx / g.n[0];
  double kap, D;
  if (!coeffs_cell_fast(g, ph, K, E, rho, eps, idx, (int)(idx % g.n[0]), (int)(r % g.n[1]), (int)(r / g.n[1]), kap,
                        D))
    atomicOr(status, kStatNonpositive);
  if (kappa_out) kappa_out[idx] = kap;
  D_out[idx] = D;
}

struct DAxes {
  const double* d[3];
};

template <class TW>
__global__ void k_faces(GridDev g, double dt, DAxes D, double* __restrict__ w0,
                        double* __restrict__ w1, double* __restrict__ w2, TW* __restrict__ t0, TW* __restrict__ t1,
                        TW* __restrict__ t2, float* __restrict__ l0, float* __restrict__ l1, float* __restrict__ l2) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  faces_cell<TW>(g, dt, D.d, idx, w0, w1, w2, t0, t1, t2, l0, l1, l2);
}

static inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <bool MIXED>
__global__ void k_opacity(long long n, const __grid_constant__ Opacity op, double gamma, double gas_R,
                          const double* __restrict__ rho, const double* __restrict__ eps, double* __restrict__ kappa) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double rh = rho[i], T = temperature(gamma, gas_R, rh, eps[i]);
  kappa[i] = (MIXED && op.model == FLD_OPACITY_TABLE) ? opacity_table_df(op, rh, T) : opacity(op, rh, T);
}

cudaError_t launch_opacity(long long n, const Opacity& op, double gamma, double gas_R, bool mixed, const double* rho,
                           const double* eps, double* kappa, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  if (mixed) k_opacity<true><<<blocks_for(n), kBlock, 0, s>>>(n, op, gamma, gas_R, rho, eps, kappa);
  else k_opacity<false><<<blocks_for(n), kBlock, 0, s>>>(n, op, gamma, gas_R, rho, eps, kappa);
  return cudaGetLastError();
}

cudaError_t launch_coeffs_range(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                                int limiter, const double* E, const double* rho, const double* eps, double* kappa_out,
                                double* D_out, unsigned* status, long long first, long long count, cudaStream_t s,
                                bool plain64) {
  if (count <= 0) return cudaSuccess;
  TraceScope ts("coeffs", s);
  CoeffPhys ph{op, c, gamma, gas_R, limiter};
  CoeffDf K = make_coeff_df(ph, g);
  if (plain64) K.ok = 0;  // every cell takes the FP64 formula
  if (g.ncell < (1ll << 32) - kBlock)
    note_launch(),
        k_coeffs<<<blocks_for(count), kBlock, 0, s>>>(g, ph, K, make_fastdiv((unsigned)g.n[0]),
                                                       make_fastdiv((unsigned)g.n[1]), (unsigned)first,
                                                       (unsigned)(first + count), E, rho, eps, kappa_out, D_out, status);
  else
    note_launch(),
        k_coeffs64<<<blocks_for(count), kBlock, 0, s>>>(g, ph, K, first, first + count, E, rho, eps, kappa_out, D_out,
                                                         status);
  return cudaGetLastError();
}

cudaError_t launch_coeffs(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                          int limiter, const double* E, const double* rho, const double* eps,
                          double* kappa_out, double* D_out, unsigned* status, cudaStream_t s, bool plain64) {
  if (g.ncell == 0) return cudaSuccess;
  return launch_coeffs_range(g, op, c, gamma, gas_R, limiter, E, rho, eps, kappa_out, D_out, status, 0, g.ncell, s,
                             plain64);
}

cudaError_t launch_faces(const GridDev& g, double dt, const double* const Dax[3], double* const w64[3],
                         float* const w32[3], float* const w32lo[3], cudaStream_t s) {
  TraceScope ts("faces", s);
  const DAxes D{{Dax[0], Dax[1], Dax[2]}};
  if (w32 && w32[0])
    note_launch(),
        k_faces<float><<<blocks_for(g.ncell), kBlock, 0, s>>>(g, dt, D, w64[0], w64[1], w64[2], w32[0], w32[1], w32[2],
                                                               w32lo ? w32lo[0] : nullptr, w32lo ? w32lo[1] : nullptr,
                                                               w32lo ? w32lo[2] : nullptr);
  else
    note_launch(),
        k_faces<double><<<blocks_for(g.ncell), kBlock, 0, s>>>(g, dt, D, w64[0], w64[1], w64[2], nullptr, nullptr,
                                                                nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace fld

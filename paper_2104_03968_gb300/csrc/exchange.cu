// Point-implicit gas-radiation energy exchange over independent cells (arXiv 2104.03968,
// Sect. 3.3); the per-cell solve is in exchange.cuh.
#include "exchange.cuh"
#include "kernels.h"
#include "trace.h"

namespace fld {

// p is __grid_constant__ so that the out-of-line FP64 fallback can take its address without a
// per-thread local copy; six blocks of 256 per SM (40 registers), as the double-float chains are
// latency-bound (measured 4 % faster than five).
__global__ void __launch_bounds__(kBlock, 6)
    k_exchange(long long n, const __grid_constant__ ExchangeParams p, Opacity op, const double* __restrict__ rho,
               const double* __restrict__ kappa_in, double* __restrict__ eps, double* __restrict__ E,
               int* __restrict__ info_iters, int* __restrict__ info_bisect, unsigned* __restrict__ status) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int iters = 0, bis = 0;
  if (idx < n) {
    double r = rho[idx], e = eps[idx], En = E[idx];
    double k = kappa_in ? kappa_in[idx] : opacity(op, r, temperature(p.gamma, p.gas_R, r, e));
    if (exchange_cell_fast(p, r, k, e, En, iters, bis)) {
      eps[idx] = e;
      E[idx] = En;
    } else {
      atomicOr(status, kStatNonpositive);
    }
  }
  exchange_report(iters, bis, info_iters, info_bisect);
}

cudaError_t launch_exchange(long long n, const ExchangeParams& p, const Opacity& op, const double* rho,
                            const double* kappa, double* eps, double* E, int* info_iters, int* info_bisect,
                            unsigned* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  unsigned blocks = (unsigned)((n + kBlock - 1) / kBlock);
  TraceScope ts("exchange", s);
  note_launch(), k_exchange<<<blocks, kBlock, 0, s>>>(n, p, op, rho, kappa, eps, E, info_iters, info_bisect, status);
  return cudaGetLastError();
}

// Midpoint IMEX recombination (Sect. 3.1): E = E0 + 2 (E_mid - E_half), eps = eps0 -- the state
// u^n plus dt times the implicit (diffusion) increment of the half step.
__global__ void k_midpoint_combine(long long n, const double* __restrict__ E0, const double* __restrict__ eps0,
                                   const double* __restrict__ Eh, double* __restrict__ E, double* __restrict__ eps) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  E[idx] = fma(2.0, E[idx] - Eh[idx], E0[idx]);
  eps[idx] = eps0[idx];
}

cudaError_t launch_midpoint_combine(long long n, const double* E0, const double* eps0, const double* Eh, double* E,
                                    double* eps, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  TraceScope ts("midpoint_combine", s);
  note_launch(), k_midpoint_combine<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, E0, eps0, Eh, E, eps);
  return cudaGetLastError();
}

}  // namespace fld

// Internal launcher declarations of the GB300 FLD library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "fld_common.cuh"

namespace fld {

// plain64: the FP64 formula in every cell (the FP64 solver); else double-float with FP64 fallback
cudaError_t launch_coeffs(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                          int limiter, const double* E, const double* rho, const double* eps,
                          double* kappa_out, double* D_out, unsigned* status, cudaStream_t s, bool plain64 = false);
// the same for cells [first, first + count) only (the whole grid is the stencil's domain)
cudaError_t launch_coeffs_range(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                                int limiter, const double* E, const double* rho, const double* eps, double* kappa_out,
                                double* D_out, unsigned* status, long long first, long long count, cudaStream_t s,
                                bool plain64 = false);

// kappa per cell from rho and eps (gas law for T); mixed: the table model's logarithms and power
// of ten in double-float (dfmath.cuh), else opacity() in FP64
cudaError_t launch_opacity(long long n, const Opacity& op, double gamma, double gas_R, bool mixed, const double* rho,
                           const double* eps, double* kappa, cudaStream_t s);

// w64[a] (and w32[a] when non-null) receive the face weights of axis a (layout of fld_common.cuh);
// with w32lo, w32 holds the truncated leading 24 bits of each weight and w32lo the remainder.
// Dax[a]: cell-centred D of axis a (the same pointer three times for a scalar D).
cudaError_t launch_faces(const GridDev& g, double dt, const double* const Dax[3], double* const w64[3],
                         float* const w32[3], float* const w32lo[3], cudaStream_t s);

// E = E0 + 2 (E - Eh), eps = eps0 (midpoint IMEX recombination)
cudaError_t launch_midpoint_combine(long long n, const double* E0, const double* eps0, const double* Eh, double* E,
                                    double* eps, cudaStream_t s);

// explicit radiation terms (sources.cu); null output pointers are skipped; sg = the pseudo-planar
// source of E with x0 the radius of the grid's lower x face
cudaError_t launch_radiation_terms(const GridDev& g, const Opacity& op, double c, double gamma, double gas_R,
                                   int limiter, const double* E, const double* rho, const double* eps,
                                   const double* const v[3], double* const F[3], double* const fr[3], double* work,
                                   double* fedd, double* const P[6], double* tiring, double* sg, double x0,
                                   unsigned* status, cudaStream_t s);
// E += a * S
cudaError_t launch_explicit_update(long long n, double a, const double* S, double* E, unsigned* status,
                                   cudaStream_t s);

cudaError_t launch_exchange(long long n, const ExchangeParams& p, const Opacity& op, const double* rho,
                            const double* kappa, double* eps, double* E, int* info_iters, int* info_bisect,
                            unsigned* status, cudaStream_t s);

}  // namespace fld

// Batched 1-D radial columns: fused coefficients + tridiagonal diffusion + exchange.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "fld_common.cuh"

namespace fld {

constexpr int kColumnMaxCells = 2048;

// CAK parameters (NULL is valid: no CAK term)
bool cak_valid(const fld_cak* c);
fld_status columns_validate(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo, int bc_hi,
                            const double* v_lo, const double* v_hi, const double* dt, std::string* err);

// geom: device scratch of at least 4*ncell + 4 doubles (per-cell geometry factors)
cudaError_t launch_columns_step(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo, int bc_hi,
                                const double* v_lo, const double* v_hi, const fld_params& p, const double* dt,
                                const double* rho, double* eps, double* E, double* geom, int* info_iters,
                                int* info_bisect, unsigned* status, cudaStream_t s);

cudaError_t launch_columns_diffuse(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo, int bc_hi,
                                   const double* v_lo, const double* v_hi, const fld_params& p, const double* dt,
                                   const double* D_cell, const double* E_old, double* E_new, double* geom,
                                   cudaStream_t s);

}  // namespace fld

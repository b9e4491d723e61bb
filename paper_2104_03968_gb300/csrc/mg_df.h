// Double-float setup kernels of the mixed multigrid solver (mg_df.cu).
#pragma once

#include <cuda_runtime.h>

#include "fld_common.cuh"
#include "mg.h"

namespace fld {

// per-call constants, split into hi + lo floats on the host: dt / dx_a^2 per axis, the boundary
// values and the Neumann gradient times dx per face
struct DfConst {
  float s_hi[3], s_lo[3];
  float v_hi[6], v_lo[6];
  float gdx_hi[6], gdx_lo[6];
};

DfConst make_df_const(const GridDev& g, double dt);

// face weights w = dt D_f / dx^2 (harmonic-mean faces) as hi + lo floats; *flag |= 1 where a
// value left the double-float window
cudaError_t launch_faces_df(const GridDev& g, const DfConst& K, const double* D, float* const w[3],
                            float* const wlo[3], unsigned* flag, cudaStream_t s);

// diagonal (hi, lo), 1/diag, right-hand side b (hi, lo) and ||b||^2 into scal[1], 1/rms(b) into
// scal[4]
cudaError_t launch_fine_setup_df(const GridDev& g, const DfConst& K, const LevelDev<float>& L,
                                 const LevelDev<float>& Llo, const double* E_old, float* dhi, float* dlo, float* invd,
                                 float* bhi, float* blo, double* parts, int nparts, double* scal, unsigned* flag,
                                 cudaStream_t s);

// r = b - A x (hi, lo) with x = E_old copied into x64; parts[0..nparts) = sum (scal[4] r)^2,
// parts[nparts..2 nparts) = the error measure's squares
cudaError_t launch_residual0_df(int ndim, const LevelDev<float>& L, const LevelDev<float>& Llo, const float* dhi,
                                const float* dlo, const float* bhi, const float* blo, const double* x, double* x64,
                                float* rhi, float* rlo, const double* scal, int nparts, double* parts,
                                cudaStream_t s);

// defined in mg.cu
__global__ void k_reduce(const double* __restrict__ parts, int n, double* __restrict__ out);

}  // namespace fld

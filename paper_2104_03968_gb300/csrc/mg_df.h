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

// face weights w = dt D_f / dx^2 (harmonic-mean faces) as hi + lo floats, and (dc not null) each
// cell's 1 / (dt D / dx_0^2) in FP32; *flag |= 1 where a value left the double-float window
cudaError_t launch_faces_df(const GridDev& g, const DfConst& K, const double* D, float* const w[3],
                            float* const wlo[3], float* dc, unsigned* flag, cudaStream_t s);

// diagonal (hi, lo) and 1/diag of the finest level, and the first outer residual r = b - A x
// (hi, lo) with x = E_old, copied into x64 unless it is null; scal[0] = ||r||^2, scal[1] = ||b||^2,
// scal[2] = the squared error measure of r's terms.  parts holds 3 nparts doubles.
cudaError_t launch_setup_res0_df(const GridDev& g, const DfConst& K, const LevelDev<float>& L,
                                 const LevelDev<float>& Llo, const double* x, double* x64, float* dhi, float* dlo,
                                 float* invd, float* rhi, float* rlo, int nparts, double* parts, double* scal,
                                 unsigned* flag, cudaStream_t s);

// defined in mg.cu
__global__ void k_reduce(const double* __restrict__ parts, int n, double* __restrict__ out);

}  // namespace fld

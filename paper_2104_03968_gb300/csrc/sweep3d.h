// Red-black Gauss-Seidel sweep of the mixed solver's FP32 finest level on 3-D grids, one launch
// per full sweep, from the cell-centred diffusion coefficient (host side).
#pragma once

#include <cuda_runtime.h>

namespace fld {

struct Sweep3dArgs {
  int nx, ny, nz;
  int bc[6];
  float ra[3];          // dx_0^2 / dx_a^2: axis a's faces weigh harmonic(dc) * ra[a]
  const float* dc;      // per cell, 1 / (dt D_cell / dx_0^2) (FP32; inf where D = 0)
  const float* r;       // right-hand side of the correction equation
  const float* xin;     // iterate before the sweep; nullptr: the sweep starts from x = 0
  float* xout;          // iterate after the sweep (a different array from xin)
  double* x64;          // if set, each cell's new value is also added to this FP64 array
  int c0;               // the first half-sweep updates the cells with (i + j + k) & 1 == c0
  unsigned* err;        // if set, a wait for staged planes that ran out of its bound ORs 1 into it
};

// Levels the tiled sweep takes: 3-D, nx a multiple of 64 (and at least 64), ny of 16, nz even
// and >= 4, fewer than 2^31 cells.
bool sweep3d_eligible(int nx, int ny, int nz);

// One full sweep (both colours).  Asynchronous on s.  Every array must start on a 16-byte boundary
// (the planes are fetched in 16-byte copies and TMA boxes).
cudaError_t launch_sweep3d(const Sweep3dArgs& a, cudaStream_t s);

// dc = 1 / (float)(dt D_cell / dx_0^2) per cell, from the FP64 D (the solver's FP64 set-up path).
cudaError_t launch_dcell32(long long ncell, double scale, const double* D, float* dc, cudaStream_t s);

}  // namespace fld

// Many independent 2-D/3-D grids advanced by one call: one CUDA graph per batch shape, with a
// device-side WHILE loop over the multigrid iterations.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "mg.h"

namespace fld {

class BatchedSolver {
 public:
  BatchedSolver() = default;
  ~BatchedSolver();
  BatchedSolver(const BatchedSolver&) = delete;
  BatchedSolver& operator=(const BatchedSolver&) = delete;

  fld_status run(int ngrids, const fld_grid* grids, const fld_params* params, const double* dt,
                 const double* const* rho, double* const* eps, double* const* E, fld_info* infos, cudaStream_t s,
                 std::string* err);

  // smoothing counts and tile size chosen for the current batch shape (after the first run)
  int nu1() const { return nu1_; }
  int nu2() const { return nu2_; }
  int tile() const { return tile_; }

 private:
  struct Impl;
  Impl* impl_ = nullptr;
  int nu1_ = 0, nu2_ = 0, tile_ = 0;
};

}  // namespace fld

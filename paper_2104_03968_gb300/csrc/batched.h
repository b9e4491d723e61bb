// Many independent 2-D/3-D grids advanced by one call.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "mg.h"

namespace fld {

class BatchedSolver {
 public:
  BatchedSolver() = default;
  ~BatchedSolver();
  fld_status run(int ngrids, const fld_grid* grids, const fld_params* params, const double* dt,
                 const double* const* rho, double* const* eps, double* const* E, fld_info* infos, cudaStream_t s,
                 std::string* err);

 private:
  std::vector<std::unique_ptr<Multigrid>> mg_;
  double* D_ = nullptr;
  double* kappa_ = nullptr;
  size_t cap_ = 0;
  unsigned* d_status_ = nullptr;
  int* d_info_ = nullptr;
  int* h_info_ = nullptr;
};

}  // namespace fld

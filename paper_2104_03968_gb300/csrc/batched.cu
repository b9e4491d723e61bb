// Many independent grids per call: coefficients, multigrid diffusion and exchange per grid.
#include <cstdio>
#include <cstring>

#include "batched.h"
#include "kernels.h"

namespace fld {

BatchedSolver::~BatchedSolver() {
  cudaFree(D_);
  cudaFree(kappa_);
  cudaFree(d_status_);
  cudaFree(d_info_);
  if (h_info_) cudaFreeHost(h_info_);
}

static GridDev grid_dev(const fld_grid& g) {
  GridDev d{};
  d.ndim = g.ndim;
  for (int a = 0; a < 3; ++a) {
    d.n[a] = g.n[a];
    d.dx[a] = a < g.ndim ? g.dx[a] : 1.0;
  }
  for (int f = 0; f < 6; ++f) {
    d.bc[f] = (f / 2) < g.ndim ? g.bc[f] : FLD_BC_PERIODIC;
    d.bc_val[f] = (f / 2) < g.ndim ? g.bc_val[f] : 0.0;
  }
  d.ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  return d;
}

static Opacity opacity_of(const fld_params& p) {
  Opacity o{};
  o.model = p.opacity;
  o.kappa0 = p.kappa0;
  o.kr_a = p.kr_a;
  o.kr_b = p.kr_b;
  o.table = p.table;
  o.tn0 = p.tn[0];
  o.tn1 = p.tn[1];
  o.tlo0 = p.tlo[0];
  o.tlo1 = p.tlo[1];
  o.thi0 = p.thi[0];
  o.thi1 = p.thi[1];
  return o;
}

fld_status BatchedSolver::run(int ngrids, const fld_grid* grids, const fld_params* params, const double* dt,
                              const double* const* rho, double* const* eps, double* const* E, fld_info* infos,
                              cudaStream_t s, std::string* err) {
  char buf[256];
  auto cuda_err = [&](cudaError_t e, const char* where) {
    snprintf(buf, sizeof(buf), "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
    *err = buf;
    return FLD_ERR_CUDA;
  };
  size_t maxcells = 0;
  for (int i = 0; i < ngrids; ++i) maxcells = std::max(maxcells, (size_t)grid_dev(grids[i]).ncell);
  cudaError_t e = cudaSuccess;
  if (!d_status_) {
    e = cudaMalloc(&d_status_, 64);
    if (e == cudaSuccess) e = cudaMalloc(&d_info_, 64);
    if (e == cudaSuccess) e = cudaMallocHost(&h_info_, 64);
    if (e != cudaSuccess) return cuda_err(e, "batched status allocation");
  }
  if (maxcells > cap_) {
    cudaFree(D_);
    cudaFree(kappa_);
    D_ = kappa_ = nullptr;
    cap_ = 0;
    e = cudaMalloc(&D_, maxcells * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&kappa_, maxcells * sizeof(double));
    if (e != cudaSuccess) return cuda_err(e, "batched scratch allocation");
    cap_ = maxcells;
  }
  if ((int)mg_.size() < ngrids) mg_.resize(ngrids);
  fld_status worst = FLD_OK;
  for (int i = 0; i < ngrids; ++i) {
    const fld_params& p = params[i];
    GridDev g = grid_dev(grids[i]);
    if (!mg_[i]) mg_[i].reset(new Multigrid());
    Multigrid& mg = *mg_[i];
    Opacity op = opacity_of(p);
    ExchangeParams xp{p.c, p.a_rad * p.c / 4.0, p.gamma, p.gas_R, dt[i], p.exch_maxit > 0 ? p.exch_maxit : 100};
    if ((e = cudaMemsetAsync(d_status_, 0, 4, s)) != cudaSuccess) return cuda_err(e, "status reset");
    if ((e = cudaMemsetAsync(d_info_, 0, 8, s)) != cudaSuccess) return cuda_err(e, "status reset");
    if (p.order == FLD_ORDER_EXCHANGE_THEN_DIFFUSE) {
      e = launch_exchange(g.ncell, xp, op, rho[i], nullptr, eps[i], E[i], d_info_, d_info_ + 1, d_status_, s);
      if (e != cudaSuccess) return cuda_err(e, "exchange");
    }
    e = launch_coeffs(g, op, p.c, p.gamma, p.gas_R, p.limiter, E[i], rho[i], eps[i], kappa_, D_, d_status_, s);
    if (e != cudaSuccess) return cuda_err(e, "coeffs");
    if ((e = mg.configure(g, p.precision)) != cudaSuccess) return cuda_err(e, "multigrid allocation");
    if ((e = mg.setup(dt[i], D_, E[i], d_status_, s)) != cudaSuccess) return cuda_err(e, "multigrid setup");
    SolveStats st;
    int maxc = p.max_cycles > 0 ? p.max_cycles : 100;
    e = mg.solve(E[i], E[i], p.rtol, maxc, p.nu1 > 0 ? p.nu1 : 2, p.nu2 > 0 ? p.nu2 : 2, &st, s);
    if (e != cudaSuccess) return cuda_err(e, "multigrid solve");
    if (p.order == FLD_ORDER_DIFFUSE_THEN_EXCHANGE) {
      e = launch_exchange(g.ncell, xp, op, rho[i], kappa_, eps[i], E[i], d_info_, d_info_ + 1, d_status_, s);
      if (e != cudaSuccess) return cuda_err(e, "exchange");
    }
    e = cudaMemcpyAsync(h_info_, d_info_, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_info_ + 2, d_status_, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e, "status read-back");
    int status = st.status;
    if (h_info_[2] & kStatNonpositive) status = FLD_ERR_NONPOSITIVE;
    if (infos) {
      memset(&infos[i], 0, sizeof(fld_info));
      infos[i].cycles = st.cycles;
      infos[i].rel_residual = st.relres;
      infos[i].exch_max_iters = h_info_[0];
      infos[i].bisection_fallbacks = h_info_[1];
      infos[i].status = status;
    }
    if (status != FLD_OK && worst == FLD_OK) {
      worst = (fld_status)status;
      snprintf(buf, sizeof(buf), "grid %d: status %d (relative residual %.3e after %d cycles)", i, status, st.relres,
               st.cycles);
      *err = buf;
    }
  }
  return worst;
}

}  // namespace fld

// Geometric multigrid for the backward-Euler FLD diffusion problem of arXiv 2104.03968,
// Sect. 3.4: E^{n+1}/dt - div(D^n grad E^{n+1}) = E^n/dt, discretised by Eq. (discdiff) with
// harmonic-mean face coefficients.  The system is scaled by dt:
//     (A x)_c = x_c + sum_faces w_f (x_c - x_nb),   w_f = dt D_f / dx^2,   b = E^n (+ boundary)
//
// Structure (the paper's solver is a CPU octree multigrid library; this is a GPU design):
//   outer loop (FP64):  r = b - A x;  ||r||/||b|| <= rtol ?;  A d ~= r by one V-cycle;  x += d
//   V-cycle (type T):   red-black Gauss-Seidel (nu1 before, nu2 after, reversed colours),
//                       residual + 2^d-cell averaging restriction fused in one kernel,
//                       piecewise-constant prolongation, coarse faces = mean of the fine faces
//                       they cover / 4 (rediscretisation), one-block coarsest solve.
// T = double is the plain FP64 solver; T = float gives the mixed form whose smoother,
// restriction and prolongation run in FP32 while the residual, update and norm stay FP64.
#include <array>
#include <cstdio>

#include "kernels.h"
#include "mg.h"
#include "mg_device.cuh"
#include "trace.h"

namespace fld {

// ----------------------------------------------------------------------------- arena

DeviceArena::~DeviceArena() { release(); }

cudaError_t DeviceArena::reserve(size_t bytes) {
  release();
  cudaError_t e = cudaMalloc(&base_, bytes);
  if (e != cudaSuccess) {
    base_ = nullptr;
    return e;
  }
  cap_ = bytes;
  used_ = 0;
  return cudaSuccess;
}

void* DeviceArena::take(size_t bytes) {
  size_t off = (used_ + 255) & ~(size_t)255;
  if (off + bytes > cap_) return nullptr;
  used_ = off + bytes;
  return base_ + off;
}

void DeviceArena::release() {
  if (base_) cudaFree(base_);
  base_ = nullptr;
  cap_ = used_ = 0;
}

// deterministic second stage: one block sums the per-block partials in a fixed order
__global__ void k_reduce(const double* __restrict__ parts, int n, double* __restrict__ out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += parts[i];
  v = block_sum(v);
  if (threadIdx.x == 0) *out = v;
}

__global__ void k_sumsq(const double* __restrict__ x, long long n, double* __restrict__ parts) {
  double v = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double t = x[i];
    v += t * t;
  }
  v = block_sum(v);
  if (threadIdx.x == 0) parts[blockIdx.x] = v;
}

// ----------------------------------------------------------------------------- setup kernels
// (the per-cell bodies are in mg_device.cuh, shared with the batched solver)

template <class T>
__global__ void k_fine_setup(LevelDev<double> L, GridDev g, const double* __restrict__ E_old, double* __restrict__ b,
                             double* __restrict__ diag, T* __restrict__ invd) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  fine_setup_cell<T>(L, g, E_old, idx, b, diag, invd);
}

template <class T>
__global__ void k_invd(LevelDev<T> L, long long ncell, T* __restrict__ invd) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncell) return;
  int i, j, k;
  unflatten(L.n, idx, i, j, k);
  invd[idx] = T(1) / diag_of(L, i, j, k, idx);
}

template <class T>
__global__ void k_coarse_faces(int a, int ndim, std::array<int, 3> nf, std::array<int, 3> nc, const T* __restrict__ wf,
                               T* __restrict__ wc) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int m[3] = {nc[0], nc[1], nc[2]};
  m[a] += 1;
  if (idx >= (long long)m[0] * m[1] * m[2]) return;
  wc[idx] = coarse_face_value<T>(a, ndim, nf.data(), m, idx, wf);
}

// ----------------------------------------------------------------------------- cycle kernels

template <class T>
__global__ void __launch_bounds__(256, 4) k_residual64(LevelDev<double> L, long long ncell, const double* x_in, double* x_out,
                             const double* __restrict__ b, const double* __restrict__ diag, T* __restrict__ r_out,
                             double* __restrict__ parts) {
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ncell;
       idx += (long long)gridDim.x * blockDim.x)
    acc = fma_residual_cell<T>(L, x_in, x_out, b, diag, r_out, idx, acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

// x64 += d (used only when no post-smoothing sweep carries the update)
template <class T>
__global__ void k_add_correction(long long ncell, const T* __restrict__ d, double* __restrict__ x64) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < ncell) x64[idx] += (double)d[idx];
}

template <class T, bool ZERO, bool UPDATE = false>
__global__ void k_smooth(LevelDev<T> L, const T* __restrict__ invd, const T* __restrict__ r, T* __restrict__ x,
                         int color, double* __restrict__ x64 = nullptr) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  smooth_colour_cell<T, ZERO, UPDATE>(L, invd, r, x, color, t, x64);
}

template <class T>
__global__ void k_residual_restrict(LevelDev<T> F, const T* __restrict__ rf, const T* __restrict__ xf,
                                    std::array<int, 3> nc, T* __restrict__ rc, T* __restrict__ xc_zero) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nc[0] * nc[1] * nc[2]) return;
  rc[idx] = restrict_value<T>(F, rf, xf, nc.data(), idx);
  if (xc_zero) xc_zero[idx] = T(0);
}

template <class T>
__global__ void k_prolong(std::array<int, 3> nf, int ndim, const T* __restrict__ xc, std::array<int, 3> nc,
                          T* __restrict__ xf) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nf[0] * nf[1] * nf[2]) return;
  prolong_cell<T>(nf.data(), ndim, xc, nc.data(), xf, idx);
}

template <class T>
__global__ void __launch_bounds__(512) k_coarse_solve(LevelDev<T> L, long long ncell, const T* __restrict__ invd, const T* __restrict__ r,
                               T* __restrict__ x, T* __restrict__ tmp, int sweeps, int use_rb) {
  coarse_solve_block<T>(L, ncell, invd, r, x, tmp, sweeps, use_rb);
}

// ----------------------------------------------------------------------------- host side

static inline unsigned nblk(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

Multigrid::~Multigrid() {
  if (host_scal_) cudaFreeHost(host_scal_);
}

static inline long long cells3(const std::array<int, 3>& n) { return (long long)n[0] * n[1] * n[2]; }

static inline long long faces3(const std::array<int, 3>& n, int a) {
  long long c = 1;
  for (int b = 0; b < 3; ++b) c *= (b == a) ? n[b] + 1 : n[b];
  return c;
}

cudaError_t Multigrid::configure(const GridDev& g, int precision) {
  bool same = configured_ && precision == precision_ && g.ndim == g_.ndim;
  for (int a = 0; a < 3 && same; ++a) same = g.n[a] == g_.n[a];
  for (int f = 0; f < 6 && same; ++f) same = g.bc[f] == g_.bc[f];
  g_ = g;  // dx and bc values may change freely
  if (same) return cudaSuccess;
  configured_ = false;
  precision_ = precision;
  dims_.clear();
  std::array<int, 3> d = {g.n[0], g.n[1], g.n[2]};
  dims_.push_back(d);
  for (;;) {
    bool ok = cells3(d) > 64;
    for (int a = 0; a < g.ndim && ok; ++a) ok = (d[a] % 2 == 0) && d[a] >= 4;
    if (!ok) break;
    for (int a = 0; a < g.ndim; ++a) d[a] /= 2;
    dims_.push_back(d);
  }
  const size_t es = precision == FLD_PREC_MIXED ? sizeof(float) : sizeof(double);
  long long N = cells3(dims_[0]);
  nparts_ = 152 * 16;
  size_t bytes = 0;
  auto add = [&](size_t b) { bytes += (b + 511) & ~(size_t)255; };
  for (int a = 0; a < g.ndim; ++a) add(faces3(dims_[0], a) * sizeof(double));
  for (int k = 0; k < 2; ++k) add(N * sizeof(double));  // b, diag
  add(nparts_ * sizeof(double));
  add(4 * sizeof(double));
  for (size_t l = 0; l < dims_.size(); ++l) {
    long long n = cells3(dims_[l]);
    if (l > 0 || precision == FLD_PREC_MIXED)
      for (int a = 0; a < g.ndim; ++a) add(faces3(dims_[l], a) * es);
    for (int k = 0; k < 4; ++k) add(n * es);  // invd, x, r, tmp
  }
  cudaError_t e = arena_.reserve(bytes + 4096);
  if (e != cudaSuccess) return e;
  for (int a = 0; a < 3; ++a) w64_[a] = a < g.ndim ? (double*)arena_.take(faces3(dims_[0], a) * sizeof(double)) : nullptr;
  b64_ = (double*)arena_.take(N * sizeof(double));
  diag64_ = (double*)arena_.take(N * sizeof(double));
  partials_ = (double*)arena_.take(nparts_ * sizeof(double));
  scal_ = (double*)arena_.take(4 * sizeof(double));
  if (!host_scal_) {
    e = cudaMallocHost(&host_scal_, 4 * sizeof(double));
    if (e != cudaSuccess) return e;
  }
  lv_.assign(dims_.size(), LevelBuf{});
  for (size_t l = 0; l < dims_.size(); ++l) {
    long long n = cells3(dims_[l]);
    for (int a = 0; a < 3; ++a) {
      if (a >= g.ndim) lv_[l].w[a] = nullptr;
      else if (l == 0 && precision != FLD_PREC_MIXED) lv_[l].w[a] = w64_[a];
      else lv_[l].w[a] = arena_.take(faces3(dims_[l], a) * es);
    }
    lv_[l].invd = arena_.take(n * es);
    lv_[l].x = arena_.take(n * es);
    lv_[l].r = arena_.take(n * es);
    lv_[l].tmp = arena_.take(n * es);
    if (!lv_[l].invd || !lv_[l].x || !lv_[l].r || !lv_[l].tmp) return cudaErrorMemoryAllocation;
    for (int a = 0; a < g.ndim; ++a)
      if (!lv_[l].w[a]) return cudaErrorMemoryAllocation;
  }
  if (!b64_ || !diag64_ || !partials_ || !scal_) return cudaErrorMemoryAllocation;
  configured_ = true;
  return cudaSuccess;
}

template <class T>
static LevelDev<T> level_dev(const GridDev& g, const std::array<int, 3>& n, void* const w[3]) {
  LevelDev<T> L;
  for (int a = 0; a < 3; ++a) L.n[a] = n[a];
  L.ndim = g.ndim;
  for (int f = 0; f < 6; ++f) L.bc[f] = g.bc[f];
  for (int a = 0; a < 3; ++a) L.w[a] = (const T*)w[a];
  return L;
}

template <class T>
cudaError_t Multigrid::setup_t(double dt, const double* D_cell, const double* E_old, cudaStream_t s) {
  float* w32[3] = {nullptr, nullptr, nullptr};
  if (precision_ == FLD_PREC_MIXED)
    for (int a = 0; a < g_.ndim; ++a) w32[a] = (float*)lv_[0].w[a];
  cudaError_t e = launch_faces(g_, dt, D_cell, w64_, w32, s);
  if (e != cudaSuccess) return e;
  void* w64v[3] = {w64_[0], w64_[1], w64_[2]};
  LevelDev<double> L64 = level_dev<double>(g_, dims_[0], w64v);
  {
    TraceScope ts("fine_setup", s);
    k_fine_setup<T><<<nblk(g_.ncell), kBlock, 0, s>>>(L64, g_, E_old, b64_, diag64_, (T*)lv_[0].invd);
  }
  for (size_t l = 1; l < dims_.size(); ++l) {
    TraceScope ts("coarse_setup", s);
    for (int a = 0; a < g_.ndim; ++a)
      k_coarse_faces<T><<<nblk(faces3(dims_[l], a)), kBlock, 0, s>>>(a, g_.ndim, dims_[l - 1], dims_[l],
                                                                      (const T*)lv_[l - 1].w[a], (T*)lv_[l].w[a]);
    LevelDev<T> L = level_dev<T>(g_, dims_[l], lv_[l].w);
    k_invd<T><<<nblk(cells3(dims_[l])), kBlock, 0, s>>>(L, cells3(dims_[l]), (T*)lv_[l].invd);
  }
  // ||b||^2
  {
    TraceScope ts("norm_b", s);
    k_sumsq<<<nparts_, kBlock, 0, s>>>(b64_, g_.ncell, partials_);
    k_reduce<<<1, 1024, 0, s>>>(partials_, nparts_, scal_ + 1);
  }
  return cudaGetLastError();
}

cudaError_t Multigrid::setup(double dt, const double* D_cell, const double* E_old, unsigned* status, cudaStream_t s) {
  (void)status;
  return precision_ == FLD_PREC_MIXED ? setup_t<float>(dt, D_cell, E_old, s) : setup_t<double>(dt, D_cell, E_old, s);
}

template <class T>
cudaError_t Multigrid::vcycle(int l, int nu1, int nu2, double* x64, cudaStream_t s) {
  const std::array<int, 3>& n = dims_[l];
  long long ncell = cells3(n);
  LevelDev<T> L = level_dev<T>(g_, n, lv_[l].w);
  T* x = (T*)lv_[l].x;
  T* r = (T*)lv_[l].r;
  T* invd = (T*)lv_[l].invd;
  if (l == (int)dims_.size() - 1) {
    bool rb = true;
    for (int a = 0; a < g_.ndim; ++a)
      if ((n[a] & 1) && (g_.bc[2 * a] == FLD_BC_PERIODIC)) rb = false;
    int sweeps = rb ? 40 : 80;
    TraceScope ts("coarse_solve", s);
    k_coarse_solve<T><<<1, 512, 0, s>>>(L, ncell, invd, r, x, (T*)lv_[l].tmp, sweeps, rb ? 1 : 0);
    if (x64) k_add_correction<T><<<nblk(ncell), kBlock, 0, s>>>(ncell, x, x64);
    return cudaGetLastError();
  }
  long long nhalf = (long long)((n[0] + 1) / 2) * n[1] * n[2];
  unsigned gb = nblk(nhalf);
  // pre-smoothing from a zero initial guess: red, black, ...
  const char* sm_name = l == 0 ? "smooth_L0" : "smooth_Lc";
  for (int it = 0; it < nu1; ++it) {
    {
      TraceScope ts(it == 0 ? (l == 0 ? "smooth_L0_zero" : "smooth_Lc") : sm_name, s);
      if (it == 0) k_smooth<T, true><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
      else k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
    }
    TraceScope ts(sm_name, s);
    k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1);
  }
  const std::array<int, 3>& nc = dims_[l + 1];
  {
    TraceScope ts(l == 0 ? "restrict_L0" : "restrict_Lc", s);
    k_residual_restrict<T><<<nblk(cells3(nc)), kBlock, 0, s>>>(L, r, x, nc, (T*)lv_[l + 1].r, nullptr);
  }
  cudaError_t e = vcycle<T>(l + 1, nu1, nu2, nullptr, s);
  if (e != cudaSuccess) return e;
  {
    TraceScope ts(l == 0 ? "prolong_L0" : "prolong_Lc", s);
    k_prolong<T><<<nblk(ncell), kBlock, 0, s>>>(n, g_.ndim, (const T*)lv_[l + 1].x, nc, x);
  }
  // post-smoothing, colours reversed; on the finest level the last sweep also adds each colour's
  // final correction to the FP64 iterate
  for (int it = 0; it < nu2; ++it) {
    bool last = x64 && it == nu2 - 1;
    {
      TraceScope ts(sm_name, s);
      if (last) k_smooth<T, false, true><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1, x64);
      else k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1);
    }
    TraceScope ts(sm_name, s);
    if (last) k_smooth<T, false, true><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0, x64);
    else k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
  }
  if (x64 && nu2 == 0) {
    TraceScope ts("add_correction", s);
    k_add_correction<T><<<nblk(ncell), kBlock, 0, s>>>(ncell, x, x64);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t Multigrid::solve_t(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                               SolveStats* st, cudaStream_t s) {
  void* w64v[3] = {w64_[0], w64_[1], w64_[2]};
  LevelDev<double> L64 = level_dev<double>(g_, dims_[0], w64v);
  // the FP64 iterate lives in E_new; the first residual copies E_old into it
  const double* x_in = E_old;
  double* x = E_new;
  double bb = 0.0;
  int cycles = 0;
  double rel = 0.0;
  int status = FLD_ERR_NOT_CONVERGED;
  for (;;) {
    {
      TraceScope ts("residual", s);
      k_residual64<T><<<nparts_, kBlock, 0, s>>>(L64, g_.ncell, x_in, x, b64_, diag64_, (T*)lv_[0].r, partials_);
    }
    {
      TraceScope ts("reduce", s);
      k_reduce<<<1, 1024, 0, s>>>(partials_, nparts_, scal_);
    }
    x_in = x;
    cudaError_t e = cudaMemcpyAsync(host_scal_, scal_, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    bb = host_scal_[1];
    double rr = host_scal_[0];
    rel = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
    if (!(rel == rel) || rel > 1e300) {
      status = FLD_ERR_NONFINITE;
      break;
    }
    if (rel <= rtol) {
      status = FLD_OK;
      break;
    }
    if (cycles >= max_cycles) break;
    // one V-cycle on A d = r; its last finest-level sweep adds d to x
    e = vcycle<T>(0, nu1, nu2, x, s);
    if (e != cudaSuccess) return e;
    ++cycles;
  }
  st->cycles = cycles;
  st->relres = rel;
  st->status = status;
  return cudaStreamSynchronize(s);
}

cudaError_t Multigrid::solve(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                             SolveStats* st, cudaStream_t s) {
  return precision_ == FLD_PREC_MIXED ? solve_t<float>(E_old, E_new, rtol, max_cycles, nu1, nu2, st, s)
                                      : solve_t<double>(E_old, E_new, rtol, max_cycles, nu1, nu2, st, s);
}

}  // namespace fld

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

// ----------------------------------------------------------------------------- face visitor

enum FaceKind { kInterior = 0, kDirichlet = 1, kNeumann = 2, kContinuous = 3 };

// Calls f(w, kind, nb) for each face of cell (i,j,k): kind kInterior (nb = the cell across the
// face, periodic faces included), kDirichlet / kNeumann (no neighbour), kContinuous (nb = the
// next cell inward, the ghost being the linear extrapolation 2 x_c - x_nb).
template <class W, class F>
__device__ __forceinline__ void for_each_face(const LevelDev<W>& L, int i, int j, int k, long long idx, F&& f) {
  const int q[3] = {i, j, k};
  long long stride = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= L.ndim) break;
    const int n = L.n[a];
    const int p = q[a];
    const W wl = L.w[a][face_index(L.n, a, i, j, k, p)];
    const W wu = L.w[a][face_index(L.n, a, i, j, k, p + 1)];
    if (p > 0) {
      f(wl, kInterior, idx - stride);
    } else {
      int bc = L.bc[2 * a];
      if (bc == FLD_BC_PERIODIC) f(wl, kInterior, idx + (long long)(n - 1) * stride);
      else if (bc == FLD_BC_DIRICHLET) f(wl, kDirichlet, idx);
      else if (bc == FLD_BC_NEUMANN) f(wl, kNeumann, idx);
      else f(wl, kContinuous, idx + stride);
    }
    if (p < n - 1) {
      f(wu, kInterior, idx + stride);
    } else {
      int bc = L.bc[2 * a + 1];
      if (bc == FLD_BC_PERIODIC) f(wu, kInterior, idx - (long long)(n - 1) * stride);
      else if (bc == FLD_BC_DIRICHLET) f(wu, kDirichlet, idx);
      else if (bc == FLD_BC_NEUMANN) f(wu, kNeumann, idx);
      else f(wu, kContinuous, idx - stride);
    }
    stride *= n;
  }
}

template <class T>
__device__ __forceinline__ T diag_of(const LevelDev<T>& L, int i, int j, int k, long long idx) {
  T d = T(1);
  for_each_face(L, i, j, k, idx, [&](T w, int kind, long long) {
    if (kind == kInterior || kind == kDirichlet) d += w;
    else if (kind == kContinuous) d -= w;
  });
  return d;
}

__device__ __forceinline__ void unflatten(const int n[3], long long idx, int& i, int& j, int& k) {
  i = (int)(idx % n[0]);
  long long r = idx / n[0];
  j = (int)(r % n[1]);
  k = (int)(r / n[1]);
}

// ----------------------------------------------------------------------------- reductions

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;  // valid in thread 0
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

// b = E_old + boundary constants (Dirichlet ghost value, Neumann gradient); 1/diagonal in T.
template <class T>
__global__ void k_fine_setup(LevelDev<double> L, GridDev g, const double* __restrict__ E_old, double* __restrict__ b,
                             T* __restrict__ invd) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  int i, j, k;
  unflatten(g.n, idx, i, j, k);
  double d = 1.0, cst = 0.0;
  const int q[3] = {i, j, k};
  int face = 0;
  // boundary constants need to know which side each boundary face is on
  for_each_face(L, i, j, k, idx, [&](double w, int kind, long long) {
    int a = face >> 1, side = face & 1;
    ++face;
    if (kind == kInterior) d += w;
    else if (kind == kDirichlet) {
      d += w;
      cst += w * g.bc_val[2 * a + side];
    } else if (kind == kNeumann) {
      double m = w * g.bc_val[2 * a + side] * g.dx[a];
      cst += side ? m : -m;
    } else {
      d -= w;
    }
    (void)q;
  });
  b[idx] = E_old[idx] + cst;
  invd[idx] = (T)(1.0 / d);
}

template <class T>
__global__ void k_invd(LevelDev<T> L, long long ncell, T* __restrict__ invd) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncell) return;
  int i, j, k;
  unflatten(L.n, idx, i, j, k);
  invd[idx] = T(1) / diag_of(L, i, j, k, idx);
}

// coarse face = mean of the 2^(d-1) fine faces it covers, / 4 (dx doubles)
template <class T>
__global__ void k_coarse_faces(int a, int ndim, std::array<int, 3> nf, std::array<int, 3> nc, const T* __restrict__ wf,
                               T* __restrict__ wc) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int m[3] = {nc[0], nc[1], nc[2]};
  m[a] += 1;
  long long total = (long long)m[0] * m[1] * m[2];
  if (idx >= total) return;
  int q[3];
  q[0] = (int)(idx % m[0]);
  long long r = idx / m[0];
  q[1] = (int)(r % m[1]);
  q[2] = (int)(r / m[1]);
  int mf[3] = {nf[0], nf[1], nf[2]};
  mf[a] += 1;
  T s = T(0);
  int cnt = 0;
  int o1max = (ndim > 1) ? 2 : 1, o2max = (ndim > 2) ? 2 : 1;
  for (int o2 = 0; o2 < o2max; ++o2)
    for (int o1 = 0; o1 < o1max; ++o1) {
      int f[3];
      // the two transverse axes in increasing order
      int t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;
      f[a] = 2 * q[a];
      f[t1] = (t1 < ndim) ? 2 * q[t1] + o1 : q[t1];
      f[t2] = (t2 < ndim) ? 2 * q[t2] + o2 : q[t2];
      s += wf[(long long)f[0] + (long long)mf[0] * ((long long)f[1] + (long long)mf[1] * f[2])];
      ++cnt;
    }
  wc[idx] = s / (T)(4 * cnt);
}

// ----------------------------------------------------------------------------- cycle kernels

// r_out = b - A (x_in + d); x_out = x_in + d; per-block partial sums of r^2.  FP64 operator.
template <class T>
__global__ void k_update_residual(LevelDev<double> L, long long ncell, const double* __restrict__ x_in,
                                  const T* __restrict__ d, const double* __restrict__ b, double* __restrict__ x_out,
                                  T* __restrict__ r_out, double* __restrict__ parts) {
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ncell;
       idx += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten(L.n, idx, i, j, k);
    auto X = [&](long long c) -> double { return d ? x_in[c] + (double)d[c] : x_in[c]; };
    double xc = X(idx);
    double ax = xc;
    for_each_face(L, i, j, k, idx, [&](double w, int kind, long long nb) {
      if (kind == kInterior) ax += w * (xc - X(nb));
      else if (kind == kDirichlet) ax += w * xc;
      else if (kind == kContinuous) ax += w * (X(nb) - xc);
    });
    double r = b[idx] - ax;
    x_out[idx] = xc;
    r_out[idx] = (T)r;
    acc += r * r;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

// One colour of a red-black Gauss-Seidel sweep: x_c = (r_c + sum w x_nb) / diag on the cells
// with (i+j+k) % 2 == color.  ZERO: the sweep starts from x = 0 (neighbours read as zero).
template <class T, bool ZERO>
__global__ void k_smooth(LevelDev<T> L, const T* __restrict__ invd, const T* __restrict__ r, T* __restrict__ x,
                         int color) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int nxh = (L.n[0] + 1) >> 1;
  long long rows = (long long)L.n[1] * L.n[2];
  if (t >= (long long)nxh * rows) return;
  int m = (int)(t % nxh);
  long long row = t / nxh;
  int j = (int)(row % L.n[1]);
  int k = (int)(row / L.n[1]);
  int i = 2 * m + ((color + j + k) & 1);
  if (i >= L.n[0]) return;
  long long idx = (long long)i + (long long)L.n[0] * row;
  T v = r[idx];
  if (!ZERO) {
    for_each_face(L, i, j, k, idx, [&](T w, int kind, long long nb) {
      if (kind == kInterior) v += w * x[nb];
      else if (kind == kContinuous) v -= w * x[nb];
    });
  }
  x[idx] = v * invd[idx];
}

// coarse rhs = average over the 2^d children of the fine residual r - A x
template <class T>
__global__ void k_residual_restrict(LevelDev<T> F, const T* __restrict__ rf, const T* __restrict__ xf,
                                    std::array<int, 3> nc, T* __restrict__ rc, T* __restrict__ xc_zero) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long ncell = (long long)nc[0] * nc[1] * nc[2];
  if (idx >= ncell) return;
  int I = (int)(idx % nc[0]);
  long long rr = idx / nc[0];
  int J = (int)(rr % nc[1]);
  int K = (int)(rr / nc[1]);
  int o1max = F.ndim > 1 ? 2 : 1, o2max = F.ndim > 2 ? 2 : 1;
  T s = T(0);
  for (int o2 = 0; o2 < o2max; ++o2)
    for (int o1 = 0; o1 < o1max; ++o1)
      for (int o0 = 0; o0 < 2; ++o0) {
        int i = 2 * I + o0, j = F.ndim > 1 ? 2 * J + o1 : J, k = F.ndim > 2 ? 2 * K + o2 : K;
        long long c = cell_index(F.n, i, j, k);
        T xv = xf[c];
        T ax = xv;
        for_each_face(F, i, j, k, c, [&](T w, int kind, long long nb) {
          if (kind == kInterior) ax += w * (xv - xf[nb]);
          else if (kind == kDirichlet) ax += w * xv;
          else if (kind == kContinuous) ax += w * (xf[nb] - xv);
        });
        s += rf[c] - ax;
      }
  rc[idx] = s / (T)(2 * o1max * o2max);
  if (xc_zero) xc_zero[idx] = T(0);
}

// x_f += x_c(parent): piecewise-constant prolongation of the coarse correction
template <class T>
__global__ void k_prolong(std::array<int, 3> nf, int ndim, const T* __restrict__ xc, std::array<int, 3> nc,
                          T* __restrict__ xf) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long ncell = (long long)nf[0] * nf[1] * nf[2];
  if (idx >= ncell) return;
  int i = (int)(idx % nf[0]);
  long long r = idx / nf[0];
  int j = (int)(r % nf[1]);
  int k = (int)(r / nf[1]);
  int I = i >> 1, J = ndim > 1 ? j >> 1 : j, K = ndim > 2 ? k >> 1 : k;
  xf[idx] += xc[(long long)I + (long long)nc[0] * ((long long)J + (long long)nc[1] * K)];
}

// Coarsest level, one block: x = 0, then `sweeps` red-black Gauss-Seidel sweeps (or damped
// Jacobi when a periodic axis has odd length and the colouring does not close).
template <class T>
__global__ void k_coarse_solve(LevelDev<T> L, long long ncell, const T* __restrict__ invd, const T* __restrict__ r,
                               T* __restrict__ x, T* __restrict__ tmp, int sweeps, int use_rb) {
  for (long long c = threadIdx.x; c < ncell; c += blockDim.x) x[c] = T(0);
  __syncthreads();
  for (int s = 0; s < sweeps; ++s) {
    if (use_rb) {
      for (int color = 0; color < 2; ++color) {
        for (long long c = threadIdx.x; c < ncell; c += blockDim.x) {
          int i, j, k;
          unflatten(L.n, c, i, j, k);
          if (((i + j + k) & 1) != color) continue;
          T v = r[c];
          for_each_face(L, i, j, k, c, [&](T w, int kind, long long nb) {
            if (kind == kInterior) v += w * x[nb];
            else if (kind == kContinuous) v -= w * x[nb];
          });
          x[c] = v * invd[c];
        }
        __syncthreads();
      }
    } else {
      for (long long c = threadIdx.x; c < ncell; c += blockDim.x) {
        int i, j, k;
        unflatten(L.n, c, i, j, k);
        T v = r[c];
        for_each_face(L, i, j, k, c, [&](T w, int kind, long long nb) {
          if (kind == kInterior) v += w * x[nb];
          else if (kind == kContinuous) v -= w * x[nb];
        });
        tmp[c] = T(0.2) * x[c] + T(0.8) * v * invd[c];
      }
      __syncthreads();
      for (long long c = threadIdx.x; c < ncell; c += blockDim.x) x[c] = tmp[c];
      __syncthreads();
    }
  }
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
  nparts_ = 152 * 4;
  size_t bytes = 0;
  auto add = [&](size_t b) { bytes += (b + 511) & ~(size_t)255; };
  for (int a = 0; a < g.ndim; ++a) add(faces3(dims_[0], a) * sizeof(double));
  for (int k = 0; k < 3; ++k) add(N * sizeof(double));  // b, xa, xb
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
  xa_ = (double*)arena_.take(N * sizeof(double));
  xb_ = (double*)arena_.take(N * sizeof(double));
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
  if (!b64_ || !xa_ || !xb_ || !partials_ || !scal_) return cudaErrorMemoryAllocation;
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
    k_fine_setup<T><<<nblk(g_.ncell), kBlock, 0, s>>>(L64, g_, E_old, b64_, (T*)lv_[0].invd);
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
cudaError_t Multigrid::vcycle(int l, int nu1, int nu2, cudaStream_t s) {
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
    k_coarse_solve<T><<<1, 1024, 0, s>>>(L, ncell, invd, r, x, (T*)lv_[l].tmp, sweeps, rb ? 1 : 0);
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
  cudaError_t e = vcycle<T>(l + 1, nu1, nu2, s);
  if (e != cudaSuccess) return e;
  {
    TraceScope ts(l == 0 ? "prolong_L0" : "prolong_Lc", s);
    k_prolong<T><<<nblk(ncell), kBlock, 0, s>>>(n, g_.ndim, (const T*)lv_[l + 1].x, nc, x);
  }
  for (int it = 0; it < nu2; ++it) {
    {
      TraceScope ts(sm_name, s);
      k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1);
    }
    TraceScope ts(sm_name, s);
    k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t Multigrid::solve_t(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                               SolveStats* st, cudaStream_t s) {
  void* w64v[3] = {w64_[0], w64_[1], w64_[2]};
  LevelDev<double> L64 = level_dev<double>(g_, dims_[0], w64v);
  const double* x_in = E_old;
  double* bufs[2] = {xa_, xb_};
  int which = 0;
  const T* d = nullptr;
  double bb = 0.0;
  int cycles = 0;
  double rel = 0.0;
  int status = FLD_ERR_NOT_CONVERGED;
  for (int it = 0;; ++it) {
    double* x_out = bufs[which];
    {
      TraceScope ts("update_residual", s);
      k_update_residual<T><<<nparts_, kBlock, 0, s>>>(L64, g_.ncell, x_in, d, b64_, x_out, (T*)lv_[0].r, partials_);
    }
    {
      TraceScope ts("reduce", s);
      k_reduce<<<1, 1024, 0, s>>>(partials_, nparts_, scal_);
    }
    cudaError_t e = cudaMemcpyAsync(host_scal_, scal_, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    bb = host_scal_[1];
    double rr = host_scal_[0];
    rel = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
    x_in = x_out;
    which ^= 1;
    if (!(rel == rel) || rel > 1e300) {
      status = FLD_ERR_NONFINITE;
      break;
    }
    if (rel <= rtol) {
      status = FLD_OK;
      break;
    }
    if (cycles >= max_cycles) break;
    e = vcycle<T>(0, nu1, nu2, s);
    if (e != cudaSuccess) return e;
    d = (const T*)lv_[0].x;
    ++cycles;
  }
  if (x_in != E_new) {
    cudaError_t e = cudaMemcpyAsync(E_new, x_in, g_.ncell * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
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

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
#include <algorithm>
#include <cstdint>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "mg.h"
#include "df.cuh"
#include "mg_df.h"
#include "mg_device.cuh"
#include "sweep3d.h"
#include "trace.h"

namespace fld {

// Device state of the graph-driven solve (Multigrid::solve_async): the outer loop of solve_t kept
// on the device.  pending: what the last residual was (the double-float first residual, an exact
// residual, or a double-float update); kc_*: the kernels of each branch of the loop body.
struct Multigrid::SolveDev {
  double rtol, N;
  int max_cycles, mixed, fmg_start, idx32;
  int cycles, status, pending, updates, fp64_op;
  float scale;
  double rel, drift;
  unsigned long long kernels;
  unsigned long long kc_check, kc_fmg, kc_vcyc, kc_fp64, kc_add, kc_exact, kc_upd;
};

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

// With dhi/dlo (mixed solver): also the diagonal as a double-float for the residual updates.
template <class T>
__global__ void k_fine_setup(LevelDev<double> L, GridDev g, const double* __restrict__ E_old, double* __restrict__ b,
                             double* __restrict__ diag, T* __restrict__ invd, float* __restrict__ dhi,
                             float* __restrict__ dlo) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  fine_setup_cell<T>(L, g, E_old, idx, b, diag, invd);
  if (dhi) split_f64(diag[idx], dhi[idx], dlo[idx]);
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

// The same two kernels with 32-bit indices, the coordinates from divisions by invariant divisors
// (levels whose faces number fewer than 2^31 per axis); the face sum is taken in the same order.
template <class T>
__global__ void k_coarse_faces32(int a, int ndim, std::array<int, 3> nf, FastDiv d0, FastDiv d1, unsigned nfaces,
                                 const T* __restrict__ wf, T* __restrict__ wc) {
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nfaces) return;
  const unsigned r = fast_div(idx, d0), q2 = fast_div(r, d1);
  const int q[3] = {(int)(idx - r * d0.d), (int)(r - q2 * d1.d), (int)q2};
  int mf[3] = {nf[0], nf[1], nf[2]};
  mf[a] += 1;
  const int o1max = (ndim > 1) ? 2 : 1, o2max = (ndim > 2) ? 2 : 1;
  const int t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;  // the transverse axes
  T sum = T(0);
  for (int o2 = 0; o2 < o2max; ++o2)
    for (int o1 = 0; o1 < o1max; ++o1) {
      int f[3];
      f[a] = 2 * q[a];
      f[t1] = (t1 < ndim) ? 2 * q[t1] + o1 : q[t1];
      f[t2] = (t2 < ndim) ? 2 * q[t2] + o2 : q[t2];
      sum += wf[f[0] + mf[0] * (f[1] + mf[1] * f[2])];
    }
  wc[idx] = sum / (T)(4 * o1max * o2max);
}

// Faces of a transverse axis a (1 or 2) for FP32 levels with the fine nx a multiple of 4: each
// thread averages two adjacent coarse faces (I, I+1) from one float4 of fine faces per fine row
// (2 rows in 2-D, 4 in 3-D); coarse faces of axis a are rows of ncx values, fine ones rows of nx.
// d1 divides the coarse face row index by the coarse rows per plane of the axis's face layout.
template <int NDIM>
__global__ void k_coarse_faces_t4(int a, std::array<int, 3> nf, int ncx, FastDiv d1, unsigned npairs,
                                  const float* __restrict__ wf, float* __restrict__ wc) {
  const unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int nph = ncx >> 1;                     // pairs per coarse row
  const unsigned crow = p / (unsigned)nph;      // coarse face row: J + m1 * K in the face layout
  const int I2 = 2 * (int)(p - crow * (unsigned)nph);  // first of the two coarse faces
  const unsigned K = fast_div(crow, d1), J = crow - K * d1.d;
  // fine face layout of axis a: x fastest, then the axis-1 index (ny + 1 faces for a = 1), then z
  const int m1 = a == 1 ? nf[1] + 1 : nf[1];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int o1n = a == 1 ? 1 : 2, o2n = (NDIM == 3 && a == 1) ? 2 : 1;
  for (int o2 = 0; o2 < o2n; ++o2)
    for (int o1 = 0; o1 < o1n; ++o1) {
      // a = 1: fine (2I.., 2J, 2K + o2); a = 2: fine (2I.., 2J + o1, 2K)
      const int fj = a == 1 ? 2 * (int)J : 2 * (int)J + o1;
      const int fk = a == 1 ? (NDIM == 3 ? 2 * (int)K + o2 : 0) : 2 * (int)K;
      const float4 v = *reinterpret_cast<const float4*>(wf + 2 * I2 + nf[0] * (fj + m1 * fk));
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  const float inv = 1.0f / (float)(4 * 2 * o1n * o2n);
  *reinterpret_cast<float2*>(wc + I2 + ncx * crow) = make_float2((acc.x + acc.y) * inv, (acc.z + acc.w) * inv);
}

template <class T>
__global__ void k_invd32(LevelDev<T> L, FastDiv d0, FastDiv d1, unsigned ncell, T* __restrict__ invd) {
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncell) return;
  const unsigned r = fast_div(idx, d0), k = fast_div(r, d1);
  invd[idx] = T(1) / diag_of(L, (int)(idx - r * d0.d), (int)(r - k * d1.d), (int)k, idx);
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

// Both mixed-solver residual kernels walk whole x rows (one row per block iteration), so the
// division of a cell index into (i, j, k) happens once per row rather than once per cell.

// Mixed solver, exact outer residual: r = b - A x in FP64, stored as the double-float (rhi, rlo);
// rhi is the FP32 right-hand side of the next V-cycle.  parts: per-block sum of r^2.
__global__ void __launch_bounds__(256, 4) k_residual64_df(LevelDev<double> L, const double* x_in, double* x_out,
                                                          const double* __restrict__ b, const double* __restrict__ diag,
                                                          float* __restrict__ rhi, float* __restrict__ rlo,
                                                          double* __restrict__ parts) {
  const int nx = L.n[0], ny = L.n[1];
  const long long rows = (long long)ny * L.n[2];
  double acc = 0.0;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = (int)(row % ny), k = (int)(row / ny);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long idx = (long long)i + (long long)nx * row;
      const double xc = x_in[idx];
      double s = fma(-diag[idx], xc, b[idx]);
      for_each_face(L, i, j, k, idx, [&](double w, int kind, long long nb) {
        if (kind == kInterior) s = fma(w, x_in[nb], s);
        else if (kind == kContinuous) s = fma(-w, x_in[nb], s);
      });
      if (x_out != x_in) x_out[idx] = xc;
      split_f64(s, rhi[idx], rlo[idx]);
      acc = fma(s, s, acc);
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

// Mixed solver, updated outer residual after a V-cycle that computed the correction d:
//   x += d (FP64),  r_new = r_old - A d,
// in double-float arithmetic: A's weights and diagonal as hi + lo floats, d exact in FP32, every
// product exact (two_prod) and the sum carried as s + e.  The error per cell is a small multiple
// of 2^-48 m, m = |r_old| + diag |d| + sum |w d_nb|.  parts[blk] = sum (scale r_new)^2,
// parts[nparts + blk] = sum (scale m)^2, summed in FP32 per thread (they steer the iteration and
// bound its error; neither needs more digits).
// One face term of the update, branch-free (as wave_face): the neighbour (the cell itself where the
// face has none, with coefficient 0) and the sign (+1 interior or periodic, -1 extrapolated).
__device__ __forceinline__ void df_face(bool inside, int bc, int idx, int across, int wrap, int mirror, float whi,
                                        float wlo, const float* __restrict__ d, float& s, float& e, float& m) {
  const bool per = bc == FLD_BC_PERIODIC, cont = bc == FLD_BC_CONTINUOUS;
  const int nb = inside ? across : (per ? wrap : (cont ? mirror : idx));
  const float sg = (inside || per) ? 1.f : (cont ? -1.f : 0.f);
  const float xn = sg * d[nb];
  float t, te, s2, e2;
  two_prod(whi, xn, t, te);
  te = fmaf(wlo, xn, te);
  two_sum(s, t, s2, e2);
  s = s2;
  e += e2 + te;
  m += fabsf(t);
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_residual_update(LevelDev<float> L, LevelDev<float> Llo,
                                                         const float* __restrict__ dhi, const float* __restrict__ dlo,
                                                         const float* __restrict__ d, float* __restrict__ rhi,
                                                         float* __restrict__ rlo, double* __restrict__ x64, float scale,
                                                         const float* __restrict__ scale_p, int nparts,
                                                         double* __restrict__ parts) {
  // 32-bit indices: the caller guarantees fewer than 2^31 cells and faces per axis
  if (scale_p) scale = *scale_p;  // the graph-driven solve keeps the scale on the device
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int rows = ny * nz, sy = nx, sz = nx * ny;
  float ss = 0.f, mm = 0.f;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const int idx = i + nx * row;
      const float dc = d[idx];
      const float ro = rhi[idx];
      x64[idx] += (double)dc;  // the V-cycle's correction joins the FP64 iterate here
      // s + e = r_old - diag * dc
      float p, pe, s, e;
      two_prod(dhi[idx], dc, p, pe);
      pe = fmaf(dlo[idx], dc, pe);
      two_sum(ro, -p, s, e);
      e += rlo[idx] - pe;
      float m = fabsf(ro) + fabsf(p);
      const int fx = i + (nx + 1) * row;
      df_face(i > 0, L.bc[0], idx, idx - 1, idx + (nx - 1), idx + 1, L.w[0][fx], Llo.w[0][fx], d, s, e, m);
      df_face(i < nx - 1, L.bc[1], idx, idx + 1, idx - (nx - 1), idx - 1, L.w[0][fx + 1], Llo.w[0][fx + 1], d, s, e, m);
      if (NDIM >= 2) {
        const int fy = i + nx * (j + (ny + 1) * k);
        df_face(j > 0, L.bc[2], idx, idx - sy, idx + (ny - 1) * sy, idx + sy, L.w[1][fy], Llo.w[1][fy], d, s, e, m);
        df_face(j < ny - 1, L.bc[3], idx, idx + sy, idx - (ny - 1) * sy, idx - sy, L.w[1][fy + nx], Llo.w[1][fy + nx],
                d, s, e, m);
      }
      if (NDIM == 3) {
        df_face(k > 0, L.bc[4], idx, idx - sz, idx + (nz - 1) * sz, idx + sz, L.w[2][idx], Llo.w[2][idx], d, s, e, m);
        df_face(k < nz - 1, L.bc[5], idx, idx + sz, idx - (nz - 1) * sz, idx - sz, L.w[2][idx + sz],
                Llo.w[2][idx + sz], d, s, e, m);
      }
      float rh, rl;
      quick_two_sum(s, e, rh, rl);
      rhi[idx] = rh;
      rlo[idx] = rl;
      const float rs = rh * scale, ms = m * scale;
      ss = fmaf(rs, rs, ss);
      mm = fmaf(ms, ms, mm);
    }
  }
  const double bs = block_sum((double)ss);
  __syncthreads();  // block_sum's shared scratch is reused
  const double bm = block_sum((double)mm);
  if (threadIdx.x == 0) {
    parts[blockIdx.x] = bs;
    parts[nparts + blockIdx.x] = bm;
  }
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

// rc = mean of the 2^d children of each coarse cell (the full-multigrid start restricts the
// right-hand side itself down the hierarchy)
template <class T>
__global__ void k_restrict_avg(std::array<int, 3> nf, int ndim, const T* __restrict__ rf, std::array<int, 3> nc,
                               T* __restrict__ rc) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nc[0] * nc[1] * nc[2]) return;
  int I, J, K;
  unflatten(nc.data(), idx, I, J, K);
  const int o1 = ndim > 1 ? 2 : 1, o2 = ndim > 2 ? 2 : 1;
  T sum = T(0);
  for (int b = 0; b < o2; ++b)
    for (int a = 0; a < o1; ++a)
      for (int c = 0; c < 2; ++c) {
        const int i = 2 * I + c, j = ndim > 1 ? 2 * J + a : J, k = ndim > 2 ? 2 * K + b : K;
        sum += rf[cell_index(nf.data(), i, j, k)];
      }
  rc[idx] = sum / T(2 * o1 * o2);
}

// Row-wise restriction and prolongation for levels with long x rows (32-bit indices).  A block
// takes one coarse row (J, K); each thread owns fine x positions i and sums the residuals r - A x
// of its 2^(d-1) fine rows; lanes i and i^1 then add their sums (one shuffle) and the even lane
// writes the coarse cell.  The face terms are branch-free (selects), as in the wavefront sweep.
template <class T>
__device__ __forceinline__ void restrict_face(bool inside, int bc, int idx, int across, int wrap, int mirror, T w, T xv,
                                              const T* __restrict__ x, T& ax) {
  const bool per = bc == FLD_BC_PERIODIC, cont = bc == FLD_BC_CONTINUOUS, dir = bc == FLD_BC_DIRICHLET;
  const int nb = inside ? across : (per ? wrap : (cont ? mirror : idx));
  const T cx = (inside || per || dir) ? T(1) : (cont ? T(-1) : T(0));
  const T cn = (inside || per) ? T(1) : (cont ? T(-1) : T(0));
  ax = fma(w, cx * xv - cn * x[nb], ax);
}

// Three blocks per SM (up to 80 registers): with the loads of all 2^(d-1) fine rows in flight at
// once the kernel runs 1.6x faster than at four blocks and 64 registers.
template <class T, int NDIM>
__global__ void __launch_bounds__(256, 3) k_restrict_rows(LevelDev<T> F, const T* __restrict__ rf, const T* __restrict__ xf,
                                                       int ncy, int crows, T* __restrict__ rc) {
  const int nx = F.n[0], ny = F.n[1], nz = F.n[2];
  const int sy = nx, sz = nx * ny, ncx = nx >> 1;
  const int iters = (nx + blockDim.x - 1) / blockDim.x;
  for (int crow = blockIdx.x; crow < crows; crow += gridDim.x) {
    const int J = NDIM > 1 ? crow % ncy : 0, K = NDIM > 2 ? crow / ncy : 0;
    for (int it = 0; it < iters; ++it) {
      const int i0 = it * blockDim.x + threadIdx.x;
      const int i = min(i0, nx - 1);
      T acc = T(0);
#pragma unroll
      for (int o = 0; o < (1 << (NDIM - 1)); ++o) {
        const int j = NDIM > 1 ? 2 * J + (o & 1) : 0;
        const int k = NDIM > 2 ? 2 * K + (o >> 1) : 0;
        const int idx = i + sy * j + sz * k;
        const T xv = xf[idx];
        T ax = xv;
        const int fx = i + (nx + 1) * (j + ny * k);
        restrict_face<T>(i > 0, F.bc[0], idx, idx - 1, idx + (nx - 1), idx + 1, F.w[0][fx], xv, xf, ax);
        restrict_face<T>(i < nx - 1, F.bc[1], idx, idx + 1, idx - (nx - 1), idx - 1, F.w[0][fx + 1], xv, xf, ax);
        if (NDIM >= 2) {
          const int fy = i + nx * (j + (ny + 1) * k);
          restrict_face<T>(j > 0, F.bc[2], idx, idx - sy, idx + (ny - 1) * sy, idx + sy, F.w[1][fy], xv, xf, ax);
          restrict_face<T>(j < ny - 1, F.bc[3], idx, idx + sy, idx - (ny - 1) * sy, idx - sy, F.w[1][fy + nx], xv, xf,
                           ax);
        }
        if (NDIM == 3) {
          restrict_face<T>(k > 0, F.bc[4], idx, idx - sz, idx + (nz - 1) * sz, idx + sz, F.w[2][idx], xv, xf, ax);
          restrict_face<T>(k < nz - 1, F.bc[5], idx, idx + sz, idx - (nz - 1) * sz, idx - sz, F.w[2][idx + sz], xv, xf,
                           ax);
        }
        acc += rf[idx] - ax;
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (!(i0 & 1) && i0 < nx) rc[(i0 >> 1) + ncx * crow] = acc * T(1.0 / (1 << NDIM));
    }
  }
}

// xf += P xc (piecewise constant), or xf = P xc with ASSIGN (the FMG's start on a finer level),
// one fine row per block iteration
template <class T, int NDIM, bool ASSIGN = false>
__global__ void __launch_bounds__(256) k_prolong_rows(int nx, int ny, int rows, const T* __restrict__ xc, int ncy,
                                                      T* __restrict__ xf) {
  const int ncx = nx >> 1;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    const int crow = NDIM == 3 ? (j >> 1) + ncy * (k >> 1) : (NDIM == 2 ? (j >> 1) : 0);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      if (ASSIGN) xf[i + nx * row] = xc[(i >> 1) + ncx * crow];
      else xf[i + nx * row] += xc[(i >> 1) + ncx * crow];
    }
  }
}

// The same for FP32 levels with nx a multiple of 4: each thread takes four fine cells (one float4
// of xf from one float2 of xc) and four such quads per iteration, loads first, so that the memory
// accesses are wide and several are in flight.  32-bit indices (rows * nx < 2^31).
template <int NDIM, bool ASSIGN>
__global__ void __launch_bounds__(256) k_prolong_rows4(int nx, int ny, int rows, const float* __restrict__ xc,
                                                       int ncy, float* __restrict__ xf) {
  constexpr int U = 4;
  const int nq = nx >> 2, ncx = nx >> 1;
  const int total = rows * nq;
  const int stride = (int)(gridDim.x * blockDim.x);
  for (int q0 = (int)(blockIdx.x * blockDim.x + threadIdx.x); q0 < total; q0 += U * stride) {
    float2 c[U];
    float4 f[U];
    int row[U], iq[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = min(q0 + u * stride, total - 1);
      row[u] = q / nq;
      iq[u] = q - row[u] * nq;
      const int j = row[u] % ny, k = row[u] / ny;
      const int crow = NDIM == 3 ? (j >> 1) + ncy * (k >> 1) : (j >> 1);
      c[u] = reinterpret_cast<const float2*>(xc + ncx * crow)[iq[u]];
      if (!ASSIGN) f[u] = reinterpret_cast<const float4*>(xf + nx * row[u])[iq[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (q0 + u * stride >= total) continue;
      float4 v = make_float4(c[u].x, c[u].x, c[u].y, c[u].y);
      if (!ASSIGN) v = make_float4(f[u].x + v.x, f[u].y + v.y, f[u].z + v.z, f[u].w + v.w);
      reinterpret_cast<float4*>(xf + nx * row[u])[iq[u]] = v;
    }
  }
}

template <class T>
__global__ void k_prolong(std::array<int, 3> nf, int ndim, const T* __restrict__ xc, std::array<int, 3> nc,
                          T* __restrict__ xf) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nf[0] * nf[1] * nf[2]) return;
  prolong_cell<T>(nf.data(), ndim, xc, nc.data(), xf, idx);
}

// The coarsest level, one block.  With in_smem the iterate (and the Jacobi scratch) live in shared
// memory: the sweeps are a chain of block barriers, and each round trip through global memory
// would otherwise set their pace.
template <class T>
__global__ void __launch_bounds__(512, 1) k_coarse_solve(LevelDev<T> L, long long ncell, const T* __restrict__ invd,
                                                      const T* __restrict__ r, T* __restrict__ x, T* __restrict__ tmp,
                                                      int sweeps, int use_rb, int in_smem) {
  extern __shared__ __align__(16) unsigned char coarse_smem[];
  if (in_smem) {
    T* xs = reinterpret_cast<T*>(coarse_smem);
    if (ncell <= (long long)blockDim.x) coarse_solve_small<T>(L, (int)ncell, invd, r, xs, xs + ncell, sweeps, use_rb);
    else coarse_solve_block<T>(L, ncell, invd, r, xs, xs + ncell, sweeps, use_rb);
    __syncthreads();
    for (long long c = threadIdx.x; c < ncell; c += blockDim.x) x[c] = xs[c];
  } else {
    coarse_solve_block<T>(L, ncell, invd, r, x, tmp, sweeps, use_rb);
  }
}


// ----------------------------------------------------------------------------- wavefront sweeps
//
// One launch performs a full red-black sweep (colour c0, then the other colour) on a large 3-D
// level in one pass over HBM.  The work is cut into items (half-sweep h in {0, 1}, z-plane k,
// chunk of rows); blocks take items in ticket order from an atomic counter.  Item (1, k) may start
// once (0, k-1), (0, k) and (0, k+1) are finished -- the values it reads are final and the values
// it overwrites have been read.  The host orders the tickets so that half-sweep 1 trails
// half-sweep 0 by `skew` planes: the planes it revisits are still in L2, and its dependencies were
// handed out long before, so blocks rarely wait.  A block only ever waits for smaller tickets,
// which running blocks hold, so the scheme cannot deadlock; every wait is bounded all the same
// and sets the error word when it runs out.  Ordering: the compute warps' stores, a barrier among
// them, then one of them increments the plane's counter with release semantics; a dependent
// block's scheduling thread observes the counters and fences (acquire), and the block barrier
// orders its compute warps' reads after that.
// The arithmetic per cell is the one of k_smooth, so the result equals two k_smooth launches.
constexpr int kWaveThreads = 256;
constexpr int kWaveCompute = kWaveThreads - 32;  // warps 1..7 compute, warp 0 schedules
constexpr int kWaveUnroll = 4;
constexpr int kWaveItem = 2 * kWaveCompute * kWaveUnroll;  // colour cells per item (rows of a plane)
constexpr long long kWaveSpinLimit = 1LL << 21;  // with up to 1 us sleeps: about two seconds

struct WaveDev {
  const int* order;
  unsigned* ctl;
  int nchunk, rows;
  unsigned total;
};

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until the previous half-sweep has finished planes k-1, k and k+1 (on a bounded z
// axis the missing neighbour is replaced by k itself), then fence: the relaxed reads and the fence
// form an acquire, and the block barrier that follows extends it to the other threads.
__device__ __forceinline__ bool wave_wait(unsigned* ctl, const unsigned* done_prev, int k, int nz, bool periodic, unsigned target) {
  const int km = k > 0 ? k - 1 : (periodic ? nz - 1 : k);
  const int kp = k < nz - 1 ? k + 1 : (periodic ? 0 : k);
  unsigned ns = 32;
  for (long long it = 0;; ++it) {
    const unsigned a = ld_relaxed_gpu(done_prev + km), b = ld_relaxed_gpu(done_prev + k),
                   c = ld_relaxed_gpu(done_prev + kp);
    if (a >= target && b >= target && c >= target) break;
    if (it > kWaveSpinLimit || *(volatile unsigned*)ctl != 0u) {
      atomicOr(ctl, 1u);
      return false;
    }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return true;
}

// One face of a cell, branch-free: the cell across it (the cell itself where the face has none, so
// that the load stays valid), cv multiplying w x_nb in the sum and cd multiplying w in the diagonal:
// interior or periodic (+1, +1), Dirichlet ghost (0, +1), Neumann (0, 0), linear extrapolation
// (-1, -1) -- the same terms, in the same order and rounding, as for_each_face in k_smooth.
template <class T>
__device__ __forceinline__ void wave_face(bool inside, int bc, int idx, int across, int wrap, int mirror, T w, const T* x,
                                          T& a, T& d) {
  const bool per = bc == FLD_BC_PERIODIC, cont = bc == FLD_BC_CONTINUOUS, dir = bc == FLD_BC_DIRICHLET;
  const int nb = inside ? across : (per ? wrap : (cont ? mirror : idx));
  const T cv = (inside || per) ? T(1) : (cont ? T(-1) : T(0));
  const T cd = (inside || per || dir) ? T(1) : (cont ? T(-1) : T(0));
  a = fma(cv * w, x[nb], a);
  d = fma(cd, w, d);
}

// New value of cell (i, j, k) of a 3-D level (32-bit indices: the level has fewer than 2^31 cells
// and faces per axis).
template <class T>
__device__ __forceinline__ T wave_cell(const LevelDev<T>& L, const T* __restrict__ invd, const T* __restrict__ r,
                                       const T* x, int i, int j, int k, bool zero) {
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int sy = nx, sz = nx * ny;
  const int idx = i + sy * j + sz * k;
  T a = r[idx];
  if (zero) return a * invd[idx];
  T d = T(1);
  const int fx = i + (nx + 1) * (j + ny * k);
  const int fy = i + nx * (j + (ny + 1) * k);
  wave_face<T>(i > 0, L.bc[0], idx, idx - 1, idx + (nx - 1), idx + 1, L.w[0][fx], x, a, d);
  wave_face<T>(i < nx - 1, L.bc[1], idx, idx + 1, idx - (nx - 1), idx - 1, L.w[0][fx + 1], x, a, d);
  wave_face<T>(j > 0, L.bc[2], idx, idx - sy, idx + (ny - 1) * sy, idx + sy, L.w[1][fy], x, a, d);
  wave_face<T>(j < ny - 1, L.bc[3], idx, idx + sy, idx - (ny - 1) * sy, idx - sy, L.w[1][fy + nx], x, a, d);
  wave_face<T>(k > 0, L.bc[4], idx, idx - sz, idx + (nz - 1) * sz, idx + sz, L.w[2][idx], x, a, d);
  wave_face<T>(k < nz - 1, L.bc[5], idx, idx + sz, idx - (nz - 1) * sz, idx - sz, L.w[2][idx + sz], x, a, d);
  if constexpr (sizeof(T) == sizeof(float)) return __fdividef(a, d);
  else return a * invd[idx];
}

template <class T, bool ZERO, bool UPDATE>
__global__ void __launch_bounds__(kWaveThreads, 4) k_wave_sweep(LevelDev<T> L, const T* __restrict__ invd,
                                                                const T* __restrict__ r, T* x, int c0,
                                                                double* __restrict__ x64, WaveDev W) {
  // Warp 0 is the control warp: its thread 0 takes the next ticket and waits for that item's
  // dependencies while warps 1..7 compute the current item; the ticket is handed over at the block
  // barrier.  The compute warps publish their own item's completion (a barrier among themselves,
  // then a release increment), so a completion never waits on a control warp.
  __shared__ unsigned s_ticket[2];
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int nxh = (nx + 1) >> 1;
  const bool zper = L.bc[4] == FLD_BC_PERIODIC;
  unsigned* done = W.ctl + 2;
  const int ct = (int)threadIdx.x - 32;  // compute thread, 0 .. kWaveCompute - 1
  auto take = [&]() -> unsigned {
    unsigned t = atomicAdd(W.ctl + 1, 1u);
    if (t < W.total) {
      const int g = (int)(t / (unsigned)W.nchunk);
      const int h = W.order[2 * g], k = W.order[2 * g + 1];
      if (h > 0 && !wave_wait(W.ctl, done + (h - 1) * nz, k, nz, zper, (unsigned)W.nchunk)) t = W.total;
    }
    return t;
  };
  if (threadIdx.x == 0) s_ticket[0] = take();
  for (int cur = 0;; cur ^= 1) {
    __syncthreads();
    const unsigned t = s_ticket[cur];
    if (t >= W.total) return;
    if (ct < 0) {
      if (threadIdx.x == 0) s_ticket[cur ^ 1] = take();
      continue;
    }
    const int g = (int)(t / (unsigned)W.nchunk);
    const int h = W.order[2 * g], k = W.order[2 * g + 1];
    const int colour = c0 ^ h;
    const int j0 = (int)(t % (unsigned)W.nchunk) * W.rows;
    const int cells = (min(ny, j0 + W.rows) - j0) * nxh;
    const bool zero = ZERO && h == 0;
    constexpr int U = sizeof(T) == sizeof(float) ? kWaveUnroll : kWaveUnroll / 2;  // FP64: registers
    for (int base = 0; base < cells; base += kWaveCompute * U) {
      T v[U];
      int id[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        // branch-free, so that the loads of all U cells are in flight together; a slot
        // past the end of the item computes a valid cell and skips the store
        const int q = base + u * kWaveCompute + ct;
        const int qq = min(q, cells - 1);
        const int j = j0 + qq / nxh;
        int i = 2 * (qq % nxh) + ((colour + j + k) & 1);
        ok[u] = q < cells && i < nx;
        i = min(i, nx - 1);
        v[u] = wave_cell<T>(L, invd, r, x, i, j, k, zero);
        id[u] = i + nx * (j + ny * k);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        x[id[u]] = v[u];
        if (UPDATE) x64[id[u]] += (double)v[u];
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kWaveCompute) : "memory");
    if (ct == 0) red_release_gpu_add(done + h * nz + k, 1u);
  }
}

// ----------------------------------------------------------------------------- host side

static inline unsigned nblk(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

Multigrid::~Multigrid() {
  drop_graphs();
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
  for (cudaStream_t b : body_s_)
    if (b) cudaStreamDestroy(b);
  if (out_h_) cudaFreeHost(out_h_);
  if (host_scal_) cudaFreeHost(host_scal_);
  if (tune_x_) cudaFree(tune_x_);
}

void Multigrid::drop_graphs() {
  for (auto& g : graphs_) cudaGraphExecDestroy(g.exec);
  graphs_.clear();
  if (sexec_) cudaGraphExecDestroy(sexec_);
  sexec_ = nullptr;
}

static inline long long cells3(const std::array<int, 3>& n) { return (long long)n[0] * n[1] * n[2]; }

template <class T>
static LevelDev<T> level_dev(const GridDev& g, const std::array<int, 3>& n, void* const w[3]) {
  LevelDev<T> L;
  for (int a = 0; a < 3; ++a) L.n[a] = n[a];
  L.ndim = g.ndim;
  for (int f = 0; f < 6; ++f) L.bc[f] = g.bc[f];
  for (int a = 0; a < 3; ++a) L.w[a] = (const T*)w[a];
  return L;
}

static inline long long faces3(const std::array<int, 3>& n, int a) {
  long long c = 1;
  for (int b = 0; b < 3; ++b) c *= (b == a) ? n[b] + 1 : n[b];
  return c;
}

// Levels that take the wavefront sweep: 3-D and too large to stay in L2 between two passes
// (4 Mi cells; FLD_WAVE_MIN_CELLS overrides the threshold).
static long long wave_min_cells() {
  const char* v = getenv("FLD_WAVE_MIN_CELLS");
  return v ? std::max(1LL, atoll(v)) : (1LL << 22);
}

static bool wave_eligible(const GridDev& g, const std::array<int, 3>& n) {
  const long long faces_x = (long long)(n[0] + 1) * n[1] * n[2];
  return g.ndim == 3 && cells3(n) >= wave_min_cells() && n[2] >= 4 && faces_x < (1LL << 31) &&
         (long long)n[0] * (n[1] + 1) * n[2] < (1LL << 31) && (long long)n[0] * n[1] * (n[2] + 1) < (1LL << 31);
}

// The mixed solver's finest level takes the tiled sweep when it is 3-D, of a shape the tiles
// cover, and at least 1 Mi cells (FLD_SWEEP3D_MIN_CELLS overrides the threshold; FLD_SWEEP3D=0
// turns the tiled sweep off).
static bool tiled_level(const GridDev& g, const std::array<int, 3>& n) {
  const char* off = getenv("FLD_SWEEP3D");
  if (off && off[0] == '0') return false;
  const char* v = getenv("FLD_SWEEP3D_MIN_CELLS");
  const long long min_cells = v ? std::max(0LL, atoll(v)) : (1LL << 20);
  return g.ndim == 3 && cells3(n) >= min_cells && sweep3d_eligible(n[0], n[1], n[2]);
}

// Ticket order of the (half-sweep, plane) groups.  Half-sweep 1 trails half-sweep 0 by `skew`
// positions.  On a periodic z axis the planes are visited folded (0, nz-1, 1, nz-2, ...), which
// puts every pair of ring neighbours, the wrap-around pair included, within two positions.
static std::vector<int> wave_order(int nz, bool periodic, int skew) {
  const int sk = std::max(skew, periodic ? 2 : 1);
  auto plane = [&](int p) { return periodic ? ((p & 1) ? nz - 1 - (p >> 1) : (p >> 1)) : p; };
  std::vector<int> o;
  o.reserve(4 * (size_t)nz);
  for (int t = 0; t < nz + sk; ++t)
    for (int h = 0; h < 2; ++h) {
      const int p = t - sk * h;
      if (p >= 0 && p < nz) {
        o.push_back(h);
        o.push_back(plane(p));
      }
    }
  return o;
}

cudaError_t Multigrid::configure_wave() {
  wave_.assign(dims_.size(), WaveLevel{});
  wave_ctl_ = (unsigned*)arena_.take((2 + 2 * (size_t)dims_[0][2]) * sizeof(unsigned));
  if (!wave_ctl_) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemset(wave_ctl_, 0, (2 + 2 * (size_t)dims_[0][2]) * sizeof(unsigned));
  if (e != cudaSuccess) return e;
  const char* skew_env = getenv("FLD_WAVE_SKEW");
  for (size_t l = 0; l < dims_.size(); ++l) {
    const std::array<int, 3>& n = dims_[l];
    if (!wave_eligible(g_, n)) continue;
    WaveLevel& W = wave_[l];
    const int nxh = (n[0] + 1) / 2;
    W.rows = std::max(1, kWaveItem / nxh);
    W.nchunk = (n[1] + W.rows - 1) / W.rows;
    // half-sweep 1 trails by about 2 Mi cells' worth of planes: far enough (in tickets) that its
    // dependencies are done when it starts, near enough that those planes are still in L2
    const long long plane = (long long)n[0] * n[1];
    const int skew = skew_env ? std::max(1, atoi(skew_env)) : (int)std::max(2LL, ((1LL << 21) + plane - 1) / plane);
    std::vector<int> o = wave_order(n[2], g_.bc[4] == FLD_BC_PERIODIC, skew);
    W.order = (int*)arena_.take(o.size() * sizeof(int));
    if (!W.order) return cudaErrorMemoryAllocation;
    e = cudaMemcpy(W.order, o.data(), o.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  if (!wave_blocks_[0]) {
    int dev = 0, sms = 0, bf = 0, bd = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_wave_sweep<float, false, true>, kWaveThreads, 0);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_wave_sweep<double, false, true>, kWaveThreads, 0);
    if (e != cudaSuccess) return e;
    wave_blocks_[0] = std::max(1, bf) * sms;
    wave_blocks_[1] = std::max(1, bd) * sms;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t Multigrid::wave_sweep(int l, bool zero, int c0, double* x64, cudaStream_t s) {
  const std::array<int, 3>& n = dims_[l];
  const WaveLevel& W = wave_[l];
  cudaError_t e = cudaMemsetAsync(wave_ctl_ + 1, 0, (1 + 2 * (size_t)n[2]) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  WaveDev d{W.order, wave_ctl_, W.nchunk, W.rows, (unsigned)(2LL * n[2] * W.nchunk)};
  LevelDev<T> L = level_dev<T>(g_, n, lv_[l].w);
  const unsigned grid = std::min<unsigned>(d.total, (unsigned)wave_blocks_[sizeof(T) == sizeof(float) ? 0 : 1]);
  const T* invd = (const T*)lv_[l].invd;
  const T* r = (const T*)lv_[l].r;
  T* x = (T*)lv_[l].x;
  if (zero) note_launch(), k_wave_sweep<T, true, false><<<grid, kWaveThreads, 0, s>>>(L, invd, r, x, c0, nullptr, d);
  else if (x64) note_launch(), k_wave_sweep<T, false, true><<<grid, kWaveThreads, 0, s>>>(L, invd, r, x, c0, x64, d);
  else note_launch(), k_wave_sweep<T, false, false><<<grid, kWaveThreads, 0, s>>>(L, invd, r, x, c0, nullptr, d);
  return cudaGetLastError();
}

template <class T>
cudaError_t Multigrid::tiled_sweep(bool zero, int c0, double* x64, cudaStream_t s) {
  const std::array<int, 3>& n = dims_[0];
  Sweep3dArgs a{};
  a.nx = n[0];
  a.ny = n[1];
  a.nz = n[2];
  for (int f = 0; f < 6; ++f) a.bc[f] = g_.bc[f];
  for (int ax = 0; ax < 3; ++ax) a.ra[ax] = (float)(g_.inv_dx2[ax] / g_.inv_dx2[0]);
  a.dc = dc32_;
  a.r = (const float*)lv_[0].r;
  a.xin = zero ? nullptr : (const float*)lv_[0].x;
  a.xout = (float*)lv_[0].tmp;
  // the sweep adds its result to x64 in 16-byte accesses; other alignments add it afterwards
  const bool aligned = ((uintptr_t)x64 & 15u) == 0;
  a.x64 = aligned ? x64 : nullptr;
  a.c0 = c0;
  a.err = wave_ctl_;  // the solve loop turns a bounded wait that ran out into FLD_ERR_DEVICE_TIMEOUT
  cudaError_t e = launch_sweep3d(a, s);
  std::swap(lv_[0].x, lv_[0].tmp);  // the iterate now lives in the other array
  if (e == cudaSuccess && x64 && !aligned)
    note_launch(), k_add_correction<T><<<nblk(g_.ncell), kBlock, 0, s>>>(g_.ncell, (const T*)lv_[0].x, x64);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t Multigrid::configure(const GridDev& g, int precision) {
  bool same = configured_ && precision == precision_ && g.ndim == g_.ndim;
  for (int a = 0; a < 3 && same; ++a) same = g.n[a] == g_.n[a];
  for (int f = 0; f < 6 && same; ++f) same = g.bc[f] == g_.bc[f];
  g_ = g;  // dx and bc values may change freely
  if (same) return cudaSuccess;
  configured_ = false;
  tuned_.clear();
  drop_graphs();
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
  add(3 * nparts_ * sizeof(double));
  add(8 * sizeof(double));
  const bool df = precision == FLD_PREC_MIXED;  // double-float residual updates
  if (df) {
    for (int a = 0; a < g.ndim; ++a) add(faces3(dims_[0], a) * sizeof(float));  // weights, low parts
    for (int k = 0; k < 3; ++k) add(N * sizeof(float));                           // diag hi, lo; r lo
    add(sizeof(unsigned));
  }
  const bool tiled = df && tiled_level(g, dims_[0]);
  if (tiled) add(N * sizeof(float));  // dt D / dx_0^2 of the tiled sweep
  for (size_t l = 0; l < dims_.size(); ++l) {
    long long n = cells3(dims_[l]);
    if (l > 0 || precision == FLD_PREC_MIXED)
      for (int a = 0; a < g.ndim; ++a) add(faces3(dims_[l], a) * es);
    for (int k = 0; k < 4; ++k) add(n * es);  // invd, x, r, tmp
    if (wave_eligible(g, dims_[l])) add(4 * (size_t)dims_[l][2] * sizeof(int));
  }
  add((2 + 2 * (size_t)dims_[0][2]) * sizeof(unsigned));
  add(sizeof(SolveDev));
  cudaError_t e = arena_.reserve(bytes + 4096);
  if (e != cudaSuccess) return e;
  for (int a = 0; a < 3; ++a) w64_[a] = a < g.ndim ? (double*)arena_.take(faces3(dims_[0], a) * sizeof(double)) : nullptr;
  b64_ = (double*)arena_.take(N * sizeof(double));
  diag64_ = (double*)arena_.take(N * sizeof(double));
  partials_ = (double*)arena_.take(3 * nparts_ * sizeof(double));
  scal_ = (double*)arena_.take(8 * sizeof(double));
  if (!host_scal_) {
    e = cudaMallocHost(&host_scal_, 8 * sizeof(double));
    if (e != cudaSuccess) return e;
  }
  for (int a = 0; a < 3; ++a) w32lo_[a] = nullptr;
  dhi_ = dlo_ = rlo_ = nullptr;
  df_flag_ = nullptr;
  if (df) {
    for (int a = 0; a < g.ndim; ++a)
      if (!(w32lo_[a] = (float*)arena_.take(faces3(dims_[0], a) * sizeof(float)))) return cudaErrorMemoryAllocation;
    dhi_ = (float*)arena_.take(N * sizeof(float));
    dlo_ = (float*)arena_.take(N * sizeof(float));
    rlo_ = (float*)arena_.take(N * sizeof(float));
    df_flag_ = (unsigned*)arena_.take(sizeof(unsigned));
    if (!dhi_ || !dlo_ || !rlo_ || !df_flag_) return cudaErrorMemoryAllocation;
  }
  dc32_ = nullptr;
  if (tiled && !(dc32_ = (float*)arena_.take(N * sizeof(float)))) return cudaErrorMemoryAllocation;
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
  if (!(sd_ = (SolveDev*)arena_.take(sizeof(SolveDev)))) return cudaErrorMemoryAllocation;
  e = configure_wave();
  if (e != cudaSuccess) return e;
  configured_ = true;
  return cudaSuccess;
}


template <class T>
cudaError_t Multigrid::fp64_operator(cudaStream_t s) {
  float* w32[3] = {nullptr, nullptr, nullptr};
  if (precision_ == FLD_PREC_MIXED)
    for (int a = 0; a < g_.ndim; ++a) w32[a] = (float*)lv_[0].w[a];
  cudaError_t e = launch_faces(g_, dt_, D_ax_, w64_, w32, dhi_ ? w32lo_ : nullptr, s);
  if (e != cudaSuccess) return e;
  if (tiled_) {
    e = launch_dcell32(g_.ncell, dt_ * g_.inv_dx2[0], D_ax_[0], dc32_, s);
    if (e != cudaSuccess) return e;
  }
  void* w64v[3] = {w64_[0], w64_[1], w64_[2]};
  LevelDev<double> L64 = level_dev<double>(g_, dims_[0], w64v);
  {
    TraceScope ts("fine_setup", s);
    note_launch(),
        k_fine_setup<T><<<nblk(g_.ncell), kBlock, 0, s>>>(L64, g_, E_old_, b64_, diag64_, (T*)lv_[0].invd, dhi_, dlo_);
  }
  {
    TraceScope ts("norm_b", s);
    const int gs = front_grid((const void*)k_sumsq, nparts_);
    note_launch(), k_sumsq<<<gs, kBlock, 0, s>>>(b64_, g_.ncell, partials_);
    note_launch(), k_reduce<<<1, 1024, 0, s>>>(partials_, gs, scal_ + 1);
  }
  fp64_op_ = true;
  return cudaGetLastError();
}

template <class T>
cudaError_t Multigrid::setup_t(double dt, const double* const D_cell[3], const double* E_old, double rtol,
                               cudaStream_t s) {
  dt_ = dt;
  for (int a = 0; a < 3; ++a) D_ax_[a] = D_cell[a];
  E_old_ = E_old;
  fp64_op_ = false;
  // double-float setup: mixed solver, a tolerance the certified updates reach, one scalar D,
  // 32-bit indices
  long long maxf = g_.ncell;
  for (int a = 0; a < g_.ndim; ++a) maxf = std::max(maxf, faces3(dims_[0], a));
  df_mode_ = sizeof(T) == sizeof(float) && dhi_ != nullptr && rtol >= 1e-10 && D_cell[1] == D_cell[0] &&
             D_cell[2] == D_cell[0] && maxf < (1LL << 31);
  // the tiled finest-level sweep needs one scalar D (it forms the face means from dc32_)
  tiled_ = sizeof(T) == sizeof(float) && dc32_ != nullptr && D_cell[1] == D_cell[0] && D_cell[2] == D_cell[0];
  cudaError_t e;
  if (df_mode_) {
    e = cudaMemsetAsync(df_flag_, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const DfConst K = make_df_const(g_, dt);
    float* w32[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < g_.ndim; ++a) w32[a] = (float*)lv_[0].w[a];
    // the diagonal, 1/diag and b follow in the first residual's pass (solve_t)
    e = launch_faces_df(g_, K, D_cell[0], w32, w32lo_, tiled_ ? dc32_ : nullptr, df_flag_, s);
    if (e != cudaSuccess) return e;
  } else {
    e = fp64_operator<T>(s);
    if (e != cudaSuccess) return e;
  }
  for (size_t l = 1; l < dims_.size(); ++l) {
    TraceScope ts("coarse_setup", s);
    for (int a = 0; a < g_.ndim; ++a) {
      std::array<int, 3> m = dims_[l];
      m[a] += 1;
      const bool small = faces3(dims_[l - 1], a) < (1LL << 31);
      if (sizeof(T) == sizeof(float) && a > 0 && dims_[l - 1][0] % 4 == 0 && small) {
        const unsigned npairs = (unsigned)(faces3(dims_[l], a) / 2);
        if (g_.ndim == 3)
          note_launch(),
              k_coarse_faces_t4<3><<<nblk(npairs), kBlock, 0, s>>>(a, dims_[l - 1], m[0], make_fastdiv((unsigned)m[1]),
                                                                   npairs, (const float*)lv_[l - 1].w[a],
                                                                   (float*)lv_[l].w[a]);
        else
          note_launch(),
              k_coarse_faces_t4<2><<<nblk(npairs), kBlock, 0, s>>>(a, dims_[l - 1], m[0], make_fastdiv((unsigned)m[1]),
                                                                   npairs, (const float*)lv_[l - 1].w[a],
                                                                   (float*)lv_[l].w[a]);
      } else if (small)
        note_launch(), k_coarse_faces32<T><<<nblk(faces3(dims_[l], a)), kBlock, 0, s>>>(
                           a, g_.ndim, dims_[l - 1], make_fastdiv((unsigned)m[0]), make_fastdiv((unsigned)m[1]),
                           (unsigned)faces3(dims_[l], a), (const T*)lv_[l - 1].w[a], (T*)lv_[l].w[a]);
      else
        note_launch(),
            k_coarse_faces<T><<<nblk(faces3(dims_[l], a)), kBlock, 0, s>>>(a, g_.ndim, dims_[l - 1], dims_[l],
                                                                            (const T*)lv_[l - 1].w[a], (T*)lv_[l].w[a]);
    }
    LevelDev<T> L = level_dev<T>(g_, dims_[l], lv_[l].w);
    if (cells3(dims_[l]) < (1LL << 31))
      note_launch(),
          k_invd32<T><<<nblk(cells3(dims_[l])), kBlock, 0, s>>>(L, make_fastdiv((unsigned)dims_[l][0]),
                                                                 make_fastdiv((unsigned)dims_[l][1]),
                                                                 (unsigned)cells3(dims_[l]), (T*)lv_[l].invd);
    else
      note_launch(), k_invd<T><<<nblk(cells3(dims_[l])), kBlock, 0, s>>>(L, cells3(dims_[l]), (T*)lv_[l].invd);
  }
  return cudaGetLastError();
}

cudaError_t Multigrid::setup(double dt, const double* const D_cell[3], const double* E_old, double rtol,
                             unsigned* status, cudaStream_t s) {
  (void)status;
  return precision_ == FLD_PREC_MIXED ? setup_t<float>(dt, D_cell, E_old, rtol, s)
                                      : setup_t<double>(dt, D_cell, E_old, rtol, s);
}

// Levels that take the row-wise transfer kernels: 2-D or 3-D, rows of at least 128 cells (the
// kernels work on whole rows), 32-bit indices.
bool Multigrid::rows_ok(int l) const {
  const std::array<int, 3>& n = dims_[l];
  long long mf = cells3(n);
  for (int a = 0; a < g_.ndim; ++a) mf = std::max(mf, faces3(n, a));
  return g_.ndim >= 2 && n[0] >= 128 && mf < (1LL << 31);
}

template <class T>
cudaError_t Multigrid::vcycle(int l, int nu1, int nu2, double* x64, cudaStream_t s, bool zero_init) {
  // graphs: the levels without a wavefront sweep, below the finest, when no FP64 iterate is
  // updated and the per-launch trace is off (its events are host-side bookkeeping)
  const bool graph = graphs_ok_ && !capturing_ && l > 0 && wave_[l].order == nullptr && x64 == nullptr &&
                     !(tracer().on && !tracer().major_only);
  if (graph) {
    cudaError_t e = vcycle_graph<T>(l, nu1, nu2, s, zero_init);
    if (e == cudaSuccess) return e;
    cudaGetLastError();  // capture unavailable here: run the launches directly from now on
    graphs_ok_ = false;
  }
  return vcycle_direct<T>(l, nu1, nu2, x64, s, zero_init);
}

template <class T>
cudaError_t Multigrid::vcycle_graph(int l, int nu1, int nu2, cudaStream_t s, bool zero_init) {
  for (const auto& g : graphs_)
    if (g.l == l && g.nu1 == nu1 && g.nu2 == nu2 && g.zero == (int)zero_init) {
      note_launch(g.kernels);
      return cudaGraphLaunch(g.exec, s);
    }
  cudaError_t e = cudaSuccess;
  if (!cap_stream_) e = cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  // the captured work reads what earlier launches on s wrote: capture is only recording, the
  // replay below is ordered on s
  e = cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const unsigned long long c0 = launch_count();
  capturing_ = true;
  cudaError_t ec = vcycle_direct<T>(l, nu1, nu2, nullptr, cap_stream_, zero_init);
  capturing_ = false;
  const unsigned long long kernels = launch_count() - c0;  // counted now, for the launch below
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap_stream_, &graph);
  if (ec != cudaSuccess || e != cudaSuccess) {
    unnote_launches(kernels);
    if (graph) cudaGraphDestroy(graph);
    return ec != cudaSuccess ? ec : e;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    unnote_launches(kernels);
    return e;
  }
  graphs_.push_back({l, nu1, nu2, (int)zero_init, exec, kernels});
  return cudaGraphLaunch(exec, s);
}

template <class T>
cudaError_t Multigrid::vcycle_direct(int l, int nu1, int nu2, double* x64, cudaStream_t s, bool zero_init) {
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
    const size_t smem = 2 * (size_t)ncell * sizeof(T);
    const int in_smem = smem <= 48 * 1024 ? 1 : 0;
    note_launch(),
        k_coarse_solve<T><<<1, 512, in_smem ? smem : 0, s>>>(L, ncell, invd, r, x, (T*)lv_[l].tmp, sweeps, rb ? 1 : 0,
                                                             in_smem);
    if (x64) note_launch(), k_add_correction<T><<<nblk(ncell), kBlock, 0, s>>>(ncell, x, x64);
    return cudaGetLastError();
  }
  long long nhalf = (long long)((n[0] + 1) / 2) * n[1] * n[2];
  unsigned gb = nblk(nhalf);
  const bool wave = wave_[l].order != nullptr;
  const bool tiled = l == 0 && tiled_ && sizeof(T) == sizeof(float);
  // pre-smoothing (from a zero initial guess unless the caller set one): red, black, ...
  const char* sm_name = l == 0 ? "smooth_L0" : "smooth_Lc";
  for (int it = 0; it < nu1; ++it) {
    const bool zero = it == 0 && zero_init;
    if (tiled) {
      TraceScope ts(zero ? "sweep_L0_zero" : "sweep_L0", s);
      cudaError_t e = tiled_sweep<T>(zero, 0, nullptr, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    if (wave) {
      TraceScope ts(l == 0 ? (zero ? "wave_L0_zero" : "wave_L0") : "wave_Lc", s);
      cudaError_t e = wave_sweep<T>(l, zero, 0, nullptr, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    {
      TraceScope ts(zero ? (l == 0 ? "smooth_L0_zero" : "smooth_Lc") : sm_name, s);
      if (zero) note_launch(), k_smooth<T, true><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
      else note_launch(), k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
    }
    TraceScope ts(sm_name, s);
    note_launch(), k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1);
  }
  x = (T*)lv_[l].x;  // the tiled sweeps move the iterate between x and tmp
  const std::array<int, 3>& nc = dims_[l + 1];
  {
    TraceScope ts(l == 0 ? "restrict_L0" : "restrict_Lc", s);
    if (rows_ok(l)) {
      const int crows = nc[1] * nc[2];
      const unsigned gr = (unsigned)front_grid((const void*)k_restrict_rows<T, 3>, std::min(crows, 152 * 16));
      if (g_.ndim == 3) note_launch(),
          k_restrict_rows<T, 3><<<gr, kBlock, 0, s>>>(L, r, x, nc[1], crows, (T*)lv_[l + 1].r);
      else note_launch(), k_restrict_rows<T, 2><<<gr, kBlock, 0, s>>>(L, r, x, nc[1], crows, (T*)lv_[l + 1].r);
    } else {
      note_launch(), k_residual_restrict<T><<<nblk(cells3(nc)), kBlock, 0, s>>>(L, r, x, nc, (T*)lv_[l + 1].r, nullptr);
    }
  }
  cudaError_t e = vcycle<T>(l + 1, nuc1_, nuc2_, nullptr, s, true);  // coarser levels: their own counts
  if (e != cudaSuccess) return e;
  {
    TraceScope ts(l == 0 ? "prolong_L0" : "prolong_Lc", s);
    if (rows_ok(l)) {
      const int rows = n[1] * n[2];
      const unsigned gr = (unsigned)std::min(rows, 152 * 16);
      if (sizeof(T) == sizeof(float) && n[0] % 4 == 0) {
        const float* xc = (const float*)lv_[l + 1].x;
        if (g_.ndim == 3) note_launch(),
            k_prolong_rows4<3, false><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, xc, nc[1], (float*)x);
        else note_launch(), k_prolong_rows4<2, false><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, xc, nc[1], (float*)x);
      } else if (g_.ndim == 3) {
        note_launch(), k_prolong_rows<T, 3><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, (const T*)lv_[l + 1].x, nc[1], x);
      } else {
        note_launch(), k_prolong_rows<T, 2><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, (const T*)lv_[l + 1].x, nc[1], x);
      }
    } else {
      note_launch(), k_prolong<T><<<nblk(ncell), kBlock, 0, s>>>(n, g_.ndim, (const T*)lv_[l + 1].x, nc, x);
    }
  }
  // post-smoothing, colours reversed; on the finest level the last sweep also adds each colour's
  // final correction to the FP64 iterate
  for (int it = 0; it < nu2; ++it) {
    bool last = x64 && it == nu2 - 1;
    if (tiled) {
      TraceScope ts(last ? "sweep_L0_update" : "sweep_L0", s);
      cudaError_t e = tiled_sweep<T>(false, 1, last ? x64 : nullptr, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    if (wave) {
      TraceScope ts(l == 0 ? (last ? "wave_L0_update" : "wave_L0") : "wave_Lc", s);
      cudaError_t e = wave_sweep<T>(l, false, 1, last ? x64 : nullptr, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    {
      TraceScope ts(sm_name, s);
      if (last) note_launch(), k_smooth<T, false, true><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1, x64);
      else note_launch(), k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 1);
    }
    TraceScope ts(sm_name, s);
    if (last) note_launch(), k_smooth<T, false, true><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0, x64);
    else note_launch(), k_smooth<T, false><<<gb, kBlock, 0, s>>>(L, invd, r, x, 0);
  }
  x = (T*)lv_[l].x;
  if (x64 && nu2 == 0) {
    TraceScope ts("add_correction", s);
    note_launch(), k_add_correction<T><<<nblk(ncell), kBlock, 0, s>>>(ncell, x, x64);
  }
  return cudaGetLastError();
}

// Full-multigrid cycle for A d = r (r on the finest level, d from zero): restrict r down the
// hierarchy, solve on the coarsest level, then on each finer level start from the prolonged
// coarse solution and run one V-cycle (Sect. 3.4: FMG first, V-cycles after).  The finest
// V-cycle's last sweep adds d to x64 when x64 is given.
template <class T>
cudaError_t Multigrid::fmg(int nu1, int nu2, double* x64, cudaStream_t s) {
  const int top = (int)dims_.size() - 1;
  if (top == 0) return vcycle<T>(0, nu1, nu2, x64, s, true);
  // nu1, nu2: the finest level's counts; the coarser levels use nuc1_, nuc2_
  {
    TraceScope ts("fmg_restrict", s);
    for (int l = 0; l < top; ++l)
      note_launch(),
          k_restrict_avg<T><<<nblk(cells3(dims_[l + 1])), kBlock, 0, s>>>(dims_[l], g_.ndim, (const T*)lv_[l].r,
                                                                         dims_[l + 1], (T*)lv_[l + 1].r);
  }
  cudaError_t e = vcycle<T>(top, nuc1_, nuc2_, nullptr, s, true);
  if (e != cudaSuccess) return e;
  for (int l = top - 1; l >= 0; --l) {
    const std::array<int, 3>& n = dims_[l];
    const std::array<int, 3>& nc = dims_[l + 1];
    T* x = (T*)lv_[l].x;
    {
      TraceScope ts(l == 0 ? "prolong_L0" : "prolong_Lc", s);
      if (rows_ok(l)) {
        const int rows = n[1] * n[2];
        const unsigned gr = (unsigned)std::min(rows, 152 * 16);
        if (sizeof(T) == sizeof(float) && n[0] % 4 == 0) {
          const float* xc = (const float*)lv_[l + 1].x;
          if (g_.ndim == 3) note_launch(),
              k_prolong_rows4<3, true><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, xc, nc[1], (float*)x);
          else note_launch(), k_prolong_rows4<2, true><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, xc, nc[1], (float*)x);
        } else if (g_.ndim == 3) {
          note_launch(),
              k_prolong_rows<T, 3, true><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, (const T*)lv_[l + 1].x, nc[1], x);
        } else {
          note_launch(),
              k_prolong_rows<T, 2, true><<<gr, kBlock, 0, s>>>(n[0], n[1], rows, (const T*)lv_[l + 1].x, nc[1], x);
        }
      } else {
        e = cudaMemsetAsync(x, 0, cells3(n) * sizeof(T), s);
        if (e != cudaSuccess) return e;
        note_launch(), k_prolong<T><<<nblk(cells3(n)), kBlock, 0, s>>>(n, g_.ndim, (const T*)lv_[l + 1].x, nc, x);
      }
    }
    e = vcycle<T>(l, l == 0 ? nu1 : nuc1_, l == 0 ? nu2 : nuc2_, l == 0 ? x64 : nullptr, s, false);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// Outer loop.  FP64 solver: every iteration computes the exact residual b - A x in FP64.  Mixed
// solver: after a V-cycle the residual is updated, r <- r - A d, in double-float arithmetic (the
// correction d is exact in FP32; see k_residual_update) instead of being recomputed in FP64.  The
// update's rounding error is bounded per iteration by kDrift ||m|| (m per cell = |r_old| +
// diag |d| + sum |w d_nb|, relative to ||b||), summed over the updates since the last exact
// residual; convergence is accepted when the updated residual plus that bound is within rtol, else
// an exact FP64 residual decides.
template <class T>
cudaError_t Multigrid::solve_t(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                               bool fmg_start, SolveStats* st, cudaStream_t s) {
  // per-cell error of a double-float residual over m (|b or r_old| + |diag x| + sum |w x_nb|): the
  // operations' roundings plus the 2^-45 representation error of the double-float weights
  constexpr double kDrift = 0x1p-42;
  void* w64v[3] = {w64_[0], w64_[1], w64_[2]};
  LevelDev<double> L64 = level_dev<double>(g_, dims_[0], w64v);
  const bool mixed = sizeof(T) == sizeof(float) && dhi_ != nullptr;
  LevelDev<float> L32{}, L32lo{};
  if (mixed) {
    void* wlo[3] = {w32lo_[0], w32lo_[1], w32lo_[2]};
    L32 = level_dev<float>(g_, dims_[0], lv_[0].w);
    L32lo = level_dev<float>(g_, dims_[0], wlo);
  }
  const double N = (double)g_.ncell;
  // one front of resident blocks for the row-walking residual kernels
  const int gu = front_grid((const void*)k_residual_update<3>, nparts_);
  const int gx = mixed ? front_grid((const void*)k_residual64_df, nparts_)
                       : front_grid((const void*)k_residual64<T>, nparts_);
  // the FP64 iterate lives in E_new; the first residual copies E_old into it
  const double* x_in = E_old;
  double* x = E_new;
  double bb = 0.0;
  int cycles = 0;
  double rel = 0.0;
  int status = FLD_ERR_NOT_CONVERGED;
  unsigned* wave_err = reinterpret_cast<unsigned*>(host_scal_ + 7);
  *wave_err = 0u;
  {
    cudaError_t e = cudaMemsetAsync(wave_ctl_, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
  }
  bool updates = false;   // residual updates allowed (decided at the first exact residual)
  bool exact = true;      // next residual: exact FP64 (else an update)
  bool df_res = false;    // this residual came from the double-float setup
  unsigned* df_flag = reinterpret_cast<unsigned*>(host_scal_ + 6);
  *df_flag = 0u;
  double drift = 0.0;
  float scale = 0.f;
  for (;;) {
    const bool upd = !exact;
    if (upd) {
      df_res = false;  // an update's sums are scaled by 1/rms(b), and its drift adds to the bound
      TraceScope ts("residual_update", s);
      const float* dv = (const float*)lv_[0].x;
      float* rv = (float*)lv_[0].r;
      if (g_.ndim == 3)
        note_launch(),
            k_residual_update<3><<<gu, kBlock, 0, s>>>(L32, L32lo, dhi_, dlo_, dv, rv, rlo_, x, scale, nullptr, gu,
                                                         partials_);
      else if (g_.ndim == 2)
        note_launch(),
            k_residual_update<2><<<gu, kBlock, 0, s>>>(L32, L32lo, dhi_, dlo_, dv, rv, rlo_, x, scale, nullptr, gu,
                                                         partials_);
      else
        note_launch(),
            k_residual_update<1><<<gu, kBlock, 0, s>>>(L32, L32lo, dhi_, dlo_, dv, rv, rlo_, x, scale, nullptr, gu,
                                                         partials_);
      note_launch(), k_reduce<<<1, 1024, 0, s>>>(partials_, gu, scal_);
      note_launch(), k_reduce<<<1, 1024, 0, s>>>(partials_ + gu, gu, scal_ + 2);
    } else {
      TraceScope ts("residual", s);
      df_res = mixed && df_mode_ && !fp64_op_ && cycles == 0;
      if (df_res) {
        // the finest level's diagonal and the double-float first residual in one pass from the
        // double-float weights (no FP64 operator exists yet)
        cudaError_t e = launch_setup_res0_df(g_, make_df_const(g_, dt_), L32, L32lo, x_in, x != x_in ? x : nullptr,
                                             dhi_, dlo_, (float*)lv_[0].invd, (float*)lv_[0].r, rlo_, nparts_,
                                             partials_, scal_, df_flag_, s);
        if (e != cudaSuccess) return e;
      } else {
        if (mixed && !fp64_op_) {
          cudaError_t e = fp64_operator<T>(s);  // an exact residual after a double-float setup
          if (e != cudaSuccess) return e;
        }
        if (mixed)
          note_launch(),
              k_residual64_df<<<gx, kBlock, 0, s>>>(L64, x_in, x, b64_, diag64_, (float*)lv_[0].r, rlo_, partials_);
        else
          note_launch(), k_residual64<T><<<gx, kBlock, 0, s>>>(L64, g_.ncell, x_in, x, b64_, diag64_, (T*)lv_[0].r,
                                                               partials_);
        note_launch(), k_reduce<<<1, 1024, 0, s>>>(partials_, gx, scal_);
      }
    }
    cudaError_t e = cudaMemcpyAsync(host_scal_, scal_, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if (cycles > 0) e = cudaMemcpyAsync(wave_err, wave_ctl_, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if (df_res) e = cudaMemcpyAsync(df_flag, df_flag_, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (*wave_err) {
      status = FLD_ERR_DEVICE_TIMEOUT;
      break;
    }
    if (df_res && *df_flag) {
      // a value left the double-float window: redo the setup and this residual in FP64
      e = fp64_operator<T>(s);
      if (e != cudaSuccess) return e;
      continue;
    }
    x_in = x;
    bb = host_scal_[1];
    if (df_res) {
      // unscaled sums: ||r||^2, ||b||^2 and the error measure's ||m||^2
      rel = bb > 0 ? sqrt(host_scal_[0] / bb) : sqrt(host_scal_[0]);
      drift = kDrift * (bb > 0 ? sqrt(host_scal_[2] / bb) : sqrt(host_scal_[2]));
      const double rms = sqrt(bb / N);
      updates = rms * std::max(rtol, 1e-16) * 1e-3 >= 0x1p-76 && rms <= 0x1p90;
      scale = (float)(1.0 / rms);
    } else if (upd) {
      // scaled sums: sum (r / rms(b))^2 = N ||r||^2 / ||b||^2
      rel = sqrt(host_scal_[0] / N);
      drift += kDrift * sqrt(host_scal_[2] / N);
    } else {
      const double rr = host_scal_[0];
      rel = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
      drift = 0.0;
      if (cycles == 0 && mixed && bb > 0) {
        // updates need the residuals (down to ~1e-3 rtol rms(b)) and their error terms in the
        // normal FP32 range
        const double rms = sqrt(bb / N);
        long long maxf = g_.ncell;
        for (int a = 0; a < g_.ndim; ++a) maxf = std::max(maxf, faces3(dims_[0], a));
        updates = rms * std::max(rtol, 1e-16) * 1e-3 >= 0x1p-76 && rms <= 0x1p90 && maxf < (1LL << 31);
        scale = (float)(1.0 / rms);
      }
    }
    if (!(rel == rel) || rel > 1e300) {
      status = FLD_ERR_NONFINITE;
      break;
    }
    if (rel + drift <= rtol) {
      status = FLD_OK;
      break;
    }
    if (upd && rel <= rtol) {
      exact = true;  // the estimate is converged but the bound does not certify it
      continue;
    }
    if (cycles >= max_cycles) break;
    // one V-cycle on A d = r; d joins x in its last finest-level sweep, or in the residual update
    // that follows
    if (cycles == 0 && fmg_start) e = fmg<T>(nu1, nu2, updates ? nullptr : x, s);
    else e = vcycle<T>(0, nu1, nu2, updates ? nullptr : x, s, true);
    if (e != cudaSuccess) return e;
    ++cycles;
    exact = !updates;
  }
  st->cycles = cycles;
  st->relres = rel;
  st->status = status;
  return cudaStreamSynchronize(s);
}

cudaError_t Multigrid::autotune(const double* E_old, double rtol, int max_cycles, bool fmg_start, int nu[4],
                                cudaStream_t s) {
  // (finest pre, finest post, coarser pre, coarser post)
  static const int cand[kTuneCands][4] = {{2, 2, 2, 2}, {3, 3, 3, 3}, {4, 4, 2, 1}, {5, 3, 2, 1}, {4, 4, 2, 2},
                                          {3, 3, 2, 1}, {4, 2, 2, 1}, {6, 4, 2, 1}, {2, 1, 2, 1}, {1, 1, 1, 1},
                                          {6, 6, 2, 2}, {5, 5, 3, 3}};
  size_t ti = tuned_.size();
  for (size_t q = 0; q < tuned_.size(); ++q)
    if (tuned_[q].rtol == rtol && tuned_[q].fmg == fmg_start) ti = q;
  if (ti < tuned_.size() && tuned_[ti].rounds >= kTuneRounds) {
    for (int k = 0; k < 4; ++k) nu[k] = cand[tuned_[ti].best][k];
    return cudaSuccess;
  }
  // the first solve of a configuration is often not typical of the ones that follow (a time
  // step's initial state differs from the states the stepping settles into), so the candidates are
  // timed on the first kTuneRounds solves and chosen by their summed time
  if (ti == tuned_.size()) {
    Tuned t{};
    t.rtol = rtol;
    t.fmg = fmg_start;
    tuned_.push_back(t);
  }
  const size_t n = (size_t)g_.ncell;
  if (tune_cap_ < n) {
    if (tune_x_) cudaFree(tune_x_);
    tune_x_ = nullptr;
    tune_cap_ = 0;
    cudaError_t e = cudaMalloc(&tune_x_, n * sizeof(double));
    if (e != cudaSuccess) return e;
    tune_cap_ = n;
  }
  static const bool log = getenv("FLD_AUTOTUNE_LOG") != nullptr;  // each candidate's timing on stderr
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return e;
  float ms_k[kTuneCands];
  bool ok_k[kTuneCands];
  for (int k = 0; k < kTuneCands; ++k) {
    const int* c = cand[k];
    nuc1_ = c[2];
    nuc2_ = c[3];
    SolveStats cs;
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess)
      e = precision_ == FLD_PREC_MIXED
              ? solve_t<float>(E_old, tune_x_, rtol, max_cycles, c[0], c[1], fmg_start, &cs, s)
              : solve_t<double>(E_old, tune_x_, rtol, max_cycles, c[0], c[1], fmg_start, &cs, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) break;
    ms_k[k] = ms;
    ok_k[k] = cs.status == FLD_OK;
    if (log)
      fprintf(stderr, "fld autotune: nu (%d,%d,%d,%d) %.3f ms, %d cycles, status %d, residual %.3e\n", c[0], c[1], c[2],
              c[3], ms, cs.cycles, cs.status, cs.relres);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  Tuned& t = tuned_[ti];
  for (int k = 0; k < kTuneCands; ++k) t.sum[k] = ok_k[k] ? t.sum[k] + ms_k[k] : INFINITY;
  t.rounds += 1;
  t.best = 0;
  for (int k = 1; k < kTuneCands; ++k)
    if (t.sum[k] < t.sum[t.best]) t.best = k;
  for (int k = 0; k < 4; ++k) nu[k] = cand[t.best][k];
  return cudaSuccess;
}

// ----------------------------------------------------------------------------- graph-driven solve
//
// The outer loop of solve_t with its decisions on the device.  The graph runs the first residual,
// then a WHILE node whose body is: k_solve_check (one thread: evaluates the last residual exactly as
// solve_t does and sets the conditions below and the loop's), then IF nodes for the full-multigrid
// cycle, the V-cycle, the FP64 operator (the redo of a double-float set-up that left its window,
// or the certification of an update), the addition of the correction to the FP64 iterate, the
// exact residual and the double-float residual update.  Its last kernel writes the result into
// pinned host memory.  Nothing on the host waits for a cycle.

enum { kPendDf = 0, kPendExact = 1, kPendUpdate = 2 };

struct SolveHandles {
  cudaGraphConditionalHandle loop, fmg, vcyc, fp64, add, exact, upd;
};

__global__ void k_solve_init(Multigrid::SolveDev* S, double rtol, double N, int max_cycles, int mixed, int fmg_start,
                             int idx32, int pending, int fp64_op, unsigned long long kernels) {
  S->rtol = rtol;
  S->N = N;
  S->max_cycles = max_cycles;
  S->mixed = mixed;
  S->fmg_start = fmg_start;
  S->idx32 = idx32;
  S->cycles = 0;
  S->status = FLD_ERR_NOT_CONVERGED;
  S->pending = pending;
  S->updates = 0;
  S->fp64_op = fp64_op;
  S->scale = 0.0f;
  S->rel = 0.0;
  S->drift = 0.0;
  S->kernels = kernels;
}

__global__ void k_solve_check(Multigrid::SolveDev* S, const double* __restrict__ scal, const unsigned* df_flag,
                              const unsigned* wave_err, SolveHandles h) {
  constexpr double kDrift = 0x1p-42;  // as solve_t
  int do_fmg = 0, do_v = 0, do_fp = 0, do_add = 0, do_exact = 0, do_upd = 0;
  bool go = true;
  const int pend = S->pending;
  if (*wave_err) {
    S->status = FLD_ERR_DEVICE_TIMEOUT;
    go = false;
  } else if (pend == kPendDf && df_flag && *df_flag) {
    // a value left the double-float window: the FP64 operator, then an exact residual from the
    // copy of E_old the set-up pass left in the iterate
    do_fp = 1;
    do_exact = 1;
    S->fp64_op = 1;
    S->pending = kPendExact;
  } else {
    const double N = S->N, bb = scal[1];
    double rel, drift = S->drift;
    if (pend == kPendDf) {
      rel = bb > 0 ? sqrt(scal[0] / bb) : sqrt(scal[0]);
      drift = kDrift * (bb > 0 ? sqrt(scal[2] / bb) : sqrt(scal[2]));
      const double rms = sqrt(bb / N);
      S->updates = rms * fmax(S->rtol, 1e-16) * 1e-3 >= 0x1p-76 && rms <= 0x1p90;
      S->scale = (float)(1.0 / rms);
    } else if (pend == kPendUpdate) {
      rel = sqrt(scal[0] / N);
      drift += kDrift * sqrt(scal[2] / N);
    } else {
      rel = bb > 0 ? sqrt(scal[0] / bb) : sqrt(scal[0]);
      drift = 0.0;
      if (S->cycles == 0 && S->mixed && bb > 0) {
        const double rms = sqrt(bb / N);
        S->updates = rms * fmax(S->rtol, 1e-16) * 1e-3 >= 0x1p-76 && rms <= 0x1p90 && S->idx32;
        S->scale = (float)(1.0 / rms);
      }
    }
    S->rel = rel;
    S->drift = drift;
    if (!(rel == rel) || rel > 1e300) {
      S->status = FLD_ERR_NONFINITE;
      go = false;
    } else if (rel + drift <= S->rtol) {
      S->status = FLD_OK;
      go = false;
    } else if (pend == kPendUpdate && rel <= S->rtol) {
      // the estimate is converged but the bound does not certify it: an exact residual
      do_exact = 1;
      do_fp = S->mixed && !S->fp64_op;
      S->fp64_op |= do_fp;
      S->pending = kPendExact;
    } else if (S->cycles >= S->max_cycles) {
      S->status = FLD_ERR_NOT_CONVERGED;
      go = false;
    } else {
      do_fmg = S->cycles == 0 && S->fmg_start;
      do_v = !do_fmg;
      S->cycles += 1;
      if (S->updates) {
        do_upd = 1;
        S->pending = kPendUpdate;
      } else {
        do_add = 1;
        do_exact = 1;
        do_fp = S->mixed && !S->fp64_op;
        S->fp64_op |= do_fp;
        S->pending = kPendExact;
      }
    }
  }
  cudaGraphSetConditional(h.loop, go ? 1u : 0u);
  cudaGraphSetConditional(h.fmg, (unsigned)do_fmg);
  cudaGraphSetConditional(h.vcyc, (unsigned)do_v);
  cudaGraphSetConditional(h.fp64, (unsigned)do_fp);
  cudaGraphSetConditional(h.add, (unsigned)do_add);
  cudaGraphSetConditional(h.exact, (unsigned)do_exact);
  cudaGraphSetConditional(h.upd, (unsigned)do_upd);
  S->kernels += S->kc_check + do_fmg * S->kc_fmg + do_v * S->kc_vcyc + do_fp * S->kc_fp64 + do_add * S->kc_add +
                do_exact * S->kc_exact + do_upd * S->kc_upd;
}

__global__ void k_solve_done(const Multigrid::SolveDev* S, Multigrid::SolveOut* out) {
  out->cycles = S->cycles;
  out->status = S->status;
  out->relres = S->rel;
  out->kernels = S->kernels;  // the loop's kernels (the host counts the rest at launch)
}

// Adds a conditional node (type WHILE or IF, condition h) at the capture position of s and returns
// its body graph.
static cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                   cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaGraph_t capg = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, &deps, &edata, &ndeps);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, capg, deps, edata, ndeps, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

template <class T>
cudaError_t Multigrid::build_solve_graph(const SolveKey& k, cudaStream_t s0) {
  if (sexec_) cudaGraphExecDestroy(sexec_);
  sexec_ = nullptr;
  cudaError_t e = cudaSuccess;
  if (!cap_stream_) e = cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking);
  for (int q = 0; q < 2 && e == cudaSuccess; ++q)
    if (!body_s_[q]) e = cudaStreamCreateWithFlags(&body_s_[q], cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  // the state the capture changes on the host: restored afterwards
  void* const x0 = lv_[0].x;
  void* const t0 = lv_[0].tmp;
  const bool fp64_op0 = fp64_op_;
  const bool mixed = sizeof(T) == sizeof(float) && dhi_ != nullptr;
  const bool df_first = mixed && df_mode_ && !fp64_op_;
  long long maxf = g_.ncell;
  for (int a = 0; a < g_.ndim; ++a) maxf = std::max(maxf, faces3(dims_[0], a));
  const double* E_old = k.E_old;
  double* x = k.E_new;
  const int nu1 = k.nu[0], nu2 = k.nu[1];
  const int tswaps = (tiled_ && sizeof(T) == sizeof(float)) ? nu1 + nu2 : 0;  // finest sweeps that swap x, tmp
  void* const A = x0;  // where every branch leaves the correction d
  void* const B = t0;
  cudaGraph_t graph = nullptr;
  e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return e;
  cudaStream_t s = cap_stream_;
  e = cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return e;
  }
  capturing_ = true;
  unsigned long long kc[7] = {0, 0, 0, 0, 0, 0, 0};  // check, fmg, vcyc, fp64, add, exact, upd
  const unsigned long long c0 = launch_count();
  void* w64v[3] = {w64_[0], w64_[1], w64_[2]};
  LevelDev<double> L64 = level_dev<double>(g_, dims_[0], w64v);
  LevelDev<float> L32{}, L32lo{};
  if (mixed) {
    void* wlo[3] = {w32lo_[0], w32lo_[1], w32lo_[2]};
    L32 = level_dev<float>(g_, dims_[0], lv_[0].w);
    L32lo = level_dev<float>(g_, dims_[0], wlo);
  }
  const int gu = front_grid((const void*)k_residual_update<3>, nparts_);
  const int gx = mixed ? front_grid((const void*)k_residual64_df, nparts_)
                       : front_grid((const void*)k_residual64<T>, nparts_);
  auto exact_residual = [&](cudaStream_t b, const double* xin) {
    if (mixed)
      note_launch(), k_residual64_df<<<gx, kBlock, 0, b>>>(L64, xin, x, b64_, diag64_, (float*)lv_[0].r, rlo_,
                                                           partials_);
    else
      note_launch(), k_residual64<T><<<gx, kBlock, 0, b>>>(L64, g_.ncell, xin, x, b64_, diag64_, (T*)lv_[0].r,
                                                           partials_);
    note_launch(), k_reduce<<<1, 1024, 0, b>>>(partials_, gx, scal_);
  };
  // pre-loop: the error word, the state and the first residual (the set-up ran before the graph)
  e = cudaMemsetAsync(wave_ctl_, 0, sizeof(unsigned), s);
  note_launch(), k_solve_init<<<1, 1, 0, s>>>(sd_, k.rtol, (double)g_.ncell, k.max_cycles, mixed ? 1 : 0, k.fmg,
                                              maxf < (1LL << 31) ? 1 : 0, df_first ? kPendDf : kPendExact,
                                              fp64_op_ ? 1 : 0, 0ull);
  if (df_first) {
    if (e == cudaSuccess)
      e = launch_setup_res0_df(g_, make_df_const(g_, dt_), L32, L32lo, E_old, x != E_old ? x : nullptr, dhi_, dlo_,
                               (float*)lv_[0].invd, (float*)lv_[0].r, rlo_, nparts_, partials_, scal_, df_flag_, s);
  } else {
    exact_residual(s, E_old);
  }
  const unsigned long long c_pre = launch_count() - c0 + 1;  // + k_solve_done
  // the loop
  cudaGraphConditionalHandle hloop;
  cudaGraph_t bodyg = nullptr;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hloop, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = add_conditional(s, hloop, cudaGraphCondTypeWhile, &bodyg);
  cudaStream_t b1 = body_s_[0], b2 = body_s_[1];
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b1, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    SolveHandles h{};
    h.loop = hloop;
    cudaGraphConditionalHandle* hs[6] = {&h.fmg, &h.vcyc, &h.fp64, &h.add, &h.exact, &h.upd};
    for (int q = 0; q < 6 && e == cudaSuccess; ++q) e = cudaGraphConditionalHandleCreate(hs[q], bodyg, 0, 0);
    unsigned long long c = launch_count();
    if (e == cudaSuccess)
      note_launch(), k_solve_check<<<1, 1, 0, b1>>>(sd_, scal_, df_first ? df_flag_ : nullptr, wave_ctl_, h);
    kc[0] = launch_count() - c;
    // one IF node per branch, its body captured on b2
    auto branch = [&](cudaGraphConditionalHandle hh, int slot, auto&& fill) {
      if (e != cudaSuccess) return;
      cudaGraph_t ifg = nullptr;
      e = add_conditional(b1, hh, cudaGraphCondTypeIf, &ifg);
      if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b2, ifg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return;
      const unsigned long long cb = launch_count();
      cudaError_t ef = fill(b2);
      kc[slot] = launch_count() - cb;
      cudaGraph_t tmp = nullptr;
      e = cudaStreamEndCapture(b2, &tmp);
      if (e == cudaSuccess) e = ef;
    };
    // full multigrid: the prolongation assigns into lv_[0].x, then nu1 + nu2 finest sweeps swap it
    branch(h.fmg, 1, [&](cudaStream_t b) {
      lv_[0].x = (tswaps % 2 == 0) ? A : B;
      lv_[0].tmp = (tswaps % 2 == 0) ? B : A;
      return fmg<T>(nu1, nu2, nullptr, b);
    });
    // V-cycle from zero: its first finest sweep writes lv_[0].tmp
    branch(h.vcyc, 2, [&](cudaStream_t b) {
      lv_[0].tmp = (tswaps % 2 == 1) ? A : B;
      lv_[0].x = (tswaps % 2 == 1) ? B : A;
      return vcycle<T>(0, nu1, nu2, nullptr, b, true);
    });
    if (e == cudaSuccess && lv_[0].x != A) e = cudaErrorInvalidValue;  // both branches end in A
    branch(h.fp64, 3, [&](cudaStream_t b) { return fp64_operator<T>(b); });
    branch(h.add, 4, [&](cudaStream_t b) {
      note_launch(), k_add_correction<T><<<nblk(g_.ncell), kBlock, 0, b>>>(g_.ncell, (const T*)A, x);
      return cudaGetLastError();
    });
    branch(h.exact, 5, [&](cudaStream_t b) {
      exact_residual(b, x);
      return cudaGetLastError();
    });
    branch(h.upd, 6, [&](cudaStream_t b) {
      if (!mixed) return cudaSuccess;
      const float* dv = (const float*)A;
      float* rv = (float*)lv_[0].r;
      const float* sp = &sd_->scale;
      if (g_.ndim == 3)
        note_launch(), k_residual_update<3><<<gu, kBlock, 0, b>>>(L32, L32lo, dhi_, dlo_, dv, rv, rlo_, x, 0.f, sp, gu,
                                                                 partials_);
      else if (g_.ndim == 2)
        note_launch(), k_residual_update<2><<<gu, kBlock, 0, b>>>(L32, L32lo, dhi_, dlo_, dv, rv, rlo_, x, 0.f, sp, gu,
                                                                 partials_);
      else
        note_launch(), k_residual_update<1><<<gu, kBlock, 0, b>>>(L32, L32lo, dhi_, dlo_, dv, rv, rlo_, x, 0.f, sp, gu,
                                                                 partials_);
      note_launch(), k_reduce<<<1, 1024, 0, b>>>(partials_, gu, scal_);
      note_launch(), k_reduce<<<1, 1024, 0, b>>>(partials_ + gu, gu, scal_ + 2);
      return cudaGetLastError();
    });
    cudaGraph_t tmp = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b1, &tmp);
    if (e == cudaSuccess) e = ee;
  }
  if (e == cudaSuccess) note_launch(), k_solve_done<<<1, 1, 0, s>>>(sd_, out_h_);
  cudaGraph_t done = nullptr;
  cudaError_t ee = cudaStreamEndCapture(s, &done);
  if (e == cudaSuccess) e = ee;
  capturing_ = false;
  unnote_launches(launch_count() - c0);  // captured, not run: the graph's last kernel counts what ran
  lv_[0].x = x0;
  lv_[0].tmp = t0;
  fp64_op_ = fp64_op0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sexec_, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    sexec_ = nullptr;
    return e;
  }
  // the per-branch kernel counts, and the pre-loop's in the initial count
  SolveDev init{};
  init.kc_check = kc[0];
  init.kc_fmg = kc[1];
  init.kc_vcyc = kc[2];
  init.kc_fp64 = kc[3];
  init.kc_add = kc[4];
  init.kc_exact = kc[5];
  init.kc_upd = kc[6];
  e = cudaMemcpyAsync(&sd_->kc_check, &init.kc_check, 7 * sizeof(unsigned long long), cudaMemcpyHostToDevice, s0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
  pre_kernels_ = c_pre;
  skey_ = k;
  return e;
}

// The graph-driven solve, unless the event tracer is on (its per-launch events are host-side
// bookkeeping) or FLD_SOLVE_GRAPH=0 asks for the host-driven loop.
bool Multigrid::async_ready() const {
  static const bool off = [] {
    const char* v = getenv("FLD_SOLVE_GRAPH");
    return v && atoi(v) == 0;
  }();
  return !off && !tracer().on;
}

cudaError_t Multigrid::solve_async(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1,
                                   int nu2, bool fmg_start, SolveStats* st, const SolveOut** out, cudaStream_t s) {
  int nu[4] = {nu1 ? nu1 : 2, nu2 ? nu2 : 2, nu1 ? nu1 : 2, nu2 ? nu2 : 2};
  if (nu1 == 0 && nu2 == 0) {
    // the first solve of a configuration times candidate sweep counts (synchronises); later ones
    // find them cached
    cudaError_t e = autotune(E_old, rtol, max_cycles, fmg_start, nu, s);
    if (e != cudaSuccess) return e;
  }
  nuc1_ = nu[2];
  nuc2_ = nu[3];
  st->nu1 = nu[0];
  st->nu2 = nu[1];
  st->nu1_coarse = nu[2];
  st->nu2_coarse = nu[3];
  if (!out_h_) {
    cudaError_t e = cudaMallocHost(&out_h_, sizeof(SolveOut));
    if (e != cudaSuccess) return e;
  }
  SolveKey k{};
  k.E_old = E_old;
  k.E_new = E_new;
  for (int a = 0; a < 3; ++a) k.D[a] = D_ax_[a];
  k.dt = dt_;
  k.rtol = rtol;
  k.max_cycles = max_cycles;
  for (int q = 0; q < 4; ++q) k.nu[q] = nu[q];
  k.fmg = fmg_start ? 1 : 0;
  k.df = df_mode_ ? 1 : 0;
  // whether the FP64 operator is already built (the autotuner's solves may have built it): a graph
  // made for that state has no double-float set-up pass and reads the FP64 b and diagonal as they
  // are, so it serves only calls that start in the same state
  k.fp64op = fp64_op_ ? 1 : 0;
  k.prec = precision_;
  if (!sexec_ || !(k == skey_)) {
    cudaError_t e = precision_ == FLD_PREC_MIXED ? build_solve_graph<float>(k, s) : build_solve_graph<double>(k, s);
    if (e != cudaSuccess) return e;
  }
  note_launch(pre_kernels_);  // the pre-loop kernels; the loop's are added when the result is read
  *out = out_h_;
  return cudaGraphLaunch(sexec_, s);
}

cudaError_t Multigrid::solve(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                             bool fmg_start, SolveStats* st, cudaStream_t s) {
  int nu[4] = {nu1 ? nu1 : 2, nu2 ? nu2 : 2, nu1 ? nu1 : 2, nu2 ? nu2 : 2};
  if (nu1 == 0 && nu2 == 0) {
    cudaError_t e = autotune(E_old, rtol, max_cycles, fmg_start, nu, s);
    if (e != cudaSuccess) return e;
  }
  nuc1_ = nu[2];
  nuc2_ = nu[3];
  st->nu1 = nu[0];
  st->nu2 = nu[1];
  st->nu1_coarse = nu[2];
  st->nu2_coarse = nu[3];
  return precision_ == FLD_PREC_MIXED ? solve_t<float>(E_old, E_new, rtol, max_cycles, nu[0], nu[1], fmg_start, st, s)
                                      : solve_t<double>(E_old, E_new, rtol, max_cycles, nu[0], nu[1], fmg_start, st, s);
}

}  // namespace fld

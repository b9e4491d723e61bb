// Device helpers shared by the single-grid and batched multigrid kernels.
#pragma once

#include "fld_common.cuh"
#include "mg.h"

namespace fld {

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

// The same for a level of fewer than 2^32 cells, with the divisions by n[0] and n[1] done by
// multiplication (f0, f1 = make_fastdiv(n[0]), make_fastdiv(n[1])).
__device__ __forceinline__ void unflatten32(unsigned idx, const FastDiv& f0, const FastDiv& f1, int& i, int& j,
                                            int& k) {
  const unsigned r = fast_div(idx, f0);
  const unsigned kk = fast_div(r, f1);
  i = (int)(idx - r * f0.d);
  j = (int)(r - kk * f1.d);
  k = (int)kk;
}


// Sum over the block (valid in thread 0); every thread of the block must call it.
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


// ----------------------------------------------------------------------------- per-cell bodies

// b = E_old + boundary constants (Dirichlet ghost value, Neumann gradient); the FP64 diagonal
// of the outer operator and its inverse in T for the finest inner level.
template <class T>
__device__ __forceinline__ double fine_setup_at(const LevelDev<double>& L, const GridDev& g,
                                                const double* __restrict__ E_old, int i, int j, int k, long long idx,
                                                double* __restrict__ b, double* __restrict__ diag,
                                                T* __restrict__ invd) {
  double d = 1.0, cst = 0.0, wsum = 0.0;
  int face = 0;
  // boundary constants need to know which side each boundary face is on
  for_each_face(L, i, j, k, idx, [&](double w, int kind, long long) {
    int a = face >> 1, side = face & 1;
    ++face;
    wsum += w;
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
  });
  b[idx] = E_old[idx] + cst;
  diag[idx] = d;
  if (sizeof(T) == sizeof(float)) invd[idx] = (T)(1.0f / (float)d);  // the FP32 smoother's 1/diag
  else invd[idx] = (T)(1.0 / d);
  return fma(2.0, wsum, 1.0);  // bound on the row's absolute sum: |diag| + sum |off-diagonal|
}

template <class T>
__device__ __forceinline__ double fine_setup_cell(const LevelDev<double>& L, const GridDev& g,
                                                  const double* __restrict__ E_old, long long idx,
                                                  double* __restrict__ b, double* __restrict__ diag,
                                                  T* __restrict__ invd) {
  int i, j, k;
  unflatten(g.n, idx, i, j, k);
  return fine_setup_at<T>(L, g, E_old, i, j, k, idx, b, diag, invd);
}

// Coarse face `idx` of axis a (coarse face layout m = coarse dims with m[a] + 1): the mean of the
// 2^(d-1) fine faces it covers, divided by 4 because dx doubles.
template <class T>
__device__ __forceinline__ T coarse_face_at(int a, int ndim, const int nf[3], const int (&q)[3],
                                            const T* __restrict__ wf) {
  int mf[3] = {nf[0], nf[1], nf[2]};
  mf[a] += 1;
  T s = T(0);
  int cnt = 0;
  int o1max = (ndim > 1) ? 2 : 1, o2max = (ndim > 2) ? 2 : 1;
  int t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;  // the transverse axes
  for (int o2 = 0; o2 < o2max; ++o2)
    for (int o1 = 0; o1 < o1max; ++o1) {
      int f[3];
      f[a] = 2 * q[a];
      f[t1] = (t1 < ndim) ? 2 * q[t1] + o1 : q[t1];
      f[t2] = (t2 < ndim) ? 2 * q[t2] + o2 : q[t2];
      s += wf[(long long)f[0] + (long long)mf[0] * ((long long)f[1] + (long long)mf[1] * f[2])];
      ++cnt;
    }
  return s / (T)(4 * cnt);
}

template <class T>
__device__ __forceinline__ T coarse_face_value(int a, int ndim, const int nf[3], const int m[3], long long idx,
                                               const T* __restrict__ wf) {
  int q[3];
  q[0] = (int)(idx % m[0]);
  long long r = idx / m[0];
  q[1] = (int)(r % m[1]);
  q[2] = (int)(r / m[1]);
  return coarse_face_at<T>(a, ndim, nf, q, wf);
}

// r = b - A x in FP64 with the stored diagonal: r_c = b_c - d_c x_c + sum_f w_f x_nb (minus the
// continuous-boundary terms), written in T for the inner V-cycle; returns acc + r^2.
// x_out = x_in (the first iteration copies E_old into the iterate; later ones run in place,
// x_out == x_in, where the store rewrites the value just read).
template <class T>
__device__ __forceinline__ double fma_residual_at(const LevelDev<double>& L, const double* x_in, double* x_out,
                                                  const double* __restrict__ b, const double* __restrict__ diag,
                                                  T* __restrict__ r_out, int i, int j, int k, long long idx,
                                                  double acc) {
  double xc = x_in[idx];
  double s = fma(-diag[idx], xc, b[idx]);
  for_each_face(L, i, j, k, idx, [&](double w, int kind, long long nb) {
    if (kind == kInterior) s = fma(w, x_in[nb], s);
    else if (kind == kContinuous) s = fma(-w, x_in[nb], s);
  });
  if (x_out != x_in) x_out[idx] = xc;
  r_out[idx] = (T)s;
  return fma(s, s, acc);
}

template <class T>
__device__ __forceinline__ double fma_residual_cell(const LevelDev<double>& L, const double* x_in, double* x_out,
                                                    const double* __restrict__ b, const double* __restrict__ diag,
                                                    T* __restrict__ r_out, long long idx, double acc) {
  int i, j, k;
  unflatten(L.n, idx, i, j, k);
  return fma_residual_at<T>(L, x_in, x_out, b, diag, r_out, i, j, k, idx, acc);
}

// Red-black Gauss-Seidel, thread t of one colour: x_c = (r_c + sum w x_nb) / diag on the cells
// with (i+j+k) % 2 == color.  ZERO: the sweep starts from x = 0 (neighbours read as zero).
// UPDATE (last sweep of the finest level): the colour's final correction is also added to the
// FP64 iterate, x64_c += x_c.
template <class T, bool ZERO, bool UPDATE>
__device__ __forceinline__ void smooth_at(const LevelDev<T>& L, const T* __restrict__ invd, const T* __restrict__ r,
                                          T* __restrict__ x, int i, int j, int k, long long idx,
                                          double* __restrict__ x64) {
  T v = r[idx];
  if (!ZERO) {
    // FP32 sweeps rebuild the diagonal from the face weights they read anyway (saves the 1/diag
    // stream); FP64 sweeps read the stored 1/diag rather than pay an FP64 division.
    constexpr bool kOwnDiag = sizeof(T) == sizeof(float);
    T d = T(1);
    for_each_face(L, i, j, k, idx, [&](T w, int kind, long long nb) {
      if (kind == kInterior) {
        v = fma(w, x[nb], v);
        if (kOwnDiag) d += w;
      } else if (kind == kContinuous) {
        v = fma(-w, x[nb], v);
        if (kOwnDiag) d -= w;
      } else if (kind == kDirichlet) {
        if (kOwnDiag) d += w;
      }
    });
    if constexpr (kOwnDiag) v = __fdividef(v, d);
    else v *= invd[idx];
  } else {
    v *= invd[idx];
  }
  x[idx] = v;
  if (UPDATE && x64) x64[idx] += (double)v;
}

template <class T, bool ZERO, bool UPDATE>
__device__ __forceinline__ void smooth_colour_cell(const LevelDev<T>& L, const T* __restrict__ invd,
                                                   const T* __restrict__ r, T* __restrict__ x, int color, long long t,
                                                   double* __restrict__ x64) {
  int nxh = (L.n[0] + 1) >> 1;
  long long rows = (long long)L.n[1] * L.n[2];
  if (t >= (long long)nxh * rows) return;
  int m = (int)(t % nxh);
  long long row = t / nxh;
  int j = (int)(row % L.n[1]);
  int k = (int)(row / L.n[1]);
  int i = 2 * m + ((color + j + k) & 1);
  if (i >= L.n[0]) return;
  smooth_at<T, ZERO, UPDATE>(L, invd, r, x, i, j, k, (long long)i + (long long)L.n[0] * row, x64);
}

// coarse rhs of coarse cell idx = average over its 2^d children of the fine residual r - A x
template <class T>
__device__ __forceinline__ T restrict_at(const LevelDev<T>& F, const T* __restrict__ rf, const T* __restrict__ xf,
                                         int I, int J, int K) {
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
  return s / (T)(2 * o1max * o2max);
}

template <class T>
__device__ __forceinline__ T restrict_value(const LevelDev<T>& F, const T* __restrict__ rf, const T* __restrict__ xf,
                                            const int nc[3], long long idx) {
  int I = (int)(idx % nc[0]);
  long long rr = idx / nc[0];
  int J = (int)(rr % nc[1]);
  int K = (int)(rr / nc[1]);
  return restrict_at<T>(F, rf, xf, I, J, K);
}

// x_f += x_c(parent): piecewise-constant prolongation of the coarse correction
template <class T>
__device__ __forceinline__ void prolong_at(int ndim, const T* __restrict__ xc, const int nc[3], T* __restrict__ xf,
                                           int i, int j, int k, long long idx) {
  int I = i >> 1, J = ndim > 1 ? j >> 1 : j, K = ndim > 2 ? k >> 1 : k;
  xf[idx] += xc[(long long)I + (long long)nc[0] * ((long long)J + (long long)nc[1] * K)];
}

template <class T>
__device__ __forceinline__ void prolong_cell(const int nf[3], int ndim, const T* __restrict__ xc, const int nc[3],
                                             T* __restrict__ xf, long long idx) {
  int i = (int)(idx % nf[0]);
  long long r = idx / nf[0];
  int j = (int)(r % nf[1]);
  int k = (int)(r / nf[1]);
  prolong_at<T>(ndim, xc, nc, xf, i, j, k, idx);
}

// Coarsest level, executed by one whole block: x = 0, then `sweeps` red-black Gauss-Seidel
// sweeps (or damped Jacobi when a periodic axis has odd length and the colouring does not close).
template <class T>
__device__ __forceinline__ void coarse_solve_block(const LevelDev<T>& L, long long ncell, const T* __restrict__ invd,
                                                   const T* __restrict__ r, T* __restrict__ x, T* __restrict__ tmp,
                                                   int sweeps, int use_rb) {
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

// coarse_solve_block for a level of at most one cell per thread (xs and ts in shared memory):
// each thread gathers its cell's stencil once -- right-hand side, 1/diag, and for each face the
// signed weight (+w across interior and periodic faces, -w for the extrapolated neighbour of a
// continuous face, 0 otherwise) and the neighbour's index -- so that a sweep is six shared-memory
// reads and FMAs per cell between barriers.  The terms and their order are those of
// for_each_face, so the iterates equal coarse_solve_block's.
template <class T>
__device__ __forceinline__ void coarse_solve_small(const LevelDev<T>& L, int ncell, const T* __restrict__ invd,
                                                   const T* __restrict__ r, T* xs, T* ts, int sweeps, int use_rb) {
  const int c = threadIdx.x;
  const bool act = c < ncell;
  T cw[6], rv = T(0), id = T(0);
  int nb[6], par = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    cw[f] = T(0);
    nb[f] = act ? c : 0;
  }
  if (act) {
    int i, j, k;
    unflatten(L.n, c, i, j, k);
    par = (i + j + k) & 1;
    rv = r[c];
    id = invd[c];
    const int q[3] = {i, j, k};
    int stride = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < L.ndim) {
        const int n = L.n[a], p = q[a];
        const T wl = L.w[a][face_index(L.n, a, i, j, k, p)];
        const T wu = L.w[a][face_index(L.n, a, i, j, k, p + 1)];
        const int bl = L.bc[2 * a], bu = L.bc[2 * a + 1];
        if (p > 0) {
          cw[2 * a] = wl;
          nb[2 * a] = c - stride;
        } else if (bl == FLD_BC_PERIODIC) {
          cw[2 * a] = wl;
          nb[2 * a] = c + (n - 1) * stride;
        } else if (bl == FLD_BC_CONTINUOUS) {
          cw[2 * a] = -wl;
          nb[2 * a] = c + stride;
        }
        if (p < n - 1) {
          cw[2 * a + 1] = wu;
          nb[2 * a + 1] = c + stride;
        } else if (bu == FLD_BC_PERIODIC) {
          cw[2 * a + 1] = wu;
          nb[2 * a + 1] = c - (n - 1) * stride;
        } else if (bu == FLD_BC_CONTINUOUS) {
          cw[2 * a + 1] = -wu;
          nb[2 * a + 1] = c - stride;
        }
        stride *= n;
      }
    }
    xs[c] = T(0);
  }
  __syncthreads();
  for (int s = 0; s < sweeps; ++s) {
    if (use_rb) {
      for (int color = 0; color < 2; ++color) {
        if (act && par == color) {
          T v = rv;
#pragma unroll
          for (int f = 0; f < 6; ++f) v += cw[f] * xs[nb[f]];
          xs[c] = v * id;
        }
        __syncthreads();
      }
    } else {
      if (act) {
        T v = rv;
#pragma unroll
        for (int f = 0; f < 6; ++f) v += cw[f] * xs[nb[f]];
        ts[c] = T(0.2) * xs[c] + T(0.8) * v * id;
      }
      __syncthreads();
      if (act) xs[c] = ts[c];
      __syncthreads();
    }
  }
}

}  // namespace fld

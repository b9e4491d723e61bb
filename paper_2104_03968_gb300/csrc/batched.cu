// Many independent grids of uneven sizes, opacities and time steps advanced in one graph launch
// (the per-grid mathematics is that of fld_step: Sect. 2.2 coefficients, Sect. 3.4
// multigrid diffusion, Sect. 3.3 exchange).
//
// Design: every kernel of the single-grid path exists here in a level-synchronous batched
// form.  A kernel launch covers one operation for ALL grids: its blocks walk a tile list of
// (grid, level, first cell, count) entries, read the grid's descriptor, and run the same
// per-cell code as the single-grid kernels (coeffs.cuh, mg_device.cuh, exchange.cuh).  Grids
// have their own sizes, number of levels, opacity, time step and tolerance.  One step is one
// CUDA graph:
//     [exchange first]  coefficients  faces  fine setup  coarse operators  ||b||
//     WHILE (some grid not converged):  residual  check  V-cycle (levels down, coarsest, up)
//     [exchange last]
// The WHILE is a conditional graph node whose condition the check kernel sets on the device, so
// a step is a single graph launch with no host round trip between cycles.  Converged grids
// drop out: their blocks return at once.  The loop is bounded: every grid stops after its
// max_cycles, and the check kernel ends the loop after the largest max_cycles + 1 passes.
//
// Autotuning: on the first three calls for a batch shape, each (nu1, nu2, tile) candidate runs
// the step on scratch copies of the state; the candidate with the least summed time is kept for
// that shape (the first step alone is not typical of the ones that follow).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "batched.h"
#include "coeffs.cuh"
#include "exchange.cuh"
#include "kernels.h"
#include "mg_device.cuh"
#include "trace.h"

namespace fld {

namespace {

constexpr int kMaxLev = 16;
constexpr int kCheckThreads = 1024;

struct Tile {
  int grid;
  int level;
  long long start;
  long long count;
};

struct BFine {
  GridDev g;
  CoeffPhys ph;
  CoeffDf cdf;  // constants of the double-float coefficient path
  ExchangeParams xp;
  double dt;
  int order;
  int nlev;
  double* w64[3];
  double* b;
  double* diag;
  double* D;
  double* kappa;
  double* p;  // search direction of the conjugate-gradient outer loop (FP64, fine cells)
  const double* rho;
  double* eps;
  double* E;
};

template <class T>
struct BLev {
  LevelDev<T> L;
  T* invd;
  T* x;
  T* r;
  T* tmp;
  long long ncell;
  FastDiv f0, f1, fh;  // division by n[0], n[1] and (n[0] + 1) / 2: 32-bit index splitting
};

struct BState {
  int active;
  int cycles;
  int status;
  unsigned bad;
  int xiters;
  int xbis;
  int max_cycles;
  int tile_begin;
  int tile_end;
  int f64res;  // the residual of this grid is evaluated in FP64 (else double-float with a bound)
  int pcg;     // the outer loop is preconditioned conjugate gradients (symmetric operator)
  double rz, beta, alpha;  // its r.z of the last cycle and step coefficients
  double bb;
  double rel;
  double rtol;
};

__device__ __forceinline__ LevelDev<double> fine_level(const BFine& f) {
  LevelDev<double> L;
  for (int a = 0; a < 3; ++a) L.n[a] = f.g.n[a];
  L.ndim = f.g.ndim;
  for (int k = 0; k < 6; ++k) L.bc[k] = f.g.bc[k];
  for (int a = 0; a < 3; ++a) L.w[a] = f.w64[a];
  return L;
}

// ----------------------------------------------------------------------------- kernels

__global__ void kb_reset(int ng, BState* __restrict__ st, int* __restrict__ ctl) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng) {
    st[g].active = 1;
    st[g].cycles = 0;
    st[g].status = FLD_ERR_NOT_CONVERGED;
    st[g].bad = 0;
    st[g].xiters = 0;
    st[g].xbis = 0;
    st[g].rel = 0.0;
    st[g].f64res = 0;
    st[g].rz = st[g].beta = st[g].alpha = 0.0;
  }
  if (g == 0) ctl[0] = ctl[1] = 0;
}

// phase 0: grids whose order is exchange-then-diffuse (kappa from the opacity model);
// phase 1: grids whose order is diffuse-then-exchange (kappa^n from the coefficient stage)
__global__ void kb_exchange(const Tile* __restrict__ tiles, const BFine* __restrict__ fine, BState* __restrict__ st,
                            int phase) {
  const Tile tl = tiles[blockIdx.x];
  const BFine& f = fine[tl.grid];
  bool mine = (f.order == FLD_ORDER_EXCHANGE_THEN_DIFFUSE) == (phase == 0);
  if (!mine) return;
  int iters = 0, bis = 0;
  bool bad = false;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    long long idx = tl.start + c;
    double r = f.rho[idx], e = f.eps[idx], En = f.E[idx];
    double k = phase == 0 ? opacity(f.ph.op, r, temperature(f.ph.gamma, f.ph.gas_R, r, e)) : f.kappa[idx];
    int it = 0, bi = 0;
    if (exchange_cell_fast(f.xp, r, k, e, En, it, bi)) {
      f.eps[idx] = e;
      f.E[idx] = En;
    } else {
      bad = true;
    }
    iters = max(iters, it);
    bis += bi;
  }
  if (bad) atomicOr(&st[tl.grid].bad, kStatNonpositive);
  exchange_report(iters, bis, &st[tl.grid].xiters, &st[tl.grid].xbis);
}

__global__ void kb_coeffs(const Tile* __restrict__ tiles, const BFine* __restrict__ fine, BState* __restrict__ st) {
  const Tile tl = tiles[blockIdx.x];
  const BFine& f = fine[tl.grid];
  bool bad = false;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    long long idx = tl.start + c;
    double kap, D;
    const int ic = (int)idx, r = ic / f.g.n[0];  // a grid of the batch has fewer than 2^31 cells
    if (!coeffs_cell_fast(f.g, f.ph, f.cdf, f.E, f.rho, f.eps, idx, ic - r * f.g.n[0], r % f.g.n[1], r / f.g.n[1], kap,
                          D))
      bad = true;
    f.kappa[idx] = kap;
    f.D[idx] = D;
  }
  if (bad) atomicOr(&st[tl.grid].bad, kStatNonpositive);
}

template <class T>
__global__ void kb_faces(const Tile* __restrict__ tiles, const BFine* __restrict__ fine, const BLev<T>* __restrict__ lev) {
  const Tile tl = tiles[blockIdx.x];
  const BFine& f = fine[tl.grid];
  const BLev<T>& L0 = lev[tl.grid * kMaxLev];
  const bool copy = sizeof(T) == sizeof(float);
  const double* const Dax[3] = {f.D, f.D, f.D};
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int q[3];
    unflatten32(idx, L0.f0, L0.f1, q[0], q[1], q[2]);
    if (copy)
      faces_cell_at<float>(f.g, f.dt, Dax, q, idx, f.w64[0], f.w64[1], f.w64[2], (float*)L0.L.w[0],
                           (float*)L0.L.w[1], (float*)L0.L.w[2]);
    else
      faces_cell_at<double>(f.g, f.dt, Dax, q, idx, f.w64[0], f.w64[1], f.w64[2], nullptr, nullptr, nullptr);
  }
}

template <class T>
__global__ void kb_fine_setup(const Tile* __restrict__ tiles, const BFine* __restrict__ fine,
                              const BLev<T>* __restrict__ lev) {
  const Tile tl = tiles[blockIdx.x];
  const BFine& f = fine[tl.grid];
  LevelDev<double> L = fine_level(f);
  const BLev<T>& L0 = lev[tl.grid * kMaxLev];
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int i, j, k;
    unflatten32(idx, L0.f0, L0.f1, i, j, k);
    fine_setup_at<T>(L, f.g, f.E, i, j, k, idx, f.b, f.diag, L0.invd);
  }
}

// coarse level l (tile list over its cells): lower faces of each cell and the faces n_a it owns,
// from the level l-1 faces; then 1/diagonal in a second kernel
template <class T>
__global__ void kb_coarse_faces(const Tile* __restrict__ tiles, const BLev<T>* __restrict__ lev) {
  const Tile tl = tiles[blockIdx.x];
  const BLev<T>& C = lev[tl.grid * kMaxLev + tl.level];
  const BLev<T>& F = lev[tl.grid * kMaxLev + tl.level - 1];
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int q[3];
    unflatten32(idx, C.f0, C.f1, q[0], q[1], q[2]);
    for (int a = 0; a < C.L.ndim; ++a) {
      long long f0 = face_index(C.L.n, a, q[0], q[1], q[2], q[a]);
      T* wc = const_cast<T*>(C.L.w[a]);
      wc[f0] = coarse_face_at<T>(a, C.L.ndim, F.L.n, q, F.L.w[a]);
      bool periodic = C.L.bc[2 * a + 1] == FLD_BC_PERIODIC;
      if ((periodic && q[a] == 0) || (!periodic && q[a] == C.L.n[a] - 1)) {
        long long fn = face_index(C.L.n, a, q[0], q[1], q[2], C.L.n[a]);
        int qn[3] = {q[0], q[1], q[2]};
        qn[a] = C.L.n[a];
        wc[fn] = coarse_face_at<T>(a, C.L.ndim, F.L.n, qn, F.L.w[a]);
      }
    }
  }
}

template <class T>
__global__ void kb_invd(const Tile* __restrict__ tiles, const BLev<T>* __restrict__ lev) {
  const Tile tl = tiles[blockIdx.x];
  const BLev<T>& C = lev[tl.grid * kMaxLev + tl.level];
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int i, j, k;
    unflatten32(idx, C.f0, C.f1, i, j, k);
    C.invd[idx] = T(1) / diag_of(C.L, i, j, k, idx);
  }
}

__global__ void kb_sumsq_b(const Tile* __restrict__ tiles, const BFine* __restrict__ fine, double* __restrict__ parts) {
  const Tile tl = tiles[blockIdx.x];
  const double* b = fine[tl.grid].b;
  double v = 0.0;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) v = fma(b[tl.start + c], b[tl.start + c], v);
  v = block_sum(v);
  if (threadIdx.x == 0) parts[blockIdx.x] = v;
}

__global__ void kb_bnorm(int ng, const double* __restrict__ parts, BState* __restrict__ st) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  double s = 0.0;
  for (int t = st[g].tile_begin; t < st[g].tile_end; ++t) s += parts[t];
  st[g].bb = s;
}

// r = b - A x of one fine cell in FP64 (out of line: the fallback of the double-float path)
static __device__ __noinline__ double residual_f64(const LevelDev<double>& L, const double* __restrict__ x,
                                                   const double* __restrict__ b, const double* __restrict__ diag,
                                                   int i, int j, int k, long long idx) {
  double s = fma(-diag[idx], x[idx], b[idx]);
  for_each_face(L, i, j, k, idx, [&](double w, int kind, long long nb) {
    if (kind == kInterior) s = fma(w, x[nb], s);
    else if (kind == kContinuous) s = fma(-w, x[nb], s);
  });
  return s;
}

// The same in double-float on the FP32 pipe (~16 splits and operations of relative error below
// 2^-46 each, so the error is below 2^-41 times the sum of the terms' magnitudes, returned in mag
// as that bound).  ok is false when an input lies outside the double-float window.
__device__ __forceinline__ dfl residual_df(const LevelDev<double>& L, const double* __restrict__ x,
                                           const double* __restrict__ b, const double* __restrict__ diag, int i,
                                           int j, int k, long long idx, float& bound, bool& ok) {
  dfl xc, bc, dc;
  bool o1, o2, o3;
  split_f64_try(x[idx], xc.hi, xc.lo, o1);
  split_f64_try(b[idx], bc.hi, bc.lo, o2);
  split_f64_try(diag[idx], dc.hi, dc.lo, o3);
  ok = o1 && o2 && o3;
  const dfl dx = df_mul(dc, xc);
  dfl s = df_add(bc, df_neg(dx));
  float mag = fabsf(bc.hi) + fabsf(dx.hi);
  for_each_face(L, i, j, k, idx, [&](double w, int kind, long long nb) {
    if (kind != kInterior && kind != kContinuous) return;
    dfl wf, xn;
    bool ow, ox;
    split_f64_try(w, wf.hi, wf.lo, ow);
    split_f64_try(x[nb], xn.hi, xn.lo, ox);
    ok = ok && ow && ox;
    const dfl p = df_mul(wf, xn);
    s = df_add(s, kind == kInterior ? p : df_neg(p));
    mag += fabsf(p.hi);
  });
  ok = ok && mag < 1e30f;
  bound = 0x1p-41f * mag * 1.01f;  // 1.01: the FP32 sum of the magnitudes
  return s;
}

// r = b - A x on the fine cells of a tile in T for the inner V-cycle.  parts[blk] = sum r^2 and,
// in the double-float form (mixed precision, unless the grid fell back to FP64), parts[nt + blk] =
// sum of the squared per-cell error bounds.
template <class T>
__global__ void __launch_bounds__(256, 4)
    kb_residual(const Tile* __restrict__ tiles, const BFine* __restrict__ fine, const BLev<T>* __restrict__ lev,
                const BState* __restrict__ st, double* __restrict__ parts) {
  const Tile tl = tiles[blockIdx.x];
  if (!st[tl.grid].active) return;
  const BFine& f = fine[tl.grid];
  LevelDev<double> L = fine_level(f);
  const BLev<T>& L0 = lev[tl.grid * kMaxLev];
  const bool use_df = sizeof(T) == sizeof(float) && !st[tl.grid].f64res;
  double acc = 0.0, err = 0.0;
  // the double-float form sums r^2 and bound^2 of its cells in FP32 (a tile gives a thread at most
  // tile / blockDim cells), then once in FP64.  Both are first scaled by 2^-e, 2^(e-1) <= rms(b) <
  // 2^e, so that grids of any magnitude neither underflow nor overflow in the squares: relative to
  // rms(b) a converging residual stays far above 2^-63 and the bounds near 2^-41.  Scaled values of
  // 2^60 or more take the FP64 accumulator.
  int e2 = 0;
  if (use_df) {
    const double bb = st[tl.grid].bb;
    const double ncell = (double)f.g.n[0] * (double)f.g.n[1] * (double)f.g.n[2];
    if (bb > 0.0) (void)frexp(sqrt(bb / ncell), &e2);
  }
  const float sc = ldexpf(1.0f, -e2);
  float facc = 0.0f, ferr = 0.0f;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int i, j, k;
    unflatten32(idx, L0.f0, L0.f1, i, j, k);
    if (!use_df) {
      acc = fma_residual_at<T>(L, f.E, f.E, f.b, f.diag, L0.r, i, j, k, idx, acc);
      continue;
    }
    float bound;
    bool ok;
    const dfl s = residual_df(L, f.E, f.b, f.diag, i, j, k, idx, bound, ok);
    const float hs = s.hi * sc, bs = bound * sc;
    if (ok && fabsf(hs) < 0x1p60f && bs < 0x1p60f) {
      L0.r[idx] = (T)(s.hi + s.lo);
      facc = fmaf(hs, hs, facc);
      ferr = fmaf(bs, bs, ferr);
    } else {
      const double r = residual_f64(L, f.E, f.b, f.diag, i, j, k, idx);
      L0.r[idx] = (T)r;
      acc = fma(r, r, acc);
    }
  }
  acc += ldexp((double)facc, 2 * e2);
  err += ldexp((double)ferr, 2 * e2);
  acc = block_sum(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
  if (use_df) {
    __syncthreads();  // block_sum's shared scratch is reused
    err = block_sum(err);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = err;
  }
}

// One block: per-grid convergence decision, then the WHILE condition for the next pass.  A grid
// whose residual was double-float (mixed, nt = the residual's tile count) converges when the
// residual plus the bound on its error meets the tolerance, so the true residual does; while the
// bound is above a quarter of the tolerance it could stall convergence, and the grid's later
// residuals are FP64.
__global__ void kb_check(int ng, const double* __restrict__ parts, BState* __restrict__ st, int* __restrict__ ctl,
                         int iter_cap, int mixed, int nt, cudaGraphConditionalHandle handle) {
  __shared__ int nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  int mine = 0;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    BState& s = st[g];
    if (!s.active) continue;
    double rr = 0.0;
    for (int t = s.tile_begin; t < s.tile_end; ++t) rr += parts[t];
    double rel = s.bb > 0 ? sqrt(rr / s.bb) : sqrt(rr);
    double bnd = 0.0;
    if (mixed && !s.f64res) {
      double ee = 0.0;
      for (int t = s.tile_begin; t < s.tile_end; ++t) ee += parts[nt + t];
      // 1.001 and 2^-18 rel: the FP32 partial sums of the squares (relative error below
      // (tile / blockDim) 2^-24 <= 2^-19)
      bnd = 1.001 * (s.bb > 0 ? sqrt(ee / s.bb) : sqrt(ee)) + 0x1p-18 * rel;
    }
    s.rel = rel;
    if (!(rel == rel) || rel > 1e300) {
      s.active = 0;
      s.status = FLD_ERR_NONFINITE;
    } else if (rel + bnd <= s.rtol) {
      s.active = 0;
      s.status = FLD_OK;
    } else if (s.cycles >= s.max_cycles) {
      s.active = 0;
      s.status = FLD_ERR_NOT_CONVERGED;
    } else {
      s.cycles += 1;  // a V-cycle follows in this pass
      if (bnd > 0.25 * s.rtol) s.f64res = 1;
      ++mine;
    }
  }
  if (mine) atomicAdd(&nact, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    int it = ++ctl[1];
    ctl[0] = nact;
    cudaGraphSetConditional(handle, (nact > 0 && it <= iter_cap) ? 1u : 0u);
  }
}

template <class T, bool ZERO, bool UPDATE>
__global__ void kb_smooth(const Tile* __restrict__ tiles, const BLev<T>* __restrict__ lev, const BState* __restrict__ st,
                          const BFine* __restrict__ fine, int color) {
  const Tile tl = tiles[blockIdx.x];
  if (!st[tl.grid].active) return;
  const BLev<T>& B = lev[tl.grid * kMaxLev + tl.level];
  // a conjugate-gradient grid takes the V-cycle's result as its preconditioned residual instead
  double* x64 = UPDATE && !st[tl.grid].pcg ? fine[tl.grid].E : nullptr;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    // thread t of the colour: half-row position m, row (j, k); the tile list covers exactly
    // ((n[0] + 1) / 2) n[1] n[2] threads
    const unsigned t = (unsigned)(tl.start + c);
    const unsigned row = fast_div(t, B.fh);
    const unsigned kk = fast_div(row, B.f1);
    const int m = (int)(t - row * B.fh.d), j = (int)(row - kk * B.f1.d), k = (int)kk;
    const int i = 2 * m + ((color + j + k) & 1);
    if (i >= B.L.n[0]) continue;
    smooth_at<T, ZERO, UPDATE>(B.L, B.invd, B.r, B.x, i, j, k, (long long)i + (long long)B.L.n[0] * row, x64);
  }
}

// Where a 2-D level's iterate is: the fused sweeps alternate between x and tmp (a sweep cannot
// update the array its neighbouring tiles are still reading), the host tracks which one holds it
// at each point of the V-cycle.  Levels of 3-D grids and coarsest levels keep it in x.
template <class T>
__device__ __forceinline__ T* iterate_of(const BLev<T>& B, bool in_tmp) {
  return (in_tmp && B.L.ndim == 2) ? B.tmp : B.x;
}

// tiles over the coarse cells of level l+1 (tile.level = l); f_tmp: level l's iterate is in tmp
template <class T>
__global__ void kb_restrict(const Tile* __restrict__ tiles, const BLev<T>* __restrict__ lev, const BState* __restrict__ st,
                            int f_tmp) {
  const Tile tl = tiles[blockIdx.x];
  if (!st[tl.grid].active) return;
  const BLev<T>& F = lev[tl.grid * kMaxLev + tl.level];
  const BLev<T>& C = lev[tl.grid * kMaxLev + tl.level + 1];
  const T* xf = iterate_of(F, f_tmp);
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int I, J, K;
    unflatten32(idx, C.f0, C.f1, I, J, K);
    C.r[idx] = restrict_at<T>(F.L, F.r, xf, I, J, K);
  }
}

// tiles over the cells of level l (tile.level = l); f_tmp / c_tmp: where the iterates of levels l
// and l+1 are (a grid's coarsest level is always in x)
template <class T>
__global__ void kb_prolong(const Tile* __restrict__ tiles, const BLev<T>* __restrict__ lev, const BState* __restrict__ st,
                           const BFine* __restrict__ fine, int f_tmp, int c_tmp) {
  const Tile tl = tiles[blockIdx.x];
  if (!st[tl.grid].active) return;
  const BLev<T>& F = lev[tl.grid * kMaxLev + tl.level];
  const BLev<T>& C = lev[tl.grid * kMaxLev + tl.level + 1];
  T* xf = iterate_of(F, f_tmp);
  const T* xc = iterate_of(C, c_tmp && tl.level + 1 < fine[tl.grid].nlev - 1);
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const unsigned idx = (unsigned)(tl.start + c);
    int i, j, k;
    unflatten32(idx, F.f0, F.f1, i, j, k);
    prolong_at<T>(F.L.ndim, xc, C.L.n, xf, i, j, k, idx);
  }
}

// ----------------------------------------------------------------------------- conjugate gradients
//
// On a grid with no linear-extrapolation face the operator A of Eq. discdiff (harmonic-mean faces,
// Dirichlet, Neumann or periodic boundaries) is symmetric positive definite, and its outer loop runs
// preconditioned conjugate gradients with the V-cycle as the preconditioner: z = V(r),
// beta = (r.z) / (r.z)_previous (0 on the grid's first cycle), p = z + beta p,
// alpha = (r.z) / (p.A p), x += alpha p.  The r of each pass is the true residual b - A x
// (kb_residual), so the convergence test and its error bound are those of the plain loop, and a
// cycle costs one more application of A.  Grids with such a face keep the plain loop x += z.

// where a grid's level-0 V-cycle result is: in tmp for 2-D grids whose fused sweeps left it there
template <class T>
__device__ __forceinline__ const T* vcycle_out(const BFine& f, const BLev<T>& L0, int z2d_tmp) {
  return (f.g.ndim == 2 && f.nlev > 1 && z2d_tmp) ? L0.tmp : L0.x;
}

// parts[blk] = sum of r z over the tile (0 for the tiles of other grids)
template <class T>
__global__ void kb_pcg_rz(const Tile* __restrict__ tiles, const BFine* __restrict__ fine,
                          const BLev<T>* __restrict__ lev, const BState* __restrict__ st, double* __restrict__ parts,
                          int z2d_tmp) {
  const Tile tl = tiles[blockIdx.x];
  double acc = 0.0;
  if (st[tl.grid].active && st[tl.grid].pcg) {
    const BLev<T>& L0 = lev[tl.grid * kMaxLev];
    const T* z = vcycle_out(fine[tl.grid], L0, z2d_tmp);
    for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
      const long long idx = tl.start + c;
      acc = fma((double)L0.r[idx], (double)z[idx], acc);
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

// one block: each conjugate-gradient grid's r.z and beta
__global__ void kb_pcg_beta(int ng, const double* __restrict__ parts, BState* __restrict__ st) {
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    BState& s = st[g];
    if (!s.active || !s.pcg) continue;
    double rz = 0.0;
    for (int t = s.tile_begin; t < s.tile_end; ++t) rz += parts[t];
    s.beta = (s.cycles <= 1 || !(s.rz > 0.0) || !(rz == rz)) ? 0.0 : rz / s.rz;
    s.rz = rz;
  }
}

// p = z + beta p (p = z where beta is 0: p holds the previous step's direction); parts[blk] =
// sum of p (A p) over the tile, A in FP64 from the fine weights and diagonal
template <class T>
__global__ void kb_pcg_dir(const Tile* __restrict__ tiles, const BFine* __restrict__ fine,
                           const BLev<T>* __restrict__ lev, const BState* __restrict__ st, int z2d_tmp) {
  const Tile tl = tiles[blockIdx.x];
  const BState& s = st[tl.grid];
  if (!s.active || !s.pcg) return;
  const BFine& f = fine[tl.grid];
  const T* z = vcycle_out(f, lev[tl.grid * kMaxLev], z2d_tmp);
  const double beta = s.beta;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const long long idx = tl.start + c;
    f.p[idx] = beta == 0.0 ? (double)z[idx] : fma(beta, f.p[idx], (double)z[idx]);
  }
}

template <class T>
__global__ void kb_pcg_ap(const Tile* __restrict__ tiles, const BFine* __restrict__ fine,
                          const BLev<T>* __restrict__ lev, const BState* __restrict__ st,
                          double* __restrict__ parts) {
  const Tile tl = tiles[blockIdx.x];
  double acc = 0.0;
  if (st[tl.grid].active && st[tl.grid].pcg) {
    const BFine& f = fine[tl.grid];
    const BLev<T>& L0 = lev[tl.grid * kMaxLev];
    const LevelDev<double> L = fine_level(f);
    const double* __restrict__ p = f.p;
    for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
      const unsigned idx = (unsigned)(tl.start + c);
      int i, j, k;
      unflatten32(idx, L0.f0, L0.f1, i, j, k);
      const double pc = p[idx];
      double ap = f.diag[idx] * pc;
      for_each_face(L, i, j, k, (long long)idx, [&](double w, int kind, long long nb) {
        if (kind == kInterior) ap = fma(-w, p[nb], ap);
        else if (kind == kContinuous) ap = fma(w, p[nb], ap);
      });
      acc = fma(pc, ap, acc);
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

// one block: alpha = r.z / p.A p (1 where p.A p is not positive: the plain correction)
__global__ void kb_pcg_alpha(int ng, const double* __restrict__ parts, BState* __restrict__ st) {
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    BState& s = st[g];
    if (!s.active || !s.pcg) continue;
    double pap = 0.0;
    for (int t = s.tile_begin; t < s.tile_end; ++t) pap += parts[t];
    const double a = s.rz / pap;
    s.alpha = (pap > 0.0 && a == a && a > 0.0 && a < 1e300) ? a : 1.0;
  }
}

// x += alpha p
__global__ void kb_pcg_x(const Tile* __restrict__ tiles, const BFine* __restrict__ fine,
                         const BState* __restrict__ st) {
  const Tile tl = tiles[blockIdx.x];
  const BState& s = st[tl.grid];
  if (!s.active || !s.pcg) return;
  const BFine& f = fine[tl.grid];
  const double a = s.alpha;
  for (long long c = threadIdx.x; c < tl.count; c += blockDim.x) {
    const long long idx = tl.start + c;
    f.E[idx] = fma(a, f.p[idx], f.E[idx]);
  }
}

// ----------------------------------------------------------------------------- fused 2-D sweep
//
// One red-black Gauss-Seidel sweep of a 2-D level (colour c0, then 1 - c0) in a single pass over
// memory.  A block owns a kSwX x kSwY tile of one grid's level and stages the iterate of the tile
// and two cells around it in shared memory (wrapped across periodic boundaries).  It updates
// colour c0 on the tile and one cell around it -- the cells around are updated again by the tiles
// that own them, from the same inputs with the same operations, so the copies agree -- then
// colour 1 - c0 on the tile, whose neighbours are now all final, and writes the tile.  The
// per-cell arithmetic is smooth_at's, term for term, so the iterates equal those of two
// colour launches.  Because neighbouring tiles stage cells this block writes, a sweep reads one
// array and writes the other (x <-> tmp); the first sweep from zero reads no iterate and writes x.

constexpr int kSwX = 64, kSwY = 32;  // cells of a tile

struct Tile2 {
  int grid;
  int level;
  int i0;
  int j0;
};

// grid coordinate of a staged position p in [-2, n + 2): wrapped on a periodic axis (n >= 4 on a
// smoothed level), false beyond a non-periodic boundary
__device__ __forceinline__ bool sw_coord(int p, int n, bool periodic, int& out) {
  if (p >= 0 && p < n) {
    out = p;
    return true;
  }
  if (!periodic) return false;
  out = p < 0 ? p + n : p - n;
  return true;
}

// contribution of one face, as for_each_face classifies it: across = the neighbour through the
// face (interior or periodic), inward = the next cell inward (the continuous boundary's ghost)
template <class T>
__device__ __forceinline__ void sw_face(T w, bool inner, int bc, T across, T inward, T& v, T& d) {
  constexpr bool kOwnDiag = sizeof(T) == sizeof(float);
  if (inner || bc == FLD_BC_PERIODIC) {
    v = fma(w, across, v);
    if (kOwnDiag) d += w;
  } else if (bc == FLD_BC_DIRICHLET) {
    if (kOwnDiag) d += w;
  } else if (bc == FLD_BC_CONTINUOUS) {
    v = fma(-w, inward, v);
    if (kOwnDiag) d -= w;
  }
}

// Asynchronous global -> shared copy of one element (cp.async, sm_80 and later): a thread issues
// all its copies before waiting on any, so a tile's loads are in flight together.
template <class T>
__device__ __forceinline__ void sw_copy(T* smem, const T* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(sizeof(T)));
}
__device__ __forceinline__ void sw_copy_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Staged arrays of a tile with a halo of H cells: each (kSwY + 2H) x (kSwX + 2H), holding the
// iterate, the right-hand side, the lower x- and y-faces of each position, and 1/diag (the FP64
// smoother, and the first sweep from zero).  H = 2 for a sweep; H = 3 for the last pre-sweep,
// which also restricts its residual (below).
template <int H>
struct SwShape {
  static constexpr int W = kSwX + 2 * H;  // staged row length
  static constexpr int S = (kSwY + 2 * H) * W;
};
template <class T, bool ZERO>
__host__ __device__ constexpr int sw_arrays() {
  return (ZERO || sizeof(T) == sizeof(double)) ? 5 : 4;
}

// smooth_at for a 2-D cell at staged position e (global gi, gj): the upper faces are the lower
// faces of the next positions, except on the last row / column, whose own upper face (index n)
// is read from memory
template <class T, int W>
__device__ __forceinline__ T sw_cell(const BLev<T>& B, const T* xs, const T* rs, const T* wxs, const T* wys,
                                     const T* is, int e, int gi, int gj) {
  const int n0 = B.L.n[0], n1 = B.L.n[1];
  T v = rs[e], d = T(1);
  const T wxu = gi < n0 - 1 ? wxs[e + 1] : B.L.w[0][n0 + (long long)(n0 + 1) * gj];
  const T wyu = gj < n1 - 1 ? wys[e + W] : B.L.w[1][gi + (long long)n0 * n1];
  sw_face<T>(wxs[e], gi > 0, B.L.bc[0], xs[e - 1], xs[e + 1], v, d);
  sw_face<T>(wxu, gi < n0 - 1, B.L.bc[1], xs[e + 1], xs[e - 1], v, d);
  sw_face<T>(wys[e], gj > 0, B.L.bc[2], xs[e - W], xs[e + W], v, d);
  sw_face<T>(wyu, gj < n1 - 1, B.L.bc[3], xs[e + W], xs[e - W], v, d);
  if constexpr (sizeof(T) == sizeof(float)) return __fdividef(v, d);
  else return v * is[e];
}

// (A x)_c of restrict_at's residual for a staged cell, its terms in for_each_face's order
template <class T>
__device__ __forceinline__ void sw_ax_face(T w, bool inner, int bc, T xv, T across, T inward, T& ax) {
  if (inner || bc == FLD_BC_PERIODIC) ax += w * (xv - across);
  else if (bc == FLD_BC_DIRICHLET) ax += w * xv;
  else if (bc == FLD_BC_CONTINUOUS) ax += w * (inward - xv);
}
template <class T, int W>
__device__ __forceinline__ T sw_ax(const BLev<T>& B, const T* xs, const T* wxs, const T* wys, int e, int gi, int gj) {
  const int n0 = B.L.n[0], n1 = B.L.n[1];
  const T xv = xs[e];
  const T wxu = gi < n0 - 1 ? wxs[e + 1] : B.L.w[0][n0 + (long long)(n0 + 1) * gj];
  const T wyu = gj < n1 - 1 ? wys[e + W] : B.L.w[1][gi + (long long)n0 * n1];
  T ax = xv;
  sw_ax_face<T>(wxs[e], gi > 0, B.L.bc[0], xv, xs[e - 1], xs[e + 1], ax);
  sw_ax_face<T>(wxu, gi < n0 - 1, B.L.bc[1], xv, xs[e + 1], xs[e - 1], ax);
  sw_ax_face<T>(wys[e], gj > 0, B.L.bc[2], xv, xs[e - W], xs[e + W], ax);
  sw_ax_face<T>(wyu, gj < n1 - 1, B.L.bc[3], xv, xs[e + W], xs[e - W], ax);
  return ax;
}

// ZERO: the sweep starts from x = 0 (writes x); otherwise it reads x (from_tmp = 0) or tmp and
// writes the other.  UPDATE: the finest level's last sweep also adds the result to the FP64
// iterate.  RESTRICT (the last pre-sweep): the halo is three cells, colour c0 is updated two cells
// around the tile and colour 1 - c0 one cell around it, so that every neighbour of a tile cell is
// final; the block then forms the residual r - A x of its cells and writes the average of each
// 2 x 2 block to the next level's right-hand side (restrict_at, term for term; tile origins and
// the sizes of smoothed levels are even).  Dynamic shared memory: sw_smem_bytes().
template <class T, bool ZERO, bool UPDATE, bool RESTRICT>
__global__ void __launch_bounds__(256) kb_sweep2d(const Tile2* __restrict__ tiles, const BLev<T>* __restrict__ lev,
                                                  const BState* __restrict__ st, const BFine* __restrict__ fine,
                                                  int c0, int from_tmp) {
  constexpr int H = RESTRICT ? 3 : 2;
  constexpr int W = SwShape<H>::W, S = SwShape<H>::S;
  extern __shared__ __align__(16) unsigned char sw_smem[];
  T* xs = reinterpret_cast<T*>(sw_smem);
  T* rs = xs + S;
  T* wxs = rs + S;
  T* wys = wxs + S;
  T* is = wys + S;  // only with sw_arrays() == 5
  constexpr bool kInvd = sw_arrays<T, ZERO>() == 5;
  const Tile2 tl = tiles[blockIdx.x];
  if (!st[tl.grid].active) return;
  const BLev<T>& B = lev[tl.grid * kMaxLev + tl.level];
  const int n0 = B.L.n[0], n1 = B.L.n[1];
  const bool px = B.L.bc[0] == FLD_BC_PERIODIC, py = B.L.bc[2] == FLD_BC_PERIODIC;
  const int w = min(kSwX, n0 - tl.i0), h = min(kSwY, n1 - tl.j0);
  const int nst = (h + 2 * H) * W;
  T* dst = (ZERO || from_tmp) ? B.x : B.tmp;
  const T* src = from_tmp ? B.tmp : B.x;
  for (int e = threadIdx.x; e < nst; e += blockDim.x) {
    const int lj = e / W, li = e - lj * W;
    int gi, gj;
    if (li < w + 2 * H && sw_coord(tl.i0 + li - H, n0, px, gi) && sw_coord(tl.j0 + lj - H, n1, py, gj)) {
      const long long idx = gi + (long long)n0 * gj;
      if (!ZERO) sw_copy(xs + e, src + idx);
      sw_copy(rs + e, B.r + idx);
      sw_copy(wxs + e, B.L.w[0] + gi + (long long)(n0 + 1) * gj);
      sw_copy(wys + e, B.L.w[1] + idx);
      if (kInvd) sw_copy(is + e, B.invd + idx);
    }
  }
  sw_copy_wait();
  __syncthreads();
  // A smoothed level has even sizes, so wrapping keeps parities and the tile origin is even: in
  // staged row lj the cells of a colour are the staged columns li with li = colour + j0 + lj (mod 2).
  // Each half-sweep walks only its colour's cells, W / 2 per staged row.
  for (int ph = 0; ph < 2; ++ph) {
    const int colour = ph ? 1 - c0 : c0;
    const int m = H - (ph ? (RESTRICT ? 1 : 0) : (RESTRICT ? 2 : 1));  // first staged row / column updated
    const int nrow = h + 2 * H - 2 * m;
    for (int t = threadIdx.x; t < nrow * (W / 2); t += blockDim.x) {
      const int q = t / (W / 2), lj = q + m;
      const int li = 2 * (t - q * (W / 2)) + ((colour + tl.j0 + lj) & 1);
      if (li < m || li >= w + 2 * H - m) continue;
      int gi, gj;
      if (!sw_coord(tl.i0 + li - H, n0, px, gi) || !sw_coord(tl.j0 + lj - H, n1, py, gj)) continue;
      const int e = lj * W + li;
      xs[e] = (ZERO && ph == 0) ? rs[e] * is[e] : sw_cell<T, W>(B, xs, rs, wxs, wys, is, e, gi, gj);
    }
    __syncthreads();
  }
  double* x64 = UPDATE && !st[tl.grid].pcg ? fine[tl.grid].E : nullptr;
  for (int e = threadIdx.x; e < h * W; e += blockDim.x) {
    const int lj = e / W, li = e - lj * W;
    if (li >= w) continue;
    const long long idx = (tl.i0 + li) + (long long)n0 * (tl.j0 + lj);
    const T v = xs[e + H * W + H];
    dst[idx] = v;
    if (UPDATE && x64) x64[idx] += (double)v;
  }
  if (RESTRICT) {
    const BLev<T>& C = lev[tl.grid * kMaxLev + tl.level + 1];
    const int wc = w >> 1, hc = h >> 1;
    for (int t = threadIdx.x; t < hc * (kSwX / 2); t += blockDim.x) {
      const int J = t / (kSwX / 2), I = t - J * (kSwX / 2);
      if (I >= wc) continue;
      T sum = T(0);
      for (int o1 = 0; o1 < 2; ++o1)
        for (int o0 = 0; o0 < 2; ++o0) {
          const int li = 2 * I + o0, lj = 2 * J + o1;
          const int e = (lj + H) * W + li + H;
          sum += rs[e] - sw_ax<T, W>(B, xs, wxs, wys, e, tl.i0 + li, tl.j0 + lj);
        }
      C.r[(tl.i0 / 2 + I) + (long long)C.L.n[0] * (tl.j0 / 2 + J)] = sum / T(4);
    }
  }
}

template <class T, bool ZERO, bool UPDATE, bool RESTRICT>
constexpr size_t sw_smem_bytes() {
  return (size_t)sw_arrays<T, ZERO>() * SwShape<RESTRICT ? 3 : 2>::S * sizeof(T);
}

// one block per grid at its coarsest level (tile.level); a single-level grid adds its
// correction to the FP64 iterate here.  A level of at most one cell per thread keeps its stencil
// in registers and the iterate in shared memory (the same iterates as the global-memory form).
constexpr int kCoarseThreads = 1024;

template <class T>
__global__ void __launch_bounds__(kCoarseThreads, 1)
    kb_coarse(const Tile* __restrict__ tiles, const BLev<T>* __restrict__ lev, const BState* __restrict__ st,
              const BFine* __restrict__ fine) {
  __shared__ T xs[2 * kCoarseThreads];
  const Tile tl = tiles[blockIdx.x];
  if (!st[tl.grid].active) return;
  const BLev<T>& B = lev[tl.grid * kMaxLev + tl.level];
  bool rb = true;
  for (int a = 0; a < B.L.ndim; ++a)
    if ((B.L.n[a] & 1) && B.L.bc[2 * a] == FLD_BC_PERIODIC) rb = false;
  if (B.ncell <= (long long)blockDim.x) {
    const int n = (int)B.ncell;
    coarse_solve_small<T>(B.L, n, B.invd, B.r, xs, xs + n, rb ? 40 : 80, rb ? 1 : 0);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) B.x[c] = xs[c];
  } else {
    coarse_solve_block<T>(B.L, B.ncell, B.invd, B.r, B.x, B.tmp, rb ? 40 : 80, rb ? 1 : 0);
  }
  if (tl.level == 0) {
    __syncthreads();
    double* E = fine[tl.grid].E;
    for (long long c = threadIdx.x; c < B.ncell; c += blockDim.x) E[c] += (double)B.x[c];
  }
}

// ----------------------------------------------------------------------------- host helpers

GridDev grid_dev(const fld_grid& g) {
  GridDev d{};
  d.ndim = g.ndim;
  for (int a = 0; a < 3; ++a) {
    d.n[a] = g.n[a];
    d.dx[a] = a < g.ndim ? g.dx[a] : 1.0;
    d.inv_dx2[a] = 1.0 / (d.dx[a] * d.dx[a]);
  }
  for (int f = 0; f < 6; ++f) {
    d.bc[f] = (f / 2) < g.ndim ? g.bc[f] : FLD_BC_PERIODIC;
    d.bc_val[f] = (f / 2) < g.ndim ? g.bc_val[f] : 0.0;
  }
  d.ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  return d;
}

Opacity opacity_of(const fld_params& p) { return make_opacity(p); }

long long cells_of(const std::array<int, 3>& n) { return (long long)n[0] * n[1] * n[2]; }

long long faces_of(const std::array<int, 3>& n, int a) {
  long long c = 1;
  for (int b = 0; b < 3; ++b) c *= (b == a) ? n[b] + 1 : n[b];
  return c;
}

unsigned blocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ----------------------------------------------------------------------------- implementation

struct BatchedSolver::Impl {
  // shape signature
  int ng = 0;
  int precision = -1;
  std::vector<int> sig;
  // per grid
  std::vector<std::vector<std::array<int, 3>>> dims;  // [grid][level]
  std::vector<GridDev> gd;
  DeviceArena arena;
  std::vector<BFine> fine_h;
  BFine* fine_d = nullptr;
  void* lev_d = nullptr;  // BLev<T>[ng * kMaxLev]
  BState* st_d = nullptr;
  std::vector<BState> st_h;
  BState* st_pinned = nullptr;
  BFine* fine_pinned = nullptr;
  int* ctl_d = nullptr;
  double* parts_d = nullptr;
  size_t parts_cap = 0;
  // tile lists
  int tile = 0;
  Tile* tiles_d = nullptr;
  size_t tiles_cap = 0;
  struct Range {
    int off = 0, n = 0;
  };
  Range fine_r;
  std::vector<Range> cell_r, smooth_r, restrict_r, prolong_r;  // per level (smooth_r: 3-D grids)
  Tile2* tiles2_d = nullptr;  // tiles of the fused sweeps of 2-D grids
  size_t tiles2_cap = 0;
  std::vector<Range> sweep_r;  // per level, into tiles2_d
  Range coarse_r;
  int maxlev = 0;
  bool pcg_any = false;  // some grid of the batch runs the conjugate-gradient outer loop
  // graph
  cudaGraphExec_t exec = nullptr;
  // kernels of one graph replay: those outside the WHILE node, and those of one pass of its body
  unsigned long long k_outer = 0, k_body = 0;
  // after a replay has finished: count its kernels (the body ran once per pass, ctl_d[1] passes)
  void count_replay() {
    int passes = 0;
    if (cudaMemcpy(&passes, ctl_d + 1, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
      note_launch(k_outer + k_body * (unsigned long long)(passes > 0 ? passes : 0));
  }
  cudaStream_t cap = nullptr, body = nullptr;
  int nu1 = 2, nu2 = 2;
  // autotune rounds done for this shape and each candidate's summed step time
  static constexpr int kCands = 9, kTuneRounds = 3;
  int tune_rounds = 0;
  float tune_sum[kCands] = {};
  // autotune scratch
  double* scratch = nullptr;
  size_t scratch_cells = 0;

  ~Impl() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (body) cudaStreamDestroy(body);
    cudaFree(fine_d);
    cudaFree(lev_d);
    cudaFree(st_d);
    cudaFree(ctl_d);
    cudaFree(parts_d);
    cudaFree(tiles_d);
    cudaFree(tiles2_d);
    cudaFree(scratch);
    if (st_pinned) cudaFreeHost(st_pinned);
    if (fine_pinned) cudaFreeHost(fine_pinned);
  }

  cudaError_t configure(int n, const fld_grid* grids, const fld_params* params);
  template <class T>
  cudaError_t build_levels();
  cudaError_t build_tiles(int tile_cells);
  template <class T>
  cudaError_t build_graph(int nu1_, int nu2_);
  cudaError_t build_graph_any(int nu1_, int nu2_) {
    return precision == FLD_PREC_MIXED ? build_graph<float>(nu1_, nu2_) : build_graph<double>(nu1_, nu2_);
  }
  cudaError_t upload(const fld_params* params, const double* dt, const double* const* rho, double* const* eps,
                     double* const* E, cudaStream_t s);
};

BatchedSolver::~BatchedSolver() { delete impl_; }

cudaError_t BatchedSolver::Impl::configure(int n, const fld_grid* grids, const fld_params* params) {
  std::vector<int> s;
  s.push_back(n);
  s.push_back(params[0].precision);
  for (int i = 0; i < n; ++i) {
    s.push_back(grids[i].ndim);
    for (int a = 0; a < 3; ++a) s.push_back(grids[i].n[a]);
    for (int f = 0; f < 6; ++f) s.push_back(grids[i].bc[f]);
  }
  if (s == sig && exec) return cudaSuccess;
  // new shape: rebuild everything
  if (exec) {
    cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  sig = s;
  ng = n;
  precision = params[0].precision;
  tune_rounds = 0;
  for (float& t : tune_sum) t = 0.0f;
  dims.assign(n, {});
  gd.resize(n);
  maxlev = 0;
  for (int i = 0; i < n; ++i) {
    gd[i] = grid_dev(grids[i]);
    std::array<int, 3> d = {grids[i].n[0], grids[i].n[1], grids[i].n[2]};
    dims[i].push_back(d);
    for (;;) {
      bool ok = cells_of(d) > 64 && (int)dims[i].size() < kMaxLev;
      for (int a = 0; a < grids[i].ndim && ok; ++a) ok = (d[a] % 2 == 0) && d[a] >= 4;
      if (!ok) break;
      for (int a = 0; a < grids[i].ndim; ++a) d[a] /= 2;
      dims[i].push_back(d);
    }
    maxlev = std::max(maxlev, (int)dims[i].size());
  }
  cudaError_t e = precision == FLD_PREC_MIXED ? build_levels<float>() : build_levels<double>();
  if (e != cudaSuccess) return e;
  if (!cap) {
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t BatchedSolver::Impl::build_levels() {
  const size_t es = sizeof(T);
  size_t bytes = 0;
  auto add = [&](size_t b) { bytes += (b + 511) & ~(size_t)255; };
  for (int i = 0; i < ng; ++i) {
    long long N = cells_of(dims[i][0]);
    for (int a = 0; a < gd[i].ndim; ++a) add(faces_of(dims[i][0], a) * 8);
    for (int k = 0; k < 5; ++k) add(N * 8);  // b, diag, D, kappa, p
    for (size_t l = 0; l < dims[i].size(); ++l) {
      long long n = cells_of(dims[i][l]);
      if (l > 0 || es == 4)
        for (int a = 0; a < gd[i].ndim; ++a) add(faces_of(dims[i][l], a) * es);
      for (int k = 0; k < 4; ++k) add(n * es);
    }
  }
  cudaError_t e = arena.reserve(bytes + 4096);
  if (e != cudaSuccess) return e;
  fine_h.assign(ng, BFine{});
  std::vector<BLev<T>> lev_h((size_t)ng * kMaxLev);
  memset(lev_h.data(), 0, lev_h.size() * sizeof(BLev<T>));
  for (int i = 0; i < ng; ++i) {
    BFine& f = fine_h[i];
    long long N = cells_of(dims[i][0]);
    f.g = gd[i];
    f.nlev = (int)dims[i].size();
    for (int a = 0; a < 3; ++a) f.w64[a] = a < gd[i].ndim ? (double*)arena.take(faces_of(dims[i][0], a) * 8) : nullptr;
    f.b = (double*)arena.take(N * 8);
    f.diag = (double*)arena.take(N * 8);
    f.D = (double*)arena.take(N * 8);
    f.kappa = (double*)arena.take(N * 8);
    f.p = (double*)arena.take(N * 8);
    if (!f.b || !f.diag || !f.D || !f.kappa || !f.p) return cudaErrorMemoryAllocation;
    for (size_t l = 0; l < dims[i].size(); ++l) {
      BLev<T>& B = lev_h[(size_t)i * kMaxLev + l];
      long long n = cells_of(dims[i][l]);
      for (int a = 0; a < 3; ++a) B.L.n[a] = dims[i][l][a];
      B.L.ndim = gd[i].ndim;
      for (int k = 0; k < 6; ++k) B.L.bc[k] = gd[i].bc[k];
      for (int a = 0; a < 3; ++a) {
        if (a >= gd[i].ndim) B.L.w[a] = nullptr;
        else if (l == 0 && es == 8) B.L.w[a] = (const T*)f.w64[a];
        else B.L.w[a] = (const T*)arena.take(faces_of(dims[i][l], a) * es);
        if (a < gd[i].ndim && !B.L.w[a]) return cudaErrorMemoryAllocation;
      }
      B.invd = (T*)arena.take(n * es);
      B.x = (T*)arena.take(n * es);
      B.r = (T*)arena.take(n * es);
      B.tmp = (T*)arena.take(n * es);
      B.ncell = n;
      B.f0 = make_fastdiv((unsigned)dims[i][l][0]);
      B.f1 = make_fastdiv((unsigned)dims[i][l][1]);
      B.fh = make_fastdiv((unsigned)((dims[i][l][0] + 1) / 2));
      if (!B.invd || !B.x || !B.r || !B.tmp) return cudaErrorMemoryAllocation;
    }
  }
  cudaFree(fine_d);
  cudaFree(lev_d);
  cudaFree(st_d);
  cudaFree(ctl_d);
  fine_d = nullptr;
  lev_d = nullptr;
  st_d = nullptr;
  ctl_d = nullptr;
  if ((e = cudaMalloc(&fine_d, ng * sizeof(BFine))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&lev_d, lev_h.size() * sizeof(BLev<T>))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&st_d, ng * sizeof(BState))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ctl_d, 4 * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(lev_d, lev_h.data(), lev_h.size() * sizeof(BLev<T>), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if (st_pinned) cudaFreeHost(st_pinned);
  if (fine_pinned) cudaFreeHost(fine_pinned);
  st_pinned = nullptr;
  fine_pinned = nullptr;
  if ((e = cudaMallocHost(&st_pinned, ng * sizeof(BState))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&fine_pinned, ng * sizeof(BFine))) != cudaSuccess) return e;
  st_h.assign(ng, BState{});
  return cudaSuccess;
}

cudaError_t BatchedSolver::Impl::build_tiles(int tile_cells) {
  tile = tile_cells;
  std::vector<Tile> t;
  auto add_range = [&](int g, int l, long long count) {
    for (long long s0 = 0; s0 < count; s0 += tile_cells) t.push_back({g, l, s0, std::min<long long>(tile_cells, count - s0)});
  };
  // fine cells, grouped by grid (contiguous per grid for the segmented reductions)
  fine_r.off = 0;
  // conjugate gradients on the grids whose operator is symmetric (no linear-extrapolation face);
  // FLD_BATCHED_PCG=0 keeps the plain defect correction everywhere
  static const bool pcg_env = [] {
    const char* v = getenv("FLD_BATCHED_PCG");
    return !(v && v[0] == '0');
  }();
  pcg_any = false;
  for (int g = 0; g < ng; ++g) {
    st_h[g].tile_begin = (int)t.size();
    add_range(g, 0, cells_of(dims[g][0]));
    st_h[g].tile_end = (int)t.size();
    bool sym = pcg_env;
    for (int f = 0; f < 2 * gd[g].ndim; ++f) sym = sym && gd[g].bc[f] != FLD_BC_CONTINUOUS;
    st_h[g].pcg = sym ? 1 : 0;
    pcg_any = pcg_any || sym;
  }
  fine_r.n = (int)t.size();
  cell_r.assign(maxlev, {});
  smooth_r.assign(maxlev, {});
  restrict_r.assign(maxlev, {});
  prolong_r.assign(maxlev, {});
  for (int l = 1; l < maxlev; ++l) {
    cell_r[l].off = (int)t.size();
    for (int g = 0; g < ng; ++g)
      if (l < (int)dims[g].size()) add_range(g, l, cells_of(dims[g][l]));
    cell_r[l].n = (int)t.size() - cell_r[l].off;
  }
  std::vector<Tile2> t2;
  sweep_r.assign(maxlev, {});
  for (int l = 0; l < maxlev; ++l) {
    smooth_r[l].off = (int)t.size();
    sweep_r[l].off = (int)t2.size();
    for (int g = 0; g < ng; ++g)
      if (l < (int)dims[g].size() - 1) {
        const auto& n = dims[g][l];
        if (gd[g].ndim == 2) {
          for (int j0 = 0; j0 < n[1]; j0 += kSwY)
            for (int i0 = 0; i0 < n[0]; i0 += kSwX) t2.push_back({g, l, i0, j0});
        } else {
          add_range(g, l, (long long)((n[0] + 1) / 2) * n[1] * n[2]);
        }
      }
    smooth_r[l].n = (int)t.size() - smooth_r[l].off;
    sweep_r[l].n = (int)t2.size() - sweep_r[l].off;
    restrict_r[l].off = (int)t.size();  // 2-D grids restrict inside their last pre-sweep
    for (int g = 0; g < ng; ++g)
      if (l < (int)dims[g].size() - 1 && gd[g].ndim != 2) add_range(g, l, cells_of(dims[g][l + 1]));
    restrict_r[l].n = (int)t.size() - restrict_r[l].off;
    prolong_r[l].off = (int)t.size();
    for (int g = 0; g < ng; ++g)
      if (l < (int)dims[g].size() - 1) add_range(g, l, cells_of(dims[g][l]));
    prolong_r[l].n = (int)t.size() - prolong_r[l].off;
  }
  coarse_r.off = (int)t.size();
  for (int g = 0; g < ng; ++g) t.push_back({g, (int)dims[g].size() - 1, 0, cells_of(dims[g].back())});
  coarse_r.n = (int)t.size() - coarse_r.off;
  cudaError_t e;
  if (t.size() > tiles_cap) {
    cudaFree(tiles_d);
    tiles_d = nullptr;
    if ((e = cudaMalloc(&tiles_d, t.size() * sizeof(Tile))) != cudaSuccess) return e;
    tiles_cap = t.size();
  }
  if ((e = cudaMemcpy(tiles_d, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if (t2.size() > tiles2_cap) {
    cudaFree(tiles2_d);
    tiles2_d = nullptr;
    if ((e = cudaMalloc(&tiles2_d, t2.size() * sizeof(Tile2))) != cudaSuccess) return e;
    tiles2_cap = t2.size();
  }
  if (!t2.empty() &&
      (e = cudaMemcpy(tiles2_d, t2.data(), t2.size() * sizeof(Tile2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if (2 * (size_t)fine_r.n > parts_cap) {  // sums of r^2, then of the squared error bounds
    cudaFree(parts_d);
    parts_d = nullptr;
    if ((e = cudaMalloc(&parts_d, 2 * (size_t)fine_r.n * sizeof(double))) != cudaSuccess) return e;
    parts_cap = 2 * (size_t)fine_r.n;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t BatchedSolver::Impl::build_graph(int nu1_, int nu2_) {
  if (exec) {
    cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  const BLev<T>* lev = (const BLev<T>*)lev_d;
  const Tile* tl = tiles_d;
  const int B = kBlock;
  int iter_cap = 0;
  for (int g = 0; g < ng; ++g) iter_cap = std::max(iter_cap, st_h[g].max_cycles);
  iter_cap += 1;

  // the fused sweeps stage more than the default 48 KB of shared memory per block
  cudaError_t e = cudaSuccess;
  auto allow = [&](const void* k, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  allow((const void*)kb_sweep2d<T, true, false, false>, sw_smem_bytes<T, true, false, false>());
  allow((const void*)kb_sweep2d<T, false, false, false>, sw_smem_bytes<T, false, false, false>());
  allow((const void*)kb_sweep2d<T, false, true, false>, sw_smem_bytes<T, false, true, false>());
  allow((const void*)kb_sweep2d<T, true, false, true>, sw_smem_bytes<T, true, false, true>());
  allow((const void*)kb_sweep2d<T, false, false, true>, sw_smem_bytes<T, false, false, true>());
  if (e != cudaSuccess) return e;
  cudaGraph_t graph;
  e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return e;
  }
  cudaStream_t s = cap;
  const unsigned long long c0 = launch_count();
  note_launch(), kb_reset<<<blocks(ng, 256), 256, 0, s>>>(ng, st_d, ctl_d);
  note_launch(), kb_exchange<<<fine_r.n, B, 0, s>>>(tl + fine_r.off, fine_d, st_d, 0);
  note_launch(), kb_coeffs<<<fine_r.n, B, 0, s>>>(tl + fine_r.off, fine_d, st_d);
  note_launch(), kb_faces<T><<<fine_r.n, B, 0, s>>>(tl + fine_r.off, fine_d, lev);
  note_launch(), kb_fine_setup<T><<<fine_r.n, B, 0, s>>>(tl + fine_r.off, fine_d, lev);
  for (int l = 1; l < maxlev; ++l) {
    if (!cell_r[l].n) continue;
    note_launch(), kb_coarse_faces<T><<<cell_r[l].n, B, 0, s>>>(tl + cell_r[l].off, lev);
    note_launch(), kb_invd<T><<<cell_r[l].n, B, 0, s>>>(tl + cell_r[l].off, lev);
  }
  note_launch(), kb_sumsq_b<<<fine_r.n, B, 0, s>>>(tl + fine_r.off, fine_d, parts_d);
  note_launch(), kb_bnorm<<<blocks(ng, 256), 256, 0, s>>>(ng, parts_d, st_d);

  const unsigned long long c1 = launch_count();
  // the WHILE node over the cycles
  cudaGraphConditionalHandle handle;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaGraph_t capg = nullptr;
  e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, &deps, &edata, &ndeps);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNode_t wnode = nullptr;
  cudaGraph_t bodyg = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, graph, deps, edata, ndeps, &np);
    if (e == cudaSuccess) bodyg = np.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(body, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaStream_t b = body;
    note_launch(), kb_residual<T><<<fine_r.n, B, 0, b>>>(tl + fine_r.off, fine_d, lev, st_d, parts_d);
    note_launch(), kb_check<<<1, kCheckThreads, 0, b>>>(ng, parts_d, st_d, ctl_d, iter_cap,
                                                       sizeof(T) == sizeof(float) ? 1 : 0, fine_r.n, handle);
    // V-cycle.  3-D grids smooth with one launch per colour on x; 2-D grids with one fused launch
    // per sweep, alternating x and tmp: pre_tmp[l] / post_tmp[l] record that their level-l iterate
    // is in tmp after the pre- / post-smoothing (the first sweep, from zero, writes x).
    std::vector<int> pre_tmp(maxlev, 0), post_tmp(maxlev, 0);
    const Tile2* t2 = tiles2_d;
    for (int l = 0; l + 1 < maxlev; ++l) {
      const Range& sr = smooth_r[l];
      const Range& wr = sweep_r[l];
      if (!sr.n && !wr.n) continue;
      int in_tmp = 0;
      for (int it = 0; it < nu1_; ++it) {
        if (sr.n) {
          if (it == 0) note_launch(), kb_smooth<T, true, false><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 0);
          else note_launch(), kb_smooth<T, false, false><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 0);
          note_launch(), kb_smooth<T, false, false><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 1);
        }
        if (wr.n) {
          // the last pre-sweep also restricts the residual to level l + 1
          const bool last = it == nu1_ - 1;
          const Tile2* tw = t2 + wr.off;
          if (it == 0 && last) {
            note_launch(), kb_sweep2d<T, true, false, true>
                               <<<wr.n, B, sw_smem_bytes<T, true, false, true>(), b>>>(tw, lev, st_d, fine_d, 0, 0);
          } else if (it == 0) {
            note_launch(), kb_sweep2d<T, true, false, false>
                               <<<wr.n, B, sw_smem_bytes<T, true, false, false>(), b>>>(tw, lev, st_d, fine_d, 0, 0);
          } else if (last) {
            note_launch(), kb_sweep2d<T, false, false, true><<<wr.n, B, sw_smem_bytes<T, false, false, true>(), b>>>(
                               tw, lev, st_d, fine_d, 0, in_tmp);
            in_tmp ^= 1;
          } else {
            note_launch(), kb_sweep2d<T, false, false, false><<<wr.n, B, sw_smem_bytes<T, false, false, false>(), b>>>(
                               tw, lev, st_d, fine_d, 0, in_tmp);
            in_tmp ^= 1;
          }
        }
      }
      pre_tmp[l] = in_tmp;
      if (restrict_r[l].n)  // 3-D grids
        note_launch(), kb_restrict<T><<<restrict_r[l].n, B, 0, b>>>(tl + restrict_r[l].off, lev, st_d, pre_tmp[l]);
    }
    note_launch(), kb_coarse<T><<<coarse_r.n, kCoarseThreads, 0, b>>>(tl + coarse_r.off, lev, st_d, fine_d);
    // levels up
    for (int l = maxlev - 2; l >= 0; --l) {
      const Range& sr = smooth_r[l];
      const Range& wr = sweep_r[l];
      if (!sr.n && !wr.n) continue;
      note_launch(), kb_prolong<T><<<prolong_r[l].n, B, 0, b>>>(tl + prolong_r[l].off, lev, st_d, fine_d, pre_tmp[l],
                                                               post_tmp[l + 1]);
      int in_tmp = pre_tmp[l];
      for (int it = 0; it < nu2_; ++it) {
        bool last = (l == 0) && it == nu2_ - 1;
        if (sr.n) {
          if (last) {
            note_launch(), kb_smooth<T, false, true><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 1);
            note_launch(), kb_smooth<T, false, true><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 0);
          } else {
            note_launch(), kb_smooth<T, false, false><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 1);
            note_launch(), kb_smooth<T, false, false><<<sr.n, B, 0, b>>>(tl + sr.off, lev, st_d, fine_d, 0);
          }
        }
        if (wr.n) {
          const Tile2* tw = t2 + wr.off;
          if (last)
            note_launch(), kb_sweep2d<T, false, true, false><<<wr.n, B, sw_smem_bytes<T, false, true, false>(), b>>>(
                               tw, lev, st_d, fine_d, 1, in_tmp);
          else
            note_launch(), kb_sweep2d<T, false, false, false><<<wr.n, B, sw_smem_bytes<T, false, false, false>(), b>>>(
                               tw, lev, st_d, fine_d, 1, in_tmp);
          in_tmp ^= 1;
        }
      }
      post_tmp[l] = in_tmp;
    }
    if (pcg_any) {  // the conjugate-gradient update of the grids that use it (kb_pcg_*)
      const int z2d = post_tmp[0];
      const Tile* tf = tl + fine_r.off;
      note_launch(), kb_pcg_rz<T><<<fine_r.n, B, 0, b>>>(tf, fine_d, lev, st_d, parts_d, z2d);
      note_launch(), kb_pcg_beta<<<1, kCheckThreads, 0, b>>>(ng, parts_d, st_d);
      note_launch(), kb_pcg_dir<T><<<fine_r.n, B, 0, b>>>(tf, fine_d, lev, st_d, z2d);
      note_launch(), kb_pcg_ap<T><<<fine_r.n, B, 0, b>>>(tf, fine_d, lev, st_d, parts_d);
      note_launch(), kb_pcg_alpha<<<1, kCheckThreads, 0, b>>>(ng, parts_d, st_d);
      note_launch(), kb_pcg_x<<<fine_r.n, B, 0, b>>>(tf, fine_d, st_d);
    }
    cudaGraph_t tmp = nullptr;
    e = cudaStreamEndCapture(b, &tmp);
  }
  const unsigned long long c2 = launch_count();
  if (e == cudaSuccess) {
    note_launch(), kb_exchange<<<fine_r.n, B, 0, s>>>(tl + fine_r.off, fine_d, st_d, 1);
  }
  // captured, not run: the replays count them (count_replay)
  const unsigned long long c3 = launch_count();
  k_outer = (c1 - c0) + (c3 - c2);
  k_body = c2 - c1;
  unnote_launches(c3 - c0);
  cudaGraph_t done = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &done);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) {
    nu1 = nu1_;
    nu2 = nu2_;
  }
  return e;
}

cudaError_t BatchedSolver::Impl::upload(const fld_params* params, const double* dt, const double* const* rho,
                                        double* const* eps, double* const* E, cudaStream_t s) {
  for (int g = 0; g < ng; ++g) {
    BFine& f = fine_h[g];
    const fld_params& p = params[g];
    f.ph.op = opacity_of(p);
    f.ph.c = p.c;
    f.ph.gamma = p.gamma;
    f.ph.gas_R = p.gas_R;
    f.ph.limiter = p.limiter;
    f.cdf = make_coeff_df(f.ph, f.g);
    const bool plain64 = params[0].precision == FLD_PREC_FP64;  // the batch shares one precision
    if (plain64) f.cdf.ok = 0;  // FP64 coefficients in every cell
    f.xp = make_exchange(p.c, p.a_rad, p.gamma, p.gas_R, dt[g], p.exch_maxit > 0 ? p.exch_maxit : 100, plain64);
    f.dt = dt[g];
    f.order = p.order;
    f.rho = rho[g];
    f.eps = eps[g];
    f.E = E[g];
    st_h[g].rtol = p.rtol;
    st_h[g].max_cycles = p.max_cycles > 0 ? p.max_cycles : 100;
  }
  memcpy(fine_pinned, fine_h.data(), ng * sizeof(BFine));
  memcpy(st_pinned, st_h.data(), ng * sizeof(BState));
  cudaError_t e = cudaMemcpyAsync(fine_d, fine_pinned, ng * sizeof(BFine), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st_d, st_pinned, ng * sizeof(BState), cudaMemcpyHostToDevice, s);
  return e;
}

fld_status BatchedSolver::run(int ngrids, const fld_grid* grids, const fld_params* params, const double* dt,
                              const double* const* rho, double* const* eps, double* const* E, fld_info* infos,
                              cudaStream_t s, std::string* err) {
  char buf[256];
  auto cuda_err = [&](cudaError_t e, const char* where) {
    snprintf(buf, sizeof(buf), "batched %s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
    *err = buf;
    return FLD_ERR_CUDA;
  };
  for (int i = 1; i < ngrids; ++i)
    if (params[i].precision != params[0].precision) {
      *err = "all grids of a batch must use the same precision";
      return FLD_ERR_UNSUPPORTED;
    }
  if (!impl_) impl_ = new Impl();
  Impl& I = *impl_;
  bool fresh = !I.exec;
  cudaError_t e = I.configure(ngrids, grids, params);
  if (e != cudaSuccess) return cuda_err(e, "configure");
  if (!I.exec) fresh = true;
  // dx / bc values of the fine grids may differ from the previous call
  for (int g = 0; g < ngrids; ++g) {
    GridDev d = grid_dev(grids[g]);
    I.fine_h[g].g = d;
  }
  if (fresh || I.tune_rounds < Impl::kTuneRounds) {
    // autotune (nu1, nu2, tile) on scratch copies of the state, then keep the candidate with the
    // least time summed over the rounds so far
    size_t cells = 0;
    for (int g = 0; g < ngrids; ++g) cells += (size_t)I.gd[g].ncell;
    if (cells > I.scratch_cells) {
      cudaFree(I.scratch);
      I.scratch = nullptr;
      if ((e = cudaMalloc(&I.scratch, 2 * cells * sizeof(double))) != cudaSuccess) return cuda_err(e, "scratch");
      I.scratch_cells = cells;
    }
    std::vector<double*> se(ngrids), sE(ngrids);
    size_t off = 0;
    for (int g = 0; g < ngrids; ++g) {
      se[g] = I.scratch + off;
      sE[g] = I.scratch + cells + off;
      off += I.gd[g].ncell;
    }
    struct Cand {
      int nu1, nu2, tile;
    };
    const Cand cands[Impl::kCands] = {{2, 2, 2048}, {1, 1, 2048}, {3, 3, 2048}, {4, 4, 2048}, {4, 2, 2048},
                                      {2, 2, 8192}, {3, 3, 8192}, {4, 4, 8192}, {1, 1, 8192}};
    float ms_k[Impl::kCands] = {};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < Impl::kCands; ++k) {
      const Cand& c = cands[k];
      if ((e = I.build_tiles(c.tile)) != cudaSuccess) break;
      if ((e = I.upload(params, dt, rho, se.data(), sE.data(), s)) != cudaSuccess) break;
      if ((e = I.build_graph_any(c.nu1, c.nu2)) != cudaSuccess) break;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        for (int g = 0; g < ngrids; ++g) {
          cudaMemcpyAsync(se[g], eps[g], I.gd[g].ncell * sizeof(double), cudaMemcpyDeviceToDevice, s);
          cudaMemcpyAsync(sE[g], E[g], I.gd[g].ncell * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
        cudaEventRecord(e0, s);
        e = cudaGraphLaunch(I.exec, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        I.count_replay();
        cudaEventElapsedTime(&ms, e0, e1);
      }
      if (e != cudaSuccess) break;
      ms_k[k] = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_err(e, "autotune");
    int best = 0;
    for (int k = 0; k < Impl::kCands; ++k) {
      I.tune_sum[k] += ms_k[k];
      if (I.tune_sum[k] < I.tune_sum[best]) best = k;
    }
    I.tune_rounds += 1;
    const Cand pick = cands[best];
    if ((e = I.build_tiles(pick.tile)) != cudaSuccess) return cuda_err(e, "tiles");
    if ((e = I.upload(params, dt, rho, eps, E, s)) != cudaSuccess) return cuda_err(e, "upload");
    if ((e = I.build_graph_any(pick.nu1, pick.nu2)) != cudaSuccess) return cuda_err(e, "graph");
    nu1_ = pick.nu1;
    nu2_ = pick.nu2;
    tile_ = pick.tile;
  }
  {
    TraceScope ts("batched_step", s);
    if ((e = I.upload(params, dt, rho, eps, E, s)) != cudaSuccess) return cuda_err(e, "upload");
    if ((e = cudaGraphLaunch(I.exec, s)) != cudaSuccess) return cuda_err(e, "graph launch");
  }
  e = cudaMemcpyAsync(I.st_pinned, I.st_d, ngrids * sizeof(BState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "result read-back");
  I.count_replay();
  fld_status worst = FLD_OK;
  for (int g = 0; g < ngrids; ++g) {
    const BState& st = I.st_pinned[g];
    int status = st.status;
    if (st.bad & kStatNonpositive) status = FLD_ERR_NONPOSITIVE;
    if (infos) {
      memset(&infos[g], 0, sizeof(fld_info));
      infos[g].cycles = st.cycles;
      infos[g].rel_residual = st.rel;
      infos[g].exch_max_iters = st.xiters;
      infos[g].bisection_fallbacks = st.xbis;
      infos[g].status = status;
    }
    if (status != FLD_OK && worst == FLD_OK) {
      worst = (fld_status)status;
      snprintf(buf, sizeof(buf), "grid %d: status %d (relative residual %.3e after %d cycles)", g, status, st.rel,
               st.cycles);
      *err = buf;
    }
  }
  return worst;
}

}  // namespace fld

// Batched 1-D radial columns (arXiv 2104.03968: the Sect. 3.4 diffusion with the spherical
// geometry its Appendix A treats by source terms, written here directly as finite volumes).
//
// One thread block advances one column of n <= 2048 cells entirely on chip:
//   1. opacity kappa(rho, T) and D = c lambda(R)/(kappa rho) per cell (Sect. 2.2), the gradient
//      in R by the 3-point non-uniform central difference of the stretched grid;
//   2. rows of the backward-Euler finite-volume operator
//        x_i + (dt/V_i) [A_+ D_+ (x_i - x_{i+1})/h_+ + A_- D_- (x_i - x_{i-1})/h_-] = E_i,
//      D on faces by harmonic mean, A = r^2 and V = (r_+^3 - r_-^3)/3 (or 1 and the width);
//   3. a direct tridiagonal solve: every thread eliminates its chunk of rows down to two
//      interface rows, parallel cyclic reduction solves the 2P-row interface system in shared
//      memory, and the chunks back-substitute;
//   4. the point-implicit exchange (Sect. 3.3) per cell.
// HBM traffic is one read of rho, eps, E and one write of eps, E per cell.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "columns.h"
#include "dfmath.cuh"
#include "exchange.cuh"
#include "trace.h"

namespace fld {

enum { kColStep = 0, kColStepExchangeFirst = 1, kColDiffuse = 2, kColStepMidpoint = 3 };

// geometry factors shared by all columns: [gl n][gu n][cm n][cp n][hl hr flo fhi]
__global__ void k_col_geometry(int n, const double* __restrict__ rf, int geometry, double* __restrict__ geom,
                               unsigned* __restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto rc = [&](int k) -> double {
    if (k < 0) return 0.5 * (rf[0] + rf[1]) - (rf[1] - rf[0]);
    if (k >= n) return 0.5 * (rf[n - 1] + rf[n]) + (rf[n] - rf[n - 1]);
    return 0.5 * (rf[k] + rf[k + 1]);
  };
  double rl = rf[i], rr = rf[i + 1];
  if (!(rr > rl) || (geometry == FLD_GEOM_SPHERICAL && !(rl >= 0.0))) {
    if (status) atomicOr(status, kStatNonpositive);
  }
  double c0 = rc(i);
  double hm = c0 - rc(i - 1), hp = rc(i + 1) - c0;
  bool sph = geometry == FLD_GEOM_SPHERICAL;
  double V = sph ? (rr * rr * rr - rl * rl * rl) / 3.0 : rr - rl;
  double Al = sph ? rl * rl : 1.0, Ar = sph ? rr * rr : 1.0;
  geom[i] = Al / (V * hm);
  geom[n + i] = Ar / (V * hp);
  geom[2 * n + i] = hp / (hm * (hm + hp));
  geom[3 * n + i] = hm / (hp * (hm + hp));
  if (i == 0) {
    geom[4 * n + 0] = hm;
    geom[4 * n + 2] = hm / (rc(1) - rc(0));
  }
  if (i == n - 1) {
    geom[4 * n + 1] = hp;
    geom[4 * n + 3] = hp / (rc(n - 1) - rc(n - 2));
  }
}

struct ColArgs {
  int n;
  int bc_lo, bc_hi;
  const double* rf;  // r_faces (n + 1)
  // CAK line opacity (cak_v null: none)
  const double* cak_v;
  double cak_kQ, cak_rstar, cak_a_in, cak_a_out, cak_x_in, cak_x_out;
  const double* v_lo;
  const double* v_hi;
  const double* dt;
  const double* geom;
  const double* rho;
  const double* Din;
  const double* Ein;
  double* eps;
  double* Eout;
  double c, gamma, gas_R, sigma;
  int limiter, maxit;
  int plain64;  // the FP64 precision: the exchange in FP64 arithmetic throughout
  Opacity op;
  int* info_iters;
  int* info_bisect;
  unsigned* status;
};

__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

constexpr int kColMaxRows = 8;  // rows per thread: n <= 2048 with at most 256 threads per column

// FP32 solve of the tridiagonal system whose rows s0..s0+m-1 this thread holds in registers
// (sub A, diagonal B, super C, rhs Dv): the chunk is eliminated down to its two interface rows,
// parallel cyclic reduction solves the 2P interface rows in shared memory (fa..fd), and the
// chunk back-substitutes into X.  Every thread of the block must call it (it synchronises).
__device__ __forceinline__ void chunk_solve_f32(int t, int P, int m, const float (&Ain)[kColMaxRows],
                                                const float (&Bin)[kColMaxRows], const float (&Cin)[kColMaxRows],
                                                const float (&Din)[kColMaxRows], float* fa, float* fb, float* fc,
                                                float* fd, float (&X)[kColMaxRows]) {
  float a[kColMaxRows], b[kColMaxRows], c[kColMaxRows], d[kColMaxRows];
#pragma unroll
  for (int k = 0; k < kColMaxRows; ++k) {
    a[k] = Ain[k];
    b[k] = Bin[k];
    c[k] = Cin[k];
    d[k] = Din[k];
  }
  float Ra0 = 0.f, Rb0 = 1.f, Rc0 = 0.f, Rd0 = 0.f, Ra1 = 0.f, Rb1 = 1.f, Rc1 = 0.f, Rd1 = 0.f;
  if (m == 1) {
    Ra0 = a[0];
    Rb0 = b[0];
    Rc0 = c[0];
    Rd0 = d[0];
  } else if (m >= 2) {
#pragma unroll
    for (int k = 2; k < kColMaxRows; ++k)
      if (k < m) {
        float f = a[k] / b[k - 1];
        a[k] = -f * a[k - 1];
        b[k] -= f * c[k - 1];
        d[k] -= f * d[k - 1];
      }
#pragma unroll
    for (int k = 1; k < kColMaxRows; ++k)
      if (k == m - 1) {
        Ra1 = a[k];
        Rb1 = b[k];
        Rc1 = c[k];
        Rd1 = d[k];
      }
#pragma unroll
    for (int k = kColMaxRows - 2; k >= 1; --k)
      if (k <= m - 2) {
        float inv = 1.0f / b[k];
        if (k == m - 2) {
          a[k] *= inv;
          c[k] *= inv;
          d[k] *= inv;
        } else {
          float g = c[k];
          a[k] = (a[k] - g * a[k + 1]) * inv;
          d[k] = (d[k] - g * d[k + 1]) * inv;
          c[k] = -g * c[k + 1] * inv;
        }
      }
    Ra0 = a[0];
    if (m == 2) {
      Rb0 = b[0];
      Rc0 = c[0];
      Rd0 = d[0];
    } else {
      float g = c[0];
      Rb0 = b[0] - g * a[1];
      Rc0 = -g * c[1];
      Rd0 = d[0] - g * d[1];
    }
  }
  __syncthreads();  // the interface arrays may still be read by a previous solve
  fa[2 * t] = Ra0;
  fb[2 * t] = Rb0;
  fc[2 * t] = Rc0;
  fd[2 * t] = Rd0;
  fa[2 * t + 1] = Ra1;
  fb[2 * t + 1] = Rb1;
  fc[2 * t + 1] = Rc1;
  fd[2 * t + 1] = Rd1;
  __syncthreads();
  const int R = 2 * P;
  for (int st = 1; st < R; st <<= 1) {
    float na[2], nb[2], nc[2], nd[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int i = 2 * t + h;
      float am = 0.f, bm = 1.f, cm_ = 0.f, dm = 0.f, ap = 0.f, bp = 1.f, cp_ = 0.f, dp = 0.f;
      if (i - st >= 0) {
        am = fa[i - st];
        bm = fb[i - st];
        cm_ = fc[i - st];
        dm = fd[i - st];
      }
      if (i + st < R) {
        ap = fa[i + st];
        bp = fb[i + st];
        cp_ = fc[i + st];
        dp = fd[i + st];
      }
      float k1 = fa[i] / bm, k2 = fc[i] / bp;
      na[h] = -am * k1;
      nc[h] = -cp_ * k2;
      nb[h] = fb[i] - cm_ * k1 - ap * k2;
      nd[h] = fd[i] - dm * k1 - dp * k2;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int i = 2 * t + h;
      fa[i] = na[h];
      fb[i] = nb[h];
      fc[i] = nc[h];
      fd[i] = nd[h];
    }
    __syncthreads();
  }
  const float xs = fd[2 * t] / fb[2 * t];
  const float xe = fd[2 * t + 1] / fb[2 * t + 1];
#pragma unroll
  for (int k = 0; k < kColMaxRows; ++k) {
    float v = 0.f;
    if (k == 0) v = xs;
    else if (k == m - 1) v = xe;
    else if (k < m - 1) v = d[k] - a[k] * xs - c[k] * xe;
    X[k] = v;
  }
}

// kappa of a cell: the mixed precision takes the table's logarithms and power of ten in
// double-float (dfmath.cuh), the FP64 precision opacity() as it is
template <bool MIXED>
__device__ __forceinline__ double col_opacity(const Opacity& o, double rho, double T) {
  if (MIXED && o.model == FLD_OPACITY_TABLE) return opacity_table_df(o, rho, T);
  return opacity(o, rho, T);
}

template <int MODE, bool MIXED>
__global__ void k_columns(ColArgs A) {
  extern __shared__ double sm[];
  const int n = A.n, P = blockDim.x, t = threadIdx.x;
  const int M = (n + P - 1) / P;
  double* sx = sm;       // E^n, then E^{n+1}
  double* sr = sx + n;   // rho
  double* se = sr + n;   // eps
  double* sk = se + n;   // kappa
  double* sD = sk + n;   // cell D
  double* sa = sD + n;   // sub-diagonal, then elimination coefficients
  double* sb = sa + n;
  double* sc = sb + n;
  double* sd = sc + n;
  double* ra = sd + n;   // interface system, 2P rows
  double* rb = ra + 2 * P;
  double* rc = rb + 2 * P;
  double* rd = rc + 2 * P;
  double* sh = rd + 2 * P;  // midpoint IMEX: E after the half-step exchange
  double* sq = sh + (MODE == kColStepMidpoint ? n : 0);  // CAK line opacity per cell
  const bool cak = MODE != kColDiffuse && A.cak_v != nullptr;
  const long long base = (long long)blockIdx.x * n;
  const double dtc = A.dt[blockIdx.x];
  const double dtd = MODE == kColStepMidpoint ? 0.5 * dtc : dtc;  // the diffusion stage's step
  const double vlo = A.v_lo ? A.v_lo[blockIdx.x] : 0.0, vhi = A.v_hi ? A.v_hi[blockIdx.x] : 0.0;
  const double *gl = A.geom, *gu = A.geom + n, *cm = A.geom + 2 * n, *cp = A.geom + 3 * n;
  const double hl = A.geom[4 * n], hr = A.geom[4 * n + 1], flo = A.geom[4 * n + 2], fhi = A.geom[4 * n + 3];
  const ExchangeParams xp = make_exchange(A.c, 4.0 * A.sigma / A.c, A.gamma, A.gas_R, dtc, A.maxit, A.plain64 != 0);
  const ExchangeParams xp1 =
      MODE == kColStepMidpoint ? make_exchange(A.c, 4.0 * A.sigma / A.c, A.gamma, A.gas_R, 0.5 * dtc, A.maxit,
                                               A.plain64 != 0)
                               : xp;  // the first exchange stage
  int iters = 0, bis = 0;
  bool bad = false;

  for (int i = t; i < n; i += P) {
    sx[i] = A.Ein[base + i];
    if (MODE == kColDiffuse) {
      sD[i] = A.Din[base + i];
    } else {
      sr[i] = A.rho[base + i];
      se[i] = A.eps[base + i];
    }
  }
  __syncthreads();
  if (cak) {
    // Sect. 5.1, Eq. kap_cak: alpha(1 - R*/r), dv/dr central (one-sided at the ends)
    for (int i = t; i < n; i += P) {
      auto rc = [&](int k) { return 0.5 * (A.rf[k] + A.rf[k + 1]); };
      const double r = rc(i), x = 1.0 - A.cak_rstar / r;
      const double alpha = x <= A.cak_x_in    ? A.cak_a_in
                           : x >= A.cak_x_out ? A.cak_a_out
                                              : A.cak_a_in + (A.cak_a_out - A.cak_a_in) * (x - A.cak_x_in) /
                                                                 (A.cak_x_out - A.cak_x_in);
      const int lo = i > 0 ? i - 1 : 0, hi = i < n - 1 ? i + 1 : n - 1;
      const double dvdr = (A.cak_v[base + lo] - A.cak_v[base + hi]) / (rc(lo) - rc(hi));
      sq[i] = A.cak_kQ / (1.0 - alpha) * pow(fabs(dvdr) / (A.c * A.cak_kQ * sr[i]), alpha);
    }
    __syncthreads();
  }
  const int s0 = t * M, s1 = min(s0 + M, n);

  if (MODE == kColStepExchangeFirst || MODE == kColStepMidpoint) {
    for (int i = s0; i < s1; ++i) {
      double e = se[i], E = sx[i];
      double k = col_opacity<MIXED>(A.op, sr[i], temperature(A.gamma, A.gas_R, sr[i], e)) + (cak ? sq[i] : 0.0);
      if (exchange_cell_fast(xp1, sr[i], k, e, E, iters, bis)) {
        se[i] = e;
        sx[i] = E;
      } else {
        bad = true;
      }
      if (MODE == kColStepMidpoint) sh[i] = sx[i];
    }
    __syncthreads();
  }
  if (MODE != kColDiffuse) {
    for (int i = s0; i < s1; ++i) {
      double e = sx[i], rh = sr[i];
      double k = col_opacity<MIXED>(A.op, rh, temperature(A.gamma, A.gas_R, rh, se[i])) + (cak ? sq[i] : 0.0);
      sk[i] = k;
      if (!(e > 0.0) || !(rh > 0.0) || !(k > 0.0) || !(se[i] >= 0.0)) bad = true;
      double em, ep;
      if (i > 0) em = sx[i - 1];
      else if (A.bc_lo == FLD_BC_DIRICHLET) em = vlo;
      else if (A.bc_lo == FLD_BC_NEUMANN) em = e - vlo * hl;
      else em = e - (sx[1] - e) * flo;
      if (i < n - 1) ep = sx[i + 1];
      else if (A.bc_hi == FLD_BC_DIRICHLET) ep = vhi;
      else if (A.bc_hi == FLD_BC_NEUMANN) ep = e + vhi * hr;
      else ep = e + (e - sx[n - 2]) * fhi;
      double gm = fabs(cp[i] * (ep - e) + cm[i] * (e - em));
      const double D = limited_D(A.limiter, A.c, k * rh, e, gm * gm, gm);
      sD[i] = D;
    }
    __syncthreads();
  }

  // rows of the dt-scaled operator
  for (int i = s0; i < s1; ++i) {
    double Dl = i > 0 ? harm(sD[i - 1], sD[i]) : sD[0];
    double Du = i < n - 1 ? harm(sD[i], sD[i + 1]) : sD[n - 1];
    double wl = dtd * Dl * gl[i], wu = dtd * Du * gu[i];
    double a = 0.0, b = 1.0, c = 0.0, d = sx[i];
    if (i > 0) {
      a = -wl;
      b += wl;
    } else if (A.bc_lo == FLD_BC_DIRICHLET) {
      b += wl;
      d += wl * vlo;
    } else if (A.bc_lo == FLD_BC_NEUMANN) {
      d -= wl * vlo * hl;
    } else if (A.bc_lo == FLD_BC_LUMINOSITY) {
      // Sect. 5.2: ghost = E_0 + L hl / (4 pi r_0^2 D_0)
      const double r0 = 0.5 * (A.rf[0] + A.rf[1]);
      d += wl * vlo * hl / (4.0 * 3.14159265358979323846 * r0 * r0 * sD[0]);
    } else {
      b -= wl * flo;
      c += wl * flo;
    }
    if (i < n - 1) {
      c -= wu;
      b += wu;
    } else if (A.bc_hi == FLD_BC_DIRICHLET) {
      b += wu;
      d += wu * vhi;
    } else if (A.bc_hi == FLD_BC_NEUMANN) {
      d += wu * vhi * hr;
    } else {
      b -= wu * fhi;
      a += wu * fhi;
    }
    sa[i] = a;
    sb[i] = b;
    sc[i] = c;
    sd[i] = d;
  }

  const int m = s1 - s0;
  if constexpr (MIXED) {
    // FP32 solves inside FP64 iterative refinement: x = solve32(d); twice r = d - A x (FP64),
    // x += solve32(r).  The rows stay in FP64 in shared memory for the residual.
    float* fa = reinterpret_cast<float*>(ra);
    float* fb = fa + 2 * P;
    float* fc = fb + 2 * P;
    float* fd = fc + 2 * P;
    float A32[kColMaxRows], B32[kColMaxRows], C32[kColMaxRows], R32[kColMaxRows], X32[kColMaxRows];
#pragma unroll
    for (int k = 0; k < kColMaxRows; ++k) {
      bool in = k < m;
      A32[k] = in ? (float)sa[s0 + k] : 0.0f;
      B32[k] = in ? (float)sb[s0 + k] : 1.0f;
      C32[k] = in ? (float)sc[s0 + k] : 0.0f;
      R32[k] = in ? (float)sd[s0 + k] : 0.0f;
    }
    chunk_solve_f32(t, P, m, A32, B32, C32, R32, fa, fb, fc, fd, X32);
#pragma unroll
    for (int k = 0; k < kColMaxRows; ++k)
      if (k < m) sx[s0 + k] = (double)X32[k];
    for (int pass = 0; pass < 2; ++pass) {
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kColMaxRows; ++k) {
        R32[k] = 0.0f;
        if (k < m) {
          int i = s0 + k;
          double r = fma(-sb[i], sx[i], sd[i]);
          if (i > 0) r = fma(-sa[i], sx[i - 1], r);
          if (i < n - 1) r = fma(-sc[i], sx[i + 1], r);
          R32[k] = (float)r;
        }
      }
      chunk_solve_f32(t, P, m, A32, B32, C32, R32, fa, fb, fc, fd, X32);  // synchronises before any update
#pragma unroll
      for (int k = 0; k < kColMaxRows; ++k)
        if (k < m) sx[s0 + k] += (double)X32[k];
    }
  } else {
  // chunk elimination down to the interface rows (x_s, x_e) of this thread
  double Ra0 = 0.0, Rb0 = 1.0, Rc0 = 0.0, Rd0 = 0.0;  // row of x_s
  double Ra1 = 0.0, Rb1 = 1.0, Rc1 = 0.0, Rd1 = 0.0;  // row of x_e
  if (m == 1) {
    Ra0 = sa[s0];
    Rb0 = sb[s0];
    Rc0 = sc[s0];  // zero: the single-row chunk is the last row
    Rd0 = sd[s0];
  } else if (m >= 2) {
    const int s = s0, e = s1 - 1;
    // downward: alpha_i x_s + beta_i x_i + c_i x_{i+1} = delta_i  (i = s+1 .. e)
    for (int i = s + 2; i <= e; ++i) {
      double f = sa[i] / sb[i - 1];
      sa[i] = -f * sa[i - 1];
      sb[i] = sb[i] - f * sc[i - 1];
      sd[i] = sd[i] - f * sd[i - 1];
    }
    Ra1 = sa[e];
    Rb1 = sb[e];
    Rc1 = sc[e];
    Rd1 = sd[e];
    // upward: x_i = d'_i - a'_i x_s - c'_i x_e  (i = e-1 .. s+1)
    for (int i = e - 1; i > s; --i) {
      double inv = 1.0 / sb[i];
      if (i == e - 1) {
        sa[i] = sa[i] * inv;
        sc[i] = sc[i] * inv;
        sd[i] = sd[i] * inv;
      } else {
        double g = sc[i];
        sa[i] = (sa[i] - g * sa[i + 1]) * inv;
        sd[i] = (sd[i] - g * sd[i + 1]) * inv;
        sc[i] = -g * sc[i + 1] * inv;
      }
    }
    Ra0 = sa[s];
    if (m == 2) {
      Rb0 = sb[s];
      Rc0 = sc[s];
      Rd0 = sd[s];
    } else {
      double g = sc[s];
      Rb0 = sb[s] - g * sa[s + 1];
      Rc0 = -g * sc[s + 1];
      Rd0 = sd[s] - g * sd[s + 1];
    }
  }
  ra[2 * t] = Ra0;
  rb[2 * t] = Rb0;
  rc[2 * t] = Rc0;
  rd[2 * t] = Rd0;
  ra[2 * t + 1] = Ra1;
  rb[2 * t + 1] = Rb1;
  rc[2 * t + 1] = Rc1;
  rd[2 * t + 1] = Rd1;
  __syncthreads();

  // parallel cyclic reduction on the 2P interface rows
  const int R = 2 * P;
  for (int st = 1; st < R; st <<= 1) {
    double na[2], nb[2], nc[2], nd[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int i = 2 * t + h;
      double a = ra[i], b = rb[i], c = rc[i], d = rd[i];
      double am = 0, bm = 1, cm_ = 0, dm = 0, ap = 0, bp = 1, cp_ = 0, dp = 0;
      if (i - st >= 0) {
        am = ra[i - st];
        bm = rb[i - st];
        cm_ = rc[i - st];
        dm = rd[i - st];
      }
      if (i + st < R) {
        ap = ra[i + st];
        bp = rb[i + st];
        cp_ = rc[i + st];
        dp = rd[i + st];
      }
      double k1 = a / bm, k2 = c / bp;
      na[h] = -am * k1;
      nc[h] = -cp_ * k2;
      nb[h] = b - cm_ * k1 - ap * k2;
      nd[h] = d - dm * k1 - dp * k2;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int i = 2 * t + h;
      ra[i] = na[h];
      rb[i] = nb[h];
      rc[i] = nc[h];
      rd[i] = nd[h];
    }
    __syncthreads();
  }
  const double xs = rd[2 * t] / rb[2 * t];
  const double xe = rd[2 * t + 1] / rb[2 * t + 1];
  if (m >= 1) sx[s0] = xs;
  if (m >= 2) {
    sx[s1 - 1] = xe;
    for (int i = s0 + 1; i < s1 - 1; ++i) sx[i] = sd[i] - sa[i] * xs - sc[i] * xe;
  }
  }  // FP64 solve

  if (MODE == kColStep) {
    for (int i = s0; i < s1; ++i) {
      double e = se[i], E = sx[i];
      if (exchange_cell_fast(xp, sr[i], sk[i], e, E, iters, bis)) {
        se[i] = e;
        sx[i] = E;
      } else {
        bad = true;
      }
    }
  }
  if (MODE == kColStepMidpoint) {
    // Sect. 3.1: from u^n plus twice the half-step diffusion increment, the exchange over dt
    // (u^n is still in global memory: the column is written back at the end)
    for (int i = s0; i < s1; ++i) {
      double E = fma(2.0, sx[i] - sh[i], A.Ein[base + i]);
      double e = A.eps[base + i];
      double k = col_opacity<MIXED>(A.op, sr[i], temperature(A.gamma, A.gas_R, sr[i], e)) + (cak ? sq[i] : 0.0);
      if (exchange_cell_fast(xp, sr[i], k, e, E, iters, bis)) {
        se[i] = e;
        sx[i] = E;
      } else {
        bad = true;
        se[i] = e;
        sx[i] = E;
      }
    }
  }
  __syncthreads();
  for (int i = t; i < n; i += P) {
    A.Eout[base + i] = sx[i];
    if (MODE != kColDiffuse) A.eps[base + i] = se[i];
  }
  if (MODE != kColDiffuse) {
    if (bad) atomicOr(A.status, kStatNonpositive);
    exchange_report(iters, bis, A.info_iters, A.info_bisect);
  }
}

bool cak_valid(const fld_cak* c) {
  if (!c) return true;
  return c->v && c->kappa_e_Qbar > 0 && c->r_star > 0 && c->alpha_in >= 0 && c->alpha_in < 1 && c->alpha_out >= 0 &&
         c->alpha_out < 1 && c->x_in <= c->x_out;
}

fld_status columns_validate(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo, int bc_hi,
                            const double* v_lo, const double* v_hi, const double* dt, std::string* err) {
  char buf[256];
  auto bad = [&](const char* m) {
    *err = m;
    return FLD_ERR_INVALID_ARG;
  };
  if (ncol < 0) return bad("ncol must be >= 0");
  if (ncell < 2 || ncell > kColumnMaxCells) {
    snprintf(buf, sizeof(buf), "ncell must be in [2, %d] (got %d)", kColumnMaxCells, ncell);
    *err = buf;
    return ncell > kColumnMaxCells ? FLD_ERR_UNSUPPORTED : FLD_ERR_INVALID_ARG;
  }
  if (geometry != FLD_GEOM_CARTESIAN && geometry != FLD_GEOM_SPHERICAL) return bad("unknown geometry");
  for (int bc : {bc_lo, bc_hi})
    if (bc != FLD_BC_DIRICHLET && bc != FLD_BC_NEUMANN && bc != FLD_BC_CONTINUOUS && bc != FLD_BC_LUMINOSITY)
      return bad("column boundaries must be Dirichlet, Neumann, continuous or (inner) luminosity");
  if (bc_hi == FLD_BC_LUMINOSITY) return bad("the luminosity boundary is for the inner face only");
  if (ncol == 0) return FLD_OK;  // an empty batch reads no array
  if ((bc_lo != FLD_BC_CONTINUOUS && !v_lo) || (bc_hi != FLD_BC_CONTINUOUS && !v_hi))
    return bad("v_lo / v_hi are required for Dirichlet, Neumann and luminosity boundaries");
  if (!r_faces) return bad("r_faces is NULL");
  if (!dt) return bad("dt is NULL");
  return FLD_OK;
}

static int col_threads(int n) {
  int need = (n + 7) / 8;
  int P = 32;
  while (P < need && P < 256) P <<= 1;
  return P;
}

static size_t col_smem(int n, int P, int mode, bool cak) {
  return (size_t)((9 + (mode == kColStepMidpoint ? 1 : 0) + (cak ? 1 : 0)) * n + 8 * P) * sizeof(double);
}

template <int MODE, bool MIXED>
static cudaError_t launch_kernel(int ncol, int ncell, ColArgs& A, cudaStream_t s) {
  int P = col_threads(ncell);
  size_t smem = col_smem(ncell, P, MODE, MODE != kColDiffuse && A.cak_v != nullptr);
  cudaError_t e = cudaFuncSetAttribute(k_columns<MODE, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  note_launch(), k_columns<MODE, MIXED><<<ncol, P, smem, s>>>(A);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(int ncol, int ncell, const double* r_faces, int geometry, ColArgs& A, unsigned* status,
                               int precision, cudaStream_t s) {
  note_launch(),
      k_col_geometry<<<(ncell + 255) / 256, 256, 0, s>>>(ncell, r_faces, geometry, const_cast<double*>(A.geom), status);
  TraceScope ts(precision == FLD_PREC_MIXED ? "columns_mixed" : "columns", s);
  return precision == FLD_PREC_MIXED ? launch_kernel<MODE, true>(ncol, ncell, A, s)
                                     : launch_kernel<MODE, false>(ncol, ncell, A, s);
}

static ColArgs col_args(int ncell, const double* r_faces, int bc_lo, int bc_hi, const double* v_lo,
                        const double* v_hi, const fld_params& p, const double* dt, double* geom) {
  ColArgs A{};
  A.n = ncell;
  A.rf = r_faces;
  A.bc_lo = bc_lo;
  A.bc_hi = bc_hi;
  if (p.cak) {
    A.cak_v = p.cak->v;
    A.cak_kQ = p.cak->kappa_e_Qbar;
    A.cak_rstar = p.cak->r_star;
    A.cak_a_in = p.cak->alpha_in;
    A.cak_a_out = p.cak->alpha_out;
    A.cak_x_in = p.cak->x_in;
    A.cak_x_out = p.cak->x_out;
  }
  A.v_lo = v_lo;
  A.v_hi = v_hi;
  A.dt = dt;
  A.geom = geom;
  A.c = p.c;
  A.gamma = p.gamma;
  A.gas_R = p.gas_R;
  A.sigma = p.a_rad * p.c / 4.0;
  A.limiter = p.limiter;
  A.maxit = p.exch_maxit > 0 ? p.exch_maxit : 100;
  A.plain64 = p.precision == FLD_PREC_FP64 ? 1 : 0;
  A.op = make_opacity(p);
  return A;
}

cudaError_t launch_columns_step(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo, int bc_hi,
                                const double* v_lo, const double* v_hi, const fld_params& p, const double* dt,
                                const double* rho, double* eps, double* E, double* geom, int* info_iters,
                                int* info_bisect, unsigned* status, cudaStream_t s) {
  ColArgs A = col_args(ncell, r_faces, bc_lo, bc_hi, v_lo, v_hi, p, dt, geom);
  A.rho = rho;
  A.Ein = E;
  A.Eout = E;
  A.eps = eps;
  A.info_iters = info_iters;
  A.info_bisect = info_bisect;
  A.status = status;
  if (p.order == FLD_ORDER_EXCHANGE_THEN_DIFFUSE)
    return launch_mode<kColStepExchangeFirst>(ncol, ncell, r_faces, geometry, A, status, p.precision, s);
  if (p.order == FLD_ORDER_IMEX_MIDPOINT)
    return launch_mode<kColStepMidpoint>(ncol, ncell, r_faces, geometry, A, status, p.precision, s);
  return launch_mode<kColStep>(ncol, ncell, r_faces, geometry, A, status, p.precision, s);
}

cudaError_t launch_columns_diffuse(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo, int bc_hi,
                                   const double* v_lo, const double* v_hi, const fld_params& p, const double* dt,
                                   const double* D_cell, const double* E_old, double* E_new, double* geom,
                                   cudaStream_t s) {
  ColArgs A = col_args(ncell, r_faces, bc_lo, bc_hi, v_lo, v_hi, p, dt, geom);
  A.Din = D_cell;
  A.Ein = E_old;
  A.Eout = E_new;
  return launch_mode<kColDiffuse>(ncol, ncell, r_faces, geometry, A, nullptr, p.precision, s);
}

// ----------------------------------------------------------------------------- no-allocation entry

// Scratch of fld_columns_step_static, resident on every device that loads the library: the
// per-cell geometry factors of up to FLD_STATIC_MAX_CELLS cells (4 n + 4 doubles) followed by
// the status word and the two exchange counters (one double slot each).
constexpr int kStaticGeom = 4 * FLD_STATIC_MAX_CELLS + 4;
static __device__ __align__(256) double g_static_scratch[kStaticGeom + 4];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device (looked up once per device).  In
// host code the symbol name is only a host-side handle, so kernels must receive this address.
cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

bool static_params_ok(const fld_params* p) {
  if (!p || !(p->c > 0) || !(p->a_rad > 0) || !(p->gamma > 1) || !(p->gas_R > 0)) return false;
  if (p->limiter < FLD_LIMITER_LP || p->limiter > FLD_LIMITER_MINERBO) return false;
  if (p->opacity < FLD_OPACITY_CONST || p->opacity > FLD_OPACITY_TABLE) return false;
  if (p->opacity != FLD_OPACITY_TABLE && !(p->kappa0 > 0)) return false;
  if (p->opacity == FLD_OPACITY_TABLE &&
      (!p->table || p->tn[0] < 2 || p->tn[1] < 2 || !(p->thi[0] > p->tlo[0]) || !(p->thi[1] > p->tlo[1])))
    return false;
  if (p->exch_maxit < 0 || !cak_valid(p->cak)) return false;
  return p->order == FLD_ORDER_DIFFUSE_THEN_EXCHANGE || p->order == FLD_ORDER_EXCHANGE_THEN_DIFFUSE ||
         p->order == FLD_ORDER_IMEX_MIDPOINT;
}

}  // namespace

}  // namespace fld

extern "C" fld_status fld_columns_step_static(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo,
                                              int bc_hi, const double* v_lo, const double* v_hi, const fld_params* p,
                                              const double* dt, const double* rho, double* eps, double* E,
                                              fld_info* info, void* stream) {
  using namespace fld;
  if (ncell > FLD_STATIC_MAX_CELLS) return FLD_ERR_UNSUPPORTED;
  std::string err;
  fld_status st = columns_validate(ncol, ncell, r_faces, geometry, bc_lo, bc_hi, v_lo, v_hi, dt, &err);
  if (st != FLD_OK) return st;
  if (!static_params_ok(p) || (ncol > 0 && (!rho || !eps || !E))) return FLD_ERR_INVALID_ARG;
  if (info) memset(info, 0, sizeof(*info));
  if (ncol == 0) return FLD_OK;
  double* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return FLD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  double* geom = scratch;
  unsigned* status = reinterpret_cast<unsigned*>(scratch + kStaticGeom);
  int* iters = reinterpret_cast<int*>(scratch + kStaticGeom + 1);
  int* bisect = reinterpret_cast<int*>(scratch + kStaticGeom + 2);
  // the counters keep the previous call's values: clear them
  if (cudaMemsetAsync(scratch + kStaticGeom, 0, 3 * sizeof(double), s) != cudaSuccess) return FLD_ERR_CUDA;
  ColArgs A = col_args(ncell, r_faces, bc_lo, bc_hi, v_lo, v_hi, *p, dt, geom);
  A.rho = rho;
  A.Ein = E;
  A.Eout = E;
  A.eps = eps;
  A.info_iters = iters;
  A.info_bisect = bisect;
  A.status = status;
  note_launch(), k_col_geometry<<<(ncell + 255) / 256, 256, 0, s>>>(ncell, r_faces, geometry, geom, status);
  const bool mixed = p->precision == FLD_PREC_MIXED;
  cudaError_t e;
  if (p->order == FLD_ORDER_EXCHANGE_THEN_DIFFUSE)
    e = mixed ? launch_kernel<kColStepExchangeFirst, true>(ncol, ncell, A, s)
              : launch_kernel<kColStepExchangeFirst, false>(ncol, ncell, A, s);
  else if (p->order == FLD_ORDER_IMEX_MIDPOINT)
    e = mixed ? launch_kernel<kColStepMidpoint, true>(ncol, ncell, A, s)
              : launch_kernel<kColStepMidpoint, false>(ncol, ncell, A, s);
  else
    e = mixed ? launch_kernel<kColStep, true>(ncol, ncell, A, s) : launch_kernel<kColStep, false>(ncol, ncell, A, s);
  if (e != cudaSuccess) return FLD_ERR_CUDA;
  if (info) {
    unsigned sbits = 0;
    e = cudaMemcpyAsync(&sbits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&info->exch_max_iters, iters, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&info->bisection_fallbacks, bisect, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return FLD_ERR_CUDA;
    info->status = (sbits & kStatNonpositive) ? FLD_ERR_NONPOSITIVE : FLD_OK;
    if (info->status != FLD_OK) return FLD_ERR_NONPOSITIVE;
  }
  return FLD_OK;
}

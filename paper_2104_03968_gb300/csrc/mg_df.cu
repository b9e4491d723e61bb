// Double-float setup of the mixed solver's finest level: face weights, diagonal, right-hand side
// and the first outer residual, computed on the FP32 and integer pipes (see df.cuh) instead of in
// FP64.  The mixed solver only ever consumes these quantities as hi + lo float pairs (the FP32
// V-cycle takes the hi parts, the residual updates both), so no FP64 copy is made.
//
// The arithmetic is exponent-scaled where the physical values may leave the FP32 range (D in cgs
// units): each face's D values are scaled by the same power of two before the harmonic mean and
// the weight is scaled back.  A cell whose values leave the window where the double-float parts
// stay normal floats (|value| outside [2^-77, 2^90)) sets a flag; the solver then redoes the
// setup in FP64.
#include <algorithm>

#include "df.cuh"
#include "kernels.h"
#include "mg_df.h"
#include "mg_device.cuh"
#include "trace.h"

namespace fld {

namespace {

// x * 2^k exactly for a normal float, 0 where the result would not be a normal float
__device__ __forceinline__ float scale2(float x, int k) {
  const int bits = __float_as_int(x);
  const int e = (bits >> 23) & 0xff;
  if (e == 0 || e + k <= 0) return 0.0f;
  return __int_as_float(bits + (k << 23));
}

// |x| in [2^-77, 2^90): the low part and the error terms (2^-48 below) stay normal floats
__device__ __forceinline__ bool in_window(float x) {
  const int e = ((__float_as_int(x) >> 23) & 0xff) - 127;
  return x == 0.0f || (e > -78 && e < 90);
}

// s * 2 Dc Dn / (Dc + Dn) (pair) or s * Dc (boundary face) as a double-float.  c = Dc 2^-sh is
// the cell's own value, split once per cell; Dn is scaled by the same power of two.
__device__ __forceinline__ dfl face_weight_df(dfl c, int sh, double Dn, bool pair, dfl s, unsigned& bad) {
  dfl w;
  if (pair) {
    float nh, nl;
    bool ok;
    split_f64_scaled(Dn, sh, nh, nl, ok);
    if (!ok) bad = 1u;
    const dfl n{nh, nl};
    const dfl h = df_div(df_mul(c, n), df_add_pos(c, n));
    w = df_scale(df_mul(h, s), 2.0f);
  } else {
    w = df_mul(c, s);
  }
  const int e = ((__float_as_int(w.hi) >> 23) & 0xff) - 127 + sh;
  if (!(w.hi > 0.0f) || e <= -78 || e >= 90) bad = 1u;
  return {scale2(w.hi, sh), scale2(w.lo, sh)};
}

}  // namespace

// Whole x rows per block iteration, 32-bit indices (the caller guarantees < 2^31 cells and faces
// per axis).
__global__ void __launch_bounds__(256) k_faces_df(GridDev g, DfConst K, const double* __restrict__ D,
                                                  float* __restrict__ w0, float* __restrict__ w1,
                                                  float* __restrict__ w2, float* __restrict__ l0,
                                                  float* __restrict__ l1, float* __restrict__ l2,
                                                  unsigned* __restrict__ flag) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int rows = ny * nz;
  const bool per[3] = {g.bc[0] == FLD_BC_PERIODIC, g.bc[2] == FLD_BC_PERIODIC, g.bc[4] == FLD_BC_PERIODIC};
  const bool perh[3] = {g.bc[1] == FLD_BC_PERIODIC, g.bc[3] == FLD_BC_PERIODIC, g.bc[5] == FLD_BC_PERIODIC};
  unsigned bad = 0u;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const int idx = i + nx * row;
      const double Dc = D[idx];
      const int sh = exponent_f64(Dc);
      dfl c;
      {
        bool ok;
        split_f64_scaled(Dc, sh, c.hi, c.lo, ok);
        if (!ok) bad = 1u;
      }
      // x faces: lower face i of row (j, k), and face nx when this cell owns it
      {
        const dfl s{K.s_hi[0], K.s_lo[0]};
        const bool pair = i > 0 || per[0];
        const double Dn = pair ? D[i > 0 ? idx - 1 : idx + (nx - 1)] : Dc;
        const dfl w = face_weight_df(c, sh, Dn, pair, s, bad);
        const int f = i + (nx + 1) * row;
        w0[f] = w.hi;
        l0[f] = w.lo;
        if ((perh[0] && i == 0) || (!perh[0] && i == nx - 1)) {
          const dfl wu = perh[0] ? w : face_weight_df(c, sh, Dc, false, s, bad);
          w0[f - i + nx] = wu.hi;
          l0[f - i + nx] = wu.lo;
        }
      }
      if (g.ndim >= 2) {
        const dfl s{K.s_hi[1], K.s_lo[1]};
        const bool pair = j > 0 || per[1];
        const double Dn = pair ? D[j > 0 ? idx - nx : idx + (ny - 1) * nx] : Dc;
        const dfl w = face_weight_df(c, sh, Dn, pair, s, bad);
        const int f = i + nx * (j + (ny + 1) * k);
        w1[f] = w.hi;
        l1[f] = w.lo;
        if ((perh[1] && j == 0) || (!perh[1] && j == ny - 1)) {
          const dfl wu = perh[1] ? w : face_weight_df(c, sh, Dc, false, s, bad);
          const int fu = i + nx * (ny + (ny + 1) * k);
          w1[fu] = wu.hi;
          l1[fu] = wu.lo;
        }
      }
      if (g.ndim == 3) {
        const int sz = nx * ny;
        const dfl s{K.s_hi[2], K.s_lo[2]};
        const bool pair = k > 0 || per[2];
        const double Dn = pair ? D[k > 0 ? idx - sz : idx + (nz - 1) * sz] : Dc;
        const dfl w = face_weight_df(c, sh, Dn, pair, s, bad);
        w2[idx] = w.hi;
        l2[idx] = w.lo;
        if ((perh[2] && k == 0) || (!perh[2] && k == nz - 1)) {
          const dfl wu = perh[2] ? w : face_weight_df(c, sh, Dc, false, s, bad);
          const int fu = i + nx * (j + ny * nz);
          w2[fu] = wu.hi;
          l2[fu] = wu.lo;
        }
      }
    }
  }
  if (bad) atomicOr(flag, 1u);
}

// diag = 1 + sum of the face terms, b = E_old + boundary constants, 1/diag for the smoother, and
// per-block sums of (b_hi 2^-30)^2 (scaled back by 2^60 in FP64 at the block level).  Whole x rows
// per block iteration, 32-bit indices (the caller guarantees < 2^31 cells and faces per axis).
__device__ __forceinline__ void setup_face(bool inside, int bc, int side, dfl w, dfl vb, dfl gdx, dfl& d, dfl& cst) {
  if (inside || bc == FLD_BC_PERIODIC) {
    d = df_add(d, w);
  } else if (bc == FLD_BC_DIRICHLET) {
    d = df_add(d, w);
    cst = df_add(cst, df_mul(w, vb));
  } else if (bc == FLD_BC_NEUMANN) {
    // ghost = x -/+ g dx: the constant +/- w g dx moves to the right-hand side
    const dfl m = df_mul(w, gdx);
    cst = df_add(cst, side ? m : df_neg(m));
  } else {
    d = df_add(d, df_neg(w));
  }
}

__global__ void __launch_bounds__(256) k_fine_setup_df(GridDev g, DfConst K, LevelDev<float> L, LevelDev<float> Llo,
                                                       const double* __restrict__ E_old, float* __restrict__ dhi,
                                                       float* __restrict__ dlo, float* __restrict__ invd,
                                                       float* __restrict__ bhi, float* __restrict__ blo,
                                                       double* __restrict__ parts, unsigned* __restrict__ flag) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int rows = ny * nz;
  float acc = 0.0f;
  unsigned bad = 0u;
  auto V = [&](int f) { return dfl{K.v_hi[f], K.v_lo[f]}; };
  auto G = [&](int f) { return dfl{K.gdx_hi[f], K.gdx_lo[f]}; };
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const int idx = i + nx * row;
      dfl d{1.0f, 0.0f}, cst{0.0f, 0.0f};
      const int fx = i + (nx + 1) * row;
      setup_face(i > 0, g.bc[0], 0, {L.w[0][fx], Llo.w[0][fx]}, V(0), G(0), d, cst);
      setup_face(i < nx - 1, g.bc[1], 1, {L.w[0][fx + 1], Llo.w[0][fx + 1]}, V(1), G(1), d, cst);
      if (g.ndim >= 2) {
        const int fy = i + nx * (j + (ny + 1) * k);
        setup_face(j > 0, g.bc[2], 0, {L.w[1][fy], Llo.w[1][fy]}, V(2), G(2), d, cst);
        setup_face(j < ny - 1, g.bc[3], 1, {L.w[1][fy + nx], Llo.w[1][fy + nx]}, V(3), G(3), d, cst);
      }
      if (g.ndim == 3) {
        const int fz = idx, sz = nx * ny;
        setup_face(k > 0, g.bc[4], 0, {L.w[2][fz], Llo.w[2][fz]}, V(4), G(4), d, cst);
        setup_face(k < nz - 1, g.bc[5], 1, {L.w[2][fz + sz], Llo.w[2][fz + sz]}, V(5), G(5), d, cst);
      }
      float eh, el;
      bool ok;
      split_f64_scaled(E_old[idx], 0, eh, el, ok);
      if (!ok || !in_window(eh)) bad = 1u;
      const dfl b = df_add({eh, el}, cst);
      dhi[idx] = d.hi;
      dlo[idx] = d.lo;
      invd[idx] = __frcp_rn(d.hi);
      bhi[idx] = b.hi;
      blo[idx] = b.lo;
      const float bs = scale2(b.hi, -30);
      acc = fmaf(bs, bs, acc);
    }
  }
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = s * 0x1p60;
  if (bad) atomicOr(flag, 1u);
}

// scal[4] = 1 / rms(b) = sqrt(N / ||b||^2), for the residual kernels' scaled sums
__global__ void k_residual_scale(double* scal, double ncell) {
  if (threadIdx.x == 0 && blockIdx.x == 0) scal[4] = scal[1] > 0.0 ? sqrt(ncell / scal[1]) : 1.0;
}

// one face term of the first residual: sign (+1 interior/periodic, -1 extrapolated, 0 none) times
// w x_nb, with x_nb split from the FP64 state; branch-free like wave_face
__device__ __forceinline__ void df0_face(bool inside, int bc, int idx, int across, int wrap, int mirror, float whi,
                                         float wlo, const double* __restrict__ x, float& s, float& e, float& m) {
  const bool per = bc == FLD_BC_PERIODIC, cont = bc == FLD_BC_CONTINUOUS;
  const int nb = inside ? across : (per ? wrap : (cont ? mirror : idx));
  const float sg = (inside || per) ? 1.f : (cont ? -1.f : 0.f);
  float xh, xl;
  split_f64(x[nb], xh, xl);
  xh *= sg;
  xl *= sg;
  float t, te, s2, e2;
  two_prod(whi, xh, t, te);
  te = fmaf(whi, xl, te);
  te = fmaf(wlo, xh, te);
  two_sum(s, t, s2, e2);
  s = s2;
  e += e2 + te;
  m += fabsf(t);
}

// First outer residual of the mixed solver, r = b - A x with x = E_old (copied to the FP64
// iterate x64), all in double-float; as k_residual_update otherwise (32-bit indices).
template <int NDIM>
__global__ void __launch_bounds__(256) k_residual0_df(LevelDev<float> L, LevelDev<float> Llo,
                                                      const float* __restrict__ dhi, const float* __restrict__ dlo,
                                                      const float* __restrict__ bhi, const float* __restrict__ blo,
                                                      const double* __restrict__ x, double* __restrict__ x64,
                                                      float* __restrict__ rhi, float* __restrict__ rlo,
                                                      const double* __restrict__ scal, int nparts,
                                                      double* __restrict__ parts) {
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int rows = ny * nz, sy = nx, sz = nx * ny;
  const float scale = (float)scal[4];
  float ss = 0.f, mm = 0.f;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const int idx = i + nx * row;
      const double xc = x[idx];
      if (x64 != x) x64[idx] = xc;
      float xh, xl;
      split_f64(xc, xh, xl);
      const float bh = bhi[idx];
      // s + e = b - diag x
      float p, pe, s, e;
      const float dh = dhi[idx];
      two_prod(dh, xh, p, pe);
      pe = fmaf(dh, xl, pe);
      pe = fmaf(dlo[idx], xh, pe);
      two_sum(bh, -p, s, e);
      e += blo[idx] - pe;
      float m = fabsf(bh) + fabsf(p);
      const int fx = i + (nx + 1) * row;
      df0_face(i > 0, L.bc[0], idx, idx - 1, idx + (nx - 1), idx + 1, L.w[0][fx], Llo.w[0][fx], x, s, e, m);
      df0_face(i < nx - 1, L.bc[1], idx, idx + 1, idx - (nx - 1), idx - 1, L.w[0][fx + 1], Llo.w[0][fx + 1], x, s,
               e, m);
      if (NDIM >= 2) {
        const int fy = i + nx * (j + (ny + 1) * k);
        df0_face(j > 0, L.bc[2], idx, idx - sy, idx + (ny - 1) * sy, idx + sy, L.w[1][fy], Llo.w[1][fy], x, s, e, m);
        df0_face(j < ny - 1, L.bc[3], idx, idx + sy, idx - (ny - 1) * sy, idx - sy, L.w[1][fy + nx],
                 Llo.w[1][fy + nx], x, s, e, m);
      }
      if (NDIM == 3) {
        df0_face(k > 0, L.bc[4], idx, idx - sz, idx + (nz - 1) * sz, idx + sz, L.w[2][idx], Llo.w[2][idx], x, s, e,
                 m);
        df0_face(k < nz - 1, L.bc[5], idx, idx + sz, idx - (nz - 1) * sz, idx - sz, L.w[2][idx + sz],
                 Llo.w[2][idx + sz], x, s, e, m);
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

// ----------------------------------------------------------------------------- launchers

DfConst make_df_const(const GridDev& g, double dt) {
  DfConst K{};
  auto split_host = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  for (int a = 0; a < 3; ++a) split_host(dt * g.inv_dx2[a], K.s_hi[a], K.s_lo[a]);
  for (int f = 0; f < 6; ++f) {
    split_host(g.bc_val[f], K.v_hi[f], K.v_lo[f]);
    split_host(g.bc_val[f] * g.dx[f / 2], K.gdx_hi[f], K.gdx_lo[f]);
  }
  return K;
}

cudaError_t launch_faces_df(const GridDev& g, const DfConst& K, const double* D, float* const w[3],
                            float* const wlo[3], unsigned* flag, cudaStream_t s) {
  TraceScope ts("faces", s);
  const int rows = g.n[1] * g.n[2];
  k_faces_df<<<(unsigned)std::min(rows, 152 * 16), 256, 0, s>>>(g, K, D, w[0], w[1], w[2], wlo[0], wlo[1], wlo[2], flag);
  return cudaGetLastError();
}

cudaError_t launch_fine_setup_df(const GridDev& g, const DfConst& K, const LevelDev<float>& L,
                                 const LevelDev<float>& Llo, const double* E_old, float* dhi, float* dlo, float* invd,
                                 float* bhi, float* blo, double* parts, int nparts, double* scal, unsigned* flag,
                                 cudaStream_t s) {
  TraceScope ts("fine_setup", s);
  k_fine_setup_df<<<nparts, 256, 0, s>>>(g, K, L, Llo, E_old, dhi, dlo, invd, bhi, blo, parts, flag);
  k_reduce<<<1, 1024, 0, s>>>(parts, nparts, scal + 1);
  k_residual_scale<<<1, 32, 0, s>>>(scal, (double)g.ncell);
  return cudaGetLastError();
}

cudaError_t launch_residual0_df(int ndim, const LevelDev<float>& L, const LevelDev<float>& Llo, const float* dhi,
                                const float* dlo, const float* bhi, const float* blo, const double* x, double* x64,
                                float* rhi, float* rlo, const double* scal, int nparts, double* parts,
                                cudaStream_t s) {
  if (ndim == 3)
    k_residual0_df<3><<<nparts, 256, 0, s>>>(L, Llo, dhi, dlo, bhi, blo, x, x64, rhi, rlo, scal, nparts, parts);
  else if (ndim == 2)
    k_residual0_df<2><<<nparts, 256, 0, s>>>(L, Llo, dhi, dlo, bhi, blo, x, x64, rhi, rlo, scal, nparts, parts);
  else
    k_residual0_df<1><<<nparts, 256, 0, s>>>(L, Llo, dhi, dlo, bhi, blo, x, x64, rhi, rlo, scal, nparts, parts);
  return cudaGetLastError();
}

}  // namespace fld

// Double-float setup of the mixed solver's finest level: face weights, then the diagonal,
// right-hand side and first outer residual in one pass, computed on the FP32 and integer pipes
// (see df.cuh) instead of in FP64.  The mixed solver only ever consumes these quantities as hi + lo
// float pairs (the FP32 V-cycle takes the hi parts, the residual updates both), so no FP64 copy is
// made.
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
// per axis); eight blocks of 256 per SM (32 registers).
__global__ void __launch_bounds__(256, 8) k_faces_df(GridDev g, DfConst K, const double* __restrict__ D,
                                                  float* __restrict__ w0, float* __restrict__ w1,
                                                  float* __restrict__ w2, float* __restrict__ l0,
                                                  float* __restrict__ l1, float* __restrict__ l2,
                                                  float* __restrict__ dc, unsigned* __restrict__ flag) {
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
      // the reciprocal of the cell's dt D / dx_0^2 in FP32, for the smoother that forms its face
      // means on chip (inf where the product leaves the FP32 range downwards)
      if (dc) dc[idx] = __frcp_rn(scale2(c.hi * K.s_hi[0], sh));
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

// One face's share of the diagonal (diag = 1 + sum of the face terms) and of the boundary
// constants of b: interior and periodic faces add w; a Dirichlet face adds w and w v to b; a
// Neumann face (ghost = x -/+ g dx) moves the constant +/- w g dx to b; a continuous face
// (linear extrapolation) subtracts w.
__device__ __forceinline__ void setup_face(bool inside, int bc, int side, dfl w, dfl vb, dfl gdx, dfl& d, dfl& cst) {
  if (inside || bc == FLD_BC_PERIODIC) {
    d = df_add_pos(d, w);
  } else if (bc == FLD_BC_DIRICHLET) {
    d = df_add_pos(d, w);
    cst = df_add(cst, df_mul(w, vb));
  } else if (bc == FLD_BC_NEUMANN) {
    const dfl m = df_mul(w, gdx);
    cst = df_add(cst, side ? m : df_neg(m));
  } else {
    d = df_add(d, df_neg(w));
  }
}

// One face's term of the first residual: sign (+1 interior/periodic, -1 extrapolated, 0 none)
// times w x_nb, with x_nb split from the FP64 state, summed into s + e (m: the sum of magnitudes);
// branch-free like wave_face.
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

// The finest level's set-up and the first outer residual of the mixed solver in one pass, in
// double-float arithmetic: diag = 1 + sum of the face terms (hi, lo) and 1/diag for the smoother,
// b = E_old + boundary constants (not stored), and r = b - A x with x = E_old, which is also copied
// into the FP64 iterate x64 unless x64 is null.  Per-block sums: parts[0..n) = sum r_hi^2 in FP64,
// parts[n..2n) = sum m^2 (m: the magnitudes of the residual's terms, for the drift bound of the
// updates) and parts[2n..3n) = sum b_hi^2, both accumulated as (v 2^-30)^2 in FP32 and scaled
// back by 2^60.  *flag |= 1 where E_old leaves the double-float window.  Whole x rows per block
// iteration, 32-bit indices (the caller guarantees < 2^31 cells and faces per axis).  Six blocks
// per SM (40 registers): the pass is bound by memory latency, and more warps in flight measured
// 15 % faster than five.
template <int NDIM>
__global__ void __launch_bounds__(256, 6) k_setup_res0_df(GridDev g, DfConst K, LevelDev<float> L, LevelDev<float> Llo,
                                                       const double* __restrict__ x, double* __restrict__ x64,
                                                       float* __restrict__ dhi, float* __restrict__ dlo,
                                                       float* __restrict__ invd, float* __restrict__ rhi,
                                                       float* __restrict__ rlo, int nparts, double* __restrict__ parts,
                                                       unsigned* __restrict__ flag) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int rows = ny * nz, sy = nx, sz = nx * ny;
  float acc_b = 0.f, acc_m = 0.f;
  double acc_r = 0.0;
  unsigned bad = 0u;
  auto V = [&](int f) { return dfl{K.v_hi[f], K.v_lo[f]}; };
  auto G = [&](int f) { return dfl{K.gdx_hi[f], K.gdx_lo[f]}; };
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const int idx = i + nx * row;
      const double xc = x[idx];
      if (x64) x64[idx] = xc;
      float xh, xl;
      bool ok;
      split_f64_scaled(xc, 0, xh, xl, ok);
      if (!ok || !in_window(xh)) bad = 1u;
      dfl d{1.0f, 0.0f}, cst{0.0f, 0.0f};
      float s = 0.f, e = 0.f, m = 0.f;
      {
        const int fx = i + (nx + 1) * row;
        const float w0h = L.w[0][fx], w0l = Llo.w[0][fx], w1h = L.w[0][fx + 1], w1l = Llo.w[0][fx + 1];
        setup_face(i > 0, g.bc[0], 0, {w0h, w0l}, V(0), G(0), d, cst);
        setup_face(i < nx - 1, g.bc[1], 1, {w1h, w1l}, V(1), G(1), d, cst);
        df0_face(i > 0, g.bc[0], idx, idx - 1, idx + (nx - 1), idx + 1, w0h, w0l, x, s, e, m);
        df0_face(i < nx - 1, g.bc[1], idx, idx + 1, idx - (nx - 1), idx - 1, w1h, w1l, x, s, e, m);
      }
      if (NDIM >= 2) {
        const int fy = i + nx * (j + (ny + 1) * k);
        const float w0h = L.w[1][fy], w0l = Llo.w[1][fy], w1h = L.w[1][fy + nx], w1l = Llo.w[1][fy + nx];
        setup_face(j > 0, g.bc[2], 0, {w0h, w0l}, V(2), G(2), d, cst);
        setup_face(j < ny - 1, g.bc[3], 1, {w1h, w1l}, V(3), G(3), d, cst);
        df0_face(j > 0, g.bc[2], idx, idx - sy, idx + (ny - 1) * sy, idx + sy, w0h, w0l, x, s, e, m);
        df0_face(j < ny - 1, g.bc[3], idx, idx + sy, idx - (ny - 1) * sy, idx - sy, w1h, w1l, x, s, e, m);
      }
      if (NDIM == 3) {
        const float w0h = L.w[2][idx], w0l = Llo.w[2][idx], w1h = L.w[2][idx + sz], w1l = Llo.w[2][idx + sz];
        setup_face(k > 0, g.bc[4], 0, {w0h, w0l}, V(4), G(4), d, cst);
        setup_face(k < nz - 1, g.bc[5], 1, {w1h, w1l}, V(5), G(5), d, cst);
        df0_face(k > 0, g.bc[4], idx, idx - sz, idx + (nz - 1) * sz, idx + sz, w0h, w0l, x, s, e, m);
        df0_face(k < nz - 1, g.bc[5], idx, idx + sz, idx - (nz - 1) * sz, idx - sz, w1h, w1l, x, s, e, m);
      }
      const dfl b = df_add({xh, xl}, cst);
      // r = b - diag x + (s + e)
      float p, pe;
      two_prod(d.hi, xh, p, pe);
      pe = fmaf(d.hi, xl, pe);
      pe = fmaf(d.lo, xh, pe);
      float s1, e1, s2, e2;
      two_sum(b.hi, -p, s1, e1);
      two_sum(s1, s, s2, e2);
      float rh, rl;
      quick_two_sum(s2, ((e1 + e2) + (e + b.lo)) - pe, rh, rl);
      m += fabsf(b.hi) + fabsf(p);
      dhi[idx] = d.hi;
      dlo[idx] = d.lo;
      invd[idx] = __frcp_rn(d.hi);
      rhi[idx] = rh;
      rlo[idx] = rl;
      const float bs = scale2(b.hi, -30), ms = scale2(m, -30);
      acc_b = fmaf(bs, bs, acc_b);
      acc_m = fmaf(ms, ms, acc_m);
      const double rd = f32_to_f64(rh);
      acc_r = fma(rd, rd, acc_r);
    }
  }
  const double sr = block_sum(acc_r);
  __syncthreads();  // block_sum's shared scratch is reused
  const double sm = block_sum((double)acc_m);
  __syncthreads();
  const double sb = block_sum((double)acc_b);
  if (threadIdx.x == 0) {
    parts[blockIdx.x] = sr;
    parts[nparts + blockIdx.x] = sm * 0x1p60;
    parts[2 * nparts + blockIdx.x] = sb * 0x1p60;
  }
  if (bad) atomicOr(flag, 1u);
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
                            float* const wlo[3], float* dc, unsigned* flag, cudaStream_t s) {
  TraceScope ts("faces", s);
  const int rows = g.n[1] * g.n[2];
  // two fronts of resident blocks measured faster here than one (1.86 against 2.07 ms at 512^3)
  const unsigned grid = (unsigned)std::min(rows, 152 * 16);
  note_launch(),
      k_faces_df<<<grid, 256, 0, s>>>(g, K, D, w[0], w[1], w[2], wlo[0], wlo[1], wlo[2], dc, flag);
  return cudaGetLastError();
}

cudaError_t launch_setup_res0_df(const GridDev& g, const DfConst& K, const LevelDev<float>& L,
                                 const LevelDev<float>& Llo, const double* x, double* x64, float* dhi, float* dlo,
                                 float* invd, float* rhi, float* rlo, int nparts, double* parts, double* scal,
                                 unsigned* flag, cudaStream_t s) {
  // one front of resident blocks (at most nparts, the partial-sum capacity)
  nparts = front_grid((const void*)k_setup_res0_df<3>, nparts);
  if (g.ndim == 3)
    note_launch(),
        k_setup_res0_df<3><<<nparts, 256, 0, s>>>(g, K, L, Llo, x, x64, dhi, dlo, invd, rhi, rlo, nparts, parts, flag);
  else if (g.ndim == 2)
    note_launch(),
        k_setup_res0_df<2><<<nparts, 256, 0, s>>>(g, K, L, Llo, x, x64, dhi, dlo, invd, rhi, rlo, nparts, parts, flag);
  else
    note_launch(),
        k_setup_res0_df<1><<<nparts, 256, 0, s>>>(g, K, L, Llo, x, x64, dhi, dlo, invd, rhi, rlo, nparts, parts, flag);
  note_launch(), k_reduce<<<1, 1024, 0, s>>>(parts, nparts, scal);
  note_launch(), k_reduce<<<1, 1024, 0, s>>>(parts + nparts, nparts, scal + 2);
  note_launch(), k_reduce<<<1, 1024, 0, s>>>(parts + 2 * nparts, nparts, scal + 1);
  return cudaGetLastError();
}

}  // namespace fld

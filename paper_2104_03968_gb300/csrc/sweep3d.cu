// Red-black Gauss-Seidel sweep of the backward-Euler diffusion operator of Sect. 3.4 (Eq.
// discdiff, dt-scaled: (A x)_c = x_c + sum_faces w_f (x_c - x_nb)) on the FP32 finest level of a
// 3-D grid, both colours in one pass over HBM.
//
// The face weights are not read from memory: the kernel stages each cell's reciprocal
// coefficient ic = 1 / (dt D / dx_0^2) and forms the harmonic-mean weight of a face (Sect. 3.4) on
// chip as w = 2 ra / (ic_a + ic_b), one reciprocal per face, so a sweep moves r, ic and x in and x
// out (16 bytes per cell) instead of r, three face arrays and x (24).  A cell with D = 0 has
// ic = inf and its faces weigh 0.
//
// Blocking: a block of 128 threads owns a 64 x 16 tile of the x-y plane and a run of z-planes (a
// z-chunk), and marches through them.  At step s it updates the first colour on plane s (on the
// tile and a one-cell ring around it) and the second colour on plane s - 1 (on the tile), so that
// every value the second colour reads is final.
//
// Each thread owns a patch of 2 x 4 cells (two rows, four cells along x) at a fixed (i, j) and
// keeps the patch's x and ic on planes s - 2 .. s + 1 in registers, so the neighbours along z,
// along the strip and across the patch's two rows never go through shared memory.  A 16-byte
// shared load brings the row above or below the patch, and the cells beyond the strip's ends come
// from the neighbouring lane by a warp shuffle (from shared memory at the tile's border).  The
// colours occupy alternate cells, and the second colour's cells on plane s - 1 sit at the same
// patch positions as the first colour's on plane s; with z-chunks that start on even planes the
// position class of each step of the plane loop (unrolled over the four register slots) and of
// each colour order is fixed at compile time, so every register index is static.
//
// Shared memory holds four slots of staged x and ic planes (two-cell halo) and two of r planes
// (one-cell halo; the second colour keeps the r of its cells in registers from the step before),
// 57 KB per block, so four blocks share an SM within its registers (at most 128 per thread).
// The planes are fetched one step ahead by tensor-memory-accelerator (TMA) box loads: one thread
// issues one 72 x 20 (x, ic) or 72 x 18 (r) box per staged plane, completing on an mbarrier that
// every thread waits on, with an iteration bound, at the end of the step.  Box
// cells beyond a non-periodic face arrive as zeros and are only ever read by boundary faces, which
// ignore them.  A box does not wrap, so tiles whose halo crosses a periodic face fetch their
// planes with 16-byte asynchronous copies (cp.async) from the wrapped addresses instead.  After its
// first-colour pass a thread writes its patch back to the plane's slot, where the next step's
// second colour reads it; second-colour values go from registers straight to global memory.  The
// ring's first-colour cells (82 per plane, threads 0..81) are computed from the slots with the same
// function and operand order as the tile's cells, so they equal the neighbouring blocks' values
// bit for bit, and the sweep reads x from one array and writes another: no block waits for another.
// Periodic faces read the wrapped halo; Dirichlet, Neumann and linear-extrapolation faces take the
// interior cell's coefficient, as in the FP64 operator, with the face terms summed in the same
// order as on interior cells (grids with such faces run an instantiation that checks every cell).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fld_common.cuh"
#include "sweep3d.h"

namespace fld {

namespace {

constexpr int TX = 64, TY = 16;        // tile of a plane
constexpr int P = TX + 8;              // row pitch in shared memory: 4 cells each side (16-byte aligned)
constexpr int RXR = TY + 4;            // rows of a staged x or ic plane (2 halo rows each side)
constexpr int RRR = TY + 2;            // rows of a staged r plane (1 halo row each side)
constexpr int CH = P / 4;              // 16-byte chunks per staged row
constexpr int NS = 4;                  // slots: planes s - 1 .. s + 2 (s - 2 lives in registers only)
constexpr int XPL = RXR * P, RPL = RRR * P;
constexpr int RPS = 1312;              // r slot stride: 128-byte aligned slots for the TMA
constexpr int kThreads = 128;
constexpr int kXChunks = RXR * CH, kRChunks = RRR * CH;  // 360, 324: at most three per thread each
constexpr int kRingHalf = TX + 2 + TY;  // 82 ring cells of each parity around the tile
constexpr int NR = 2;                  // r slots: planes s and s + 1 (the second colour keeps its r in registers)
constexpr size_t kBarOffset = (size_t)(2 * NS * XPL + NR * RPS) * sizeof(float);
constexpr size_t kSmemBytes = kBarOffset + 16;  // slots, then one mbarrier
static_assert((XPL * 4) % 128 == 0 && (RPS * 4) % 128 == 0 && RPS >= RPL, "128-byte aligned TMA slots");
static_assert(kRingHalf <= kThreads && kXChunks <= 3 * kThreads && kRChunks <= 3 * kThreads, "thread shares");
static_assert(kThreads * 8 == TX * TY, "one 2 x 4 patch per thread");

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// the slots' generic-proxy accesses (loads, first-colour stores) before later TMA writes to them
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces the bytes the step's TMA copies will deliver (0: none)
__device__ __forceinline__ void mbar_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// wait for the phase of the given parity to complete; false after the iteration bound
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  for (int it = 0; it < (1 << 20); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// TMA box load of the map's box at (x, y, z) into dst, completing on bar
__device__ __forceinline__ void tma3(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// one hardware reciprocal (rcp.approx, about 1 ulp; 0 for inf): the smoother's arithmetic is FP32
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void lds4(float* d, const float* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  d[0] = v.x, d[1] = v.y, d[2] = v.z, d[3] = v.w;
}
__device__ __forceinline__ void sts4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// One face's contribution: returns its diagonal term and adds its neighbour term to a.  Interior
// and periodic faces pair the cell (reciprocal coefficient ic) with the one across (ia, value xa);
// a Dirichlet face adds the cell's own weight to the diagonal only; a Neumann face adds nothing; a
// linear-extrapolation face (ghost 2 x_c - x_m, xm the opposite neighbour) subtracts w x_m and w.
template <bool NOX>
__device__ __forceinline__ float face_term(bool pair, int bc, float t, float ra, float ic, float ia, float xa, float xm,
                                           float& a) {
  if (pair) {
    const float w = t * rcp_fast(ic + ia);
    if (!NOX) a = fmaf(w, xa, a);
    return w;
  }
  if (bc == FLD_BC_DIRICHLET) return ra * rcp_fast(ic);
  if (bc == FLD_BC_CONTINUOUS) {
    const float w = ra * rcp_fast(ic);
    if (!NOX) a = fmaf(-w, xm, a);
    return -w;
  }
  return 0.0f;
}

// New value of a cell from its right-hand side rv, its ic and its six neighbours' ic (cn) and x
// (xn), faces ordered x-, x+, y-, y+, z-, z+.  NOX: x is zero everywhere (first colour of a sweep
// from zero).  BND: bit f of bm marks face f as a non-periodic boundary face.  On a cell with no
// boundary face both forms give the same bits.
template <bool NOX, bool BND>
__device__ __forceinline__ float cell(const Sweep3dArgs& A, const float tr[3], float rv, float ic, const float (&cn)[6],
                                      const float (&xn)[6], unsigned bm) {
  float a = rv, w[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (BND) {
      w[f] = face_term<NOX>(!((bm >> f) & 1u), A.bc[f], tr[f >> 1], A.ra[f >> 1], ic, cn[f], xn[f], xn[f ^ 1], a);
    } else {
      w[f] = tr[f >> 1] * rcp_fast(ic + cn[f]);
      if (!NOX) a = fmaf(w[f], xn[f], a);
    }
  }
  const float d = 1.0f + (((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]));
  return a * rcp_fast(d);
}

__device__ __forceinline__ unsigned bnd_mask(const Sweep3dArgs& A, int i, int j, int k) {
  unsigned m = 0u;
  m |= (i == 0 && A.bc[0] != FLD_BC_PERIODIC) ? 1u : 0u;
  m |= (i == A.nx - 1 && A.bc[1] != FLD_BC_PERIODIC) ? 2u : 0u;
  m |= (j == 0 && A.bc[2] != FLD_BC_PERIODIC) ? 4u : 0u;
  m |= (j == A.ny - 1 && A.bc[3] != FLD_BC_PERIODIC) ? 8u : 0u;
  m |= (k == 0 && A.bc[4] != FLD_BC_PERIODIC) ? 16u : 0u;
  m |= (k == A.nz - 1 && A.bc[5] != FLD_BC_PERIODIC) ? 32u : 0u;
  return m;
}

__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool periodic) {
  if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// A thread's share of a tile.
//  - Its patch: warp w, lanes 0-15 take rows 4 w and 4 w + 1, lanes 16-31 rows 4 w + 2 and
//    4 w + 3; lane % 16 is the strip along x (four cells from column 4 (lane % 16)).  oA is the
//    staged offset of the patch's first row in an x or ic slot (the second row: oA + P; r slots
//    have one halo row fewer: oA - P).
//  - Threads 0..81 each own one ring cell of either parity class (iu + ju even or odd; 82 each:
//    33 in the row below the tile, 33 above, 8 in each side column).
struct Share {
  int oA, rowA, sx;
  int ring_o[2];
};

__device__ __forceinline__ Share make_share() {
  Share sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  sh.rowA = 4 * warp + 2 * (lane >> 4);
  sh.sx = lane & 15;
  sh.oA = (2 + sh.rowA) * P + 4 + 4 * sh.sx;
  // ring: with i0 and j0 even, the staged position (ii, jj) has parity (iu + ju) & 1 = (ii + jj) & 1
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int q = min(t, kRingHalf - 1);
    int ii, jj;
    if (q < TX / 2 + 1) ii = 3 + c + 2 * q, jj = 1;                             // row j0 - 1
    else if (q < TX + 2) ii = 4 - c + 2 * (q - (TX / 2 + 1)), jj = RXR - 2;      // row j0 + 16
    else if (q < TX + 2 + TY / 2) ii = 3, jj = 3 - c + 2 * (q - (TX + 2));       // column i0 - 1
    else ii = P - 4, jj = 2 + c + 2 * (q - (TX + 2 + TY / 2));                   // column i0 + 64
    sh.ring_o[c] = jj * P + ii;
  }
  return sh;
}

// cp.async staging of one tile (tiles whose halo wraps): each thread copies up to three 16-byte
// chunks of a staged x and ic plane and of an r plane; xg / rg are their in-plane source offsets
// (-1: none), xo their offsets in a slot (the same for the x and r chunks of one thread).  A chunk
// beyond a periodic face wraps; beyond a non-periodic one it is clamped into the grid (the
// boundary faces do not read it).
struct Chunks {
  int xg[3], xo[3], rg[3];
};

__device__ __forceinline__ Chunks make_chunks(int i0, int j0, const Sweep3dArgs& A, bool xper, bool yper) {
  Chunks ch;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int tt = threadIdx.x + c * kThreads;
    auto chunk = [&](int q, int jlo, int& g, int& o) {
      const int jj = q / CH, cc = q % CH;
      const int j = wrap_or_clamp(j0 + jlo + jj, A.ny, yper);
      int i = i0 - 4 + 4 * cc;
      i = xper ? (i < 0 ? i + A.nx : (i >= A.nx ? i - A.nx : i)) : min(max(i, 0), A.nx - 4);
      g = j * A.nx + i;
      o = jj * P + 4 * cc;
    };
    if (tt < kXChunks) chunk(tt, -2, ch.xg[c], ch.xo[c]);
    else ch.xg[c] = -1, ch.xo[c] = 0;
    int ro;
    if (tt < kRChunks) chunk(tt, -1, ch.rg[c], ro);
    else ch.rg[c] = -1;
  }
  return ch;
}

// Box maps of the staged arrays (x_in, ic: 72 x 20 x 1 boxes; r: 72 x 18 x 1), encoded on the host.
struct Sweep3dMaps {
  CUtensorMap x, c, r;
};

// One colour pass over a thread's patch on one plane: row A's cells at strip positions Q and
// Q + 2, row B's at 1 - Q and 3 - Q.  xo/co: the plane's registers (row A 0..3, row B 4..7);
// xm/cm, xp/cp: the planes below and above; xs, cs: the plane's slots (the rows above A and below
// B, and the strip ends of the tile's border lanes); rs: its r slot.  The new values replace the
// updated cells of xo.  Every x it reads is of the other colour, which this pass does not change.
template <int Q, bool NOX, bool BND>
__device__ __forceinline__ void patch_pass(const Sweep3dArgs& A, const float tr[3], const Share& sh, int i0, int j0,
                                           int kw, const float* xs, const float* cs, const float (&ra)[4],
                                           const float (&rb)[4], float (&xo)[8],
                                           const float (&co)[8], const float (&xm)[8], const float (&cm)[8],
                                           const float (&xp)[8], const float (&cp)[8]) {
  const int oA = sh.oA, oB = oA + P;
  float ca[4], cb[4], xa[4] = {0.f, 0.f, 0.f, 0.f}, xb[4] = {0.f, 0.f, 0.f, 0.f};
  lds4(ca, cs + oA - P);
  lds4(cb, cs + oB + P);
  if (!NOX) {
    lds4(xa, xs + oA - P);
    lds4(xb, xs + oB + P);
  }
  // Strip ends: row A needs its left neighbour for Q = 0 (right for Q = 1), row B the other side.
  // The neighbouring strip belongs to the next lane of the 16-lane row group.
  const unsigned full = 0xffffffffu;
  float eAc, eBc, eAx = 0.f, eBx = 0.f;
  if (Q == 0) {
    eAc = __shfl_up_sync(full, co[3], 1, 16);
    eBc = __shfl_down_sync(full, co[4], 1, 16);
    if (!NOX) {
      eAx = __shfl_up_sync(full, xo[3], 1, 16);
      eBx = __shfl_down_sync(full, xo[4], 1, 16);
    }
    if (sh.sx == 0) {
      eAc = cs[oA - 1];
      if (!NOX) eAx = xs[oA - 1];
    }
    if (sh.sx == 15) {
      eBc = cs[oB + 4];
      if (!NOX) eBx = xs[oB + 4];
    }
  } else {
    eAc = __shfl_down_sync(full, co[0], 1, 16);
    eBc = __shfl_up_sync(full, co[7], 1, 16);
    if (!NOX) {
      eAx = __shfl_down_sync(full, xo[0], 1, 16);
      eBx = __shfl_up_sync(full, xo[7], 1, 16);
    }
    if (sh.sx == 15) {
      eAc = cs[oA + 4];
      if (!NOX) eAx = xs[oA + 4];
    }
    if (sh.sx == 0) {
      eBc = cs[oB - 1];
      if (!NOX) eBx = xs[oB - 1];
    }
  }
  const int iA = i0 + 4 * sh.sx, jA = j0 + sh.rowA;
  float v[4];
#pragma unroll
  for (int u = 0; u < 2; ++u) {  // row A
    const int p = Q + 2 * u;
    const float cn[6] = {p == 0 ? eAc : co[p > 0 ? p - 1 : 0], p == 3 ? eAc : co[p < 3 ? p + 1 : 3], ca[p],
                         co[4 + p], cm[p], cp[p]};
    const float xn[6] = {p == 0 ? eAx : xo[p > 0 ? p - 1 : 0], p == 3 ? eAx : xo[p < 3 ? p + 1 : 3], xa[p],
                         xo[4 + p], xm[p], xp[p]};
    const unsigned bm = BND ? bnd_mask(A, iA + p, jA, kw) : 0u;
    v[u] = cell<NOX, BND>(A, tr, ra[p], co[p], cn, xn, bm);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {  // row B
    const int p = 1 - Q + 2 * u;
    const float cn[6] = {p == 0 ? eBc : co[4 + (p > 0 ? p - 1 : 0)], p == 3 ? eBc : co[4 + (p < 3 ? p + 1 : 3)], co[p],
                         cb[p], cm[4 + p], cp[4 + p]};
    const float xn[6] = {p == 0 ? eBx : xo[4 + (p > 0 ? p - 1 : 0)], p == 3 ? eBx : xo[4 + (p < 3 ? p + 1 : 3)], xo[p],
                         xb[p], xm[4 + p], xp[4 + p]};
    const unsigned bm = BND ? bnd_mask(A, iA + p, jA + 1, kw) : 0u;
    v[2 + u] = cell<NOX, BND>(A, tr, rb[p], co[4 + p], cn, xn, bm);
  }
  xo[Q] = v[0];
  xo[Q + 2] = v[1];
  xo[4 + 1 - Q] = v[2];
  xo[4 + 3 - Q] = v[3];
}

// First colour of plane kw on one ring cell (staged offset o), read entirely from the slots: x and
// ic of the plane (xs, cs), below (xsm, csm) and above (xsp, csp); r from rs.
template <bool NOX, bool BND>
__device__ __noinline__ void ring_cell(const Sweep3dArgs& A, int i0, int j0, int o, int kw, float* xs, const float* cs,
                                       const float* xsm, const float* csm, const float* xsp, const float* csp,
                                       const float* rs) {
  const float tr[3] = {2.0f * A.ra[0], 2.0f * A.ra[1], 2.0f * A.ra[2]};
  const float cn[6] = {cs[o - 1], cs[o + 1], cs[o - P], cs[o + P], csm[o], csp[o]};
  float xn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (!NOX) {
    xn[0] = xs[o - 1], xn[1] = xs[o + 1], xn[2] = xs[o - P], xn[3] = xs[o + P];
    xn[4] = xsm[o], xn[5] = xsp[o];
  }
  unsigned bm = 0u;
  if (BND) {  // the ring cell's global (i, j), wrapped on periodic axes
    const int jj = o / P, ii = o - jj * P;
    const int ri = wrap_or_clamp(i0 + ii - 4, A.nx, A.bc[0] == FLD_BC_PERIODIC);
    const int rj = wrap_or_clamp(j0 + jj - 2, A.ny, A.bc[2] == FLD_BC_PERIODIC);
    bm = bnd_mask(A, ri, rj, kw);
  }
  xs[o] = cell<NOX, BND>(A, tr, rs[o - P], cs[o], cn, xn, bm);
}

// The plane loop of one item (a tile's z-chunk), with the patch registers of planes s - 2 .. s + 1.
// Plane p sits in slot (p - k0 + 2) % 4 of shared memory and of the registers.
template <int C0, bool ZERO, bool UPDATE, bool BND>
struct Sweeper {
  const Sweep3dArgs& A;
  const Sweep3dMaps& M;
  const float* tr;
  float* Xs;
  float* Cs;
  float* Rs;
  uint64_t* bar;
  const Share& sh;
  const Chunks& ch;
  int i0, j0, k0, k1;
  bool zper, use_tma;
  size_t plane;
  float (&X)[NS][8];
  float (&C)[NS][8];
  float (&RK)[2][4];  // r of the cells the second colour updates on the plane just done, by step parity

  __device__ __forceinline__ bool valid(int k) const { return zper || (k >= 0 && k < A.nz); }
  __device__ __forceinline__ int wrapk(int k) const { return k < 0 ? k + A.nz : (k >= A.nz ? k - A.nz : k); }

  // bytes the TMA boxes of x and ic of plane kx and r of plane kr deliver
  __device__ __forceinline__ unsigned box_bytes(bool do_x, int kx, bool do_r, int kr) const {
    return (do_x && valid(kx) ? (ZERO ? 1u : 2u) * (unsigned)(XPL * sizeof(float)) : 0u) +
           (do_r && valid(kr) ? (unsigned)(RPL * sizeof(float)) : 0u);
  }

  // Fetch x and ic of plane kx into slot sx (if do_x) and r of plane kr into slot sr (if do_r):
  // TMA boxes issued by thread 0 (after the step's mbar_expect), or every thread's cp.async chunks
  // on a tile whose halo wraps (committed by the caller).  Planes outside a non-periodic z range
  // are skipped.
  __device__ __forceinline__ void issue(bool do_x, int kx, int sx, bool do_r, int kr, int sr) const {
    do_x = do_x && valid(kx);
    do_r = do_r && valid(kr);
    if (use_tma) {
      if (threadIdx.x != 0) return;
      if (do_x) {
        if (!ZERO) tma3(Xs + sx * XPL, &M.x, i0 - 4, j0 - 2, wrapk(kx), bar);
        tma3(Cs + sx * XPL, &M.c, i0 - 4, j0 - 2, wrapk(kx), bar);
      }
      if (do_r) tma3(Rs + sr * RPS, &M.r, i0 - 4, j0 - 1, wrapk(kr), bar);
      return;
    }
    const size_t px = (size_t)wrapk(kx) * plane, pr = (size_t)wrapk(kr) * plane;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (do_x && ch.xg[c] >= 0) {
        if (!ZERO) cp16(Xs + sx * XPL + ch.xo[c], A.xin + px + ch.xg[c]);
        cp16(Cs + sx * XPL + ch.xo[c], A.dc + px + ch.xg[c]);
      }
      if (do_r && ch.rg[c] >= 0) cp16(Rs + sr * RPS + ch.xo[c], A.r + pr + ch.rg[c]);
    }
  }

  // one step's fetch: x and ic of plane kx into slot sx, r of plane kr into r slot sr
  __device__ __forceinline__ void stage(bool do_x, int kx, int sx, bool do_r, int kr, int sr) const {
    if (use_tma && threadIdx.x == 0) mbar_expect(bar, box_bytes(do_x, kx, do_r, kr));
    issue(do_x, kx, sx, do_r, kr, sr);
    if (!use_tma) cp_commit();
  }

  // the item's first fetch: x and ic of planes k0 - 2 .. k0 in slots 0..2, r of k0 - 1 in r slot 1
  // (plane p's r slot is (p - k0 + 2) % 2)
  __device__ __forceinline__ void stage_prologue() const {
    if (use_tma && threadIdx.x == 0)
      mbar_expect(bar, box_bytes(true, k0 - 2, false, 0) + box_bytes(true, k0 - 1, true, k0 - 1) +
                           box_bytes(true, k0, false, 0));
    issue(true, k0 - 2, 0, false, 0, 0);
    issue(true, k0 - 1, 1, true, k0 - 1, 1);
    issue(true, k0, 2, false, 0, 0);
    if (!use_tma) cp_commit();
  }

  // End of a step: the staged planes have landed and every thread is done with the slots.  True
  // (for the whole block) when a TMA wait ran out of its bound: the error word is set and the block
  // leaves after giving the copies in flight a second bound.
  __device__ __forceinline__ bool step_end(unsigned& phase) const {
    if (!use_tma) {
      cp_wait_all();
      __syncthreads();
      return false;
    }
    const int late = mbar_wait(bar, phase) ? 0 : 1;
    fence_proxy_async();
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0 && A.err) atomicOr(A.err, 1u);
      mbar_wait(bar, phase);
      return true;
    }
    phase ^= 1u;
    return false;
  }

  // registers of slot q <- the thread's patch of the plane staged in slot q
  template <int Q>
  __device__ __forceinline__ void load_patch() const {
    if (ZERO) {
#pragma unroll
      for (int c = 0; c < 8; ++c) X[Q][c] = 0.f;
    } else {
      lds4(&X[Q][0], Xs + Q * XPL + sh.oA);
      lds4(&X[Q][4], Xs + Q * XPL + sh.oA + P);
    }
    lds4(&C[Q][0], Cs + Q * XPL + sh.oA);
    lds4(&C[Q][4], Cs + Q * XPL + sh.oA + P);
  }

  template <int Q>
  __device__ __forceinline__ void store_plane(int k) const {
    const size_t g = (size_t)wrapk(k) * plane + (size_t)(j0 + sh.rowA) * A.nx + i0 + 4 * sh.sx;
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const size_t gr = g + (size_t)row * A.nx;
      const float* v = &X[Q][4 * row];
      *reinterpret_cast<float4*>(A.xout + gr) = make_float4(v[0], v[1], v[2], v[3]);
      if (UPDATE) {
        double2* p = reinterpret_cast<double2*>(A.x64 + gr);
        double2 a = p[0], b = p[1];
        a.x += (double)v[0];
        a.y += (double)v[1];
        b.x += (double)v[2];
        b.y += (double)v[3];
        p[0] = a;
        p[1] = b;
      }
    }
  }

  // Step s, with PH = (s - k0 + 1) % 4: the slots of planes s - 2 .. s + 2 and the patch position
  // class (the first colour's row-A positions on plane s, (C0 + s) & 1 with k0 even) are fixed.
  template <int PH>
  __device__ __forceinline__ bool step(int s, unsigned& phase) const {
    constexpr int SM1 = PH, S0 = (PH + 1) & 3, SP1 = (PH + 2) & 3, SP2 = (PH + 3) & 3, SM2 = SP2;
    constexpr int R0 = (PH + 1) & 1, RP1 = PH & 1;  // r slots of planes s and s + 1
    constexpr int Q = (C0 + 1 + PH) & 1;
    // x and ic of plane s + 2 (up to k1 + 1) and r of plane s + 1 (up to k1) land while this step
    // computes
    stage(s + 2 <= k1 + 1, s + 2, SP2, s + 1 <= k1, s + 1, RP1);
    if (s + 1 <= k1 + 1) load_patch<SP1>();
    if (s <= k1 && valid(s)) {
      const int kw = wrapk(s);
      float ra[4], rb[4];
      lds4(ra, Rs + R0 * RPS + sh.oA - P);
      lds4(rb, Rs + R0 * RPS + sh.oA);
      patch_pass<Q, ZERO, BND>(A, tr, sh, i0, j0, kw, Xs + S0 * XPL, Cs + S0 * XPL, ra, rb, X[S0], C[S0], X[SM1],
                               C[SM1], X[SP1], C[SP1]);
      // the r of this plane's second-colour cells (row A at 1 - Q, 3 - Q; row B at Q, Q + 2)
      RK[PH & 1][0] = ra[1 - Q];
      RK[PH & 1][1] = ra[3 - Q];
      RK[PH & 1][2] = rb[Q];
      RK[PH & 1][3] = rb[Q + 2];
      sts4(Xs + S0 * XPL + sh.oA, &X[S0][0]);
      sts4(Xs + S0 * XPL + sh.oA + P, &X[S0][4]);
      if (threadIdx.x < kRingHalf) {
        const int o = ((C0 + kw) & 1) ? sh.ring_o[1] : sh.ring_o[0];
        ring_cell<ZERO, BND>(A, i0, j0, o, kw, Xs + S0 * XPL, Cs + S0 * XPL, Xs + SM1 * XPL, Cs + SM1 * XPL,
                             Xs + SP1 * XPL, Cs + SP1 * XPL, Rs + R0 * RPS);
      }
    }
    // second colour on plane s - 1: its cells sit at the same patch positions as the first
    // colour's on plane s
    if (s - 1 >= k0 && s - 1 < k1) {
      // kept at the previous step: row A's cells at Q, Q + 2, row B's at 1 - Q, 3 - Q
      const float* k = RK[(PH + 1) & 1];
      float ra[4], rb[4];
      ra[Q] = k[0], ra[Q + 2] = k[1], rb[1 - Q] = k[2], rb[3 - Q] = k[3];
      ra[1 - Q] = ra[3 - Q] = rb[Q] = rb[Q + 2] = 0.f;
      patch_pass<Q, false, BND>(A, tr, sh, i0, j0, wrapk(s - 1), Xs + SM1 * XPL, Cs + SM1 * XPL, ra, rb, X[SM1],
                                C[SM1], X[SM2], C[SM2], X[S0], C[S0]);
      store_plane<SM1>(s - 1);
    }
    return step_end(phase);
  }
};

template <int C0, bool ZERO, bool UPDATE, bool BND>
__global__ void __launch_bounds__(kThreads, 4) k_sweep3d(const __grid_constant__ Sweep3dArgs A,
                                                         const __grid_constant__ Sweep3dMaps M, int lz, int tiles_x,
                                                         int tiles_y, int nzchunk, int tma) {
  extern __shared__ __align__(128) float sm[];
  float* Xs = sm;
  float* Cs = sm + NS * XPL;
  float* Rs = Cs + NS * XPL;
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(sm) + kBarOffset);
  const size_t plane = (size_t)A.nx * A.ny;
  const bool xper = A.bc[0] == FLD_BC_PERIODIC, yper = A.bc[2] == FLD_BC_PERIODIC;
  const bool zper = A.bc[4] == FLD_BC_PERIODIC;
  const int ntile = tiles_x * tiles_y;
  const int items = ntile * nzchunk;
  const float tr[3] = {2.0f * A.ra[0], 2.0f * A.ra[1], 2.0f * A.ra[2]};
  const Share sh = make_share();
  float X[NS][8], C[NS][8], RK[2][4];
  if (threadIdx.x == 0) mbar_init(bar);
  __syncthreads();
  unsigned phase = 0;  // parity of the mbarrier phase the next wait is for
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    // consecutive items are the z-chunks of one tile, then those of the next tile along x: the
    // blocks running together cover a few rows of tiles through the whole depth (measured at 512^3:
    // 0.532 ms per sweep, against 0.586 ms with the tiles of one z-chunk consecutive)
    const int tile = item / nzchunk, zc = item % nzchunk;
    const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
    const int k0 = zc * lz, k1 = min(A.nz, k0 + lz);  // lz even: k0 even
    // TMA boxes do not wrap: tiles whose halo crosses a periodic face stage with cp.async
    const bool use_tma =
        tma && !(xper && (i0 == 0 || i0 + TX == A.nx)) && !(yper && (j0 == 0 || j0 + TY == A.ny));
    const Chunks ch = make_chunks(i0, j0, A, xper, yper);
    const Sweeper<C0, ZERO, UPDATE, BND> W{A, M, tr, Xs, Cs, Rs, bar, sh, ch, i0, j0, k0, k1, zper, use_tma, plane,
                                           X, C, RK};
    cp_wait_all();
    fence_proxy_async();
    __syncthreads();  // the previous item's last reads of the slots are done
    W.stage_prologue();
    if (W.step_end(phase)) return;
    W.template load_patch<0>();
    W.template load_patch<1>();
    const int nsteps = k1 - k0 + 2;  // s = k0 - 1 .. k1
    for (int t = 0; t < nsteps; t += 4) {
      const int s = k0 - 1 + t;
      if (W.template step<0>(s, phase)) return;
      if (t + 1 < nsteps && W.template step<1>(s + 1, phase)) return;
      if (t + 2 < nsteps && W.template step<2>(s + 2, phase)) return;
      if (t + 3 < nsteps && W.template step<3>(s + 3, phase)) return;
    }
  }
}

// ic = 1 / (float)(scale D): the reciprocal coefficient the tiled sweep stages
__global__ void k_dcell32(long long n, double scale, const double* __restrict__ D, float* __restrict__ ic) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ic[i] = __frcp_rn((float)(scale * D[i]));
}

using SweepKernel = void (*)(const Sweep3dArgs, const Sweep3dMaps, int, int, int, int, int);

// the instantiations, indexed by c0 + 2 zero + 4 update + 8 bnd
template <int I>
constexpr SweepKernel kernel_at() {
  return k_sweep3d<I & 1, ((I >> 1) & 1) != 0, ((I >> 2) & 1) != 0, ((I >> 3) & 1) != 0>;
}
const SweepKernel kKernels[16] = {kernel_at<0>(),  kernel_at<1>(),  kernel_at<2>(),  kernel_at<3>(),
                                  kernel_at<4>(),  kernel_at<5>(),  kernel_at<6>(),  kernel_at<7>(),
                                  kernel_at<8>(),  kernel_at<9>(),  kernel_at<10>(), kernel_at<11>(),
                                  kernel_at<12>(), kernel_at<13>(), kernel_at<14>(), kernel_at<15>()};

int g_blocks_per_sm = 0, g_sms = 0;

// cuTensorMapEncodeTiled from the driver (no link against libcuda); nullptr where unavailable, in
// which case every tile stages with cp.async
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// a map of an nx x ny x nz FP32 array whose boxes are 72 x rows x 1 (zero fill beyond the array)
bool encode_box(CUtensorMap& m, const float* base, int nx, int ny, int nz, int rows) {
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)P, (cuuint32_t)rows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool sweep3d_eligible(int nx, int ny, int nz) {
  // nz even: on an odd periodic axis two cells of one colour would meet across the wrap, and the
  // chunks of neighbouring blocks would then read different values for them
  return nx >= TX && nx % TX == 0 && ny >= TY && ny % TY == 0 && nz >= 4 && nz % 2 == 0 &&
         (long long)nx * ny * nz < (1LL << 31);
}

cudaError_t launch_sweep3d(const Sweep3dArgs& a, cudaStream_t s) {
  if (!g_blocks_per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int q = 0; q < 16 && e == cudaSuccess; ++q)
      e = cudaFuncSetAttribute((const void*)kKernels[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    int b = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void*)kKernels[0], kThreads, kSmemBytes);
    if (e != cudaSuccess) return e;
    g_blocks_per_sm = std::max(1, b);
  }
  const int tiles_x = a.nx / TX, tiles_y = a.ny / TY, ntile = tiles_x * tiles_y;
  const int resident = g_blocks_per_sm * g_sms;
  // z-chunk length (even, so that chunks start on even planes): the candidate with the best product
  // of useful planes per staged plane (lz / (lz + 2)) and load balance over the resident blocks
  int lz = a.nz;
  double best = -1.0;
  for (int c : {4, 8, 16, 32, 64, 128, 256, 512}) {
    const int L = std::min(c, a.nz);
    const int nzc = (a.nz + L - 1) / L;
    const long long items = (long long)ntile * nzc;
    const long long waves = (items + resident - 1) / resident;
    const double eff = (double)L / (L + 2) * (double)items / (double)(waves * resident);
    if (eff > best + 1e-9) best = eff, lz = L;
    if (L == a.nz) break;
  }
  const int nzchunk = (a.nz + lz - 1) / lz;
  const int items = ntile * nzchunk;
  const unsigned grid = (unsigned)std::min(items, resident);
  const bool zero = a.xin == nullptr, upd = a.x64 != nullptr;
  bool bnd = false;
  for (int f = 0; f < 6; ++f) bnd = bnd || a.bc[f] != FLD_BC_PERIODIC;
  // TMA box maps of this launch's arrays (FLD_SWEEP3D_TMA=0: cp.async staging for every tile)
  static const bool tma_env = [] {
    const char* v = getenv("FLD_SWEEP3D_TMA");
    return !(v && v[0] == '0');
  }();
  Sweep3dMaps M;
  memset(&M, 0, sizeof(M));
  int tma = 0;
  if (tma_env && encode_fn()) {
    const bool ok = encode_box(M.c, a.dc, a.nx, a.ny, a.nz, RXR) && encode_box(M.r, a.r, a.nx, a.ny, a.nz, RRR) &&
                    (zero || encode_box(M.x, a.xin, a.nx, a.ny, a.nz, RXR));
    tma = ok ? 1 : 0;
  }
  const int q = (a.c0 & 1) + 2 * (zero ? 1 : 0) + 4 * (upd ? 1 : 0) + 8 * (bnd ? 1 : 0);
  note_launch();
  kKernels[q]<<<grid, kThreads, kSmemBytes, s>>>(a, M, lz, tiles_x, tiles_y, nzchunk, tma);
  return cudaGetLastError();
}

cudaError_t launch_dcell32(long long ncell, double scale, const double* D, float* dc, cudaStream_t s) {
  note_launch();
  k_dcell32<<<(unsigned)((ncell + kBlock - 1) / kBlock), kBlock, 0, s>>>(ncell, scale, D, dc);
  return cudaGetLastError();
}

}  // namespace fld

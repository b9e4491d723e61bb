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
// Blocking: a block owns a 64 x 16 tile of the x-y plane and a run of z-planes (a z-chunk), and
// marches through them.  At step s it updates the first colour on plane s (on the tile and one
// cell around it) and the second colour on plane s - 1 (on the tile), so that every value the
// second colour reads is final.  Planes of x and ic with a two-cell halo, and of r with a one-cell
// halo, stay in a ring of shared-memory slots; 16-byte asynchronous copies (cp.async), two per
// thread per staged plane, fetch the planes of the next step while step s computes.  With one step
// of prefetch a block needs 73 KB of shared memory, so three blocks (24 warps) share an SM: more
// warps to hide the shared-memory and reciprocal latencies measured faster than a second step of
// prefetch at two blocks per SM.  A colour pass computes all its cells' values before it stores
// any, so the loads of one cell do not wait behind the store of another.  The
// cells around the tile are computed again by the neighbouring blocks from the same inputs, so the
// sweep reads x from one array and writes another: no block waits for another.  Periodic faces
// read the wrapped halo; Dirichlet, Neumann and linear-extrapolation faces take the interior cell's
// coefficient, as in the FP64 operator.  Everything a thread needs for its cells (staged offsets,
// its chunks to copy, its ring cells) is worked out once per tile, so the loop over planes spends
// its instructions on the cells.
#include <algorithm>

#include "fld_common.cuh"
#include "sweep3d.h"

namespace fld {

namespace {

constexpr int TX = 64, TY = 16;        // tile of a plane
constexpr int P = TX + 8;              // row pitch in shared memory: 4 cells each side (16-byte aligned)
constexpr int RXR = TY + 4;            // rows of a staged x or ic plane (2 halo rows each side)
constexpr int RRR = TY + 2;            // rows of a staged r plane (1 halo row each side)
constexpr int CH = P / 4;              // 16-byte chunks per staged row
constexpr int NXS = 5, NRS = 3;        // ring slots: x and ic planes s-2 .. s+2, r planes s-1 .. s+1
constexpr int XPL = RXR * P, RPL = RRR * P;
constexpr int kThreads = 256;
constexpr int kXChunks = RXR * CH, kRChunks = RRR * CH;  // 360, 324: at most two per thread each
constexpr int kRingHalf = TX + 2 + TY;  // 82 ring cells of each parity around the tile
constexpr size_t kSmemBytes = (size_t)(2 * NXS * XPL + NRS * RPL) * sizeof(float);
static_assert(P % 32 == 8, "the two-row lane mapping is conflict-free for a pitch of 8 mod 32");
static_assert(kRingHalf <= kThreads && kXChunks <= 2 * kThreads && kRChunks <= 2 * kThreads, "thread shares");

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// one hardware reciprocal (rcp.approx, about 1 ulp; 0 for inf): the smoother's arithmetic is FP32
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Staged planes around the cell's plane: x and ic of the plane, below and above; r of the plane.
struct Planes {
  const float* x;
  const float* c;
  const float* xm;
  const float* cm;
  const float* xp;
  const float* cp;
  const float* r;  // indexed like x minus one row
};

// One face of a cell that may lie on a non-periodic face: interior and periodic faces pair the
// cell with the one across (x xa, reciprocal coefficient ia); a Dirichlet face adds the cell's
// own weight to the diagonal only; a Neumann face adds nothing; a linear-extrapolation face
// (ghost 2 x_c - x_m) subtracts w x_m from the sum and w from the diagonal.
__device__ __forceinline__ void face_b(bool inside, int bc, float ic, float ia, float xa, float xm, float ra,
                                       float& a, float& d) {
  if (inside || bc == FLD_BC_PERIODIC) {
    const float w = 2.0f * ra * rcp_fast(ic + ia);
    a = fmaf(w, xa, a);
    d += w;
  } else if (bc == FLD_BC_DIRICHLET) {
    d += ra * rcp_fast(ic);
  } else if (bc == FLD_BC_CONTINUOUS) {
    const float w = ra * rcp_fast(ic);
    a = fmaf(-w, xm, a);
    d -= w;
  }
}

// New value of the cell at staged offset o with right-hand side rv.  NOX: x is zero everywhere
// (the first colour of a sweep from zero).  BND: the cell may lie on a non-periodic face, so the
// face kinds are checked at its global (i, j, k) (wrapped on periodic axes); tr = 2 ra.
template <bool NOX, bool BND>
__device__ __forceinline__ float update(const Sweep3dArgs& A, const float tr[3], const Planes& S, int o, float rv,
                                        int i, int j, int k) {
  const float ic = S.c[o];
  float a = rv;
  float d = 1.0f;
  if (!BND) {
    const float w0 = tr[0] * rcp_fast(ic + S.c[o - 1]), w1 = tr[0] * rcp_fast(ic + S.c[o + 1]);
    const float w2 = tr[1] * rcp_fast(ic + S.c[o - P]), w3 = tr[1] * rcp_fast(ic + S.c[o + P]);
    const float w4 = tr[2] * rcp_fast(ic + S.cm[o]), w5 = tr[2] * rcp_fast(ic + S.cp[o]);
    d += ((w0 + w1) + (w2 + w3)) + (w4 + w5);
    if (!NOX) {
      a = fmaf(w0, S.x[o - 1], a);
      a = fmaf(w1, S.x[o + 1], a);
      a = fmaf(w2, S.x[o - P], a);
      a = fmaf(w3, S.x[o + P], a);
      a = fmaf(w4, S.xm[o], a);
      a = fmaf(w5, S.xp[o], a);
    }
  } else {
    const float z = 0.0f;
    face_b(i > 0, A.bc[0], ic, S.c[o - 1], NOX ? z : S.x[o - 1], NOX ? z : S.x[o + 1], A.ra[0], a, d);
    face_b(i < A.nx - 1, A.bc[1], ic, S.c[o + 1], NOX ? z : S.x[o + 1], NOX ? z : S.x[o - 1], A.ra[0], a, d);
    face_b(j > 0, A.bc[2], ic, S.c[o - P], NOX ? z : S.x[o - P], NOX ? z : S.x[o + P], A.ra[1], a, d);
    face_b(j < A.ny - 1, A.bc[3], ic, S.c[o + P], NOX ? z : S.x[o + P], NOX ? z : S.x[o - P], A.ra[1], a, d);
    face_b(k > 0, A.bc[4], ic, S.cm[o], NOX ? z : S.xm[o], NOX ? z : S.xp[o], A.ra[2], a, d);
    face_b(k < A.nz - 1, A.bc[5], ic, S.cp[o], NOX ? z : S.xp[o], NOX ? z : S.xm[o], A.ra[2], a, d);
  }
  return a * rcp_fast(d);
}

__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool periodic) {
  if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// A thread's share of a tile.
//  - Two tile cells per colour pass: warp w, lanes 0-15 take row 2 (w / 2) and lanes 16-31 row
//    2 (w / 2) + 1, half w % 2 of the row's 32 cells of the colour; the second cell is 8 rows below
//    the first (with the pitch at 8 mod 32 the two half-warps fall on disjoint banks).  The
//    colour's cells of a row alternate parity with the plane: o0 is the first cell's staged offset
//    for parity 0 (column 2m), o0 + 1 for parity 1.
//  - Threads 0..81 each own one ring cell of either parity class (iu + ju even or odd; 82 each:
//    33 in the row below the tile, 33 above, 8 in each side column), so a colour pass on the ring
//    occupies the first three warps only.
//  - Each thread copies up to two 16-byte chunks of a staged x and ic plane and of an r plane:
//    xg / rg are their in-plane source offsets (-1: none), xo their offset in a slot (the same for
//    the x and r chunks of one thread).  A chunk beyond a periodic face wraps; beyond a
//    non-periodic one it is clamped into the grid (the boundary faces do not read it).
// The share is kept small: with three blocks per SM a thread has at most 85 registers.
struct Share {
  int o0, row0;      // the first tile cell (parity-0 column); the second is 8 rows below
  int ring_o[2];     // per parity class: staged offset
  int xg[2], xo[2], rg[2];  // r chunks share the x chunks' slot offsets
};

__device__ __forceinline__ Share make_share(int i0, int j0, const Sweep3dArgs& A, bool xper, bool yper) {
  Share sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  sh.row0 = 2 * (warp >> 1) + (lane >> 4);        // 0 .. 7
  const int m = 16 * (warp & 1) + (lane & 15);     // colour cell within the row, 0 .. 31
  sh.o0 = (2 + sh.row0) * P + 4 + 2 * m;
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
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int tt = t + c * kThreads;
    auto chunk = [&](int q, int jlo, int& g, int& o) {
      const int jj = q / CH, cc = q % CH;
      const int j = wrap_or_clamp(j0 + jlo + jj, A.ny, yper);
      int i = i0 - 4 + 4 * cc;
      i = xper ? (i < 0 ? i + A.nx : (i >= A.nx ? i - A.nx : i)) : min(max(i, 0), A.nx - 4);
      g = j * A.nx + i;
      o = jj * P + 4 * cc;
    };
    if (tt < kXChunks) chunk(tt, -2, sh.xg[c], sh.xo[c]);
    else sh.xg[c] = -1, sh.xo[c] = 0;
    int ro;
    if (tt < kRChunks) chunk(tt, -1, sh.rg[c], ro);
    else sh.rg[c] = -1;
  }
  return sh;
}

// The cells of colour col on the tile of plane k (wrapped kw), and with RING on the ring around it
// (a ring cell outside a non-periodic face is a ghost position: computed, never read).
template <bool NOX, bool RING, bool BND>
__device__ __forceinline__ void colour_pass(const Sweep3dArgs& A, const float tr[3], const Planes& S, float* xs,
                                            const Share& sh, int col, int i0, int j0, int kw) {
  float v[2];
  int oo[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = j0 + sh.row0 + 8 * u;
    const int q = (col + j + kw) & 1;  // the same for both cells (8 rows apart)
    const int o = sh.o0 + 8 * P * u + q;
    const float rv = S.r[o - P];
    oo[u] = o;
    v[u] = update<NOX, BND>(A, tr, S, o, rv, i0 + (sh.o0 - (2 + sh.row0) * P) - 4 + q, j, kw);
  }
  float vr = 0.f;
  int orr = 0;
  if (RING && threadIdx.x < kRingHalf) {
    const bool c = ((col + kw) & 1) != 0;  // the class whose cells have this colour on plane kw
    orr = c ? sh.ring_o[1] : sh.ring_o[0];
    int ri = 0, rj = 0;
    if (BND) {  // the ring cell's global (i, j), wrapped on periodic axes
      const int jj = orr / P, ii = orr - jj * P;
      ri = wrap_or_clamp(i0 + ii - 4, A.nx, A.bc[0] == FLD_BC_PERIODIC);
      rj = wrap_or_clamp(j0 + jj - 2, A.ny, A.bc[2] == FLD_BC_PERIODIC);
    }
    vr = update<NOX, BND>(A, tr, S, orr, S.r[orr - P], ri, rj, kw);
  }
  xs[oo[0]] = v[0];
  xs[oo[1]] = v[1];
  if (RING && threadIdx.x < kRingHalf) xs[orr] = vr;
}

template <bool ZERO, bool UPDATE>
__global__ void __launch_bounds__(kThreads, 3) k_sweep3d(Sweep3dArgs A, int lz, int tiles_x, int tiles_y,
                                                         int nzchunk) {
  extern __shared__ __align__(16) float sm[];
  float* Xs = sm;
  float* Cs = sm + NXS * XPL;
  float* Rs = Cs + NXS * XPL;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const size_t plane = (size_t)nx * ny;
  const bool xper = A.bc[0] == FLD_BC_PERIODIC, yper = A.bc[2] == FLD_BC_PERIODIC;
  const bool zper = A.bc[4] == FLD_BC_PERIODIC;
  const int ntile = tiles_x * tiles_y;
  const int items = ntile * nzchunk;
  const int tid = threadIdx.x;
  const int c1 = A.c0 ^ 1;
  const float tr[3] = {2.0f * A.ra[0], 2.0f * A.ra[1], 2.0f * A.ra[2]};
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    // consecutive items are neighbouring tiles of one z-chunk, so the blocks running together
    // share their halos through L2
    const int tile = item % ntile, zc = item / ntile;
    const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
    const int k0 = zc * lz, k1 = min(nz, k0 + lz);
    const bool tile_bnd = (!xper && (i0 == 0 || i0 + TX == nx)) || (!yper && (j0 == 0 || j0 + TY == ny));
    const Share sh = make_share(i0, j0, A, xper, yper);
    auto valid = [&](int k) { return zper || (k >= 0 && k < nz); };
    auto wrapk = [&](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
    auto load_xc = [&](int k, int slot) {
      if (!valid(k)) return;
      const size_t pb = (size_t)wrapk(k) * plane;
      float* xs = Xs + slot * XPL;
      float* cs = Cs + slot * XPL;
#pragma unroll
      for (int c = 0; c < 2; ++c)
        if (sh.xg[c] >= 0) {
          if (!ZERO) cp16(xs + sh.xo[c], A.xin + pb + sh.xg[c]);
          cp16(cs + sh.xo[c], A.dc + pb + sh.xg[c]);
        }
    };
    auto load_r = [&](int k, int slot) {
      if (!valid(k)) return;
      const size_t pb = (size_t)wrapk(k) * plane;
      float* rs = Rs + slot * RPL;
#pragma unroll
      for (int c = 0; c < 2; ++c)
        if (sh.rg[c] >= 0) cp16(rs + sh.xo[c], A.r + pb + sh.rg[c]);
    };
    auto store = [&](int k, int slot) {
      // the tile of plane k, both colours final: one float4 per thread
      const int row = tid >> 4, q4 = tid & 15;
      const float4 v = *reinterpret_cast<const float4*>(Xs + slot * XPL + (2 + row) * P + 4 + 4 * q4);
      const size_t g = (size_t)wrapk(k) * plane + (size_t)(j0 + row) * nx + i0 + 4 * q4;
      *reinterpret_cast<float4*>(A.xout + g) = v;
      if (UPDATE) {
        double2* p = reinterpret_cast<double2*>(A.x64 + g);
        double2 a = p[0], b = p[1];
        a.x += (double)v.x;
        a.y += (double)v.y;
        b.x += (double)v.z;
        b.y += (double)v.w;
        p[0] = a;
        p[1] = b;
      }
    };
    // slots: plane k0 - 2 + q of x and ic in slot q % NXS, plane k0 - 1 + q of r in slot q % NRS
    cp_wait_all();
    __syncthreads();  // the previous item's last reads of the slots are done
    load_xc(k0 - 2, 0);
    load_xc(k0 - 1, 1);
    load_xc(k0, 2);
    load_r(k0 - 1, 0);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    auto wrap_slot = [](int v, int n) { return v >= n ? v - n : (v < 0 ? v + n : v); };
    int xs0 = 1, rs0 = 0;  // slots of plane s
    for (int s = k0 - 1; s <= k1; ++s) {
      const int xm2 = wrap_slot(xs0 - 2, NXS), xm1 = wrap_slot(xs0 - 1, NXS), xp1 = wrap_slot(xs0 + 1, NXS);
      const int xp2 = wrap_slot(xs0 + 2, NXS);
      const int rm1 = wrap_slot(rs0 - 1, NRS), rp1 = wrap_slot(rs0 + 1, NRS);
      // the planes step s + 1 adds (x and ic of plane s + 2, r of plane s + 1), in flight while
      // step s computes
      if (s + 2 <= k1 + 1) load_xc(s + 2, xp2);
      if (s + 1 <= k1) load_r(s + 1, rp1);
      cp_commit();
      // first colour on plane s, tile and ring (in place: it reads only second-colour cells)
      if (valid(s)) {
        const Planes S{Xs + xs0 * XPL, Cs + xs0 * XPL, Xs + xm1 * XPL, Cs + xm1 * XPL,
                       Xs + xp1 * XPL, Cs + xp1 * XPL, Rs + rs0 * RPL};
        const int kw = wrapk(s);
        if (tile_bnd || (!zper && (s == 0 || s == nz - 1)))
          colour_pass<ZERO, true, true>(A, tr, S, Xs + xs0 * XPL, sh, A.c0, i0, j0, kw);
        else
          colour_pass<ZERO, true, false>(A, tr, S, Xs + xs0 * XPL, sh, A.c0, i0, j0, kw);
      }
      if (s - 2 >= k0) store(s - 2, xm2);
      // second colour on plane s - 1 (tile): its neighbours of the first colour are final.  No
      // barrier is needed between the two passes: a thread's second-colour cell on plane s - 1 and
      // its first-colour cell on plane s share their (i, j), so the one value the second pass reads
      // from this step (the z+ neighbour) and the one the first pass reads from what the second
      // overwrites (the z- neighbour) are the thread's own; everything else either pass reads was
      // final at the last barrier, and the ring's second-colour cells are never written.
      if (s - 1 >= k0 && s - 1 < k1) {
        const Planes S{Xs + xm1 * XPL, Cs + xm1 * XPL, Xs + xm2 * XPL, Cs + xm2 * XPL,
                       Xs + xs0 * XPL, Cs + xs0 * XPL, Rs + rm1 * RPL};
        const int kw = wrapk(s - 1);
        if (tile_bnd || (!zper && (s - 1 == 0 || s - 1 == nz - 1)))
          colour_pass<false, false, true>(A, tr, S, Xs + xm1 * XPL, sh, c1, i0, j0, kw);
        else
          colour_pass<false, false, false>(A, tr, S, Xs + xm1 * XPL, sh, c1, i0, j0, kw);
      }
      cp_wait_all();  // the planes of step s + 1 have landed
      __syncthreads();
      xs0 = xp1;
      rs0 = wrap_slot(rs0 + 1, NRS);
    }
    // the loop ended with xs0 = slot of plane k1 + 1
    store(k1 - 1, wrap_slot(xs0 - 2, NXS));
  }
}

// ic = 1 / (float)(scale D): the reciprocal coefficient the tiled sweep stages
__global__ void k_dcell32(long long n, double scale, const double* __restrict__ D, float* __restrict__ ic) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ic[i] = __frcp_rn((float)(scale * D[i]));
}

int g_blocks_per_sm = 0, g_sms = 0;

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
    const void* ks[4] = {(const void*)k_sweep3d<false, false>, (const void*)k_sweep3d<true, false>,
                         (const void*)k_sweep3d<false, true>, (const void*)k_sweep3d<true, true>};
    for (int q = 0; q < 4 && e == cudaSuccess; ++q)
      e = cudaFuncSetAttribute(ks[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    int b = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep3d<false, false>, kThreads, kSmemBytes);
    if (e != cudaSuccess) return e;
    g_blocks_per_sm = std::max(1, b);
  }
  const int tiles_x = a.nx / TX, tiles_y = a.ny / TY, ntile = tiles_x * tiles_y;
  const int resident = g_blocks_per_sm * g_sms;
  // z-chunk length: the candidate with the best product of useful planes per staged plane
  // (lz / (lz + 2)) and load balance over the resident blocks
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
  note_launch();
  if (zero && upd) k_sweep3d<true, true><<<grid, kThreads, kSmemBytes, s>>>(a, lz, tiles_x, tiles_y, nzchunk);
  else if (zero) k_sweep3d<true, false><<<grid, kThreads, kSmemBytes, s>>>(a, lz, tiles_x, tiles_y, nzchunk);
  else if (upd) k_sweep3d<false, true><<<grid, kThreads, kSmemBytes, s>>>(a, lz, tiles_x, tiles_y, nzchunk);
  else k_sweep3d<false, false><<<grid, kThreads, kSmemBytes, s>>>(a, lz, tiles_x, tiles_y, nzchunk);
  return cudaGetLastError();
}

cudaError_t launch_dcell32(long long ncell, double scale, const double* D, float* dc, cudaStream_t s) {
  note_launch();
  k_dcell32<<<(unsigned)((ncell + kBlock - 1) / kBlock), kBlock, 0, s>>>(ncell, scale, D, dc);
  return cudaGetLastError();
}

}  // namespace fld

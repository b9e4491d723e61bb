// Red-black Gauss-Seidel sweep of the backward-Euler diffusion operator of Sect. 3.4 (Eq.
// discdiff, dt-scaled: (A x)_c = x_c + sum_faces w_f (x_c - x_nb)) on the FP32 finest level of a
// 3-D grid, both colours in one pass over HBM.
//
// The face weights are not read from memory: the kernel stages the cell-centred coefficient
// dc = dt D / dx_0^2 and forms each face's harmonic mean 2 dc_a dc_b / (dc_a + dc_b) (Sect. 3.4)
// on chip, so a sweep moves r, dc and x in and x out (16 bytes per cell) instead of r, three face
// arrays and x (24).
//
// Blocking: a block owns a 64 x 16 tile of the x-y plane and a run of z-planes (a z-chunk), and
// marches through them.  At step s it updates the first colour on plane s (on the tile and one
// cell around it) and the second colour on plane s - 1 (on the tile), so that every value the
// second colour reads is final.  Planes of x and dc with a two-cell halo, and of r with a one-cell
// halo, stay in a ring of shared-memory slots; cp.async fetches the planes of step s + 1 while
// step s computes.  The cells around the tile are computed again by the neighbouring blocks from
// the same inputs, so the sweep reads x from one array and writes another: no block waits for
// another.  Periodic faces read the wrapped halo; Dirichlet, Neumann and linear-extrapolation
// faces take the interior cell's coefficient, as in the FP64 operator.
#include <algorithm>

#include "fld_common.cuh"
#include "sweep3d.h"

namespace fld {

namespace {

constexpr int TX = 64, TY = 16;        // tile of a plane
constexpr int P = TX + 8;              // row pitch in shared memory: 4 cells each side (16-byte chunks)
constexpr int RXR = TY + 4;            // rows of a staged x or dc plane (2 halo rows each side)
constexpr int RRR = TY + 2;            // rows of a staged r plane (1 halo row each side)
constexpr int CH = P / 4;              // 16-byte chunks per staged row
constexpr int NXS = 5, NRS = 3;        // ring slots: x and dc planes s-2 .. s+2, r planes s-1 .. s+1
constexpr int XPL = RXR * P, RPL = RRR * P;
constexpr int kThreads = 256;
constexpr int kXChunks = RXR * CH, kRChunks = RRR * CH;  // 360, 324: two per thread each
constexpr size_t kSmemBytes = (size_t)(2 * NXS * XPL + NRS * RPL) * sizeof(float);
static_assert(kXChunks <= 2 * kThreads && kRChunks <= 2 * kThreads, "two chunks per thread");
static_assert(P % 32 == 8, "the two-row lane mapping is conflict-free for a pitch of 8 mod 32");

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 2 a b / (a + b), 0 where both vanish
__device__ __forceinline__ float hmean(float a, float b) {
  const float s = a + b;
  return s > 0.0f ? 2.0f * a * __fdividef(b, s) : 0.0f;
}

// One face of a cell next to a non-periodic boundary or away from it: the interior and periodic
// faces pair the cell with the one across (xa, coefficient da); a Dirichlet face adds the cell's
// own weight to the diagonal only; a Neumann face adds nothing; a linear-extrapolation face
// (ghost 2 x_c - x_m) subtracts w x_m from the sum and w from the diagonal.
__device__ __forceinline__ void face_b(bool inside, int bc, float dcen, float da, float xa, float xm, float ra,
                                       float& a, float& d) {
  if (inside || bc == FLD_BC_PERIODIC) {
    const float w = hmean(dcen, da) * ra;
    a = fmaf(w, xa, a);
    d += w;
  } else if (bc == FLD_BC_DIRICHLET) {
    d += dcen * ra;
  } else if (bc == FLD_BC_CONTINUOUS) {
    const float w = dcen * ra;
    a = fmaf(-w, xm, a);
    d -= w;
  }
}

struct Planes {
  const float* x;  // slot of the cell's plane
  const float* d;
  const float* xm; // slots of the planes below and above
  const float* dm;
  const float* xp;
  const float* dp;
  const float* r;  // r slot, indexed like x minus one row
};

// New value of the cell at staged offset o (row jj, column ii of the slot), global (i, j, k).
// NOX: x is zero everywhere (the first colour of a sweep from zero).  BND: the cell may lie on a
// non-periodic face, so the face kinds are checked; i, j must then be wrapped on periodic axes.
template <bool NOX, bool BND>
__device__ __forceinline__ float update(const Sweep3dArgs& A, const Planes& S, int o, int i, int j, int k) {
  const float dcen = S.d[o];
  float a = S.r[o - P];
  float d = 1.0f;
  if (!BND) {
    const float w0 = hmean(dcen, S.d[o - 1]) * A.ra[0], w1 = hmean(dcen, S.d[o + 1]) * A.ra[0];
    const float w2 = hmean(dcen, S.d[o - P]) * A.ra[1], w3 = hmean(dcen, S.d[o + P]) * A.ra[1];
    const float w4 = hmean(dcen, S.dm[o]) * A.ra[2], w5 = hmean(dcen, S.dp[o]) * A.ra[2];
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
    face_b(i > 0, A.bc[0], dcen, S.d[o - 1], NOX ? z : S.x[o - 1], NOX ? z : S.x[o + 1], A.ra[0], a, d);
    face_b(i < A.nx - 1, A.bc[1], dcen, S.d[o + 1], NOX ? z : S.x[o + 1], NOX ? z : S.x[o - 1], A.ra[0], a, d);
    face_b(j > 0, A.bc[2], dcen, S.d[o - P], NOX ? z : S.x[o - P], NOX ? z : S.x[o + P], A.ra[1], a, d);
    face_b(j < A.ny - 1, A.bc[3], dcen, S.d[o + P], NOX ? z : S.x[o + P], NOX ? z : S.x[o - P], A.ra[1], a, d);
    face_b(k > 0, A.bc[4], dcen, S.dm[o], NOX ? z : S.xm[o], NOX ? z : S.xp[o], A.ra[2], a, d);
    face_b(k < A.nz - 1, A.bc[5], dcen, S.dp[o], NOX ? z : S.xp[o], NOX ? z : S.xm[o], A.ra[2], a, d);
  }
  return __fdividef(a, d);
}

__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool periodic) {
  if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// Cells of one colour on the tile of one plane, and (RING) on the ring of cells around it.  A warp
// takes two rows of 32 cells, lanes 0-15 the colour's 16 cells of the first row and lanes 16-31
// those of the second: with the pitch at 8 mod 32 the two halves fall on disjoint banks.
template <bool NOX, bool RING>
__device__ __forceinline__ void colour_pass(const Sweep3dArgs& A, const Planes& S, float* xs, int col, int i0, int j0,
                                            int k, bool bnd) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kw = k < 0 ? k + A.nz : (k >= A.nz ? k - A.nz : k);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int task = warp + 8 * u;                  // 16 tasks: 8 row pairs x 2 halves of 32 cells
    const int row = 2 * (task >> 1) + (lane >> 4);  // 0 .. 15
    const int m = 16 * (task & 1) + (lane & 15);    // colour cell within the row, 0 .. 31
    const int j = j0 + row;
    const int q = (col + j + kw) & 1;
    const int ii = 4 + 2 * m + q;
    const int o = (2 + row) * P + ii;
    const float v = bnd ? update<NOX, true>(A, S, o, i0 + ii - 4, j, kw) : update<NOX, false>(A, S, o, 0, 0, 0);
    xs[o] = v;
  }
  if (RING) {
    // 164 cells around the tile: rows j0-1 and j0+16 (66 cells each), columns i0-1 and i0+64
    const int t = threadIdx.x;
    if (t < 164) {
      int ii, jj;
      if (t < 66) ii = 3 + t, jj = 1;
      else if (t < 132) ii = 3 + (t - 66), jj = RXR - 2;
      else if (t < 148) ii = 3, jj = 2 + (t - 132);
      else ii = P - 4, jj = 2 + (t - 148);
      const int i = wrap_or_clamp(i0 + ii - 4, A.nx, A.bc[0] == FLD_BC_PERIODIC);
      const int j = wrap_or_clamp(j0 + jj - 2, A.ny, A.bc[2] == FLD_BC_PERIODIC);
      const int iu = i0 + ii - 4, ju = j0 + jj - 2;  // unwrapped: the parity of the staged position
      if (((iu + ju + kw) & 1) == col) {
        const int o = jj * P + ii;
        // a ring cell outside a non-periodic face is a ghost position: computed, never read
        const float v = bnd ? update<NOX, true>(A, S, o, i, j, kw) : update<NOX, false>(A, S, o, 0, 0, 0);
        xs[o] = v;
      }
    }
  }
}

template <bool ZERO, bool UPDATE>
__global__ void __launch_bounds__(kThreads, 3) k_sweep3d(Sweep3dArgs A, int lz, int tiles_x, int tiles_y,
                                                         int nzchunk) {
  extern __shared__ __align__(16) float sm[];
  float* Xs = sm;
  float* Ds = sm + NXS * XPL;
  float* Rs = Ds + NXS * XPL;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const size_t plane = (size_t)nx * ny;
  const bool xper = A.bc[0] == FLD_BC_PERIODIC, yper = A.bc[2] == FLD_BC_PERIODIC;
  const bool zper = A.bc[4] == FLD_BC_PERIODIC;
  const int ntile = tiles_x * tiles_y;
  const int items = ntile * nzchunk;
  const int tid = threadIdx.x;
  const int c1 = A.c0 ^ 1;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    // consecutive items are neighbouring tiles of one z-chunk, so the blocks running together
    // share their halos through L2
    const int tile = item % ntile, zc = item / ntile;
    const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
    const int k0 = zc * lz, k1 = min(nz, k0 + lz);
    const bool tile_bnd = (!xper && (i0 == 0 || i0 + TX == nx)) || (!yper && (j0 == 0 || j0 + TY == ny));
    // per-thread 16-byte chunks of a staged plane: in-plane global offset and slot offset
    int xg[2], xo[2], rg[2], ro[2];
    bool xok[2], rok[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int t = tid + c * kThreads;
      xok[c] = t < kXChunks;
      rok[c] = t < kRChunks;
      const int tx = xok[c] ? t : 0, tr = rok[c] ? t : 0;
      {
        const int jj = tx / CH, cc = tx % CH;
        const int j = wrap_or_clamp(j0 - 2 + jj, ny, yper);
        int i = i0 - 4 + 4 * cc;
        i = xper ? (i < 0 ? i + nx : (i >= nx ? i - nx : i)) : min(max(i, 0), nx - 4);
        xg[c] = j * nx + i;
        xo[c] = jj * P + 4 * cc;
      }
      {
        const int jj = tr / CH, cc = tr % CH;
        const int j = wrap_or_clamp(j0 - 1 + jj, ny, yper);
        int i = i0 - 4 + 4 * cc;
        i = xper ? (i < 0 ? i + nx : (i >= nx ? i - nx : i)) : min(max(i, 0), nx - 4);
        rg[c] = j * nx + i;
        ro[c] = jj * P + 4 * cc;
      }
    }
    auto valid = [&](int k) { return zper || (k >= 0 && k < nz); };
    auto wrapk = [&](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
    auto xslot = [&](int k) { return (k - k0 + 2) % NXS; };
    auto rslot = [&](int k) { return (k - k0 + 1) % NRS; };
    auto load_xd = [&](int k) {
      if (!valid(k)) return;
      const size_t pb = (size_t)wrapk(k) * plane;
      const int s = xslot(k) * XPL;
#pragma unroll
      for (int c = 0; c < 2; ++c)
        if (xok[c]) {
          if (!ZERO) cp16(Xs + s + xo[c], A.xin + pb + xg[c]);
          cp16(Ds + s + xo[c], A.dc + pb + xg[c]);
        }
    };
    auto load_r = [&](int k) {
      if (!valid(k)) return;
      const size_t pb = (size_t)wrapk(k) * plane;
      const int s = rslot(k) * RPL;
#pragma unroll
      for (int c = 0; c < 2; ++c)
        if (rok[c]) cp16(Rs + s + ro[c], A.r + pb + rg[c]);
    };
    auto planes = [&](int k) {
      Planes S;
      S.x = Xs + xslot(k) * XPL;
      S.d = Ds + xslot(k) * XPL;
      S.xm = Xs + xslot(k - 1) * XPL;
      S.dm = Ds + xslot(k - 1) * XPL;
      S.xp = Xs + xslot(k + 1) * XPL;
      S.dp = Ds + xslot(k + 1) * XPL;
      S.r = Rs + rslot(k) * RPL;
      return S;
    };
    auto store = [&](int k) {
      // the tile of plane k, both colours final: one float4 per thread
      const int row = tid >> 4, q4 = tid & 15;
      const float4 v = *reinterpret_cast<const float4*>(Xs + xslot(k) * XPL + (2 + row) * P + 4 + 4 * q4);
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
    __syncthreads();  // the previous item's last reads of the slots are done
    load_xd(k0 - 2);
    load_xd(k0 - 1);
    load_xd(k0);
    load_r(k0 - 1);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    for (int s = k0 - 1; s <= k1; ++s) {
      if (s + 2 <= k1 + 1) load_xd(s + 2);
      if (s + 1 <= k1) load_r(s + 1);
      cp_commit();
      // first colour on plane s, tile and ring (in place: it reads only second-colour cells)
      if (valid(s)) {
        const Planes S = planes(s);
        const bool bnd = tile_bnd || (!zper && (s == 0 || s == nz - 1));
        colour_pass<ZERO, true>(A, S, Xs + xslot(s) * XPL, A.c0, i0, j0, s, bnd);
      }
      if (s - 2 >= k0) store(s - 2);
      __syncthreads();
      // second colour on plane s - 1 (tile): its neighbours of the first colour are final
      if (s - 1 >= k0 && s - 1 < k1) {
        const Planes S = planes(s - 1);
        const bool bnd = tile_bnd || (!zper && (s - 1 == 0 || s - 1 == nz - 1));
        colour_pass<false, false>(A, S, Xs + xslot(s - 1) * XPL, c1, i0, j0, s - 1, bnd);
      }
      cp_wait_all();
      __syncthreads();
    }
    store(k1 - 1);
  }
}

__global__ void k_dcell32(long long n, double scale, const double* __restrict__ D, float* __restrict__ dc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dc[i] = (float)(scale * D[i]);
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
  for (int c : {8, 16, 32, 64, 128, 256, 512}) {
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

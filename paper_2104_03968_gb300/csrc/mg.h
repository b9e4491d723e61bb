// Geometric multigrid for the backward-Euler FLD diffusion operator (host side).
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <string>
#include <vector>

#include "fld_common.cuh"

namespace fld {

// One 256-byte-aligned device allocation carved into sub-buffers.
class DeviceArena {
 public:
  DeviceArena() = default;
  ~DeviceArena();
  DeviceArena(const DeviceArena&) = delete;
  DeviceArena& operator=(const DeviceArena&) = delete;
  cudaError_t reserve(size_t bytes);
  void* take(size_t bytes);
  void release();
  size_t capacity() const { return cap_; }

 private:
  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0;
};

template <class T>
struct LevelDev {
  int n[3];
  int ndim;
  int bc[6];
  const T* w[3];
};

struct SolveStats {
  int cycles = 0;
  double relres = 0.0;
  int status = FLD_OK;
  int nu1 = 0, nu2 = 0, nu1_coarse = 0, nu2_coarse = 0;
};

// Operator A = I + dt * (-div D grad) on one grid, solved by an outer FP64 defect-correction
// loop around V-cycles in precision T (double: the plain FP64 solver; float: the mixed form).
class Multigrid {
 public:
  Multigrid() = default;
  ~Multigrid();
  Multigrid(const Multigrid&) = delete;
  Multigrid& operator=(const Multigrid&) = delete;

  // (Re)build the level hierarchy for grid g and precision; keeps buffers when unchanged.
  cudaError_t configure(const GridDev& g, int precision);
  // Face weights, diagonals and coarse operators from the cell-centred D (D_cell[a] for the faces
  // of axis a); rhs from E_old.
  // rtol: the solve's tolerance (the mixed solver sets up in double-float when rtol >= 1e-10).
  cudaError_t setup(double dt, const double* const D_cell[3], const double* E_old, double rtol, unsigned* status,
                    cudaStream_t s);
  // Outer iterations until ||b - A x||/||b|| <= rtol or max_cycles cycles; writes E_new.  With
  // fmg_start the first cycle is a full-multigrid cycle, the others V-cycles.  nu1 = nu2 = 0: the
  // sweep counts -- one pair for the finest level, one for the coarser levels -- are autotuned on
  // the first solve of this configuration (per rtol and start; the candidates run on a scratch
  // iterate, the fastest converged set is kept); otherwise every level uses (nu1, nu2).
  cudaError_t solve(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                    bool fmg_start, SolveStats* st, cudaStream_t s);

  // The result of a graph-driven solve, written by the graph's last kernel into pinned host memory:
  // valid once the stream has passed the solve.  kernels: kernels the solve's graph ran.
  struct SolveOut {
    int cycles, status;
    double relres;
    unsigned long long kernels;
  };
  struct SolveDev;  // the graph-driven solve's device state (mg.cu)
  // True when solve_async applies: per-kernel tracing (whose events are host bookkeeping) is off.
  bool async_ready() const;
  // The solve of `solve` with no host synchronisation per cycle: the whole outer loop (residuals,
  // the convergence decision, V-cycles) is one CUDA graph whose conditional nodes the device steers,
  // built on the first call for a configuration and these pointers, then replayed (the first solve
  // of a configuration with autotuned sweep counts times its candidates first, which synchronises).
  // *out receives the pinned result, valid after the stream passes the solve; st receives the sweep
  // counts.
  cudaError_t solve_async(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                          bool fmg_start, SolveStats* st, const SolveOut** out, cudaStream_t s);

  int levels() const { return (int)dims_.size(); }
  const GridDev& grid() const { return g_; }

 private:
  template <class T>
  cudaError_t setup_t(double dt, const double* const D_cell[3], const double* E_old, double rtol, cudaStream_t s);
  // the FP64 finest-level operator (weights, diagonal, rhs, ||b||) for the exact FP64 residual
  template <class T>
  cudaError_t fp64_operator(cudaStream_t s);
  template <class T>
  cudaError_t solve_t(const double* E_old, double* E_new, double rtol, int max_cycles, int nu1, int nu2,
                      bool fmg_start, SolveStats* st, cudaStream_t s);
  template <class T>
  cudaError_t vcycle(int l, int nu1, int nu2, double* x64, cudaStream_t s, bool zero_init);
  template <class T>
  cudaError_t vcycle_direct(int l, int nu1, int nu2, double* x64, cudaStream_t s, bool zero_init);
  // V-cycles of the levels below the wavefront ones replay as CUDA graphs (captured once per
  // (level, nu1, nu2, zero start) on a private stream): they are many small launches
  template <class T>
  cudaError_t vcycle_graph(int l, int nu1, int nu2, cudaStream_t s, bool zero_init);
  void drop_graphs();
  template <class T>
  cudaError_t fmg(int nu1, int nu2, double* x64, cudaStream_t s);

  // nu = (finest pre, finest post, coarser pre, coarser post)
  cudaError_t autotune(const double* E_old, double rtol, int max_cycles, bool fmg_start, int nu[4], cudaStream_t s);

  GridDev g_{};
  int precision_ = -1;
  // sweep-count tuning per (rtol, start): each candidate's solve time summed over the first
  // kTuneRounds solves of the configuration (infinite once it failed to converge), then settled
  static constexpr int kTuneCands = 12, kTuneRounds = 3;
  struct Tuned {
    double rtol;
    bool fmg;
    int rounds, best;
    float sum[kTuneCands];
  };
  std::vector<Tuned> tuned_;
  int nuc1_ = 2, nuc2_ = 2;                   // sweep counts of the levels below the finest
  struct GraphEntry {
    int l, nu1, nu2, zero;
    cudaGraphExec_t exec;
    unsigned long long kernels;  // kernel launches captured in the graph
  };
  std::vector<GraphEntry> graphs_;
  cudaStream_t cap_stream_ = nullptr;
  bool capturing_ = false;
  bool graphs_ok_ = true;
  double* tune_x_ = nullptr;                  // scratch iterate of the autotuning solves
  size_t tune_cap_ = 0;
  bool configured_ = false;
  std::vector<std::array<int, 3>> dims_;
  DeviceArena arena_;
  // FP64 outer operator and iterate
  double* w64_[3] = {nullptr, nullptr, nullptr};
  double* b64_ = nullptr;
  double* diag64_ = nullptr;
  double* partials_ = nullptr;
  double* scal_ = nullptr;      // [0] = ||r||^2, [1] = ||b||^2, [2] = update error measure (scaled)
  double* host_scal_ = nullptr; // pinned mirror ([7] holds the wavefront error word)
  // mixed solver: low parts of the finest FP32 weights, the diagonal as hi + lo, and the low part
  // of the outer residual (its high part is the V-cycle's right-hand side)
  float* w32lo_[3] = {nullptr, nullptr, nullptr};
  float* dhi_ = nullptr;
  float* dlo_ = nullptr;
  float* rlo_ = nullptr;
  // double-float setup (mixed solver, rtol >= 1e-10): the out-of-window flag and the setup inputs
  // kept for an FP64 redo
  unsigned* df_flag_ = nullptr;
  bool df_mode_ = false;
  bool fp64_op_ = false;
  double dt_ = 0.0;
  const double* D_ax_[3] = {nullptr, nullptr, nullptr};
  const double* E_old_ = nullptr;
  // Wavefront smoothing (large 3-D levels): per level, the (half-sweep, plane) of each group of
  // `nchunk` tickets in ticket order; control words [0] error, [1] ticket, [2..] finished chunks
  // per (half-sweep, plane).
  struct WaveLevel {
    int* order = nullptr;  // 2 ints (h, plane) per group
    int nchunk = 0, rows = 0;
  };
  std::vector<WaveLevel> wave_;
  unsigned* wave_ctl_ = nullptr;
  int wave_blocks_[2] = {0, 0};  // resident blocks of the sweep kernel (float, double)
  cudaError_t configure_wave();
  bool rows_ok(int l) const;
  template <class T>
  cudaError_t wave_sweep(int l, bool zero, int c0, double* x64, cudaStream_t s);
  // Graph-driven solve: device state (arena), pinned result, body capture streams and the graph of
  // the last configuration with its key.
  SolveDev* sd_ = nullptr;
  SolveOut* out_h_ = nullptr;
  cudaStream_t body_s_[2] = {nullptr, nullptr};
  struct SolveKey {
    const double* E_old;
    double* E_new;
    const double* D[3];
    double dt, rtol;
    int max_cycles, nu[4], fmg, df, fp64op, prec;
    bool operator==(const SolveKey& o) const {
      return E_old == o.E_old && E_new == o.E_new && D[0] == o.D[0] && D[1] == o.D[1] && D[2] == o.D[2] &&
             dt == o.dt && rtol == o.rtol && max_cycles == o.max_cycles && nu[0] == o.nu[0] && nu[1] == o.nu[1] &&
             nu[2] == o.nu[2] && nu[3] == o.nu[3] && fmg == o.fmg && df == o.df && fp64op == o.fp64op &&
             prec == o.prec;
    }
  };
  SolveKey skey_{};
  cudaGraphExec_t sexec_ = nullptr;
  unsigned long long pre_kernels_ = 0;  // kernels of the graph outside its loop
  template <class T>
  cudaError_t build_solve_graph(const SolveKey& k, cudaStream_t s);
  // Tiled sweep of the mixed solver's finest 3-D level (sweep3d.cu): each cell's 1 / (dt D / dx_0^2)
  // in FP32, and whether this solve uses it (scalar D, eligible shape).  The sweep reads the iterate
  // from lv_[0].x and writes lv_[0].tmp, then the two are swapped.
  float* dc32_ = nullptr;
  bool tiled_ = false;
  template <class T>
  cudaError_t tiled_sweep(bool zero, int c0, double* x64, cudaStream_t s);
  int nparts_ = 0;
  // inner levels (type-erased; cast to T per precision)
  struct LevelBuf {
    void* w[3];
    void* invd;
    void* x;
    void* r;
    void* tmp;
  };
  std::vector<LevelBuf> lv_;
};

}  // namespace fld

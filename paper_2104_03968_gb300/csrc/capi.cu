// C ABI of the GB300 FLD library: argument validation, context-owned buffers and the
// composition of the kernels into the calls declared in include/fld.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batched.h"
#include "columns.h"
#include "kernels.h"
#include "mg.h"
#include "sweep3d.h"
#include "trace.h"

using namespace fld;

// slabs (equal cell ranges) of the host-buffer step: the copies of slab i overlap the coefficient or
// exchange kernel of the slabs before it
constexpr int kHostSlabs = 8;

struct fld_ctx {
  int device = 0;
  std::string err;
  Multigrid mg;
  double* D = nullptr;
  double* kappa = nullptr;
  size_t cap = 0;  // cells of D and kappa
  unsigned* d_status = nullptr;  // [0] status bits
  int* d_info = nullptr;         // [0] max iterations, [1] bisections
  int* h_info = nullptr;         // pinned: [0..1] info, [2] status
  BatchedSolver* batched = nullptr;
  double* geom = nullptr;  // per-cell geometry of the 1-D column calls
  size_t geom_cap = 0;
  double* mid = nullptr;   // midpoint IMEX: E^n, eps^n and the half-step E (3 x cells)
  size_t mid_cap = 0;
  // fld_step_host: device copies of rho, eps and E (3 x cells), the copy stream and its events
  double* stage = nullptr;
  size_t stage_cap = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev[2 * kHostSlabs + 3] = {};
};

namespace {

fld_status fail(fld_ctx* ctx, fld_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return st;
}

fld_status cuda_fail(fld_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, FLD_ERR_CUDA, "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
}

// RAII: make the context's device current for the duration of a call
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

fld_status check_grid(fld_ctx* ctx, const fld_grid* g) {
  if (!g) return fail(ctx, FLD_ERR_INVALID_ARG, "grid is NULL");
  if (g->ndim < 1 || g->ndim > 3) return fail(ctx, FLD_ERR_INVALID_ARG, "ndim must be 1, 2 or 3 (got %d)", g->ndim);
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1) return fail(ctx, FLD_ERR_INVALID_ARG, "n[%d] must be >= 1", a);
    if (a >= g->ndim && g->n[a] != 1) return fail(ctx, FLD_ERR_INVALID_ARG, "n[%d] must be 1 for ndim=%d", a, g->ndim);
    if (a < g->ndim) {
      if (!(g->dx[a] > 0) || !std::isfinite(g->dx[a])) return fail(ctx, FLD_ERR_INVALID_ARG, "dx[%d] must be > 0", a);
      for (int s = 0; s < 2; ++s) {
        int bc = g->bc[2 * a + s];
        if (bc < FLD_BC_PERIODIC || bc > FLD_BC_CONTINUOUS)
          return fail(ctx, FLD_ERR_INVALID_ARG, "bc[%d] = %d is not a boundary condition", 2 * a + s, bc);
        if (bc != FLD_BC_PERIODIC && g->n[a] < 2)
          return fail(ctx, FLD_ERR_INVALID_ARG, "axis %d needs n >= 2 for a non-periodic boundary", a);
        if (!std::isfinite(g->bc_val[2 * a + s])) return fail(ctx, FLD_ERR_INVALID_ARG, "bc_val[%d] not finite", 2 * a + s);
      }
      if ((g->bc[2 * a] == FLD_BC_PERIODIC) != (g->bc[2 * a + 1] == FLD_BC_PERIODIC))
        return fail(ctx, FLD_ERR_INVALID_ARG, "axis %d: periodic must be set on both faces", a);
    }
  }
  long long n = (long long)g->n[0] * g->n[1] * g->n[2];
  if (n > (1LL << 34)) return fail(ctx, FLD_ERR_INVALID_ARG, "grid too large (%lld cells)", n);
  return FLD_OK;
}

fld_status check_params(fld_ctx* ctx, const fld_params* p, bool solver, bool columns = false) {
  if (!p) return fail(ctx, FLD_ERR_INVALID_ARG, "params is NULL");
  if (p->cak && !columns) return fail(ctx, FLD_ERR_INVALID_ARG, "the CAK line opacity applies to column calls only");
  if (!cak_valid(p->cak))
    return fail(ctx, FLD_ERR_INVALID_ARG, "CAK: v, kappa_e_Qbar > 0, r_star > 0, 0 <= alpha < 1, x_in <= x_out");
  if (!(p->c > 0) || !(p->a_rad > 0) || !(p->gamma > 1) || !(p->gas_R > 0))
    return fail(ctx, FLD_ERR_INVALID_ARG, "c, a_rad, gas_R must be > 0 and gamma > 1");
  if (p->start != FLD_START_FMG && p->start != FLD_START_VCYCLE)
    return fail(ctx, FLD_ERR_INVALID_ARG, "unknown start %d", p->start);
  if (p->limiter < FLD_LIMITER_LP || p->limiter > FLD_LIMITER_MINERBO)
    return fail(ctx, FLD_ERR_INVALID_ARG, "unknown limiter %d", p->limiter);
  if (p->opacity < FLD_OPACITY_CONST || p->opacity > FLD_OPACITY_TABLE)
    return fail(ctx, FLD_ERR_INVALID_ARG, "unknown opacity model %d", p->opacity);
  if (p->opacity != FLD_OPACITY_TABLE && !(p->kappa0 > 0)) return fail(ctx, FLD_ERR_INVALID_ARG, "kappa0 must be > 0");
  if (p->opacity == FLD_OPACITY_TABLE) {
    if (!p->table || p->tn[0] < 2 || p->tn[1] < 2 || !(p->thi[0] > p->tlo[0]) || !(p->thi[1] > p->tlo[1]))
      return fail(ctx, FLD_ERR_INVALID_ARG, "opacity table needs a device pointer, tn >= 2 and thi > tlo");
  }
  if (solver) {
    if (p->precision != FLD_PREC_FP64 && p->precision != FLD_PREC_MIXED)
      return fail(ctx, FLD_ERR_INVALID_ARG, "unknown precision %d", p->precision);
    if (!(p->rtol > 0) || p->rtol >= 1) return fail(ctx, FLD_ERR_INVALID_ARG, "rtol must be in (0, 1)");
    if (p->max_cycles < 0 || p->nu1 < 0 || p->nu2 < 0 || p->nu1 > 16 || p->nu2 > 16)
      return fail(ctx, FLD_ERR_INVALID_ARG, "max_cycles, nu1, nu2 out of range");
    if (p->order != FLD_ORDER_DIFFUSE_THEN_EXCHANGE && p->order != FLD_ORDER_EXCHANGE_THEN_DIFFUSE &&
        p->order != FLD_ORDER_IMEX_MIDPOINT)
      return fail(ctx, FLD_ERR_INVALID_ARG, "unknown order %d", p->order);
  }
  if (p->exch_maxit < 0) return fail(ctx, FLD_ERR_INVALID_ARG, "exch_maxit must be >= 0");
  return FLD_OK;
}

GridDev to_dev(const fld_grid* g) {
  GridDev d{};
  d.ndim = g->ndim;
  for (int a = 0; a < 3; ++a) {
    d.n[a] = g->n[a];
    d.dx[a] = a < g->ndim ? g->dx[a] : 1.0;
    d.inv_dx2[a] = 1.0 / (d.dx[a] * d.dx[a]);
  }
  for (int f = 0; f < 6; ++f) {
    d.bc[f] = (f / 2) < g->ndim ? g->bc[f] : FLD_BC_PERIODIC;
    d.bc_val[f] = (f / 2) < g->ndim ? g->bc_val[f] : 0.0;
  }
  d.ncell = (long long)g->n[0] * g->n[1] * g->n[2];
  return d;
}

Opacity to_opacity(const fld_params* p) { return make_opacity(*p); }

ExchangeParams to_exchange(const fld_params* p, double dt) {
  return make_exchange(p->c, p->a_rad, p->gamma, p->gas_R, dt, p->exch_maxit > 0 ? p->exch_maxit : 100,
                       p->precision == FLD_PREC_FP64);
}

fld_status ensure_scratch(fld_ctx* ctx, long long ncell) {
  if ((size_t)ncell <= ctx->cap) return FLD_OK;
  cudaFree(ctx->D);
  cudaFree(ctx->kappa);
  ctx->D = ctx->kappa = nullptr;
  ctx->cap = 0;
  cudaError_t e = cudaMalloc(&ctx->D, ncell * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->kappa, ncell * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation");
  ctx->cap = ncell;
  return FLD_OK;
}

fld_status ensure_mid(fld_ctx* ctx, long long ncell) {
  if ((size_t)ncell <= ctx->mid_cap) return FLD_OK;
  cudaFree(ctx->mid);
  ctx->mid = nullptr;
  ctx->mid_cap = 0;
  cudaError_t e = cudaMalloc(&ctx->mid, 3 * ncell * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "midpoint scratch allocation");
  ctx->mid_cap = ncell;
  return FLD_OK;
}

fld_status ensure_stage(fld_ctx* ctx, long long ncell) {
  if (!ctx->copy_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 * kHostSlabs + 3 && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&ctx->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream creation");
  }
  if ((size_t)ncell <= ctx->stage_cap) return FLD_OK;
  cudaFree(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_cap = 0;
  cudaError_t e = cudaMalloc(&ctx->stage, 3 * ncell * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host-step staging allocation");
  ctx->stage_cap = ncell;
  return FLD_OK;
}

fld_status reset_status(fld_ctx* ctx, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_info, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status reset");
  return FLD_OK;
}

// copy the device status/info to the host (synchronises)
fld_status read_status(fld_ctx* ctx, cudaStream_t s, unsigned* status, int* iters, int* bisect) {
  cudaError_t e = cudaMemcpyAsync(ctx->h_info, ctx->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_info + 2, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status read-back");
  if (iters) *iters = ctx->h_info[0];
  if (bisect) *bisect = ctx->h_info[1];
  if (status) *status = (unsigned)ctx->h_info[2];
  return FLD_OK;
}

// The outcome of a diffusion solve: known at once (the host-driven solve, which synchronises per
// cycle: the first solve of a configuration, which autotunes, or a traced one), or pending in pinned
// memory that the graph-driven solve writes when the stream passes it.
struct DiffuseResult {
  SolveStats ss;
  const Multigrid::SolveOut* out = nullptr;
};

// Completes a pending result once the stream has passed the solve, and counts the kernels its
// graph's loop ran.
void resolve(DiffuseResult& r) {
  if (!r.out) return;
  r.ss.cycles = r.out->cycles;
  r.ss.status = r.out->status;
  r.ss.relres = r.out->relres;
  note_launch(r.out->kernels);
  r.out = nullptr;
}

void fill_info(fld_info* inf, const SolveStats& ss, const int* h_info) {
  memset(inf, 0, sizeof(*inf));
  inf->cycles = ss.cycles;
  inf->rel_residual = ss.relres;
  inf->status = ss.status;
  inf->nu1 = ss.nu1;
  inf->nu2 = ss.nu2;
  inf->nu1_coarse = ss.nu1_coarse;
  inf->nu2_coarse = ss.nu2_coarse;
  if (h_info) {
    inf->exch_max_iters = h_info[0];
    inf->bisection_fallbacks = h_info[1];
    if ((unsigned)h_info[2] & kStatNonpositive) inf->status = FLD_ERR_NONPOSITIVE;
  }
}

// A stream host function: fills the caller's fld_info (may be null) when the stream reaches it.
struct Delivery {
  fld_info* dst;
  DiffuseResult res;
  const int* h_info;  // pinned exchange counters and status bits, or null
};

void CUDART_CB deliver(void* arg) {
  Delivery* d = static_cast<Delivery*>(arg);
  resolve(d->res);
  if (d->dst) fill_info(d->dst, d->res.ss, d->h_info);
  delete d;
}

fld_status enqueue_delivery(fld_ctx* ctx, fld_info* info, const DiffuseResult& r, const int* h_info, cudaStream_t s) {
  if (!info && !r.out) return FLD_OK;
  Delivery* d = new (std::nothrow) Delivery{info, r, h_info};
  if (!d) return fail(ctx, FLD_ERR_CUDA, "out of host memory");
  cudaError_t e = cudaLaunchHostFunc(s, deliver, d);
  if (e != cudaSuccess) {
    delete d;
    return cuda_fail(ctx, e, "result delivery");
  }
  return FLD_OK;
}

// The status of a completed step, with its message.
fld_status outcome(fld_ctx* ctx, const fld_info& inf) {
  if (inf.status == FLD_ERR_NONPOSITIVE)
    return fail(ctx, FLD_ERR_NONPOSITIVE, "rho, kappa or E <= 0 (or eps < 0) in the input or an intermediate state");
  if (inf.status != FLD_OK)
    return fail(ctx, (fld_status)inf.status, "diffusion solve stopped at relative residual %.3e after %d cycles",
                inf.rel_residual, inf.cycles);
  return FLD_OK;
}

fld_status run_diffuse(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt, const double* const D[3],
                       const double* E_old, double* E_new, DiffuseResult* r, cudaStream_t s) {
  GridDev g = to_dev(grid);
  cudaError_t e = ctx->mg.configure(g, p->precision);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "multigrid allocation");
  e = ctx->mg.setup(dt, D, E_old, p->rtol, ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "multigrid setup");
  int maxc = p->max_cycles > 0 ? p->max_cycles : 100;
  const bool fmg = p->start == FLD_START_FMG;
  r->out = nullptr;
  if (ctx->mg.async_ready())
    e = ctx->mg.solve_async(E_old, E_new, p->rtol, maxc, p->nu1, p->nu2, fmg, &r->ss, &r->out, s);
  else
    e = ctx->mg.solve(E_old, E_new, p->rtol, maxc, p->nu1, p->nu2, fmg, &r->ss, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "multigrid solve");
  return FLD_OK;
}

fld_status ensure_geom(fld_ctx* ctx, int ncell) {
  size_t need = 4 * (size_t)ncell + 4;
  if (need <= ctx->geom_cap) return FLD_OK;
  cudaFree(ctx->geom);
  ctx->geom = nullptr;
  ctx->geom_cap = 0;
  cudaError_t e = cudaMalloc(&ctx->geom, need * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "column geometry allocation");
  ctx->geom_cap = need;
  return FLD_OK;
}

fld_status check_coarsest(fld_ctx* ctx, const fld_grid* g) {
  // the coarsest multigrid level is solved by one thread block
  int n[3] = {g->n[0], g->n[1], g->n[2]};
  long long cells = (long long)n[0] * n[1] * n[2];
  for (;;) {
    bool ok = cells > 64;
    for (int a = 0; a < g->ndim && ok; ++a) ok = (n[a] % 2 == 0) && n[a] >= 4;
    if (!ok) break;
    for (int a = 0; a < g->ndim; ++a) n[a] /= 2;
    cells = (long long)n[0] * n[1] * n[2];
  }
  if (cells > 4096)
    return fail(ctx, FLD_ERR_UNSUPPORTED,
                "grid %dx%dx%d coarsens only to %lld cells (>4096); use axis lengths with more factors of 2", g->n[0],
                g->n[1], g->n[2], cells);
  return FLD_OK;
}

}  // namespace

extern "C" {

fld_status fld_ctx_create(fld_ctx** out, int device) {
  if (!out) return FLD_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FLD_ERR_INVALID_ARG;
  fld_ctx* ctx = new (std::nothrow) fld_ctx();
  if (!ctx) return FLD_ERR_CUDA;
  ctx->device = device;
  DeviceGuard dg(device);
  cudaError_t e = cudaMalloc(&ctx->d_status, 64);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_info, 64);
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_info, 64);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 64);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_info, 0, 64);
  if (e != cudaSuccess) {
    fld_ctx_destroy(ctx);
    return FLD_ERR_CUDA;
  }
  *out = ctx;
  return FLD_OK;
}

fld_status fld_ctx_destroy(fld_ctx* ctx) {
  if (!ctx) return FLD_OK;
  DeviceGuard dg(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->D);
  cudaFree(ctx->kappa);
  cudaFree(ctx->geom);
  cudaFree(ctx->mid);
  cudaFree(ctx->stage);
  for (cudaEvent_t ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_info);
  if (ctx->h_info) cudaFreeHost(ctx->h_info);
  delete ctx->batched;
  delete ctx;  // releases the multigrid buffers while the device is current
  return FLD_OK;
}

const char* fld_last_error(const fld_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

unsigned long long fld_launch_count(void) { return fld::launch_count(); }

fld_status fld_coeffs(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, const double* E, const double* rho,
                      const double* eps, double* kappa_out, double* D_out, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_grid(ctx, grid);
  if (st == FLD_OK) st = check_params(ctx, p, false);
  if (st != FLD_OK) return st;
  if (!E || !rho || !eps || !D_out) return fail(ctx, FLD_ERR_INVALID_ARG, "E, rho, eps and D_out must be non-NULL");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  GridDev g = to_dev(grid);
  cudaError_t e = launch_coeffs(g, to_opacity(p), p->c, p->gamma, p->gas_R, p->limiter, E, rho, eps, kappa_out, D_out,
                                ctx->d_status, s, p->precision == FLD_PREC_FP64);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fld_coeffs launch");
  return FLD_OK;
}

namespace {

fld_status diffuse_common(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                          const double* const Dax[3], const double* E_old, double* E_new, fld_info* info,
                          void* stream) {
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  DiffuseResult r;
  fld_status st = run_diffuse(ctx, grid, p, dt, Dax, E_old, E_new, &r, s);
  if (st != FLD_OK) return st;
  if (!r.out) {  // known already
    if (info) fill_info(info, r.ss, nullptr);
    return FLD_OK;
  }
  return enqueue_delivery(ctx, info, r, nullptr, s);
}

fld_status diffuse_checks(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt, const double* E_old,
                          double* E_new) {
  fld_status st = check_grid(ctx, grid);
  if (st == FLD_OK) st = check_params(ctx, p, true);
  if (st == FLD_OK) st = check_coarsest(ctx, grid);
  if (st != FLD_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be > 0");
  if (!E_old || !E_new) return fail(ctx, FLD_ERR_INVALID_ARG, "E_old and E_new must be non-NULL");
  return FLD_OK;
}

}  // namespace

fld_status fld_diffuse(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt, const double* D_cell,
                       const double* E_old, double* E_new, fld_info* info, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = diffuse_checks(ctx, grid, p, dt, E_old, E_new);
  if (st != FLD_OK) return st;
  if (!D_cell) return fail(ctx, FLD_ERR_INVALID_ARG, "D_cell must be non-NULL");
  const double* const Dax[3] = {D_cell, D_cell, D_cell};
  return diffuse_common(ctx, grid, p, dt, Dax, E_old, E_new, info, stream);
}

fld_status fld_diffuse_aniso(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                             const double* const* D_axis, const double* E_old, double* E_new, fld_info* info,
                             void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = diffuse_checks(ctx, grid, p, dt, E_old, E_new);
  if (st != FLD_OK) return st;
  if (!D_axis) return fail(ctx, FLD_ERR_INVALID_ARG, "D_axis must be non-NULL");
  const double* Dax[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < 3; ++a) {
    Dax[a] = a < grid->ndim ? D_axis[a] : D_axis[0];
    if (!Dax[a]) return fail(ctx, FLD_ERR_INVALID_ARG, "D_axis[%d] is NULL", a);
  }
  return diffuse_common(ctx, grid, p, dt, Dax, E_old, E_new, info, stream);
}

fld_status fld_smooth_sweep(fld_ctx* ctx, const fld_grid* grid, double dt, const double* D_cell, const float* r,
                            const float* x_in, float* x_out, int first_colour, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_grid(ctx, grid);
  if (st != FLD_OK) return st;
  if (!D_cell || !r || !x_out) return fail(ctx, FLD_ERR_INVALID_ARG, "D_cell, r and x_out must be non-NULL");
  if (x_in == x_out) return fail(ctx, FLD_ERR_INVALID_ARG, "x_out must not be x_in");
  if (((uintptr_t)r | (uintptr_t)x_in | (uintptr_t)x_out) & 15u)
    return fail(ctx, FLD_ERR_INVALID_ARG, "r, x_in and x_out must start on 16-byte boundaries");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be positive and finite");
  if (first_colour != 0 && first_colour != 1) return fail(ctx, FLD_ERR_INVALID_ARG, "first_colour must be 0 or 1");
  if (grid->ndim != 3 || !sweep3d_eligible(grid->n[0], grid->n[1], grid->n[2]))
    return fail(ctx, FLD_ERR_UNSUPPORTED,
                "the tiled sweep needs a 3-D grid with n[0] %% 64 == 0, n[1] %% 16 == 0, n[2] even and >= 4");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const GridDev g = to_dev(grid);
  if ((st = ensure_scratch(ctx, g.ncell)) != FLD_OK) return st;
  float* dc = reinterpret_cast<float*>(ctx->kappa);  // FP32 in the FP64 scratch
  cudaError_t e = launch_dcell32(g.ncell, dt * g.inv_dx2[0], D_cell, dc, s);
  Sweep3dArgs a{};
  a.nx = g.n[0];
  a.ny = g.n[1];
  a.nz = g.n[2];
  for (int f = 0; f < 6; ++f) a.bc[f] = g.bc[f];
  for (int ax = 0; ax < 3; ++ax) a.ra[ax] = (float)(g.inv_dx2[ax] / g.inv_dx2[0]);
  a.dc = dc;
  a.r = r;
  a.xin = x_in;
  a.xout = x_out;
  a.x64 = nullptr;
  a.c0 = first_colour;
  a.err = ctx->d_status;  // set by a wait for staged planes that ran out of its bound
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_sweep3d(a, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_info + 2, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fld_smooth_sweep launch");
  if (ctx->h_info[2]) return fail(ctx, FLD_ERR_DEVICE_TIMEOUT, "fld_smooth_sweep: staged planes did not arrive in time");
  return FLD_OK;
}

fld_status fld_opacity(fld_ctx* ctx, size_t n, const fld_params* p, const double* rho, const double* eps,
                       double* kappa, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_params(ctx, p, false);
  if (st != FLD_OK) return st;
  if (n == 0) return FLD_OK;
  if (!rho || !eps || !kappa) return fail(ctx, FLD_ERR_INVALID_ARG, "rho, eps and kappa must be non-NULL");
  DeviceGuard dg(ctx->device);
  cudaError_t e = launch_opacity((long long)n, to_opacity(p), p->gamma, p->gas_R, p->precision == FLD_PREC_MIXED, rho,
                                 eps, kappa, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fld_opacity launch");
  return FLD_OK;
}

fld_status fld_exchange(fld_ctx* ctx, size_t n, const fld_params* p, double dt, const double* rho, const double* kappa,
                        double* eps, double* E, fld_info* info, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_params(ctx, p, false);
  if (st != FLD_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be > 0");
  if (n == 0) {
    if (info) memset(info, 0, sizeof(*info));
    return FLD_OK;
  }
  if (!rho || !eps || !E) return fail(ctx, FLD_ERR_INVALID_ARG, "rho, eps and E must be non-NULL");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = reset_status(ctx, s)) != FLD_OK) return st;
  cudaError_t e = launch_exchange((long long)n, to_exchange(p, dt), to_opacity(p), rho, kappa, eps, E, ctx->d_info,
                                  ctx->d_info + 1, ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fld_exchange launch");
  if (info) {
    unsigned sbits;
    memset(info, 0, sizeof(*info));
    if ((st = read_status(ctx, s, &sbits, &info->exch_max_iters, &info->bisection_fallbacks)) != FLD_OK) return st;
    info->status = (sbits & kStatNonpositive) ? FLD_ERR_NONPOSITIVE : FLD_OK;
    if (info->status != FLD_OK) return fail(ctx, FLD_ERR_NONPOSITIVE, "exchange met rho, kappa <= 0 or eps, E < 0");
  }
  return FLD_OK;
}

fld_status fld_step(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt, const double* rho, double* eps,
                    double* E, fld_info* info, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_grid(ctx, grid);
  if (st == FLD_OK) st = check_params(ctx, p, true);
  if (st == FLD_OK) st = check_coarsest(ctx, grid);
  if (st != FLD_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be > 0");
  if (!rho || !eps || !E) return fail(ctx, FLD_ERR_INVALID_ARG, "rho, eps and E must be non-NULL");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  GridDev g = to_dev(grid);
  if ((st = ensure_scratch(ctx, g.ncell)) != FLD_OK) return st;
  if ((st = reset_status(ctx, s)) != FLD_OK) return st;
  Opacity op = to_opacity(p);
  ExchangeParams xp = to_exchange(p, dt);
  DiffuseResult dr;
  cudaError_t e;
  if (p->order == FLD_ORDER_IMEX_MIDPOINT) {
    // Sect. 3.1, midpoint IMEX for the static-medium subsystem: exchange over dt/2 from u^n,
    // diffusion over dt/2 (D from that state), then the exchange over dt from u^n plus twice the
    // half-step diffusion increment
    if ((st = ensure_mid(ctx, g.ncell)) != FLD_OK) return st;
    double* E0 = ctx->mid;
    double* eps0 = ctx->mid + g.ncell;
    double* Eh = ctx->mid + 2 * g.ncell;
    const size_t bytes = g.ncell * sizeof(double);
    e = cudaMemcpyAsync(E0, E, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(eps0, eps, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "midpoint copies");
    ExchangeParams xh = to_exchange(p, 0.5 * dt);
    e = launch_exchange(g.ncell, xh, op, rho, nullptr, eps, E, ctx->d_info, ctx->d_info + 1, ctx->d_status, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "exchange launch");
    e = cudaMemcpyAsync(Eh, E, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "midpoint copies");
    e = launch_coeffs(g, op, p->c, p->gamma, p->gas_R, p->limiter, E, rho, eps, ctx->kappa, ctx->D, ctx->d_status, s,
                      p->precision == FLD_PREC_FP64);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coeffs launch");
    const double* const Dax[3] = {ctx->D, ctx->D, ctx->D};
    if ((st = run_diffuse(ctx, grid, p, 0.5 * dt, Dax, E, E, &dr, s)) != FLD_OK) return st;
    e = launch_midpoint_combine(g.ncell, E0, eps0, Eh, E, eps, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "midpoint combine launch");
    e = launch_exchange(g.ncell, xp, op, rho, nullptr, eps, E, ctx->d_info, ctx->d_info + 1, ctx->d_status, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "exchange launch");
  } else {
    if (p->order == FLD_ORDER_EXCHANGE_THEN_DIFFUSE) {
      e = launch_exchange(g.ncell, xp, op, rho, nullptr, eps, E, ctx->d_info, ctx->d_info + 1, ctx->d_status, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "exchange launch");
    }
    e = launch_coeffs(g, op, p->c, p->gamma, p->gas_R, p->limiter, E, rho, eps, ctx->kappa, ctx->D, ctx->d_status,
                      s, p->precision == FLD_PREC_FP64);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coeffs launch");
    const double* const Dax[3] = {ctx->D, ctx->D, ctx->D};
    if ((st = run_diffuse(ctx, grid, p, dt, Dax, E, E, &dr, s)) != FLD_OK) return st;
    if (p->order == FLD_ORDER_DIFFUSE_THEN_EXCHANGE) {
      // eps is unchanged by the diffusion, so kappa^n from the coefficient stage is current
      e = launch_exchange(g.ncell, xp, op, rho, ctx->kappa, eps, E, ctx->d_info, ctx->d_info + 1, ctx->d_status, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "exchange launch");
    }
  }
  // the exchange counters and status bits into pinned memory, then the outcome into *info, both in
  // stream order: nothing here waits for the device
  e = cudaMemcpyAsync(ctx->h_info, ctx->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_info + 2, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status read-back");
  if (!info && !dr.out) return FLD_OK;
  Delivery* d = new (std::nothrow) Delivery{info, dr, ctx->h_info};
  if (!d) return fail(ctx, FLD_ERR_CUDA, "out of host memory");
  e = cudaLaunchHostFunc(s, deliver, d);
  if (e != cudaSuccess) {
    delete d;
    return cuda_fail(ctx, e, "result delivery");
  }
  return FLD_OK;
}

fld_status fld_step_host(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt, const double* rho,
                         double* eps, double* E, fld_info* info, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_grid(ctx, grid);
  if (st == FLD_OK) st = check_params(ctx, p, true);
  if (st == FLD_OK) st = check_coarsest(ctx, grid);
  if (st != FLD_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be > 0");
  if (!rho || !eps || !E) return fail(ctx, FLD_ERR_INVALID_ARG, "rho, eps and E must be non-NULL");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const GridDev g = to_dev(grid);
  const long long n = g.ncell;
  if ((st = ensure_stage(ctx, n)) != FLD_OK) return st;
  double* dr = ctx->stage;
  double* de = ctx->stage + n;
  double* dE = ctx->stage + 2 * n;
  const size_t cell = sizeof(double);
  cudaStream_t cs = ctx->copy_stream;
  cudaError_t e;
  if (p->order != FLD_ORDER_DIFFUSE_THEN_EXCHANGE) {
    // whole arrays in, fld_step, whole arrays out
    e = cudaMemcpyAsync(dr, rho, n * cell, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(de, eps, n * cell, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dE, E, n * cell, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copies");
    fld_info tmp;
    fld_info* inf = info ? info : &tmp;
    st = fld_step(ctx, grid, p, dt, dr, de, dE, inf, stream);
    if (st == FLD_ERR_CUDA) return st;
    const std::string msg = ctx->err;
    e = cudaMemcpyAsync(eps, de, n * cell, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E, dE, n * cell, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device-to-host copies");
    ctx->err = msg;
    if (st != FLD_OK) return st;
    return outcome(ctx, *inf);
  }
  if ((st = ensure_scratch(ctx, n)) != FLD_OK) return st;
  if ((st = reset_status(ctx, s)) != FLD_OK) return st;
  const Opacity op = to_opacity(p);
  const ExchangeParams xp = to_exchange(p, dt);
  cudaEvent_t* ev = ctx->ev;  // [0] s before the copies, [1] E in, [2 + i] slab i in, [2 + S + i] slab i out
  const int S = (int)std::min<long long>(kHostSlabs, std::max<long long>(1, n / 4096));
  auto first = [&](int i) { return n * i / S; };
  // any host copy still queued must finish before an error return, since the caller may then free
  // the host arrays
  auto drain = [&](fld_status r) {
    cudaStreamSynchronize(cs);
    return r;
  };
  // the copies start after the work already queued on the caller's stream (it may use the staging)
  e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dE, E, n * cell, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], cs);
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    const long long f = first(i), c = first(i + 1) - f;
    e = cudaMemcpyAsync(dr + f, rho + f, c * cell, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(de + f, eps + f, c * cell, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 + i], cs);
  }
  if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "host-to-device copies"));
  // coefficients slab by slab as rho and eps arrive (E, which the stencil reads across slabs, first)
  e = cudaStreamWaitEvent(s, ev[1], 0);
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(s, ev[2 + i], 0);
    if (e == cudaSuccess)
      e = launch_coeffs_range(g, op, p->c, p->gamma, p->gas_R, p->limiter, dE, dr, de, ctx->kappa, ctx->D,
                              ctx->d_status, first(i), first(i + 1) - first(i), s, p->precision == FLD_PREC_FP64);
  }
  if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "coeffs launch"));
  DiffuseResult res;
  const double* const Dax[3] = {ctx->D, ctx->D, ctx->D};
  if ((st = run_diffuse(ctx, grid, p, dt, Dax, dE, dE, &res, s)) != FLD_OK) return drain(st);
  // exchange slab by slab, each slab's eps and E copied back while the next ones are computed
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    const long long f = first(i), c = first(i + 1) - f;
    e = launch_exchange(c, xp, op, dr + f, ctx->kappa + f, de + f, dE + f, ctx->d_info, ctx->d_info + 1,
                        ctx->d_status, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 + S + i], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[2 + S + i], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(eps + f, de + f, c * cell, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E + f, dE + f, c * cell, cudaMemcpyDeviceToHost, cs);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
  if (e != cudaSuccess) return drain(cuda_fail(ctx, e, "exchange and device-to-host copies"));
  // this call returns with the host arrays complete, so it waits here and reports the outcome
  if ((st = read_status(ctx, s, nullptr, nullptr, nullptr)) != FLD_OK) return drain(st);
  resolve(res);
  fld_info tmp;
  fld_info* inf = info ? info : &tmp;
  fill_info(inf, res.ss, ctx->h_info);
  return outcome(ctx, *inf);
}

fld_status fld_radiation_terms(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, const double* E,
                               const double* rho, const double* eps, const double* const* v, double* const* F,
                               double* const* f_r, double* work, double* fedd, double* const* P, double* tiring,
                               int sync, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_grid(ctx, grid);
  if (st == FLD_OK) st = check_params(ctx, p, false);
  if (st != FLD_OK) return st;
  if (!E || !rho || !eps) return fail(ctx, FLD_ERR_INVALID_ARG, "E, rho and eps must be non-NULL");
  const int nd = grid->ndim;
  const double* vv[3] = {nullptr, nullptr, nullptr};
  double* FF[3] = {nullptr, nullptr, nullptr};
  double* ff[3] = {nullptr, nullptr, nullptr};
  double* PP[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int a = 0; a < nd; ++a) {
    if (v) {
      if (!v[a]) return fail(ctx, FLD_ERR_INVALID_ARG, "velocity component %d is NULL", a);
      vv[a] = v[a];
    }
    if (F) FF[a] = F[a];
    if (f_r) ff[a] = f_r[a];
  }
  if (P)
    for (int m = 0; m < 6; ++m) PP[m] = P[m];
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  GridDev g = to_dev(grid);
  if ((st = reset_status(ctx, s)) != FLD_OK) return st;
  cudaError_t e = launch_radiation_terms(g, to_opacity(p), p->c, p->gamma, p->gas_R, p->limiter, E, rho, eps,
                                         v ? vv : nullptr, FF, ff, work, fedd, PP, tiring, nullptr, 0.0,
                                         ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "radiation terms launch");
  if (sync) {
    unsigned sbits = 0;
    int it = 0, bi = 0;
    if ((st = read_status(ctx, s, &sbits, &it, &bi)) != FLD_OK) return st;
    if (sbits & kStatNonpositive) return fail(ctx, FLD_ERR_NONPOSITIVE, "rho, kappa or E <= 0 (or eps < 0)");
  }
  return FLD_OK;
}

fld_status fld_photon_tiring_step(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                                  const double* rho, const double* eps, const double* const* v, double* E,
                                  void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!v) return fail(ctx, FLD_ERR_INVALID_ARG, "the velocity components are required");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be > 0");
  fld_status st = check_grid(ctx, grid);
  if (st != FLD_OK) return st;
  DeviceGuard dg(ctx->device);
  GridDev g = to_dev(grid);
  if ((st = ensure_scratch(ctx, g.ncell)) != FLD_OK) return st;
  // the tiring term into the context's D scratch, then the update (the stencil reads E)
  st = fld_radiation_terms(ctx, grid, p, E, rho, eps, v, nullptr, nullptr, nullptr, nullptr, nullptr, ctx->D, 0,
                           stream);
  if (st != FLD_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_explicit_update(g.ncell, -dt, ctx->D, E, ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tiring update launch");
  unsigned sbits = 0;
  int it = 0, bi = 0;
  if ((st = read_status(ctx, s, &sbits, &it, &bi)) != FLD_OK) return st;
  if (sbits & kStatNonpositive) return fail(ctx, FLD_ERR_NONPOSITIVE, "invalid input or E <= 0 after the update");
  return FLD_OK;
}

fld_status fld_pseudo_planar_source(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double x0,
                                    const double* E, const double* rho, const double* eps, const double* const* v,
                                    double* S, int sync, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_grid(ctx, grid);
  if (st == FLD_OK) st = check_params(ctx, p, false);
  if (st != FLD_OK) return st;
  if (!(x0 >= 0) || !std::isfinite(x0)) return fail(ctx, FLD_ERR_INVALID_ARG, "x0 must be finite and >= 0");
  if (!E || !rho || !eps || !S) return fail(ctx, FLD_ERR_INVALID_ARG, "E, rho, eps and S must be non-NULL");
  const double* vv[3] = {nullptr, nullptr, nullptr};
  if (v)
    for (int a = 0; a < grid->ndim; ++a) {
      if (!v[a]) return fail(ctx, FLD_ERR_INVALID_ARG, "velocity component %d is NULL", a);
      vv[a] = v[a];
    }
  double* none3[3] = {nullptr, nullptr, nullptr};
  double* none6[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  GridDev g = to_dev(grid);
  if ((st = reset_status(ctx, s)) != FLD_OK) return st;
  cudaError_t e = launch_radiation_terms(g, to_opacity(p), p->c, p->gamma, p->gas_R, p->limiter, E, rho, eps,
                                         v ? vv : nullptr, none3, none3, nullptr, nullptr, none6, nullptr, S, x0,
                                         ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pseudo-planar source launch");
  if (sync) {
    unsigned sbits = 0;
    int it = 0, bi = 0;
    if ((st = read_status(ctx, s, &sbits, &it, &bi)) != FLD_OK) return st;
    if (sbits & kStatNonpositive) return fail(ctx, FLD_ERR_NONPOSITIVE, "rho, kappa or E <= 0 (or eps < 0)");
  }
  return FLD_OK;
}

fld_status fld_pseudo_planar_step(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt, double x0,
                                  const double* rho, const double* eps, const double* const* v, double* E,
                                  void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!(dt > 0) || !std::isfinite(dt)) return fail(ctx, FLD_ERR_INVALID_ARG, "dt must be > 0");
  fld_status st = check_grid(ctx, grid);
  if (st != FLD_OK) return st;
  DeviceGuard dg(ctx->device);
  GridDev g = to_dev(grid);
  if ((st = ensure_scratch(ctx, g.ncell)) != FLD_OK) return st;
  // the source into the context's D scratch, then the update (the stencil reads E)
  st = fld_pseudo_planar_source(ctx, grid, p, x0, E, rho, eps, v, ctx->D, 0, stream);
  if (st != FLD_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_explicit_update(g.ncell, dt, ctx->D, E, ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pseudo-planar update launch");
  unsigned sbits = 0;
  int it = 0, bi = 0;
  if ((st = read_status(ctx, s, &sbits, &it, &bi)) != FLD_OK) return st;
  if (sbits & kStatNonpositive) return fail(ctx, FLD_ERR_NONPOSITIVE, "invalid input or E <= 0 after the update");
  return FLD_OK;
}

fld_status fld_step_batched(fld_ctx* ctx, int ngrids, const fld_grid* grids, const fld_params* params, const double* dt,
                            const double* const* rho, double* const* eps, double* const* E, fld_info* infos,
                            void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ngrids < 0 || (ngrids > 0 && (!grids || !params || !dt || !rho || !eps || !E)))
    return fail(ctx, FLD_ERR_INVALID_ARG, "ngrids < 0 or NULL host arrays");
  for (int i = 0; i < ngrids; ++i) {
    fld_status st = check_grid(ctx, &grids[i]);
    if (st == FLD_OK) st = check_params(ctx, &params[i], true);
    if (st == FLD_OK) st = check_coarsest(ctx, &grids[i]);
    if (st != FLD_OK) return fail(ctx, st, "grid %d: %s", i, std::string(ctx->err).c_str());
    if (grids[i].ndim < 2) return fail(ctx, FLD_ERR_INVALID_ARG, "grid %d: batched grids need ndim 2 or 3", i);
    if ((long long)grids[i].n[0] * grids[i].n[1] * grids[i].n[2] >= (1LL << 31))
      return fail(ctx, FLD_ERR_INVALID_ARG, "grid %d: batched grids hold fewer than 2^31 cells", i);
    if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(ctx, FLD_ERR_INVALID_ARG, "grid %d: dt must be > 0", i);
    if (!rho[i] || !eps[i] || !E[i]) return fail(ctx, FLD_ERR_INVALID_ARG, "grid %d: NULL device array", i);
  }
  if (ngrids == 0) return FLD_OK;
  DeviceGuard dg(ctx->device);
  if (!ctx->batched) {
    ctx->batched = new (std::nothrow) BatchedSolver();
    if (!ctx->batched) return fail(ctx, FLD_ERR_CUDA, "out of host memory");
  }
  std::string err;
  fld_status st = ctx->batched->run(ngrids, grids, params, dt, rho, eps, E, infos, (cudaStream_t)stream, &err);
  if (st != FLD_OK) return fail(ctx, st, "%s", err.c_str());
  return FLD_OK;
}

fld_status fld_columns_step(fld_ctx* ctx, int ncol, int ncell, const double* r_faces, int geometry, int bc_lo,
                            int bc_hi, const double* v_lo, const double* v_hi, const fld_params* p, const double* dt,
                            const double* rho, double* eps, double* E, fld_info* info, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_params(ctx, p, false, true);
  if (st != FLD_OK) return st;
  if (p->order != FLD_ORDER_DIFFUSE_THEN_EXCHANGE && p->order != FLD_ORDER_EXCHANGE_THEN_DIFFUSE &&
      p->order != FLD_ORDER_IMEX_MIDPOINT)
    return fail(ctx, FLD_ERR_INVALID_ARG, "unknown order %d", p->order);
  std::string err;
  st = columns_validate(ncol, ncell, r_faces, geometry, bc_lo, bc_hi, v_lo, v_hi, dt, &err);
  if (st != FLD_OK) return fail(ctx, st, "%s", err.c_str());
  if (ncol == 0) {
    if (info) memset(info, 0, sizeof(*info));
    return FLD_OK;
  }
  if (!rho || !eps || !E) return fail(ctx, FLD_ERR_INVALID_ARG, "rho, eps and E must be non-NULL");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = reset_status(ctx, s)) != FLD_OK) return st;
  if ((st = ensure_geom(ctx, ncell)) != FLD_OK) return st;
  cudaError_t e = launch_columns_step(ncol, ncell, r_faces, geometry, bc_lo, bc_hi, v_lo, v_hi, *p, dt, rho, eps, E,
                                      ctx->geom, ctx->d_info, ctx->d_info + 1, ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fld_columns_step launch");
  if (info) {
    unsigned sbits;
    memset(info, 0, sizeof(*info));
    if ((st = read_status(ctx, s, &sbits, &info->exch_max_iters, &info->bisection_fallbacks)) != FLD_OK) return st;
    info->status = (sbits & kStatNonpositive) ? FLD_ERR_NONPOSITIVE : FLD_OK;
    if (info->status != FLD_OK) return fail(ctx, FLD_ERR_NONPOSITIVE, "rho, kappa or E <= 0 (or eps < 0) in a column");
  }
  return FLD_OK;
}

fld_status fld_columns_diffuse(fld_ctx* ctx, int ncol, int ncell, const double* r_faces, int geometry, int bc_lo,
                               int bc_hi, const double* v_lo, const double* v_hi, const fld_params* p, const double* dt,
                               const double* D_cell, const double* E_old, double* E_new, void* stream) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  ctx->err.clear();
  fld_status st = check_params(ctx, p, false, true);
  if (st != FLD_OK) return st;
  std::string err;
  st = columns_validate(ncol, ncell, r_faces, geometry, bc_lo, bc_hi, v_lo, v_hi, dt, &err);
  if (st != FLD_OK) return fail(ctx, st, "%s", err.c_str());
  if (ncol == 0) return FLD_OK;
  if (!D_cell || !E_old || !E_new) return fail(ctx, FLD_ERR_INVALID_ARG, "D_cell, E_old and E_new must be non-NULL");
  DeviceGuard dg(ctx->device);
  if ((st = ensure_geom(ctx, ncell)) != FLD_OK) return st;
  cudaError_t e = launch_columns_diffuse(ncol, ncell, r_faces, geometry, bc_lo, bc_hi, v_lo, v_hi, *p, dt, D_cell,
                                         E_old, E_new, ctx->geom, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fld_columns_diffuse launch");
  return FLD_OK;
}

fld_status fld_trace_enable(fld_ctx* ctx, int on) {
  if (!ctx) return FLD_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (on) tracer().clear();
  tracer().on = on != 0;
  tracer().major_only = on == 2;
  return FLD_OK;
}

fld_status fld_trace_report(fld_ctx* ctx, fld_trace_entry* out, int max, int* n) {
  if (!ctx || !n || (max > 0 && !out)) return FLD_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  auto rep = tracer().report();
  int k = 0;
  for (auto& e : rep) {
    if (k >= max) break;
    memset(&out[k], 0, sizeof(fld_trace_entry));
    snprintf(out[k].name, sizeof(out[k].name), "%s", e.name.c_str());
    out[k].launches = e.launches;
    out[k].total_ms = e.ms;
    ++k;
  }
  *n = k;
  return FLD_OK;
}

}  // extern "C"

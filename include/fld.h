/*
 * fld.h -- C ABI of the GB300 (sm_103a) flux-limited-diffusion radiation-energy update.
 *
 * Method: arXiv 2104.03968, "Radiation-hydrodynamics with MPI-AMRVAC: flux-limited
 * diffusion".  The update advances the radiation energy density E and the gas internal
 * energy density eps of a static medium (density rho) over one time step dt:
 *
 *   fld_coeffs    opacity kappa(rho, T), the 4th-order gradient of E (Sect. 3.2, Eq.
 *                 ileyk_flux), R = |grad E|/(kappa rho E), the Levermore-Pomraning limiter
 *                 lambda(R) (Sect. 2.2, Eq. fld_lambda) and D = c lambda/(kappa rho)
 *                 (Sect. 2.2, Eq. fld_F), per cell.
 *   fld_diffuse   the backward-Euler diffusion solve E^{n+1}/dt - div(D grad E^{n+1}) =
 *                 E^n/dt on a uniform Cartesian grid, 5/7/3-point stencil with harmonic-mean
 *                 face coefficients (Sect. 3.4, Eq. discdiff), by geometric multigrid.
 *   fld_exchange  the point-implicit gas-radiation energy exchange: the quartic in
 *                 eps^{n+1} (Sect. 3.3), root in ]0, eps^n + E^n[, then E^{n+1}.
 *   fld_step      fld_coeffs, fld_diffuse and fld_exchange in the selected order.
 *   fld_step_batched   many independent 2-D/3-D grids in one call.
 *   fld_columns_step   many independent 1-D radial columns (spherical or Cartesian finite
 *                 volumes on a stretched grid), diffusion by a tridiagonal solve.
 *
 * Conventions shared by every entry point
 *   - Arrays are caller-owned DEVICE memory, float64, contiguous, x fastest: cell (i,j,k)
 *     is element i + n[0]*(j + n[1]*k).  Column arrays are [column][cell].
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work
 *     is enqueued on it, and calls return after enqueueing unless documented otherwise.
 *     The solves (fld_diffuse, fld_diffuse_aniso, fld_step) keep their whole outer loop on
 *     the device -- residual, convergence test and V-cycles in one CUDA graph whose
 *     conditional nodes the device steers -- so they do not wait for the GPU either.  Their
 *     outcome (status, cycles, residual, sweep counts) is written into *info in stream order:
 *     keep `info` valid until the stream has passed the call, and read it after synchronising
 *     the stream.  Two exceptions wait on the stream: the first solve of a grid configuration
 *     with autotuned sweep counts (it times its candidates), and solves while per-kernel
 *     tracing is on.  fld_step_batched and fld_step_host return with their results complete.
 *   - Inputs are never modified; eps and E are updated in place where documented.
 *   - Empty batches are valid: n == 0 cells (fld_opacity, fld_exchange), ncol == 0 columns and
 *     ngrids == 0 grids launch nothing and return FLD_OK once the scalar arguments have passed
 *     their checks; the data arrays may then be NULL, and an info is zeroed (status FLD_OK).
 *     A grid (fld_grid) has at least one cell per axis.
 *   - Return value: FLD_OK, or an error code for an invalid argument or a CUDA error.  What
 *     the device finds -- a solve that did not reach rtol within max_cycles, a non-positive
 *     input met on the device, a non-finite residual -- is info->status of the asynchronous
 *     calls (and the return value of the synchronous ones).  The message of the last error is
 *     available from fld_last_error().  No exception crosses the ABI.
 *   - A context is bound to one device and is not thread-safe; use one context per host
 *     thread.  It owns the multigrid hierarchy, scratch buffers and CUDA graphs and keeps
 *     them between calls of the same shape.
 */
#ifndef FLD_H
#define FLD_H

#include <stddef.h>

#if defined(__GNUC__)
#define FLD_API __attribute__((visibility("default")))
#else
#define FLD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FLD_OK = 0,
  FLD_ERR_INVALID_ARG = 1,
  FLD_ERR_NONPOSITIVE = 2,  /* rho, kappa or E <= 0, or eps < 0, met on the device */
  FLD_ERR_NONFINITE = 3,    /* a NaN/Inf appeared in a residual norm */
  FLD_ERR_NOT_CONVERGED = 4,
  FLD_ERR_CUDA = 5,
  FLD_ERR_DEVICE_TIMEOUT = 6,
  FLD_ERR_UNSUPPORTED = 7
} fld_status;

/* boundary conditions (Sect. 3.4): ghost value, fixed gradient, linear extrapolation; and, for the
   inner face of radial columns only, a fixed luminosity L (Sect. 5.2): the ghost is
   E_0 + L dr / (4 pi r_0^2 D_0) with r_0 the first cell centre, dr the distance to the ghost centre
   and D_0 the first cell's D of the state entering the step (whose gradient there uses a linear
   extrapolation); the boundary value is L */
enum { FLD_BC_PERIODIC = 0, FLD_BC_NEUMANN = 1, FLD_BC_DIRICHLET = 2, FLD_BC_CONTINUOUS = 3, FLD_BC_LUMINOSITY = 4 };
/* Eq. fld_lambda; lambda = 1/3 (the diffusion limit); or the Minerbo limiter, the alternative
   Sect. 2.2 names: lambda = 2/(3 + sqrt(9 + 12 R^2)) for R <= 3/2, 1/(1 + R + sqrt(1 + 2R)) above */
enum { FLD_LIMITER_LP = 0, FLD_LIMITER_THIRD = 1, FLD_LIMITER_MINERBO = 2 };
enum { FLD_OPACITY_CONST = 0, FLD_OPACITY_KRAMERS = 1, FLD_OPACITY_TABLE = 2 };
enum { FLD_PREC_FP64 = 0, FLD_PREC_MIXED = 1 };
/* step order: diffusion then exchange; exchange then diffusion; or the paper's midpoint IMEX scheme
   (Sect. 3.1): exchange over dt/2 from the old state, diffusion over dt/2, then the exchange over
   dt from the old state plus twice the half-step diffusion increment */
enum { FLD_ORDER_DIFFUSE_THEN_EXCHANGE = 0, FLD_ORDER_EXCHANGE_THEN_DIFFUSE = 1, FLD_ORDER_IMEX_MIDPOINT = 2 };
/* first cycle of the multigrid solve: full multigrid (Sect. 3.4: FMG, then V-cycles) or a V-cycle */
enum { FLD_START_FMG = 0, FLD_START_VCYCLE = 1 };
enum { FLD_GEOM_CARTESIAN = 0, FLD_GEOM_SPHERICAL = 1 };

/* Uniform Cartesian grid.  ndim in {1,2,3}; unused axes have n = 1.  bc[2a] / bc[2a+1] are the
   lower / upper faces of axis a; bc_val holds the Dirichlet ghost value or the Neumann
   gradient dE/dx across the boundary face.  Every axis with a non-periodic face needs
   n >= 2. */
typedef struct {
  int ndim;
  int n[3];
  double dx[3];
  int bc[6];
  double bc_val[6];
} fld_grid;

/* CAK line opacity of radial columns (Sect. 5.1, Eq. kap_cak), added to the opacity model wherever
   the opacity enters (coefficients and exchange):
     kappa_CAK = kQ / (1 - alpha) (|dv/dr| / (c kQ rho))^alpha,
   dv/dr by the central difference of the cell-centre velocities (one-sided at the column ends),
   alpha(x), x = 1 - r_star / r: alpha_in for x <= x_in, alpha_out for x >= x_out, linear between
   (the paper: 0.66, 0.5, 0.4, 0.65). */
typedef struct {
  const double* v;            /* DEVICE, [column][cell]: radial velocity at the cell centres */
  double kappa_e_Qbar;        /* kQ, the line opacity when every line is optically thin */
  double r_star;
  double alpha_in, alpha_out; /* 0 <= alpha < 1 */
  double x_in, x_out;         /* x_in <= x_out */
} fld_cak;

typedef struct {
  /* physics (code units or cgs, consistently) */
  double c;        /* speed of light */
  double a_rad;    /* radiation constant a_r = 4 sigma / c */
  double gamma;    /* adiabatic index */
  double gas_R;    /* k_b / (mu m_p): T = (gamma-1) eps / (rho gas_R) */
  int limiter;     /* FLD_LIMITER_* */
  int opacity;     /* FLD_OPACITY_*: kappa0 | kappa0 rho^kr_a T^kr_b | table */
  double kappa0, kr_a, kr_b;
  const double* table; /* DEVICE pointer: log10 kappa on a tn[0] x tn[1] grid, row = log10 rho,
                          column (fastest) = log10 T, uniform over [tlo, thi], bilinear and
                          clamped at the edges */
  int tn[2];
  double tlo[2], thi[2];
  /* solver */
  int precision;   /* FLD_PREC_FP64: plain FP64 throughout -- the coefficients, the multigrid
                      solve and the exchange's safeguarded Halley root (Sect. 3.3).
                      FLD_PREC_MIXED: FP32 V-cycles inside a defect-correction loop whose
                      residuals, updates and norms are FP64-grade: double-float (pairs of floats,
                      ~2^-46 relative) with a certified error bound, FP64 where values leave the
                      double-float range or rtol < 1e-10; the coefficients and the exchange in
                      double-float with FP64 fallback per cell. */
  double rtol;     /* stop when ||b - A E||_2 / ||b||_2 <= rtol */
  int max_cycles;  /* outer iterations (one V-cycle each); 0 = 100 */
  int nu1, nu2;    /* red-black Gauss-Seidel sweeps before / after coarse correction.  Both 0:
                      autotuned on the first solve of a grid configuration (per rtol and start:
                      candidate sets -- a pair for the finest level, a pair for the coarser
                      ones -- are timed on a scratch iterate, the fastest converged set is kept
                      for later calls); otherwise every level uses them (0 = 2) */
  int exch_maxit;  /* Halley iterations before bisection in the exchange; 0 = 100 */
  int order;       /* FLD_ORDER_* used by fld_step */
  int start;       /* FLD_START_*: first cycle of fld_diffuse / fld_step (fld_step_batched always
                      starts with a V-cycle) */
  const fld_cak* cak; /* HOST pointer; column calls only: CAK line opacity, or NULL */
} fld_params;

typedef struct {
  int cycles;              /* outer iterations (V-cycles) used */
  double rel_residual;     /* final ||b - A E||_2 / ||b||_2 in FP64 */
  int exch_max_iters;      /* largest number of root iterations over the cells */
  int bisection_fallbacks; /* cells that fell back to bisection */
  int status;              /* fld_status of this grid / column set */
  int nu1, nu2;            /* sweep counts the multigrid solve used on the finest level */
  int nu1_coarse, nu2_coarse; /* and on the coarser levels (differ only when autotuned) */
} fld_info;

typedef struct fld_ctx fld_ctx;

/* Create a context on `device` (CUDA ordinal).  *out receives the handle. */
FLD_API fld_status fld_ctx_create(fld_ctx** out, int device);
FLD_API fld_status fld_ctx_destroy(fld_ctx* ctx);
/* Message of the last error raised on `ctx` (never NULL; empty when none). */
FLD_API const char* fld_last_error(const fld_ctx* ctx);

/* Kernels this library has launched in the calling process so far, every launch site and the
   kernels of each CUDA-graph replay included (a graph counts the kernels captured in it; the
   batched solver's WHILE node counts its body once per pass).  A diagnostic for benchmarks, with
   no counterpart in the paper; read it before and after the work to count. */
FLD_API unsigned long long fld_launch_count(void);

/* Per-cell opacity and diffusion coefficient (Sect. 2.2, Eqs. fld_lambda and fld_F, with the
   5-point gradient of Sect. 3.2).  In: E, rho, eps (N cells).  Out: kappa_out (N, may be NULL),
   D_out (N).  Asynchronous. */
FLD_API fld_status fld_coeffs(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, const double* E,
                      const double* rho, const double* eps, double* kappa_out, double* D_out,
                      void* stream);

/* Backward-Euler diffusion (Sect. 3.4, Eq. discdiff): solves
   E_new + dt*(-div D grad E_new) = E_old (with the boundary terms) to p->rtol.  D_cell is the
   cell-centred D from fld_coeffs; faces take its harmonic mean.  E_new may alias E_old.
   `info` (may be NULL) receives the status, cycles and final relative residual in stream order.
   Asynchronous (see the conventions above). */
FLD_API fld_status fld_diffuse(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                       const double* D_cell, const double* E_old, double* E_new, fld_info* info,
                       void* stream);

/* fld_diffuse with a diagonal-tensor D (the anisotropic variant Sect. 6 mentions: one diffusion
   coefficient per grid direction).  D_axis: host array of grid->ndim DEVICE pointers; D_axis[a]
   is the cell-centred D of axis a, and the faces of axis a take its harmonic mean.  Otherwise as
   fld_diffuse (asynchronous). */
FLD_API fld_status fld_diffuse_aniso(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                             const double* const* D_axis, const double* E_old, double* E_new,
                             fld_info* info, void* stream);

/* One red-black Gauss-Seidel sweep (both colours) of the smoother that the mixed-precision
   multigrid runs on the finest level of 3-D grids (Sect. 3.4: a Gauss-Seidel smoother of the
   backward-Euler operator of Eq. discdiff), exposed so that it can be checked on its own.  It
   relaxes the dt-scaled correction equation x + dt (-div D grad x) = r in FP32:
     x_c <- (r_c + sum_f w_f x_nb) / (1 + sum_f w_f),  w_f = dt D_f / dx_a^2,
   with D_f the harmonic mean of the two cells' D (a non-periodic boundary face takes the interior
   cell's D; Dirichlet, Neumann and linear-extrapolation faces as in fld_diffuse, with homogeneous
   boundary values).  D_cell: DEVICE float64, N cells.  r, x_in, x_out: DEVICE float32, N cells,
   x fastest; x_in NULL means x = 0 before the sweep; x_out must not overlap x_in.  The cells with
   (i + j + k) % 2 == first_colour are updated first, then the others from their new values.
   Supported grids: ndim 3, n[0] a multiple of 64, n[1] a multiple of 16, n[2] even and >= 4,
   fewer than 2^31 cells (FLD_ERR_UNSUPPORTED otherwise); every array starts on a 16-byte boundary.
   Uses the context's scratch (allocated on first use) for an FP32 copy of dt D / dx_0^2.
   Synchronises the stream: FLD_ERR_DEVICE_TIMEOUT if a wait of the kernel for its staged planes
   ran out of its bound (x_out is then unspecified). */
FLD_API fld_status fld_smooth_sweep(fld_ctx* ctx, const fld_grid* grid, double dt, const double* D_cell,
                                    const float* r, const float* x_in, float* x_out, int first_colour,
                                    void* stream);

/* Opacity of n independent cells (Sect. 2: T from the ideal-gas law; Sect. 5.1: the tabulated
   opacity, here a bilinear table in log10 rho and log10 T on log10 kappa, clamped to its edges; or
   the constant / Kramers-like models of p).  rho, eps, kappa: DEVICE float64, n cells.  With
   p->precision == FLD_PREC_MIXED the table's two logarithms and its power of ten are evaluated in
   double-float arithmetic (relative error ~1e-14), as the mixed column step does; otherwise in
   FP64.  Asynchronous. */
FLD_API fld_status fld_opacity(fld_ctx* ctx, size_t n, const fld_params* p, const double* rho, const double* eps,
                               double* kappa, void* stream);

/* Point-implicit exchange (Sect. 3.3) on n independent cells, in place on eps and E.  kappa may
   be NULL, in which case it is evaluated from rho and eps with the opacity model of p.
   Asynchronous; `info` (may be NULL) is filled after a stream synchronisation. */
FLD_API fld_status fld_exchange(fld_ctx* ctx, size_t n, const fld_params* p, double dt, const double* rho,
                        const double* kappa, double* eps, double* E, fld_info* info, void* stream);

/* One full radiation-energy update in place on eps and E: coefficients from the state entering
   the diffusion stage (lagged D), diffusion, exchange; p->order selects the paper's order
   (exchange first, Sect. 3.1) or diffusion first.  Asynchronous: `info` (may be NULL) receives
   the solve's outcome and the exchange's counters in stream order; its status is
   FLD_ERR_NONPOSITIVE if rho, kappa or E <= 0 (or eps < 0) was met on the device. */
FLD_API fld_status fld_step(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                    const double* rho, double* eps, double* E, fld_info* info, void* stream);

/* The update of fld_step (Sects. 3.1-3.4) on HOST arrays, for callers whose fields live in host
   memory.  rho, eps, E: HOST arrays of cells, x fastest; eps and E are updated in place.
   The library copies them into device buffers it owns (allocated on first use, kept in the
   context), runs the step on `stream`, and copies eps and E back; it returns once they are back.
   With the default order (diffusion, then exchange) the copies are pipelined in 8 equal cell
   ranges on a second stream: E first, then rho and eps range by range while the
   coefficient kernel runs on the ranges already in, and eps and E range by range while the
   exchange runs on the later ranges.  Page-locked (pinned) host memory is needed for the copies
   to overlap; pageable memory works, serialised.  Results equal fld_step's on the same data.
   Errors as fld_step; on a CUDA error the host arrays may hold a partial update. */
FLD_API fld_status fld_step_host(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                         const double* rho, double* eps, double* E, fld_info* info, void* stream);

/* fld_step on `ngrids` independent grids with their own sizes, parameters and time steps.
   grids, params and dt are HOST arrays of length ngrids; rho/eps/E are HOST arrays of DEVICE
   pointers; infos (may be NULL) receives one fld_info per grid.  Every grid must have ndim 2
   or 3 and fewer than 2^31 cells (FLD_ERR_INVALID_ARG otherwise).  Synchronises.
   All grids share params[0].precision.  The batch autotunes its own sweep counts and tile size
   on the first call for a batch shape (nu1 / nu2 of params are not used).  With
   FLD_PREC_MIXED, each grid's fine residual is double-float with a bound on its error.  The
   grid has converged when the residual plus the bound is at most its rtol, so the true residual
   is too.  A grid whose bound exceeds rtol / 4 takes FP64 residuals from its next cycle on.
   A grid with no linear-extrapolation face (a symmetric operator) runs conjugate gradients
   preconditioned by the V-cycle as its outer loop; the others add each V-cycle's correction.
   infos[g].rel_residual is the last residual computed, bound not included. */
FLD_API fld_status fld_step_batched(fld_ctx* ctx, int ngrids, const fld_grid* grids,
                            const fld_params* params, const double* dt, const double* const* rho,
                            double* const* eps, double* const* E, fld_info* infos, void* stream);

/* One full update of `ncol` independent 1-D radial columns of `ncell` cells sharing the face
   radii r_faces (DEVICE, ncell+1 values, increasing).  geometry: FLD_GEOM_SPHERICAL (areas r^2,
   volumes (r_+^3 - r_-^3)/3) or FLD_GEOM_CARTESIAN.  bc_lo/bc_hi: FLD_BC_DIRICHLET, NEUMANN or
   CONTINUOUS; v_lo/v_hi: DEVICE arrays of ncol boundary values.  dt: DEVICE array of ncol time
   steps.  rho, eps, E: DEVICE [ncol][ncell]; eps and E are updated in place.  The diffusion is
   a direct tridiagonal solve per column (exact to round-off, no rtol).  The gradient in R is
   the 3-point non-uniform central difference.  Asynchronous. */
FLD_API fld_status fld_columns_step(fld_ctx* ctx, int ncol, int ncell, const double* r_faces, int geometry,
                            int bc_lo, int bc_hi, const double* v_lo, const double* v_hi,
                            const fld_params* p, const double* dt, const double* rho,
                            double* eps, double* E, fld_info* info, void* stream);

/* Diffusion stage only of fld_columns_step, with a caller-given cell-centred D (DEVICE
   [ncol][ncell]); E_new may alias E_old.  Asynchronous. */
FLD_API fld_status fld_columns_diffuse(fld_ctx* ctx, int ncol, int ncell, const double* r_faces,
                               int geometry, int bc_lo, int bc_hi, const double* v_lo,
                               const double* v_hi, const fld_params* p, const double* dt,
                               const double* D_cell, const double* E_old, double* E_new,
                               void* stream);

/* Explicit radiation terms of the current state (Sect. 2.1-2.2 and 3.2), per cell, with every
   gradient by the 5-point stencil of Sect. 3.2:
     F     = -D grad E                                  (Eq. fld_F; D as in fld_coeffs)
     f_r   = rho kappa F / c                            (Eq. rhd_force), work = v . f_r
     f     = lambda + lambda^2 R^2                      (Eq. fld_Edd_fac, the Eddington factor)
     P     = E [(1-f)/2 I + (3f-1)/2 n n], n = grad E / |grad E| (n = 0 where grad E = 0)
                                                         (Eq. fld_Edd)
     P:grad v = sum_ab P_ab d_b v_a                     (the photon-tiring term)
   In: E, rho, eps (N cells, device); v = host array of grid->ndim DEVICE pointers to the velocity
   components, or NULL (then work and tiring are 0).  Velocity ghosts on non-periodic faces are
   linear extrapolations.  Out (each may be NULL): F and f_r = host arrays of ndim device pointers;
   P = host array of 6 device pointers (xx, yy, zz, xy, xz, yz); work, fedd, tiring = device arrays.
   sync == 0: asynchronous, and cells with rho, kappa or E <= 0 (or eps < 0) are left unwritten
   without an error.  sync != 0: synchronises and returns FLD_ERR_NONPOSITIVE if any cell was. */
FLD_API fld_status fld_radiation_terms(fld_ctx* ctx, const fld_grid* grid, const fld_params* p,
                               const double* E, const double* rho, const double* eps,
                               const double* const* v, double* const* F, double* const* f_r,
                               double* work, double* fedd, double* const* P, double* tiring,
                               int sync, void* stream);

/* The explicit radiation-energy source over dt (Sect. 3.1, first stage; Sect. 3.2):
   E <- E - dt P : grad v, in place (P and the gradients from the state on entry).  v as in
   fld_radiation_terms (required).  Synchronises; FLD_ERR_NONPOSITIVE when the input is invalid or
   the update leaves E <= 0 somewhere. */
FLD_API fld_status fld_photon_tiring_step(fld_ctx* ctx, const fld_grid* grid, const fld_params* p,
                                  double dt, const double* rho, const double* eps,
                                  const double* const* v, double* E, void* stream);

/* Pseudo-planar geometric source of the radiation energy (Appendix A).  The grid is Cartesian and
   its x axis (axis 0) stands for the radius of a radially extended problem; the spherical
   divergence differs from the Cartesian one by 2 f_x / x, which becomes a source.  Per cell
     S = -2 (E v_x + F_x) / x + 2 v_x P_xx / x,   x = x0 + (i + 1/2) dx[0]
   (the second term corrects the radiation-work term P : grad v, as printed in the appendix), with
   F and P exactly as in fld_radiation_terms.  x0 >= 0 is the radius of the grid's lower x face.
   v = host array of grid->ndim DEVICE pointers to the velocity components, or NULL (v = 0, so
   S = -2 F_x / x).  S: DEVICE array of N cells (out).  sync as in fld_radiation_terms. */
FLD_API fld_status fld_pseudo_planar_source(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double x0,
                                    const double* E, const double* rho, const double* eps,
                                    const double* const* v, double* S, int sync, void* stream);

/* E <- E + dt S with S the pseudo-planar source of the state on entry (context scratch holds
   S).  Synchronises; FLD_ERR_NONPOSITIVE when the input is invalid or the update leaves E <= 0. */
FLD_API fld_status fld_pseudo_planar_step(fld_ctx* ctx, const fld_grid* grid, const fld_params* p, double dt,
                                  double x0, const double* rho, const double* eps,
                                  const double* const* v, double* E, void* stream);

/* ---- allocation-free column update (no counterpart in the paper; a deployment convenience).
   Some callers cannot allocate device memory when they advance the radiation field: codes whose
   own memory manager has reserved the whole GPU in advance, runtimes that forbid device
   allocation inside their time-step loop (for instance while recording work for later replay),
   or real-time loops where an allocation that may fail or stall is not acceptable.  They cannot
   create an fld_ctx either, since a context allocates its scratch on first use.
   fld_columns_step_static takes the arguments of fld_columns_step without the context, does the
   same computation, and allocates nothing: its scratch (the per-cell geometry factors and three
   status counters) lives in one statically sized device array of the library, 4 *
   FLD_STATIC_MAX_CELLS + 8 doubles (about 64 KiB), which every device that loads the library
   holds until the process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
     - ncell > FLD_STATIC_MAX_CELLS is rejected with FLD_ERR_UNSUPPORTED (nothing is launched);
       the other argument checks and return codes are those of fld_columns_step.
     - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
       with that device current, and caches it.  Make that first call before any stream capture.
     - Every call on a device shares the one array and leaves its contents behind; each call
       rewrites the geometry and clears the counters before use.  Calls whose work overlaps on
       the GPU (different streams, or host threads, without ordering between them) race on the
       array and give undefined results: order them on one stream.
     - With info == NULL the call returns after enqueueing; otherwise it synchronises on the
       stream and fills info as fld_columns_step does. */
#define FLD_STATIC_MAX_CELLS 2048
FLD_API fld_status fld_columns_step_static(int ncol, int ncell, const double* r_faces, int geometry, int bc_lo,
                                           int bc_hi, const double* v_lo, const double* v_hi, const fld_params* p,
                                           const double* dt, const double* rho, double* eps, double* E,
                                           fld_info* info, void* stream);

/* ---- tracing: per-kernel launch timing with CUDA events (library diagnostics; the paper has
   no counterpart).  While enabled, every kernel launch of the library is bracketed by a pair of
   events on its stream; fld_trace_report synchronises on them and returns, per kernel name,
   the number of launches and their summed device time since the last enable. */
typedef struct {
  char name[32];
  int launches;
  double total_ms;
} fld_trace_entry;

/* on != 0 clears the record and starts tracing (on == 2: only the finest-level and per-step kernels,
   which costs fewer event records per step); on == 0 stops it (the record is kept). */
FLD_API fld_status fld_trace_enable(fld_ctx* ctx, int on);
/* Writes up to `max` entries to `out` and their count to *n.  Synchronises. */
FLD_API fld_status fld_trace_report(fld_ctx* ctx, fld_trace_entry* out, int max, int* n);

#ifdef __cplusplus
}
#endif
#endif /* FLD_H */

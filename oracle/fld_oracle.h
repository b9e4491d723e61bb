/*
 * Plain FP64 CPU oracle for the flux-limited-diffusion (FLD) radiation-energy
 * update of "Radiation-hydrodynamics with MPI-AMRVAC: flux-limited diffusion"
 * (arXiv 2104.03968).  TEST INFRASTRUCTURE ONLY: only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code with the
 * CUDA library.  Everything is single-threaded, plain loops, double precision.
 *
 * Layout: cell arrays are contiguous, x fastest (index i + nx*(j + ny*k)).
 */
#ifndef FLD_ORACLE_H
#define FLD_ORACLE_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_BC_PERIODIC = 0, ORA_BC_NEUMANN = 1, ORA_BC_DIRICHLET = 2, ORA_BC_CONTINUOUS = 3,
       ORA_BC_LUMINOSITY = 4 /* columns, inner face only: fixed luminosity (Sect. 5.2) */ };
enum { ORA_LIM_LP = 0, ORA_LIM_THIRD = 1, ORA_LIM_MINERBO = 2 };
enum { ORA_OPA_CONST = 0, ORA_OPA_KRAMERS = 1, ORA_OPA_TABLE = 2 };
enum { ORA_GEOM_CARTESIAN = 0, ORA_GEOM_SPHERICAL = 1 };

typedef struct {
  int ndim;          /* 1, 2 or 3 */
  int n[3];          /* cells per axis (unused axes = 1) */
  double dx[3];      /* uniform spacing per axis */
  int bc[6];         /* lower/upper per axis: x-,x+,y-,y+,z-,z+ */
  double bc_val[6];  /* Dirichlet value or Neumann gradient */
} ora_grid;

typedef struct {
  double c, a_rad, gamma, gas_R; /* gas_R = k_b/(mu m_p) */
  int limiter;                   /* ORA_LIM_* */
  int opacity;                   /* ORA_OPA_* */
  double kappa0, kr_a, kr_b;     /* kappa = kappa0 rho^kr_a T^kr_b (Kramers) */
  const double* table;           /* log10 kappa, [tn0][tn1], log10 T fastest */
  int tn[2];
  double tlo[2], thi[2];         /* log10 rho range, log10 T range */
} ora_phys;

double ora_lambda(double R);
double ora_lambda_minerbo(double R);
double ora_limiter(int limiter, double R);
double ora_temperature(const ora_phys* p, double rho, double eps);
double ora_kappa(const ora_phys* p, double rho, double T);
void ora_opacity(size_t n, const ora_phys* p, const double* rho, const double* eps, double* kappa);
/* explicit radiation quantities: F[ndim], fr[ndim], work, fedd, P[6] (xx yy zz xy xz yz), tiring;
   any output may be NULL; v (ndim velocity components) may be NULL */
int ora_radiation_sources(const ora_grid* g, const ora_phys* p, const double* E, const double* rho,
                          const double* kappa, const double* const* v, double* const* F, double* const* fr,
                          double* work, double* fedd, double* const* P, double* tiring);

/* pseudo-planar geometric source of E (x = x0 + (i + 1/2) dx[0]); v may be NULL (v = 0) */
int ora_pseudo_planar_source(const ora_grid* g, const ora_phys* p, double x0, const double* E,
                             const double* rho, const double* kappa, const double* const* v, double* S);

/* 4th-order 5-point gradient, |grad E|, R, lambda and D = c lambda/(kappa rho) per cell. */
int ora_coeffs(const ora_grid* g, const ora_phys* p, const double* E, const double* rho,
               const double* kappa, double* D_cell, double* gradmag);

/* Linear (homogeneous-boundary) part of the dt-scaled operator  A = I + dt*(-div D grad). */
void ora_apply(const ora_grid* g, double dt, const double* D_cell, const double* x, double* Ax);
/* Right-hand side b = E_old + boundary constants (Dirichlet value, Neumann gradient). */
void ora_rhs(const ora_grid* g, double dt, const double* D_cell, const double* E_old, double* b);
/* ||b - A x||_2 / ||b||_2 */
double ora_relres(const ora_grid* g, double dt, const double* D_cell, const double* E_old, const double* x);
/* Jacobi-preconditioned conjugate gradients (symmetric boundary conditions only). */
int ora_diffuse_cg(const ora_grid* g, double dt, const double* D_cell, const double* E_old, double* E_new,
                   double rtol, int maxit, double* relres, int* iters);
/* the same with a diagonal-tensor D: Dax[a] is the cell-centred D of axis a */
void ora_apply_aniso(const ora_grid* g, double dt, const double* const* Dax, const double* x, double* Ax);
double ora_relres_aniso(const ora_grid* g, double dt, const double* const* Dax, const double* E_old,
                        const double* x);
int ora_diffuse_cg_aniso(const ora_grid* g, double dt, const double* const* Dax, const double* E_old, double* x,
                         double rtol, int maxit, double* relres, int* iters);
/* Dense LU with partial pivoting on the assembled matrix (small grids; any boundary). */
int ora_diffuse_dense(const ora_grid* g, double dt, const double* D_cell, const double* E_old, double* E_new);

/* One 1-D column on a stretched radial grid (r_faces: n+1 values).  Finite-volume operator with
   area r^2 and volume (r+^3-r-^3)/3 (spherical) or 1 and width (Cartesian); Thomas algorithm. */
/* Sect. 5.1, Eq. (kap_cak): CAK line opacity of one column from the radial velocity v at the cell
   centres; alpha(x), x = 1 - rstar/r: a_in for x <= x_in, a_out for x >= x_out, linear between */
void ora_kappa_cak(int n, const double* rf, const double* rho, const double* v, double c, double kQ,
                   double rstar, double a_in, double a_out, double x_in, double x_out, double* out);
int ora_column_coeffs(int n, const double* r_faces, int bc_lo, int bc_hi, double v_lo, double v_hi,
                      const ora_phys* p, const double* E, const double* rho, const double* kappa,
                      double* D_cell);
int ora_column_diffuse(int n, const double* r_faces, int geometry, int bc_lo, int bc_hi, double v_lo,
                       double v_hi, double dt, const double* D_cell, const double* E_old, double* E_new);
int ora_column_diffuse_dense(int n, const double* r_faces, int geometry, int bc_lo, int bc_hi, double v_lo,
                             double v_hi, double dt, const double* D_cell, const double* E_old, double* E_new);
double ora_column_relres(int n, const double* r_faces, int geometry, int bc_lo, int bc_hi, double v_lo,
                         double v_hi, double dt, const double* D_cell, const double* E_old, const double* x);

/* Point-implicit gas-radiation exchange: quartic root by safeguarded Halley, bisection after maxit. */
int ora_exchange(size_t n, const ora_phys* p, double dt, const double* rho, const double* kappa,
                 double* eps, double* E, int maxit, int* max_iters, int* bisections);

#ifdef __cplusplus
}
#endif
#endif

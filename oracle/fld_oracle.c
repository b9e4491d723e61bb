/*
 * Plain FP64 CPU oracle for the FLD radiation-energy update of arXiv 2104.03968.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library; the CUDA library never does, and the
 * two share no source.  It is written for a reader checking it against the paper:
 * plain loops, double precision, no blocking or fusion.
 *
 * What each function follows:
 *   ora_lambda            Sect. 2.2, Eq. (fld_lambda): Levermore-Pomraning limiter.
 *   ora_kappa_cak         Sect. 5.1, Eq. (kap_cak): CAK line opacity along a radial column.
 *   ora_radiation_sources Sect. 2.1-2.2 and 3.2: flux, radiation force and work, Eddington
 *                         factor and tensor, photon tiring P : grad v.
 *   ora_pseudo_planar_source  Appendix A: the geometric source of the radiation energy on a
 *                         Cartesian grid whose x axis stands for the radius, -2(E v_x + F_x)/x,
 *                         plus the radiation-work correction 2 v_x P_xx / x as printed there.
 *   ora_lambda_minerbo    the Minerbo limiter that Sect. 2.2 names as the alternative (its
 *                         formula is not printed there; the two-branch form of Minerbo's
 *                         closure, joined at R = 3/2, is restated here).
 *   ora_coeffs            Sect. 2.2, Eqs. (fld_lambda), (fld_F) and the ratio R; Sect. 3.2,
 *                         Eq. (ileyk_flux): 4th-order 5-point gradient.
 *   face coefficients     Sect. 3.4: harmonic mean of the two cell-centred D.
 *   ora_apply / ora_rhs   Sect. 3.4, Eq. (discdiff) multiplied through by dt, with the
 *                         Dirichlet / Neumann / continuous ghost cells listed under it.
 *   ora_diffuse_*         The backward-Euler Helmholtz problem of Sect. 3.4, solved to
 *                         round-off: the result is the exact solution of the linear
 *                         system, whatever solver reaches it.
 *   ora_exchange          Sect. 3.3: the point-implicit heating/cooling equations, their
 *                         quartic in eps^{n+1} with the root in ]0, eps^n + E^n[, Halley's
 *                         method with a bisection fallback, then the E^{n+1} formula.
 *   ora_opacity           Sect. 2.1 gas law for T; Kramers-like and tabulated opacities
 *                         stand in for the tables of Sect. 5.1.
 *
 * Readings taken where the paper is silent or garbled:
 *   - a boundary face takes the D of its interior cell (ghost D = interior D);
 *   - Dirichlet fixes the ghost-cell value, Neumann the gradient across the boundary face,
 *     "continuous" extrapolates linearly from the two interior cells;
 *   - on the stretched 1-D radial grid the gradient is the 3-point non-uniform central
 *     difference (the 5-point formula assumes uniform spacing);
 *   - the exchange coefficient a1 carries the (m_p mu / k_b)^4 factor of the gas law, which
 *     the printed expression for a1 drops; with it the quartic and the E^{n+1} formula agree;
 *   - the quartic is solved for y = x / (eps^n + E^n), whose root lies in ]0, 1[.
 */
#include "fld_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double kPi = 3.14159265358979323846;

/* ------------------------------------------------------------------ physics */

double ora_lambda(double R) {
  /* Sect. 2.2, Eq. (fld_lambda) */
  return (2.0 + R) / (6.0 + 3.0 * R + R * R);
}

double ora_lambda_minerbo(double R) {
  if (R <= 1.5) return 2.0 / (3.0 + sqrt(9.0 + 12.0 * R * R));
  return 1.0 / (1.0 + R + sqrt(1.0 + 2.0 * R));
}

double ora_limiter(int limiter, double R) {
  if (limiter == ORA_LIM_THIRD) return 1.0 / 3.0;
  if (limiter == ORA_LIM_MINERBO) return ora_lambda_minerbo(R);
  return ora_lambda(R);
}

double ora_temperature(const ora_phys* p, double rho, double eps) {
  /* Sect. 2 ideal gas: p = (gamma-1) eps = rho k_b T / (mu m_p) */
  return (p->gamma - 1.0) * eps / (rho * p->gas_R);
}

double ora_kappa(const ora_phys* p, double rho, double T) {
  if (p->opacity == ORA_OPA_CONST) return p->kappa0;
  if (p->opacity == ORA_OPA_KRAMERS) return p->kappa0 * pow(rho, p->kr_a) * pow(T, p->kr_b);
  /* table of log10 kappa on a uniform (log10 rho, log10 T) grid, bilinear, clamped */
  double u = (log10(rho) - p->tlo[0]) / (p->thi[0] - p->tlo[0]) * (p->tn[0] - 1);
  double v = (log10(T) - p->tlo[1]) / (p->thi[1] - p->tlo[1]) * (p->tn[1] - 1);
  if (u < 0) u = 0;
  if (u > p->tn[0] - 1) u = p->tn[0] - 1;
  if (v < 0) v = 0;
  if (v > p->tn[1] - 1) v = p->tn[1] - 1;
  int i = (int)floor(u), j = (int)floor(v);
  if (i > p->tn[0] - 2) i = p->tn[0] - 2;
  if (j > p->tn[1] - 2) j = p->tn[1] - 2;
  double fu = u - i, fv = v - j;
  const double* t = p->table;
  int m = p->tn[1];
  double l = (1 - fu) * (1 - fv) * t[i * m + j] + (1 - fu) * fv * t[i * m + j + 1] +
             fu * (1 - fv) * t[(i + 1) * m + j] + fu * fv * t[(i + 1) * m + j + 1];
  return pow(10.0, l);
}

void ora_opacity(size_t n, const ora_phys* p, const double* rho, const double* eps, double* kappa) {
  for (size_t c = 0; c < n; ++c) kappa[c] = ora_kappa(p, rho[c], ora_temperature(p, rho[c], eps[c]));
}

/* ------------------------------------------------------------------ grid helpers */

static size_t ncells(const ora_grid* g) { return (size_t)g->n[0] * g->n[1] * g->n[2]; }

static size_t lin(const ora_grid* g, const int q[3]) {
  return (size_t)q[0] + (size_t)g->n[0] * ((size_t)q[1] + (size_t)g->n[1] * q[2]);
}

/* Value of E at integer position p along axis a (other coordinates from q), applying
   the boundary condition when p lies outside [0, n).  Ghost cells per Sect. 3.4. */
static double sample(const ora_grid* g, const double* E, const int q[3], int a, int p) {
  int n = g->n[a];
  int r[3] = {q[0], q[1], q[2]};
  if (p >= 0 && p < n) {
    r[a] = p;
    return E[lin(g, r)];
  }
  int side = p < 0 ? 0 : 1;
  int bc = g->bc[2 * a + side];
  double v = g->bc_val[2 * a + side];
  if (bc == ORA_BC_PERIODIC) {
    r[a] = ((p % n) + n) % n;
    return E[lin(g, r)];
  }
  if (bc == ORA_BC_DIRICHLET) return v;
  if (side == 0) {
    int m = -1 - p; /* mirror distance: p=-1 -> 0, p=-2 -> 1 */
    if (bc == ORA_BC_NEUMANN) {
      r[a] = m;
      return E[lin(g, r)] - (2 * m + 1) * v * g->dx[a];
    }
    r[a] = 0;
    double e0 = E[lin(g, r)];
    r[a] = 1;
    double e1 = E[lin(g, r)];
    return e0 + p * (e1 - e0);
  } else {
    int m = p - n;
    if (bc == ORA_BC_NEUMANN) {
      r[a] = n - 1 - m;
      return E[lin(g, r)] + (2 * m + 1) * v * g->dx[a];
    }
    r[a] = n - 1;
    double e1 = E[lin(g, r)];
    r[a] = n - 2;
    double e0 = E[lin(g, r)];
    return e1 + (p - (n - 1)) * (e1 - e0);
  }
}

static void unlin(const ora_grid* g, size_t c, int q[3]) {
  q[0] = (int)(c % g->n[0]);
  q[1] = (int)((c / g->n[0]) % g->n[1]);
  q[2] = (int)(c / ((size_t)g->n[0] * g->n[1]));
}

/* ------------------------------------------------------------------ coefficients */

int ora_coeffs(const ora_grid* g, const ora_phys* p, const double* E, const double* rho,
               const double* kappa, double* D_cell, double* gradmag) {
  size_t N = ncells(g);
  for (size_t c = 0; c < N; ++c) {
    if (!(E[c] > 0) || !(rho[c] > 0) || !(kappa[c] > 0)) return 2;
    int q[3];
    unlin(g, c, q);
    double g2 = 0;
    for (int a = 0; a < g->ndim; ++a) {
      int i = q[a];
      /* Sect. 3.2, Eq. (ileyk_flux) */
      double d = (sample(g, E, q, a, i - 2) / 12.0 - 2.0 / 3.0 * sample(g, E, q, a, i - 1) +
                  2.0 / 3.0 * sample(g, E, q, a, i + 1) - sample(g, E, q, a, i + 2) / 12.0) /
                 g->dx[a];
      g2 += d * d;
    }
    double gm = sqrt(g2);
    if (gradmag) gradmag[c] = gm;
    double kr = kappa[c] * rho[c];
    double R = gm / (kr * E[c]);
    double lam = ora_limiter(p->limiter, R);
    D_cell[c] = p->c * lam / kr; /* Sect. 2.2, Eq. (fld_F): F = -c lambda grad E/(kappa rho) */
  }
  return 0;
}

/* ------------------------------------------------------------------ explicit radiation terms */

/* field value at position p along axis a for the velocity components: periodic wrap, else
   linear extrapolation from the two boundary cells (velocity ghosts; the paper leaves them to
   the hydro solver) */
static double sample_extrap(const ora_grid* g, const double* f, const int q[3], int a, int p) {
  int n = g->n[a];
  int r[3] = {q[0], q[1], q[2]};
  if (p >= 0 && p < n) {
    r[a] = p;
    return f[lin(g, r)];
  }
  int side = p < 0 ? 0 : 1;
  if (g->bc[2 * a + side] == ORA_BC_PERIODIC) {
    r[a] = ((p % n) + n) % n;
    return f[lin(g, r)];
  }
  r[a] = side ? n - 1 : 0;
  double f0 = f[lin(g, r)];
  r[a] = side ? n - 2 : 1;
  double f1 = f[lin(g, r)];
  int d = side ? p - (n - 1) : -p;
  return f0 + d * (f0 - f1);
}

/* Sect. 3.2, Eq. (ileyk_flux) along axis a */
static double grad5(const ora_grid* g, const double* f, const int q[3], int a, int extrap) {
  double fm2, fm1, fp1, fp2;
  int i = q[a];
  if (extrap) {
    fm2 = sample_extrap(g, f, q, a, i - 2);
    fm1 = sample_extrap(g, f, q, a, i - 1);
    fp1 = sample_extrap(g, f, q, a, i + 1);
    fp2 = sample_extrap(g, f, q, a, i + 2);
  } else {
    fm2 = sample(g, f, q, a, i - 2);
    fm1 = sample(g, f, q, a, i - 1);
    fp1 = sample(g, f, q, a, i + 1);
    fp2 = sample(g, f, q, a, i + 2);
  }
  return (fm2 / 12.0 - 2.0 / 3.0 * fm1 + 2.0 / 3.0 * fp1 - fp2 / 12.0) / g->dx[a];
}

int ora_radiation_sources(const ora_grid* g, const ora_phys* p, const double* E, const double* rho,
                          const double* kappa, const double* const* v, double* const* F, double* const* fr,
                          double* work, double* fedd, double* const* P, double* tiring) {
  size_t N = ncells(g);
  int nd = g->ndim;
  for (size_t c = 0; c < N; ++c) {
    if (!(E[c] > 0) || !(rho[c] > 0) || !(kappa[c] > 0)) return 2;
    int q[3];
    unlin(g, c, q);
    double gE[3] = {0, 0, 0}, g2 = 0;
    for (int a = 0; a < nd; ++a) {
      gE[a] = grad5(g, E, q, a, 0);
      g2 += gE[a] * gE[a];
    }
    double gm = sqrt(g2);
    double kr = kappa[c] * rho[c];
    double R = gm / (kr * E[c]);
    double lam = ora_limiter(p->limiter, R);
    double D = p->c * lam / kr;
    double f = lam + lam * lam * R * R; /* Sect. 2.2, Eq. (fld_Edd_fac) */
    double nrm[3] = {0, 0, 0};
    if (gm > 0)
      for (int a = 0; a < nd; ++a) nrm[a] = gE[a] / gm;
    double w = 0;
    for (int a = 0; a < nd; ++a) {
      double Fa = -D * gE[a];                  /* Sect. 2.2, Eq. (fld_F) */
      double fa = rho[c] * kappa[c] * Fa / p->c; /* Sect. 2.1, Eq. (rhd_force) */
      if (F) F[a][c] = Fa;
      if (fr) fr[a][c] = fa;
      if (v) w += v[a][c] * fa;
    }
    if (work) work[c] = v ? w : 0.0;
    if (fedd) fedd[c] = f;
    /* Sect. 2.2, Eq. (fld_Edd): f_ab = (1-f)/2 delta_ab + (3f-1)/2 n_a n_b; P = f_ab E */
    double Pt[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        Pt[a][b] = E[c] * ((a == b ? 0.5 * (1.0 - f) : 0.0) + 0.5 * (3.0 * f - 1.0) * nrm[a] * nrm[b]);
    if (P) {
      P[0][c] = Pt[0][0];
      P[1][c] = Pt[1][1];
      P[2][c] = Pt[2][2];
      P[3][c] = Pt[0][1];
      P[4][c] = Pt[0][2];
      P[5][c] = Pt[1][2];
    }
    if (tiring) {
      /* Sect. 3.2: P : grad v = sum_ab P_ab d_b v_a */
      double t = 0;
      if (v)
        for (int a = 0; a < nd; ++a)
          for (int b = 0; b < nd; ++b) t += Pt[a][b] * grad5(g, v[a], q, b, 1);
      tiring[c] = t;
    }
  }
  return 0;
}

int ora_pseudo_planar_source(const ora_grid* g, const ora_phys* p, double x0, const double* E,
                             const double* rho, const double* kappa, const double* const* v, double* S) {
  /* Appendix A: x ~ r, so the spherical divergence (1/r^2) d_r (r^2 f) is the Cartesian d_x f
     plus 2 f / x, moved to the right-hand side as a source.  For the radiation energy the
     divergence carries f = E v + F; the radiation-work term gets its own correction. */
  size_t N = ncells(g);
  double* buf = (double*)malloc(9 * N * sizeof(double)); /* F (3 axes), then P (6 components) */
  if (!buf) return 3;
  double* F[3];
  double* P[6];
  for (int a = 0; a < 3; ++a) F[a] = buf + (size_t)a * N;
  for (int m = 0; m < 6; ++m) P[m] = buf + (size_t)(3 + m) * N;
  int st = ora_radiation_sources(g, p, E, rho, kappa, NULL, F, NULL, NULL, NULL, P, NULL);
  if (st == 0) {
    for (size_t c = 0; c < N; ++c) {
      int q[3];
      unlin(g, c, q);
      double x = x0 + (q[0] + 0.5) * g->dx[0]; /* the cell centre's radius */
      double vx = v ? v[0][c] : 0.0;
      S[c] = -2.0 * (E[c] * vx + F[0][c]) / x + 2.0 * vx * P[0][c] / x;
    }
  }
  free(buf);
  return st;
}

/* ------------------------------------------------------------------ operator */

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

/* Contribution of one face of cell q (axis a, side 0 = lower, 1 = upper) to the row of
   the dt-scaled operator:  self*x_q + cnb*x_nb  on the left, cconst on the right. */
static void face_term(const ora_grid* g, double dt, const double* const* Dax, const int q[3], int a, int side,
                      double* cself, long* nb, double* cnb, double* cconst) {
  int n = g->n[a];
  int i = q[a];
  int j = side ? i + 1 : i - 1;
  int r[3] = {q[0], q[1], q[2]};
  const double* D = Dax[a]; /* the diffusion coefficient of axis a (a diagonal tensor D) */
  double Di = D[lin(g, q)];
  double h2 = g->dx[a] * g->dx[a];
  *nb = -1;
  *cnb = 0;
  *cconst = 0;
  if (j >= 0 && j < n) {
    r[a] = j;
    double w = dt * harmonic(Di, D[lin(g, r)]) / h2;
    *cself = w;
    *nb = (long)lin(g, r);
    *cnb = -w;
    return;
  }
  int bc = g->bc[2 * a + side];
  double v = g->bc_val[2 * a + side];
  if (bc == ORA_BC_PERIODIC) {
    r[a] = ((j % n) + n) % n;
    double w = dt * harmonic(Di, D[lin(g, r)]) / h2;
    *cself = w;
    *nb = (long)lin(g, r);
    *cnb = -w;
    return;
  }
  double w = dt * Di / h2; /* boundary face: ghost D = interior D */
  if (bc == ORA_BC_DIRICHLET) {
    *cself = w; /* w (x_q - v) */
    *cconst = w * v;
  } else if (bc == ORA_BC_NEUMANN) {
    *cself = 0; /* ghost = x_q -/+ v dx: the flux is fixed */
    *cconst = side ? w * v * g->dx[a] : -w * v * g->dx[a];
  } else { /* continuous: ghost = 2 x_q - x_inner, so the term is w (x_inner - x_q) */
    r[a] = side ? i - 1 : i + 1;
    *cself = -w;
    *nb = (long)lin(g, r);
    *cnb = w;
  }
}

static void apply_ax(const ora_grid* g, double dt, const double* const* Dax, const double* x, double* Ax) {
  size_t N = ncells(g);
  for (size_t c = 0; c < N; ++c) {
    int q[3];
    unlin(g, c, q);
    double s = x[c];
    for (int a = 0; a < g->ndim; ++a)
      for (int side = 0; side < 2; ++side) {
        double cs, cn, cc;
        long nb;
        face_term(g, dt, Dax, q, a, side, &cs, &nb, &cn, &cc);
        s += cs * x[c];
        if (nb >= 0) s += cn * x[nb];
      }
    Ax[c] = s;
  }
}

static void rhs_ax(const ora_grid* g, double dt, const double* const* Dax, const double* E_old, double* b) {
  size_t N = ncells(g);
  for (size_t c = 0; c < N; ++c) {
    int q[3];
    unlin(g, c, q);
    double s = E_old[c];
    for (int a = 0; a < g->ndim; ++a)
      for (int side = 0; side < 2; ++side) {
        double cs, cn, cc;
        long nb;
        face_term(g, dt, Dax, q, a, side, &cs, &nb, &cn, &cc);
        s += cc;
      }
    b[c] = s;
  }
}

static double dot(size_t n, const double* a, const double* b) {
  double s = 0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double relres_ax(const ora_grid* g, double dt, const double* const* Dax, const double* E_old,
                        const double* x) {
  size_t N = ncells(g);
  double* b = malloc(N * sizeof(double));
  double* Ax = malloc(N * sizeof(double));
  rhs_ax(g, dt, Dax, E_old, b);
  apply_ax(g, dt, Dax, x, Ax);
  double rr = 0;
  for (size_t c = 0; c < N; ++c) rr += (b[c] - Ax[c]) * (b[c] - Ax[c]);
  double bb = dot(N, b, b);
  free(b);
  free(Ax);
  return sqrt(rr / bb);
}

static int diffuse_cg_ax(const ora_grid* g, double dt, const double* const* Dax, const double* E_old, double* x,
                         double rtol, int maxit, double* relres, int* iters) {
  for (int f = 0; f < 2 * g->ndim; ++f)
    if (g->bc[f] == ORA_BC_CONTINUOUS) return 1; /* not symmetric */
  size_t N = ncells(g);
  double* b = malloc(N * sizeof(double));
  double* r = malloc(N * sizeof(double));
  double* z = malloc(N * sizeof(double));
  double* pv = malloc(N * sizeof(double));
  double* Ap = malloc(N * sizeof(double));
  double* dinv = malloc(N * sizeof(double));
  rhs_ax(g, dt, Dax, E_old, b);
  for (size_t c = 0; c < N; ++c) {
    int q[3];
    unlin(g, c, q);
    double d = 1.0;
    for (int a = 0; a < g->ndim; ++a)
      for (int side = 0; side < 2; ++side) {
        double cs, cn, cc;
        long nb;
        face_term(g, dt, Dax, q, a, side, &cs, &nb, &cn, &cc);
        d += cs;
      }
    dinv[c] = 1.0 / d;
    x[c] = E_old[c];
  }
  double bnorm = sqrt(dot(N, b, b));
  apply_ax(g, dt, Dax, x, Ap);
  for (size_t c = 0; c < N; ++c) r[c] = b[c] - Ap[c];
  for (size_t c = 0; c < N; ++c) z[c] = dinv[c] * r[c];
  memcpy(pv, z, N * sizeof(double));
  double rz = dot(N, r, z);
  int it = 0;
  double best = sqrt(dot(N, r, r)) / bnorm;
  int since_check = 0;
  while (it < maxit && best > rtol) {
    apply_ax(g, dt, Dax, pv, Ap);
    double alpha = rz / dot(N, pv, Ap);
    for (size_t c = 0; c < N; ++c) {
      x[c] += alpha * pv[c];
      r[c] -= alpha * Ap[c];
    }
    ++it;
    ++since_check;
    double rn = sqrt(dot(N, r, r)) / bnorm;
    if (rn <= rtol || since_check >= 50) {
      /* replace the recursive residual by the true one */
      apply_ax(g, dt, Dax, x, Ap);
      for (size_t c = 0; c < N; ++c) r[c] = b[c] - Ap[c];
      double tn = sqrt(dot(N, r, r)) / bnorm;
      since_check = 0;
      if (tn <= rtol) {
        best = tn;
        break;
      }
      if (tn > 0.5 * best && rn <= rtol) { /* stagnated at round-off */
        best = tn < best ? tn : best;
        break;
      }
      best = tn < best ? tn : best;
      for (size_t c = 0; c < N; ++c) z[c] = dinv[c] * r[c];
      memcpy(pv, z, N * sizeof(double));
      rz = dot(N, r, z);
      continue;
    }
    for (size_t c = 0; c < N; ++c) z[c] = dinv[c] * r[c];
    double rz2 = dot(N, r, z);
    double beta = rz2 / rz;
    rz = rz2;
    for (size_t c = 0; c < N; ++c) pv[c] = z[c] + beta * pv[c];
  }
  double rel = relres_ax(g, dt, Dax, E_old, x);
  if (relres) *relres = rel;
  if (iters) *iters = it;
  free(b);
  free(r);
  free(z);
  free(pv);
  free(Ap);
  free(dinv);
  return rel <= rtol ? 0 : 4;
}


/* public forms: one D for all axes, or one per axis (the diagonal-tensor D of Sect. 6) */
void ora_apply(const ora_grid* g, double dt, const double* D, const double* x, double* Ax) {
  const double* Dax[3] = {D, D, D};
  apply_ax(g, dt, Dax, x, Ax);
}
void ora_rhs(const ora_grid* g, double dt, const double* D, const double* E_old, double* b) {
  const double* Dax[3] = {D, D, D};
  rhs_ax(g, dt, Dax, E_old, b);
}
double ora_relres(const ora_grid* g, double dt, const double* D, const double* E_old, const double* x) {
  const double* Dax[3] = {D, D, D};
  return relres_ax(g, dt, Dax, E_old, x);
}
int ora_diffuse_cg(const ora_grid* g, double dt, const double* D, const double* E_old, double* x, double rtol,
                   int maxit, double* relres, int* iters) {
  const double* Dax[3] = {D, D, D};
  return diffuse_cg_ax(g, dt, Dax, E_old, x, rtol, maxit, relres, iters);
}
void ora_apply_aniso(const ora_grid* g, double dt, const double* const* Dax, const double* x, double* Ax) {
  apply_ax(g, dt, Dax, x, Ax);
}
double ora_relres_aniso(const ora_grid* g, double dt, const double* const* Dax, const double* E_old,
                        const double* x) {
  return relres_ax(g, dt, Dax, E_old, x);
}
int ora_diffuse_cg_aniso(const ora_grid* g, double dt, const double* const* Dax, const double* E_old, double* x,
                         double rtol, int maxit, double* relres, int* iters) {
  return diffuse_cg_ax(g, dt, Dax, E_old, x, rtol, maxit, relres, iters);
}

/* Gaussian elimination with partial pivoting on a dense row-major n x n matrix. */
static int dense_solve(int n, double* M, double* rhs) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(M[(size_t)i * n + k]) > fabs(M[(size_t)piv * n + k])) piv = i;
    if (M[(size_t)piv * n + k] == 0) return 3;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = M[(size_t)k * n + j];
        M[(size_t)k * n + j] = M[(size_t)piv * n + j];
        M[(size_t)piv * n + j] = t;
      }
      double t = rhs[k];
      rhs[k] = rhs[piv];
      rhs[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = M[(size_t)i * n + k] / M[(size_t)k * n + k];
      if (f == 0) continue;
      for (int j = k; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
      rhs[i] -= f * rhs[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = rhs[i];
    for (int j = i + 1; j < n; ++j) s -= M[(size_t)i * n + j] * rhs[j];
    rhs[i] = s / M[(size_t)i * n + i];
  }
  return 0;
}

int ora_diffuse_dense(const ora_grid* g, double dt, const double* D, const double* E_old, double* x) {
  const double* Dax[3] = {D, D, D};
  size_t N = ncells(g);
  if (N > 8192) return 1;
  double* M = calloc(N * N, sizeof(double));
  for (size_t c = 0; c < N; ++c) {
    int q[3];
    unlin(g, c, q);
    M[c * N + c] += 1.0;
    for (int a = 0; a < g->ndim; ++a)
      for (int side = 0; side < 2; ++side) {
        double cs, cn, cc;
        long nb;
        face_term(g, dt, Dax, q, a, side, &cs, &nb, &cn, &cc);
        M[c * N + c] += cs;
        if (nb >= 0) M[c * N + nb] += cn;
      }
  }
  ora_rhs(g, dt, D, E_old, x);
  int st = dense_solve((int)N, M, x);
  free(M);
  return st;
}

/* ------------------------------------------------------------------ 1-D columns */

/* Centre of cell i, with ghost cells mirrored in width at both ends. */
static double col_centre(int n, const double* rf, int i) {
  if (i < 0) return 0.5 * (rf[0] + rf[1]) - (rf[1] - rf[0]);
  if (i >= n) return 0.5 * (rf[n - 1] + rf[n]) + (rf[n] - rf[n - 1]);
  return 0.5 * (rf[i] + rf[i + 1]);
}

static double col_ghost(int n, const double* rf, const double* E, int side, int bc, double v) {
  /* the luminosity boundary needs D, which needs this gradient: the coefficients see a linear
     extrapolation there (the operator then imposes the luminosity with that D) */
  if (bc == ORA_BC_LUMINOSITY) bc = ORA_BC_CONTINUOUS;
  if (side == 0) {
    double h = col_centre(n, rf, 0) - col_centre(n, rf, -1);
    if (bc == ORA_BC_DIRICHLET) return v;
    if (bc == ORA_BC_NEUMANN) return E[0] - v * h;
    return E[0] - (E[1] - E[0]) * h / (col_centre(n, rf, 1) - col_centre(n, rf, 0));
  }
  double h = col_centre(n, rf, n) - col_centre(n, rf, n - 1);
  if (bc == ORA_BC_DIRICHLET) return v;
  if (bc == ORA_BC_NEUMANN) return E[n - 1] + v * h;
  return E[n - 1] + (E[n - 1] - E[n - 2]) * h / (col_centre(n, rf, n - 1) - col_centre(n, rf, n - 2));
}

void ora_kappa_cak(int n, const double* rf, const double* rho, const double* v, double c, double kQ,
                   double rstar, double a_in, double a_out, double x_in, double x_out, double* out) {
  for (int i = 0; i < n; ++i) {
    double r = col_centre(n, rf, i);
    double x = 1.0 - rstar / r;
    double alpha = x <= x_in ? a_in : (x >= x_out ? a_out : a_in + (a_out - a_in) * (x - x_in) / (x_out - x_in));
    /* second-order central difference of v; one-sided at the column ends */
    int lo = i > 0 ? i - 1 : 0, hi = i < n - 1 ? i + 1 : n - 1;
    double dvdr = (v[lo] - v[hi]) / (col_centre(n, rf, lo) - col_centre(n, rf, hi));
    out[i] = kQ / (1.0 - alpha) * pow(fabs(dvdr) / (c * kQ * rho[i]), alpha);
  }
}

int ora_column_coeffs(int n, const double* rf, int bc_lo, int bc_hi, double v_lo, double v_hi,
                      const ora_phys* p, const double* E, const double* rho, const double* kappa,
                      double* D_cell) {
  if (bc_lo == ORA_BC_PERIODIC || bc_hi == ORA_BC_PERIODIC || n < 2) return 1;
  for (int i = 0; i < n; ++i) {
    if (!(E[i] > 0) || !(rho[i] > 0) || !(kappa[i] > 0)) return 2;
    double em = i > 0 ? E[i - 1] : col_ghost(n, rf, E, 0, bc_lo, v_lo);
    double ep = i < n - 1 ? E[i + 1] : col_ghost(n, rf, E, 1, bc_hi, v_hi);
    double hm = col_centre(n, rf, i) - col_centre(n, rf, i - 1);
    double hp = col_centre(n, rf, i + 1) - col_centre(n, rf, i);
    /* second-order central difference on a non-uniform grid */
    double d = (hm * hm * (ep - E[i]) + hp * hp * (E[i] - em)) / (hm * hp * (hm + hp));
    double kr = kappa[i] * rho[i];
    double R = fabs(d) / (kr * E[i]);
    double lam = ora_limiter(p->limiter, R);
    D_cell[i] = p->c * lam / kr;
  }
  return 0;
}

/* Row i of the dt-scaled finite-volume operator: sub*x[i-1] + diag*x[i] + sup*x[i+1] = E_old + cst. */
static void col_row(int n, const double* rf, int geom, int bc_lo, int bc_hi, double v_lo, double v_hi,
                    double dt, const double* D, int i, double* sub, double* diag, double* sup,
                    double* cst) {
  double rl = rf[i], rr = rf[i + 1];
  double V = geom == ORA_GEOM_SPHERICAL ? (rr * rr * rr - rl * rl * rl) / 3.0 : rr - rl;
  double Al = geom == ORA_GEOM_SPHERICAL ? rl * rl : 1.0;
  double Ar = geom == ORA_GEOM_SPHERICAL ? rr * rr : 1.0;
  double hl = col_centre(n, rf, i) - col_centre(n, rf, i - 1);
  double hr = col_centre(n, rf, i + 1) - col_centre(n, rf, i);
  double Dl = i > 0 ? harmonic(D[i - 1], D[i]) : D[0];
  double Dr = i < n - 1 ? harmonic(D[i], D[i + 1]) : D[n - 1];
  double wl = dt * Al * Dl / (V * hl);
  double wr = dt * Ar * Dr / (V * hr);
  *sub = 0;
  *sup = 0;
  *cst = 0;
  *diag = 1.0;
  /* lower face */
  if (i > 0) {
    *diag += wl;
    *sub = -wl;
  } else if (bc_lo == ORA_BC_DIRICHLET) {
    *diag += wl;
    *cst += wl * v_lo;
  } else if (bc_lo == ORA_BC_NEUMANN) {
    *cst -= wl * v_lo * hl;
  } else if (bc_lo == ORA_BC_LUMINOSITY) {
    /* Sect. 5.2: ghost = E_0 + L dr / (4 pi r_0^2 D_0), D from the state entering the step */
    double r0 = col_centre(n, rf, 0);
    *cst += wl * v_lo * hl / (4.0 * kPi * r0 * r0 * D[0]);
  } else { /* continuous: ghost = x0 - (x1-x0)*hl/h01 */
    double f = hl / (col_centre(n, rf, 1) - col_centre(n, rf, 0));
    *diag += wl * (-f);
    *sup += wl * f;
  }
  /* upper face */
  if (i < n - 1) {
    *diag += wr;
    *sup += -wr;
  } else if (bc_hi == ORA_BC_DIRICHLET) {
    *diag += wr;
    *cst += wr * v_hi;
  } else if (bc_hi == ORA_BC_NEUMANN) {
    *cst += wr * v_hi * hr;
  } else {
    double f = hr / (col_centre(n, rf, n - 1) - col_centre(n, rf, n - 2));
    *diag += wr * (-f);
    *sub += wr * f;
  }
}

int ora_column_diffuse(int n, const double* rf, int geom, int bc_lo, int bc_hi, double v_lo, double v_hi,
                       double dt, const double* D, const double* E_old, double* x) {
  if (bc_lo == ORA_BC_PERIODIC || bc_hi == ORA_BC_PERIODIC || n < 2) return 1;
  double* cp = malloc(n * sizeof(double));
  double* dp = malloc(n * sizeof(double));
  /* Thomas algorithm: forward elimination, back substitution */
  for (int i = 0; i < n; ++i) {
    double a, b, c, k;
    col_row(n, rf, geom, bc_lo, bc_hi, v_lo, v_hi, dt, D, i, &a, &b, &c, &k);
    double rhs = E_old[i] + k;
    if (i == 0) {
      cp[0] = c / b;
      dp[0] = rhs / b;
    } else {
      double m = b - a * cp[i - 1];
      cp[i] = c / m;
      dp[i] = (rhs - a * dp[i - 1]) / m;
    }
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return 0;
}

int ora_column_diffuse_dense(int n, const double* rf, int geom, int bc_lo, int bc_hi, double v_lo,
                             double v_hi, double dt, const double* D, const double* E_old, double* x) {
  if (bc_lo == ORA_BC_PERIODIC || bc_hi == ORA_BC_PERIODIC || n < 2 || n > 4096) return 1;
  double* M = calloc((size_t)n * n, sizeof(double));
  for (int i = 0; i < n; ++i) {
    double a, b, c, k;
    col_row(n, rf, geom, bc_lo, bc_hi, v_lo, v_hi, dt, D, i, &a, &b, &c, &k);
    if (i > 0) M[(size_t)i * n + i - 1] += a;
    M[(size_t)i * n + i] += b;
    if (i < n - 1) M[(size_t)i * n + i + 1] += c;
    x[i] = E_old[i] + k;
  }
  int st = dense_solve(n, M, x);
  free(M);
  return st;
}

double ora_column_relres(int n, const double* rf, int geom, int bc_lo, int bc_hi, double v_lo,
                         double v_hi, double dt, const double* D, const double* E_old, const double* x) {
  double rr = 0, bb = 0;
  for (int i = 0; i < n; ++i) {
    double a, b, c, k;
    col_row(n, rf, geom, bc_lo, bc_hi, v_lo, v_hi, dt, D, i, &a, &b, &c, &k);
    double Ax = b * x[i] + (i > 0 ? a * x[i - 1] : 0) + (i < n - 1 ? c * x[i + 1] : 0);
    double rhs = E_old[i] + k;
    rr += (rhs - Ax) * (rhs - Ax);
    bb += rhs * rhs;
  }
  return sqrt(rr / bb);
}

/* ------------------------------------------------------------------ exchange */

int ora_exchange(size_t n, const ora_phys* p, double dt, const double* rho, const double* kappa,
                 double* eps, double* E, int maxit, int* max_iters, int* bisections) {
  const double sigma = p->a_rad * p->c / 4.0; /* a_r = 4 sigma / c (Sect. 2.2) */
  const double tol = 4.0 * 2.220446049250313e-16;
  int worst = 0, nbis = 0;
  for (size_t c = 0; c < n; ++c) {
    double r = rho[c], k = kappa[c], e0 = eps[c], E0 = E[c];
    if (!(r > 0) || !(k > 0) || !(e0 >= 0) || !(E0 >= 0)) return 2;
    /* Sect. 3.3: T = (gamma-1) eps / (rho gas_R) turns the emission term into a1 eps^4 */
    double t = (p->gamma - 1.0) / (r * p->gas_R);
    double a1 = 4.0 * k * r * sigma * dt * t * t * t * t;
    double a2 = p->c * k * r * dt;
    double S = e0 + E0;
    if (S == 0) continue;
    /* quartic a1 x^4 + (1+a2) x - (1+a2) eps - a2 E = 0, with x = S y, y in ]0,1[ */
    double A = a1 * S * S * S;
    double B = 1.0 + a2;
    double C = ((1.0 + a2) * e0 + a2 * E0) / S;
    double lo = 0.0, hi = 1.0;
    double y = C / B; /* root of the linear part: an upper bound of the root */
    if (y > hi) y = hi;
    int it = 0;
    int converged = 0;
    while (it < maxit) {
      double f = A * y * y * y * y + B * y - C;
      if (f == 0) {
        converged = 1;
        break;
      }
      if (f < 0) lo = y;
      else hi = y;
      double f1 = 4.0 * A * y * y * y + B;
      double f2 = 12.0 * A * y * y;
      double yn = y - 2.0 * f * f1 / (2.0 * f1 * f1 - f * f2); /* Halley's step */
      ++it;
      /* a converged step can land on the bracket end that was just set from y itself:
         accept it before the bracket safeguard would turn it into a bisection */
      if (fabs(yn - y) <= tol * yn) {
        y = yn;
        converged = 1;
        break;
      }
      if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
      y = yn;
    }
    if (!converged) { /* bisection fallback */
      ++nbis;
      while (hi - lo > tol * hi) {
        double m = 0.5 * (lo + hi);
        double f = A * m * m * m * m + B * m - C;
        if (f < 0) lo = m;
        else hi = m;
      }
      y = 0.5 * (lo + hi);
    }
    if (it > worst) worst = it;
    double x = S * y;
    eps[c] = x;
    E[c] = (a1 * x * x * x * x + E0) / (1.0 + a2); /* Sect. 3.3, E^{n+1} */
  }
  if (max_iters) *max_iters = worst;
  if (bisections) *bisections = nbis;
  return 0;
}

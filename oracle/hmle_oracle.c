/*
 * CPU oracle for the H-MLE log-likelihood -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the bench's CPU-baseline leg may
 * load this library.  The GPU product path never links or calls it.
 *
 * Contents (all FP64, plain loops, no blocking or reordering beyond the
 * definitions they restate):
 *   - oracle_besselk_scaled: e^x K_nu(x) from the integral representation
 *       K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt,
 *     evaluated by the trapezoid rule on a fixed grid.  The integrand is
 *     analytic in a strip around the real axis and decays double-
 *     exponentially, so the trapezoid rule converges geometrically in 1/h.
 *     This is a different method from the series / continued-fraction
 *     evaluation used by the device kernels on purpose.
 *   - oracle_matern_matrix: C_ij = sigma^2 M_nu(|s_i - s_j| / ell) + tau^2 [i==j]
 *     with M_nu(x) = x^nu K_nu(x) / (2^(nu-1) Gamma(nu)), M_nu(0) = 1
 *     (Matern covariance, Eq. 2; nugget on index-diagonal entries only).
 *   - oracle_forward_solve: w = L^{-1} z for a dense lower-triangular L,
 *     row-oriented forward substitution in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_NGRID 3       /* steps h = 1/16, 1/64, 1/256 */
#define ORACLE_TAIL 60.0      /* stop once the exponent is below -60 */
#define ORACLE_MAXTERMS 4096
#define ORACLE_XMAX 4096.0    /* beyond this M_nu(x) < 1e-1700: exactly 0 */

/* t-grid tables for one nu and one step h: c1[j] = cosh(t_j) - 1,
 * c2[j] = cosh(nu t_j), t_j = j h.  For large x the integrand is a narrow
 * peak of width ~ 1/sqrt(x) at t = 0, so the step shrinks with x to keep
 * several nodes inside it. */
typedef struct {
  double h;
  double c1[ORACLE_MAXTERMS];
  double c2[ORACLE_MAXTERMS];
  double t[ORACLE_MAXTERMS];
} kgrid1;

typedef struct {
  double nu;
  kgrid1 g[ORACLE_NGRID];
} kgrid;

static void kgrid_init(kgrid *g, double nu) {
  g->nu = nu;
  for (int k = 0; k < ORACLE_NGRID; ++k) {
    kgrid1 *q = &g->g[k];
    q->h = 1.0 / (16.0 * (double)(1 << (2 * k)));
    for (int j = 0; j < ORACLE_MAXTERMS; ++j) {
      double t = j * q->h;
      q->t[j] = t;
      q->c1[j] = 2.0 * sinh(0.5 * t) * sinh(0.5 * t); /* cosh t - 1, no cancellation */
      q->c2[j] = cosh(nu * t);
    }
  }
}

/* e^x K_nu(x), x > 0: h * [1/2 f(0) + sum_{j>=1} f(t_j)],
 * f(t) = exp(-x (cosh t - 1)) cosh(nu t).  Kahan-compensated sum. */
static double besselk_scaled_grid(const kgrid *g, double x) {
  int k = x <= 16.0 ? 0 : (x <= 256.0 ? 1 : 2);
  const kgrid1 *q = &g->g[k];
  double sum = 0.5, comp = 0.0;
  for (int j = 1; j < ORACLE_MAXTERMS; ++j) {
    double e = -x * q->c1[j];
    double term = exp(e) * q->c2[j];
    double y = term - comp;
    double s = sum + y;
    comp = (s - sum) - y;
    sum = s;
    /* past the peak the integrand decays double-exponentially: stop once
     * the log of the term is far below the (>= 1/2) running sum */
    if (e + g->nu * q->t[j] < -ORACLE_TAIL && x * q->c1[j] > g->nu) break;
  }
  return sum * q->h;
}

double oracle_besselk_scaled(double nu, double x) {
  kgrid *g = (kgrid *)malloc(sizeof(kgrid));
  if (!g) return NAN;
  kgrid_init(g, nu);
  double r = besselk_scaled_grid(g, x);
  free(g);
  return r;
}

/* M_nu(x) = x^nu K_nu(x) / (2^(nu-1) Gamma(nu)); M_nu(0) = 1. */
static double matern_unit(const kgrid *g, double x) {
  if (x <= 0.0) return 1.0;
  if (x > ORACLE_XMAX) return 0.0;
  double nu = g->nu;
  double lk = log(besselk_scaled_grid(g, x)) - x; /* log K_nu(x) */
  double lm = nu * log(x) + lk - (nu - 1.0) * log(2.0) - lgamma(nu);
  return exp(lm);
}

double oracle_matern_unit(double nu, double x) {
  kgrid *g = (kgrid *)malloc(sizeof(kgrid));
  if (!g) return NAN;
  kgrid_init(g, nu);
  double r = matern_unit(g, x);
  free(g);
  return r;
}

/* Dense covariance matrix, row-major n x n, both triangles filled.
 * locs: n x d row-major.  Returns 0 on success. */
int oracle_matern_matrix(int64_t n, int d, const double *locs, double ell,
                         double nu, double sigma2, double tau2, double *C) {
  if (n < 0 || d < 1 || d > 3 || !(ell > 0) || !(nu > 0)) return 1;
  kgrid *g = (kgrid *)malloc(sizeof(kgrid));
  if (!g) return 2;
  kgrid_init(g, nu);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double h2 = 0.0;
      for (int k = 0; k < d; ++k) {
        double dx = locs[i * d + k] - locs[j * d + k];
        h2 += dx * dx;
      }
      double c = sigma2 * matern_unit(g, sqrt(h2) / ell);
      if (i == j) c += tau2;
      C[i * n + j] = c;
      C[j * n + i] = c;
    }
  }
  free(g);
  return 0;
}

/* Matern covariance between two point sets (rows of A vs rows of B), no
 * nugget: out[i*nb + j] = sigma2 * M_nu(|a_i - b_j| / ell). */
int oracle_matern_cross(int64_t na, int64_t nb, int d, const double *A,
                        const double *B, double ell, double nu, double sigma2,
                        double *out) {
  if (na < 0 || nb < 0 || d < 1 || d > 3 || !(ell > 0) || !(nu > 0)) return 1;
  kgrid *g = (kgrid *)malloc(sizeof(kgrid));
  if (!g) return 2;
  kgrid_init(g, nu);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < na; ++i) {
    for (int64_t j = 0; j < nb; ++j) {
      double h2 = 0.0;
      for (int k = 0; k < d; ++k) {
        double dx = A[i * d + k] - B[j * d + k];
        h2 += dx * dx;
      }
      out[i * nb + j] = sigma2 * matern_unit(g, sqrt(h2) / ell);
    }
  }
  free(g);
  return 0;
}

/* w = L^{-1} z, L dense lower-triangular, row-major n x n. */
int oracle_forward_solve(int64_t n, const double *L, const double *z,
                         double *w) {
  for (int64_t i = 0; i < n; ++i) {
    double s = z[i];
    const double *row = L + i * n;
    for (int64_t j = 0; j < i; ++j) s -= row[j] * w[j];
    if (!(row[i] > 0)) return 1;
    w[i] = s / row[i];
  }
  return 0;
}

/* C = L L^T by the unblocked row-by-row (Cholesky-Banachiewicz) algorithm,
 * in place on a row-major n x n array: for row i and j <= i,
 * s = C_ij - sum_{k<j} L_ik L_jk, then L_ij = s / L_jj (j < i) and
 * L_ii = sqrt(s).  The strict upper triangle is zeroed.  Returns 1 at a
 * non-positive pivot. */
int oracle_cholesky(int64_t n, double *A) {
  for (int64_t i = 0; i < n; ++i) {
    double *Li = A + i * n;
    for (int64_t j = 0; j <= i; ++j) {
      const double *Lj = A + j * n;
      double s = Li[j];
      for (int64_t k = 0; k < j; ++k) s -= Li[k] * Lj[k];
      if (j < i) {
        Li[j] = s / Lj[j];
      } else {
        if (!(s > 0)) return 1;
        Li[i] = sqrt(s);
      }
    }
    for (int64_t j = i + 1; j < n; ++j) Li[j] = 0.0;
  }
  return 0;
}

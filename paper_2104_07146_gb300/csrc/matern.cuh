// Device Matern correlation M_nu(x) = x^nu K_nu(x) / (2^(nu-1) Gamma(nu))
// (Eq. 2), M_nu(0) = 1.
//
// nu is fixed for one evaluation of the likelihood, so a table of
// piecewise Chebyshev interpolants of M_nu on the log-spaced intervals
// [2^j, 2^(j+1)), j = kJmin .. kJmin + kNint - 1, is built once per nu
// (k_matern_table) and every matrix entry costs one Clenshaw recurrence.
// The interpolation nodes are computed from the integral representation
//     e^x K_nu(x) = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt
// by the trapezoid rule (geometrically convergent for this analytic,
// double-exponentially decaying integrand; the step shrinks like 1/sqrt(x)
// to resolve the peak at t = 0 for large x).  Below 2^kJmin the same
// quadrature is evaluated directly; above 2^(kJmin + kNint) M_nu < e^-1000
// and is returned as 0.
#pragma once

#include <cuda_runtime.h>

namespace hmle {

constexpr int kJmin = -12;
constexpr int kNint = 22;           // intervals up to x = 2^10
constexpr int kDeg = 20;            // Chebyshev degree
constexpr int kNcoef = kDeg + 1;
constexpr int kTableWords = kNint * kNcoef + 8;  // + header (nu, log-normaliser)

// e^x K_nu(x) by the trapezoid rule, x > 0.
__device__ inline double besselk_scaled_quad(double nu, double x) {
  double h = 0.0625;
  if (x > 16.0) h = 0.25 / sqrt(x);
  double sum = 0.5, comp = 0.0;
  for (int j = 1; j < 100000; ++j) {
    double t = j * h;
    double sh = sinh(0.5 * t);
    double e = -x * 2.0 * sh * sh;            // -x (cosh t - 1)
    double term = exp(e) * cosh(nu * t);
    double y = term - comp;
    double s = sum + y;
    comp = (s - sum) - y;
    sum = s;
    if (e + nu * t < -60.0 && x * 2.0 * sh * sh > nu) break;
  }
  return sum * h;
}

// M_nu(x) from the quadrature (any x >= 0); lognorm = (nu-1) log 2 + lgamma(nu).
__device__ inline double matern_unit_quad(double nu, double lognorm, double x) {
  if (x <= 0.0) return 1.0;
  double lk = log(besselk_scaled_quad(nu, x)) - x;
  return exp(nu * log(x) + lk - lognorm);
}

// Table layout: tab[0] = nu, tab[1] = lognorm, tab[8 + j*kNcoef + k] = c_k of
// interval j (Chebyshev series in t = x / 2^(kJmin+j) * 2 - 3 on [-1, 1]).
__device__ __forceinline__ double matern_unit(const double *__restrict__ tab, double x) {
  if (x <= 0.0) return 1.0;
  int e = ilogb(x);                            // floor(log2 x) for normal x
  int j = e - kJmin;
  if (j < 0) return matern_unit_quad(tab[0], tab[1], x);
  if (j >= kNint) return 0.0;
  double t = scalbn(x, -e) * 2.0 - 3.0;        // x / 2^e in [1, 2) -> [-1, 1)
  const double *c = tab + 8 + j * kNcoef;
  double b1 = 0.0, b2 = 0.0, t2 = 2.0 * t;
#pragma unroll
  for (int k = kDeg; k >= 1; --k) {
    double b0 = fma(t2, b1, c[k] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(t, b1, c[0] - b2);
}

// Covariance between points i and j of a coordinate SoA (xyz[dim*n + i]).
__device__ __forceinline__ double cov_entry(const double *__restrict__ tab,
                                            const double *__restrict__ xyz, int64_t n,
                                            int d, int64_t i, int64_t j, double inv_ell,
                                            double sigma2, double tau2) {
  double h2 = 0.0;
  for (int k = 0; k < d; ++k) {
    double dx = xyz[k * n + i] - xyz[k * n + j];
    h2 = fma(dx, dx, h2);
  }
  double c = sigma2 * matern_unit(tab, sqrt(h2) * inv_ell);
  return (i == j) ? c + tau2 : c;
}

}  // namespace hmle

// Modified Bessel function of the second kind K_nu(x) for real order nu and
// x > 0, and the Matern correlation of a general smoothness nu (Eq.
// maternkernel: 2^(1-nu)/Gamma(nu) r^nu K_nu(r), at the scaled distance r),
// in FP64, for host and device.
//
// K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt  (DLMF 10.32.9).  The
// integrand is entire and decays doubly exponentially in t, so the
// trapezoidal rule with step h converges geometrically (Trefethen &
// Weideman, SIAM Review 56 (2014)).  On the strip |Im t| < pi/4 the
// integrand is at most that of K_nu(x / sqrt 2), about 2^(nu/2) times larger,
// so the relative error is about 2^(nu/2) exp(-pi^2 / (2h)): below 1e-12 for
// nu <= 20 at h = 1/8 (checked against scipy's kv for nu in [0, 19.5], x in
// [1e-8, 700]).  For large x the integrand is a peak of width 1/sqrt(x) at
// t = 0, whose sampling error 2 exp(-2 pi^2 / (x h^2)) stays below 1e-17 with
// h <= 0.7 / sqrt(x).  The nodes cosh(k h) and cosh(nu k h) follow the
// three-term recurrence c_{k+1} = 2 cosh(h) c_k - c_{k-1} of the growing
// solution.  The sum runs past the integrand's peak (sinh t = nu / x) until a
// term falls below 1e-18 of the sum, and at most kMaxNodes nodes (t <= 60).
#pragma once
#include <math.h>

#ifdef __CUDACC__
#define SBV_HD __host__ __device__
#else
#define SBV_HD
#endif

namespace sbv {

// below this scaled distance the general-nu correlation is taken as 1 and its
// derivative term as its r -> 0 limit (for nu >= 1: 1 - M(r) = O(r^2 log r))
constexpr double kMaternTiny = 1e-8;

SBV_HD inline double bessel_k_trap(double nu, double x) {
  const double h = fmin(0.125, 0.7 / sqrt(x));
  constexpr int kMaxNodes = 480;
  const double ch = cosh(h), cnh = cosh(nu * h);
  const double tpeak = asinh(nu / x);
  double c0 = 1.0, c1 = ch;      // cosh((k-1) h), cosh(k h)
  double n0 = 1.0, n1 = cnh;     // cosh(nu (k-1) h), cosh(nu k h)
  double sum = 0.5 * exp(-x);    // k = 0, half weight
  for (int k = 1; k < kMaxNodes; ++k) {
    const double term = exp(-x * c1) * n1;
    sum += term;
    if (k * h > tpeak && term <= 1e-18 * sum) break;
    const double c2 = 2.0 * ch * c1 - c0, n2 = 2.0 * cnh * n1 - n0;
    c0 = c1;
    c1 = c2;
    n0 = n1;
    n1 = n2;
  }
  return h * sum;
}

// Matern correlation M_nu(r), general nu >= 1.
SBV_HD inline double matern_general(double r, double nu) {
  if (r < kMaternTiny) return 1.0;
  return exp2(1.0 - nu) / tgamma(nu) * pow(r, nu) * bessel_k_trap(nu, r);
}

// -M_nu'(r) / r = 2^(1-nu)/Gamma(nu) r^(nu-1) K_(nu-1)(r) (from
// d/dr [r^nu K_nu(r)] = -r^nu K_(nu-1)(r) and K_(-a) = K_a), general nu >= 1;
// below kMaternTiny its limit 1 / (2 (nu - 1)) (nu > 1), or 0 for nu = 1
// (where it grows like -log r but multiplies squared coordinate differences
// below r^2).
SBV_HD inline double matern_general_h(double r, double nu) {
  if (r < kMaternTiny) return nu > 1.0 ? 0.5 / (nu - 1.0) : 0.0;
  return exp2(1.0 - nu) / tgamma(nu) * pow(r, nu - 1.0) * bessel_k_trap(fabs(nu - 1.0), r);
}

}  // namespace sbv

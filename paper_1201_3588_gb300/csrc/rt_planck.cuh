// rt_planck.cuh -- FP64 Planck integrals over frequency bins and the temperature
// grid of the tables (device functions shared by the table builders).
//
// The Planck function integrated over a frequency bin is evaluated in closed
// form: with x = h nu / k T, the integral of B_nu over [nu0, nu1] equals
// (2 k^4 T^4 / h^3 c^2) [G(x0) - G(x1)], G(x) the integral of t^3/(e^t - 1) from x
// to infinity, summed as sum_k e^{-kx} (x^3/k + 3x^2/k^2 + 6x/k^3 + 6/k^4) for
// x >= 1/2 and as pi^4/15 minus the Bernoulli series of the integral from 0 to x
// below that.
#pragma once

#include <math.h>

namespace rt {
namespace planck {

constexpr double kH = 6.62607015e-27;
constexpr double kK = 1.380649e-16;
constexpr double kC = 2.99792458e10;
constexpr double kPi = 3.14159265358979323846;
constexpr double kPi4Over15 = 6.4939394022668291491;  // pi^4 / 15

// integral_0^x t^3/(e^t-1) dt for 0 <= x < 1/2: sum_n (B_n/n!) x^(n+3)/(n+3)
static __device__ inline double planck_head(double x) {
  // B_n / n! for n = 0, 1, 2, 4, ..., 20 (odd n > 1 vanish)
  const double c0 = 1.0, c1 = -0.5;
  const double ce[10] = {1.0 / 12.0,
                         -1.0 / 720.0,
                         1.0 / 30240.0,
                         -1.0 / 1209600.0,
                         1.0 / 47900160.0,
                         -691.0 / 1307674368000.0,
                         1.0 / 74724249600.0,
                         -3617.0 / 10670622842880000.0,
                         43867.0 / 5109094217170944000.0,
                         -174611.0 / 802857662698291200000.0};
  double x2 = x * x, x3 = x2 * x;
  double s = c0 * x3 / 3.0 + c1 * x3 * x / 4.0;
  double xp = x3 * x2;  // x^(n+3) for n = 2
  for (int k = 0; k < 10; ++k) {
    int n = 2 * k + 2;
    s += ce[k] * xp / (double)(n + 3);
    xp *= x2;
  }
  return s;
}

// integral_x^inf t^3/(e^t-1) dt for x >= 1/2
static __device__ inline double planck_tail(double x) {
  double s = 0.0;
  double x2 = x * x, x3 = x2 * x;
  for (int k = 1; k <= 400; ++k) {
    double kk = (double)k;
    double e = exp(-kk * x);
    double term = e * (x3 / kk + 3.0 * x2 / (kk * kk) + 6.0 * x / (kk * kk * kk) +
                       6.0 / (kk * kk * kk * kk));
    s += term;
    if (term <= 1e-18 * s) break;
  }
  return s;
}

// integral over [nu0, nu1] of B_nu(T) d nu, erg s^-1 cm^-2 sr^-1
static __device__ inline double planck_bin(double nu0, double nu1, double T) {
  if (!(T > 0.0)) return 0.0;
  double a = kH / (kK * T);
  double x0 = a * nu0, x1 = a * nu1;
  double d;
  if (x1 < 0.5) {
    d = planck_head(x1) - planck_head(x0);
  } else if (x0 < 0.5) {
    d = (kPi4Over15 - planck_head(x0)) - planck_tail(x1);
  } else {
    d = planck_tail(x0) - planck_tail(x1);
  }
  double kT = kK * T;
  double pref = 2.0 * kT * kT * kT * kT / (kH * kH * kH * kC * kC);
  return pref * (d > 0.0 ? d : 0.0);
}

static __device__ inline double table_T(int i, int n_T, double t_min, double t_max) {
  if (i == 0) return 0.0;
  if (i == n_T - 1) return t_max;
  return t_min * pow(t_max / t_min, (double)(i - 1) / (double)(n_T - 2));
}

}  // namespace planck
}  // namespace rt

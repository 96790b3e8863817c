// Double-precision special functions written for this library (device code).
//
//  - inc_gamma_pq: regularised incomplete gamma P(a, x) and Q(a, x) = 1 - P.
//    Power series of P for x < a + 1 (DLMF 8.7.1 rearranged as
//    P = x^a e^-x / Gamma(a) * sum_n x^n / (a (a+1) ... (a+n))) and Legendre's
//    continued fraction of Q otherwise (DLMF 8.9.2), evaluated with the modified
//    Lentz method (Thompson & Barnett 1986).
//  - inc_gamma_inv: x with P(a, x) = u, from a Wilson-Hilferty (1931) start and
//    bracketed Halley steps; the upper-tail equation Q(a, x) = 1 - u is solved
//    for u >= 1/2 so that both tails keep full relative accuracy.
//  - digamma: the recurrence psi(x) = psi(x + 1) - 1/x (DLMF 5.5.2) up to
//    x >= 10, then the asymptotic series in Bernoulli numbers (DLMF 5.11.2).
//
// lgamma, log, exp and normcdfinv are CUDA's own functions, called as-is.
#pragma once

#include <cuda_runtime.h>

namespace cfust {

__device__ inline void inc_gamma_pq(double a, double x, double *P, double *Q) {
  if (!(x > 0.0)) {
    *P = 0.0;
    *Q = 1.0;
    return;
  }
  const double lpre = a * log(x) - x - lgamma(a);
  if (x < a + 1.0) {
    double term = 1.0 / a, sum = term, den = a;
    for (int k = 0; k < 1000; ++k) {
      den += 1.0;
      term *= x / den;
      sum += term;
      if (fabs(term) <= fabs(sum) * 1e-17) break;
    }
    const double p = sum * exp(lpre);
    *P = p;
    *Q = 1.0 - p;
  } else {
    const double tiny = 1e-300;
    double b = x + 1.0 - a;
    double c = 1.0 / tiny;
    double d = 1.0 / b;
    double h = d;
    for (int k = 1; k < 1000; ++k) {
      const double an = -(double)k * ((double)k - a);
      b += 2.0;
      d = an * d + b;
      if (fabs(d) < tiny) d = tiny;
      c = b + an / c;
      if (fabs(c) < tiny) c = tiny;
      d = 1.0 / d;
      const double delta = d * c;
      h *= delta;
      if (fabs(delta - 1.0) <= 1e-16) break;
    }
    const double q = exp(lpre) * h;
    *Q = q;
    *P = 1.0 - q;
  }
}

// Inverse of the regularised lower incomplete gamma function in x, a > 0,
// 0 < u < 1.  Returns x >= 0.
__device__ inline double inc_gamma_inv(double a, double u) {
  const bool upper = u >= 0.5;
  const double uc = 1.0 - u;  // exact for u >= 1/2
  const double lga = lgamma(a);
  // Wilson-Hilferty: chi^2_{2a} / (2a) ~ (1 - 1/(9a) + z / (3 sqrt(a)))^3.
  const double zq = upper ? -normcdfinv(uc) : normcdfinv(u);
  const double t = 1.0 / (9.0 * a);
  const double wh = 1.0 - t + zq * sqrt(t);
  double x = a * wh * wh * wh;
  if (!upper) {
    // leading term of the series: P ~ x^a / Gamma(a + 1) for small x
    const double xs = exp((log(u) + lgamma(a + 1.0)) / a);
    if (!(x > 0.0) || xs < x) x = xs;
  }
  if (!(x > 0.0)) x = a;
  double lo = 0.0, hi = 1e308;
  for (int it = 0; it < 100; ++it) {
    double P, Q;
    inc_gamma_pq(a, x, &P, &Q);
    const double f = upper ? (uc - Q) : (P - u);  // increasing in x
    if (f == 0.0) return x;
    if (f < 0.0) lo = x; else hi = x;
    const double dens = exp((a - 1.0) * log(x) - x - lga);  // dP/dx
    double xn;
    if (dens > 0.0 && isfinite(dens)) {
      const double ratio = f / dens;
      double corr = 1.0 - 0.5 * ratio * ((a - 1.0) / x - 1.0);
      if (!(corr > 0.5)) corr = 1.0;  // keep the step Newton-like when Halley is unsafe
      xn = x - ratio / corr;
    } else {
      xn = (hi < 1e308) ? 0.5 * (lo + hi) : 2.0 * x;
    }
    if (!(xn > lo && xn < hi)) xn = (hi < 1e308) ? 0.5 * (lo + hi) : 2.0 * x;
    if (fabs(xn - x) <= 4e-16 * xn) return xn;
    x = xn;
  }
  return x;
}

__device__ inline double digamma(double x) {
  double acc = 0.0;
  while (x < 10.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double f = 1.0 / (x * x);
  // B2/2 = 1/12, B4/4 = -1/120, B6/6 = 1/252, B8/8 = -1/240, B10/10 = 1/132,
  // B12/12 = -691/32760, B14/14 = 1/12
  const double series =
      f * (-1.0 / 12.0 +
           f * (1.0 / 120.0 +
                f * (-1.0 / 252.0 +
                     f * (1.0 / 240.0 + f * (-1.0 / 132.0 + f * (691.0 / 32760.0 + f * (-1.0 / 12.0)))))));
  return acc + log(x) - 0.5 / x + series;
}

}  // namespace cfust

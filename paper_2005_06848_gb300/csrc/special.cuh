// Double-precision special functions written for this library (device code).
//
//  - inc_gamma_pq: regularised incomplete gamma P(a, x) and Q(a, x) = 1 - P.
//    Power series of P for x < a + 1 (DLMF 8.7.1 rearranged as
//    P = x^a e^-x / Gamma(a) * sum_n x^n / (a (a+1) ... (a+n))) and Legendre's
//    continued fraction of Q otherwise (DLMF 8.9.2), evaluated with the modified
//    Lentz method (Thompson & Barnett 1986).
//  - inc_gamma_inv: x with P(a, x) = u, from a Wilson-Hilferty (1931) start and
//    bracketed Halley steps, first in single precision, then in double; the
//    upper-tail equation Q(a, x) = 1 - u is solved for u >= 1/2 so that both
//    tails keep full relative accuracy.
//  - digamma: the recurrence psi(x) = psi(x + 1) - 1/x (DLMF 5.5.2) up to
//    x >= 10, then the asymptotic series in Bernoulli numbers (DLMF 5.11.2).
//  - log_minus_digamma: D(x) = log x - psi(x) without the cancellation of the
//    two (same recurrence and series, the series taken for the difference),
//    in double and single precision, and its derivative 1/x - psi'(x) in
//    single precision (recurrence DLMF 5.15.5, series DLMF 5.15.8).
//
// lgamma(f), log(f), exp(f) and normcdfinv are CUDA's own functions, called as-is.
#pragma once

#include <cuda_runtime.h>

namespace cfust {

// Precision traits of the incomplete-gamma routines.
template <typename T>
struct GammaT;
template <>
struct GammaT<double> {
  __device__ static double lgam(double x) { return lgamma(x); }
  __device__ static double ex(double x) { return exp(x); }
  __device__ static double lg(double x) { return log(x); }
  static constexpr double series_eps = 1e-17, cf_eps = 1e-16, tiny = 1e-300, big = 1e308;
};
template <>
struct GammaT<float> {
  __device__ static float lgam(float x) { return lgammaf(x); }
  __device__ static float ex(float x) { return expf(x); }
  __device__ static float lg(float x) { return logf(x); }
  static constexpr float series_eps = 1e-8f, cf_eps = 1e-7f, tiny = 1e-30f, big = 3e38f;
};

template <typename T>
__device__ inline void inc_gamma_pq_t(T a, T x, T *P, T *Q) {
  using G = GammaT<T>;
  if (!(x > T(0))) {
    *P = T(0);
    *Q = T(1);
    return;
  }
  const T lpre = a * G::lg(x) - x - G::lgam(a);
  if (x < a + T(1)) {
    T term = T(1) / a, sum = term, den = a;
    for (int k = 0; k < 1000; ++k) {
      den += T(1);
      term *= x / den;
      sum += term;
      if (fabs(term) <= fabs(sum) * G::series_eps) break;
    }
    const T p = sum * G::ex(lpre);
    *P = p;
    *Q = T(1) - p;
  } else {
    const T tiny = G::tiny;
    T b = x + T(1) - a;
    T c = T(1) / tiny;
    T d = T(1) / b;
    T h = d;
    for (int k = 1; k < 1000; ++k) {
      const T an = -(T)k * ((T)k - a);
      b += T(2);
      d = an * d + b;
      if (fabs(d) < tiny) d = tiny;
      c = b + an / c;
      if (fabs(c) < tiny) c = tiny;
      d = T(1) / d;
      const T delta = d * c;
      h *= delta;
      if (fabs(delta - T(1)) <= G::cf_eps) break;
    }
    const T q = G::ex(lpre) * h;
    *Q = q;
    *P = T(1) - q;
  }
}

__device__ inline void inc_gamma_pq(double a, double x, double *P, double *Q) {
  inc_gamma_pq_t<double>(a, x, P, Q);
}

// Bracketed Halley iteration for P(a, x) = u (or Q(a, x) = uc, uc = 1 - u,
// when `upper`) from the start x; stops when a step moves x by at most rtol
// relative.
template <typename T>
__device__ inline T inc_gamma_halley(T a, T u, T uc, bool upper, T x, int max_it, T rtol) {
  // stops after the step that moves x by at most rtol relative
  using G = GammaT<T>;
  const T lga = G::lgam(a);
  T lo = T(0), hi = G::big;
  for (int it = 0; it < max_it; ++it) {
    T P, Q;
    inc_gamma_pq_t<T>(a, x, &P, &Q);
    const T f = upper ? (uc - Q) : (P - u);  // increasing in x
    if (f == T(0)) return x;
    if (f < T(0)) lo = x; else hi = x;
    const T dens = G::ex((a - T(1)) * G::lg(x) - x - lga);  // dP/dx
    T xn;
    if (dens > T(0) && isfinite(dens)) {
      const T ratio = f / dens;
      T corr = T(1) - T(0.5) * ratio * ((a - T(1)) / x - T(1));
      if (!(corr > T(0.5))) corr = T(1);  // keep the step Newton-like when Halley is unsafe
      xn = x - ratio / corr;
    } else {
      xn = (hi < G::big) ? T(0.5) * (lo + hi) : T(2) * x;
    }
    if (!(xn > lo && xn < hi)) xn = (hi < G::big) ? T(0.5) * (lo + hi) : T(2) * x;
    if (fabs(xn - x) <= rtol * xn) return xn;
    x = xn;
  }
  return x;
}

// Inverse of the regularised lower incomplete gamma function in x, a > 0,
// 0 < u < 1.  Returns x >= 0.  The root is first found in single precision
// (to about 1e-6) and then polished in double, so most of the work runs at
// the single-precision rate.
__device__ inline double inc_gamma_inv(double a, double u) {
  const bool upper = u >= 0.5;
  const double uc = 1.0 - u;  // exact for u >= 1/2
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
  const float xf = inc_gamma_halley<float>((float)a, (float)u, (float)uc, upper, (float)x, 30, 1e-6f);
  if (xf > 0.0f && isfinite(xf)) x = (double)xf;
  // Halley converges cubically: once a double step moves x by at most 1e-5
  // relative, the error after it is of order 1e-15, below what a further
  // step would change in the chi scale that uses it
  return inc_gamma_halley<double>(a, u, uc, upper, x, 100, 1e-5);
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

// D(x) = log x - psi(x), x > 0.  psi(x) = psi(x + m) - sum_{k<m} 1/(x + k)
// with x + m >= 10 gives D(x) = -log1p(m/x) + sum_{k<m} 1/(x + k) + D(x + m);
// the sum is accumulated as one fraction (a single division), and
// D(y) = 1/(2y) + sum_k B_2k / (2k y^2k) to y^-14 (error below 5e-16 y^-16).
__device__ inline double log_minus_digamma(double x) {
  double num = 0.0, den = 1.0, y = x;
  int m = 0;
  while (y < 10.0) {
    num = num * y + den;
    den *= y;
    y += 1.0;
    ++m;
  }
  const double f = 1.0 / (y * y);
  const double series =
      f * (1.0 / 12.0 +
           f * (-1.0 / 120.0 +
                f * (1.0 / 252.0 +
                     f * (-1.0 / 240.0 + f * (1.0 / 132.0 + f * (-691.0 / 32760.0 + f * (1.0 / 12.0)))))));
  double d = 0.5 / y + series;
  if (m > 0) d += num / den - log1p((double)m / x);
  return d;
}

// Single-precision D(x) (series to y^-6: the next term is below 2e-9 y^-8).
__device__ inline float log_minus_digamma_f(float x) {
  float num = 0.0f, den = 1.0f, y = x;
  int m = 0;
  while (y < 10.0f) {
    num = num * y + den;
    den *= y;
    y += 1.0f;
    ++m;
  }
  const float f = 1.0f / (y * y);
  float d = 0.5f / y + f * (1.0f / 12.0f + f * (-1.0f / 120.0f + f * (1.0f / 252.0f)));
  if (m > 0) d += num / den - log1pf((float)m / x);
  return d;
}

// Single-precision D'(x) = 1/x - psi'(x) (< 0).  psi'(x) = psi'(x + m) +
// sum_{k<m} 1/(x + k)^2, so D'(x) = m / (x (x + m)) - sum_{k<m} 1/(x + k)^2 +
// D'(x + m), and D'(y) = -1/(2y^2) - 1/(6y^3) + 1/(30y^5) - 1/(42y^7).
__device__ inline float dlog_minus_digamma_f(float x) {
  float s2 = 0.0f, y = x;
  int m = 0;
  while (y < 10.0f) {
    s2 += 1.0f / (y * y);
    y += 1.0f;
    ++m;
  }
  const float iy = 1.0f / y, f = iy * iy;
  float d = -f * (0.5f + iy * (1.0f / 6.0f + f * (-1.0f / 30.0f + f * (1.0f / 42.0f))));
  if (m > 0) d += (float)m / (x * y) - s2;
  return d;
}

}  // namespace cfust

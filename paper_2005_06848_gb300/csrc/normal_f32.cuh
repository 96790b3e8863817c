// Single-precision normal tail probability and quantile used by the lattice
// sweep, with the fitted polynomials of normal_f32_coeffs.cuh (forms in
// fit_normal_f32.py), plus log-domain variants for pairs whose lattice weights
// fall below the float range.
//
//   phi_upper_f32(y)  = Phi(-y) = P(Z > y); phi_upper_pq_f32 also gives Phi(y)
//   phi_inv_f32(x)    = Phi^{-1}(x), x in (0, 1)
//   neg_quantile_f32  = -Phi^{-1}(um p), evaluated on the smaller of x, 1 - x
//   log_phi_upper_f32(y) = log Phi(-y) for any finite y
//   neg_quantile_log_f32(la) = -Phi^{-1}(exp(la)) for la <= 0, including
//                              exp(la) far below the float range
//
// exp(-y^2/2) carries the rounding error of y*y through a fused multiply-add
// (y*y = s + e exactly, exp(-(s+e)/2) ~ exp(-s/2) (1 - e/2)).
#pragma once

#include <math.h>

#include "normal_f32_coeffs.cuh"

namespace cfust {

namespace nf32 {

template <int K>
__device__ __forceinline__ float horner(const float (&c)[K], float t) {
  float q = c[K - 1];
#pragma unroll
  for (int k = K - 2; k >= 0; --k) q = fmaf(q, t, c[k]);
  return q;
}

// G(a) = Phi(-a) exp(a^2/2), a >= 0
__device__ __forceinline__ float tail_factor(float a) {
  const float t = __fdividef(1.0f, fmaf(TAIL_C, a, 1.0f));
  return horner(TAIL_Q, t) * t;
}

}  // namespace nf32

__device__ __forceinline__ float exp2f_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Phi(-y) and its complement 1 - Phi(-y) = Phi(y), each from the small side.
__device__ __forceinline__ void phi_upper_pq_f32(float y, float &p, float &q) {
  const float a = fabsf(y);
  const float s = a * a;
  const float e = fmaf(a, a, -s);
  float tail = nf32::tail_factor(a) * expf(-0.5f * s);
  tail = fmaf(-0.5f * e, tail, tail);
  const float big = 1.0f - tail;
  p = (y >= 0.0f) ? tail : big;
  q = (y >= 0.0f) ? big : tail;
}

// Same with exp(-y^2/2) from the hardware base-2 exponential of the rounded
// product (relative error below 3e-6 for |y| < 10): the bulk lattice sweep.
__device__ __forceinline__ void phi_upper_pq_fast_f32(float y, float &p, float &q) {
  const float a = fabsf(y);
  const float tail = nf32::tail_factor(a) * exp2f_approx(-0.72134752044f * (a * a));
  const float big = 1.0f - tail;
  p = (y >= 0.0f) ? tail : big;
  q = (y >= 0.0f) ? big : tail;
}

__device__ __forceinline__ float phi_upper_f32(float y) {
  float p, q;
  phi_upper_pq_f32(y, p, q);
  return p;
}

__device__ __forceinline__ float phi_inv_f32(float x) {
  const float w = -__logf(4.0f * x * (1.0f - x));
  const float v = fmaf(2.0f, x, -1.0f);
  float p;
  if (w < 5.0f) {
    p = nf32::horner(nf32::Q_P0, w - nf32::Q_W0);
  } else {
    const float sw = w * rsqrtf(w);
    p = (w < 16.0f) ? nf32::horner(nf32::Q_P1, sw - nf32::Q_S1) : nf32::horner(nf32::Q_P2, sw - nf32::Q_S2);
  }
  return 1.41421356237f * v * p;
}

// z = -Phi^{-1}(x) for x = um * p, given also u = 1 - um and q = 1 - p; when
// x > 1/2 the quantile is taken of 1 - x = u + um q, which keeps full relative
// precision where x itself is within rounding of 1.
__device__ __forceinline__ float neg_quantile_f32(float um, float u, float p, float q) {
  const float x = um * p;
  const bool lower = x <= 0.5f;
  const float xs = lower ? fmaxf(x, 1.17549435e-38f) : fmaf(um, q, u);
  const float zq = phi_inv_f32(xs);
  return lower ? -zq : zq;
}

__device__ __forceinline__ float log_phi_upper_f32(float y) {
  const float a = fabsf(y);
  if (y < 0.0f) return log1pf(-phi_upper_f32(a));
  const float s = a * a;
  const float e = fmaf(a, a, -s);
  float G;
  if (a <= 40.0f) {
    G = nf32::tail_factor(a);
  } else {
    // asymptotic series of Mills' ratio: G = (1 - 1/a^2 + 3/a^4) / (a sqrt(2 pi))
    const float ia2 = 1.0f / s;
    G = 0.398942280f / a * fmaf(ia2, fmaf(3.0f, ia2, -1.0f), 1.0f);
  }
  return logf(G) - 0.5f * s - 0.5f * e;
}

__device__ __forceinline__ float neg_quantile_log_f32(float la) {
  if (la > -0.693147181f) {
    // x = exp(la) > 1/2: use 1 - x = -expm1(la) from the small side
    return phi_inv_f32(-expm1f(la));
  }
  if (la > -80.0f) return -phi_inv_f32(expf(la));
  // far tail: z solves log Phi(-z) = la; fixed-point start from
  // z^2 = -2 la - 2 log z - log(2 pi), then Newton steps on log Phi(-z) whose
  // derivative is -1 / (sqrt(2 pi) G(z))
  const float L2 = -2.0f * la;
  float z = sqrtf(L2);
  z = sqrtf(L2 - 2.0f * logf(z) - 1.837877066f);
  z = sqrtf(L2 - 2.0f * logf(z) - 1.837877066f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float h = log_phi_upper_f32(z) - la;
    float G;
    if (z <= 40.0f) {
      G = nf32::tail_factor(z);
    } else {
      const float ia2 = 1.0f / (z * z);
      G = 0.398942280f / z * fmaf(ia2, fmaf(3.0f, ia2, -1.0f), 1.0f);
    }
    z = fmaf(h * 2.506628275f, G, z);
  }
  return z;
}

}  // namespace cfust

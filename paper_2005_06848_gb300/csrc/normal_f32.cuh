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

// ---- paired forms: two independent evaluations per FP32x2 instruction ------
// Coefficients (the sweep's shorter set, see fit_normal_f32.py) duplicated
// into (c, c) pairs in constant memory.
namespace nf32 {
struct Pairs {
  float2 tail_q[7];
  float2 p0[7];
  float2 p3[10];  // the tail quantile piece times -sqrt(ln 2) (see neg_quantile_x2)
};
constexpr float NSQRT_LN2 = -0.832554611158f;
__constant__ Pairs kPairs = {
    {{TAIL_QF[0], TAIL_QF[0]}, {TAIL_QF[1], TAIL_QF[1]}, {TAIL_QF[2], TAIL_QF[2]}, {TAIL_QF[3], TAIL_QF[3]},
     {TAIL_QF[4], TAIL_QF[4]}, {TAIL_QF[5], TAIL_QF[5]}, {TAIL_QF[6], TAIL_QF[6]}},
    {{Q_P0F[0], Q_P0F[0]}, {Q_P0F[1], Q_P0F[1]}, {Q_P0F[2], Q_P0F[2]}, {Q_P0F[3], Q_P0F[3]}, {Q_P0F[4], Q_P0F[4]},
     {Q_P0F[5], Q_P0F[5]}, {Q_P0F[6], Q_P0F[6]}},
    {{Q_P3[0] * NSQRT_LN2, Q_P3[0] * NSQRT_LN2}, {Q_P3[1] * NSQRT_LN2, Q_P3[1] * NSQRT_LN2},
     {Q_P3[2] * NSQRT_LN2, Q_P3[2] * NSQRT_LN2}, {Q_P3[3] * NSQRT_LN2, Q_P3[3] * NSQRT_LN2},
     {Q_P3[4] * NSQRT_LN2, Q_P3[4] * NSQRT_LN2}, {Q_P3[5] * NSQRT_LN2, Q_P3[5] * NSQRT_LN2},
     {Q_P3[6] * NSQRT_LN2, Q_P3[6] * NSQRT_LN2}, {Q_P3[7] * NSQRT_LN2, Q_P3[7] * NSQRT_LN2},
     {Q_P3[8] * NSQRT_LN2, Q_P3[8] * NSQRT_LN2}, {Q_P3[9] * NSQRT_LN2, Q_P3[9] * NSQRT_LN2}}};

template <int K>
__device__ __forceinline__ float2 horner2(const float2 (&c)[K], float2 t) {
  float2 q = c[K - 1];
#pragma unroll
  for (int k = K - 2; k >= 0; --k) q = __ffma2_rn(q, t, c[k]);
  return q;
}
}  // namespace nf32

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Paired counterpart of phi_upper_pq_fast_f32 with the sweep's degree-6 tail
// factor (fitted for y <= 14; beyond, exp2 of -y^2/2 flushes the weight to 0).
__device__ __forceinline__ void phi_upper_pq_x2(float2 y, float2 &p, float2 &q) {
  const float2 a = make_float2(fabsf(y.x), fabsf(y.y));
  const float2 den = __ffma2_rn(f2(nf32::TAIL_CF), a, f2(1.0f));
  const float2 t = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
  const float2 G = __fmul2_rn(nf32::horner2(nf32::kPairs.tail_q, t), t);
  const float2 k = __fmul2_rn(__fmul2_rn(a, a), f2(-0.72134752044f));
  const float2 tail = __fmul2_rn(G, make_float2(exp2f_approx(k.x), exp2f_approx(k.y)));
  const float2 big = __ffma2_rn(tail, f2(-1.0f), f2(1.0f));
  p = make_float2(y.x >= 0.0f ? tail.x : big.x, y.y >= 0.0f ? tail.y : big.y);
  q = make_float2(y.x >= 0.0f ? big.x : tail.x, y.y >= 0.0f ? big.y : tail.y);
}

// Paired, branch-free neg_quantile_f32: central piece below w = 5, single
// tail piece P = sqrt(w) T(1/sqrt(w)) above.
// um and u may differ between the halves (two lattice points side by side).
__device__ __forceinline__ float2 neg_quantile_x2v(float2 um, float2 u, float2 p, float2 q) {
  const float2 x = __fmul2_rn(um, p);
  const float2 c = __ffma2_rn(um, q, u);  // 1 - x
  const bool lx = x.x <= 0.5f, ly = x.y <= 0.5f;
  const float2 xs = make_float2(lx ? fmaxf(x.x, 1.17549435e-38f) : c.x, ly ? fmaxf(x.y, 1.17549435e-38f) : c.y);
  const float2 prod = __fmul2_rn(xs, __ffma2_rn(xs, f2(-4.0f), f2(4.0f)));  // 4 x (1 - x), exactly
  // with l = log2(4 x (1 - x)) <= 0, w = -ln2 l: the central argument is one
  // fused step from l, and 1/sqrt(w) = rsqrt(-l)/sqrt(ln2), sqrt(w) =
  // -sqrt(ln2) l rsqrt(-l), the constant factor living in the tail coefficients
  const float2 l = make_float2(__log2f(prod.x), __log2f(prod.y));
  const float2 pc = nf32::horner2(nf32::kPairs.p0, __ffma2_rn(l, f2(-0.69314718056f), f2(-nf32::Q_W0F)));
  const float2 rn = make_float2(rsqrtf(-l.x), rsqrtf(-l.y));
  const float2 pt = __fmul2_rn(nf32::horner2(nf32::kPairs.p3, __ffma2_rn(rn, f2(1.20112240879f), f2(-nf32::Q_U3))),
                               __fmul2_rn(l, rn));
  // w < 5  <=>  l > -5 / ln2
  const float2 P = make_float2(l.x > -7.21347520444f ? pc.x : pt.x, l.y > -7.21347520444f ? pc.y : pt.y);
  const float2 v = __ffma2_rn(f2(2.82842712475f), xs, f2(-1.41421356237f));  // sqrt(2) (2x - 1)
  const float2 zq = __fmul2_rn(v, P);
  return make_float2(lx ? -zq.x : zq.x, ly ? -zq.y : zq.y);
}

// The same with one lattice point's (1 - u, u) for both halves (passes A and B).
__device__ __forceinline__ float2 neg_quantile_x2(float um, float u, float2 p, float2 q) {
  return neg_quantile_x2v(f2(um), f2(u), p, q);
}

// One lane of neg_quantile_x2: the same coefficients and the same operations in
// the same order (a packed FP32x2 operation rounds each half as its scalar
// counterpart does), so the result equals that lane's bit for bit.  For a
// draw only one pass of the pair needs.
__device__ __forceinline__ float neg_quantile_x1(float um, float u, float p, float q) {
  const float x = um * p;
  const float c = fmaf(um, q, u);  // 1 - x
  const bool lx = x <= 0.5f;
  const float xs = lx ? fmaxf(x, 1.17549435e-38f) : c;
  const float prod = xs * fmaf(xs, -4.0f, 4.0f);
  const float l = __log2f(prod);
  const float tc = fmaf(l, -0.69314718056f, -nf32::Q_W0F);
  float pc = nf32::kPairs.p0[6].x;
#pragma unroll
  for (int k = 5; k >= 0; --k) pc = fmaf(pc, tc, nf32::kPairs.p0[k].x);
  const float rn = rsqrtf(-l);
  const float tt = fmaf(rn, 1.20112240879f, -nf32::Q_U3);
  float pt = nf32::kPairs.p3[9].x;
#pragma unroll
  for (int k = 8; k >= 0; --k) pt = fmaf(pt, tt, nf32::kPairs.p3[k].x);
  pt = pt * (l * rn);
  const float P = l > -7.21347520444f ? pc : pt;
  const float v = fmaf(2.82842712475f, xs, -1.41421356237f);
  const float zq = v * P;
  return lx ? -zq : zq;
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

// Shared by the posterior / M-step sums kernel (mstep.cu) and the fused
// E-step + sums kernel (fused.cu): the layout of one component's sum vector
// and the double-float arithmetic of the single-precision sums.
#pragma once

#include "cfust_internal.cuh"

namespace cfust {
namespace {

// Entry ent of a component's sum vector (Section 3.2's S1..S8, packed as
// sums_width(p, r) doubles): the weight column w of the tile rows
// (0 tau, 1 tau e1, 2 + t tau e3_t, 2 + r + t tau e4_t, 2 + r + rp tau (e2 - e1))
// and the observation coordinates it is multiplied by (-1 for none).
__device__ __forceinline__ void entry_desc(int ent, int p, int r, int *w, int *y1, int *y2) {
  const int rp = r * (r + 1) / 2;
  *y1 = -1;
  *y2 = -1;
  if (ent == 0) { *w = 0; return; }                 // S1
  if (ent == 1) { *w = 1; return; }                 // S2
  ent -= 2;
  if (ent < p) { *w = 1; *y1 = ent; return; }       // S3[a]
  ent -= p;
  if (ent < r) { *w = 2 + ent; return; }            // S4[t]
  ent -= r;
  if (ent < p * r) { *w = 2 + ent % r; *y1 = ent / r; return; }  // S5[a][t]
  ent -= p * r;
  if (ent < rp) { *w = 2 + r + ent; return; }       // S6 packed
  ent -= rp;
  if (ent < p * (p + 1) / 2) {                      // S7 packed (a, b), b <= a
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= ent) ++a;
    *w = 1;
    *y1 = a;
    *y2 = ent - a * (a + 1) / 2;
    return;
  }
  *w = 2 + r + rp;                                  // S8
}

// Double-float numbers (hi + lo, two floats): products formed exactly by
// Dekker's two-product (hi = fl(a b), lo = fma(a, b, -hi) is the exact rest),
// cross terms of a double-float product in single precision (their own error
// is of order 2^-48 of the product).
__device__ __forceinline__ float2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return make_float2(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  return make_float2(p, e);
}
// a + b exactly as an unevaluated pair (Knuth's two-sum)
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp)));
}
// hi + lo += v.x + v.y (two-sum on the leading parts, the rests added to lo)
__device__ __forceinline__ void df_acc(float &hi, float &lo, float2 v) {
  const float s = __fadd_rn(hi, v.x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v.x, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, v.y));
}

}  // namespace
}  // namespace cfust

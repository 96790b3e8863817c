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


// The columns of one sum entry in a tile staged as rows of tj values:
// tau[g][tj] followed by e1[g][tj], e2[g][tj], e3[g][r][tj], e4[g][r(r+1)/2][tj]
// (g the tile's components).  Entry e is component e / K, entry e % K of the
// packing above: tau times the weight column (kind 0: the weight is 1; kind 1:
// one column; kind 2: e2 - e1), times the observation coordinates y1, y2.
struct TileCols {
  int kind;  // 0: tau; 1: tau col; 2: tau (col - col1)
  const void *col, *col1;
  int y1, y2;
};

template <typename T>
__device__ __forceinline__ TileCols tile_cols(const T *out, int g, int tj, int p, int r, int K, int e) {
  const int rp = r * (r + 1) / 2;
  const int i = e / K;
  int w, y1, y2;
  entry_desc(e % K, p, r, &w, &y1, &y2);
  const T *e1 = out + (size_t)g * tj, *e2 = out + (size_t)2 * g * tj, *e3 = out + (size_t)3 * g * tj;
  const T *e4 = e3 + (size_t)g * r * tj;
  TileCols c;
  c.y1 = y1;
  c.y2 = y2;
  c.col1 = nullptr;
  c.col = nullptr;
  if (w == 0) {
    c.kind = 0;
  } else if (w == 1) {
    c.kind = 1;
    c.col = e1 + (size_t)i * tj;
  } else if (w < 2 + r) {
    c.kind = 1;
    c.col = e3 + ((size_t)i * r + (w - 2)) * tj;
  } else if (w < 2 + r + rp) {
    c.kind = 1;
    c.col = e4 + ((size_t)i * rp + (w - 2 - r)) * tj;
  } else {
    c.kind = 2;
    c.col = e2 + (size_t)i * tj;
    c.col1 = e1 + (size_t)i * tj;
  }
  return c;
}

__device__ __forceinline__ float2 tile_term_f32(const TileCols &c, float t, int jj, const float2 *ys, int p) {
  float2 v;
  if (c.kind == 0) {
    v = make_float2(t, 0.0f);
  } else if (c.kind == 1) {
    v = two_prod(t, reinterpret_cast<const float *>(c.col)[jj]);
  } else {
    // e2 - e1 as an exact float pair (two-sum), then times tau
    const float v2 = reinterpret_cast<const float *>(c.col)[jj];
    const float v1 = reinterpret_cast<const float *>(c.col1)[jj];
    const float d = __fsub_rn(v2, v1);
    const float bp = __fsub_rn(d, v2);
    const float dlo = __fadd_rn(__fsub_rn(v2, __fsub_rn(d, bp)), __fsub_rn(-v1, bp));
    v = two_prod(t, d);
    v.y = __fmaf_rn(t, dlo, v.y);
  }
  if (c.y1 >= 0) v = df_mul(v, ys[jj * p + c.y1]);
  if (c.y2 >= 0) v = df_mul(v, ys[jj * p + c.y2]);
  return v;
}

__device__ __forceinline__ double tile_term_f64(const TileCols &c, double t, int jj) {
  if (c.kind == 0) return t;
  const double *col = reinterpret_cast<const double *>(c.col);
  if (c.kind == 1) return t * col[jj];
  return t * (col[jj] - reinterpret_cast<const double *>(c.col1)[jj]);
}

}  // namespace
}  // namespace cfust

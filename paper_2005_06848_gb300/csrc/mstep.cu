// Posterior memberships, log-likelihood and the M-step (Algorithms 2 and 3).
//
// posterior_kernel: for every observation j, tau_ij = exp(log pi_i + log f_ij
// - LSE_i(...)) (Eq. 4) and log f_j = LSE (Eq. 3), then per component the
// eight sums of Section 3.2 (derived from the expected complete-data
// log-likelihood):
//   S1 = sum tau, S2 = sum tau e1, S3 = sum tau e1 y, S4 = sum tau e3,
//   S5 = sum tau y e3^T, S6 = sum tau e4, S7 = sum tau e1 y y^T, S8 = sum tau (e2 - e1)
// as block-level segmented reductions in double precision: each block walks
// its tiles of 64 observations, stages per-observation weight rows and y in
// shared memory, and every thread owns fixed entries of the sum vectors.  The
// per-block partials are reduced in a fixed order, so results do not depend
// on scheduling.
//
// mstep_finalize_kernel: one block per component, conditional maximisation
// (pi, then mu with the old Delta, then Delta, then Sigma, then nu).
#include <math.h>

#include "cfust_internal.cuh"
#include "special.cuh"
#include "sums.cuh"

namespace cfust {

namespace {

constexpr int TJ = 64;       // observations per tile
constexpr int MAXOWN = 8;    // sum entries per thread
constexpr int THREADS = 256;

// Single-precision E-step outputs (CFUST_FP32).  Double-precision work costs
// 64 times single-precision work on this GPU, so the double-precision parts
// run as double-float arithmetic on the single-precision pipe where they are
// bulk work: the M-step sums take the exact products of the single-precision
// tau, e1..e4 and the double-precision observations (y split into two
// floats), summed within a 64-observation tile with two-sum compensation
// (about 2^-42 of the sum of |terms| per tile) and across tiles in double:
// double-precision sums of the same inputs up to ~1e-13.  log pi_i + log f_ij
// is formed exactly as a float pair (two-sum), its maximum and the
// differences (the log-sum-exp's exponents) from the pairs, and
// l_j = max + log s_j and its sum over the observations in native double;
// the exponentials and tau are single precision (tau to ~1e-7 relative, the
// level of the single-precision log f_ij it comes from), and so is log s_j
// (s_j in [1, g]: 1e-7 absolute).
//
// Each tile's rows (log f of every component or the given tau, e1..e4 of
// the block's components, y) are staged in shared memory by asynchronous
// copies issued one tile ahead into the other of two buffers, so the loads of
// tile t + 1 are in flight while tile t is summed.

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// One staging buffer of the single-precision kernel, in floats: tau rows of
// the block's gc components (written from log f, or copied from the given
// tau), then their e1, e2, e3 (r rows each), e4 (r(r+1)/2 rows each), all of
// TJP values (the row layout tile_cols reads; TJP = TJ + 1 so that the lanes
// of a warp reading one observation of different rows hit different banks);
// then log f of all g components when given; then y as TJ x p doubles.  Two
// buffers, then y's float pairs.
constexpr int TJP = TJ + 1;

struct PostTile {
  int lf, y, size;
};

__host__ __device__ inline PostTile post_tile(int g, int gc, int p, int r, bool sums, bool have_lf) {
  const int rp = r * (r + 1) / 2;
  PostTile t;
  int off = gc * TJP;
  if (sums) off += gc * TJP * (2 + r + rp);
  t.lf = off;
  if (have_lf) off += g * TJP;
  off = (off + 1) & ~1;
  t.y = off;
  if (sums) off += TJ * p * 2;
  t.size = (off + 3) & ~3;
  return t;
}

__host__ __device__ inline size_t post_smem_f32(int g, int gc, int p, int r, bool sums, bool have_lf) {
  return (size_t)2 * post_tile(g, gc, p, r, sums, have_lf).size * 4 + (sums ? (size_t)TJ * p * 8 : 0);
}

// Issues the asynchronous copies of tile [j0, j0 + nt) into `buf`.
__device__ __forceinline__ void post_issue(const PosteriorArgs &a, int c0, int gc, int64_t j0, int nt, float *buf,
                                           const PostTile &L) {
  const int g = a.g, p = a.p, r = a.r, rp = r * (r + 1) / 2;
  const int64_t n = a.n;
  if (a.logf != nullptr) {
    const float *lf = reinterpret_cast<const float *>(a.logf);
    for (int idx = threadIdx.x; idx < g * nt; idx += THREADS) {
      const int row = idx / nt, jj = idx - row * nt;
      cp_async4(buf + L.lf + row * TJP + jj, lf + (int64_t)row * n + j0 + jj);
    }
  } else if (a.want_sums) {
    const float *ti = reinterpret_cast<const float *>(a.tau_in);
    for (int idx = threadIdx.x; idx < gc * nt; idx += THREADS) {
      const int row = idx / nt, jj = idx - row * nt;
      cp_async4(buf + row * TJP + jj, ti + (int64_t)(c0 + row) * n + j0 + jj);
    }
  }
  if (!a.want_sums) return;
  const float *e1 = reinterpret_cast<const float *>(a.e1), *e2 = reinterpret_cast<const float *>(a.e2);
  const float *e3 = reinterpret_cast<const float *>(a.e3), *e4 = reinterpret_cast<const float *>(a.e4);
  const int nr = gc * (2 + r + rp);
  for (int idx = threadIdx.x; idx < nr * nt; idx += THREADS) {
    const int row = idx / nt, jj = idx - row * nt;
    const float *src;
    if (row < gc)
      src = e1 + (int64_t)(c0 + row) * n;
    else if (row < 2 * gc)
      src = e2 + (int64_t)(c0 + row - gc) * n;
    else if (row < 2 * gc + gc * r)
      src = e3 + (int64_t)(c0 * r + row - 2 * gc) * n;
    else
      src = e4 + (int64_t)(c0 * rp + row - 2 * gc - gc * r) * n;
    cp_async4(buf + (gc + row) * TJP + jj, src + j0 + jj);
  }
  const double *yt = a.Y + j0 * a.p;
  for (int idx = threadIdx.x; idx < nt * p; idx += THREADS) cp_async8(buf + L.y + 2 * idx, yt + idx);
}

__device__ __forceinline__ void posterior_block_f32(const PosteriorArgs &a, int c0, int c1, int blk, int nblk,
                                                    unsigned char *smem_raw) {
  const int p = a.p, r = a.r, g = a.g;
  const int K = sums_width(p, r);
  const int gc = c1 - c0;
  const int64_t n = a.n;
  const bool have_lf = a.logf != nullptr;
  const PostTile L = post_tile(g, gc, p, r, a.want_sums, have_lf);
  float *bufs = reinterpret_cast<float *>(smem_raw);
  float2 *ys = reinterpret_cast<float2 *>(bufs + 2 * L.size);  // [TJ][p] (hi, lo) of y
  __shared__ double red[THREADS];
  float *tau_out = reinterpret_cast<float *>(a.tau_out);

  double acc[MAXOWN];
#pragma unroll
  for (int k = 0; k < MAXOWN; ++k) acc[k] = 0.0;
  const int E = a.want_sums ? gc * K : 0;
  // With few sum entries (a small mixture), S adjacent threads share one
  // entry: each sums every S-th row of the tile, and the S partial sums are
  // merged by shuffles in a fixed order, so more of the block's threads work
  // on the tile's column sums.  S = 1 keeps one entry per thread and step.
  const int S = (E > 0 && 4 * E <= THREADS) ? 4 : ((E > 0 && 2 * E <= THREADS) ? 2 : 1);
  const int split = threadIdx.x % S;
  const int per = THREADS / S;
  double llacc = 0.0;
  int bad = 0;
  const int64_t ntiles = (n + TJ - 1) / TJ;
  const bool first_chunk = (c0 == 0);
  // log pi_i as a float pair (hi + lo to double precision), so that the
  // log-sum-exp's exponents log pi_i + log f_ij - max are formed on the
  // single-precision pipe
  __shared__ float2 lpi2[CFUST_GMAX];
  for (int i = threadIdx.x; i < g; i += THREADS) {
    const double l = log(a.pi[i]);
    const float hi = (float)l;
    lpi2[i] = make_float2(hi, (float)(l - (double)hi));
  }
  if (blk < ntiles) {
    const int64_t j0 = (int64_t)blk * TJ;
    post_issue(a, c0, gc, j0, (int)((n - j0) < TJ ? (n - j0) : TJ), bufs, L);
  }
  cp_async_commit();

  int it = 0;
  for (int64_t tile = blk; tile < ntiles; tile += nblk, ++it) {
    const int64_t j0 = tile * TJ;
    const int nt = (int)((n - j0) < TJ ? (n - j0) : TJ);
    float *buf = bufs + (it & 1) * L.size;
    const int64_t next = tile + nblk;
    if (next < ntiles) {
      const int64_t jn = next * TJ;
      post_issue(a, c0, gc, jn, (int)((n - jn) < TJ ? (n - jn) : TJ), bufs + ((it + 1) & 1) * L.size, L);
    }
    cp_async_commit();
    cp_async_wait_prev();  // this thread's copies of the current tile have landed
    __syncthreads();       // and everyone's
    if (have_lf && (int)threadIdx.x < nt) {
      const int jj = threadIdx.x;
      const int64_t j = j0 + jj;
      const float *lf = buf + L.lf;
      // a_i = log pi_i + log f_ij as a float pair (exact sum of the float
      // log f and the pair of log pi); the shift is the largest a_i
      float2 mx = make_float2(-INFINITY, 0.0f);
      for (int i = 0; i < g; ++i) {
        float2 ai = two_sum(lpi2[i].x, lf[i * TJP + jj]);
        ai.y = __fadd_rn(ai.y, lpi2[i].y);
        if (ai.x > mx.x || (ai.x == mx.x && ai.y > mx.y)) mx = ai;
      }
      if (!isfinite(mx.x)) {
        // no component gives the observation a positive density: flagged,
        // and its weights are zero so that the sums stay defined
        bad = 1;
        if (a.want_sums)
          for (int i = c0; i < c1; ++i) buf[(i - c0) * TJP + jj] = 0.0f;
        if (tau_out != nullptr && first_chunk)
          for (int i = 0; i < g; ++i) tau_out[(int64_t)i * n + j] = 0.0f;
      } else {
        float s = 0.0f;
        for (int i = 0; i < g; ++i) {
          float2 ai = two_sum(lpi2[i].x, lf[i * TJP + jj]);
          ai.y = __fadd_rn(ai.y, lpi2[i].y);
          // the exponent a_i - max (exact leading difference where the two
          // are within a factor two, else rounded: 2^-24 of an exponent
          // whose exponential is then below e^-1 of the largest)
          const float dx = __fadd_rn(__fsub_rn(ai.x, mx.x), __fsub_rn(ai.y, mx.y));
          s = __fadd_rn(s, (ai.x == -INFINITY) ? 0.0f : expf(dx));
        }
        // s is in [1, g]: its single-precision logarithm is good to 1e-7
        // absolute, below the error of the log f_ij it sums; l_j in double
        const double lse = (double)mx.x + (double)mx.y + (double)logf(s);
        if (!isfinite(lse)) bad = 1;
        llacc += lse;
        const float inv = 1.0f / s;
        for (int i = 0; i < g; ++i) {
          float2 ai = two_sum(lpi2[i].x, lf[i * TJP + jj]);
          ai.y = __fadd_rn(ai.y, lpi2[i].y);
          const float dx = __fadd_rn(__fsub_rn(ai.x, mx.x), __fsub_rn(ai.y, mx.y));
          const float t = ((ai.x == -INFINITY) ? 0.0f : expf(dx)) * inv;
          if (a.want_sums && i >= c0 && i < c1) buf[(i - c0) * TJP + jj] = t;
          if (tau_out != nullptr && first_chunk) tau_out[(int64_t)i * n + j] = t;
        }
      }
    }
    if (a.want_sums) {
      const double *yb = reinterpret_cast<const double *>(buf + L.y);
      for (int idx = threadIdx.x; idx < nt * p; idx += THREADS) {
        const double y = yb[idx];
        const float yh = (float)y;
        ys[idx] = make_float2(yh, (float)(y - (double)yh));
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < MAXOWN; ++k) {
        const int e0 = k * per;
        if (e0 >= E) continue;  // uniform over the block
        const int e = e0 + (int)threadIdx.x / S;
        // two compensated chains (rows jj and jj + S) for instruction-level
        // parallelism, merged by a further two-sum; this thread's rows are
        // split, split + S, ...
        float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
        if (e < E) {
          const TileCols c = tile_cols<float>(buf, gc, TJP, p, r, K, e);
          const float *ti = buf + (e / K) * TJP;
          int jj = split;
          for (; jj + S < nt; jj += 2 * S) {
            df_acc(h0, l0, tile_term_f32(c, ti[jj], jj, ys, p));
            df_acc(h1, l1, tile_term_f32(c, ti[jj + S], jj + S, ys, p));
          }
          if (jj < nt) df_acc(h0, l0, tile_term_f32(c, ti[jj], jj, ys, p));
          df_acc(h0, l0, make_float2(h1, l1));
        }
        // the entry's S partial sums, from adjacent lanes, in a fixed order
        for (int o = 1; o < S; o <<= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, h0, o), l2 = __shfl_xor_sync(0xffffffffu, l0, o);
          df_acc(h0, l0, make_float2(h2, l2));
        }
        if (e < E && split == 0) acc[k] += (double)h0 + (double)l0;
      }
    }
    __syncthreads();  // this buffer is refilled two tiles on
  }

  if (a.want_sums) {
    double *dst = a.partials + (int64_t)blk * g * K;
#pragma unroll
    for (int k = 0; k < MAXOWN; ++k) {
      const int e = k * per + (int)threadIdx.x / S;
      if (k * per < E && e < E && split == 0) dst[(int64_t)c0 * K + e] = acc[k];
    }
  }
  if (a.want_ll && first_chunk) {
    red[threadIdx.x] = llacc;
    __syncthreads();
    for (int s = THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) a.ll_partials[blk] = red[0];
  }
  if (bad) atomicOr(a.d_status, ERR_ZERO_DENSITY);
}

// One block's share of the posterior / sums work of one fit: tiles blk,
// blk + nblk, ...; partial sums and the log-likelihood partial go to row blk.
template <typename ET>
__device__ __forceinline__ void posterior_block(const PosteriorArgs &a, int c0, int c1, int blk, int nblk,
                                                unsigned char *smem_raw) {
  if constexpr (sizeof(ET) == 4) {
    posterior_block_f32(a, c0, c1, blk, nblk, smem_raw);
    return;
  }
  double *smem = reinterpret_cast<double *>(smem_raw);
  const int p = a.p, r = a.r, g = a.g;
  const int rp = r * (r + 1) / 2;
  const int K = sums_width(p, r);
  const int WR = 3 + r + rp;
  const int gc = c1 - c0;
  const int64_t n = a.n;
  double *ys = smem;                     // [TJ][p]
  double *ws = ys + TJ * p;              // [gc][TJ][WR]
  __shared__ double red[THREADS];

  const ET *logf = reinterpret_cast<const ET *>(a.logf);
  const ET *tau_in = reinterpret_cast<const ET *>(a.tau_in);
  const ET *e1 = reinterpret_cast<const ET *>(a.e1);
  const ET *e2 = reinterpret_cast<const ET *>(a.e2);
  const ET *e3 = reinterpret_cast<const ET *>(a.e3);
  const ET *e4 = reinterpret_cast<const ET *>(a.e4);
  ET *tau_out = reinterpret_cast<ET *>(a.tau_out);

  int own_w[MAXOWN], own_y1[MAXOWN], own_y2[MAXOWN], own_c[MAXOWN];
  double acc[MAXOWN];
  const int E = a.want_sums ? gc * K : 0;
#pragma unroll
  for (int k = 0; k < MAXOWN; ++k) {
    const int e = threadIdx.x + k * THREADS;
    acc[k] = 0.0;
    own_c[k] = -1;
    own_w[k] = 0;
    own_y1[k] = own_y2[k] = -1;
    if (e < E) {
      own_c[k] = e / K;
      entry_desc(e % K, p, r, &own_w[k], &own_y1[k], &own_y2[k]);
    }
  }
  double llacc = 0.0;
  int bad = 0;
  const int64_t ntiles = (n + TJ - 1) / TJ;
  const bool first_chunk = (c0 == 0);
  // log pi_i once per block (a double logarithm costs ~40 operations of the
  // 1/64-rate pipe; per observation it was taken three times per component)
  __shared__ double lpi[CFUST_GMAX];
  for (int i = threadIdx.x; i < g; i += THREADS) lpi[i] = log(a.pi[i]);
  __syncthreads();

  for (int64_t tile = blk; tile < ntiles; tile += nblk) {
    const int64_t j0 = tile * TJ;
    const int nt = (int)((n - j0) < TJ ? (n - j0) : TJ);
    if (a.want_sums)
      for (int idx = threadIdx.x; idx < nt * p; idx += THREADS) ys[idx] = a.Y[j0 * p + idx];
    if (threadIdx.x < nt) {
      const int jj = threadIdx.x;
      const int64_t j = j0 + jj;
      if (logf != nullptr) {
        double mx = -INFINITY;
        for (int i = 0; i < g; ++i) mx = fmax(mx, lpi[i] + (double)logf[(int64_t)i * n + j]);
        // tau_ij = exp(a_i - mx) / sum_h exp(a_h - mx): the exponentials of the
        // sum are kept (in the tile's rows) and scaled once the sum is known
        double s = 0.0;
        for (int i = 0; i < g; ++i) {
          const double e = exp(lpi[i] + (double)logf[(int64_t)i * n + j] - mx);
          s += e;
          if (a.want_sums && i >= c0 && i < c1) ws[((i - c0) * TJ + jj) * WR] = e;
        }
        const double lse = mx + log(s);
        if (!isfinite(lse)) bad = 1;
        llacc += lse;
        const double inv = 1.0 / s;
        if (a.want_sums)
          for (int i = c0; i < c1; ++i) ws[((i - c0) * TJ + jj) * WR] *= inv;
        if (tau_out != nullptr && first_chunk)
          for (int i = 0; i < g; ++i)
            tau_out[(int64_t)i * n + j] = (ET)(exp(lpi[i] + (double)logf[(int64_t)i * n + j] - mx) * inv);
      } else if (a.want_sums) {
        for (int i = c0; i < c1; ++i) ws[((i - c0) * TJ + jj) * WR] = (double)tau_in[(int64_t)i * n + j];
      }
    }
    __syncthreads();
    if (a.want_sums) {
      for (int idx = threadIdx.x; idx < gc * nt; idx += THREADS) {
        const int ic = idx / nt, jj = idx % nt;
        const int i = c0 + ic;
        const int64_t j = j0 + jj;
        double *row = ws + (ic * TJ + jj) * WR;
        const double t = row[0];
        const double v1 = (double)e1[(int64_t)i * n + j];
        row[1] = t * v1;
        for (int q = 0; q < r; ++q) row[2 + q] = t * (double)e3[((int64_t)i * r + q) * n + j];
        for (int q = 0; q < rp; ++q) row[2 + r + q] = t * (double)e4[((int64_t)i * rp + q) * n + j];
        row[2 + r + rp] = t * ((double)e2[(int64_t)i * n + j] - v1);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < MAXOWN; ++k) {
        if (own_c[k] >= 0) {
          const double *col = ws + own_c[k] * TJ * WR + own_w[k];
          const int y1 = own_y1[k], y2 = own_y2[k];
          // four interleaved partial sums (fixed order): independent chains
          // of the long-latency double multiply-add
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int jj = 0;
          if (y1 < 0) {
            for (; jj + 4 <= nt; jj += 4) {
              s0 += col[jj * WR];
              s1 += col[(jj + 1) * WR];
              s2 += col[(jj + 2) * WR];
              s3 += col[(jj + 3) * WR];
            }
            for (; jj < nt; ++jj) s0 += col[jj * WR];
          } else if (y2 < 0) {
            for (; jj + 4 <= nt; jj += 4) {
              s0 = fma(col[jj * WR], ys[jj * p + y1], s0);
              s1 = fma(col[(jj + 1) * WR], ys[(jj + 1) * p + y1], s1);
              s2 = fma(col[(jj + 2) * WR], ys[(jj + 2) * p + y1], s2);
              s3 = fma(col[(jj + 3) * WR], ys[(jj + 3) * p + y1], s3);
            }
            for (; jj < nt; ++jj) s0 = fma(col[jj * WR], ys[jj * p + y1], s0);
          } else {
            for (; jj + 4 <= nt; jj += 4) {
              s0 = fma(col[jj * WR] * ys[jj * p + y1], ys[jj * p + y2], s0);
              s1 = fma(col[(jj + 1) * WR] * ys[(jj + 1) * p + y1], ys[(jj + 1) * p + y2], s1);
              s2 = fma(col[(jj + 2) * WR] * ys[(jj + 2) * p + y1], ys[(jj + 2) * p + y2], s2);
              s3 = fma(col[(jj + 3) * WR] * ys[(jj + 3) * p + y1], ys[(jj + 3) * p + y2], s3);
            }
            for (; jj < nt; ++jj) s0 = fma(col[jj * WR] * ys[jj * p + y1], ys[jj * p + y2], s0);
          }
          acc[k] += (s0 + s1) + (s2 + s3);
        }
      }
    }
    __syncthreads();
  }

  if (a.want_sums) {
    double *dst = a.partials + (int64_t)blk * g * K;
#pragma unroll
    for (int k = 0; k < MAXOWN; ++k) {
      const int e = threadIdx.x + k * THREADS;
      if (e < E) dst[(int64_t)c0 * K + e] = acc[k];
    }
  }
  if (a.want_ll && first_chunk) {
    red[threadIdx.x] = llacc;
    __syncthreads();
    for (int s = THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) a.ll_partials[blk] = red[0];
  }
  if (bad) atomicOr(a.d_status, ERR_ZERO_DENSITY);
}

template <typename ET>
__global__ void __launch_bounds__(THREADS) posterior_kernel(PosteriorArgs a, int c0, int c1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  posterior_block<ET>(a, c0, c1, blockIdx.x, gridDim.x, smem_raw);
}

__global__ void reduce_ll_kernel(const double *part, int nb, double *out, double *trace, int *iter) {
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) s += part[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = red[0];
    if (trace != nullptr) {
      trace[*iter] = red[0];
      *iter += 1;
    }
  }
}

__device__ bool chol_inplace(double *S, int n, int ld) {
  for (int j = 0; j < n; ++j) {
    double s = S[j * ld + j];
    for (int k = 0; k < j; ++k) s -= S[j * ld + k] * S[j * ld + k];
    if (!(s > 0.0) || !isfinite(s)) return false;
    const double d = sqrt(s);
    S[j * ld + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = S[i * ld + j];
      for (int k = 0; k < j; ++k) t -= S[i * ld + k] * S[j * ld + k];
      S[i * ld + j] = t / d;
    }
  }
  return true;
}

// Root of h(nu) = log(nu/2) - psi(nu/2) + 1 + c in [lo, hi]; h decreases in
// nu, so the bound is returned when there is no sign change.  Double-precision
// work costs 64 times single-precision work on this GPU and a warp
// instruction of it costs the same whatever the number of active lanes, so
// warp 0 brackets the root with single-precision evaluations (32 interior
// points per round, the bracket shrinks 33-fold per round, to ~1e-7
// relative) and finishes with Newton steps on the double-precision h; h is
// convex, so the steps approach the root monotonically once on its left, and
// each is clamped to the bracket that the double-precision end values
// certify.  The derivative enters only the step length, so its single-precision
// value costs no accuracy.  All threads of the block must call it with the
// same arguments.
__device__ double solve_nu_block(double c, double lo, double hi) {
  __shared__ double nu_out;
  if (threadIdx.x < 32) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    const double he = log_minus_digamma(0.5 * ((lane & 1) ? hi : lo)) + 1.0 + c;
    const double h_lo = __shfl_sync(full, he, 0), h_hi = __shfl_sync(full, he, 1);
    double nu;
    if (h_hi >= 0.0) {
      nu = hi;
    } else if (h_lo <= 0.0) {
      nu = lo;
    } else {
      float flo = (float)lo, fhi = (float)hi;
      const float cp = (float)(1.0 + c);
      for (int round = 0; round < 6; ++round) {
        const float w = (fhi - flo) * (1.0f / 33.0f);
        const float x = flo + (float)(lane + 1) * w;
        const int npos = __popc(__ballot_sync(full, log_minus_digamma_f(0.5f * x) + cp > 0.0f));
        const float nlo = (npos == 0) ? flo : flo + (float)npos * w;
        const float nhi = (npos == 32) ? fhi : flo + (float)(npos + 1) * w;
        flo = nlo;
        fhi = nhi;
      }
      nu = 0.5 * ((double)flo + (double)fhi);
      for (int it = 0; it < 6; ++it) {
        const double h = log_minus_digamma(0.5 * nu) + 1.0 + c;
        const double dh = 0.5 * (double)dlog_minus_digamma_f((float)(0.5 * nu));
        const double nn = fmin(fmax(nu - h / dh, lo), hi);
        // a step of 1e-8 relative leaves an error of order 1e-16 after it
        const bool done = fabs(nn - nu) <= 1e-8 * nu;
        nu = nn;
        if (done) break;
      }
    }
    if (lane == 0) nu_out = nu;
  }
  __syncthreads();
  return nu_out;
}

// Thread 0 of the finalize block: pi, mu, Delta, Sigma of component i from its
// sums S (Algorithm 3); false (status flagged) when the update is not defined.
// *nu_c receives the constant S8 / S1 of the nu equation.
__device__ bool mstep_update_thread0(const double *S, double total_weight, int g, int p, int r, int64_t n,
                                     double *params, int *status, int i, double *nu_c) {
  const int rp = r * (r + 1) / 2;
  const double S1 = S[0], S2 = S[1];
  const double *S3 = S + 2;
  const double *S4 = S3 + p;
  const double *S5 = S4 + r;          // [p][r]
  const double *S6p = S5 + p * r;     // packed lower
  const double *S7p = S6p + rp;       // packed lower
  const double S8 = S7p[p * (p + 1) / 2];
  if (!(S1 > 1e-10 * (double)n) || !(S2 > 0.0)) {
    atomicOr(status, ERR_DEGENERATE);
    return false;
  }
  ParamView pv = param_view(params, g, p, r);
  double *mu = pv.mu + (int64_t)i * p;
  double *Sig = pv.Sigma + (int64_t)i * p * p;
  double *Del = pv.Delta + (int64_t)i * p * r;

  double m[PMAX], C[PMAX * RMAX], D[PMAX * RMAX], S6[RMAX * RMAX], Lc[RMAX * RMAX];
  for (int a = 0; a < p; ++a) {
    double s = S3[a];
    for (int t = 0; t < r; ++t) s -= Del[a * r + t] * S4[t];
    m[a] = s / S2;
  }
  for (int a = 0; a < p; ++a)
    for (int t = 0; t < r; ++t) C[a * RMAX + t] = S5[a * r + t] - m[a] * S4[t];
  for (int t = 0; t < r; ++t)
    for (int h = 0; h <= t; ++h) S6[t * RMAX + h] = S6[h * RMAX + t] = S6p[t * (t + 1) / 2 + h];
  for (int t = 0; t < r; ++t)
    for (int h = 0; h < r; ++h) Lc[t * RMAX + h] = S6[t * RMAX + h];
  if (!chol_inplace(Lc, r, RMAX)) {
    atomicOr(status, ERR_NOTPD_S6);
    return false;
  }
  // Delta row a solves S6 x = C[a, :]^T
  for (int a = 0; a < p; ++a) {
    double x[RMAX];
    for (int t = 0; t < r; ++t) {
      double s = C[a * RMAX + t];
      for (int k = 0; k < t; ++k) s -= Lc[t * RMAX + k] * x[k];
      x[t] = s / Lc[t * RMAX + t];
    }
    for (int t = r - 1; t >= 0; --t) {
      double s = x[t];
      for (int k = t + 1; k < r; ++k) s -= Lc[k * RMAX + t] * x[k];
      x[t] = s / Lc[t * RMAX + t];
    }
    for (int t = 0; t < r; ++t) D[a * RMAX + t] = x[t];
  }
  double Sn[PMAX * PMAX];
  for (int a = 0; a < p; ++a)
    for (int b = 0; b <= a; ++b) {
      double s = S7p[a * (a + 1) / 2 + b] - S3[a] * m[b] - m[a] * S3[b] + S2 * m[a] * m[b];
      for (int t = 0; t < r; ++t) s -= C[a * RMAX + t] * D[b * RMAX + t] + D[a * RMAX + t] * C[b * RMAX + t];
      for (int t = 0; t < r; ++t)
        for (int h = 0; h < r; ++h) s += D[a * RMAX + t] * S6[t * RMAX + h] * D[b * RMAX + h];
      Sn[a * PMAX + b] = Sn[b * PMAX + a] = s / S1;
    }
  double Lt[PMAX * PMAX];
  for (int a = 0; a < p * PMAX; ++a) Lt[a] = Sn[a];
  if (!chol_inplace(Lt, p, PMAX)) {
    atomicOr(status, ERR_NOTPD_SIGMA);
    return false;
  }
  // pi_i maximises sum_i S1_i log pi_i subject to sum_i pi_i = 1
  pv.pi[i] = S1 / total_weight;
  for (int a = 0; a < p; ++a) {
    mu[a] = m[a];
    for (int t = 0; t < r; ++t) Del[a * r + t] = D[a * RMAX + t];
    for (int b = 0; b < p; ++b) Sig[a * p + b] = Sn[a * PMAX + b];
  }
  *nu_c = S8 / S1;
  return true;
}

// Conditional-maximisation update of component i of one fit from the
// per-block partial sums (block of 128 threads).
__device__ void mstep_finalize_block(const double *partials, int nb, int g, int p, int r, int64_t n,
                                     double nu_min, double nu_max, double *params, int *status, int i) {
  __shared__ double S[3 + PMAX + RMAX + PMAX * RMAX + RMAX * (RMAX + 1) / 2 + PMAX * (PMAX + 1) / 2];
  __shared__ double red[128];
  const int K = sums_width(p, r);
  // every warp takes a share of the blocks' partial sums (double-precision
  // adds issue at 1/64 rate: one warp alone would run nb of them in a row),
  // combined in a fixed order
  const int splits = (int)blockDim.x / K < 8 ? (int)blockDim.x / K : 8;
  if (splits > 1) {
    const int e = threadIdx.x % K, sp = threadIdx.x / K;
    if (sp < splits) {
      double s0 = 0.0, s1 = 0.0;
      int b = sp;
      for (; b + splits < nb; b += 2 * splits) {
        s0 += partials[(int64_t)b * g * K + (int64_t)i * K + e];
        s1 += partials[(int64_t)(b + splits) * g * K + (int64_t)i * K + e];
      }
      if (b < nb) s0 += partials[(int64_t)b * g * K + (int64_t)i * K + e];
      red[threadIdx.x] = s0 + s1;
    }
    __syncthreads();
    if (threadIdx.x < K) {
      double s = 0.0;
      for (int q = 0; q < splits; ++q) s += red[q * K + threadIdx.x];
      S[threadIdx.x] = s;
    }
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < K; e += blockDim.x) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += partials[(int64_t)b * g * K + (int64_t)i * K + e];
      S[e] = s;
    }
  }
  // total posterior weight over all components (= n when every tau row sums to 1)
  double tw = 0.0;
  for (int q = threadIdx.x; q < g * nb; q += blockDim.x) {
    const int ic = q / nb, b = q % nb;
    tw += partials[(int64_t)b * g * K + (int64_t)ic * K];
  }
  red[threadIdx.x] = tw;
  __syncthreads();
  for (int h = 64; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  __shared__ double nu_c;
  __shared__ int nu_go;
  if (threadIdx.x == 0) nu_go = mstep_update_thread0(S, red[0], g, p, r, n, params, status, i, &nu_c) ? 1 : 0;
  __syncthreads();
  if (!nu_go) return;
  // nu = inf selects the skew-normal limit, a model choice the update keeps
  if (isinf(param_view(params, g, p, r).nu[i])) return;
  const double nu = solve_nu_block(nu_c, nu_min, nu_max);
  if (threadIdx.x == 0) param_view(params, g, p, r).nu[i] = nu;
}

__global__ void mstep_finalize_kernel(const double *partials, int nb, int g, int p, int r, int64_t n,
                                      double nu_min, double nu_max, double *params, int *status) {
  mstep_finalize_block(partials, nb, g, p, r, n, nu_min, nu_max, params, status, blockIdx.x);
}

template <typename ET>
__global__ void __launch_bounds__(THREADS) posterior_batched_kernel(BatchDev b, int p, int r, const BlockRef *blocks,
                                                                     double *partials, double *ll_partials,
                                                                     bool want_sums) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BlockRef br = blocks[blockIdx.x];
  const FitDesc fd = b.fits[br.fit];
  const int rp = r * (r + 1) / 2;
  PosteriorArgs a{};
  a.Y = fd.Y;
  a.n = fd.n;
  a.g = fd.g;
  a.p = p;
  a.r = r;
  a.pi = param_view(b.params + fd.param_off, fd.g, p, r).pi;
  a.logf = reinterpret_cast<const ET *>(b.logf) + fd.pair_off;
  a.e1 = reinterpret_cast<const ET *>(b.e1) + fd.pair_off;
  a.e2 = reinterpret_cast<const ET *>(b.e2) + fd.pair_off;
  a.e3 = reinterpret_cast<const ET *>(b.e3) + fd.pair_off * r;
  a.e4 = reinterpret_cast<const ET *>(b.e4) + fd.pair_off * rp;
  a.want_sums = want_sums;
  a.want_ll = true;
  a.partials = partials + fd.part_off;
  a.ll_partials = ll_partials + fd.blk0;
  a.d_status = b.fit_status + br.fit;
  a.nblocks = fd.nblk;
  posterior_block<ET>(a, 0, fd.g, br.lb, fd.nblk, smem_raw);
}

__global__ void reduce_ll_batched_kernel(BatchDev b, const double *part, double *trace, int stride, int *iter) {
  __shared__ double red[256];
  const FitDesc fd = b.fits[blockIdx.x];
  double s = 0.0;
  for (int k = threadIdx.x; k < fd.nblk; k += 256) s += part[fd.blk0 + k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) trace[(int64_t)blockIdx.x * stride + *iter] = red[0];
}

__global__ void advance_iter_kernel(int *iter) { *iter += 1; }

__global__ void finalize_batched_kernel(BatchDev b, int p, int r, const double *partials, double nu_min,
                                        double nu_max) {
  const CompRef cr = b.comps[blockIdx.x];
  const FitDesc fd = b.fits[cr.fit];
  mstep_finalize_block(partials + fd.part_off, fd.nblk, fd.g, p, r, fd.n, nu_min, nu_max,
                       b.params + fd.param_off, b.fit_status + cr.fit, cr.i);
}

}  // namespace

cudaError_t launch_posterior_batched(int precision, const BatchDev &b, int p, int r, const BlockRef *blocks,
                                     int nblocks, double *partials, double *ll_partials, bool want_sums,
                                     int g_max, cudaStream_t st) {
  const int WR = 3 + r + r * (r + 1) / 2;
  const int K = sums_width(p, r);
  if (want_sums && g_max * K > MAXOWN * THREADS) return cudaErrorInvalidValue;
  // every fit's block takes all its components in one pass (the log f rows of
  // all of them are staged in single precision): sized for the largest g
  const size_t smem = precision == CFUST_FP64
                          ? (want_sums ? ((size_t)TJ * p + (size_t)g_max * TJ * WR) * 8 : 16)
                          : post_smem_f32(g_max, g_max, p, r, want_sums, true);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (precision == CFUST_FP64) {
    e = raise_smem_limit((const void *)posterior_batched_kernel<double>, (size_t)((int)smem));
    if (e != cudaSuccess) return e;
    posterior_batched_kernel<double><<<nblocks, THREADS, smem, st>>>(b, p, r, blocks, partials, ll_partials,
                                                                     want_sums);
  } else {
    e = raise_smem_limit((const void *)posterior_batched_kernel<float>, (size_t)((int)smem));
    if (e != cudaSuccess) return e;
    posterior_batched_kernel<float><<<nblocks, THREADS, smem, st>>>(b, p, r, blocks, partials, ll_partials,
                                                                    want_sums);
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_ll_batched(const BatchDev &b, const double *ll_partials, double *trace, int stride,
                                     int *iter, cudaStream_t st) {
  reduce_ll_batched_kernel<<<b.nfits, 256, 0, st>>>(b, ll_partials, trace, stride, iter);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  advance_iter_kernel<<<1, 1, 0, st>>>(iter);
  return cudaGetLastError();
}

cudaError_t launch_finalize_batched(const BatchDev &b, int p, int r, const double *partials, double nu_min,
                                    double nu_max, cudaStream_t st) {
  finalize_batched_kernel<<<b.G, 128, 0, st>>>(b, p, r, partials, nu_min, nu_max);
  return cudaGetLastError();
}

int posterior_nblocks(int64_t n) {
  const int64_t ntiles = (n + TJ - 1) / TJ;
  const int64_t cap = (int64_t)sm_count() * 4;
  return (int)(ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
}

cudaError_t launch_posterior(int precision, const PosteriorArgs &a, cudaStream_t st) {
  const int K = sums_width(a.p, a.r);
  const int WR = 3 + a.r + a.r * (a.r + 1) / 2;
  const bool f32 = precision != CFUST_FP64;
  const bool have_lf = a.logf != nullptr;
  // components per launch: bounded by the per-thread entries and by shared memory
  int gc = a.g;
  if (a.want_sums) {
    const int by_entries = (MAXOWN * THREADS) / K;
    gc = a.g < by_entries ? a.g : by_entries;
    if (f32) {
      while (gc > 1 && post_smem_f32(a.g, gc, a.p, a.r, true, have_lf) > 200u * 1024u) --gc;
    } else {
      const int by_smem = (int)((96 * 1024 - (size_t)TJ * a.p * 8) / ((size_t)TJ * WR * 8));
      gc = gc < by_smem ? gc : by_smem;
    }
    if (gc < 1) return cudaErrorInvalidValue;
  }
  for (int c0 = 0; c0 < a.g; c0 += gc) {
    const int c1 = (c0 + gc < a.g) ? c0 + gc : a.g;
    cudaError_t e;
    if (!f32) {
      const size_t smem = a.want_sums ? ((size_t)TJ * a.p + (size_t)(c1 - c0) * TJ * WR) * 8 : 16;
      e = raise_smem_limit((const void *)posterior_kernel<double>, smem);
      if (e != cudaSuccess) return e;
      posterior_kernel<double><<<a.nblocks, THREADS, smem, st>>>(a, c0, c1);
    } else {
      const size_t smem = post_smem_f32(a.g, c1 - c0, a.p, a.r, a.want_sums, have_lf);
      e = raise_smem_limit((const void *)posterior_kernel<float>, smem);
      if (e != cudaSuccess) return e;
      posterior_kernel<float><<<a.nblocks, THREADS, smem, st>>>(a, c0, c1);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!a.want_sums) break;
  }
  return cudaSuccess;
}

cudaError_t launch_reduce_ll(const double *ll_partials, int nblocks, double *ll_out, double *trace,
                             int *iter, cudaStream_t st) {
  reduce_ll_kernel<<<1, 256, 0, st>>>(ll_partials, nblocks, ll_out, trace, iter);
  return cudaGetLastError();
}

namespace {
__global__ void sum_partials_kernel(const double *partials, int nb, int gK, double *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= gK) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partials[(int64_t)b * gK + e];
  out[e] = s;
}
}  // namespace

cudaError_t launch_sum_partials(const double *partials, int nblocks, int gK, double *out, cudaStream_t st) {
  if (gK <= 0) return cudaSuccess;
  sum_partials_kernel<<<(gK + 127) / 128, 128, 0, st>>>(partials, nblocks, gK, out);
  return cudaGetLastError();
}

cudaError_t launch_mstep_finalize(const double *partials, int nblocks, int g, int p, int r, int64_t n,
                                  double nu_min, double nu_max, double *d_params, int *d_status,
                                  cudaStream_t st) {
  mstep_finalize_kernel<<<g, 128, 0, st>>>(partials, nblocks, g, p, r, n, nu_min, nu_max, d_params,
                                           d_status);
  return cudaGetLastError();
}

}  // namespace cfust

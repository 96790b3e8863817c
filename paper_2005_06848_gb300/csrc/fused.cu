// Fused E-step and M-step sums: one kernel per EM iteration that takes every
// observation through all g components and leaves only the eight per-component
// sums of Section 3.2 and the log-likelihood partial (the per-block partial
// sums of Algorithm 2, combined by Algorithm 3's M-step).  The per-pair
// E-step outputs log f_ij, e1..e4 (17 numbers per pair at r = 4) live only in
// shared memory; nothing of size g n is read or written in HBM.
//
// Work unit: a tile of TJ = 8 ppw consecutive observations.  A CTA takes its
// tiles round-robin (tile = blockIdx.x, + gridDim.x, ...; a fixed assignment, so
// results do not depend on scheduling) and for each tile
//   1. for each group of components (all g when their chi tables fit beside
//      the tile: then they are staged once per CTA): stages the group's tables
//      (bulk asynchronous copy, bounded mbarrier wait, one phase per stage) and
//      paired factors, and its warps sweep the tile's (i, j) pairs exactly as
//      the per-pair sweep kernel does (pair_sweep, sweep.cuh), the outputs
//      going to shared memory;
//   2. single precision: pairs whose float sums underflowed are triaged against
//      the observation's final log f values or recomputed by the whole CTA with
//      the log-domain sweep (pair_sweep_log_cta), in (i, j) order;
//   3. tau_ij = exp(log pi_i + log f_ij - LSE_j) (Eq. 4) and l_j = LSE_j (Eq. 3),
//      then every sum entry of every component over the tile, added into the
//      CTA's own row of the partials: the same arithmetic as the posterior
//      kernel (double-float exact products and compensated tile sums in single
//      precision, double in double precision).
// The M-step finalize and the log-likelihood reduction then read the rows
// [gridDim.x][g][K] and [gridDim.x] exactly as after the posterior kernel.
#include <math.h>

#include "sums.cuh"
#include "sweep.cuh"

namespace cfust {

namespace {

constexpr int FT = 256;  // threads per CTA (8 warps)

struct FusedArgs {
  const CompT<double> *c64;  // double-precision constants of the log-domain rescue
  const double *chi64;       // [g][2][N] double chi tables of the rescue
  double *partials;          // [gridDim.x][g][K]
  double *ll_partials;       // [gridDim.x]
  int r, K, tj;
  int ntiles;
  int gs;  // components staged together (a group); gs >= g: staged once per CTA
  // the dynamic shared memory layout (fused_layout), passed in so that the
  // kernel forms its pointers from constants rather than holding them
  unsigned pcs, bar, wpc, out, flag, ys, tab_stride;
};

// Byte offsets of the CTA's dynamic shared memory: the chi tables of a group
// of gs components (component c0 + k's at k * tab_stride elements; none when
// the tables are read from global memory), the group's paired factors
// -L_th / L_tt (read at every lattice point), the staging mbarrier, the
// prioritised sweep's per-warp slots, the tile's per-pair outputs, the
// rescue flags and the tile's observations.  The per-component constants
// stay in global memory: only each pair's set-up reads them.
struct FusedLayout {
  size_t pcs, bar, wpc, out, flag, ys, total;
  int tab_stride;
};

__host__ __device__ inline FusedLayout fused_layout(size_t es, int N, int g, int p, int r, int tj, int gs, bool dens,
                                                    bool prio, bool staged) {
  const int rp = r * (r + 1) / 2;
  const int nvo = dens ? 1 : 3 + r + rp;
  FusedLayout L;
  L.tab_stride = (dens ? 1 : 2) * N;
  L.pcs = staged ? align16((size_t)gs * L.tab_stride * es) : 0;
  L.bar = L.pcs + align16((size_t)gs * sizeof(PairedConsts));
  L.wpc = L.bar + 16;
  L.out = L.wpc + (prio ? align16(8 * sizeof(PairedConsts)) : 0);
  L.flag = L.out + align16((size_t)g * tj * nvo * es);
  L.ys = L.flag + align16((size_t)g * tj);
  L.total = L.ys + (dens ? 0 : align16((size_t)tj * p * 8));
  return L;
}

__device__ __forceinline__ void fence_proxy_async_cta() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Stages components [c0, c1): their chi tables by one bulk asynchronous
// copy (one per component for the density sweep, which reads pass A's half)
// completing phase `parity` of the mbarrier, and their paired factors from
// the constants in global memory.  The caller has synchronised the CTA after
// the last read of the previous group.  Returns false after flagging
// ERR_TIMEOUT when the copy did not land in time (the block first lets it
// land, bounded, then the kernel returns).
template <typename T, bool DENS>
__device__ __forceinline__ bool fused_stage(const EArgs &a, int c0, int c1, bool staged, T *tab, PairedConsts *pcs,
                                            uint64_t *bar, uint32_t parity, int *s_fail) {
  const int N = a.N;
  const T *chi = reinterpret_cast<const T *>(a.chi);
  const CompT<T> *cs = reinterpret_cast<const CompT<T> *>(a.comp);
  if (threadIdx.x == 0) {
    *s_fail = 0;
    if (staged) {
      // the generic-proxy reads of the previous tables are ordered before the
      // asynchronous copy that overwrites them
      fence_proxy_async_cta();
      const uint32_t per = static_cast<uint32_t>((DENS ? 1 : 2) * N * sizeof(T));
      mbar_expect_tx(bar, per * (uint32_t)(c1 - c0));
      if (DENS) {
        for (int i = c0; i < c1; ++i) bulk_copy_g2s(tab + (size_t)(i - c0) * N, chi + (int64_t)i * 2 * N, per, bar);
      } else {
        bulk_copy_g2s(tab, chi + (int64_t)c0 * 2 * N, per * (uint32_t)(c1 - c0), bar);
      }
    }
  }
  for (int x = threadIdx.x; x < (c1 - c0) * RMAX * RMAX; x += blockDim.x) {
    const int k = x / (RMAX * RMAX), t = (x / RMAX) % RMAX, h = x % RMAX;
    if (h <= t) {
      const float v = -(float)cs[c0 + k].L[t * RMAX + h] * (float)cs[c0 + k].Linv[t];
      pcs[k].nL[t * (t + 1) / 2 + h] = make_float2(v, v);
    }
  }
  __syncthreads();
  if (staged) {
    if (!mbar_wait_bounded(bar, parity, a.wait_polls)) atomicOr(s_fail, 1);
    __syncthreads();
    if (*s_fail) {
      if (threadIdx.x == 0) {
        mbar_wait_bounded(bar, parity, 1 << 22);
        atomicOr(a.status, ERR_TIMEOUT);
      }
      __syncthreads();
      return false;
    }
  }
  return true;
}

// Step 2 for single precision: every flagged pair of the tile, in (i, j)
// order, by the whole CTA.  The triage compares the pair's density bound with
// the best FINAL value of the observation (pairs still flagged do not count:
// their bounds are upper bounds), so a pair is dropped only when some
// component is known to outweigh it by exp(tnats).
template <int R, bool DENS, bool SHR>
__device__ __noinline__ void fused_rescue(const EArgs &a, const FusedArgs &f, const FitView &fv, unsigned char *flag,
                                          int nt, int tj, double *sm, Prologue<R> *spr, int *skip) {
  constexpr int RP = R * (R + 1) / 2;
  const int g = fv.g;
  const float *lf = reinterpret_cast<const float *>(fv.out.logf);
  for (int i = 0; i < g; ++i) {
    for (int jj = 0; jj < nt; ++jj) {
      if (!flag[i * tj + jj]) continue;  // uniform: every thread reads the same byte
      if (threadIdx.x == 0) {
        atomicAdd(a.rescue_count, 1u);
        *skip = 0;
        if (a.triage) {
          double best = -INFINITY;
          for (int h = 0; h < g; ++h)
            if (!flag[h * tj + jj]) best = fmax(best, log(fv.pi[h]) + (double)lf[h * tj + jj]);
          const double mine = log(fv.pi[i]) + pending_bound_decode(lf[i * tj + jj]);
          if (isfinite(best) && mine < best - (double)a.tnats) {
            *skip = 1;
            const int64_t ij = (int64_t)i * tj + jj;
            store<float>(fv.out.logf, ij, -INFINITY);
            if (!DENS) {
              store<float>(fv.out.e1, ij, 0.0);
              store<float>(fv.out.e2, ij, 0.0);
              for (int t = 0; t < R; ++t) store<float>(fv.out.e3, ((int64_t)i * R + t) * tj + jj, 0.0);
              for (int t = 0; t < RP; ++t) store<float>(fv.out.e4, ((int64_t)i * RP + t) * tj + jj, 0.0);
            }
          }
        }
        if (!*skip) *spr = prologue<double, R>(a, fv, f.c64[i], jj);
      }
      __syncthreads();
      if (!*skip) {
        const double *tab = f.chi64 + (int64_t)i * 2 * a.N;
        pair_sweep_log_cta<R, DENS, SHR>(a, fv, f.c64[i], *spr, tab, tab + a.N, i, jj, sm);
      }
      if (threadIdx.x == 0) flag[i * tj + jj] = 0;
      __syncthreads();
    }
  }
}

// Step 3, log-sum-exp part, for observation jj of the tile (one thread each):
// single precision forms log pi_i + log f_ij as an exact float pair and the
// exponentials from the pairs' differences (the posterior kernel's
// arithmetic); double precision takes the plain definition.  With TAU the
// tile's log f row of every component is overwritten by tau.  Returns l_j;
// `bad` is set when no component gives the observation a positive density.
template <typename T, bool TAU>
__device__ __forceinline__ double fused_lse(T *lf, int g, int tj, int jj, const void *lpi_raw, int &bad) {
  if constexpr (sizeof(T) == 4) {
    const float2 *lpi2 = reinterpret_cast<const float2 *>(lpi_raw);
    float2 mx = make_float2(-INFINITY, 0.0f);
    for (int i = 0; i < g; ++i) {
      float2 ai = two_sum(lpi2[i].x, lf[i * tj + jj]);
      ai.y = __fadd_rn(ai.y, lpi2[i].y);
      if (ai.x > mx.x || (ai.x == mx.x && ai.y > mx.y)) mx = ai;
    }
    if (!isfinite(mx.x)) {
      bad = 1;
      if (TAU)
        for (int i = 0; i < g; ++i) lf[i * tj + jj] = 0.0f;
      return -INFINITY;
    }
    float s = 0.0f;
    for (int i = 0; i < g; ++i) {
      float2 ai = two_sum(lpi2[i].x, lf[i * tj + jj]);
      ai.y = __fadd_rn(ai.y, lpi2[i].y);
      const float dx = __fadd_rn(__fsub_rn(ai.x, mx.x), __fsub_rn(ai.y, mx.y));
      const float ex = (ai.x == -INFINITY) ? 0.0f : expf(dx);
      s = __fadd_rn(s, ex);
      if (TAU) lf[i * tj + jj] = ex;
    }
    const double lse = (double)mx.x + (double)mx.y + (double)logf(s);
    if (!isfinite(lse)) bad = 1;
    if (TAU) {
      const float inv = 1.0f / s;
      for (int i = 0; i < g; ++i) lf[i * tj + jj] *= inv;
    }
    return lse;
  } else {
    const double *lpi = reinterpret_cast<const double *>(lpi_raw);
    double mx = -INFINITY;
    for (int i = 0; i < g; ++i) mx = fmax(mx, lpi[i] + (double)lf[i * tj + jj]);
    double s = 0.0;
    for (int i = 0; i < g; ++i) {
      const double e = exp(lpi[i] + (double)lf[i * tj + jj] - mx);
      s += e;
      if (TAU) lf[i * tj + jj] = e;
    }
    const double lse = mx + log(s);
    if (!isfinite(lse)) bad = 1;
    if (TAU) {
      const double inv = 1.0 / s;
      for (int i = 0; i < g; ++i) lf[i * tj + jj] *= inv;
    }
    return lse;
  }
}

// Step 3, sums part: entry e of the tile's g K sums (component e / K, entry
// e % K of Section 3.2's packing) over observations split, split + S, ...
// of the tile, from tau (in the log f rows), e1..e4 and the staged y.
// Single precision: tau times the weight as an exact product (two-product),
// times y's float pairs (double-float), two compensated chains merged by a
// two-sum; double: the posterior kernel's four interleaved chains.
// Adds the tile's sums to the CTA's partial row (`first`: the row starts here).
template <typename T>
__device__ __forceinline__ void fused_tile_sums(const T *out, const void *ys_raw, int g, int tj, int p, int r, int K,
                                                int nt, double *prow, bool first) {
  const int E = g * K;
  const T *tau = out;  // the log f rows now hold tau
  if constexpr (sizeof(T) == 4) {
    const float2 *ys = reinterpret_cast<const float2 *>(ys_raw);
    // with few entries, S adjacent threads share one (rows split, split + S, ...)
    const int S = (4 * E <= FT) ? 4 : ((2 * E <= FT) ? 2 : 1);
    const int split = threadIdx.x % S;
    const int per = FT / S;
    for (int e0 = 0; e0 < E; e0 += per) {
      const int e = e0 + (int)threadIdx.x / S;
      float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
      if (e < E) {
        const TileCols c = tile_cols<float>(out, g, tj, p, r, K, e);
        const float *ti = tau + (size_t)(e / K) * tj;
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
      if (e < E && split == 0) prow[e] = (first ? 0.0 : prow[e]) + ((double)h0 + (double)l0);
    }
  } else {
    const double *ys = reinterpret_cast<const double *>(ys_raw);
    for (int e = threadIdx.x; e < E; e += FT) {
      const TileCols c = tile_cols<double>(out, g, tj, p, r, K, e);
      const double *ti = tau + (size_t)(e / K) * tj;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int jj = 0;
      if (c.y1 < 0) {
        for (; jj + 4 <= nt; jj += 4) {
          s0 += tile_term_f64(c, ti[jj], jj);
          s1 += tile_term_f64(c, ti[jj + 1], jj + 1);
          s2 += tile_term_f64(c, ti[jj + 2], jj + 2);
          s3 += tile_term_f64(c, ti[jj + 3], jj + 3);
        }
        for (; jj < nt; ++jj) s0 += tile_term_f64(c, ti[jj], jj);
      } else if (c.y2 < 0) {
        for (; jj + 4 <= nt; jj += 4) {
          s0 = fma(tile_term_f64(c, ti[jj], jj), ys[jj * p + c.y1], s0);
          s1 = fma(tile_term_f64(c, ti[jj + 1], jj + 1), ys[(jj + 1) * p + c.y1], s1);
          s2 = fma(tile_term_f64(c, ti[jj + 2], jj + 2), ys[(jj + 2) * p + c.y1], s2);
          s3 = fma(tile_term_f64(c, ti[jj + 3], jj + 3), ys[(jj + 3) * p + c.y1], s3);
        }
        for (; jj < nt; ++jj) s0 = fma(tile_term_f64(c, ti[jj], jj), ys[jj * p + c.y1], s0);
      } else {
        for (; jj + 4 <= nt; jj += 4) {
          s0 = fma(tile_term_f64(c, ti[jj], jj) * ys[jj * p + c.y1], ys[jj * p + c.y2], s0);
          s1 = fma(tile_term_f64(c, ti[jj + 1], jj + 1) * ys[(jj + 1) * p + c.y1], ys[(jj + 1) * p + c.y2], s1);
          s2 = fma(tile_term_f64(c, ti[jj + 2], jj + 2) * ys[(jj + 2) * p + c.y1], ys[(jj + 2) * p + c.y2], s2);
          s3 = fma(tile_term_f64(c, ti[jj + 3], jj + 3) * ys[(jj + 3) * p + c.y1], ys[(jj + 3) * p + c.y2], s3);
        }
        for (; jj < nt; ++jj) s0 = fma(tile_term_f64(c, ti[jj], jj) * ys[jj * p + c.y1], ys[jj * p + c.y2], s0);
      }
      prow[e] = (first ? 0.0 : prow[e]) + ((s0 + s1) + (s2 + s3));
    }
  }
}

// Step 1 for one group of components [c0, c1): warp w sweeps observations
// [w ppw, w ppw + ppw) of the tile through every component of the group
// without waiting for the other warps; lane k ppw + b first computes the
// double prologue of (component c0 + k, observation b) ((c1 - c0) ppw <= 32),
// and the pairs needing the rescue are recorded.
template <typename T, int R, bool DENS, bool PRIO, bool SHR>
__device__ __forceinline__ void fused_sweep_group(const EArgs &a, const FitView &fv, const PairedConsts *pcs,
                                                  PairedConsts *wpc, const T *tab, int tab_stride, int c0, int c1,
                                                  int nt, unsigned char *flag) {
  const CompT<T> *cs = reinterpret_cast<const CompT<T> *>(a.comp);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tj = (int)fv.n, ppw = a.ppw;
  const int jw0 = warp * ppw;
  const int cnt = (nt - jw0) < ppw ? ((nt - jw0) > 0 ? (nt - jw0) : 0) : ppw;
  Prologue<R> mine;
  PrioLane<R, T> pmine;
  {
    const int c = c0 + lane / ppw, b = lane % ppw;
    if (c < c1 && b < cnt) {
      mine = prologue<T, R>(a, fv, cs[c], jw0 + b);
      if constexpr (PRIO) prio_lane<R, T>(mine.q, cs[c].lam, cs[c].lamd, &pmine);
    }
  }
  for (int i = c0; i < c1; ++i) {
    const T *tA = tab + (size_t)(i - c0) * tab_stride;
    for (int b = 0; b < cnt; ++b) {
      const int src = (i - c0) * ppw + b;
      const Prologue<R> pr = shfl_prologue<R>(mine, src);
      PrioLane<R, T> pp;
      if constexpr (PRIO) pp = shfl_prio<R, T>(pmine, src);
      const bool need = pair_sweep<T, T, R, DENS, PRIO, 1, SHR>(a, fv, cs[i], pr, tA, tA + a.N, i, jw0 + b,
                                                                lane, sizeof(T) == 4, pcs + (i - c0), wpc, &pp);
      if (lane == 0) flag[i * tj + jw0 + b] = need ? 1 : 0;
    }
  }
}

template <typename T, int R, bool DENS, bool PRIO, bool SHR = false>
__global__ void __launch_bounds__(FT, sizeof(T) == 4 ? CFUST_ESTEP_MINB : 1) fused_em_kernel(EArgs a, FusedArgs f) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int RP = R * (R + 1) / 2;
  __shared__ int s_fail, s_skip, s_bad;
  __shared__ Prologue<R> s_pr;
  __shared__ double s_rsm[8 * (2 + 3 + R + RP)];
  __shared__ double s_red[FT];  // per-thread log-likelihood sums, then the block's
  __shared__ FitView s_fv;      // the tile as a fit (see below); read where used
  __shared__ __align__(16) unsigned char s_lpi[CFUST_GMAX * 8];

  const int g = a.g, p = a.p, tj = f.tj, gs = f.gs;
  const bool staged = a.staged != 0;
  T *const stab = reinterpret_cast<T *>(smem);
#define FUSED_PCS reinterpret_cast<PairedConsts *>(smem + f.pcs)
#define FUSED_BAR reinterpret_cast<uint64_t *>(smem + f.bar)
#define FUSED_WPC (PRIO ? reinterpret_cast<PairedConsts *>(smem + f.wpc) + (threadIdx.x >> 5) : nullptr)
#define FUSED_OUT reinterpret_cast<T *>(smem + f.out)
#define FUSED_FLAG (smem + f.flag)
#define FUSED_YS reinterpret_cast<void *>(smem + f.ys)

  // log pi_i once per CTA: a float pair in single precision, else a double
  for (int i = threadIdx.x; i < g; i += FT) {
    const double l = log(a.pi[i]);
    if constexpr (sizeof(T) == 4) {
      const float hi = (float)l;
      reinterpret_cast<float2 *>(s_lpi)[i] = make_float2(hi, (float)(l - (double)hi));
    } else {
      reinterpret_cast<double *>(s_lpi)[i] = l;
    }
  }
  s_red[threadIdx.x] = 0.0;
  if (threadIdx.x == 0) {
    s_bad = 0;
    if (staged) mbar_init(FUSED_BAR, 1);
    // the tile's pairs as a fit of tj observations whose outputs are the
    // shared-memory rows (stride tj): pair_sweep and the rescue address them
    // as they address the per-pair arrays
    const size_t gt = (size_t)g * tj;
    T *out = FUSED_OUT;
    s_fv.n = tj;
    s_fv.g = g;
    s_fv.pi = a.pi;
    s_fv.Y = a.Y;
    s_fv.out.logf = out;
    s_fv.out.e1 = DENS ? nullptr : out + gt;
    s_fv.out.e2 = DENS ? nullptr : out + 2 * gt;
    s_fv.out.e3 = DENS ? nullptr : out + 3 * gt;
    s_fv.out.e4 = DENS ? nullptr : out + (3 + R) * gt;
  }
  __syncthreads();
  // one group holding every component: staged once for all tiles
  const bool once = (gs >= g);
  if (once && !fused_stage<T, DENS>(a, 0, g, staged, stab, FUSED_PCS, FUSED_BAR, 0u, &s_fail)) return;
  uint32_t stage = once ? 1u : 0u;
  for (int tile = blockIdx.x; tile < f.ntiles; tile += gridDim.x) {
    const int64_t j0 = (int64_t)tile * tj;
    const int nt = (int)((a.n - j0) < tj ? (a.n - j0) : tj);
    __syncthreads();  // the previous tile's outputs, tau and staged y are no longer read
    if (threadIdx.x == 0) s_fv.Y = a.Y + j0 * p;
    __syncthreads();
    for (int c0 = 0; c0 < g; c0 += gs) {
      const int c1 = (c0 + gs < g) ? c0 + gs : g;
      if (!once) {
        if (c0 > 0) __syncthreads();  // every warp is done with the previous group
        if (!fused_stage<T, DENS>(a, c0, c1, staged, stab, FUSED_PCS, FUSED_BAR, stage & 1u, &s_fail)) return;
        ++stage;
      }
      const T *tab = staged ? stab : reinterpret_cast<const T *>(a.chi) + (int64_t)c0 * 2 * a.N;
      fused_sweep_group<T, R, DENS, PRIO, SHR>(a, s_fv, FUSED_PCS, FUSED_WPC, tab, staged ? (int)f.tab_stride : 2 * a.N,
                                          c0, c1, nt, FUSED_FLAG);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) fused_rescue<R, DENS, SHR>(a, f, s_fv, FUSED_FLAG, nt, tj, s_rsm, &s_pr, &s_skip);
    if ((int)threadIdx.x < nt) {
      int bad = 0;
      s_red[threadIdx.x] += fused_lse<T, !DENS>(FUSED_OUT, g, tj, threadIdx.x, s_lpi, bad);
      if (bad) s_bad = 1;
    }
    if constexpr (!DENS) {
      const double *yt = a.Y + j0 * p;
      for (int idx = threadIdx.x; idx < nt * p; idx += FT) {
        const double y = yt[idx];
        if constexpr (sizeof(T) == 4) {
          const float yh = (float)y;
          reinterpret_cast<float2 *>(FUSED_YS)[idx] = make_float2(yh, (float)(y - (double)yh));
        } else {
          reinterpret_cast<double *>(FUSED_YS)[idx] = y;
        }
      }
      __syncthreads();
      fused_tile_sums<T>(FUSED_OUT, FUSED_YS, g, tj, p, R, f.K, nt, f.partials + (int64_t)blockIdx.x * g * f.K,
                         tile == (int)blockIdx.x);
    }
  }
  __syncthreads();
  for (int h = FT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s_red[threadIdx.x] += s_red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    f.ll_partials[blockIdx.x] = s_red[0];
    if (s_bad) atomicOr(a.status, ERR_ZERO_DENSITY);
  }
#undef FUSED_PCS
#undef FUSED_BAR
#undef FUSED_WPC
#undef FUSED_OUT
#undef FUSED_FLAG
#undef FUSED_YS
}

// Tile size and staging for one launch: tiles of 8 ppw observations with
// about 64 tiles per resident CTA (at most 4 observations per warp), and
// groups of as many components as fit beside the tile, gs ppw <= 32 (every
// component at once when possible: then they are staged once per CTA).  In
// single precision a CTA keeps to about 100 KB so that two share an SM; when
// not even one component fits (in up to 220 KB) the tables are read from
// global memory.
struct FusedPlan {
  int ppw, gs, staged;
  size_t smem;
};

template <typename T, int R, bool DENS, bool PRIO>
bool fused_plan(int N, int g, int p, int64_t n, int ppw_req, FusedPlan *pl) {
  constexpr size_t LIMIT = 220u * 1024u;  // the static shared memory stays below 7 KB
  const size_t pair_limit = sizeof(T) == 4 ? 100u * 1024u : LIMIT;
  int ppw0 = ppw_req;
  if (ppw0 <= 0) {
    const int64_t v = n / ((int64_t)sm_count() * 2 * 8 * 64);
    ppw0 = (int)(v < 1 ? 1 : (v > 4 ? 4 : v));
  }
  for (const size_t lim : {pair_limit, LIMIT})
    for (int ppw = ppw0; ppw >= 1; ppw = (ppw > 1 ? ppw / 2 : 0))
      for (int gs = (g < 32 / ppw ? g : 32 / ppw); gs >= 1; --gs) {
        const FusedLayout L = fused_layout(sizeof(T), N, g, p, R, 8 * ppw, gs, DENS, PRIO, true);
        if (L.total <= lim) {
          *pl = FusedPlan{ppw, gs, 1, L.total};
          return true;
        }
      }
  for (int ppw = ppw0; ppw >= 1; ppw = (ppw > 1 ? ppw / 2 : 0)) {
    const int gs = g < 32 / ppw ? g : 32 / ppw;
    const FusedLayout L = fused_layout(sizeof(T), N, g, p, R, 8 * ppw, gs, DENS, PRIO, false);
    if (L.total <= LIMIT) {
      *pl = FusedPlan{ppw, gs, 0, L.total};
      return true;
    }
  }
  return false;
}

template <typename T, int R, bool DENS, bool PRIO, bool SHR = false>
cudaError_t fused_launch(EArgs a, FusedArgs f, int64_t n, int ppw_req, cudaStream_t st, SweepTiming tm,
                         int *nblocks) {
  FusedPlan pl;
  if (!fused_plan<T, R, DENS, PRIO>(a.N, a.g, a.p, n, ppw_req, &pl)) return cudaErrorInvalidValue;
  const void *kern = (const void *)fused_em_kernel<T, R, DENS, PRIO, SHR>;
  cudaError_t e = raise_smem_limit(kern, pl.smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, FT, pl.smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  a.ppw = pl.ppw;
  a.staged = pl.staged;
  f.gs = pl.gs;
  {
    const FusedLayout L = fused_layout(sizeof(T), a.N, a.g, a.p, R, 8 * pl.ppw, pl.gs, DENS, PRIO, pl.staged != 0);
    f.pcs = (unsigned)L.pcs;
    f.bar = (unsigned)L.bar;
    f.wpc = (unsigned)L.wpc;
    f.out = (unsigned)L.out;
    f.flag = (unsigned)L.flag;
    f.ys = (unsigned)L.ys;
    f.tab_stride = (unsigned)L.tab_stride;
  }
  f.tj = 8 * pl.ppw;
  const int64_t ntiles = (n + f.tj - 1) / f.tj;
  if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  f.ntiles = (int)ntiles;
  int64_t nb = (int64_t)occ * sm_count();
  if (nb > fused_max_blocks()) nb = fused_max_blocks();
  if (nb > f.ntiles) nb = f.ntiles;
  *nblocks = (int)nb;
  if (sizeof(T) == 4) {
    e = cudaMemsetAsync(a.rescue_count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  const unsigned evflag = tm.capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (tm.start) {
    e = cudaEventRecordWithFlags(tm.start, st, evflag);
    if (e != cudaSuccess) return e;
  }
  fused_em_kernel<T, R, DENS, PRIO, SHR><<<(unsigned)nb, FT, pl.smem, st>>>(a, f);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (tm.stop) e = cudaEventRecordWithFlags(tm.stop, st, evflag);
  return e;
}

// pass B on pass A's points (shr) has its own instantiations for full sweeps
template <typename T, bool DENS>
cudaError_t fused_dispatch(int r, bool prio, bool shr, EArgs a, FusedArgs f, int64_t n, int ppw, cudaStream_t st,
                           SweepTiming tm, int *nb) {
  shr = shr && !DENS;
  switch (r) {
    case 1:
      return shr ? fused_launch<T, 1, DENS, false, !DENS>(a, f, n, ppw, st, tm, nb)
                 : fused_launch<T, 1, DENS, false>(a, f, n, ppw, st, tm, nb);
#define CFUST_FUSED_R(R)                                                                  \
  case R:                                                                                 \
    if (shr)                                                                              \
      return prio ? fused_launch<T, R, DENS, true, !DENS>(a, f, n, ppw, st, tm, nb)       \
                  : fused_launch<T, R, DENS, false, !DENS>(a, f, n, ppw, st, tm, nb);     \
    return prio ? fused_launch<T, R, DENS, true>(a, f, n, ppw, st, tm, nb)                \
                : fused_launch<T, R, DENS, false>(a, f, n, ppw, st, tm, nb);
    CFUST_FUSED_R(2)
    CFUST_FUSED_R(3)
    CFUST_FUSED_R(4)
    CFUST_FUSED_R(5)
    CFUST_FUSED_R(6)
#undef CFUST_FUSED_R
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int fused_max_blocks() { return sm_count() * 4; }

cudaError_t launch_fused(int precision, const double *Y, int64_t n, int g, int p, int r, const LatticeDev &lat,
                         const CompT<double> *c64, const CompT<float> *c32, const double *chi64, const float *chi32,
                         bool density_only, int e2_mode, int *d_status, unsigned *rescue_count, int pairs_per_warp,
                         double *partials, double *ll_partials, const double *d_pi, float tnats, int prio,
                         int shared, cudaStream_t st, SweepTiming tm, int *nblocks) {
  if (n <= 0 || g < 1 || g > CFUST_GMAX || r < 1 || r > RMAX) return cudaErrorInvalidValue;
  EArgs a{};
  a.Y = Y;
  a.n = n;
  a.g = g;
  a.p = p;
  a.N = lat.n;
  for (int t = 0; t <= RMAX; ++t) {
    a.z[t] = lat.z[t];
    a.step[t] = lat.step[t];
    a.sint[t] = lat.sint[t];
    a.sfrac[t] = lat.sfrac[t];
  }
  a.utab = lat.utab;
  a.utab2 = lat.utab2;
  a.e2_mode = e2_mode;
  a.ppw = 1;
  a.staged = 1;
  a.rescue_list = nullptr;
  a.rescue_count = rescue_count;
  a.status = d_status;
  a.triage = 1;
  a.pi = d_pi;
  a.tnats = tnats;
  a.prio = prio ? 1 : 0;
  a.shr = shared ? 1 : 0;
  a.wait_polls = lat.wait_polls;
  FusedArgs f{};
  f.c64 = c64;
  f.chi64 = chi64;
  f.partials = partials;
  f.ll_partials = ll_partials;
  f.r = r;
  f.K = sums_width(p, r);
  const bool pr = prio != 0, sh = shared != 0;
  if (precision == CFUST_FP64) {
    a.comp = c64;
    a.chi = chi64;
    return density_only ? fused_dispatch<double, true>(r, pr, sh, a, f, n, pairs_per_warp, st, tm, nblocks)
                        : fused_dispatch<double, false>(r, pr, sh, a, f, n, pairs_per_warp, st, tm, nblocks);
  }
  a.comp = c32;
  a.chi = chi32;
  return density_only ? fused_dispatch<float, true>(r, pr, sh, a, f, n, pairs_per_warp, st, tm, nblocks)
                      : fused_dispatch<float, false>(r, pr, sh, a, f, n, pairs_per_warp, st, tm, nblocks);
}

}  // namespace cfust

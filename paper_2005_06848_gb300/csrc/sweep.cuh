// Device building blocks of the E-step lattice sweeps, shared by the
// per-pair sweep kernels (estep.cu) and the fused E-step + M-step-sums kernel
// (fused.cu).  Everything here has internal linkage: each translation unit
// compiles its own copy.
//
// E-step lattice sweeps: one warp per (observation j, component i) pair, the
// lattice points spread over the 32 lanes, warp-shuffle reductions.
//
// For pair (i, j), with z = A (y_j - mu_i), d = z^T z, q = B z (Eq. 2; this
// prologue always in double, one lane per pair, broadcast by shuffles):
//   log f_ij = c0 - ((nu+p)/2) log(1 + d/nu) + log T_A
//   pass A: T_A = P(L V > a_A), V ~ t_r(0, I, nu+p),   a_A = -q sqrt((nu+p)/(nu+d))
//   pass B: T_B, E[V], E[V V^T] for V ~ t_r(0, I, nu+p+2), a_B = -q sqrt((nu+p+2)/(nu+d))
// each probability by Genz's separation of variables over the shifted lattice:
//   lim_t = (a_t s - sum_{h<t} L_th z_h) / L_tt,  p_t = Phi(-lim_t),
//   z_t = -Phi^{-1}(max((1 - u_t) p_t, tiny)),   weight w = prod_t p_t,  V = z / s,
// s the chi scale of the point (a per-component table).  Both passes share
// the lattice point and run interleaved in one sweep; with shared_points,
// pass B is instead estimated on pass A's draws with the weight s^2 (the
// chi-square density ratio x / (nu+p), x = (nu+p) s^2).  The per-pair outputs
// are the E-step expectations of the latent gamma W and truncated normal U:
//   e1 = (nu+p)/(nu+d) T_B/T_A,  sigma = sqrt((nu+d)/(nu+p+2)),
//   e3 = e1 (q + sigma L E[V]),
//   e4 = e1 (q q^T + sigma (q (L E[V])^T + (L E[V]) q^T) + sigma^2 L E[V V^T] L^T),
//   e2 = e1 - log((nu+d)/2) - (nu+p)/(nu+d) + psi((nu+p)/2)     (e2_mode 0)
//      = E_w[log chi^2_{nu+p}] - log(nu+d)                         (e2_mode 1).
// Where T_A or T_B is 0, e1..e4 are 0 (their posterior weight is 0).
//
// Single precision: the sweep runs in float with this library's normal tail
// and quantile approximations (normal_f32.cuh); a pair whose lattice sum falls
// below 1e-20 N in either pass (point weights near the float underflow) or whose
// result is not finite is queued and recomputed by rescue_kernel, a float sweep
// that carries every point weight as a logarithm and accumulates with a running
// maximum.  Double precision calls CUDA's normcdf / normcdfinv.
#pragma once

#include <math.h>

#include "cfust_internal.cuh"
#include "normal_f32.cuh"

namespace cfust {

namespace {

template <typename T>
struct Num;

// upper_pq(y): p = Phi(-y) and q = 1 - p; neg_quantile(um, u, p, q) =
// -Phi^{-1}(um p) with u = 1 - um.  The float versions take the quantile on
// the smaller side (normal_f32.cuh); the double versions follow the plain
// definition, -Phi^{-1}(max(um p, tiny)).
template <>
struct Num<float> {
  __device__ static void upper_pq(float y, float &p, float &q) { phi_upper_pq_fast_f32(y, p, q); }
  __device__ static float neg_quantile(float um, float u, float p, float q) {
    return neg_quantile_f32(um, u, p, q);
  }
  // 2^-53, the same clamp as double precision: a normal float, so the small
  // side of a lattice coordinate keeps its value down to where the oracle clamps
  __device__ static constexpr float umin() { return 1.1102230246251565e-16f; }
  __device__ static float lg(float x) { return logf(x); }
  __device__ static float sq(float x) { return sqrtf(x); }
  __device__ static float ab(float x) { return fabsf(x); }
  __device__ static float mn(float x, float y) { return fminf(x, y); }
  __device__ static float mx(float x, float y) { return fmaxf(x, y); }
};

template <>
struct Num<double> {
  __device__ static void upper_pq(double y, double &p, double &q) {
    p = normcdf(-y);
    q = 1.0 - p;
  }
  __device__ static double neg_quantile(double um, double, double p, double) {
    return -normcdfinv(fmax(um * p, 2.2250738585072014e-308));
  }
  __device__ static constexpr double umin() { return 1.1102230246251565e-16; }  // 2^-53
  __device__ static double lg(double x) { return log(x); }
  __device__ static double sq(double x) { return sqrt(x); }
  __device__ static double ab(double x) { return fabs(x); }
  __device__ static double mn(double x, double y) { return fmin(x, y); }
  __device__ static double mx(double x, double y) { return fmax(x, y); }
};

struct EArgs {
  const double *Y;
  int64_t n;
  int g, p, N;
  int z[RMAX + 1];
  int step[RMAX + 1];
  int sint[RMAX + 1];
  double sfrac[RMAX + 1];
  const float *utab; // lattice uniforms, [N][uniform_stride(r)] (single precision sweeps)
  const float *utab2; // the same, pair-interleaved for the shared-points sweep (LatticeDev::utab2)
  const void *comp;  // CompT<T>[g]
  const void *chi;   // T[g][2][N]
  EstepOut out;
  int e2_mode;
  int ppw;           // pairs per warp (observations of one component)
  int staged;
  unsigned long long *rescue_list;
  unsigned *rescue_count;
  int *status;
  int triage;          // 1: skip queued pairs whose posterior weight is provably negligible
  const double *pi;    // device [g], read by the triage
  float tnats;         // the triage's margin: tau_ij < exp(-tnats) counts as negligible
  int prio;            // 1: variable prioritisation (every sweep and its rescue)
  int shr;             // 1: pass B estimated on pass A's lattice points (see pair_sweep)
  int wait_polls;      // polls of the staging wait before it gives up (LatticeDev::wait_polls)
};

// The per-fit part of a sweep: observations, their count, the component
// count, the per-pair output arrays and the mixing proportions.  A single fit
// takes it from EArgs; the batched sweep builds one per work item.
struct FitView {
  const double *Y;
  int64_t n;
  int g;
  EstepOut out;
  const double *pi;
};

__device__ __forceinline__ FitView fit_view(const EArgs &a) {
  FitView f;
  f.Y = a.Y;
  f.n = a.n;
  f.g = a.g;
  f.out = a.out;
  f.pi = a.pi;
  return f;
}

// Queued pair: component index in the high 32 bits, observation in the low.
__device__ __forceinline__ unsigned long long pair_id(int i, int64_t j) {
  return ((unsigned long long)(unsigned)i << 32) | (unsigned long long)j;
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ---- bulk async copy global -> shared, completion on an mbarrier ---------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, "
      "P;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait: gives up after `limit` polls (each poll itself blocks for a
// hardware-chosen interval), so a lost completion can never hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename OT, typename T>
__device__ __forceinline__ void store(void *base, int64_t idx, T v) {
  reinterpret_cast<OT *>(base)[idx] = static_cast<OT>(v);
}

// Per-component operands of the paired sweep, duplicated into (x, x) pairs,
// kept in shared memory so they occupy no registers.
struct PairedConsts {
  float2 nL[RMAX * (RMAX + 1) / 2];  // -L_th / L_tt (h < t), packed lower triangle
};

// One pair's variable order and the factor of its permuted Lambda (variable
// prioritisation), written by one thread, read by the warp (or CTA) sweeping it.
struct PrioSlot {
  double q[RMAX];                      // q in the prioritised order
  double L[RMAX * (RMAX + 1) / 2];     // Cholesky factor of the permuted Lambda, packed lower
  double Li[RMAX];                     // 1 / L_tt
  int ord[RMAX];                       // original coordinate of position t
  PairedConsts pc;                     // -L_th / L_tt pairs for the paired sweep
};

// Variable prioritisation (Genz's reordering, this library's reading): the
// coordinates are integrated in decreasing order of the standardised limit
// -q_t / sqrt(Lambda_tt) (pass B's limits are a positive multiple of pass
// A's, so one order serves both), ties keeping the lower index, with the
// Cholesky factor of the permuted Lambda.  The order is decided in double
// from the double prologue, as the oracle decides it; the factor is formed
// in the sweep's precision T (double work costs 64 times single on this GPU,
// and the single-precision sweep rounds the factor to float anyway).  Not
// inlined: its dynamically indexed arrays stay out of the sweep's registers.
template <int R, typename T>
__device__ __noinline__ void prio_setup(const double *q, const double *lam, const double *lamd, PrioSlot *s) {
  int ord[R];
  double key[R];
  for (int t = 0; t < R; ++t) {
    ord[t] = t;
    key[t] = -q[t] * lamd[t];
  }
  for (int t = 1; t < R; ++t) {  // stable insertion sort, descending
    const int o = ord[t];
    const double k = key[t];
    int u = t - 1;
    while (u >= 0 && key[u] < k) {
      key[u + 1] = key[u];
      ord[u + 1] = ord[u];
      --u;
    }
    key[u + 1] = k;
    ord[u + 1] = o;
  }
  T Lm[R * R];
  for (int t = 0; t < R; ++t)
    for (int h = 0; h <= t; ++h) {
      const int x = ord[t] > ord[h] ? ord[t] : ord[h], y = ord[t] > ord[h] ? ord[h] : ord[t];
      Lm[t * R + h] = static_cast<T>(lam[x * (x + 1) / 2 + y]);
    }
  for (int j = 0; j < R; ++j) {
    T d = Lm[j * R + j];
    for (int k = 0; k < j; ++k) d -= Lm[j * R + k] * Lm[j * R + k];
    // a permutation of a positive definite Lambda stays so
    d = Num<T>::sq(d > T(0) ? d : static_cast<T>(sizeof(T) == 4 ? 1e-30 : 1e-300));
    Lm[j * R + j] = d;
    for (int i = j + 1; i < R; ++i) {
      T v = Lm[i * R + j];
      for (int k = 0; k < j; ++k) v -= Lm[i * R + k] * Lm[j * R + k];
      Lm[i * R + j] = v / d;
    }
  }
  for (int t = 0; t < R; ++t) {
    s->ord[t] = ord[t];
    s->q[t] = q[ord[t]];
    const T li = T(1) / Lm[t * R + t];
    s->Li[t] = (double)li;
    for (int h = 0; h <= t; ++h) {
      s->L[t * (t + 1) / 2 + h] = (double)Lm[t * R + h];
      const float v = -(float)Lm[t * R + h] * (float)li;
      s->pc.nL[t * (t + 1) / 2 + h] = make_float2(v, v);
    }
  }
}

// The same order and factor held per lane: in a warp's chunk of pairs every
// lane prepares its own pair (as it computes its prologue), and the warp
// takes pair b's values by shuffles when it sweeps it.  ord packs the
// original coordinate of position t in bits 3t .. 3t + 2.
template <int R, typename T>
struct PrioLane {
  T q[R];
  T L[R * (R + 1) / 2];
  T Li[R];
  int ord;
};

template <int R, typename T>
__device__ __noinline__ void prio_lane(const double *q, const double *lam, const double *lamd, PrioLane<R, T> *o) {
  PrioSlot s;
  prio_setup<R, T>(q, lam, lamd, &s);
  int packed = 0;
  for (int t = 0; t < R; ++t) {
    packed |= s.ord[t] << (3 * t);
    o->q[t] = static_cast<T>(s.q[t]);
    o->Li[t] = static_cast<T>(s.Li[t]);
    for (int h = 0; h <= t; ++h) o->L[t * (t + 1) / 2 + h] = static_cast<T>(s.L[t * (t + 1) / 2 + h]);
  }
  o->ord = packed;
}

template <int R, typename T>
__device__ __forceinline__ PrioLane<R, T> shfl_prio(const PrioLane<R, T> &m, int src) {
  PrioLane<R, T> o;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    o.q[t] = __shfl_sync(0xffffffffu, m.q[t], src);
    o.Li[t] = __shfl_sync(0xffffffffu, m.Li[t], src);
  }
#pragma unroll
  for (int k = 0; k < R * (R + 1) / 2; ++k) o.L[k] = __shfl_sync(0xffffffffu, m.L[k], src);
  o.ord = __shfl_sync(0xffffffffu, m.ord, src);
  return o;
}

// Lattice constants of coordinate t for the double-precision sweep (the
// single-precision sweep reads its uniforms from the lattice table).
__device__ __forceinline__ double lat_sf(const EArgs &a, int t) { return a.sfrac[t]; }
__device__ __forceinline__ double lat_two_sf(const EArgs &a, int t) { return 2.0 * a.sfrac[t]; }
__device__ __forceinline__ double lat_step2(const EArgs &a, int t) { return (double)(2 * a.step[t]); }

// A pair left to the double-precision rescue keeps an upper bound of its
// log f in its log f slot until the rescue, stored as a quiet NaN whose
// payload is the bound (ceil(8 ub) + 2^21 in 22 bits: eighths of a nat over
// +-262144 nats; a bound below that range is stored as its lower end, still
// an upper bound; the top payload means +inf).  A maximum over an
// observation's log f values (fmax) skips it, so a triage compares with final
// values only, and the pair's own test decodes its bound.
__device__ __forceinline__ float pending_bound_encode(double ub) {
  unsigned payload = 0x3FFFFFu;
  if (ub < 262143.0) {
    const double c = ceil(ub * 8.0) + 2097152.0;
    payload = c > 0.0 ? (unsigned)c : 0u;
  }
  return __uint_as_float(0x7FC00000u | payload);
}
__device__ __forceinline__ double pending_bound_decode(float v) {
  const unsigned payload = __float_as_uint(v) & 0x3FFFFFu;
  return payload == 0x3FFFFFu ? INFINITY : ((double)payload - 2097152.0) * 0.125;
}

// Per-pair prologue in double precision: z = A (y - mu), d = z^T z, q = B z and
// the log of the t_p factor with the constant c0 of Eq. 2.
template <int R>
struct Prologue {
  double d, logt;
  double q[R];
};

template <typename T, int R>
__device__ __forceinline__ Prologue<R> prologue(const EArgs &a, const FitView &fv, const CompT<T> &c,
                                                int64_t j) {
  Prologue<R> pr;
  const int p = a.p;
  const double *yj = fv.Y + j * (int64_t)p;
  double yc[PMAX];
#pragma unroll
  for (int k = 0; k < PMAX; ++k) yc[k] = (k < p) ? yj[k] - c.mu[k] : 0.0;
#pragma unroll
  for (int t = 0; t < R; ++t) pr.q[t] = 0.0;
  double d = 0.0;
#pragma unroll
  for (int k = 0; k < PMAX; ++k) {
    if (k < p) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l <= k; ++l) acc += c.A[k * PMAX + l] * yc[l];
      d += acc * acc;
#pragma unroll
      for (int t = 0; t < R; ++t) pr.q[t] += c.B[t * PMAX + k] * acc;
    }
  }
  pr.d = d;
  // log t_p, or log phi_p at nu = inf (the skew-normal limit)
  pr.logt = isinf(c.nu) ? c.c0 - 0.5 * d : c.c0 - 0.5 * c.mA * log1p(d / c.nu);
  return pr;
}

template <int R>
__device__ __forceinline__ Prologue<R> shfl_prologue(const Prologue<R> &mine, int src) {
  Prologue<R> o;
  o.d = __shfl_sync(0xffffffffu, mine.d, src);
  o.logt = __shfl_sync(0xffffffffu, mine.logt, src);
#pragma unroll
  for (int t = 0; t < R; ++t) o.q[t] = __shfl_sync(0xffffffffu, mine.q[t], src);
  return o;
}

// Single-precision sums of one pair with pass B on pass A's lattice points.
// Pass B's law differs from pass A's only in the chi variable (dof m_B = m_A + 2
// for m_A = nu + p), and chi2_{m+2}(x) = chi2_m(x) x / m: with x = m_A s^2 at
// pass A's chi scale s of a point, pass B's scaled limit equals pass A's, so
// pass B takes pass A's weight w and draws z with the extra weight s^2, and
// V = z / (s c), c = sqrt(m_A / m_B).  Returned: SA = sum w, SB = sum w s^2,
// M1 = sum w s z (= c sum w_B V), M2 = sum w z z^T (= c^2 sum w_B V V^T), SL
// (e2_mode 1) = sum w (log m_A + 2 log s).  Each lane takes the points k and
// k + 32 side by side in FP32x2 operations (.x and .y); a second point past
// N repeats the first and gets weight 0.
template <int R>
__device__ __forceinline__ void shared_point_sums(const EArgs &a, int lane, const float *__restrict__ tA,
                                                  const float2 (&ab2)[R], const PairedConsts *pcu, bool e2lat,
                                                  float logmA, float &SA, float &SB, float &SL, float (&M1)[R],
                                                  float (&M2)[R * (R + 1) / 2]) {
  constexpr int RP = R * (R + 1) / 2;
  constexpr int US = uniform_stride(R);
  const int N = a.N;
  float2 sa2 = make_float2(0.f, 0.f), sb2 = make_float2(0.f, 0.f);
  float2 m1[R], m2[RP];
#pragma unroll
  for (int t = 0; t < R; ++t) m1[t] = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < RP; ++t) m2[t] = make_float2(0.f, 0.f);
  float sl = 0.f;
  for (int k = lane; k < N; k += 2 * WARP) {
    const bool two = k + WARP < N;
    const int k2 = two ? k + WARP : k;
    // the uniforms of points k and k + 32 as (k, k + 32) pairs, column by
    // column: entry (k / 64, lane) of the pair-interleaved table
    const float4 *rp = reinterpret_cast<const float4 *>(a.utab2) + (size_t)((k >> 6) * WARP + lane) * (US / 2);
    float2 v2[US];
#pragma unroll
    for (int q4 = 0; q4 < US / 2; ++q4) {
      const float4 f = __ldg(rp + q4);
      v2[2 * q4] = make_float2(f.x, f.y);
      v2[2 * q4 + 1] = make_float2(f.z, f.w);
    }
    const float2 s2 = make_float2(tA[k], tA[k2]);
    float2 w2;
    float2 z2[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float2 acc2 = __fmul2_rn(ab2[t], s2);
#pragma unroll
      for (int h = 0; h < t; ++h) acc2 = __ffma2_rn(pcu->nL[t * (t + 1) / 2 + h], z2[h], acc2);
      float2 p2, q2;
      phi_upper_pq_x2(acc2, p2, q2);
      w2 = (t == 0) ? p2 : __fmul2_rn(w2, p2);
      z2[t] = neg_quantile_x2v(v2[t], v2[R + t], p2, q2);
    }
    if (!two) w2.y = 0.0f;
    sa2 = __fadd2_rn(sa2, w2);
    if (e2lat) sl += w2.x * (logmA + 2.0f * logf(s2.x)) + w2.y * (logmA + 2.0f * logf(s2.y));
    const float2 ws = __fmul2_rn(w2, s2);
    sb2 = __ffma2_rn(ws, s2, sb2);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      m1[t] = __ffma2_rn(ws, z2[t], m1[t]);
      const float2 u = __fmul2_rn(w2, z2[t]);
#pragma unroll
      for (int h = 0; h <= t; ++h) m2[t * (t + 1) / 2 + h] = __ffma2_rn(u, z2[h], m2[t * (t + 1) / 2 + h]);
    }
  }
  SA = sa2.x + sa2.y;
  SB = sb2.x + sb2.y;
  SL = sl;
#pragma unroll
  for (int t = 0; t < R; ++t) M1[t] = m1[t].x + m1[t].y;
#pragma unroll
  for (int t = 0; t < RP; ++t) M2[t] = m2[t].x + m2[t].y;
}

// One (i, j) pair on one warp, its prologue given.  Returns true (uniformly
// over the warp) when `check` is set and the single-precision sweep needs the
// double rescue; in that case nothing is written.  With SHR, pass B is
// estimated on pass A's lattice points (shared_point_sums; the
// double-precision sweep does the same per point): one conditional chain per
// point instead of two.  PTS > 1 lets the paired two-pass loop keep two
// lattice points in flight.
template <typename T, typename OT, int R, bool DENS, bool PRIO = false, int PTS = 1, bool SHR = false>
__device__ __forceinline__ bool pair_sweep(const EArgs &a, const FitView &fv, const CompT<T> &c,
                                           const Prologue<R> &pr,
                                           const T *__restrict__ tA, const T *__restrict__ tB,
                                           int i, int64_t j, int lane, bool check,
                                           const PairedConsts *pc, PairedConsts *wpc,
                                           const PrioLane<R, T> *pp) {
  using M = Num<T>;
  constexpr int RP = R * (R + 1) / 2;
  constexpr bool PAIRED = (sizeof(T) == 4) && !DENS;
  const int N = a.N;
  // per-pair scalars, run by every lane: in the precision of the sweep (FP64
  // divides, roots and logarithms cost 64x on this GPU, and in single
  // precision every one of these rounds to float anyway)
  // at nu = inf (the skew-normal limit) W = 1: both passes take the limits
  // -q with scale 1, so their sums agree bit for bit and e1 = 1, e2 = 0
  const bool nrm = isinf(c.nu);
  const T nud = static_cast<T>(c.nu + pr.d);
  const T mAT = static_cast<T>(c.mA), mBT = static_cast<T>(c.mB);
  const T fA = nrm ? T(1) : M::sq(mAT / nud), fB = nrm ? T(1) : M::sq(mBT / nud);
  T q[R], aA[R], aB[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    q[t] = static_cast<T>(pr.q[t]);
    aA[t] = -q[t] * fA;
    aB[t] = -q[t] * fB;
  }
  T Lc[RP], Li[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    Li[t] = c.Linv[t];
#pragma unroll
    for (int h = 0; h <= t; ++h) Lc[t * (t + 1) / 2 + h] = c.L[t * RMAX + h];
  }
  // variable prioritisation: the pair's order and permuted factor (prepared
  // lane-parallel with the prologues); the sweep runs in that order and the
  // moments are stored back at their original coordinates
  int ord[R];
#pragma unroll
  for (int t = 0; t < R; ++t) ord[t] = t;
  const PairedConsts *pcu = pc;
  if constexpr (PRIO) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      ord[t] = (pp->ord >> (3 * t)) & 7;
      q[t] = pp->q[t];
      aA[t] = -q[t] * fA;
      aB[t] = -q[t] * fB;
      Li[t] = pp->Li[t];
#pragma unroll
      for (int h = 0; h <= t; ++h) Lc[t * (t + 1) / 2 + h] = pp->L[t * (t + 1) / 2 + h];
    }
    if constexpr (PAIRED) {
      // the paired loop reads -L_th / L_tt from shared memory: this warp's slot
      __syncwarp();  // every lane is done with the slot's previous pair
#pragma unroll
      for (int t = 1; t < R; ++t)
#pragma unroll
        for (int h = 0; h < t; ++h) {
          const int k = t * (t + 1) / 2 + h;
          if (lane == k) {
            const float v = -(float)Lc[k] * (float)Li[t];
            wpc->nL[k] = make_float2(v, v);
          }
        }
      __syncwarp();
      pcu = wpc;
    }
  }
  // paired operands: (pass A, pass B) limits; -L and 1/L_tt pairs come from shared memory
  // (pass A, pass B) limits over L_tt: with the staged -L_th / L_tt the
  // standardised limit of coordinate t is one multiply-add chain per point
  float2 ab2[R];
  if constexpr (PAIRED) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const float li = (float)Li[t];
      ab2[t] = make_float2((float)aA[t] * li, (float)aB[t] * li);
    }
  }

  // lattice state: fm_t = 2 m_t - N with m_t = (k z_t + sint_t) mod N for this
  // lane's point; integers below 2^17 are exact in float, so the update is exact
  T fm[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int m0 = static_cast<int>(((int64_t)lane * a.z[t + 1] + a.sint[t + 1]) % N);
    fm[t] = static_cast<T>(2 * m0 - N);
  }
  const T fN = static_cast<T>(N);
  const T invN = T(1) / fN;
  const T umin = M::umin();
  const T umax = T(1) - (sizeof(T) == 4 ? T(5.9604644775390625e-08) : umin);  // largest value below 1
  const bool e2lat = (a.e2_mode == 1);
  const T logmA = static_cast<T>(c.logmA);

  T SA = T(0), SL = T(0), SB = T(0);
  T M1[R], M2[RP];
#pragma unroll
  for (int t = 0; t < R; ++t) M1[t] = T(0);
#pragma unroll
  for (int t = 0; t < RP; ++t) M2[t] = T(0);

  // paired sweeps up to r = 4 keep two lattice points in flight per lane:
  // their dependency chains (a point's conditional draws are sequential in t)
  // interleave, and each lane's sums still take the points in the same order.
  // Larger r and the prioritised form would spill at the register cap.
  constexpr int kPoints = (PAIRED && !PRIO && R <= 4) ? PTS : 1;
  float2 SAB = make_float2(0.0f, 0.0f);  // paired sweeps: (SA, SB) side by side
  if constexpr (PAIRED && SHR) {
    float2 abs2[R];
#pragma unroll
    for (int t = 0; t < R; ++t) abs2[t] = make_float2(ab2[t].x, ab2[t].x);
    float sa, sb, sl;
    shared_point_sums<R>(a, lane, tA, abs2, pcu, e2lat, logmA, sa, sb, sl, M1, M2);
    SAB = make_float2(sa, sb);
    SL = sl;
  } else {
#pragma unroll kPoints
  for (int k = lane; k < N; k += WARP) {
    // 1 - u_t = |2 m - N + 2 sfrac| / N and u_t = 2 min(m + sfrac, N - m - sfrac) / N,
    // each formed from an exact integer and the fraction so the small side stays exact;
    // in single precision they come from the lattice's table (the same numbers)
    T um[R], uu[R];
    if constexpr (sizeof(T) == 4) {
      constexpr int US = uniform_stride(R);
      const float4 *row = reinterpret_cast<const float4 *>(a.utab) + (size_t)k * (US / 4);
      float v[US];
#pragma unroll
      for (int q4 = 0; q4 < US / 4; ++q4) {
        const float4 f4 = __ldg(row + q4);
        v[4 * q4] = f4.x;
        v[4 * q4 + 1] = f4.y;
        v[4 * q4 + 2] = f4.z;
        v[4 * q4 + 3] = f4.w;
      }
#pragma unroll
      for (int t = 0; t < R; ++t) {
        um[t] = v[t];
        uu[t] = v[R + t];
      }
    } else {
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const T sf = static_cast<T>(lat_sf(a, t + 1));
        const T mm = T(0.5) * (fm[t] + fN);
        const T lo = mm + sf, hi = (fN - mm) - sf;
        um[t] = M::mn(M::mx(M::ab(fm[t] + static_cast<T>(lat_two_sf(a, t + 1))) * invN, umin), umax);
        uu[t] = M::mx(T(2) * M::mn(lo, hi) * invN, umin);
        fm[t] += static_cast<T>(lat_step2(a, t + 1));
        if (fm[t] >= fN) fm[t] -= T(2) * fN;
      }
    }
    if constexpr (PAIRED) {
      // passes A and B side by side in FP32x2: .x is pass A, .y pass B
      const float2 s2 = make_float2(tA[k], tB[k]);
      float2 w2;
      float2 z2[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float2 acc2 = __fmul2_rn(ab2[t], s2);
#pragma unroll
        for (int h = 0; h < t; ++h) acc2 = __ffma2_rn(pcu->nL[t * (t + 1) / 2 + h], z2[h], acc2);
        float2 p2, q2;
        phi_upper_pq_x2(acc2, p2, q2);
        w2 = (t == 0) ? p2 : __fmul2_rn(w2, p2);
        // the last draw feeds pass B's moments only: pass A's half is not formed
        if (t + 1 < R)
          z2[t] = neg_quantile_x2(um[t], uu[t], p2, q2);
        else
          z2[t] = make_float2(0.0f, neg_quantile_x1(um[t], uu[t], p2.y, q2.y));
      }
      SAB = __fadd2_rn(SAB, w2);
      if (e2lat) SL += w2.x * (logmA + T(2) * M::lg(s2.x));
      const float isB = __fdividef(1.0f, s2.y);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const float wv = w2.y * (z2[t].y * isB);
#pragma unroll
        for (int h = 0; h <= t; ++h) M2[t * (t + 1) / 2 + h] += wv * (z2[h].y * isB);
        M1[t] += wv;
      }
    } else {
    // pass A: density integral
      const T sA = tA[k];
      T wA = T(1);
      T zA[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        T acc = aA[t] * sA;
#pragma unroll
        for (int h = 0; h < t; ++h) acc -= Lc[t * (t + 1) / 2 + h] * zA[h];
        T pt, qt;
        M::upper_pq(acc * Li[t], pt, qt);
        wA *= pt;
        if (SHR || t + 1 < R) zA[t] = M::neg_quantile(um[t], uu[t], pt, qt);
      }
      SA += wA;
      if (e2lat) SL += wA * (logmA + T(2) * M::lg(sA));
      if constexpr (SHR && !DENS) {
        // pass B on pass A's point: weight w s^2, sums as shared_point_sums
        const T ws = wA * sA;
        SB += ws * sA;
#pragma unroll
        for (int t = 0; t < R; ++t) {
          M1[t] += ws * zA[t];
          const T u = wA * zA[t];
#pragma unroll
          for (int h = 0; h <= t; ++h) M2[t * (t + 1) / 2 + h] += u * zA[h];
        }
      } else if (!DENS) {
        // pass B: the e1 numerator and the truncated moments
        const T sB = tB[k];
        const T isB = T(1) / sB;
        T wB = T(1);
        T zB[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          T acc = aB[t] * sB;
#pragma unroll
          for (int h = 0; h < t; ++h) acc -= Lc[t * (t + 1) / 2 + h] * zB[h];
          T pt, qt;
          M::upper_pq(acc * Li[t], pt, qt);
          wB *= pt;
          zB[t] = M::neg_quantile(um[t], uu[t], pt, qt);
        }
        SB += wB;
#pragma unroll
        for (int t = 0; t < R; ++t) {
          const T wv = wB * (zB[t] * isB);
#pragma unroll
          for (int h = 0; h <= t; ++h) M2[t * (t + 1) / 2 + h] += wv * (zB[h] * isB);
          M1[t] += wv;
        }
      }
      }
  }
  }

  if constexpr (PAIRED) {
    SA = SAB.x;
    SB = SAB.y;
  }
  SA = warp_sum(SA);
  if (e2lat) SL = warp_sum(SL);
  if (!DENS) {
    SB = warp_sum(SB);
#pragma unroll
    for (int t = 0; t < R; ++t) M1[t] = warp_sum(M1[t]);
#pragma unroll
    for (int t = 0; t < RP; ++t) M2[t] = warp_sum(M2[t]);
  }
  if constexpr (SHR && !DENS) {
    // sum w s z = c sum w_B V and sum w z z^T = c^2 sum w_B V V^T, c = sqrt(m_A / m_B)
    const T ic = nrm ? T(1) : M::sq(mBT / mAT);
#pragma unroll
    for (int t = 0; t < R; ++t) M1[t] *= ic;
#pragma unroll
    for (int t = 0; t < RP; ++t) M2[t] *= ic * ic;
  }

  // double precision: a probability below the smallest normal double counts
  // as underflowed (log f = -inf, expectations 0); a single-precision sum that
  // small is queued for the log-domain rescue below
  constexpr bool dbl = sizeof(T) == 8;
  const T tiny_sum = dbl ? static_cast<T>(2.2250738585072014e-308 * (double)N) : T(0);
  const T logf = (dbl && !(SA >= tiny_sum)) ? static_cast<T>(-INFINITY)
                                             : static_cast<T>(pr.logt) + M::lg(SA) - M::lg(static_cast<T>(N));
  const int64_t n = fv.n;
  const int64_t ij = (int64_t)i * n + j;
  if (check) {
    const T thr = T(1e-20) * static_cast<T>(N);
    // pass B on pass A's points: pass B's sum no longer falls first for pairs
    // far in the tails, whose single-precision log f degrades with the size
    // of their conditional limits, so pass A's own threshold is raised to
    // 1e-15 N (the pairs the separate pass B sends to the rescue lie below it)
    const T thrA = SHR ? T(1e-15) * static_cast<T>(N) : thr;
    const bool densok = (SA >= thrA) && isfinite(logf);
    bool need = !densok;
    if (!DENS) need = need || !(SB >= thr);
    if (need) {
      // upper bound of log f for the triage: the float sum misses only point
      // weights that fell below the float range, so T <= max(S_A / N, 1e-37) up
      // to rounding; one nat of margin; +inf when the sum is not finite
      if constexpr (sizeof(OT) == 4) {
        if (a.triage && fv.out.logf != nullptr && lane == 0) {
          const double sa = (double)SA / (double)N;
          const double ub = isfinite(sa) ? pr.logt + log(fmax(sa, 1e-37)) + 1.0 : INFINITY;
          reinterpret_cast<float *>(fv.out.logf)[ij] = pending_bound_encode(ub);
        }
      }
      return true;
    }
  }
  if (fv.out.logf != nullptr && lane == 0) store<OT>(fv.out.logf, ij, logf);
  if (DENS) return false;

  const bool ok = dbl ? (SA >= tiny_sum && SB >= tiny_sum) : (SA > T(0) && SB > T(0));
  const T ratio = nrm ? T(1) : mAT / nud;
  const T e1 = ok ? ratio * (SB / SA) : T(0);
  const T sig = nrm ? T(1) : M::sq(nud / mBT);
  // the weighted means M / S_B (S_B at least the smallest normal times N here,
  // so 1 / S_B stays finite)
  const T iSB = ok ? T(1) / SB : T(0);
  const auto mean_of = [&](T m) -> T { return ok ? m * iSB : T(0); };
  T LEV[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    T s = T(0);
#pragma unroll
    for (int h = 0; h <= t; ++h) s += Lc[t * (t + 1) / 2 + h] * mean_of(M1[h]);
    LEV[t] = s;
  }
  T e2;
  if (nrm)
    e2 = T(0);
  else if (e2lat)
    e2 = ok ? SL / SA - M::lg(nud) : T(0);
  else
    e2 = ok ? e1 - (M::lg(T(0.5) * nud) + ratio - static_cast<T>(c.psiA)) : T(0);

  // lane-parallel stores: lane 0 wrote logf; lane 1 e1, lane 2 e2, lanes 3.. e3 then e4
  if (lane == 1) store<OT>(fv.out.e1, ij, e1);
  if (lane == 2) store<OT>(fv.out.e2, ij, e2);
#pragma unroll
  for (int t = 0; t < R; ++t) {
    if (lane == 3 + t) store<OT>(fv.out.e3, ((int64_t)i * R + ord[t]) * n + j, e1 * (q[t] + sig * LEV[t]));
  }
  // E[V V^T] in the L basis: (L EVV L^T)_th = sum_{a<=t} sum_{b<=h} L_ta EVV_ab L_hb
#pragma unroll
  for (int t = 0; t < R; ++t) {
#pragma unroll
    for (int h = 0; h <= t; ++h) {
      const int o = 3 + R + t * (t + 1) / 2 + h;
      if (lane == (o & 31)) {
        T s = T(0);
#pragma unroll
        for (int aa = 0; aa <= t; ++aa) {
#pragma unroll
          for (int bb = 0; bb <= h; ++bb) {
            const T evv = mean_of(aa >= bb ? M2[aa * (aa + 1) / 2 + bb] : M2[bb * (bb + 1) / 2 + aa]);
            s += Lc[t * (t + 1) / 2 + aa] * evv * Lc[h * (h + 1) / 2 + bb];
          }
        }
        const T exx = q[t] * q[h] + sig * (q[t] * LEV[h] + LEV[t] * q[h]) + sig * sig * s;
        // entry (t, h) of the prioritised order is (ord_t, ord_h) of the original
        const int x = ord[t] > ord[h] ? ord[t] : ord[h], y = ord[t] > ord[h] ? ord[h] : ord[t];
        store<OT>(fv.out.e4, ((int64_t)i * RP + x * (x + 1) / 2 + y) * n + j, e1 * exx);
      }
    }
  }
  return false;
}

// Minimum resident CTAs per SM the compiler must allow for the sweep kernel
// (caps its registers at 65536 / (256 * CFUST_ESTEP_MINB)).
#ifndef CFUST_ESTEP_MINB
#define CFUST_ESTEP_MINB 2
#endif

// Stages component i's chi tables (bulk async copy, bounded mbarrier wait),
// its constants and the paired single-precision factors into shared memory.
// Returns false, after flagging ERR_TIMEOUT, when the copy did not land.
template <typename T, bool DENS>
__device__ __forceinline__ bool stage_block(const EArgs &a, int i, unsigned char *smem, const T *&tA,
                                            const T *&tB, CompT<T> *&cs, PairedConsts *&pcs) {
  const int N = a.N;
  const size_t tab_bytes = a.staged ? (size_t)(DENS ? 1 : 2) * N * sizeof(T) : 0;
  T *tab = reinterpret_cast<T *>(smem);
  cs = reinterpret_cast<CompT<T> *>(smem + align16(tab_bytes));
  pcs = reinterpret_cast<PairedConsts *>(smem + align16(tab_bytes) + align16(sizeof(CompT<T>)));
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + align16(tab_bytes) + align16(sizeof(CompT<T>)) +
                                               align16(sizeof(PairedConsts)));
  const T *gtab = reinterpret_cast<const T *>(a.chi) + (int64_t)i * 2 * N;

  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  if (a.staged && threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, static_cast<uint32_t>(tab_bytes));
    bulk_copy_g2s(tab, gtab, static_cast<uint32_t>(tab_bytes), bar);
  }
  const uint32_t *src = reinterpret_cast<const uint32_t *>(reinterpret_cast<const CompT<T> *>(a.comp) + i);
  uint32_t *dst = reinterpret_cast<uint32_t *>(cs);
  for (int w = threadIdx.x; w < (int)(sizeof(CompT<T>) / 4); w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  if (threadIdx.x < RMAX * RMAX) {
    const int t = threadIdx.x / RMAX, h = threadIdx.x % RMAX;
    if (h <= t) {
      const float v = -(float)cs->L[t * RMAX + h] * (float)cs->Linv[t];
      pcs->nL[t * (t + 1) / 2 + h] = make_float2(v, v);
    }
  }
  __syncthreads();
  if (a.staged) {
    // the decision to give up is the block's, never a single thread's: a lane
    // that left alone would break the warp's full-mask shuffles in the sweep
    if (!mbar_wait_bounded(bar, 0, a.wait_polls)) atomicOr(&s_fail, 1);
    __syncthreads();
    if (s_fail) {
      // the copy may still be in flight: let it land (bounded) before the
      // block's shared memory is released, then report the timeout
      if (threadIdx.x == 0) {
        mbar_wait_bounded(bar, 0, 1 << 22);
        atomicOr(a.status, ERR_TIMEOUT);
      }
      __syncthreads();
      return false;
    }
  }
  tA = a.staged ? tab : gtab;
  tB = tA + N;
  return true;
}

// One coordinate of the log-domain sweep: log p for p = Phi(-lim) and the
// conditional draw z = -Phi^{-1}((1 - u) p).  While p is a normal float the
// direct single-precision forms are used; beyond, log p = log G(lim) - lim^2/2
// with the square in double and z from the log-domain quantile.
__device__ __forceinline__ float tail_factor_any(float a) {
  if (a <= 40.0f) return nf32::tail_factor(a);
  const float ia2 = 1.0f / (a * a);
  return 0.398942280f / a * fmaf(ia2, fmaf(3.0f, ia2, -1.0f), 1.0f);
}

__device__ __forceinline__ void rescue_dim(double lim, float um, float u, double &lp, float &z) {
  const float limf = (float)lim;
  const float lum = logf(um);
  if (limf < 12.0f) {
    float p, q;
    phi_upper_pq_f32(limf, p, q);
    lp = (double)logf(p);
    z = neg_quantile_f32(um, u, p, q);
  } else {
    lp = (double)logf(tail_factor_any(limf)) - 0.5 * lim * lim;
    z = neg_quantile_log_f32(lum + (float)lp);
  }
  if (z > 1.0f) {
    // one Newton step on log Phi(-z) = log(1 - u) + log p, the residual formed in
    // double from float logarithms: d/dz log Phi(-z) = -1 / (sqrt(2 pi) G(z))
    const float G = tail_factor_any(z);
    const double lpz = (double)logf(G) - 0.5 * (double)z * (double)z;
    const double h = lpz - ((double)lum + lp);
    z = fmaf((float)h * 2.50662827f, G, z);
  }
}

// Running log-sum-exp accumulator: value = exp(m) * s.
__device__ __forceinline__ void lse_add(double &m, float &s, double lw, float &scale_old, float &w_new) {
  if (lw > m) {
    scale_old = (m == -INFINITY) ? 0.f : expf((float)(m - lw));
    w_new = 1.0f;
    m = lw;
  } else {
    scale_old = 1.0f;
    w_new = expf((float)(lw - m));
  }
  s = fmaf(s, scale_old, w_new);
}

// Log-domain sweep of one queued pair by a whole CTA: the warps split the
// lattice points, each point weight is carried as log w = sum_t log Phi(-lim_t)
// (limits and log weights in double arithmetic, every transcendental in float)
// and accumulated against a running maximum, per lane, warp and CTA, so nothing
// underflows.  `sm` is shared scratch of at least 8 * (4 + 3 + R + R(R+1)/2) words.
template <int R, bool DENS, bool SHR = false>
__device__ void pair_sweep_log_cta(const EArgs &a, const FitView &fv, const CompT<double> &c,
                                   const Prologue<R> &pr,
                                   const double *__restrict__ tA, const double *__restrict__ tB, int i,
                                   int64_t j, double *sm) {
  constexpr int RP = R * (R + 1) / 2;
  constexpr int NV = 3 + R + RP;  // SA, SL, SB, M1, M2
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int N = a.N;
  const bool nrm = isinf(c.nu);  // the skew-normal limit: scale 1, e1 = 1, e2 = 0
  const double nud64 = c.nu + pr.d;
  const double fA = nrm ? 1.0 : sqrt(c.mA / nud64), fB = nrm ? 1.0 : sqrt(c.mB / nud64);
  const double cshr = nrm ? 1.0 : sqrt(c.mA / c.mB);  // c of pass B on pass A's points
  double aA[R], aB[R], Lc[RP], Li[R], qv[R];
  int ord[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    qv[t] = pr.q[t];
    ord[t] = t;
    Li[t] = c.Linv[t];
#pragma unroll
    for (int h = 0; h <= t; ++h) Lc[t * (t + 1) / 2 + h] = c.L[t * RMAX + h];
  }
  if (a.prio) {
    // the variable order and permuted factor of the single-precision sweep,
    // so the rescued pair is integrated by the same rule
    __shared__ PrioSlot rslot;
    __syncthreads();
    if (threadIdx.x == 0) prio_setup<R, double>(pr.q, c.lam, c.lamd, &rslot);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < R; ++t) {
      ord[t] = rslot.ord[t];
      qv[t] = rslot.q[t];
      Li[t] = rslot.Li[t];
#pragma unroll
      for (int h = 0; h <= t; ++h) Lc[t * (t + 1) / 2 + h] = rslot.L[t * (t + 1) / 2 + h];
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    aA[t] = -qv[t] * fA;
    aB[t] = -qv[t] * fB;
  }
  const int k0 = warp * WARP + lane, kstride = nw * WARP;
  float fm[R], fstep[R], two_sf[R], sf[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int m0 = (int)(((int64_t)k0 * a.z[t + 1] + a.sint[t + 1]) % N);
    fm[t] = (float)(2 * m0 - N);
    fstep[t] = (float)(2 * (int)(((int64_t)kstride * a.z[t + 1]) % N));
    two_sf[t] = (float)(2.0 * a.sfrac[t + 1]);
    sf[t] = (float)a.sfrac[t + 1];
  }
  const float fN = (float)N, invN = 1.0f / fN;
  const float umin = 1.1102230246251565e-16f, umax = 1.0f - 5.9604644775390625e-08f;
  const bool e2lat = (a.e2_mode == 1);

  double mA = -INFINITY, mB = -INFINITY;
  float v[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = 0.f;

  for (int k = k0; k < N; k += kstride) {
    float um[R], uu[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const float mm = 0.5f * (fm[t] + fN);
      const float lo = mm + sf[t], hi = (fN - mm) - sf[t];
      um[t] = fminf(fmaxf(fabsf(fm[t] + two_sf[t]) * invN, umin), umax);
      uu[t] = fmaxf(2.0f * fminf(lo, hi) * invN, umin);
      fm[t] += fstep[t];
      if (fm[t] >= fN) fm[t] -= 2.0f * fN;
    }
    const double sA = tA[k];
    double lw = 0.0;
    float z[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      double acc = aA[t] * sA;
#pragma unroll
      for (int h = 0; h < t; ++h) acc -= Lc[t * (t + 1) / 2 + h] * (double)z[h];
      double lp;
      rescue_dim(acc * Li[t], um[t], uu[t], lp, z[t]);
      lw += lp;
    }
    float so, wn;
    lse_add(mA, v[0], lw, so, wn);
    if (e2lat) v[1] = fmaf(v[1], so, wn * (float)(c.logmA + 2.0 * (double)logf((float)sA)));
    if (!DENS) {
      double lwb = 0.0;
      float isB;
      if constexpr (SHR) {
        // pass B on this point of pass A: weight s_A^2, V = z / (s_A c)
        lwb = lw + 2.0 * (double)logf((float)sA);
        isB = (float)(1.0 / (sA * cshr));
      } else {
        const double sB = tB[k];
        isB = (float)(1.0 / sB);
#pragma unroll
        for (int t = 0; t < R; ++t) {
          double acc = aB[t] * sB;
#pragma unroll
          for (int h = 0; h < t; ++h) acc -= Lc[t * (t + 1) / 2 + h] * (double)z[h];
          double lp;
          rescue_dim(acc * Li[t], um[t], uu[t], lp, z[t]);
          lwb += lp;
        }
      }
      lse_add(mB, v[2], lwb, so, wn);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const float vt = z[t] * isB;
        v[3 + t] = fmaf(v[3 + t], so, wn * vt);
#pragma unroll
        for (int h = 0; h <= t; ++h)
          v[3 + R + t * (t + 1) / 2 + h] = fmaf(v[3 + R + t * (t + 1) / 2 + h], so, wn * vt * (z[h] * isB));
      }
    }
  }
  // combine: per warp against the warp maximum, then across warps in shared memory
  double wmA = mA, wmB = mB;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wmA = fmax(wmA, __shfl_xor_sync(0xffffffffu, wmA, o));
    wmB = fmax(wmB, __shfl_xor_sync(0xffffffffu, wmB, o));
  }
  const float scA = (mA == -INFINITY) ? 0.f : expf((float)(mA - wmA));
  const float scB = (mB == -INFINITY) ? 0.f : expf((float)(mB - wmB));
  v[0] = warp_sum(v[0] * scA);
  v[1] = warp_sum(v[1] * scA);
#pragma unroll
  for (int t = 2; t < NV; ++t) v[t] = warp_sum(v[t] * scB);
  double *row = sm + warp * (2 + NV);
  if (lane == 0) {
    row[0] = wmA;
    row[1] = wmB;
#pragma unroll
    for (int t = 0; t < NV; ++t) row[2 + t] = (double)v[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gA = -INFINITY, gB = -INFINITY;
    for (int w = 0; w < nw; ++w) {
      gA = fmax(gA, sm[w * (2 + NV)]);
      gB = fmax(gB, sm[w * (2 + NV) + 1]);
    }
    double tot[NV];
    for (int t = 0; t < NV; ++t) tot[t] = 0.0;
    for (int w = 0; w < nw; ++w) {
      const double *rw = sm + w * (2 + NV);
      const double fa = (rw[0] == -INFINITY) ? 0.0 : exp(rw[0] - gA);
      const double fb = (rw[1] == -INFINITY) ? 0.0 : exp(rw[1] - gB);
      tot[0] += rw[2] * fa;
      tot[1] += rw[3] * fa;
      for (int t = 2; t < NV; ++t) tot[t] += rw[2 + t] * fb;
    }
    const int64_t n = fv.n;
    const int64_t ij = (int64_t)i * n + j;
    const double logTA = gA + log(tot[0]) - log((double)N);
    const double logf_out = pr.logt + logTA;
    if (!isfinite(logf_out)) atomicOr(a.status, ERR_NUMERIC);
    if (fv.out.logf != nullptr) store<float>(fv.out.logf, ij, logf_out);
    if (!DENS) {
      const double logTB = gB + log(tot[2]) - log((double)N);
      const bool ok = isfinite(logTA) && isfinite(logTB);
      const double e1 = ok ? (nrm ? 1.0 : c.mA / nud64) * exp(logTB - logTA) : 0.0;
      const double sig = nrm ? 1.0 : sqrt(nud64 / c.mB);
      const double iSB = ok ? 1.0 / tot[2] : 0.0;
      double LEV[R];
      for (int t = 0; t < R; ++t) {
        double sacc = 0.0;
        for (int h = 0; h <= t; ++h) sacc += Lc[t * (t + 1) / 2 + h] * (tot[3 + h] * iSB);
        LEV[t] = sacc;
      }
      double e2;
      if (nrm)
        e2 = 0.0;
      else if (e2lat)
        e2 = ok ? tot[1] / tot[0] - log(nud64) : 0.0;
      else
        e2 = ok ? e1 - (log(0.5 * nud64) + c.mA / nud64 - c.psiA) : 0.0;
      store<float>(fv.out.e1, ij, e1);
      store<float>(fv.out.e2, ij, e2);
      for (int t = 0; t < R; ++t) store<float>(fv.out.e3, ((int64_t)i * R + ord[t]) * n + j, e1 * (qv[t] + sig * LEV[t]));
      for (int t = 0; t < R; ++t)
        for (int h = 0; h <= t; ++h) {
          double sacc = 0.0;
          for (int aa = 0; aa <= t; ++aa)
            for (int bb = 0; bb <= h; ++bb) {
              const double evv = (aa >= bb ? tot[3 + R + aa * (aa + 1) / 2 + bb] : tot[3 + R + bb * (bb + 1) / 2 + aa]) * iSB;
              sacc += Lc[t * (t + 1) / 2 + aa] * evv * Lc[h * (h + 1) / 2 + bb];
            }
          const double exx = qv[t] * qv[h] + sig * (qv[t] * LEV[h] + LEV[t] * qv[h]) + sig * sig * sacc;
          const int x = ord[t] > ord[h] ? ord[t] : ord[h], y = ord[t] > ord[h] ? ord[h] : ord[t];
          store<float>(fv.out.e4, ((int64_t)i * RP + x * (x + 1) / 2 + y) * n + j, e1 * exx);
        }
    }
  }
  __syncthreads();
}

}  // namespace
}  // namespace cfust

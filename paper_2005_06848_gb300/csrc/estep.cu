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
#include "sweep.cuh"

namespace cfust {

namespace {

// One warp sweeps observations [jw0, jw0 + ppw) of component i of a fit: lane b
// computes the double prologue of the b-th observation, then the warp sweeps
// them one at a time.  `qi` is the component index recorded for queued pairs
// (the fit's own index, or the global one in a batch).
template <typename T, int R, bool DENS, bool PRIO = false, bool SHR = false>
__device__ __forceinline__ void sweep_warp_pairs(const EArgs &a, const FitView &fv, const CompT<T> &c,
                                                 const PairedConsts *pcs, const T *tA, const T *tB,
                                                 int i, int qi, int64_t jw0, int ppw, PairedConsts *wpc) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  if (jw0 < fv.n) cnt = (int)((fv.n - jw0) < ppw ? (fv.n - jw0) : ppw);
  Prologue<R> mine;
  if (lane < cnt) mine = prologue<T, R>(a, fv, c, jw0 + lane);
  PrioLane<R, T> pmine;
  if constexpr (PRIO) {
    if (lane < cnt) prio_lane<R, T>(mine.q, c.lam, c.lamd, &pmine);
  }
  const bool check = (sizeof(T) == 4);
  for (int b = 0; b < cnt; ++b) {
    const Prologue<R> pr = shfl_prologue<R>(mine, b);
    PrioLane<R, T> pp;
    if constexpr (PRIO) pp = shfl_prio<R, T>(pmine, b);
    const int64_t j = jw0 + b;
    const bool need = pair_sweep<T, T, R, DENS, PRIO, 2, SHR>(a, fv, c, pr, tA, tB, i, j, lane, check, pcs, wpc,
                                                              &pp);
    if (need && lane == 0) {
      const unsigned slot = atomicAdd(a.rescue_count, 1u);
      a.rescue_list[slot] = pair_id(qi, j);
    }
  }
}

template <typename T, int R, bool DENS, bool PRIO, bool SHR = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? CFUST_ESTEP_MINB : 1) estep_kernel(EArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int i = blockIdx.y;
  const T *tA, *tB;
  CompT<T> *cs;
  PairedConsts *pcs;
  if (!stage_block<T, DENS>(a, i, smem, tA, tB, cs, pcs)) return;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t jw0 = ((int64_t)blockIdx.x * nw + warp) * a.ppw;
  // with prioritisation, one order-and-factor slot per warp after the staged constants
  PairedConsts *wpc = nullptr;
  if constexpr (PRIO) {
    const size_t tab_bytes = a.staged ? (size_t)(DENS ? 1 : 2) * a.N * sizeof(T) : 0;
    wpc = reinterpret_cast<PairedConsts *>(smem + align16(tab_bytes) + align16(sizeof(CompT<T>)) +
                                           align16(sizeof(PairedConsts)) + 16) + warp;
  }
  sweep_warp_pairs<T, R, DENS, PRIO, SHR>(a, fit_view(a), *cs, pcs, tA, tB, i, i, jw0, a.ppw, wpc);
}

// Triage of a listed pair (single precision outputs): with log f of every
// component of observation j in place (values, or upper bounds for pairs still
// to be swept, +inf where none is known), a pair whose log pi_i + log f_ij
// trails the best component by more than tnats has tau_ij < exp(-tnats); it gets
// log f = -inf and zero expectations instead of a sweep.  Unknown entries do
// not count towards the best (that only makes the test more cautious).
template <int R, bool DENS>
__device__ bool triage_listed(const FitView &fv, int i, int64_t j, float tnats) {
  const float *lf = reinterpret_cast<const float *>(fv.out.logf);
  float best = -INFINITY;
  for (int h = 0; h < fv.g; ++h) {
    const float v = lf[(int64_t)h * fv.n + j];
    if (v < INFINITY) best = fmaxf(best, logf((float)fv.pi[h]) + v);
  }
  const float mine = logf((float)fv.pi[i]) + lf[(int64_t)i * fv.n + j];
  if (!(isfinite(best) && mine < best - tnats)) return false;
  const int64_t ij = (int64_t)i * fv.n + j;
  constexpr int RP = R * (R + 1) / 2;
  store<float>(fv.out.logf, ij, -INFINITY);
  if (!DENS) {
    store<float>(fv.out.e1, ij, 0.0);
    store<float>(fv.out.e2, ij, 0.0);
    for (int t = 0; t < R; ++t) store<float>(fv.out.e3, ((int64_t)i * R + t) * fv.n + j, 0.0);
    for (int t = 0; t < RP; ++t) store<float>(fv.out.e4, ((int64_t)i * RP + t) * fv.n + j, 0.0);
  }
  return true;
}

// The same sweep over an explicit list of observations per component:
// list[i * stride + k] for k < count[i] (the pairs a surrogate E-step leaves
// to the lattice rule).  Warps stride over the list in chunks of ppw.
template <typename T, int R, bool DENS, bool PRIO = false, bool SHR = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? CFUST_ESTEP_MINB : 1)
    estep_list_kernel(EArgs a, const int *list, const unsigned *count, int64_t stride) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int i = blockIdx.y;
  const int64_t cnt = count[i];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((int64_t)blockIdx.x * nw * a.ppw >= cnt) return;  // uniform over the block
  const T *tA, *tB;
  CompT<T> *cs;
  PairedConsts *pcs;
  if (!stage_block<T, DENS>(a, i, smem, tA, tB, cs, pcs)) return;
  const FitView fv = fit_view(a);
  const int *li = list + (int64_t)i * stride;
  const int lane = threadIdx.x & 31;
  const bool check = (sizeof(T) == 4);
  // with prioritisation, one order-and-factor slot per warp after the staged constants
  PairedConsts *wpc = nullptr;
  if constexpr (PRIO) {
    const size_t tab_bytes = a.staged ? (size_t)(DENS ? 1 : 2) * a.N * sizeof(T) : 0;
    wpc = reinterpret_cast<PairedConsts *>(smem + align16(tab_bytes) + align16(sizeof(CompT<T>)) +
                                           align16(sizeof(PairedConsts)) + 16) + warp;
  }
  for (int64_t base = ((int64_t)blockIdx.x * nw + warp) * a.ppw; base < cnt;
       base += (int64_t)gridDim.x * nw * a.ppw) {
    const int m = (int)((cnt - base) < a.ppw ? (cnt - base) : a.ppw);
    Prologue<R> mine;
    int64_t myj = 0;
    bool myskip = false;
    PrioLane<R, T> pmine;
    if (lane < m) {
      myj = li[base + lane];
      if (a.triage) myskip = triage_listed<R, DENS>(fv, i, myj, a.tnats);
      if (!myskip) {
        mine = prologue<T, R>(a, fv, *cs, myj);
        if constexpr (PRIO) prio_lane<R, T>(mine.q, cs->lam, cs->lamd, &pmine);
      }
    }
    const unsigned skipped = __ballot_sync(0xffffffffu, myskip);
    for (int b = 0; b < m; ++b) {
      if ((skipped >> b) & 1u) continue;
      const Prologue<R> pr = shfl_prologue<R>(mine, b);
      PrioLane<R, T> pp;
      if constexpr (PRIO) pp = shfl_prio<R, T>(pmine, b);
      const int64_t j = __shfl_sync(0xffffffffu, myj, b);
      const bool need = pair_sweep<T, T, R, DENS, PRIO, 2, SHR>(a, fv, *cs, pr, tA, tB, i, j, lane, check, pcs, wpc,
                                                                &pp);
      if (need && lane == 0) {
        const unsigned slot = atomicAdd(a.rescue_count, 1u);
        a.rescue_list[slot] = pair_id(i, j);
      }
    }
  }
}

// The triage of a queued pair (single precision): with the log f of every
// component of observation j in place, final values or pending bounds, a pair
// whose bound log pi_i + ub_ij trails the best final value by tnats has
// tau_ij < exp(-tnats) and is dropped instead of recomputed.  Pending bounds
// of the observation's other pairs do not count towards the best (they are
// upper bounds), and the decisions are all taken before any rescue writes.
__device__ __forceinline__ bool triage_drops(const FitView &fv, int i, int64_t j, float tnats) {
  const float *lf = reinterpret_cast<const float *>(fv.out.logf);
  double best = -INFINITY;
  for (int h = 0; h < fv.g; ++h) best = fmax(best, log(fv.pi[h]) + (double)lf[(int64_t)h * fv.n + j]);
  const double mine = log(fv.pi[i]) + pending_bound_decode(lf[(int64_t)i * fv.n + j]);
  return isfinite(best) && mine < best - (double)tnats;
}

constexpr unsigned long long RESCUE_DROP = 1ull << 63;  // marks a queued pair the triage dropped

__global__ void rescue_triage_kernel(EArgs a) {
  const unsigned cnt = *a.rescue_count;
  const FitView fv = fit_view(a);
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x) {
    const unsigned long long id = a.rescue_list[w];
    if (triage_drops(fv, static_cast<int>(id >> 32), static_cast<int64_t>(id & 0xffffffffull), a.tnats))
      a.rescue_list[w] = id | RESCUE_DROP;
  }
}

// Log-domain recomputation of one queued pair by the whole CTA, or, when the
// triage dropped it, log f = -inf and zero expectations.
template <int R, bool DENS, bool SHR = false>
__device__ void rescue_one(const EArgs &a, const FitView &fv, const CompT<double> &comp, const double *tab,
                           int i, int64_t j, bool dropped, double *sm, Prologue<R> &spr) {
  if (dropped) {
    if (threadIdx.x == 0) {
      const int64_t ij = (int64_t)i * fv.n + j;
      const int RP = R * (R + 1) / 2;
      store<float>(fv.out.logf, ij, -INFINITY);
      if (!DENS) {
        store<float>(fv.out.e1, ij, 0.0);
        store<float>(fv.out.e2, ij, 0.0);
        for (int t = 0; t < R; ++t) store<float>(fv.out.e3, ((int64_t)i * R + t) * fv.n + j, 0.0);
        for (int t = 0; t < RP; ++t) store<float>(fv.out.e4, ((int64_t)i * RP + t) * fv.n + j, 0.0);
      }
    }
    return;  // uniform over the block
  }
  if (threadIdx.x == 0) spr = prologue<double, R>(a, fv, comp, j);
  __syncthreads();
  const Prologue<R> pr = spr;
  pair_sweep_log_cta<R, DENS, SHR>(a, fv, comp, pr, tab, tab + a.N, i, j, sm);
}

template <int R, bool DENS, bool SHR = false>
__global__ void __launch_bounds__(256) rescue_kernel(EArgs a, const CompT<double> *comp,
                                                      const double *chi) {
  constexpr int NV = 3 + R + R * (R + 1) / 2;
  __shared__ double sm[8 * (2 + NV)];
  __shared__ Prologue<R> spr;
  const unsigned cnt = *a.rescue_count;
  const FitView fv = fit_view(a);
  for (unsigned w = blockIdx.x; w < cnt; w += gridDim.x) {
    const unsigned long long id = a.rescue_list[w];
    const int i = static_cast<int>((id & ~RESCUE_DROP) >> 32);
    const int64_t j = static_cast<int64_t>(id & 0xffffffffull);
    rescue_one<R, DENS, SHR>(a, fv, comp[i], chi + (int64_t)i * 2 * a.N, i, j, (id & RESCUE_DROP) != 0, sm,
                             spr);
  }
}

template <typename T, int R, bool DENS>
cudaError_t launch_r(EArgs a, int g, int64_t n, cudaStream_t st, bool fp32,
                     const CompT<double> *c64, const double *chi64, SweepTiming tm) {
  const size_t tab_bytes = (size_t)(DENS ? 1 : 2) * a.N * sizeof(T);
  a.staged = tab_bytes <= 160u * 1024u ? 1 : 0;
  const size_t smem = (a.staged ? align16(tab_bytes) : 0) + align16(sizeof(CompT<T>)) +
                      align16(sizeof(PairedConsts)) + 16 + (a.prio ? 8 * sizeof(PairedConsts) : 0);
  // the prioritised sweep is its own instantiation (r >= 2), so the default
  // one carries none of its registers
  const bool prio = a.prio && R >= 2;
  // pass B on pass A's points: its own instantiations (full sweeps)
  const bool shr = a.shr && !DENS;
  const void *kern = prio ? (shr ? (const void *)estep_kernel<T, R, DENS, (R >= 2), !DENS>
                                 : (const void *)estep_kernel<T, R, DENS, (R >= 2)>)
                          : (shr ? (const void *)estep_kernel<T, R, DENS, false, !DENS>
                                 : (const void *)estep_kernel<T, R, DENS, false>);
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  const int64_t per_cta = (int64_t)a.ppw * 8;
  const int64_t bx = (n + per_cta - 1) / per_cta;
  if (bx > 0x7fffffff) return cudaErrorInvalidValue;
  dim3 grid((unsigned)bx, g);
  if (fp32) {
    e = cudaMemsetAsync(a.rescue_count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  const unsigned evflag = tm.capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (tm.start) {
    e = cudaEventRecordWithFlags(tm.start, st, evflag);
    if (e != cudaSuccess) return e;
  }
  if (prio && shr)
    estep_kernel<T, R, DENS, (R >= 2), !DENS><<<grid, 256, smem, st>>>(a);
  else if (prio)
    estep_kernel<T, R, DENS, (R >= 2)><<<grid, 256, smem, st>>>(a);
  else if (shr)
    estep_kernel<T, R, DENS, false, !DENS><<<grid, 256, smem, st>>>(a);
  else
    estep_kernel<T, R, DENS, false><<<grid, 256, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (tm.stop) {
    e = cudaEventRecordWithFlags(tm.stop, st, evflag);
    if (e != cudaSuccess) return e;
  }
  if (!fp32) return e;
  if (a.triage) {
    rescue_triage_kernel<<<sm_count() * 2, 256, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (shr)
    rescue_kernel<R, DENS, !DENS><<<sm_count() * 4, 256, 0, st>>>(a, c64, chi64);
  else
    rescue_kernel<R, DENS><<<sm_count() * 4, 256, 0, st>>>(a, c64, chi64);
  return cudaGetLastError();
}

template <typename T, bool DENS>
cudaError_t dispatch_r(int r, EArgs a, int g, int64_t n, cudaStream_t st, bool fp32,
                       const CompT<double> *c64, const double *chi64, SweepTiming tm) {
  switch (r) {
    case 1: return launch_r<T, 1, DENS>(a, g, n, st, fp32, c64, chi64, tm);
    case 2: return launch_r<T, 2, DENS>(a, g, n, st, fp32, c64, chi64, tm);
    case 3: return launch_r<T, 3, DENS>(a, g, n, st, fp32, c64, chi64, tm);
    case 4: return launch_r<T, 4, DENS>(a, g, n, st, fp32, c64, chi64, tm);
    case 5: return launch_r<T, 5, DENS>(a, g, n, st, fp32, c64, chi64, tm);
    case 6: return launch_r<T, 6, DENS>(a, g, n, st, fp32, c64, chi64, tm);
    default: return cudaErrorInvalidValue;
  }
}


// ---------------------------------------------------------------------------
// Batched fits
// ---------------------------------------------------------------------------

template <typename OT>
__device__ __forceinline__ FitView batch_view(const BatchDev &b, const FitDesc &fd, int p, int r) {
  FitView f;
  f.Y = fd.Y;
  f.n = fd.n;
  f.g = fd.g;
  const int rp = r * (r + 1) / 2;
  f.out.logf = reinterpret_cast<OT *>(b.logf) + fd.pair_off;
  f.out.e1 = reinterpret_cast<OT *>(b.e1) + fd.pair_off;
  f.out.e2 = reinterpret_cast<OT *>(b.e2) + fd.pair_off;
  f.out.e3 = reinterpret_cast<OT *>(b.e3) + fd.pair_off * r;
  f.out.e4 = reinterpret_cast<OT *>(b.e4) + fd.pair_off * rp;
  f.pi = param_view(b.params + fd.param_off, fd.g, p, r).pi;
  return f;
}

// Persistent sweep over many fits: each CTA pulls (component, observation
// tile) items from an atomic counter until none are left; the component's
// chi tables are restaged by one bulk copy (bounded mbarrier wait) and its
// constants copied only when the component changes from the CTA's previous
// item.  Items are ordered component by component, so a CTA mostly stays on
// one component.  A lost copy ends the whole CTA with ERR_TIMEOUT.
template <typename T, int R, bool DENS, bool PRIO = false, bool SHR = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? CFUST_ESTEP_MINB : 1)
    estep_batched_kernel(EArgs a, BatchDev b, const SweepItem *items, int nitems, unsigned *counter) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  __shared__ int s_fail;
  const int N = a.N;
  const size_t tab_bytes = a.staged ? (size_t)(DENS ? 1 : 2) * N * sizeof(T) : 0;
  T *tab = reinterpret_cast<T *>(smem);
  CompT<T> *cs = reinterpret_cast<CompT<T> *>(smem + align16(tab_bytes));
  PairedConsts *pcs = reinterpret_cast<PairedConsts *>(smem + align16(tab_bytes) + align16(sizeof(CompT<T>)));
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + align16(tab_bytes) + align16(sizeof(CompT<T>)) +
                                               align16(sizeof(PairedConsts)));
  const T *gtab_base = reinterpret_cast<const T *>(a.chi);
  const CompT<T> *gcomp = reinterpret_cast<const CompT<T> *>(a.comp);
  if (threadIdx.x == 0) {
    if (a.staged) mbar_init(bar, 1);
    s_fail = 0;
  }
  __syncthreads();
  int cur = -1;
  uint32_t phase = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const SweepItem item = items[it];
    if (item.gc != cur) {
      // every warp finished the previous item at the barrier above
      if (a.staged && threadIdx.x == 0) {
        mbar_expect_tx(bar, static_cast<uint32_t>(tab_bytes));
        bulk_copy_g2s(tab, gtab_base + (int64_t)item.gc * 2 * N, static_cast<uint32_t>(tab_bytes), bar);
      }
      const uint32_t *src = reinterpret_cast<const uint32_t *>(gcomp + item.gc);
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
      if (a.staged && !mbar_wait_bounded(bar, phase, a.wait_polls)) atomicOr(&s_fail, 1);
      __syncthreads();
      if (s_fail) {
        // let the copy in flight land (bounded) before the block exits
        if (threadIdx.x == 0) {
          mbar_wait_bounded(bar, phase, 1 << 22);
          atomicOr(a.status, ERR_TIMEOUT);
        }
        __syncthreads();
        return;
      }
      phase ^= 1u;
      cur = item.gc;
    }
    const T *tA = a.staged ? tab : gtab_base + (int64_t)cur * 2 * N;
    const T *tB = tA + N;
    const CompRef cr = b.comps[item.gc];
    const FitDesc fd = b.fits[cr.fit];
    const FitView fv = batch_view<T>(b, fd, a.p, R);
    const int warp = threadIdx.x >> 5;
    const int64_t jw0 = (int64_t)item.j0 + (int64_t)warp * a.ppw;
    // with prioritisation, one order-and-factor slot per warp after the mbarrier
    PairedConsts *wpc = nullptr;
    if constexpr (PRIO)
      wpc = reinterpret_cast<PairedConsts *>(reinterpret_cast<unsigned char *>(bar) + 16) + warp;
    sweep_warp_pairs<T, R, DENS, PRIO, SHR>(a, fv, *cs, pcs, tA, tB, cr.i, item.gc, jw0, a.ppw, wpc);
    __syncthreads();
  }
}

// The triage of the batch's queued pairs (see rescue_triage_kernel).
__global__ void rescue_triage_batched_kernel(EArgs a, BatchDev b, int r) {
  const unsigned cnt = *a.rescue_count;
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x) {
    const unsigned long long id = a.rescue_list[w];
    const int gc = static_cast<int>(id >> 32);
    const CompRef cr = b.comps[gc];
    const FitDesc fd = b.fits[cr.fit];
    const FitView fv = batch_view<float>(b, fd, a.p, r);
    if (triage_drops(fv, cr.i, static_cast<int64_t>(id & 0xffffffffull), a.tnats))
      a.rescue_list[w] = id | RESCUE_DROP;
  }
}

template <int R, bool DENS, bool SHR = false>
__global__ void __launch_bounds__(256) rescue_batched_kernel(EArgs a, BatchDev b, const CompT<double> *comp,
                                                              const double *chi) {
  constexpr int NV = 3 + R + R * (R + 1) / 2;
  __shared__ double sm[8 * (2 + NV)];
  __shared__ Prologue<R> spr;
  const unsigned cnt = *a.rescue_count;
  for (unsigned w = blockIdx.x; w < cnt; w += gridDim.x) {
    const unsigned long long id = a.rescue_list[w];
    const int gc = static_cast<int>((id & ~RESCUE_DROP) >> 32);
    const int64_t j = static_cast<int64_t>(id & 0xffffffffull);
    const CompRef cr = b.comps[gc];
    const FitDesc fd = b.fits[cr.fit];
    const FitView fv = batch_view<float>(b, fd, a.p, R);
    rescue_one<R, DENS, SHR>(a, fv, comp[gc], chi + (int64_t)gc * 2 * a.N, cr.i, j, (id & RESCUE_DROP) != 0, sm,
                             spr);
  }
}

template <typename T, int R, bool DENS>
cudaError_t launch_batched_r(EArgs a, const BatchDev &b, const SweepItem *items, int nitems, unsigned *counter,
                             int ctas_per_sm, cudaStream_t st, bool fp32, const CompT<double> *c64,
                             const double *chi64, SweepTiming tm) {
  const size_t tab_bytes = (size_t)(DENS ? 1 : 2) * a.N * sizeof(T);
  a.staged = tab_bytes <= 160u * 1024u ? 1 : 0;
  const bool prio = a.prio && R >= 2;
  const size_t smem = (a.staged ? align16(tab_bytes) : 0) + align16(sizeof(CompT<T>)) +
                      align16(sizeof(PairedConsts)) + 16 + (prio ? 8 * sizeof(PairedConsts) : 0);
  const bool shr = a.shr && !DENS;
  const void *kern = prio ? (shr ? (const void *)estep_batched_kernel<T, R, DENS, (R >= 2), !DENS>
                                 : (const void *)estep_batched_kernel<T, R, DENS, (R >= 2)>)
                          : (shr ? (const void *)estep_batched_kernel<T, R, DENS, false, !DENS>
                                 : (const void *)estep_batched_kernel<T, R, DENS, false>);
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
  if (fp32 && (e = cudaMemsetAsync(a.rescue_count, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
  const unsigned evflag = tm.capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (tm.start && (e = cudaEventRecordWithFlags(tm.start, st, evflag)) != cudaSuccess) return e;
  const unsigned grid = (unsigned)(sm_count() * (ctas_per_sm > 0 ? ctas_per_sm : 2));
  if (prio && shr)
    estep_batched_kernel<T, R, DENS, (R >= 2), !DENS><<<grid, 256, smem, st>>>(a, b, items, nitems, counter);
  else if (prio)
    estep_batched_kernel<T, R, DENS, (R >= 2)><<<grid, 256, smem, st>>>(a, b, items, nitems, counter);
  else if (shr)
    estep_batched_kernel<T, R, DENS, false, !DENS><<<grid, 256, smem, st>>>(a, b, items, nitems, counter);
  else
    estep_batched_kernel<T, R, DENS, false><<<grid, 256, smem, st>>>(a, b, items, nitems, counter);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (tm.stop && (e = cudaEventRecordWithFlags(tm.stop, st, evflag)) != cudaSuccess) return e;
  if (!fp32) return cudaSuccess;
  if (a.triage) {
    rescue_triage_batched_kernel<<<sm_count() * 2, 256, 0, st>>>(a, b, R);
    const cudaError_t et = cudaGetLastError();
    if (et != cudaSuccess) return et;
  }
  if (shr)
    rescue_batched_kernel<R, DENS, !DENS><<<sm_count() * 4, 256, 0, st>>>(a, b, c64, chi64);
  else
    rescue_batched_kernel<R, DENS><<<sm_count() * 4, 256, 0, st>>>(a, b, c64, chi64);
  return cudaGetLastError();
}

template <typename T, bool DENS>
cudaError_t dispatch_batched(int r, EArgs a, const BatchDev &b, const SweepItem *items, int nitems,
                             unsigned *counter, int cps, cudaStream_t st, bool fp32, const CompT<double> *c64,
                             const double *chi64, SweepTiming tm) {
  switch (r) {
    case 1: return launch_batched_r<T, 1, DENS>(a, b, items, nitems, counter, cps, st, fp32, c64, chi64, tm);
    case 2: return launch_batched_r<T, 2, DENS>(a, b, items, nitems, counter, cps, st, fp32, c64, chi64, tm);
    case 3: return launch_batched_r<T, 3, DENS>(a, b, items, nitems, counter, cps, st, fp32, c64, chi64, tm);
    case 4: return launch_batched_r<T, 4, DENS>(a, b, items, nitems, counter, cps, st, fp32, c64, chi64, tm);
    case 5: return launch_batched_r<T, 5, DENS>(a, b, items, nitems, counter, cps, st, fp32, c64, chi64, tm);
    case 6: return launch_batched_r<T, 6, DENS>(a, b, items, nitems, counter, cps, st, fp32, c64, chi64, tm);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void normal_f32_kernel(const float *x, float *out, int64_t n, int which) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[k];
    float r;
    switch (which) {
      case 0: r = phi_upper_f32(v); break;
      case 1: r = phi_inv_f32(v); break;
      case 2: r = normcdff(-v); break;
      case 3: r = normcdfinvf(v); break;
      case 4: r = log_phi_upper_f32(v); break;
      default: r = neg_quantile_log_f32(v); break;
    }
    out[k] = r;
  }
}

}  // namespace

cudaError_t launch_normal_f32(const float *x, float *out, int64_t n, int which, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  const int64_t bcap = (int64_t)sm_count() * 16;
  normal_f32_kernel<<<(unsigned)(blocks < bcap ? blocks : bcap), 256, 0, st>>>(x, out, n, which);
  return cudaGetLastError();
}

cudaError_t launch_estep_batched(int precision, const BatchDev &b, int p, int r, const LatticeDev &lat,
                                 const CompT<double> *c64, const CompT<float> *c32, const double *chi64,
                                 const float *chi32, const SweepItem *items, int nitems,
                                 unsigned *item_counter, bool density_only, int e2_mode, int ppw,
                                 int ctas_per_sm, unsigned long long *rescue_list, unsigned *rescue_count,
                                 int *d_status, int triage, cudaStream_t st, SweepTiming tm, int prio,
                                 int shared) {
  if (nitems <= 0) return cudaSuccess;
  EArgs a{};
  a.Y = nullptr;
  a.n = 0;
  a.g = 0;
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
  a.ppw = ppw < 1 ? 1 : (ppw > 32 ? 32 : ppw);
  a.rescue_list = rescue_list;
  a.rescue_count = rescue_count;
  a.status = d_status;
  a.triage = triage ? 1 : 0;
  a.tnats = 30.f;
  a.prio = prio ? 1 : 0;
  a.shr = shared ? 1 : 0;
  a.wait_polls = lat.wait_polls;
  if (precision == CFUST_FP64) {
    a.comp = c64;
    a.chi = chi64;
    return density_only
               ? dispatch_batched<double, true>(r, a, b, items, nitems, item_counter, ctas_per_sm, st, false, c64, chi64, tm)
               : dispatch_batched<double, false>(r, a, b, items, nitems, item_counter, ctas_per_sm, st, false, c64, chi64, tm);
  }
  a.comp = c32;
  a.chi = chi32;
  return density_only
             ? dispatch_batched<float, true>(r, a, b, items, nitems, item_counter, ctas_per_sm, st, true, c64, chi64, tm)
             : dispatch_batched<float, false>(r, a, b, items, nitems, item_counter, ctas_per_sm, st, true, c64, chi64, tm);
}

// One thread per slot k of the padded lattice (ceil(n / 64) * 64 slots): the
// row of point k (k < n) and its place in the pair-interleaved table, where a
// second point past n repeats the first of its pair.
__global__ void uniform_table_kernel(LatticeDev lat, int r, int us, float *tab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = lat.n;
  const int npad = (N + 63) / 64 * 64;
  if (k >= npad) return;
  const int src = k < N ? k : (k - 32 < N ? k - 32 : N - 1);
  const float fN = (float)N, invN = 1.0f / fN;
  const float umin = 1.1102230246251565e-16f, umax = 1.0f - 5.9604644775390625e-08f;
  float *row = tab + (int64_t)k * us;
  float *pair = tab + (int64_t)N * us + ((int64_t)(k >> 6) * 32 + (k & 31)) * 2 * us + ((k >> 5) & 1);
  for (int t = 0; t < r; ++t) {
    const int m = (int)(((int64_t)src * lat.z[t + 1] + lat.sint[t + 1]) % N);
    const float fm = (float)(2 * m - N);
    const float sf = (float)lat.sfrac[t + 1], two_sf = (float)(2.0 * lat.sfrac[t + 1]);
    const float mm = 0.5f * (fm + fN);
    const float lo = mm + sf, hi = (fN - mm) - sf;
    const float um = fminf(fmaxf(fabsf(fm + two_sf) * invN, umin), umax);
    const float uu = fmaxf(2.0f * fminf(lo, hi) * invN, umin);
    if (k < N) {
      row[t] = um;
      row[r + t] = uu;
    }
    pair[2 * t] = um;
    pair[2 * (r + t)] = uu;
  }
  for (int t = 2 * r; t < us; ++t) {
    if (k < N) row[t] = 0.0f;
    pair[2 * t] = 0.0f;
  }
}

template <bool DENS>
cudaError_t launch_list_r3(EArgs a, int g, int64_t n, const int *list, const unsigned *count,
                           const CompT<double> *c64, const double *chi64, cudaStream_t st) {
  const size_t tab_bytes = (size_t)(DENS ? 1 : 2) * a.N * sizeof(float);
  a.staged = tab_bytes <= 160u * 1024u ? 1 : 0;
  const size_t smem = (a.staged ? align16(tab_bytes) : 0) + align16(sizeof(CompT<float>)) +
                      align16(sizeof(PairedConsts)) + 16 + (a.prio ? 8 * sizeof(PairedConsts) : 0);
  const bool shr = a.shr && !DENS;
  const void *kern = a.prio ? (shr ? (const void *)estep_list_kernel<float, 3, DENS, true, !DENS>
                                   : (const void *)estep_list_kernel<float, 3, DENS, true>)
                            : (shr ? (const void *)estep_list_kernel<float, 3, DENS, false, !DENS>
                                   : (const void *)estep_list_kernel<float, 3, DENS, false>);
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  // 16 listed pairs per warp chunk: their FP64 prologues and triage tests run
  // lane-parallel, which matters at the small lattices this path serves
  a.ppw = 16;
  // the list lengths live on the device: size every component's column of
  // the grid for a full list, capped near four waves of two CTAs per SM;
  // blocks past the end of their list return at once.  The lists are often
  // lopsided (one component's far tail can hold most listed pairs), so each
  // column gets the whole cap rather than a 1/g share of it
  const int64_t need = (n + 8 * a.ppw - 1) / (8 * a.ppw);
  const int64_t cap = (int64_t)sm_count() * 2 * 4;
  const int64_t bx = need < cap ? need : cap;
  e = cudaMemsetAsync(a.rescue_count, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)(bx < 1 ? 1 : bx), g);
  if (a.prio && shr)
    estep_list_kernel<float, 3, DENS, true, !DENS><<<grid, 256, smem, st>>>(a, list, count, n);
  else if (a.prio)
    estep_list_kernel<float, 3, DENS, true><<<grid, 256, smem, st>>>(a, list, count, n);
  else if (shr)
    estep_list_kernel<float, 3, DENS, false, !DENS><<<grid, 256, smem, st>>>(a, list, count, n);
  else
    estep_list_kernel<float, 3, DENS, false><<<grid, 256, smem, st>>>(a, list, count, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.triage) {
    rescue_triage_kernel<<<sm_count() * 2, 256, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (shr)
    rescue_kernel<3, DENS, !DENS><<<sm_count() * 4, 256, 0, st>>>(a, c64, chi64);
  else
    rescue_kernel<3, DENS><<<sm_count() * 4, 256, 0, st>>>(a, c64, chi64);
  return cudaGetLastError();
}

EArgs make_args(const double *Y, int64_t n, int g, int p, const LatticeDev &lat, EstepOut out, int e2_mode,
                unsigned long long *rescue_list, unsigned *rescue_count, int *d_status, int triage,
                const double *d_pi, float tnats, int prio = 0, int shared = 0) {
  EArgs a;
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
  a.out = out;
  a.utab = lat.utab;
  a.utab2 = lat.utab2;
  a.e2_mode = e2_mode;
  a.ppw = 1;
  a.staged = 1;
  a.rescue_list = rescue_list;
  a.rescue_count = rescue_count;
  a.status = d_status;
  a.triage = (triage && out.logf != nullptr) ? 1 : 0;
  a.tnats = tnats;
  a.prio = prio ? 1 : 0;
  a.shr = shared ? 1 : 0;
  a.wait_polls = lat.wait_polls;
  a.pi = d_pi;
  a.comp = nullptr;
  a.chi = nullptr;
  return a;
}

cudaError_t launch_estep_list(const double *Y, int64_t n, int g, int p, int r, const LatticeDev &lat,
                              const CompT<double> *c64, const CompT<float> *c32, const double *chi64,
                              const float *chi32, EstepOut out, bool density_only, int e2_mode,
                              const int *list, const unsigned *count, unsigned long long *rescue_list,
                              unsigned *rescue_count, int *d_status, cudaStream_t st, int triage,
                              const double *d_pi, float tnats, int prio, int shared) {
  if (n <= 0) return cudaSuccess;
  if (r != 3) return cudaErrorInvalidValue;
  EArgs a = make_args(Y, n, g, p, lat, out, e2_mode, rescue_list, rescue_count, d_status, triage, d_pi, tnats,
                      prio, shared);
  a.comp = c32;
  a.chi = chi32;
  return density_only ? launch_list_r3<true>(a, g, n, list, count, c64, chi64, st)
                      : launch_list_r3<false>(a, g, n, list, count, c64, chi64, st);
}

cudaError_t launch_uniform_table(const LatticeDev &lat, int r, float *tab, cudaStream_t st) {
  if (lat.n <= 0 || r < 1 || r > RMAX) return cudaErrorInvalidValue;
  const int npad = (lat.n + 63) / 64 * 64;
  uniform_table_kernel<<<(npad + 255) / 256, 256, 0, st>>>(lat, r, uniform_stride(r), tab);
  return cudaGetLastError();
}

cudaError_t launch_estep(int precision, const double *Y, int64_t n, int g, int p, int r,
                         const LatticeDev &lat, const CompT<double> *c64, const CompT<float> *c32,
                         const double *chi64, const float *chi32, EstepOut out, bool density_only,
                         int e2_mode, unsigned long long *rescue_list, unsigned *rescue_count, int *d_status,
                         int pairs_per_warp, cudaStream_t st, SweepTiming tm, int triage,
                         const double *d_pi, float tnats, int prio, int shared) {
  if (n <= 0) return cudaSuccess;
  EArgs a = make_args(Y, n, g, p, lat, out, e2_mode, rescue_list, rescue_count, d_status, triage, d_pi, tnats,
                      prio, shared);
  if (pairs_per_warp <= 0) {
    // about sixteen waves of two resident CTAs per SM (8 warps each), so the
    // last wave's imbalance stays small; 1..32 pairs per warp (measured best
    // near 8 on the p=4, r=4, g=3, n=100000 workload)
    const int64_t target_ctas = (int64_t)sm_count() * 2 * 16;
    int64_t ppw = ((int64_t)g * n) / (target_ctas * 8);
    pairs_per_warp = (int)(ppw < 1 ? 1 : (ppw > 32 ? 32 : ppw));
  }
  a.ppw = pairs_per_warp > 32 ? 32 : pairs_per_warp;
  if (precision == CFUST_FP64) {
    a.comp = c64;
    a.chi = chi64;
    return density_only ? dispatch_r<double, true>(r, a, g, n, st, false, c64, chi64, tm)
                        : dispatch_r<double, false>(r, a, g, n, st, false, c64, chi64, tm);
  }
  a.comp = c32;
  a.chi = chi32;
  return density_only ? dispatch_r<float, true>(r, a, g, n, st, true, c64, chi64, tm)
                      : dispatch_r<float, false>(r, a, g, n, st, true, c64, chi64, tm);
}

}  // namespace cfust

// Internal declarations shared by the CUDA translation units of libcfust.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cfust.h"

namespace cfust {

constexpr int PMAX = CFUST_PMAX;

// Streaming multiprocessors of the current CUDA device (cudaDevAttrMultiProcessorCount,
// queried once per device ordinal and cached).  Persistent grids and block caps
// are sized from it.
int sm_count();

// Raises the dynamic shared-memory limit of a kernel on the current device to
// at least `bytes` (never lowers it; nothing to do up to the default, which is
// 48 KB less the function's static shared memory).
// A limit that went down after a launch was captured into a CUDA graph could
// leave the graph's launch above it, so every kernel of this library sets its
// limit through here.
cudaError_t raise_smem_limit(const void *func, size_t bytes);
constexpr int RMAX = CFUST_RMAX;
constexpr int WARP = 32;

// Device-side error bits (OR-ed into the context's status word).
enum : int {
  ERR_NOTPD_OMEGA = 1 << 0,
  ERR_NOTPD_LAMBDA = 1 << 1,
  ERR_NOTPD_S6 = 1 << 2,
  ERR_NOTPD_SIGMA = 1 << 3,
  ERR_NUMERIC = 1 << 4,
  ERR_DEGENERATE = 1 << 5,
  ERR_TIMEOUT = 1 << 6,
  ERR_ZERO_DENSITY = 1 << 7,
  ERR_BAD_LABEL = 1 << 8,    // a partition label outside 0..g-1
  ERR_INIT_GROUP = 1 << 9,   // a partition group with < p + 1 members or a singular covariance
};

// Per-component constants of Eq. 2, produced in double by the precompute
// kernel and read by the E-step.  The per-pair prologue (z, d, q) always runs
// in double; the lattice sweep reads L and 1/L_tt in its own precision T.
//   A = chol(Omega)^{-1} (lower), B = (A Delta)^T, L = chol(Lambda) with
//   Lambda = I - B B^T = I - Delta^T Omega^{-1} Delta,
//   c0 = r log 2 + lgamma((nu+p)/2) - lgamma(nu/2) - (p/2) log(nu pi) - (1/2) log|Omega|.
template <typename T>
struct CompT {
  double mu[PMAX];
  double A[PMAX * PMAX];  // row-major, stride PMAX, lower triangle used
  double B[RMAX * PMAX];  // r x p, stride PMAX
  double c0;
  double nu, mA, mB;      // nu, nu + p, nu + p + 2
  double psiA;            // digamma((nu + p) / 2)
  double logmA;           // log(nu + p)
  T L[RMAX * RMAX];       // r x r, stride RMAX, lower triangle used
  T Linv[RMAX];           // 1 / L_tt
  double lamd[RMAX];      // 1 / sqrt(Lambda_tt): standardises the limits for the variable order
  double lam[RMAX * (RMAX + 1) / 2];  // Lambda, packed lower (t, h <= t at t(t+1)/2 + h)
  // single-precision copies for code that runs in float throughout (the
  // surrogate E-step), so it converts nothing per pair
  float fmu[PMAX], fA[PMAX * PMAX], fB[RMAX * PMAX];
  float fc0, fnu, fmA, fmB, fpsiA;
};

// Layout of the device parameter block (doubles): pi[g] mu[g][p] Sigma[g][p][p]
// Delta[g][p][r] nu[g], exactly the host cfust_params arrays back to back.
struct ParamView {
  double *pi, *mu, *Sigma, *Delta, *nu;
};

__host__ __device__ inline int64_t param_block_size(int g, int p, int r) {
  return (int64_t)g * (2 + p + p * p + p * r);
}

__host__ __device__ inline ParamView param_view(double *base, int g, int p, int r) {
  ParamView v;
  v.pi = base;
  v.mu = v.pi + g;
  v.Sigma = v.mu + (int64_t)g * p;
  v.Delta = v.Sigma + (int64_t)g * p * p;
  v.nu = v.Delta + (int64_t)g * p * r;
  return v;
}

// Number of doubles in one component's M-step sum vector:
// S1, S2, S3[p], S4[r], S5[p][r], S6[r(r+1)/2], S7[p(p+1)/2], S8.
__host__ __device__ inline int sums_width(int p, int r) {
  return 3 + p + r + p * r + r * (r + 1) / 2 + p * (p + 1) / 2;
}

// ---------------------------------------------------------------------------
// Launchers (one translation unit each)
// ---------------------------------------------------------------------------

// Lattice rule on the device.  For coordinate t, frac(k z_t / n + shift_t) * n
// = m + sfrac_t with the integer m = (k z_t + sint_t) mod n, sint_t = floor(shift_t n)
// and sfrac_t = shift_t n - sint_t in [0, 1).  The baker-transformed point is
// u = 1 - |2 (m + sfrac_t)/n - 1|; the sweep needs 1 - u = |2m - n + 2 sfrac_t| / n,
// which this integer/fraction split keeps accurate in single precision.
struct LatticeDev {
  int n;                 // points
  int z[RMAX + 1];       // generator vector mod n
  int step[RMAX + 1];    // (32 z) mod n: advance of one lane between its points
  int sint[RMAX + 1];
  double sfrac[RMAX + 1];
  double shift[RMAX + 1];
  // polls of a bounded mbarrier wait (the sweeps' staging of this lattice's
  // tables) before it gives up with ERR_TIMEOUT; 2^22 unless a test lowers it
  int wait_polls = 1 << 22;
  // single-precision uniforms of every point for the r normal coordinates:
  // row k = [1 - u_1 .. 1 - u_r, u_1 .. u_r, padding] with a row stride of
  // uniform_stride(r) floats (device memory; built by launch_uniform_table)
  const float *utab = nullptr;
  // the same values in the order of the shared-points sweep, which takes the
  // points k and k + 32 side by side: for k = 64 b + l (l < 32), entry
  // (b, l) holds, for each of the uniform_stride(r) columns c, the pair
  // (row k [c], row k + 32 [c]) (row k again where k + 32 >= n); entries for
  // ceil(n / 64) blocks, right after the row table in the same allocation
  const float *utab2 = nullptr;
};

__host__ __device__ constexpr int uniform_stride(int r) { return ((2 * r + 3) / 4) * 4; }

// Floats of the two uniform tables of an n-point lattice for r normal
// coordinates (the row table, then the pair-interleaved one).
__host__ __device__ constexpr int64_t uniform_table_floats(int n, int r) {
  return ((int64_t)n + ((int64_t)n + 63) / 64 * 64) * uniform_stride(r);
}

// Fill the uniform tables of `lat` for r normal coordinates into tab (row
// table [lat.n][uniform_stride(r)], then the pair-interleaved table, see
// LatticeDev::utab2; uniform_table_floats(lat.n, r) floats), with the same
// single-precision arithmetic as the sweep used to form them per point.
cudaError_t launch_uniform_table(const LatticeDev &lat, int r, float *tab, cudaStream_t st);

// Precompute: factorisations, constants and chi-scale tables for every component.
cudaError_t launch_precompute(const double *d_params, int g, int p, int r, const LatticeDev &lat,
                              CompT<double> *c64, CompT<float> *c32, double *chi64, float *chi32,
                              int *d_status, cudaStream_t st);

struct EstepOut {
  void *logf, *e1, *e2, *e3, *e4;
};

// Optional CUDA events recorded right before and after the sweep kernel;
// `capturing` selects external event-record nodes inside a stream capture.
struct SweepTiming {
  cudaEvent_t start = nullptr, stop = nullptr;
  bool capturing = false;
};

// E-step lattice sweeps for all (i, j).  precision: CFUST_FP64 / CFUST_FP32.
// In FP32 mode, pairs whose sweep underflows are appended to rescue_list and
// recomputed by the log-domain rescue pass (both launched here).  With
// `triage`, a queued pair whose posterior weight is below exp(-tnats) of the
// best component of its observation (judged from an upper bound of its
// density) gets log f = -inf and e = 0 instead (fit and log-likelihood paths).
cudaError_t launch_estep(int precision, const double *Y, int64_t n, int g, int p, int r,
                         const LatticeDev &lat, const CompT<double> *c64, const CompT<float> *c32,
                         const double *chi64, const float *chi32, EstepOut out, bool density_only,
                         int e2_mode, unsigned long long *rescue_list, unsigned *rescue_count, int *d_status,
                         int pairs_per_warp, cudaStream_t st, SweepTiming tm = SweepTiming(),
                         int triage = 0, const double *d_pi = nullptr, float tnats = 30.f, int prio = 0,
                         int shared = 0);

// FP32 lattice sweep (r = 3 only) of the observations listed per component:
// list[i * n + k], k < count[i] (device counts), followed by the rescue pass.
// Serves the pairs a surrogate E-step leaves to the lattice rule.
cudaError_t launch_estep_list(const double *Y, int64_t n, int g, int p, int r, const LatticeDev &lat,
                              const CompT<double> *c64, const CompT<float> *c32, const double *chi64,
                              const float *chi32, EstepOut out, bool density_only, int e2_mode,
                              const int *list, const unsigned *count, unsigned long long *rescue_list,
                              unsigned *rescue_count, int *d_status, cudaStream_t st, int triage,
                              const double *d_pi, float tnats = 30.f, int prio = 0, int shared = 0);

// Device view of a trained surrogate network (owned by cfust_surrogate):
// packed BF16 weights W1 [16][128], W2, W3 [128][128], W4 [128][16] (input x
// output, zero padded), FP32 biases and the 20 target-normalisation values.
struct SurrogateDev {
  const void *W1, *W2, *W3, *W4;
  const float *b1, *b2, *b3, *b4;
  const float *norm;
};

SurrogateDev surrogate_dev(const cfust_surrogate *s);

// Standardised problems (network inputs, two rows per pair) of every
// stride-th pair in the network's domain into x_out [max_rows][7]; the number
// of rows wanted goes to *count (device).
cudaError_t launch_surrogate_problems(const double *Y, int64_t n, int g, int p, const CompT<float> *c32,
                                      int64_t stride, float *x_out, int64_t max_rows, unsigned long long *count,
                                      cudaStream_t st);

// Both network inputs of every pair as the surrogate E-step forms them
// (BF16-rounded values as floats) into x_out [g n][2][7], and each pair's
// domain class into kind [g n].
cudaError_t launch_surrogate_inputs(const double *Y, int64_t n, int g, int p, const CompT<float> *c32, float *x_out,
                                    int *kind, cudaStream_t st);

// Surrogate E-step (FP32 outputs, r = 3): for every pair whose standardised
// problem lies in the training domain the network gives log T_A, T_B and the
// pass-B moments, from which log f and e1..e4 are formed as in the lattice
// sweep; other pairs are appended to fb_list[i * n + k] / fb_count[i] (both
// zeroed here first) for launch_estep_list.
cudaError_t launch_surrogate_estep(const SurrogateDev &sd, const double *Y, int64_t n, int g, int p,
                                   const CompT<float> *c32, EstepOut out, bool density_only, int *fb_list,
                                   unsigned *fb_count, int *status, cudaStream_t st);

// Elementwise single-precision normal functions (see cfust_normal_f32).
cudaError_t launch_normal_f32(const float *x, float *out, int64_t n, int which, cudaStream_t st);

// Posterior memberships (Eq. 4), log-likelihood partials (Eq. 3) and the
// M-step sum partials of Section 3.2 for components [0, g).
struct PosteriorArgs {
  const double *Y;
  int64_t n;
  int g, p, r;
  const double *pi;       // device, [g]
  const void *logf;       // [g][n] or NULL when tau_in is given
  const void *tau_in;     // [g][n] or NULL
  const void *e1, *e2, *e3, *e4;
  void *tau_out;          // may be NULL
  bool want_sums;
  bool want_ll;
  double *partials;       // [nblocks][g * K]
  double *ll_partials;    // [nblocks]
  int *d_status;
  int nblocks;
};
cudaError_t launch_posterior(int precision, const PosteriorArgs &a, cudaStream_t st);
int posterior_nblocks(int64_t n);

// Fused E-step + M-step sums (fused.cu): every observation through all g
// components per tile of observations, the per-pair outputs in shared memory
// only; writes the partial sums [*nblocks][g][K] and the log-likelihood
// partials [*nblocks] that the M-step finalize and reduce_ll read (only the
// log-likelihood partials when density_only).  *nblocks <= fused_max_blocks().
int fused_max_blocks();
cudaError_t launch_fused(int precision, const double *Y, int64_t n, int g, int p, int r, const LatticeDev &lat,
                         const CompT<double> *c64, const CompT<float> *c32, const double *chi64, const float *chi32,
                         bool density_only, int e2_mode, int *d_status, unsigned *rescue_count, int pairs_per_warp,
                         double *partials, double *ll_partials, const double *d_pi, float tnats, int prio,
                         int shared, cudaStream_t st, SweepTiming tm, int *nblocks);

// Sum the per-block log-likelihood partials in a fixed order: *ll_out = sum,
// and when trace != NULL also trace[*iter] = sum and ++*iter.
cudaError_t launch_reduce_ll(const double *ll_partials, int nblocks, double *ll_out,
                             double *trace, int *iter, cudaStream_t st);

// Totals of the per-block partial sums, out[e] = sum_b partials[b][e] for
// e < gK, added block by block in order (one thread per entry).
cudaError_t launch_sum_partials(const double *partials, int nblocks, int gK, double *out, cudaStream_t st);

// Algorithm 3: per-component conditional-maximisation update from the sums.
cudaError_t launch_mstep_finalize(const double *partials, int nblocks, int g, int p, int r,
                                  int64_t n, double nu_min, double nu_max, double *d_params,
                                  int *d_status, cudaStream_t st);

// ---------------------------------------------------------------------------
// Batched fits: many independent fits (same p, r and lattice; own n and g)
// advanced together, one persistent sweep launch per EM iteration.
// ---------------------------------------------------------------------------

struct FitDesc {
  const double *Y;    // device [n][p]
  int64_t n;
  int g;
  int comp0;          // global index of this fit's first component
  int64_t pair_off;   // this fit's rows in the per-pair buffers: sum of g n over earlier fits
  int64_t param_off;  // offset (doubles) of this fit's parameter block
  int64_t part_off;   // offset (doubles) of this fit's per-block partial sums
  int blk0, nblk;     // this fit's posterior blocks (global block index, count)
};

struct CompRef {
  int fit, i;         // global component -> (fit, component within the fit)
};

struct SweepItem {
  int gc;             // global component
  unsigned j0;        // first observation of the item
};

struct BlockRef {
  int fit, lb;        // global posterior block -> (fit, block within the fit)
};

struct BatchDev {
  const FitDesc *fits;
  const CompRef *comps;
  int nfits, G;
  double *params;     // all parameter blocks back to back
  void *logf, *e1, *e2, *e3, *e4;  // per-pair buffers (precision of the context)
  int *fit_status;    // [nfits] error bits per fit
};

cudaError_t launch_precompute_batched(const BatchDev &b, int p, int r, const LatticeDev &lat,
                                      CompT<double> *c64, CompT<float> *c32, double *chi64, float *chi32,
                                      cudaStream_t st);

cudaError_t launch_estep_batched(int precision, const BatchDev &b, int p, int r, const LatticeDev &lat,
                                 const CompT<double> *c64, const CompT<float> *c32, const double *chi64,
                                 const float *chi32, const SweepItem *items, int nitems,
                                 unsigned *item_counter, bool density_only, int e2_mode, int ppw,
                                 int ctas_per_sm, unsigned long long *rescue_list, unsigned *rescue_count,
                                 int *d_status, int triage, cudaStream_t st, SweepTiming tm = SweepTiming(),
                                 int prio = 0, int shared = 0);

cudaError_t launch_posterior_batched(int precision, const BatchDev &b, int p, int r, const BlockRef *blocks,
                                     int nblocks, double *partials, double *ll_partials, bool want_sums,
                                     int g_max, cudaStream_t st);

// trace[f * stride + *iter] = sum of fit f's log-likelihood partials; then ++*iter.
cudaError_t launch_reduce_ll_batched(const BatchDev &b, const double *ll_partials, double *trace, int stride,
                                     int *iter, cudaStream_t st);

cudaError_t launch_finalize_batched(const BatchDev &b, int p, int r, const double *partials, double nu_min,
                                    double nu_max, cudaStream_t st);


// Initial values of Algorithm 1 (init.cu): per-group sums of a partition
// (mode 0: counts and sums, optionally assigning nearest centres first;
// mode 1: central second and third moments about given means), the k-means
// centre update, the group means, and the moment rule for Psi^(0).
int group_sums_width(int mode, int p);
int group_sums_nblocks(int64_t n);
cudaError_t launch_group_sums(int mode, const double *Y, int64_t n, int p, int g, int32_t *labels,
                              const double *cm, int assign, int first, double *partials, int nblk,
                              unsigned long long *changed, int *status, cudaStream_t st);
cudaError_t launch_kmeans_update(const double *partials, int nblk, int g, int p, double *centers, cudaStream_t st);
cudaError_t launch_group_means(const double *partials, int nblk, int g, int p, double *means, double *counts,
                               cudaStream_t st);
cudaError_t launch_moment_finalize(const double *partials, int nblk, const double *counts, const double *means,
                                   int64_t n, int g, int p, int r, double nu0, double lam, double *params,
                                   double *lam_used, int *status, cudaStream_t st);

}  // namespace cfust

/*
 * cfust.h - C ABI of the GB300 CFUST-mixture EM library (libcfust.so).
 *
 * The library fits finite mixtures of canonical fundamental skew t (CFUST)
 * distributions by EM, the model of Eq. 1 and Eq. 2 of Lee, McLachlan and
 * Leemaqz, "Multi-Node EM Algorithm for Finite Mixture Models"
 * (arXiv:2005.06848):
 *
 *   f(y; Psi)   = sum_i pi_i f_i(y; theta_i)                       (Eq. 1)
 *   f_i(y)      = 2^r t_p(y; mu, Omega, nu)
 *                 T_r(Delta^T Omega^{-1}(y - mu) sqrt((nu+p)/(nu+d)); 0, Lambda, nu+p)  (Eq. 2)
 *   Omega = Sigma + Delta Delta^T,  Lambda = I_r - Delta^T Omega^{-1} Delta,
 *   d = (y-mu)^T Omega^{-1} (y-mu).
 *
 * The paper writes the skew dimension as q; it is r here.  Every call runs its
 * arithmetic in this library's CUDA kernels (sm_103a); nothing falls back to
 * the host.
 *
 * Conventions
 *  - The caller owns every buffer.  Y and the per-pair E-step arrays are DEVICE
 *    pointers on the context's stream; cfust_params and the scalar outputs
 *    (log-likelihood, traces) are HOST memory.
 *  - Y is row-major [n][p] double, 8-byte aligned.
 *  - Per-pair arrays are component-major and coalesced in the observation
 *    index j: tau[g][n], logf[g][n], e1[g][n], e2[g][n], e3[g][r][n],
 *    e4[g][r(r+1)/2][n] with e4 packed as the lower triangle row by row
 *    (entry (t, h), h <= t, at t(t+1)/2 + h).  Their element type is double in
 *    CFUST_FP64 mode and float in CFUST_FP32 mode.
 *  - Calls that return host scalars synchronise the context's stream; the
 *    others are stream-ordered.  No call aborts: errors come back as a
 *    negative cfust_status, and cfust_last_error() gives a message.
 *  - Limits: 1 <= p <= CFUST_PMAX, 1 <= r <= CFUST_RMAX, 1 <= g <= CFUST_GMAX,
 *    32 <= lattice points <= CFUST_NMAX with the count a multiple of 32.
 */
#ifndef CFUST_H
#define CFUST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CFUST_PMAX 16
#define CFUST_RMAX 6
#define CFUST_GMAX 64
#define CFUST_NMAX 65536

typedef int cfust_status;
#define CFUST_OK           0
#define CFUST_EINVAL      -1   /* bad argument or parameter (message says which) */
#define CFUST_ENOTPD      -2   /* Omega, Lambda, S6 or an updated Sigma not positive definite */
#define CFUST_ENUMERIC    -3   /* NaN/Inf, or an observation with zero density under every component */
#define CFUST_EDEGENERATE -4   /* a component's sum of tau fell below 1e-10 n */
#define CFUST_ETIMEOUT    -5   /* a bounded device wait ran out (no fault is raised) */
#define CFUST_ECUDA       -6   /* a CUDA runtime call failed */
#define CFUST_ENOMEM      -7   /* device allocation failed */

#define CFUST_FP64 0   /* every step in double precision (parity mode) */
#define CFUST_FP32 1   /* lattice sweeps and posterior exponentials in float; the M-step sums to
                          double accuracy as double-float arithmetic (exact products, two-sum
                          compensated tile sums, tile totals in double); factorisations, per-pair
                          prologue, log-sum-exp, log-likelihood and the update in double */

/* Mixture parameters Psi = (pi_1..pi_g, theta_1..theta_g), theta_i = (mu_i, Sigma_i, Delta_i, nu_i)
 * (Section 2).  Host memory, row-major:
 *   pi[g], mu[g][p], Sigma[g][p][p] (full symmetric), Delta[g][p][r], nu[g].
 * nu_i = +inf selects the CFUST family's skew-normal limit for component i
 * (W = 1: t_p becomes the normal density, T_r the normal orthant probability,
 * e1 = 1, e2 = 0); the M-step keeps nu_i = +inf.  A surrogate network leaves
 * such components to the lattice rule (their dof lie outside its domain). */
typedef struct {
  int g, p, r;
  double *pi;
  double *mu;
  double *Sigma;
  double *Delta;
  double *nu;
} cfust_params;

/* Shifted rank-1 lattice rule used for every r-variate t integral: point k
 * (k = 0..n-1) is u_k = frac(((k z) mod n)/n + shift), then the baker's
 * transform u <- 1 - |2u - 1| is applied.  dim must be r + 1: coordinate 0
 * drives the chi-square mixing variable, 1..r the normal variables.
 * z and shift are host arrays of length dim, read at cfust_create. */
typedef struct {
  int n;
  int dim;
  const int64_t *z;
  const double *shift;
} cfust_lattice;

typedef struct {
  int precision;          /* CFUST_FP64 or CFUST_FP32 */
  cfust_lattice lattice;
  int e2_mode;            /* 0: e2 = e1 - log((nu+d)/2) - (nu+p)/(nu+d) + psi((nu+p)/2);
                             1: lattice estimate of E[log W | y] from the density sweep */
  double nu_min, nu_max;  /* bracket of the nu update; 0, 0 selects [1, 200] */
  int max_iter;           /* EM iterations run by cfust_fit */
  double tol;             /* Aitken stopping threshold (Algorithm 4); 0 disables it */
  int use_graph;          /* 1: cfust_fit replays one CUDA graph per EM iteration */
  int timing;             /* 1: bracket every lattice-sweep kernel launch with CUDA events */
  int pairs_per_warp;     /* observations one warp sweeps in turn (1..32); 0 = chosen from n and g */
  int autotune;           /* 1: cfust_fit_batched times candidate launch shapes (pairs per warp,
                             resident CTAs per SM) on its first call for a batch and keeps the fastest */
  double triage_nats;     /* T: in the fit and log-likelihood paths a pair left to a slower rule (the
                             double-precision rescue, or the lattice rule behind a surrogate) whose
                             density bound puts tau_ij below exp(-T) gets log f = -inf, e = 0; each such
                             pair moves l by at most exp(-T).  0 selects 30; else in [1, 700]. */
  int prioritise;         /* 1: Genz variable prioritisation: each pair's r variables are integrated in
                             decreasing order of the standardised limit -q_t / sqrt(Lambda_tt) (ties
                             keep the lower index) with the Cholesky factor of the permuted Lambda;
                             the moments come back in the original order.  Same integral, much
                             smaller lattice error for pairs in the tails.  Every lattice sweep takes
                             it: single and batched fits, and the pairs a surrogate leaves to the
                             lattice rule (the network's own pairs are not integrated). */
  int test_wait_polls;    /* for tests of the timeout path only; 0 in normal use.  The lattice sweeps
                             stage a component's chi tables with an asynchronous bulk copy and wait on
                             its completion for a bounded number of polls (2^22 by default) before they
                             give up with CFUST_ETIMEOUT; k > 0 sets that bound, -1 makes the wait give
                             up at once.  On giving up a block first lets its copy land (bounded by the
                             default), then returns: no fault, no hang, the context stays usable. */
  int fused;              /* 1: cfust_fit (and cfust_fit_begin/step/end) and cfust_loglik run each E-step
                             and the M-step sums of Section 3.2 (Algorithm 2's per-block partial sums) as
                             one kernel: a CTA takes a tile of observations through all g components,
                             keeps log f_ij and e1..e4 in shared memory only, forms tau (Eq. 4), l_j
                             (Eq. 3) and every sum entry, and writes per-block partials that the M-step
                             (Algorithm 3) combines.  Nothing of size g x n is allocated or moved: the
                             fit holds Y and the partial sums only.  Same rule and per-pair arithmetic as
                             the unfused path (results agree to summation order; pairs needing the
                             double-precision rescue are recomputed by the tile's CTA).  cfust_estep,
                             cfust_mstep*, cfust_fit_batched and the explicit E-step outputs keep the
                             unfused kernels; a fit or log-likelihood with a surrogate attached and
                             fused = 1 fails with CFUST_EINVAL. */
  int shared_points;      /* 1: pass B (T_B and the truncated moments at dof nu+p+2 that give e1, e3, e4,
                             the E-step expectations of Section 2's latent gamma and truncated normal
                             variables) is estimated on pass A's lattice points.  The two laws differ only in the
                             chi-square variable x, and chi2_{nu+p+2}(x) = chi2_{nu+p}(x) x / (nu+p): at
                             pass A's x of a point pass B's scaled limits equal pass A's, so pass A's
                             conditional draws serve both, pass B with the extra weight x / (nu+p).  The
                             same integrals with one conditional chain per point instead of two (about
                             half the normal-function work); log f and l are pass A's, unchanged, and
                             e1..e4 move within the rule's error.  0 keeps the two separate sweeps.
                             Taken by every lattice sweep in both precisions and either variable order:
                             cfust_estep, cfust_loglik, the single and batched fits, the fused pass, and
                             the pairs a surrogate leaves to the lattice rule. */
} cfust_opts;

typedef struct cfust_ctx cfust_ctx;

/* Create a context bound to the current CUDA device and to cuda_stream (a
 * cudaStream_t; NULL means the legacy default stream).  Copies opts and the
 * lattice spec.  Allocates per-context device scratch lazily on first use. */
cfust_status cfust_create(cfust_ctx **ctx, const cfust_opts *opts, void *cuda_stream);

/* Free the context and its device scratch.  NULL is accepted. */
cfust_status cfust_destroy(cfust_ctx *ctx);

/* l(Psi) = sum_j log sum_i pi_i f_i(y_j) (Eq. 1, Eq. 3), one density sweep per pair.
 * Y: device [n][p].  loglik: host, written on success.  Synchronises. */
cfust_status cfust_loglik(cfust_ctx *ctx, const double *Y, int64_t n,
                          const cfust_params *params, double *loglik);

/* E-step of Section 2 (Algorithm 2's per-pair work): for every (i, j),
 * tau_ij = pi_i f_ij / f_j (Eq. 4) and the conditional expectations
 * e1 = E[W|y], e2 = E[log W|y], e3 = E[W U|y], e4 = E[W U U^T|y] of the latent
 * gamma W and truncated-normal U.  logf (log f_i(y_j)) may be NULL; the
 * others must be device arrays in the layout above.  loglik (host, may be
 * NULL) receives l(Psi).  Synchronises when loglik is not NULL. */
cfust_status cfust_estep(cfust_ctx *ctx, const double *Y, int64_t n,
                         const cfust_params *params,
                         void *logf, void *tau, void *e1, void *e2, void *e3, void *e4,
                         double *loglik);

/* M-step of Algorithm 3: accumulates the eight per-component sums of
 * Section 3.2 from tau, e1..e4 (device, same layout and element type as
 * cfust_estep's outputs) and Y, then updates params in place (host) by
 * conditional maximisation: pi, mu, Delta, Sigma, nu.  Synchronises. */
cfust_status cfust_mstep(cfust_ctx *ctx, const double *Y, int64_t n,
                         const void *tau, const void *e1, const void *e2,
                         const void *e3, const void *e4, cfust_params *params);

/* The M-step split at its one exchange point, for fits whose observations
 * are spread over several processes or devices (Algorithm 2's per-worker
 * partial sums, Section 3.2, and Algorithm 3's combine by the master,
 * Section 3.3): every worker runs cfust_estep on its own rows and
 * cfust_mstep_sums on them; the workers add their sums vectors (e.g. one
 * all-reduce of g K doubles) and every worker runs cfust_mstep_apply on the
 * totals, which gives each the same parameters.
 *
 * cfust_mstep_sums: the eight per-component sums of Section 3.2 over this
 * call's n observations into sums (host, [g][K] doubles, K = 3 + p + r + p r
 * + r(r+1)/2 + p(p+1)/2), component i's vector at i K:
 *   S1 = sum tau, S2 = sum tau e1, S3[a] = sum tau e1 y_a (p entries),
 *   S4[t] = sum tau e3_t (r), S5[a][t] = sum tau y_a e3_t (p r, a-major),
 *   S6 = sum tau e4 (packed lower triangle, r(r+1)/2), S7 = sum tau e1 y y^T
 *   (packed lower triangle, p(p+1)/2), S8 = sum tau (e2 - e1).
 * Inputs as for cfust_mstep; params: host, read only (its g, p, r give the
 * shapes).  Synchronises.
 *
 * cfust_mstep_apply: Algorithm 3's conditional-maximisation update (the
 * same update as cfust_mstep) from sums (host [g][K], the totals over every
 * worker's rows) and the total number of observations n_total; params (host)
 * in: the current parameters (Delta enters the mu update), out: the update.
 * CFUST_ENUMERIC when a sum is not finite.  Synchronises.  Summing the
 * workers' vectors in another order changes the result only by rounding. */
cfust_status cfust_mstep_sums(cfust_ctx *ctx, const double *Y, int64_t n,
                              const void *tau, const void *e1, const void *e2,
                              const void *e3, const void *e4, const cfust_params *params,
                              double *sums);
cfust_status cfust_mstep_apply(cfust_ctx *ctx, const double *sums, int64_t n_total,
                               cfust_params *params);

/* Full EM (Section 2 outline) from params (updated in place): at most
 * opts.max_iter iterations, stopping early by Algorithm 4 when opts.tol > 0.
 * loglik_trace (host, length max_iter + 1, may be NULL) receives
 * l(Psi^(0)) .. l(Psi^(k)), each E-step yielding the log-likelihood of the
 * parameters it starts from.  iters_done (may be NULL) receives k. */
cfust_status cfust_fit(cfust_ctx *ctx, const double *Y, int64_t n,
                       cfust_params *params, double *loglik_trace, int *iters_done);

/* Stepwise form of cfust_fit for callers that drive the iterations themselves.
 * In the fit and log-likelihood paths a single-precision pair whose lattice
 * sum underflows and whose posterior weight is provably below exp(-30) of the
 * best component of its observation gets density 0 (tau = 0, e = 0) instead of
 * the log-domain recomputation that cfust_estep always performs.
 * cfust_fit_begin uploads params and binds Y (device [n][p], kept until
 * cfust_fit_end) and resets the trace.  cfust_fit_step enqueues `iters` EM
 * iterations on the context's stream without synchronising (each a replay of
 * one CUDA graph when opts.use_graph is 1); at most opts.max_iter iterations
 * in total.  cfust_fit_end runs the final density sweep, synchronises, and
 * returns the parameters, the trace l(Psi^(0)) .. l(Psi^(k)) (host, k + 1
 * entries, may be NULL) and k (may be NULL). */
cfust_status cfust_fit_begin(cfust_ctx *ctx, const double *Y, int64_t n,
                             const cfust_params *params);
cfust_status cfust_fit_step(cfust_ctx *ctx, int iters);
cfust_status cfust_fit_end(cfust_ctx *ctx, cfust_params *params, double *loglik_trace,
                           int *iters_done);

/* During a stepwise fit: synchronise and copy the log-likelihood trace so far,
 * l(Psi^(0)) .. l(Psi^(k-1)) after k cfust_fit_step iterations, into trace
 * (host, at least k entries); *count receives k. */
cfust_status cfust_fit_trace(cfust_ctx *ctx, double *trace, int *count);

/* Many independent fits advanced together (Algorithm 1's multiple starts, or
 * separate data sets): fit f has Y[f] (device [n[f]][p]) and params[f]
 * (host, updated in place); every fit shares p, r and the context's lattice,
 * g may differ.  Runs opts.max_iter EM iterations, each one CUDA graph whose
 * E-step is a single persistent sweep launch over all fits' (component,
 * observation tile) items.  loglik_trace (host [nfits][max_iter + 1], may be
 * NULL) receives each fit's l(Psi^(0)) .. l(Psi^(max_iter)).  fit_status
 * (host [nfits], may be NULL) receives each fit's cfust_status; the call
 * returns the first non-zero one.  Y pointers must stay valid during the call. */
cfust_status cfust_fit_batched(cfust_ctx *ctx, int nfits, const double *const *Y, const int64_t *n,
                               cfust_params *params, double *loglik_trace, int *fit_status);

/* Launch shape chosen for the last batched fit (by the autotuner or the
 * default rule): pairs per warp and resident CTAs per SM of the sweep. */
cfust_status cfust_batched_shape(cfust_ctx *ctx, int *pairs_per_warp, int *ctas_per_sm);

/* Multiple starts (Algorithm 1, with the largest log-likelihood kept; the
 * paper's listing selects the smallest, a misprint for maximum likelihood):
 * every start runs burn_in EM iterations (all starts together as one batched
 * fit over the same observations; burn_in = 0 compares the starts'
 * log-likelihoods directly), the start with the largest log-likelihood after
 * its burn-in is chosen and fitted further like cfust_fit (opts.max_iter,
 * opts.tol).  starts: host [nstarts], updated in place (every start holds its
 * burned-in parameters; starts[*best] the fitted ones).  trace and iters_done
 * as for cfust_fit, for the final fit.  Starts that fail their burn-in
 * (degenerate, not positive definite) are not chosen; CFUST_EDEGENERATE when
 * none survives.  The burn-in runs as a batched fit. */
cfust_status cfust_fit_multistart(cfust_ctx *ctx, const double *Y, int64_t n, cfust_params *starts, int nstarts,
                                  int burn_in, int *best, double *loglik_trace, int *iters_done);

/* Initial partitions of Algorithm 1 by k-means (Section 3.1 names k-means
 * and random partitions; the rule here is Lloyd's): each iteration assigns
 * every observation to its nearest centre (squared Euclidean distance summed
 * over the coordinates in order, each difference, square and sum rounded
 * separately in double precision; ties to the lowest index) and stops when no
 * label changed; otherwise each centre moves to the mean of its members (a
 * centre without members stays).  Y: device [n][p].  centers: host [g][p],
 * the starting centres on entry, the final ones on return.  labels: device
 * int32 [n], written.  iters_done (host, may be NULL): assignment passes run
 * (<= max_iter).  Synchronises every iteration.  CFUST_EINVAL for bad sizes
 * or max_iter < 1. */
cfust_status cfust_kmeans(cfust_ctx *ctx, const double *Y, int64_t n, int p, int g, double *centers, int max_iter,
                          int32_t *labels, int *iters_done);

/* Psi^(0) of a partition by moments (Algorithm 1's "compute Psi^(0)"; the
 * paper does not give the rule, this is the library's): for group i with n_i
 * members, pi_i = n_i / n, nu_i = nu0, Delta_i diagonal in its first
 * min(p, r) columns with Delta_i[k][k] = lam * sign(skewness_k) * sd_k (the
 * group's sample skewness and standard deviation of coordinate k, sign +1 at
 * zero), and mu_i, Sigma_i matching the group's sample mean and covariance
 * (divisor n_i) to the CFUST law's:
 *   E[Y] = mu + m1 Delta 1_r,  Cov(Y) = nu/(nu-2) Sigma + Delta C Delta^T,
 * m1 = E|U_k|, C = Cov(|U|), U ~ t_r(0, I, nu0).  lam is halved (at most 20
 * times, then 0) until Sigma_i is positive definite.  labels: device int32
 * [n] in 0..g-1 (CFUST_EINVAL otherwise).  params: host; g, p, r and the
 * arrays set by the caller, the arrays written on success.  nu0 > 2 and
 * lam >= 0 (CFUST_EINVAL otherwise).  CFUST_EDEGENERATE when a group has
 * fewer than p + 1 members or a singular sample covariance.  Synchronises. */
cfust_status cfust_init_partition(cfust_ctx *ctx, const double *Y, int64_t n, const int32_t *labels, double nu0,
                                  double lam, cfust_params *params);

/* Algorithm 1 from m partitions: Psi^(0) of each partition (cfust_init_partition),
 * then cfust_fit_multistart over the partitions that gave initial values.
 * labels: device int32 [m][n].  starts: host [m] with g, p, r and arrays set
 * by the caller; start f receives its Psi^(0) (burned in when burn_in > 0;
 * the chosen one is fitted further).  best: index into 0..m-1 of the chosen
 * partition.  loglik_trace, iters_done: as for cfust_fit.  CFUST_EDEGENERATE
 * when no partition gives initial values or no start survives its burn-in. */
cfust_status cfust_multistart_partitions(cfust_ctx *ctx, const double *Y, int64_t n, const int32_t *labels, int m,
                                         double nu0, double lam, int burn_in, cfust_params *starts, int *best,
                                         double *loglik_trace, int *iters_done);

/* l(Psi) under M shifted copies of the context's lattice rule (same
 * generator z, shift m = shifts[m][0..dim-1], host, each in [0, 1)):
 * randomised quasi-Monte Carlo.  With independent uniform shifts every
 * copy's T_r estimate is unbiased, so the spread of loglik[0..M-1] (host,
 * written) estimates the integration error of the rule: standard error
 * sd / sqrt(M) for their mean (l, a sum of logarithms, carries a bias of
 * second order in that error).  The context's own shift is restored before
 * returning (also after an error).  Works with a surrogate attached (its
 * fallback lattice is the context's).  Synchronises. */
cfust_status cfust_loglik_shifts(cfust_ctx *ctx, const double *Y, int64_t n, const cfust_params *params, int M,
                                 const double *shifts, double *loglik);

/* Number of (i, j) pairs whose single-precision lattice sweep fell below the
 * underflow guard in the last E-step and were recomputed in double precision
 * on the GPU (always 0 in CFUST_FP64 mode). */
cfust_status cfust_last_rescued(cfust_ctx *ctx, int64_t *count);

/* Device time (ms) of the last lattice-sweep kernel launch (the E-step's
 * dominant kernel), from the CUDA events recorded around it on the launching
 * stream when opts.timing is 1.  Synchronises on the stop event.
 * CFUST_EINVAL when timing is off or nothing has run yet. */
cfust_status cfust_last_sweep_ms(cfust_ctx *ctx, float *ms);

/* Device time (ms) of the last posterior / M-step-sums kernel launch of an
 * EM iteration (the eight sums of Section 3.2, unfused from the E-step),
 * from CUDA events recorded around it on the launching stream when
 * opts.timing is 1 (inside the captured graph too).  Synchronises on the
 * stop event.  CFUST_EINVAL when timing is off or no iteration has run. */
cfust_status cfust_last_mstep_ms(cfust_ctx *ctx, float *ms);

/* Single-precision normal functions of the lattice sweep, exposed for
 * verification.  x, out: device float arrays of n elements; stream: a
 * cudaStream_t (NULL = legacy default stream); stream-ordered.
 *   which 0: Phi(-x) (this library)      1: Phi^{-1}(x) (this library)
 *         2: normcdff(-x) (CUDA)          3: normcdfinvf(x) (CUDA)
 *         4: log Phi(-x) (this library)   5: -Phi^{-1}(exp(x)) (this library, x <= 0) */
cfust_status cfust_normal_f32(const float *x, float *out, int64_t n, int which, void *stream);

/* M-step without a context and without any device allocation.
 *
 * For callers that cannot allocate device memory on the call path, e.g. code
 * running under an external memory manager that forbids cudaMalloc after
 * start-up, or a host that must not grow its device footprint per call.  It
 * computes what cfust_mstep computes (the eight sums of Section 3.2 and the
 * conditional-maximisation update) from caller-owned inputs.  The paper has
 * no counterpart: this is an interface variant only.
 *
 * Scratch (status words, the device copy of params, per-block partial sums)
 * lives in one static device array of CFUST_NOALLOC_SCRATCH_BYTES (1 MiB) that
 * every GPU loading this library holds until the process exits.  The number of
 * reduction blocks is reduced to fit it, but at least CFUST_NOALLOC_MIN_BLOCKS
 * blocks' partial sums (8 * g * (3 + p + r + p r + r(r+1)/2 + p(p+1)/2) bytes
 * each) plus the parameters must fit; larger problems (e.g. g = 64, p = 16,
 * r = 6) return CFUST_EINVAL with a message naming the limit.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current).  All calls share the
 * array: calls that overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 *
 * precision: CFUST_FP64 or CFUST_FP32 (element type of tau, e1..e4).
 * Y, tau, e1..e4: device memory of the CURRENT device (checked: CFUST_EINVAL
 * otherwise), layouts as for cfust_estep; stream: a cudaStream_t of that
 * device (NULL = legacy default stream).  params: host, updated in place.
 * nu_min, nu_max: 0, 0 selects [1, 200].  Synchronises the stream.  Messages
 * come from cfust_last_error(NULL), which keeps one message per host thread. */
#define CFUST_NOALLOC_SCRATCH_BYTES (1u << 20)
#define CFUST_NOALLOC_MIN_BLOCKS 8
cfust_status cfust_mstep_noalloc(int precision, const double *Y, int64_t n,
                                 const void *tau, const void *e1, const void *e2,
                                 const void *e3, const void *e4, double nu_min, double nu_max,
                                 cfust_params *params, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the trivariate truncated-t integrals (r = 3).
 *
 * Not in the paper: an added form of the E-step.  The lattice rule's two
 * integrals per pair (T_A, and T_B with the truncated moments; Eq. 2 and the
 * E-step expectations of Section 3.1) are, after standardisation, functions
 * of a truncation point c in R^3, a correlation matrix R (3 off-diagonal
 * entries) and the degrees of freedom m:
 *   X ~ t_3(0, R, m):  log P(X > c),  E[X | X > c],  E[X X^T | X > c].
 * A network 7 -> 128 -> 128 -> 128 -> 10 (GELU, BF16 weights and activations,
 * FP32 accumulation on the tensor cores: tcgen05 MMAs with accumulators in
 * tensor memory for prediction and the E-step) maps
 *   x = (c_1, c_2, c_3, R_12, R_13, R_23, log m)
 * to y = (log P, E[X_1..3], E[X X^T] upper triangle 11 12 13 22 23 33).
 * Training domain: -8 <= c_t <= 4, |R_ht| <= 0.9, squared Cholesky pivots of
 * R >= 0.05, 3 <= m <= 30.  Training data come from the plain lattice rule on
 * this library's GPU (labeller below); training (forward, backward, Adam) runs
 * in this library's kernels.  Internally the network predicts log(-log P),
 * E[X] and the covariance E[X X^T] - E[X] E[X]^T, standardised per output;
 * the loss weighs log(-log P) 4x.
 *
 * Flat parameter vector theta (CFUST_SURROGATE_NPARAM floats): W1 [7][128]
 * (input x output, row-major), b1 [128], W2 [128][128], b2, W3 [128][128], b3,
 * W4 [128][10], b4 [10].  The network predicts (y - mean) / std per output;
 * norm = (mean[10], std[10]).
 * ------------------------------------------------------------------------- */
#define CFUST_SURROGATE_NPARAM 35338
typedef struct cfust_surrogate cfust_surrogate;

/* Create a surrogate with N(0, 1/fan_in) weights from SplitMix64(seed), zero
 * biases and unit normalisation.  lattice: the labeller's rule, dim 4 (chi
 * coordinate and three normal coordinates), n a multiple of 32 up to
 * CFUST_NMAX (8192 points is the intended size); its chi-scale tables are
 * built on a grid of 256 values of log m over [log 3, log 30] and
 * interpolated linearly in log m.  stream: cudaStream_t for all calls on
 * this object.  Messages from cfust_surrogate_last_error(NULL). */
cfust_status cfust_surrogate_create(cfust_surrogate **out, uint64_t seed, const cfust_lattice *lattice,
                                    void *cuda_stream);
cfust_status cfust_surrogate_destroy(cfust_surrogate *s);

/* Lattice-rule targets of B problems (B <= 2^30 here and in the calls below;
 * larger counts return CFUST_EINVAL).  x: device float [B][7] (as above), y:
 * device float [B][10].  A problem whose every point weight underflows gets
 * NaN targets.  Synchronises the stream. */
cfust_status cfust_surrogate_label(cfust_surrogate *s, const float *x, float *y, int64_t B);

/* Network prediction (de-normalised) for device x [B][7] into device y [B][10].
 * Inputs outside the training domain are evaluated all the same.
 * Synchronises the stream. */
cfust_status cfust_surrogate_predict(cfust_surrogate *s, const float *x, float *y, int64_t B);

/* Loss (mean over rows and outputs of the squared error of the normalised
 * prediction) and its gradient with respect to theta for device x [B][7] and
 * device targets y [B][10] (raw, normalised inside with the current norm).
 * loss: host double or NULL; grad: host float [CFUST_SURROGATE_NPARAM] or
 * NULL.  Synchronises the stream. */
cfust_status cfust_surrogate_gradient(cfust_surrogate *s, const float *x, const float *y, int64_t B,
                                      double *loss, float *grad);

/* Host copies of theta and norm (either may be NULL), and their replacement
 * (norm NULL keeps the current one). */
cfust_status cfust_surrogate_get_params(cfust_surrogate *s, float *theta, float *norm);
cfust_status cfust_surrogate_set_params(cfust_surrogate *s, const float *theta, const float *norm);

/* Train on n_train problems drawn over the training domain (SplitMix64(seed);
 * R and log m uniform, rows with a non-PD or too-thin R redrawn), labelled on
 * the GPU, target normalisation set from the labels (rows whose labels are not
 * finite are dropped).  Problems: half uniform over the box, half with c_t
 * drawn from N(-1.5, 2.5^2) clipped to it.  Adam (beta 0.9, 0.999,
 * eps 1e-8) on mini-batches of `batch` rows with a cosine-decayed step from
 * lr; `epochs` passes.  loss_trace: host float [epochs] (mean sampled batch
 * loss per epoch) or NULL.  Requires n_train >= batch >= 128. */
cfust_status cfust_surrogate_train(cfust_surrogate *s, int64_t n_train, int epochs, int batch, float lr,
                                   uint64_t seed, float *loss_trace);

/* Continue training on given problems: x device float [rows][7] (e.g. from
 * cfust_surrogate_problems), labelled by the lattice rule inside; rows without
 * finite labels are dropped and the rest shuffled (SplitMix64(seed)); the
 * target normalisation stays as trained; Adam continues from its state with a
 * step cosine-decayed from lr over `epochs` passes.  loss_trace: host float
 * [epochs] or NULL.  Requires 128 <= batch <= rows <= 2^30. */
cfust_status cfust_surrogate_finetune(cfust_surrogate *s, const float *x, int64_t rows, int epochs, int batch,
                                      float lr, uint64_t seed, float *loss_trace);

const char *cfust_surrogate_last_error(cfust_surrogate *s);

/* Attach a surrogate to a context (NULL detaches; the context does not own
 * it, and it must outlive its use).  With a surrogate attached, every E-step
 * of the context (cfust_estep, cfust_loglik, cfust_fit, the stepwise fit)
 * evaluates each pair's two standardised problems (pass A at dof nu+p and
 * pass B at nu+p+2, c = D^{-1/2} a with D = diag(Lambda)) with the network
 * when the pair lies in the domain, and with the context's lattice rule
 * otherwise.  A pair is the network's when its component's R and dof are in
 * the domain and pass B's point (the larger one) lies in [-8, 4]^3; when
 * nu+p >= 8 the lower edge is dropped and c_t < -8 is clamped to -8 (that
 * moves P by at most P(t_8 < -8) = 2.2e-5).  In the log-likelihood and fit
 * paths, a pair left to the lattice rule whose bound log pi_i + log f_ij
 * (the network at the clamped point, plus 5) trails the best component of
 * its observation by 30 is given tau = 0 without a sweep.  Batched fits
 * (cfust_fit_batched) always use the lattice rule.
 * Requires CFUST_FP32 precision, e2_mode 0 and r = 3 (checked when the E-step
 * runs).  Attaching drops a captured fit graph. */
cfust_status cfust_set_surrogate(cfust_ctx *ctx, cfust_surrogate *s);

/* The standardised problems the surrogate E-step would hand the network for
 * every stride-th (i, j) pair (pair index i n + j) in its domain at params P:
 * two rows (pass A, pass B) of (c_1, c_2, c_3, R_12, R_13, R_23, log m) per
 * pair, written to x_out (device float [max_rows][7]) in no particular order.
 * *rows (host) receives the rows written (at most max_rows).  Requires r = 3;
 * Y as for cfust_estep.  Synchronises the context's stream.  For tuning a
 * network to the problems a family of fits poses (cfust_surrogate_finetune). */
cfust_status cfust_surrogate_problems(cfust_ctx *ctx, const double *Y, int64_t n, const cfust_params *P,
                                      int64_t stride, float *x_out, int64_t max_rows, int64_t *rows);

/* Both network inputs of every (i, j) pair exactly as the surrogate E-step
 * hands them to the tensor cores at params P, for verification: the
 * standardised problem of pass A (dof nu+p) and pass B (nu+p+2), normalised
 * (c and log m mapped from their ranges onto [-1, 1], R / 0.9) and rounded to
 * BF16, written as floats to x_out (device float [g][n][2][7], pair (i, j) at
 * (i n + j)); kind (device int32 [g][n]) receives the pair's class: 2 the
 * network's, 1 its point leaves the box (lattice rule, log T bounded through
 * the clamped point), 0 R or the dof outside the domain (lattice rule).
 * Requires r = 3; Y as for cfust_estep.  Synchronises the context's stream. */
cfust_status cfust_surrogate_inputs(cfust_ctx *ctx, const double *Y, int64_t n, const cfust_params *P,
                                    float *x_out, int32_t *kind);

/* Pairs the last surrogate E-step handed to the lattice rule (outside the
 * training domain).  Synchronises the context's stream. */
cfust_status cfust_last_fallback(cfust_ctx *ctx, int64_t *count);

/* Message for the last error on ctx; with ctx NULL, the message of the last
 * failed cfust_create or cfust_mstep_noalloc call of the calling host thread
 * (kept per thread). */
const char *cfust_last_error(cfust_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CFUST_H */

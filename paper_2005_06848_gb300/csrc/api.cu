// Host side of the C ABI declared in include/cfust.h: context, argument
// checks, device buffers, and the EM driver (Section 2 outline; Algorithms
// 2-4) that chains the kernels on the context's stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "cfust_internal.cuh"

using namespace cfust;

namespace cfust {

int sm_count() {
  constexpr int kDevices = 64;
  static int cached[kDevices] = {};
  static std::mutex m;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) dev = -1;
  std::lock_guard<std::mutex> lock(m);
  if (dev >= 0 && cached[dev] > 0) return cached[dev];
  int sms = 0;
  if (dev < 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return 1;  // no device answers: one SM's worth of blocks, the launch itself will report the error
  cached[dev] = sms;
  return sms;
}

cudaError_t raise_smem_limit(const void *func, size_t bytes) {
  // the limit a launch may use without the opt-in is 48 KB less the
  // function's static shared memory: read it (cudaFuncGetAttributes) the first
  // time a function is seen on a device, then only ever raise it
  static std::mutex m;
  static std::vector<std::pair<std::pair<int, const void *>, size_t>> limits;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  std::lock_guard<std::mutex> lock(m);
  std::pair<std::pair<int, const void *>, size_t> *ent = nullptr;
  for (auto &e : limits)
    if (e.first.first == dev && e.first.second == func) ent = &e;
  if (!ent) {
    cudaFuncAttributes fa;
    const cudaError_t err = cudaFuncGetAttributes(&fa, func);
    if (err != cudaSuccess) return err;
    limits.push_back({{dev, func}, (size_t)(fa.maxDynamicSharedSizeBytes > 0 ? fa.maxDynamicSharedSizeBytes : 0)});
    ent = &limits.back();
  }
  if (bytes <= ent->second) return cudaSuccess;
  const cudaError_t err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (err == cudaSuccess) ent->second = bytes;
  return err;
}

}  // namespace cfust

struct cfust_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cfust_opts opts{};
  LatticeDev lat{};
  std::string err;

  int g = 0, p = 0, r = 0;
  int64_t n_cap = 0;       // observations the pair buffers hold
  int nb_cap = 0;          // posterior blocks the partial buffers hold

  double *d_params = nullptr;
  CompT<double> *d_c64 = nullptr;
  CompT<float> *d_c32 = nullptr;
  double *d_chi64 = nullptr;
  float *d_chi32 = nullptr;
  int *d_status = nullptr;      // [0] error bits, [1] EM iteration counter
  unsigned *d_rescue_cnt = nullptr;
  double *d_ll = nullptr;
  double *d_trace = nullptr;
  int trace_cap = 0;
  unsigned long long *d_rescue = nullptr;
  double *d_partials = nullptr;
  double *d_sums = nullptr;     // [g][K] totals of cfust_mstep_sums
  double *d_llpart = nullptr;
  void *d_logf = nullptr, *d_e1 = nullptr, *d_e2 = nullptr, *d_e3 = nullptr, *d_e4 = nullptr;

  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  cudaEvent_t ev_sweep[2] = {nullptr, nullptr};
  bool sweep_recorded = false;
  cudaEvent_t ev_post[2] = {nullptr, nullptr};  // around the posterior / M-step sums launch
  bool post_recorded = false;
  cudaGraphExec_t gexec = nullptr;
  const double *graph_Y = nullptr;
  int64_t graph_n = 0;

  // batched fits (cfust_fit_batched)
  struct Batch {
    int nfits = 0, G = 0, p = 0, r = 0, g_max = 0, nitems = 0, nblocks = 0, K = 0;
    int ppw = 0, cps = 2;
    bool tuned = false;
    std::vector<const double *> Y;
    std::vector<int64_t> n;
    std::vector<int> g;
    int64_t pairs = 0, params_len = 0, part_len = 0;
    FitDesc *d_fits = nullptr;
    CompRef *d_comps = nullptr;
    SweepItem *d_items = nullptr;
    BlockRef *d_blocks = nullptr;
    double *d_params = nullptr;
    CompT<double> *c64 = nullptr;
    CompT<float> *c32 = nullptr;
    double *chi64 = nullptr;
    float *chi32 = nullptr;
    void *logf = nullptr, *e1 = nullptr, *e2 = nullptr, *e3 = nullptr, *e4 = nullptr;
    unsigned long long *rescue = nullptr;
    unsigned *rescue_cnt = nullptr, *counter = nullptr;
    double *partials = nullptr, *llpart = nullptr, *trace = nullptr;
    int *iter = nullptr, *fit_status = nullptr, *status = nullptr;
    cudaGraphExec_t graph = nullptr;
  } batch;

  // learned surrogate E-step (not owned) and its fallback lists
  cfust_surrogate *sur = nullptr;
  float *d_utab = nullptr;       // lattice uniforms (LatticeDev::utab)
  unsigned long long *d_prob_cnt = nullptr;  // cfust_surrogate_problems row count
  int *d_fb = nullptr;           // [g][n] observations left to the lattice rule
  unsigned *d_fb_cnt = nullptr;  // [g]
  int64_t fb_cap = 0;

  // stepwise fit state
  const double *fit_Y = nullptr;
  int64_t fit_n = 0;
  int fit_done = 0;
  bool fit_open = false;
};

namespace {

void free_batch(cfust_ctx::Batch &b);

thread_local std::string g_create_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cfust_status fail(cfust_ctx *c, cfust_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

cfust_status cuda_fail(cfust_ctx *c, cudaError_t e, const char *where) {
  return fail(c, e == cudaErrorMemoryAllocation ? CFUST_ENOMEM : CFUST_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CF_CUDA(c, call)                                    \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

template <typename P>
cudaError_t realloc_dev(P **ptr, size_t bytes) {
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  if (bytes == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
}

size_t elem_size(const cfust_ctx *c) { return c->opts.precision == CFUST_FP64 ? 8 : 4; }

void drop_graph(cfust_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->graph_Y = nullptr;
  c->graph_n = 0;
}

// (Re)allocate every device buffer for shapes (g, p, r) and n observations.
// `pairs` = false leaves out the g x n per-pair buffers (the fused path's
// fits and log-likelihoods never touch them).
cfust_status ensure(cfust_ctx *c, int g, int p, int r, int64_t n, bool pairs = true) {
  const int N = c->lat.n;
  if (g != c->g || p != c->p || r != c->r) {
    drop_graph(c);
    CF_CUDA(c, realloc_dev(&c->d_params, sizeof(double) * param_block_size(g, p, r)));
    CF_CUDA(c, realloc_dev(&c->d_c64, sizeof(CompT<double>) * g));
    CF_CUDA(c, realloc_dev(&c->d_c32, sizeof(CompT<float>) * g));
    CF_CUDA(c, realloc_dev(&c->d_chi64, sizeof(double) * 2 * (size_t)N * g));
    CF_CUDA(c, realloc_dev(&c->d_chi32, sizeof(float) * 2 * (size_t)N * g));
    CF_CUDA(c, realloc_dev(&c->d_sums, sizeof(double) * (size_t)g * sums_width(p, r)));
    c->g = g;
    c->p = p;
    c->r = r;
    c->n_cap = 0;
    c->nb_cap = 0;
    c->fb_cap = 0;
  }
  if (!c->d_status) {
    CF_CUDA(c, cudaMalloc(&c->d_status, 2 * sizeof(int)));
    CF_CUDA(c, cudaMalloc(&c->d_rescue_cnt, sizeof(unsigned)));
    CF_CUDA(c, cudaMalloc(&c->d_ll, sizeof(double)));
    CF_CUDA(c, cudaMemset(c->d_rescue_cnt, 0, sizeof(unsigned)));
  }
  int nb = posterior_nblocks(n);
  if (c->opts.fused && fused_max_blocks() > nb) nb = fused_max_blocks();
  if (nb > c->nb_cap) {
    drop_graph(c);
    CF_CUDA(c, realloc_dev(&c->d_partials, sizeof(double) * (size_t)nb * g * sums_width(p, r)));
    CF_CUDA(c, realloc_dev(&c->d_llpart, sizeof(double) * (size_t)nb));
    c->nb_cap = nb;
  }
  if (pairs && n > c->n_cap) {
    drop_graph(c);
    const size_t es = elem_size(c);
    const size_t gn = (size_t)g * (size_t)n;
    const int rp = r * (r + 1) / 2;
    CF_CUDA(c, realloc_dev(&c->d_rescue, sizeof(unsigned long long) * gn));
    CF_CUDA(c, realloc_dev(&c->d_logf, es * gn));
    CF_CUDA(c, realloc_dev(&c->d_e1, es * gn));
    CF_CUDA(c, realloc_dev(&c->d_e2, es * gn));
    CF_CUDA(c, realloc_dev(&c->d_e3, es * gn * r));
    CF_CUDA(c, realloc_dev(&c->d_e4, es * gn * rp));
    c->n_cap = n;
  }
  if (c->sur && (n > c->fb_cap || !c->d_fb_cnt)) {
    drop_graph(c);
    CF_CUDA(c, realloc_dev(&c->d_fb, sizeof(int) * (size_t)g * (size_t)n));
    CF_CUDA(c, realloc_dev(&c->d_fb_cnt, sizeof(unsigned) * CFUST_GMAX));
    CF_CUDA(c, cudaMemset(c->d_fb_cnt, 0, sizeof(unsigned) * CFUST_GMAX));
    c->fb_cap = n;
  }
  return CFUST_OK;
}

cfust_status check_params(cfust_ctx *c, const cfust_params *P) {
  if (!P) return fail(c, CFUST_EINVAL, "params is NULL");
  const int g = P->g, p = P->p, r = P->r;
  if (g < 1 || g > CFUST_GMAX) return fail(c, CFUST_EINVAL, "g out of range");
  if (p < 1 || p > CFUST_PMAX) return fail(c, CFUST_EINVAL, "p out of range");
  if (r < 1 || r > CFUST_RMAX) return fail(c, CFUST_EINVAL, "r out of range");
  if (r + 1 != c->opts.lattice.dim)
    return fail(c, CFUST_EINVAL, "lattice dimension must equal r + 1");
  if (!P->pi || !P->mu || !P->Sigma || !P->Delta || !P->nu)
    return fail(c, CFUST_EINVAL, "a parameter array is NULL");
  double spi = 0.0;
  for (int i = 0; i < g; ++i) {
    if (!(P->pi[i] > 0.0) || !isfinite(P->pi[i])) return fail(c, CFUST_EINVAL, "pi_i must be > 0");
    spi += P->pi[i];
    // +inf is the skew-normal limit (kept by the M-step)
    if (!(P->nu[i] > 0.0)) return fail(c, CFUST_EINVAL, "nu_i must be > 0 (or +inf)");
    for (int a = 0; a < p; ++a)
      if (!isfinite(P->mu[i * p + a])) return fail(c, CFUST_EINVAL, "mu not finite");
    for (int a = 0; a < p * r; ++a)
      if (!isfinite(P->Delta[(size_t)i * p * r + a])) return fail(c, CFUST_EINVAL, "Delta not finite");
    const double *S = P->Sigma + (size_t)i * p * p;
    double L[CFUST_PMAX * CFUST_PMAX];
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b) {
        const double v = S[a * p + b], w = S[b * p + a];
        if (!isfinite(v)) return fail(c, CFUST_EINVAL, "Sigma not finite");
        if (fabs(v - w) > 1e-12 * (fabs(v) + fabs(w)) + 1e-300)
          return fail(c, CFUST_EINVAL, "Sigma not symmetric");
      }
    for (int j = 0; j < p; ++j) {
      double s = S[j * p + j];
      for (int k = 0; k < j; ++k) s -= L[j * p + k] * L[j * p + k];
      if (!(s > 0.0)) return fail(c, CFUST_ENOTPD, "Sigma not positive definite");
      L[j * p + j] = sqrt(s);
      for (int i2 = j + 1; i2 < p; ++i2) {
        double t = S[i2 * p + j];
        for (int k = 0; k < j; ++k) t -= L[i2 * p + k] * L[j * p + k];
        L[i2 * p + j] = t / L[j * p + j];
      }
    }
  }
  if (fabs(spi - 1.0) > 1e-10) return fail(c, CFUST_EINVAL, "pi must sum to 1");
  return CFUST_OK;
}

cfust_status upload_params(cfust_ctx *c, const cfust_params *P) {
  const int g = P->g, p = P->p, r = P->r;
  ParamView v = param_view(c->d_params, g, p, r);
  CF_CUDA(c, cudaMemcpyAsync(v.pi, P->pi, sizeof(double) * g, cudaMemcpyHostToDevice, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(v.mu, P->mu, sizeof(double) * g * p, cudaMemcpyHostToDevice, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(v.Sigma, P->Sigma, sizeof(double) * g * p * p, cudaMemcpyHostToDevice,
                             c->stream));
  CF_CUDA(c, cudaMemcpyAsync(v.Delta, P->Delta, sizeof(double) * g * p * r, cudaMemcpyHostToDevice,
                             c->stream));
  CF_CUDA(c, cudaMemcpyAsync(v.nu, P->nu, sizeof(double) * g, cudaMemcpyHostToDevice, c->stream));
  return CFUST_OK;
}

cfust_status download_params(cfust_ctx *c, cfust_params *P) {
  const int g = P->g, p = P->p, r = P->r;
  ParamView v = param_view(c->d_params, g, p, r);
  CF_CUDA(c, cudaMemcpyAsync(P->pi, v.pi, sizeof(double) * g, cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(P->mu, v.mu, sizeof(double) * g * p, cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(P->Sigma, v.Sigma, sizeof(double) * g * p * p, cudaMemcpyDeviceToHost,
                             c->stream));
  CF_CUDA(c, cudaMemcpyAsync(P->Delta, v.Delta, sizeof(double) * g * p * r, cudaMemcpyDeviceToHost,
                             c->stream));
  CF_CUDA(c, cudaMemcpyAsync(P->nu, v.nu, sizeof(double) * g, cudaMemcpyDeviceToHost, c->stream));
  return CFUST_OK;
}

cfust_status status_from_bits(cfust_ctx *c, int bits) {
  if (bits == 0) return CFUST_OK;
  if (bits & ERR_TIMEOUT) return fail(c, CFUST_ETIMEOUT, "a bounded device wait ran out");
  if (bits & ERR_NOTPD_OMEGA) return fail(c, CFUST_ENOTPD, "Omega = Sigma + Delta Delta^T not positive definite");
  if (bits & ERR_NOTPD_LAMBDA) return fail(c, CFUST_ENOTPD, "Lambda = I - Delta^T Omega^-1 Delta not positive definite");
  if (bits & ERR_NOTPD_S6) return fail(c, CFUST_ENOTPD, "sum of tau e4 not positive definite");
  if (bits & ERR_NOTPD_SIGMA) return fail(c, CFUST_ENOTPD, "updated Sigma not positive definite");
  if (bits & ERR_DEGENERATE) return fail(c, CFUST_EDEGENERATE, "a component lost its posterior weight");
  if (bits & ERR_ZERO_DENSITY) return fail(c, CFUST_ENUMERIC, "an observation has zero density under every component");
  if (bits & ERR_BAD_LABEL) return fail(c, CFUST_EINVAL, "a partition label is outside 0..g-1");
  if (bits & ERR_INIT_GROUP)
    return fail(c, CFUST_EDEGENERATE, "a partition group has fewer than p + 1 members or a singular covariance");
  return fail(c, CFUST_ENUMERIC, "non-finite value in the E-step");
}

// Read the status word (synchronises) and the rescue count.
cfust_status finish(cfust_ctx *c) {
  int bits = 0;
  CF_CUDA(c, cudaMemcpyAsync(&bits, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  return status_from_bits(c, bits);
}

cfust_status check_common(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P) {
  if (!c) return CFUST_EINVAL;
  if (!Y) return fail(c, CFUST_EINVAL, "Y is NULL");
  if (n < 1) return fail(c, CFUST_EINVAL, "n must be >= 1");
  if ((uint64_t)n >= (1ull << 32) || (uint64_t)n * (uint64_t)(P ? P->g : 1) >= (1ull << 40))
    return fail(c, CFUST_EINVAL, "n too large (n < 2^32, n g < 2^40)");
  if (reinterpret_cast<uintptr_t>(Y) % 8 != 0) return fail(c, CFUST_EINVAL, "Y must be 8-byte aligned");
  return check_params(c, P);
}

EstepOut ctx_out(cfust_ctx *c) {
  EstepOut o;
  o.logf = c->d_logf;
  o.e1 = c->d_e1;
  o.e2 = c->d_e2;
  o.e3 = c->d_e3;
  o.e4 = c->d_e4;
  return o;
}

PosteriorArgs post_args(cfust_ctx *c, const double *Y, int64_t n) {
  PosteriorArgs a{};
  a.Y = Y;
  a.n = n;
  a.g = c->g;
  a.p = c->p;
  a.r = c->r;
  a.pi = param_view(c->d_params, c->g, c->p, c->r).pi;
  a.partials = c->d_partials;
  a.ll_partials = c->d_llpart;
  a.d_status = c->d_status;
  a.nblocks = posterior_nblocks(n);
  return a;
}

double nu_lo(const cfust_ctx *c) { return c->opts.nu_min > 0 ? c->opts.nu_min : 1.0; }
double nu_hi(const cfust_ctx *c) { return c->opts.nu_max > 0 ? c->opts.nu_max : 200.0; }

SweepTiming sweep_timing(cfust_ctx *c, bool capturing) {
  SweepTiming tm;
  if (c->opts.timing && c->ev_sweep[0]) {
    tm.start = c->ev_sweep[0];
    tm.stop = c->ev_sweep[1];
    tm.capturing = capturing;
    c->sweep_recorded = true;
  }
  return tm;
}

// The E-step sweep for all pairs: the lattice rule, or with a surrogate
// attached the network for in-domain pairs and the lattice rule for the list
// of the others.  The timing events bracket the dominant kernel.
cfust_status run_estep(cfust_ctx *c, const double *Y, int64_t n, EstepOut o, bool density_only,
                       cudaStream_t st, SweepTiming tm, int triage) {
  const double *pi = param_view(c->d_params, c->g, c->p, c->r).pi;
  if (!c->sur) {
    CF_CUDA(c, launch_estep(c->opts.precision, Y, n, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32,
                            c->d_chi64, c->d_chi32, o, density_only, c->opts.e2_mode, c->d_rescue,
                            c->d_rescue_cnt, c->d_status, c->opts.pairs_per_warp, st, tm, triage, pi,
                            (float)c->opts.triage_nats, c->opts.prioritise, c->opts.shared_points));
    return CFUST_OK;
  }
  if (c->opts.precision != CFUST_FP32 || c->opts.e2_mode != 0 || c->r != 3)
    return fail(c, CFUST_EINVAL, "the surrogate E-step needs CFUST_FP32, e2_mode 0 and r = 3");
  const unsigned evflag = tm.capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (tm.start) CF_CUDA(c, cudaEventRecordWithFlags(tm.start, st, evflag));
  CF_CUDA(c, launch_surrogate_estep(surrogate_dev(c->sur), Y, n, c->g, c->p, c->d_c32, o, density_only,
                                    c->d_fb, c->d_fb_cnt, c->d_status, st));
  if (tm.stop) CF_CUDA(c, cudaEventRecordWithFlags(tm.stop, st, evflag));
  CF_CUDA(c, launch_estep_list(Y, n, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64, c->d_chi32, o,
                               density_only, c->opts.e2_mode, c->d_fb, c->d_fb_cnt, c->d_rescue,
                               c->d_rescue_cnt, c->d_status, st, triage, pi, (float)c->opts.triage_nats,
                               c->opts.prioritise, c->opts.shared_points));
  return CFUST_OK;
}

// The fused E-step + sums launch (density_only: the log-likelihood partials
// only); *nb receives the number of partial rows it writes.
cfust_status enqueue_fused(cfust_ctx *c, const double *Y, int64_t n, bool density_only, cudaStream_t st,
                           SweepTiming tm, int *nb) {
  if (c->sur)
    return fail(c, CFUST_EINVAL, "the fused pass covers the lattice rule: detach the surrogate or set fused = 0");
  const double *pi = param_view(c->d_params, c->g, c->p, c->r).pi;
  CF_CUDA(c, launch_fused(c->opts.precision, Y, n, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64,
                          c->d_chi32, density_only, c->opts.e2_mode, c->d_status, c->d_rescue_cnt,
                          c->opts.pairs_per_warp, c->d_partials, c->d_llpart, pi, (float)c->opts.triage_nats,
                          c->opts.prioritise, c->opts.shared_points, st, tm, nb));
  return CFUST_OK;
}

// One EM iteration on the stream: E-step at the device parameters (yielding
// their log-likelihood into trace[iter]), then the M-step in place.
cfust_status enqueue_iteration(cfust_ctx *c, const double *Y, int64_t n, cudaStream_t st) {
  CF_CUDA(c, launch_precompute(c->d_params, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64,
                               c->d_chi32, c->d_status, st));
  if (c->opts.fused) {
    // one kernel for the E-step and the sums; the timing events bracket it
    int nb = 0;
    cfust_status s = enqueue_fused(c, Y, n, false, st, sweep_timing(c, st == c->cap_stream), &nb);
    if (s != CFUST_OK) return s;
    CF_CUDA(c, launch_reduce_ll(c->d_llpart, nb, c->d_ll, c->d_trace, c->d_status + 1, st));
    CF_CUDA(c, launch_mstep_finalize(c->d_partials, nb, c->g, c->p, c->r, n, nu_lo(c), nu_hi(c), c->d_params,
                                     c->d_status, st));
    return CFUST_OK;
  }
  cfust_status s = run_estep(c, Y, n, ctx_out(c), false, st, sweep_timing(c, st == c->cap_stream), 1);
  if (s != CFUST_OK) return s;
  PosteriorArgs a = post_args(c, Y, n);
  a.logf = c->d_logf;
  a.e1 = c->d_e1;
  a.e2 = c->d_e2;
  a.e3 = c->d_e3;
  a.e4 = c->d_e4;
  a.want_sums = true;
  a.want_ll = true;
  const bool tpost = c->opts.timing && c->ev_post[0];
  const unsigned evflag = (st == c->cap_stream) ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (tpost) CF_CUDA(c, cudaEventRecordWithFlags(c->ev_post[0], st, evflag));
  CF_CUDA(c, launch_posterior(c->opts.precision, a, st));
  if (tpost) {
    CF_CUDA(c, cudaEventRecordWithFlags(c->ev_post[1], st, evflag));
    c->post_recorded = true;
  }
  CF_CUDA(c, launch_reduce_ll(c->d_llpart, a.nblocks, c->d_ll, c->d_trace, c->d_status + 1, st));
  CF_CUDA(c, launch_mstep_finalize(c->d_partials, a.nblocks, c->g, c->p, c->r, n, nu_lo(c), nu_hi(c),
                                   c->d_params, c->d_status, st));
  return CFUST_OK;
}

// Density-only pass: log-likelihood of the device parameters into *d_ll
// (and trace[iter] when trace is set).
cfust_status enqueue_loglik(cfust_ctx *c, const double *Y, int64_t n, double *trace) {
  CF_CUDA(c, launch_precompute(c->d_params, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64,
                               c->d_chi32, c->d_status, c->stream));
  if (c->opts.fused) {
    int nb = 0;
    cfust_status s = enqueue_fused(c, Y, n, true, c->stream, sweep_timing(c, false), &nb);
    if (s != CFUST_OK) return s;
    CF_CUDA(c, launch_reduce_ll(c->d_llpart, nb, c->d_ll, trace, c->d_status + 1, c->stream));
    return CFUST_OK;
  }
  EstepOut o{};
  o.logf = c->d_logf;
  cfust_status s = run_estep(c, Y, n, o, true, c->stream, sweep_timing(c, false), 1);
  if (s != CFUST_OK) return s;
  PosteriorArgs a = post_args(c, Y, n);
  a.logf = c->d_logf;
  a.want_ll = true;
  CF_CUDA(c, launch_posterior(c->opts.precision, a, c->stream));
  CF_CUDA(c, launch_reduce_ll(c->d_llpart, a.nblocks, c->d_ll, trace, c->d_status + 1, c->stream));
  return CFUST_OK;
}

}  // namespace

extern "C" {

cfust_status cfust_create(cfust_ctx **out, const cfust_opts *o, void *cuda_stream) {
  g_create_error.clear();
  if (!out || !o) {
    g_create_error = "ctx or opts is NULL";
    return CFUST_EINVAL;
  }
  *out = nullptr;
  const cfust_lattice &L = o->lattice;
  if (o->precision != CFUST_FP64 && o->precision != CFUST_FP32) {
    g_create_error = "precision must be CFUST_FP64 or CFUST_FP32";
    return CFUST_EINVAL;
  }
  if (L.n < 32 || L.n > CFUST_NMAX || L.n % 32 != 0) {
    g_create_error = "lattice points must be a multiple of 32 in [32, CFUST_NMAX]";
    return CFUST_EINVAL;
  }
  if (L.dim < 2 || L.dim > CFUST_RMAX + 1 || !L.z || !L.shift) {
    g_create_error = "lattice dim must be in [2, CFUST_RMAX + 1] with z and shift given";
    return CFUST_EINVAL;
  }
  if (o->e2_mode != 0 && o->e2_mode != 1) {
    g_create_error = "e2_mode must be 0 or 1";
    return CFUST_EINVAL;
  }
  if (o->pairs_per_warp < 0 || o->pairs_per_warp > 32) {
    g_create_error = "pairs_per_warp must be in [0, 32]";
    return CFUST_EINVAL;
  }
  if (o->max_iter < 0 || !(o->tol >= 0.0)) {
    g_create_error = "max_iter must be >= 0 and tol >= 0";
    return CFUST_EINVAL;
  }
  if ((o->nu_min != 0.0 || o->nu_max != 0.0) && !(o->nu_min > 0.0 && o->nu_max > o->nu_min)) {
    g_create_error = "need 0 < nu_min < nu_max";
    return CFUST_EINVAL;
  }
  if (o->prioritise != 0 && o->prioritise != 1) {
    g_create_error = "prioritise must be 0 or 1";
    return CFUST_EINVAL;
  }
  if (o->triage_nats != 0.0 && !(o->triage_nats >= 1.0 && o->triage_nats <= 700.0)) {
    g_create_error = "triage_nats must be 0 (default 30) or in [1, 700]";
    return CFUST_EINVAL;
  }
  if (o->test_wait_polls < -1) {
    g_create_error = "test_wait_polls must be -1, 0 or positive";
    return CFUST_EINVAL;
  }
  if (o->fused != 0 && o->fused != 1) {
    g_create_error = "fused must be 0 or 1";
    return CFUST_EINVAL;
  }
  if (o->shared_points != 0 && o->shared_points != 1) {
    g_create_error = "shared_points must be 0 or 1";
    return CFUST_EINVAL;
  }
  cfust_ctx *c = new cfust_ctx();
  c->opts = *o;
  c->lat.wait_polls = o->test_wait_polls == 0 ? (1 << 22) : (o->test_wait_polls < 0 ? 0 : o->test_wait_polls);
  c->opts.lattice.z = nullptr;
  c->opts.lattice.shift = nullptr;
  if (c->opts.triage_nats == 0.0) c->opts.triage_nats = 30.0;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    g_create_error = "no CUDA device";
    delete c;
    return CFUST_ECUDA;
  }
  if (o->timing) {
    if (cudaEventCreate(&c->ev_sweep[0]) != cudaSuccess || cudaEventCreate(&c->ev_sweep[1]) != cudaSuccess ||
        cudaEventCreate(&c->ev_post[0]) != cudaSuccess || cudaEventCreate(&c->ev_post[1]) != cudaSuccess) {
      g_create_error = "cudaEventCreate failed";
      delete c;
      return CFUST_ECUDA;
    }
  }
  c->lat.n = L.n;
  for (int t = 0; t <= CFUST_RMAX; ++t) {
    if (t < L.dim) {
      if (!(L.shift[t] >= 0.0 && L.shift[t] < 1.0)) {
        g_create_error = "lattice shift must lie in [0, 1)";
        delete c;
        return CFUST_EINVAL;
      }
      int64_t zz = L.z[t] % L.n;
      if (zz < 0) zz += L.n;
      c->lat.z[t] = (int)zz;
      c->lat.step[t] = (int)((32 * zz) % L.n);
      c->lat.shift[t] = L.shift[t];
      const double sn = L.shift[t] * (double)L.n;
      c->lat.sint[t] = (int)floor(sn);
      c->lat.sfrac[t] = sn - floor(sn);
    } else {
      c->lat.z[t] = 0;
      c->lat.step[t] = 0;
      c->lat.shift[t] = 0.0;
      c->lat.sint[t] = 0;
      c->lat.sfrac[t] = 0.0;
    }
  }
  {
    const int r = L.dim - 1;
    float *tab = nullptr;
    if (cudaMalloc(&tab, sizeof(float) * (size_t)uniform_table_floats(L.n, r)) != cudaSuccess) {
      g_create_error = "cudaMalloc of the lattice table failed";
      cfust_destroy(c);
      return CFUST_ENOMEM;
    }
    c->d_utab = tab;
    c->lat.utab = tab;
    c->lat.utab2 = tab + (size_t)L.n * uniform_stride(r);
    if (launch_uniform_table(c->lat, r, tab, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      g_create_error = "building the lattice table failed";
      cfust_destroy(c);
      return CFUST_ECUDA;
    }
  }
  *out = c;
  return CFUST_OK;
}

cfust_status cfust_destroy(cfust_ctx *c) {
  if (!c) return CFUST_OK;
  DeviceGuard dg(c->device);
  drop_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  free_batch(c->batch);
  for (cudaEvent_t ev : c->ev_post)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c->ev_sweep)
    if (ev) cudaEventDestroy(ev);
  void *bufs[] = {c->d_params, c->d_c64, c->d_c32, c->d_chi64, c->d_chi32, c->d_status,
                  c->d_rescue_cnt, c->d_ll, c->d_trace, c->d_rescue, c->d_partials, c->d_llpart,
                  c->d_logf, c->d_e1, c->d_e2, c->d_e3, c->d_e4, c->d_fb, c->d_fb_cnt, c->d_utab,
                  c->d_prob_cnt, c->d_sums};
  for (void *b : bufs)
    if (b) cudaFree(b);
  delete c;
  return CFUST_OK;
}

const char *cfust_last_error(cfust_ctx *c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

cfust_status cfust_set_surrogate(cfust_ctx *c, cfust_surrogate *s) {
  if (!c) return CFUST_EINVAL;
  DeviceGuard dg(c->device);
  drop_graph(c);
  c->sur = s;
  c->fb_cap = 0;  // (re)allocated by the next call that knows n
  return CFUST_OK;
}

cfust_status cfust_surrogate_problems(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P,
                                      int64_t stride, float *x_out, int64_t max_rows, int64_t *rows) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  if (P->r != 3) return fail(c, CFUST_EINVAL, "the surrogate's problems need r = 3");
  if (stride < 1 || max_rows < 0 || !rows || (max_rows > 0 && !x_out))
    return fail(c, CFUST_EINVAL, "stride >= 1, max_rows >= 0, rows and x_out required");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  if (!c->d_prob_cnt) CF_CUDA(c, cudaMalloc(&c->d_prob_cnt, sizeof(unsigned long long)));
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  CF_CUDA(c, launch_precompute(c->d_params, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64,
                               c->d_chi32, c->d_status, c->stream));
  CF_CUDA(c, launch_surrogate_problems(Y, n, c->g, c->p, c->d_c32, stride, x_out, max_rows, c->d_prob_cnt,
                                       c->stream));
  unsigned long long cnt = 0;
  CF_CUDA(c, cudaMemcpyAsync(&cnt, c->d_prob_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  if ((s = finish(c)) != CFUST_OK) return s;
  *rows = (int64_t)cnt < max_rows ? (int64_t)cnt : max_rows;
  return CFUST_OK;
}

cfust_status cfust_surrogate_inputs(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P, float *x_out,
                                    int32_t *kind) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  if (P->r != 3) return fail(c, CFUST_EINVAL, "the surrogate's inputs need r = 3");
  if (!x_out || !kind) return fail(c, CFUST_EINVAL, "x_out and kind required");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  CF_CUDA(c, launch_precompute(c->d_params, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64,
                               c->d_chi32, c->d_status, c->stream));
  CF_CUDA(c, launch_surrogate_inputs(Y, n, c->g, c->p, c->d_c32, x_out, kind, c->stream));
  return finish(c);
}

cfust_status cfust_last_fallback(cfust_ctx *c, int64_t *count) {
  if (!c || !count) return CFUST_EINVAL;
  DeviceGuard dg(c->device);
  *count = 0;
  if (!c->sur || !c->d_fb_cnt || c->g < 1) return CFUST_OK;
  unsigned v[CFUST_GMAX];
  CF_CUDA(c, cudaMemcpyAsync(v, c->d_fb_cnt, sizeof(unsigned) * c->g, cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->g; ++i) *count += v[i];
  return CFUST_OK;
}

cfust_status cfust_last_rescued(cfust_ctx *c, int64_t *count) {
  if (!c || !count) return CFUST_EINVAL;
  DeviceGuard dg(c->device);
  if (!c->d_rescue_cnt) {
    *count = 0;
    return CFUST_OK;
  }
  unsigned v = 0;
  CF_CUDA(c, cudaMemcpyAsync(&v, c->d_rescue_cnt, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  *count = (c->opts.precision == CFUST_FP32) ? (int64_t)v : 0;
  return CFUST_OK;
}

cfust_status cfust_normal_f32(const float *x, float *out, int64_t n, int which, void *stream) {
  if (n < 0 || (n > 0 && (!x || !out)) || which < 0 || which > 5) return CFUST_EINVAL;
  if (launch_normal_f32(x, out, n, which, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return CFUST_ECUDA;
  return CFUST_OK;
}

cfust_status cfust_last_mstep_ms(cfust_ctx *c, float *ms) {
  if (!c || !ms) return CFUST_EINVAL;
  if (!c->opts.timing || !c->post_recorded) return fail(c, CFUST_EINVAL, "no timed M-step recorded");
  DeviceGuard dg(c->device);
  CF_CUDA(c, cudaEventSynchronize(c->ev_post[1]));
  CF_CUDA(c, cudaEventElapsedTime(ms, c->ev_post[0], c->ev_post[1]));
  return CFUST_OK;
}

cfust_status cfust_last_sweep_ms(cfust_ctx *c, float *ms) {
  if (!c || !ms) return CFUST_EINVAL;
  if (!c->opts.timing || !c->sweep_recorded) return fail(c, CFUST_EINVAL, "no timed sweep recorded");
  DeviceGuard dg(c->device);
  CF_CUDA(c, cudaEventSynchronize(c->ev_sweep[1]));
  CF_CUDA(c, cudaEventElapsedTime(ms, c->ev_sweep[0], c->ev_sweep[1]));
  return CFUST_OK;
}

cfust_status cfust_loglik(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P,
                          double *loglik) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  if (!loglik) return fail(c, CFUST_EINVAL, "loglik is NULL");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n, !c->opts.fused)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  if ((s = enqueue_loglik(c, Y, n, nullptr)) != CFUST_OK) return s;
  double ll = 0.0;
  CF_CUDA(c, cudaMemcpyAsync(&ll, c->d_ll, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if ((s = finish(c)) != CFUST_OK) return s;
  *loglik = ll;
  return CFUST_OK;
}

cfust_status cfust_estep(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P, void *logf,
                         void *tau, void *e1, void *e2, void *e3, void *e4, double *loglik) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  if (!tau || !e1 || !e2 || !e3 || !e4) return fail(c, CFUST_EINVAL, "an E-step output is NULL");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  CF_CUDA(c, launch_precompute(c->d_params, c->g, c->p, c->r, c->lat, c->d_c64, c->d_c32, c->d_chi64,
                               c->d_chi32, c->d_status, c->stream));
  EstepOut o;
  o.logf = logf ? logf : c->d_logf;
  o.e1 = e1;
  o.e2 = e2;
  o.e3 = e3;
  o.e4 = e4;
  if ((s = run_estep(c, Y, n, o, false, c->stream, sweep_timing(c, false), 0)) != CFUST_OK) return s;
  PosteriorArgs a = post_args(c, Y, n);
  a.logf = o.logf;
  a.tau_out = tau;
  a.want_ll = true;
  CF_CUDA(c, launch_posterior(c->opts.precision, a, c->stream));
  CF_CUDA(c, launch_reduce_ll(c->d_llpart, a.nblocks, c->d_ll, nullptr, nullptr, c->stream));
  double ll = 0.0;
  CF_CUDA(c, cudaMemcpyAsync(&ll, c->d_ll, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if ((s = finish(c)) != CFUST_OK) return s;
  if (loglik) *loglik = ll;
  return CFUST_OK;
}

cfust_status cfust_mstep(cfust_ctx *c, const double *Y, int64_t n, const void *tau, const void *e1,
                         const void *e2, const void *e3, const void *e4, cfust_params *P) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  if (!tau || !e1 || !e2 || !e3 || !e4) return fail(c, CFUST_EINVAL, "an E-step input is NULL");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  PosteriorArgs a = post_args(c, Y, n);
  a.tau_in = tau;
  a.e1 = e1;
  a.e2 = e2;
  a.e3 = e3;
  a.e4 = e4;
  a.want_sums = true;
  CF_CUDA(c, launch_posterior(c->opts.precision, a, c->stream));
  CF_CUDA(c, launch_mstep_finalize(c->d_partials, a.nblocks, c->g, c->p, c->r, n, nu_lo(c), nu_hi(c),
                                   c->d_params, c->d_status, c->stream));
  if ((s = finish(c)) != CFUST_OK) return s;
  if ((s = download_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  return CFUST_OK;
}

cfust_status cfust_mstep_sums(cfust_ctx *c, const double *Y, int64_t n, const void *tau, const void *e1,
                              const void *e2, const void *e3, const void *e4, const cfust_params *P,
                              double *sums) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  if (!tau || !e1 || !e2 || !e3 || !e4 || !sums) return fail(c, CFUST_EINVAL, "an input or sums is NULL");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  PosteriorArgs a = post_args(c, Y, n);
  a.tau_in = tau;
  a.e1 = e1;
  a.e2 = e2;
  a.e3 = e3;
  a.e4 = e4;
  a.want_sums = true;
  CF_CUDA(c, launch_posterior(c->opts.precision, a, c->stream));
  const int gK = c->g * sums_width(c->p, c->r);
  CF_CUDA(c, launch_sum_partials(c->d_partials, a.nblocks, gK, c->d_sums, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(sums, c->d_sums, sizeof(double) * gK, cudaMemcpyDeviceToHost, c->stream));
  return finish(c);
}

cfust_status cfust_mstep_apply(cfust_ctx *c, const double *sums, int64_t n_total, cfust_params *P) {
  if (!c) return CFUST_EINVAL;
  cfust_status s = check_params(c, P);
  if (s != CFUST_OK) return s;
  if (!sums || n_total < 1) return fail(c, CFUST_EINVAL, "sums must be given and n_total >= 1");
  const int gK = P->g * sums_width(P->p, P->r);
  for (int e = 0; e < gK; ++e)
    if (!isfinite(sums[e])) return fail(c, CFUST_ENUMERIC, "a sum is not finite");
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, 1)) != CFUST_OK) return s;
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  // the totals enter the finalize as the partials of a single block
  CF_CUDA(c, cudaMemcpyAsync(c->d_partials, sums, sizeof(double) * gK, cudaMemcpyHostToDevice, c->stream));
  CF_CUDA(c, launch_mstep_finalize(c->d_partials, 1, c->g, c->p, c->r, n_total, nu_lo(c), nu_hi(c), c->d_params,
                                   c->d_status, c->stream));
  if ((s = finish(c)) != CFUST_OK) return s;
  if ((s = download_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  return CFUST_OK;
}

cfust_status cfust_fit_begin(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P) {
  cfust_status s = check_common(c, Y, n, P);
  if (s != CFUST_OK) return s;
  DeviceGuard dg(c->device);
  if ((s = ensure(c, P->g, P->p, P->r, n, !c->opts.fused)) != CFUST_OK) return s;
  const int K = c->opts.max_iter;
  if (K + 1 > c->trace_cap) {
    CF_CUDA(c, realloc_dev(&c->d_trace, sizeof(double) * (K + 1)));
    c->trace_cap = K + 1;
    drop_graph(c);
  }
  if ((s = upload_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream));
  if (c->opts.use_graph && (c->graph_Y != Y || c->graph_n != n)) drop_graph(c);
  if (c->opts.use_graph && !c->gexec && K > 0) {
    cudaGraph_t gr = nullptr;
    if (!c->cap_stream) CF_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CF_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
    cfust_status cs = enqueue_iteration(c, Y, n, c->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &gr);
    if (cs != CFUST_OK) {
      if (gr) cudaGraphDestroy(gr);
      return cs;
    }
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&c->gexec, gr, 0);
    cudaGraphDestroy(gr);
    if (ce != cudaSuccess) {
      c->gexec = nullptr;
      return cuda_fail(c, ce, "cudaGraphInstantiate");
    }
    c->graph_Y = Y;
    c->graph_n = n;
  }
  c->fit_Y = Y;
  c->fit_n = n;
  c->fit_done = 0;
  c->fit_open = true;
  return CFUST_OK;
}

cfust_status cfust_fit_step(cfust_ctx *c, int iters) {
  if (!c) return CFUST_EINVAL;
  if (!c->fit_open) return fail(c, CFUST_EINVAL, "cfust_fit_begin has not been called");
  if (iters < 0 || c->fit_done + iters > c->opts.max_iter)
    return fail(c, CFUST_EINVAL, "more iterations than opts.max_iter");
  DeviceGuard dg(c->device);
  for (int k = 0; k < iters; ++k) {
    if (c->opts.use_graph) {
      CF_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    } else {
      cfust_status s = enqueue_iteration(c, c->fit_Y, c->fit_n, c->stream);
      if (s != CFUST_OK) return s;
    }
    ++c->fit_done;
  }
  return CFUST_OK;
}

cfust_status cfust_fit_trace(cfust_ctx *c, double *trace, int *count) {
  if (!c || !trace || !count) return CFUST_EINVAL;
  if (!c->fit_open) return fail(c, CFUST_EINVAL, "cfust_fit_begin has not been called");
  DeviceGuard dg(c->device);
  if (c->fit_done > 0)
    CF_CUDA(c, cudaMemcpyAsync(trace, c->d_trace, sizeof(double) * c->fit_done, cudaMemcpyDeviceToHost,
                               c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  *count = c->fit_done;
  return CFUST_OK;
}

cfust_status cfust_fit_end(cfust_ctx *c, cfust_params *P, double *trace, int *iters_done) {
  if (!c) return CFUST_EINVAL;
  if (!c->fit_open) return fail(c, CFUST_EINVAL, "cfust_fit_begin has not been called");
  if (!P || P->g != c->g || P->p != c->p || P->r != c->r)
    return fail(c, CFUST_EINVAL, "params shape differs from cfust_fit_begin");
  DeviceGuard dg(c->device);
  c->fit_open = false;
  cfust_status s;
  if ((s = enqueue_loglik(c, c->fit_Y, c->fit_n, c->d_trace)) != CFUST_OK) return s;
  if ((s = finish(c)) != CFUST_OK) return s;
  if (trace)
    CF_CUDA(c, cudaMemcpyAsync(trace, c->d_trace, sizeof(double) * (c->fit_done + 1),
                               cudaMemcpyDeviceToHost, c->stream));
  if ((s = download_params(c, P)) != CFUST_OK) return s;
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (iters_done) *iters_done = c->fit_done;
  return CFUST_OK;
}

cfust_status cfust_fit(cfust_ctx *c, const double *Y, int64_t n, cfust_params *P, double *trace,
                       int *iters_done) {
  cfust_status s = cfust_fit_begin(c, Y, n, P);
  if (s != CFUST_OK) return s;
  DeviceGuard dg(c->device);
  const int K = c->opts.max_iter;
  std::vector<double> hist;
  for (int k = 0; k < K; ++k) {
    if ((s = cfust_fit_step(c, 1)) != CFUST_OK) {
      c->fit_open = false;
      return s;
    }
    if (c->opts.tol > 0.0) {
      double lk = 0.0;
      CF_CUDA(c, cudaMemcpyAsync(&lk, c->d_trace + k, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      CF_CUDA(c, cudaStreamSynchronize(c->stream));
      hist.push_back(lk);
      const size_t m = hist.size();
      if (m >= 3) {
        // Algorithm 4 with the standard Aitken asymptote
        const double l2 = hist[m - 3], l1 = hist[m - 2], l0 = hist[m - 1];
        const double den = l1 - l2;
        bool stop = (den == 0.0);
        if (!stop) {
          const double acc = (l0 - l1) / den;
          if (acc != 1.0) {
            const double linf = l1 + (l0 - l1) / (1.0 - acc);
            stop = fabs(linf - l0) < c->opts.tol;
          }
        }
        if (stop) break;
      }
    }
  }
  return cfust_fit_end(c, P, trace, iters_done);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched fits
// ---------------------------------------------------------------------------

namespace {

void free_batch(cfust_ctx::Batch &b) {
  if (b.graph) cudaGraphExecDestroy(b.graph);
  b.graph = nullptr;
  void *bufs[] = {b.d_fits, b.d_comps, b.d_items, b.d_blocks, b.d_params, b.c64, b.c32, b.chi64, b.chi32,
                  b.logf, b.e1, b.e2, b.e3, b.e4, b.rescue, b.rescue_cnt, b.counter, b.partials, b.llpart,
                  b.trace, b.iter, b.fit_status, b.status};
  for (void *p : bufs)
    if (p) cudaFree(p);
  cfust_ctx::Batch fresh;
  fresh.tuned = b.tuned;
  fresh.ppw = b.ppw;
  fresh.cps = b.cps;
  b = fresh;
}

BatchDev batch_dev(const cfust_ctx::Batch &b) {
  BatchDev d;
  d.fits = b.d_fits;
  d.comps = b.d_comps;
  d.nfits = b.nfits;
  d.G = b.G;
  d.params = b.d_params;
  d.logf = b.logf;
  d.e1 = b.e1;
  d.e2 = b.e2;
  d.e3 = b.e3;
  d.e4 = b.e4;
  d.fit_status = b.fit_status;
  return d;
}

// Sweep items for a given pairs-per-warp: component by component, tiles of
// 8 warps x ppw observations.
std::vector<SweepItem> batch_items(const cfust_ctx::Batch &b, int ppw) {
  std::vector<SweepItem> items;
  const int64_t T = 8LL * ppw;
  for (int f = 0; f < b.nfits; ++f)
    for (int i = 0; i < b.g[f]; ++i) {
      int gc = 0;
      for (int h = 0; h < f; ++h) gc += b.g[h];
      gc += i;
      for (int64_t j0 = 0; j0 < b.n[f]; j0 += T) items.push_back(SweepItem{gc, (unsigned)j0});
    }
  return items;
}

int default_batch_ppw(int64_t pairs) {
  int64_t ppw = pairs / ((int64_t)sm_count() * 2 * 16 * 8);
  return (int)(ppw < 1 ? 1 : (ppw > 32 ? 32 : ppw));
}

cfust_status upload_items(cfust_ctx *c, int ppw) {
  cfust_ctx::Batch &b = c->batch;
  std::vector<SweepItem> items = batch_items(b, ppw);
  if (b.d_items) cudaFree(b.d_items);
  b.d_items = nullptr;
  CF_CUDA(c, cudaMalloc(&b.d_items, sizeof(SweepItem) * items.size()));
  CF_CUDA(c, cudaMemcpy(b.d_items, items.data(), sizeof(SweepItem) * items.size(), cudaMemcpyHostToDevice));
  b.nitems = (int)items.size();
  b.ppw = ppw;
  return CFUST_OK;
}

cfust_status enqueue_batch_estep(cfust_ctx *c, cudaStream_t st, bool density_only) {
  cfust_ctx::Batch &b = c->batch;
  const BatchDev d = batch_dev(b);
  CF_CUDA(c, launch_precompute_batched(d, b.p, b.r, c->lat, b.c64, b.c32, b.chi64, b.chi32, st));
  CF_CUDA(c, launch_estep_batched(c->opts.precision, d, b.p, b.r, c->lat, b.c64, b.c32, b.chi64, b.chi32,
                                  b.d_items, b.nitems, b.counter, density_only, c->opts.e2_mode, b.ppw, b.cps,
                                  b.rescue, b.rescue_cnt, b.status, 1, st,
                                  sweep_timing(c, st == c->cap_stream), c->opts.prioritise,
                                  c->opts.shared_points));
  return CFUST_OK;
}

cfust_status enqueue_batch_iteration(cfust_ctx *c, cudaStream_t st) {
  cfust_ctx::Batch &b = c->batch;
  cfust_status s = enqueue_batch_estep(c, st, false);
  if (s != CFUST_OK) return s;
  const BatchDev d = batch_dev(b);
  CF_CUDA(c, launch_posterior_batched(c->opts.precision, d, b.p, b.r, b.d_blocks, b.nblocks, b.partials, b.llpart,
                                      true, b.g_max, st));
  CF_CUDA(c, launch_reduce_ll_batched(d, b.llpart, b.trace, c->opts.max_iter + 1, b.iter, st));
  CF_CUDA(c, launch_finalize_batched(d, b.p, b.r, b.partials, nu_lo(c), nu_hi(c), st));
  return CFUST_OK;
}

// Time one sweep per candidate shape on the real batch; keep the fastest.
cfust_status autotune_batch(cfust_ctx *c) {
  cfust_ctx::Batch &b = c->batch;
  const int ppws[] = {2, 4, 8, 16};
  const int cpss[] = {1, 2};
  cudaEvent_t e0, e1;
  CF_CUDA(c, cudaEventCreate(&e0));
  CF_CUDA(c, cudaEventCreate(&e1));
  const BatchDev d = batch_dev(b);
  CF_CUDA(c, launch_precompute_batched(d, b.p, b.r, c->lat, b.c64, b.c32, b.chi64, b.chi32, c->stream));
  float best = 1e30f;
  int best_ppw = b.ppw, best_cps = b.cps;
  for (int ppw : ppws) {
    cfust_status s = upload_items(c, ppw);
    if (s != CFUST_OK) return s;
    for (int cps : cpss) {
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        CF_CUDA(c, cudaEventRecord(e0, c->stream));
        CF_CUDA(c, launch_estep_batched(c->opts.precision, d, b.p, b.r, c->lat, b.c64, b.c32, b.chi64, b.chi32,
                                        b.d_items, b.nitems, b.counter, false, c->opts.e2_mode, ppw, cps,
                                        b.rescue, b.rescue_cnt, b.status, 1, c->stream, SweepTiming(),
                                        c->opts.prioritise, c->opts.shared_points));
        CF_CUDA(c, cudaEventRecord(e1, c->stream));
        CF_CUDA(c, cudaEventSynchronize(e1));
        CF_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
      }
      if (ms < best) {
        best = ms;
        best_ppw = ppw;
        best_cps = cps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b.cps = best_cps;
  b.tuned = true;
  return upload_items(c, best_ppw);
}

}  // namespace

extern "C" cfust_status cfust_batched_shape(cfust_ctx *c, int *ppw, int *cps) {
  if (!c || !ppw || !cps) return CFUST_EINVAL;
  *ppw = c->batch.ppw;
  *cps = c->batch.cps;
  return CFUST_OK;
}

extern "C" cfust_status cfust_fit_batched(cfust_ctx *c, int nfits, const double *const *Y, const int64_t *n,
                                         cfust_params *P, double *trace_out, int *fit_status_out) {
  if (!c) return CFUST_EINVAL;
  if (nfits < 1 || !Y || !n || !P) return fail(c, CFUST_EINVAL, "nfits >= 1 with Y, n and params required");
  DeviceGuard dg(c->device);
  const int p = P[0].p, r = P[0].r;
  for (int f = 0; f < nfits; ++f) {
    cfust_status s = check_common(c, Y[f], n[f], &P[f]);
    if (s != CFUST_OK) return fail(c, s, "fit " + std::to_string(f) + ": " + c->err);
    if (P[f].p != p || P[f].r != r) return fail(c, CFUST_EINVAL, "all fits must share p and r");
  }
  const int K = c->opts.max_iter;
  const int kK = sums_width(p, r);
  cfust_ctx::Batch &b = c->batch;
  bool same = b.nfits == nfits && b.p == p && b.r == r && b.graph != nullptr;
  for (int f = 0; same && f < nfits; ++f) same = b.Y[f] == Y[f] && b.n[f] == n[f] && b.g[f] == P[f].g;
  if (!same) {
    free_batch(b);
    b.nfits = nfits;
    b.p = p;
    b.r = r;
    b.K = kK;
    b.Y.assign(Y, Y + nfits);
    b.n.assign(n, n + nfits);
    b.g.resize(nfits);
    std::vector<FitDesc> fits(nfits);
    std::vector<CompRef> comps;
    std::vector<BlockRef> blocks;
    int64_t pair_off = 0, param_off = 0, part_off = 0;
    int comp0 = 0, blk0 = 0;
    for (int f = 0; f < nfits; ++f) {
      const int g = P[f].g;
      b.g[f] = g;
      b.g_max = g > b.g_max ? g : b.g_max;
      const int nb = posterior_nblocks(n[f]);
      fits[f] = FitDesc{Y[f], n[f], g, comp0, pair_off, param_off, part_off, blk0, nb};
      for (int i = 0; i < g; ++i) comps.push_back(CompRef{f, i});
      for (int lb = 0; lb < nb; ++lb) blocks.push_back(BlockRef{f, lb});
      comp0 += g;
      pair_off += (int64_t)g * n[f];
      param_off += param_block_size(g, p, r);
      part_off += (int64_t)nb * g * kK;
      blk0 += nb;
    }
    if (b.g_max * kK > 2048) return fail(c, CFUST_EINVAL, "g x sums per component too large for batched fits");
    b.G = comp0;
    b.pairs = pair_off;
    b.params_len = param_off;
    b.part_len = part_off;
    b.nblocks = blk0;
    const size_t es = elem_size(c);
    const int rp = r * (r + 1) / 2;
    const int N = c->lat.n;
    CF_CUDA(c, cudaMalloc(&b.d_fits, sizeof(FitDesc) * nfits));
    CF_CUDA(c, cudaMalloc(&b.d_comps, sizeof(CompRef) * comps.size()));
    CF_CUDA(c, cudaMalloc(&b.d_blocks, sizeof(BlockRef) * blocks.size()));
    CF_CUDA(c, cudaMalloc(&b.d_params, sizeof(double) * b.params_len));
    CF_CUDA(c, cudaMalloc(&b.c64, sizeof(CompT<double>) * b.G));
    CF_CUDA(c, cudaMalloc(&b.c32, sizeof(CompT<float>) * b.G));
    CF_CUDA(c, cudaMalloc(&b.chi64, sizeof(double) * 2 * (size_t)N * b.G));
    CF_CUDA(c, cudaMalloc(&b.chi32, sizeof(float) * 2 * (size_t)N * b.G));
    CF_CUDA(c, cudaMalloc(&b.logf, es * b.pairs));
    CF_CUDA(c, cudaMalloc(&b.e1, es * b.pairs));
    CF_CUDA(c, cudaMalloc(&b.e2, es * b.pairs));
    CF_CUDA(c, cudaMalloc(&b.e3, es * b.pairs * r));
    CF_CUDA(c, cudaMalloc(&b.e4, es * b.pairs * rp));
    CF_CUDA(c, cudaMalloc(&b.rescue, sizeof(unsigned long long) * b.pairs));
    CF_CUDA(c, cudaMalloc(&b.rescue_cnt, sizeof(unsigned)));
    CF_CUDA(c, cudaMalloc(&b.counter, sizeof(unsigned)));
    CF_CUDA(c, cudaMalloc(&b.partials, sizeof(double) * b.part_len));
    CF_CUDA(c, cudaMalloc(&b.llpart, sizeof(double) * b.nblocks));
    CF_CUDA(c, cudaMalloc(&b.trace, sizeof(double) * (size_t)nfits * (K + 1)));
    CF_CUDA(c, cudaMalloc(&b.iter, sizeof(int)));
    CF_CUDA(c, cudaMalloc(&b.fit_status, sizeof(int) * nfits));
    CF_CUDA(c, cudaMalloc(&b.status, sizeof(int)));
    CF_CUDA(c, cudaMemcpy(b.d_fits, fits.data(), sizeof(FitDesc) * nfits, cudaMemcpyHostToDevice));
    CF_CUDA(c, cudaMemcpy(b.d_comps, comps.data(), sizeof(CompRef) * comps.size(), cudaMemcpyHostToDevice));
    CF_CUDA(c, cudaMemcpy(b.d_blocks, blocks.data(), sizeof(BlockRef) * blocks.size(), cudaMemcpyHostToDevice));
  }
  // parameters: one block per fit, back to back
  {
    std::vector<double> host(b.params_len);
    int64_t off = 0;
    for (int f = 0; f < nfits; ++f) {
      const cfust_params &q = P[f];
      const int g = q.g;
      double *dst = host.data() + off;
      ParamView v = param_view(dst, g, p, r);
      memcpy(v.pi, q.pi, sizeof(double) * g);
      memcpy(v.mu, q.mu, sizeof(double) * g * p);
      memcpy(v.Sigma, q.Sigma, sizeof(double) * g * p * p);
      memcpy(v.Delta, q.Delta, sizeof(double) * g * p * r);
      memcpy(v.nu, q.nu, sizeof(double) * g);
      off += param_block_size(g, p, r);
    }
    CF_CUDA(c, cudaMemcpyAsync(b.d_params, host.data(), sizeof(double) * b.params_len, cudaMemcpyHostToDevice,
                               c->stream));
    CF_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  CF_CUDA(c, cudaMemsetAsync(b.iter, 0, sizeof(int), c->stream));
  CF_CUDA(c, cudaMemsetAsync(b.fit_status, 0, sizeof(int) * nfits, c->stream));
  CF_CUDA(c, cudaMemsetAsync(b.status, 0, sizeof(int), c->stream));
  cfust_status s;
  if (!same) {
    if (c->opts.autotune && !b.tuned) {
      if ((s = autotune_batch(c)) != CFUST_OK) return s;
      CF_CUDA(c, cudaMemsetAsync(b.fit_status, 0, sizeof(int) * nfits, c->stream));
      CF_CUDA(c, cudaMemsetAsync(b.status, 0, sizeof(int), c->stream));
    } else if ((s = upload_items(c, b.tuned ? b.ppw : (c->opts.pairs_per_warp > 0 ? c->opts.pairs_per_warp
                                                                                   : default_batch_ppw(b.pairs)))) !=
               CFUST_OK) {
      return s;
    }
    if (K > 0) {
      cudaGraph_t gr = nullptr;
      if (!c->cap_stream) CF_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      CF_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
      cfust_status cs = enqueue_batch_iteration(c, c->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &gr);
      if (cs != CFUST_OK) {
        if (gr) cudaGraphDestroy(gr);
        return cs;
      }
      if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
      ce = cudaGraphInstantiate(&b.graph, gr, 0);
      cudaGraphDestroy(gr);
      if (ce != cudaSuccess) {
        b.graph = nullptr;
        return cuda_fail(c, ce, "cudaGraphInstantiate");
      }
    }
  }
  for (int k = 0; k < K; ++k) CF_CUDA(c, cudaGraphLaunch(b.graph, c->stream));
  // final density sweep: l(Psi^(K)) of every fit
  if ((s = enqueue_batch_estep(c, c->stream, true)) != CFUST_OK) return s;
  {
    const BatchDev d = batch_dev(b);
    CF_CUDA(c, launch_posterior_batched(c->opts.precision, d, p, r, b.d_blocks, b.nblocks, b.partials, b.llpart,
                                        false, b.g_max, c->stream));
    CF_CUDA(c, launch_reduce_ll_batched(d, b.llpart, b.trace, K + 1, b.iter, c->stream));
  }
  std::vector<int> fst(nfits);
  int bits = 0;
  CF_CUDA(c, cudaMemcpyAsync(fst.data(), b.fit_status, sizeof(int) * nfits, cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(&bits, b.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  std::vector<double> host(b.params_len);
  CF_CUDA(c, cudaMemcpyAsync(host.data(), b.d_params, sizeof(double) * b.params_len, cudaMemcpyDeviceToHost,
                             c->stream));
  if (trace_out)
    CF_CUDA(c, cudaMemcpyAsync(trace_out, b.trace, sizeof(double) * (size_t)nfits * (K + 1),
                               cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bits) return status_from_bits(c, bits);
  cfust_status first = CFUST_OK;
  int64_t off = 0;
  for (int f = 0; f < nfits; ++f) {
    const int g = P[f].g;
    cfust_status fs = fst[f] ? status_from_bits(c, fst[f]) : CFUST_OK;
    if (fit_status_out) fit_status_out[f] = fs;
    if (fs != CFUST_OK && first == CFUST_OK) {
      first = fs;
      c->err = "fit " + std::to_string(f) + ": " + c->err;
    }
    if (fs == CFUST_OK) {
      ParamView v = param_view(host.data() + off, g, p, r);
      memcpy(P[f].pi, v.pi, sizeof(double) * g);
      memcpy(P[f].mu, v.mu, sizeof(double) * g * p);
      memcpy(P[f].Sigma, v.Sigma, sizeof(double) * g * p * p);
      memcpy(P[f].Delta, v.Delta, sizeof(double) * g * p * r);
      memcpy(P[f].nu, v.nu, sizeof(double) * g);
    }
    off += param_block_size(g, p, r);
  }
  return first;
}

// ---------------------------------------------------------------------------
// M-step without allocation: scratch in a static device array.
// ---------------------------------------------------------------------------

namespace {

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CFUST_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {};  // per device ordinal, looked up on first use

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

cfust_status noalloc_fail(cfust_status s, const char *msg) {
  g_create_error = msg;
  return s;
}

}  // namespace

extern "C" cfust_status cfust_mstep_noalloc(int precision, const double *Y, int64_t n, const void *tau,
                                           const void *e1, const void *e2, const void *e3,
                                           const void *e4, double nu_min, double nu_max,
                                           cfust_params *P, void *cuda_stream) {
  g_create_error.clear();
  if (precision != CFUST_FP64 && precision != CFUST_FP32)
    return noalloc_fail(CFUST_EINVAL, "precision must be CFUST_FP64 or CFUST_FP32");
  if (!Y || !tau || !e1 || !e2 || !e3 || !e4 || !P || n < 1)
    return noalloc_fail(CFUST_EINVAL, "Y, tau, e1..e4 and params must be given and n >= 1");
  const int g = P->g, p = P->p, r = P->r;
  if (g < 1 || g > CFUST_GMAX || p < 1 || p > CFUST_PMAX || r < 1 || r > CFUST_RMAX)
    return noalloc_fail(CFUST_EINVAL, "g, p or r out of range");
  if (!P->pi || !P->mu || !P->Sigma || !P->Delta || !P->nu)
    return noalloc_fail(CFUST_EINVAL, "a parameter array is NULL");
  double spi = 0.0;
  for (int i = 0; i < g; ++i) {
    if (!(P->pi[i] > 0.0) || !(P->nu[i] > 0.0)) return noalloc_fail(CFUST_EINVAL, "pi_i and nu_i must be > 0");
    spi += P->pi[i];
  }
  if (fabs(spi - 1.0) > 1e-10) return noalloc_fail(CFUST_EINVAL, "pi must sum to 1");
  if ((nu_min != 0.0 || nu_max != 0.0) && !(nu_min > 0.0 && nu_max > nu_min))
    return noalloc_fail(CFUST_EINVAL, "need 0 < nu_min < nu_max");
  const double lo = nu_min > 0 ? nu_min : 1.0, hi = nu_max > 0 ? nu_max : 200.0;

  // layout: [status: 2 ints][parameter block][per-block partial sums]
  const size_t pbytes = sizeof(double) * (size_t)param_block_size(g, p, r);
  const size_t off_params = 256, off_part = off_params + round256(pbytes);
  const size_t per_block = sizeof(double) * (size_t)g * sums_width(p, r);
  if (off_part + CFUST_NOALLOC_MIN_BLOCKS * per_block > CFUST_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(CFUST_EINVAL,
                        "parameters plus CFUST_NOALLOC_MIN_BLOCKS blocks of partial sums exceed "
                        "CFUST_NOALLOC_SCRATCH_BYTES (1 MiB): g, p or r too large for cfust_mstep_noalloc");
  int nb = posterior_nblocks(n);
  const int cap = (int)((CFUST_NOALLOC_SCRATCH_BYTES - off_part) / per_block);
  if (nb > cap) nb = cap;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(CFUST_ECUDA, "no usable current CUDA device");
  // the inputs must live on the current device, where the scratch array is
  // looked up and the kernels run (a pointer query allocates nothing)
  {
    const void *ptrs[6] = {Y, tau, e1, e2, e3, e4};
    for (const void *q : ptrs) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(CFUST_EINVAL, "Y, tau and e1..e4 must be device memory of the current device");
      }
      if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
        return noalloc_fail(CFUST_EINVAL, "Y, tau and e1..e4 must be device memory of the current device");
    }
  }
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void *addr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) return noalloc_fail(CFUST_ECUDA, "cudaGetSymbolAddress failed");
      g_noalloc_addr[dev] = addr;
    }
    base = static_cast<unsigned char *>(g_noalloc_addr[dev]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int *d_status = reinterpret_cast<int *>(base);
  double *d_params = reinterpret_cast<double *>(base + off_params);
  double *d_part = reinterpret_cast<double *>(base + off_part);
  ParamView v = param_view(d_params, g, p, r);

#define NA_CUDA(call)                                                   \
  do {                                                                  \
    if ((call) != cudaSuccess) return noalloc_fail(CFUST_ECUDA, #call); \
  } while (0)
  NA_CUDA(cudaMemsetAsync(d_status, 0, 2 * sizeof(int), st));
  NA_CUDA(cudaMemcpyAsync(v.pi, P->pi, sizeof(double) * g, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(v.mu, P->mu, sizeof(double) * g * p, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(v.Sigma, P->Sigma, sizeof(double) * g * p * p, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(v.Delta, P->Delta, sizeof(double) * g * p * r, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(v.nu, P->nu, sizeof(double) * g, cudaMemcpyHostToDevice, st));
  PosteriorArgs pa{};
  pa.Y = Y;
  pa.n = n;
  pa.g = g;
  pa.p = p;
  pa.r = r;
  pa.pi = v.pi;
  pa.tau_in = tau;
  pa.e1 = e1;
  pa.e2 = e2;
  pa.e3 = e3;
  pa.e4 = e4;
  pa.want_sums = true;
  pa.partials = d_part;
  pa.d_status = d_status;
  pa.nblocks = nb;
  NA_CUDA(launch_posterior(precision, pa, st));
  NA_CUDA(launch_mstep_finalize(d_part, nb, g, p, r, n, lo, hi, d_params, d_status, st));
  int bits = 0;
  NA_CUDA(cudaMemcpyAsync(&bits, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  if (bits != 0) {
    if (bits & (ERR_NOTPD_S6 | ERR_NOTPD_SIGMA)) return noalloc_fail(CFUST_ENOTPD, "S6 or the updated Sigma not positive definite");
    if (bits & ERR_DEGENERATE) return noalloc_fail(CFUST_EDEGENERATE, "a component lost its posterior weight");
    return noalloc_fail(CFUST_ENUMERIC, "non-finite value in the M-step");
  }
  NA_CUDA(cudaMemcpyAsync(P->pi, v.pi, sizeof(double) * g, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaMemcpyAsync(P->mu, v.mu, sizeof(double) * g * p, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaMemcpyAsync(P->Sigma, v.Sigma, sizeof(double) * g * p * p, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaMemcpyAsync(P->Delta, v.Delta, sizeof(double) * g * p * r, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaMemcpyAsync(P->nu, v.nu, sizeof(double) * g, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
  return CFUST_OK;
}

extern "C" cfust_status cfust_fit_multistart(cfust_ctx *c, const double *Y, int64_t n, cfust_params *starts,
                                            int nstarts, int burn_in, int *best, double *trace, int *iters_done) {
  if (!c) return CFUST_EINVAL;
  if (nstarts < 1 || !starts || !best || burn_in < 0)
    return fail(c, CFUST_EINVAL, "nstarts >= 1, burn_in >= 0, starts and best required");
  DeviceGuard dg(c->device);
  int chosen = 0;
  if (nstarts > 1) {
    double best_ll = -INFINITY;
    chosen = -1;
    if (burn_in == 0) {
      // select on the starts' own log-likelihoods
      for (int f = 0; f < nstarts; ++f) {
        double ll = -INFINITY;
        const cfust_status s = cfust_loglik(c, Y, n, &starts[f], &ll);
        if (s == CFUST_OK && isfinite(ll) && ll > best_ll) {
          best_ll = ll;
          chosen = f;
        }
      }
    } else {
      // every start's burn-in as one batched fit over the same observations
      std::vector<const double *> Ys(nstarts, Y);
      std::vector<int64_t> ns(nstarts, n);
      std::vector<double> tr((size_t)nstarts * (burn_in + 1));
      std::vector<int> st(nstarts, 0);
      const int keep = c->opts.max_iter;
      c->opts.max_iter = burn_in;
      free_batch(c->batch);
      const cfust_status s = cfust_fit_batched(c, nstarts, Ys.data(), ns.data(), starts, tr.data(), st.data());
      free_batch(c->batch);
      c->opts.max_iter = keep;
      // a start that degenerates (its own status) is only left out
      if (s != CFUST_OK && s != CFUST_ENOTPD && s != CFUST_ENUMERIC && s != CFUST_EDEGENERATE) return s;
      for (int f = 0; f < nstarts; ++f) {
        const double ll = tr[(size_t)f * (burn_in + 1) + burn_in];
        if (st[f] == 0 && isfinite(ll) && ll > best_ll) {
          best_ll = ll;
          chosen = f;
        }
      }
    }
    if (chosen < 0) return fail(c, CFUST_EDEGENERATE, "no start gave a finite log-likelihood");
  }
  *best = chosen;
  return cfust_fit(c, Y, n, &starts[chosen], trace, iters_done);
}

// ---------------------------------------------------------------------------
// Initial values of Algorithm 1: k-means partitions, Psi^(0) of a partition
// by moments, and the multi-start fit from partitions.
// ---------------------------------------------------------------------------

namespace {

// Device scratch of one initial-value call (freed on every return path).
struct InitScratch {
  double *partials = nullptr, *cm = nullptr, *counts = nullptr, *params = nullptr, *lam = nullptr;
  unsigned long long *changed = nullptr;
  int *status = nullptr;
  ~InitScratch() {
    cudaFree(partials);
    cudaFree(cm);
    cudaFree(counts);
    cudaFree(params);
    cudaFree(lam);
    cudaFree(changed);
    cudaFree(status);
  }
};

cfust_status check_init_shape(cfust_ctx *c, const double *Y, int64_t n, int g, int p) {
  if (!Y || n < 1) return fail(c, CFUST_EINVAL, "Y must be a device array with n >= 1 rows");
  if (g < 1 || g > CFUST_GMAX || p < 1 || p > CFUST_PMAX) return fail(c, CFUST_EINVAL, "g or p out of range");
  if (n > (int64_t)1 << 40) return fail(c, CFUST_EINVAL, "n too large");
  return CFUST_OK;
}

}  // namespace

extern "C" cfust_status cfust_kmeans(cfust_ctx *c, const double *Y, int64_t n, int p, int g, double *centers,
                                     int max_iter, int32_t *labels, int *iters_done) {
  if (!c) return CFUST_EINVAL;
  cfust_status s = check_init_shape(c, Y, n, g, p);
  if (s != CFUST_OK) return s;
  if (!centers || !labels || max_iter < 1) return fail(c, CFUST_EINVAL, "centers, labels and max_iter >= 1 required");
  DeviceGuard dg(c->device);
  const int nblk = group_sums_nblocks(n);
  const int W = group_sums_width(0, p);
  InitScratch sc;
  CF_CUDA(c, cudaMalloc(&sc.partials, sizeof(double) * nblk * g * W));
  CF_CUDA(c, cudaMalloc(&sc.cm, sizeof(double) * g * p));
  CF_CUDA(c, cudaMalloc(&sc.changed, sizeof(unsigned long long)));
  CF_CUDA(c, cudaMalloc(&sc.status, sizeof(int)));
  CF_CUDA(c, cudaMemcpyAsync(sc.cm, centers, sizeof(double) * g * p, cudaMemcpyHostToDevice, c->stream));
  CF_CUDA(c, cudaMemsetAsync(sc.status, 0, sizeof(int), c->stream));
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    unsigned long long changed = 0;
    CF_CUDA(c, cudaMemsetAsync(sc.changed, 0, sizeof(unsigned long long), c->stream));
    CF_CUDA(c, launch_group_sums(0, Y, n, p, g, labels, sc.cm, 1, it == 1, sc.partials, nblk, sc.changed,
                                 sc.status, c->stream));
    CF_CUDA(c, cudaMemcpyAsync(&changed, sc.changed, sizeof(changed), cudaMemcpyDeviceToHost, c->stream));
    CF_CUDA(c, cudaStreamSynchronize(c->stream));
    // an assignment that changed nothing leaves the centres at its groups' means
    if (changed == 0) break;
    CF_CUDA(c, launch_kmeans_update(sc.partials, nblk, g, p, sc.cm, c->stream));
  }
  if (it > max_iter) it = max_iter;
  CF_CUDA(c, cudaMemcpyAsync(centers, sc.cm, sizeof(double) * g * p, cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (iters_done) *iters_done = it;
  return CFUST_OK;
}

extern "C" cfust_status cfust_init_partition(cfust_ctx *c, const double *Y, int64_t n, const int32_t *labels,
                                             double nu0, double lam, cfust_params *P) {
  if (!c) return CFUST_EINVAL;
  if (!P || !P->pi || !P->mu || !P->Sigma || !P->Delta || !P->nu) return fail(c, CFUST_EINVAL, "params arrays required");
  cfust_status s = check_init_shape(c, Y, n, P->g, P->p);
  if (s != CFUST_OK) return s;
  if (P->r < 1 || P->r > CFUST_RMAX) return fail(c, CFUST_EINVAL, "r out of range");
  if (!labels) return fail(c, CFUST_EINVAL, "labels required");
  if (!(nu0 > 2.0) || !isfinite(nu0)) return fail(c, CFUST_EINVAL, "nu0 must exceed 2");
  if (!(lam >= 0.0) || !isfinite(lam)) return fail(c, CFUST_EINVAL, "lam must be finite and >= 0");
  const int g = P->g, p = P->p, r = P->r;
  DeviceGuard dg(c->device);
  const int nblk = group_sums_nblocks(n);
  const int W0 = group_sums_width(0, p), W1 = group_sums_width(1, p);
  InitScratch sc;
  CF_CUDA(c, cudaMalloc(&sc.partials, sizeof(double) * nblk * g * (W0 > W1 ? W0 : W1)));
  CF_CUDA(c, cudaMalloc(&sc.cm, sizeof(double) * g * p));
  CF_CUDA(c, cudaMalloc(&sc.counts, sizeof(double) * g));
  CF_CUDA(c, cudaMalloc(&sc.params, sizeof(double) * param_block_size(g, p, r)));
  CF_CUDA(c, cudaMalloc(&sc.status, sizeof(int)));
  CF_CUDA(c, cudaMemsetAsync(sc.status, 0, sizeof(int), c->stream));
  int32_t *lab = const_cast<int32_t *>(labels);  // read only when assign = 0
  CF_CUDA(c, launch_group_sums(0, Y, n, p, g, lab, nullptr, 0, 0, sc.partials, nblk, nullptr, sc.status, c->stream));
  CF_CUDA(c, launch_group_means(sc.partials, nblk, g, p, sc.cm, sc.counts, c->stream));
  CF_CUDA(c, launch_group_sums(1, Y, n, p, g, lab, sc.cm, 0, 0, sc.partials, nblk, nullptr, sc.status, c->stream));
  CF_CUDA(c, launch_moment_finalize(sc.partials, nblk, sc.counts, sc.cm, n, g, p, r, nu0, lam, sc.params, nullptr,
                                    sc.status, c->stream));
  int bits = 0;
  std::vector<double> host(param_block_size(g, p, r));
  CF_CUDA(c, cudaMemcpyAsync(&bits, sc.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CF_CUDA(c, cudaMemcpyAsync(host.data(), sc.params, sizeof(double) * host.size(), cudaMemcpyDeviceToHost,
                             c->stream));
  CF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bits) return status_from_bits(c, bits);
  ParamView v = param_view(host.data(), g, p, r);
  memcpy(P->pi, v.pi, sizeof(double) * g);
  memcpy(P->mu, v.mu, sizeof(double) * g * p);
  memcpy(P->Sigma, v.Sigma, sizeof(double) * g * p * p);
  memcpy(P->Delta, v.Delta, sizeof(double) * g * p * r);
  memcpy(P->nu, v.nu, sizeof(double) * g);
  return CFUST_OK;
}

extern "C" cfust_status cfust_multistart_partitions(cfust_ctx *c, const double *Y, int64_t n, const int32_t *labels,
                                                    int m, double nu0, double lam, int burn_in, cfust_params *starts,
                                                    int *best, double *trace, int *iters_done) {
  if (!c) return CFUST_EINVAL;
  if (m < 1 || !labels || !starts || !best) return fail(c, CFUST_EINVAL, "m >= 1, labels, starts and best required");
  std::vector<cfust_params> ok;
  std::vector<int> idx;
  for (int f = 0; f < m; ++f) {
    const cfust_status s = cfust_init_partition(c, Y, n, labels + (int64_t)f * n, nu0, lam, &starts[f]);
    if (s == CFUST_OK) {
      ok.push_back(starts[f]);
      idx.push_back(f);
    } else if (s != CFUST_EDEGENERATE) {
      return s;
    }
  }
  if (ok.empty()) return fail(c, CFUST_EDEGENERATE, "no partition gave initial values");
  int b = 0;
  const cfust_status s = cfust_fit_multistart(c, Y, n, ok.data(), (int)ok.size(), burn_in, &b, trace, iters_done);
  *best = (b >= 0 && b < (int)idx.size()) ? idx[b] : -1;
  return s;
}

// ---------------------------------------------------------------------------
// Randomised-shift error estimate of the lattice rule.
// ---------------------------------------------------------------------------

namespace {

void set_lattice_shift(LatticeDev &lat, int dim, const double *shift) {
  for (int t = 0; t < dim; ++t) {
    lat.shift[t] = shift[t];
    const double sn = shift[t] * (double)lat.n;
    lat.sint[t] = (int)floor(sn);
    lat.sfrac[t] = sn - floor(sn);
  }
}

}  // namespace

extern "C" cfust_status cfust_loglik_shifts(cfust_ctx *c, const double *Y, int64_t n, const cfust_params *P, int M,
                                            const double *shifts, double *loglik) {
  if (!c) return CFUST_EINVAL;
  if (M < 1 || !shifts || !loglik) return fail(c, CFUST_EINVAL, "M >= 1, shifts and loglik required");
  const int dim = c->opts.lattice.dim;
  for (int64_t k = 0; k < (int64_t)M * dim; ++k)
    if (!(shifts[k] >= 0.0 && shifts[k] < 1.0)) return fail(c, CFUST_EINVAL, "lattice shift must lie in [0, 1)");
  DeviceGuard dg(c->device);
  const LatticeDev saved = c->lat;
  cfust_status s = CFUST_OK;
  for (int m = 0; m < M && s == CFUST_OK; ++m) {
    set_lattice_shift(c->lat, dim, shifts + (int64_t)m * dim);
    if (launch_uniform_table(c->lat, dim - 1, c->d_utab, c->stream) != cudaSuccess) {
      s = fail(c, CFUST_ECUDA, "rebuilding the lattice table failed");
      break;
    }
    s = cfust_loglik(c, Y, n, P, &loglik[m]);
  }
  // the context's own rule again (graphs captured before hold its values)
  c->lat = saved;
  if (launch_uniform_table(c->lat, dim - 1, c->d_utab, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, CFUST_ECUDA, "restoring the lattice table failed");
  return s;
}

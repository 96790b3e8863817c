// Per-component precompute in double precision (one CUDA block column per
// component): the factorisations and constants of Eq. 2 and the chi-scale
// tables of the lattice rule.
//
// Omega = Sigma + Delta Delta^T; Lo = chol(Omega); A = Lo^{-1}; M = A Delta;
// Lambda = I - M^T M (= I - Delta^T Omega^{-1} Delta); L = chol(Lambda).
// Table entry k of pass A (dof m = nu + p) and pass B (dof m = nu + p + 2):
// s_k = sqrt(F^{-1}_{chi^2_m}(u_k0) / m), u_k0 the baker-transformed coordinate 0
// of lattice point k.
#include <math.h>

#include "cfust_internal.cuh"
#include "special.cuh"

namespace cfust {

namespace {

__device__ bool cholesky_lower(const double *S, int n, int ld, double *Lout, int ldl) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Lout[i * ldl + j] = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = S[j * ld + j];
    for (int k = 0; k < j; ++k) s -= Lout[j * ldl + k] * Lout[j * ldl + k];
    if (!(s > 0.0) || !isfinite(s)) return false;
    const double d = sqrt(s);
    Lout[j * ldl + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = S[i * ld + j];
      for (int k = 0; k < j; ++k) t -= Lout[i * ldl + k] * Lout[j * ldl + k];
      Lout[i * ldl + j] = t / d;
    }
  }
  return true;
}

__device__ inline double lattice_coord(int k, int z, int n, double shift) {
  const int64_t idx = ((int64_t)k * (int64_t)z) % n;
  double u = (double)idx / (double)n + shift;
  if (u >= 1.0) u -= 1.0;
  u = 1.0 - fabs(2.0 * u - 1.0);
  const double umin = 1.1102230246251565e-16;  // 2^-53
  return fmin(fmax(u, umin), 1.0 - umin);
}

// Component i of one fit (parameter block `params`): chi tables chi64/chi32
// ([2][N] each, this component's rows) by the threads of blocks bx = 0..nbx-1,
// and the factorisations into *o / *f by thread 0 of block nbx (a block of
// its own, so that the serial double-precision factorisation runs beside the
// tables' quantiles rather than after one of them).
__device__ void precompute_component(const double *params, int g, int p, int r, int i, const LatticeDev &lat,
                                     CompT<double> *o_out, CompT<float> *f_out, double *t64, float *t32,
                                     int *status, int bx, int nbx) {
  ParamView pv = param_view(const_cast<double *>(params), g, p, r);
  const double nu = pv.nu[i];
  const int N = lat.n;

  // chi-scale tables: [2][N], one quantile per thread (pass A rows, then pass B)
  for (int kk = bx * blockDim.x + threadIdx.x; bx < nbx && kk < 2 * N; kk += nbx * blockDim.x) {
    const int k = kk < N ? kk : kk - N;
    const double u0 = lattice_coord(k, lat.z[0], N, lat.shift[0]);
    const double m = nu + p + (kk < N ? 0.0 : 2.0);
    // nu = inf (the skew-normal limit): chi^2_m / m -> 1
    const double sc = isinf(nu) ? 1.0 : sqrt(2.0 * inc_gamma_inv(0.5 * m, u0) / m);
    t64[kk] = sc;
    t32[kk] = (float)sc;
  }

  if (bx != nbx || threadIdx.x != 0) return;

  const double *mu = pv.mu + (int64_t)i * p;
  const double *Sig = pv.Sigma + (int64_t)i * p * p;
  const double *Del = pv.Delta + (int64_t)i * p * r;

  double Om[PMAX * PMAX], Lo[PMAX * PMAX], A[PMAX * PMAX];
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      double s = Sig[a * p + b];
      for (int t = 0; t < r; ++t) s += Del[a * r + t] * Del[b * r + t];
      Om[a * PMAX + b] = s;
    }
  if (!cholesky_lower(Om, p, PMAX, Lo, PMAX)) {
    atomicOr(status, ERR_NOTPD_OMEGA);
    return;
  }
  double logdet = 0.0;
  for (int a = 0; a < p; ++a) logdet += 2.0 * log(Lo[a * PMAX + a]);
  // A = Lo^{-1} by forward substitution, one column at a time
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) A[a * PMAX + b] = 0.0;
  for (int col = 0; col < p; ++col) {
    for (int a = col; a < p; ++a) {
      double s = (a == col) ? 1.0 : 0.0;
      for (int k = col; k < a; ++k) s -= Lo[a * PMAX + k] * A[k * PMAX + col];
      A[a * PMAX + col] = s / Lo[a * PMAX + a];
    }
  }
  // M = A Delta (p x r); B = M^T; Lambda = I - M^T M
  double M[PMAX * RMAX], Lam[RMAX * RMAX], L[RMAX * RMAX];
  for (int a = 0; a < p; ++a)
    for (int t = 0; t < r; ++t) {
      double s = 0.0;
      for (int k = 0; k <= a; ++k) s += A[a * PMAX + k] * Del[k * r + t];
      M[a * RMAX + t] = s;
    }
  for (int t = 0; t < r; ++t)
    for (int h = 0; h < r; ++h) {
      double s = (t == h) ? 1.0 : 0.0;
      for (int a = 0; a < p; ++a) s -= M[a * RMAX + t] * M[a * RMAX + h];
      Lam[t * RMAX + h] = s;
    }
  for (int t = 0; t < r; ++t)
    for (int h = 0; h < t; ++h) {
      const double s = 0.5 * (Lam[t * RMAX + h] + Lam[h * RMAX + t]);
      Lam[t * RMAX + h] = Lam[h * RMAX + t] = s;
    }
  double lamd[RMAX], lamp[RMAX * (RMAX + 1) / 2];
  for (int t = 0; t < RMAX; ++t) lamd[t] = (t < r && Lam[t * RMAX + t] > 0.0) ? 1.0 / sqrt(Lam[t * RMAX + t]) : 0.0;
  for (int t = 0; t < RMAX; ++t)
    for (int h = 0; h <= t; ++h) lamp[t * (t + 1) / 2 + h] = (t < r) ? Lam[t * RMAX + h] : 0.0;
  if (!cholesky_lower(Lam, r, RMAX, L, RMAX)) {
    atomicOr(status, ERR_NOTPD_LAMBDA);
    return;
  }
  const double pi_c = 3.14159265358979323846;
  // log of 2^r times the normalising constant of t_p(.; mu, Omega, nu); at
  // nu = inf that of the normal density phi_p, (2 pi)^{-p/2} |Omega|^{-1/2}
  const double c0 = isinf(nu) ? r * 0.69314718055994530942 - 0.5 * p * log(2.0 * pi_c) - 0.5 * logdet
                              : r * 0.69314718055994530942 + lgamma(0.5 * (nu + p)) - lgamma(0.5 * nu) -
                                    0.5 * p * log(nu * pi_c) - 0.5 * logdet;

  CompT<double> &o = *o_out;
  CompT<float> &f = *f_out;
  for (int a = 0; a < PMAX; ++a) o.mu[a] = f.mu[a] = (a < p) ? mu[a] : 0.0;
  for (int a = 0; a < PMAX * PMAX; ++a) {
    const int row = a / PMAX, col = a % PMAX;
    o.A[a] = f.A[a] = (row < p && col <= row) ? A[row * PMAX + col] : 0.0;
  }
  for (int t = 0; t < RMAX; ++t)
    for (int a = 0; a < PMAX; ++a) o.B[t * PMAX + a] = f.B[t * PMAX + a] = (t < r && a < p) ? M[a * RMAX + t] : 0.0;
  for (int t = 0; t < RMAX; ++t) {
    for (int h = 0; h < RMAX; ++h) {
      const double v = (t < r && h <= t) ? L[t * RMAX + h] : 0.0;
      o.L[t * RMAX + h] = v;
      f.L[t * RMAX + h] = (float)v;
    }
    const double li = (t < r) ? 1.0 / L[t * RMAX + t] : 0.0;
    o.Linv[t] = li;
    f.Linv[t] = (float)li;
    o.lamd[t] = f.lamd[t] = lamd[t];
    for (int h = 0; h <= t; ++h) o.lam[t * (t + 1) / 2 + h] = f.lam[t * (t + 1) / 2 + h] = lamp[t * (t + 1) / 2 + h];
  }
  // psi((nu+p)/2) and log(nu+p) enter e2 only, which is 0 at nu = inf
  const double psiA = isinf(nu) ? 0.0 : digamma(0.5 * (nu + p));
  o.c0 = f.c0 = c0;
  o.nu = f.nu = nu;
  o.mA = f.mA = nu + p;
  o.mB = f.mB = nu + p + 2.0;
  o.psiA = f.psiA = psiA;
  o.logmA = f.logmA = isinf(nu) ? 0.0 : log(nu + p);
  for (int a = 0; a < PMAX; ++a) o.fmu[a] = f.fmu[a] = (float)o.mu[a];
  for (int a = 0; a < PMAX * PMAX; ++a) o.fA[a] = f.fA[a] = (float)o.A[a];
  for (int a = 0; a < RMAX * PMAX; ++a) o.fB[a] = f.fB[a] = (float)o.B[a];
  o.fc0 = f.fc0 = (float)c0;
  o.fnu = f.fnu = (float)nu;
  o.fmA = f.fmA = (float)(nu + p);
  o.fmB = f.fmB = (float)(nu + p + 2.0);
  o.fpsiA = f.fpsiA = (float)psiA;
}

__global__ void precompute_kernel(const double *params, int g, int p, int r, LatticeDev lat,
                                  CompT<double> *c64, CompT<float> *c32, double *chi64,
                                  float *chi32, int *status) {
  const int i = blockIdx.y;
  precompute_component(params, g, p, r, i, lat, c64 + i, c32 + i, chi64 + (int64_t)i * 2 * lat.n,
                       chi32 + (int64_t)i * 2 * lat.n, status, blockIdx.x, gridDim.x - 1);
}

__global__ void precompute_batched_kernel(BatchDev b, int p, int r, LatticeDev lat, CompT<double> *c64,
                                          CompT<float> *c32, double *chi64, float *chi32) {
  const int gc = blockIdx.y;
  const CompRef cr = b.comps[gc];
  const FitDesc fd = b.fits[cr.fit];
  precompute_component(b.params + fd.param_off, fd.g, p, r, cr.i, lat, c64 + gc, c32 + gc,
                       chi64 + (int64_t)gc * 2 * lat.n, chi32 + (int64_t)gc * 2 * lat.n, b.fit_status + cr.fit,
                       blockIdx.x, gridDim.x - 1);
}

}  // namespace

cudaError_t launch_precompute_batched(const BatchDev &b, int p, int r, const LatticeDev &lat,
                                      CompT<double> *c64, CompT<float> *c32, double *chi64, float *chi32,
                                      cudaStream_t st) {
  const int threads = 64;
  int bx = (2 * lat.n + threads - 1) / threads;
  if (bx < 1) bx = 1;
  // bx table blocks and one factorisation block per component
  precompute_batched_kernel<<<dim3(bx + 1, b.G), threads, 0, st>>>(b, p, r, lat, c64, c32, chi64, chi32);
  return cudaGetLastError();
}

cudaError_t launch_precompute(const double *d_params, int g, int p, int r, const LatticeDev &lat,
                              CompT<double> *c64, CompT<float> *c32, double *chi64, float *chi32,
                              int *d_status, cudaStream_t st) {
  const int threads = 64;
  int bx = (2 * lat.n + threads - 1) / threads;
  if (bx < 1) bx = 1;
  dim3 grid(bx + 1, g);  // bx table blocks and one factorisation block per component
  precompute_kernel<<<grid, threads, 0, st>>>(d_params, g, p, r, lat, c64, c32, chi64, chi32,
                                              d_status);
  return cudaGetLastError();
}

}  // namespace cfust

// Initial values of Algorithm 1 (parallel initialisation, Section 3.1): the
// initial partitions by Lloyd's k-means, and Psi^(0) of a partition by
// moments.
//
// group_sums_kernel: per block, fixed-order sums over the block's tiles of
// per-observation terms, separately for each group of the partition:
//   mode 0: 1 and y_k                      (counts and sums: group means),
//   mode 1: z_a z_b (b <= a) and z_k^3,    z = y - mean of the group
//           (central second and third moments).
// With centres given, mode 0 first assigns every observation to its nearest
// centre (squared distance accumulated over the coordinates in order, each
// difference, square and sum rounded on its own: no fused multiply-add, so
// the decision is the one a plain double-precision loop takes) and counts
// the labels that changed.
//
// kmeans_update_kernel: centre i = sum / count of group i (unchanged when the
// group is empty).  group_means_kernel: counts and means.
// moment_finalize_kernel: one thread per group, the moment rule:
//   pi_i = n_i / n, nu_i = nu0,
//   Delta_i[k][k] = lam sign(skew_k) sd_k (k < min(p, r)), 0 elsewhere,
//   mu_i = ybar_i - m1 Delta_i 1_r,
//   Sigma_i = (nu0 - 2)/nu0 (S_i - Delta_i C Delta_i^T),
// with m1 = E|U_k| = sqrt(nu/pi) Gamma((nu-1)/2) / Gamma(nu/2) and
// C = Cov(|U|) (diagonal nu/(nu-2) - m1^2, off-diagonal (2/pi) nu/(nu-2) - m1^2)
// for U ~ t_r(0, I, nu0): E[Y] = mu + m1 Delta 1 and
// Cov(Y) = nu/(nu-2) Sigma + Delta C Delta^T for the CFUST law.  lam is
// halved (at most 20 times, then 0) until Sigma_i is positive definite.
#include <math.h>

#include "cfust_internal.cuh"

namespace cfust {

namespace {

constexpr int IT = 256;  // threads per block = observations per tile

__device__ inline int packed_pair_a(int e) {
  int a = 0;
  while ((a + 1) * (a + 2) / 2 <= e) ++a;
  return a;
}

template <int MODE>
__global__ void __launch_bounds__(IT) group_sums_kernel(const double *Y, int64_t n, int p, int g, int32_t *labels,
                                                        const double *cm, int assign, int first, double *partials,
                                                        unsigned long long *changed, int *status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = MODE == 0 ? p + 1 : p * (p + 1) / 2 + p;
  const int GW = g * W;
  double *ys = reinterpret_cast<double *>(smem_raw);  // [IT][p]
  double *cms = ys + IT * p;                          // [g][p] centres or means
  double *acc = cms + g * p;                          // [GW]
  double *red = acc + GW;                             // [IT]
  int *lab = reinterpret_cast<int *>(red + IT);       // [IT]
  for (int e = threadIdx.x; e < g * p; e += IT) cms[e] = cm != nullptr ? cm[e] : 0.0;
  for (int e = threadIdx.x; e < GW; e += IT) acc[e] = 0.0;
  // each entry's rows are split over `splits` threads, combined in order
  const int splits = GW >= IT ? 1 : IT / GW;
  unsigned long long nchanged = 0;
  int bad = 0;
  __syncthreads();
  const int64_t ntiles = (n + IT - 1) / IT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t j0 = tile * IT;
    const int nt = (int)((n - j0) < IT ? (n - j0) : IT);
    for (int idx = threadIdx.x; idx < nt * p; idx += IT) ys[idx] = Y[j0 * p + idx];
    __syncthreads();
    if (threadIdx.x < nt) {
      const int jj = threadIdx.x;
      const double *y = ys + jj * p;
      int li;
      if (MODE == 0 && assign) {
        li = 0;
        double best = INFINITY;
        for (int i = 0; i < g; ++i) {
          double d = 0.0;
          for (int k = 0; k < p; ++k) {
            const double t = __dsub_rn(y[k], cms[i * p + k]);
            d = __dadd_rn(d, __dmul_rn(t, t));
          }
          if (d < best) {
            best = d;
            li = i;
          }
        }
        if (first || labels[j0 + jj] != li) ++nchanged;
        labels[j0 + jj] = li;
      } else {
        li = labels[j0 + jj];
        if (li < 0 || li >= g) {
          bad = 1;
          li = -1;
        }
      }
      lab[jj] = li;
      if (MODE == 1 && li >= 0)
        for (int k = 0; k < p; ++k) ys[jj * p + k] -= cms[li * p + k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < GW * splits; t += IT) {
      const int e = t % GW, sp = t / GW;
      const int i = e / W, w = e % W;
      double s = 0.0;
      if (MODE == 0) {
        for (int jj = sp; jj < nt; jj += splits)
          if (lab[jj] == i) s += (w == 0) ? 1.0 : ys[jj * p + w - 1];
      } else {
        const int pp = p * (p + 1) / 2;
        if (w < pp) {
          const int a = packed_pair_a(w), b = w - a * (a + 1) / 2;
          for (int jj = sp; jj < nt; jj += splits)
            if (lab[jj] == i) s += ys[jj * p + a] * ys[jj * p + b];
        } else {
          const int k = w - pp;
          for (int jj = sp; jj < nt; jj += splits)
            if (lab[jj] == i) {
              const double z = ys[jj * p + k];
              s += z * z * z;
            }
        }
      }
      if (splits > 1) red[t] = s;
      else acc[e] += s;
    }
    if (splits > 1) {
      __syncthreads();
      for (int e = threadIdx.x; e < GW; e += IT) {
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += red[sp * GW + e];
        acc[e] += s;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < GW; e += IT) partials[(int64_t)blockIdx.x * GW + e] = acc[e];
  if (MODE == 0 && assign && changed != nullptr) {
    // warp sums, one atomic per warp (the count is an integer: order-free)
    for (int o = 16; o > 0; o >>= 1) nchanged += __shfl_down_sync(0xffffffffu, nchanged, o);
    if ((threadIdx.x & 31) == 0 && nchanged) atomicAdd(changed, nchanged);
  }
  if (bad) atomicOr(status, ERR_BAD_LABEL);
}

// Sum of entry e over the blocks, in block order.
__device__ inline double block_total(const double *partials, int nblk, int GW, int e) {
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * GW + e];
  return s;
}

__global__ void kmeans_update_kernel(const double *partials, int nblk, int g, int p, double *centers) {
  const int W = p + 1, GW = g * W;
  for (int e = threadIdx.x; e < g * p; e += blockDim.x) {
    const int i = e / p, k = e % p;
    const double cnt = block_total(partials, nblk, GW, i * W);
    if (cnt > 0.0) centers[e] = block_total(partials, nblk, GW, i * W + 1 + k) / cnt;
  }
}

__global__ void group_means_kernel(const double *partials, int nblk, int g, int p, double *means, double *counts) {
  const int W = p + 1, GW = g * W;
  for (int e = threadIdx.x; e < g * p; e += blockDim.x) {
    const int i = e / p, k = e % p;
    const double cnt = block_total(partials, nblk, GW, i * W);
    means[e] = cnt > 0.0 ? block_total(partials, nblk, GW, i * W + 1 + k) / cnt : 0.0;
    if (k == 0) counts[i] = cnt;
  }
}

__device__ bool chol_pd(const double *S, int p) {
  double L[PMAX * PMAX];
  for (int j = 0; j < p; ++j) {
    double s = S[j * p + j];
    for (int k = 0; k < j; ++k) s -= L[j * PMAX + k] * L[j * PMAX + k];
    if (!(s > 0.0) || !isfinite(s)) return false;
    const double d = sqrt(s);
    L[j * PMAX + j] = d;
    for (int i = j + 1; i < p; ++i) {
      double t = S[i * p + j];
      for (int k = 0; k < j; ++k) t -= L[i * PMAX + k] * L[j * PMAX + k];
      L[i * PMAX + j] = t / d;
    }
  }
  return true;
}

__global__ void moment_finalize_kernel(const double *partials, int nblk, const double *counts, const double *means,
                                       int64_t n, int g, int p, int r, double nu0, double lam, double *params,
                                       double *lam_used, int *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g) return;
  const int pp = p * (p + 1) / 2;
  const int W = pp + p, GW = g * W;
  const double ni = counts[i];
  if (!(ni >= (double)(p + 1))) {
    atomicOr(status, ERR_INIT_GROUP);
    return;
  }
  double S[PMAX * PMAX], m3[PMAX], sd[PMAX], Sig[PMAX * PMAX], D[PMAX * RMAX];
  for (int a = 0; a < p; ++a)
    for (int b = 0; b <= a; ++b)
      S[a * p + b] = S[b * p + a] = block_total(partials, nblk, GW, i * W + a * (a + 1) / 2 + b) / ni;
  for (int k = 0; k < p; ++k) {
    m3[k] = block_total(partials, nblk, GW, i * W + pp + k) / ni;
    sd[k] = sqrt(S[k * p + k]);
  }
  if (!chol_pd(S, p)) {
    atomicOr(status, ERR_INIT_GROUP);
    return;
  }
  const double m1 = exp(0.5 * log(nu0 / M_PI) + lgamma(0.5 * (nu0 - 1.0)) - lgamma(0.5 * nu0));
  const double sv = nu0 / (nu0 - 2.0);
  const double c_diag = sv - m1 * m1, c_off = (2.0 / M_PI) * sv - m1 * m1;
  const int kd = p < r ? p : r;
  double li = lam;
  for (int h = 0; h <= 21; ++h) {
    if (h == 21) li = 0.0;
    for (int e = 0; e < p * r; ++e) D[e] = 0.0;
    for (int k = 0; k < kd; ++k) D[k * r + k] = li * (m3[k] < 0.0 ? -1.0 : 1.0) * sd[k];
    // Delta C Delta^T with Delta diagonal in its first kd columns
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b) {
        double dcd = 0.0;
        if (a < kd && b < kd) dcd = D[a * r + a] * (a == b ? c_diag : c_off) * D[b * r + b];
        Sig[a * p + b] = (nu0 - 2.0) / nu0 * (S[a * p + b] - dcd);
      }
    if (chol_pd(Sig, p)) break;
    li *= 0.5;
  }
  ParamView pv = param_view(params, g, p, r);
  pv.pi[i] = ni / (double)n;
  pv.nu[i] = nu0;
  for (int a = 0; a < p; ++a) {
    double rowsum = 0.0;
    for (int t = 0; t < r; ++t) rowsum += D[a * r + t];
    pv.mu[i * p + a] = means[i * p + a] - m1 * rowsum;
    for (int b = 0; b < p; ++b) pv.Sigma[(int64_t)i * p * p + a * p + b] = Sig[a * p + b];
    for (int t = 0; t < r; ++t) pv.Delta[(int64_t)i * p * r + a * r + t] = D[a * r + t];
  }
  if (lam_used) lam_used[i] = li;
}

size_t group_sums_smem(int mode, int p, int g) {
  const int W = mode == 0 ? p + 1 : p * (p + 1) / 2 + p;
  return sizeof(double) * ((size_t)IT * p + (size_t)g * p + (size_t)g * W + IT) + sizeof(int) * IT;
}

}  // namespace

int group_sums_width(int mode, int p) { return mode == 0 ? p + 1 : p * (p + 1) / 2 + p; }

int group_sums_nblocks(int64_t n) {
  const int64_t ntiles = (n + IT - 1) / IT;
  const int64_t cap = (int64_t)sm_count() * 2;
  return (int)(ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
}

cudaError_t launch_group_sums(int mode, const double *Y, int64_t n, int p, int g, int32_t *labels,
                              const double *cm, int assign, int first, double *partials, int nblk,
                              unsigned long long *changed, int *status, cudaStream_t st) {
  const size_t smem = group_sums_smem(mode, p, g);
  cudaError_t e;
  if (mode == 0) {
    e = raise_smem_limit((const void *)group_sums_kernel<0>, (size_t)((int)smem));
    if (e != cudaSuccess) return e;
    group_sums_kernel<0><<<nblk, IT, smem, st>>>(Y, n, p, g, labels, cm, assign, first, partials, changed, status);
  } else {
    e = raise_smem_limit((const void *)group_sums_kernel<1>, (size_t)((int)smem));
    if (e != cudaSuccess) return e;
    group_sums_kernel<1><<<nblk, IT, smem, st>>>(Y, n, p, g, labels, cm, 0, 0, partials, changed, status);
  }
  return cudaGetLastError();
}

cudaError_t launch_kmeans_update(const double *partials, int nblk, int g, int p, double *centers, cudaStream_t st) {
  kmeans_update_kernel<<<1, 256, 0, st>>>(partials, nblk, g, p, centers);
  return cudaGetLastError();
}

cudaError_t launch_group_means(const double *partials, int nblk, int g, int p, double *means, double *counts,
                               cudaStream_t st) {
  group_means_kernel<<<1, 256, 0, st>>>(partials, nblk, g, p, means, counts);
  return cudaGetLastError();
}

cudaError_t launch_moment_finalize(const double *partials, int nblk, const double *counts, const double *means,
                                   int64_t n, int g, int p, int r, double nu0, double lam, double *params,
                                   double *lam_used, int *status, cudaStream_t st) {
  moment_finalize_kernel<<<(g + 31) / 32, 32, 0, st>>>(partials, nblk, counts, means, n, g, p, r, nu0, lam, params,
                                                       lam_used, status);
  return cudaGetLastError();
}

}  // namespace cfust

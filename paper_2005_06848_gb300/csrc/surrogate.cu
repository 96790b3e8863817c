// Learned surrogate of the trivariate truncated-t integrals of the E-step.
//
// Problem: X ~ t_3(0, R, m), R a correlation matrix, truncation X > c.
//   inputs  (7):  c_1, c_2, c_3, R_12, R_13, R_23, log m
//   outputs (10): log P(X > c), E[X | X > c] (3), E[X X^T | X > c] upper
//                 triangle (11, 12, 13, 22, 23, 33)
// Network 7 -> 128 -> 128 -> 128 -> 10 with GELU (tanh form) after the hidden
// layers; BF16 weights and activations, FP32 accumulation on the tensor cores
// (tcgen05 MMAs with accumulators in tensor memory, in the fused E-step,
// prediction and the training GEMMs), FP32 master weights updated by Adam.  Inputs are
// normalised as c and log m mapped from their ranges onto [-1, 1] and R/0.9.
// The network predicts log(-log P), the first moments and the covariance
// (second moments minus the products of the first moments), standardised by
// per-output mean and standard deviation of the training labels.
//
// Labels come from the plain lattice evaluator (Genz separation of variables
// on the shifted Korobov lattice) with chi-scale tables on a grid of 256
// values of log m over [log 3, log 30], interpolated linearly in log m; the
// same evaluator judges the error.
//
// Training domain: -8 <= c_t <= 4, |R_ht| <= 0.9, every squared Cholesky
// pivot of R >= 0.05, m in [3, 30].  The E-step uses the network for a pair
// whose pass-B point lies in the box (below it too once nu + p >= 8, where a
// coordinate under -8 is clamped: it moves P by at most P(t_8 < -8)); the
// other pairs go to the lattice rule with an upper bound of their log T for
// its triage.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>

#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "cfust_internal.cuh"
#include "normal_f32.cuh"
#include "special.cuh"
#include "tcgen05.cuh"

namespace cfust {
namespace sg {

constexpr int DIN = 7, DINP = 16, H = 128, DOUT = 10, DOUTP = 16;
constexpr int NPARAM = DIN * H + H + 2 * (H * H + H) + H * DOUT + DOUT;  // 35338
constexpr int MGRID = 256;
constexpr float C_LO = -8.0f, C_HI = 4.0f, RHO_MAX = 0.9f, PIVOT_MIN = 0.05f;
// added to the network's log T at a clamped truncation point to bound the
// log T of a pair outside the box (network error and the lower clamp)
constexpr float UB_MARGIN = 5.0f;
// loss weight of log P (the moments weigh 1): the log-likelihood depends on it directly
constexpr float LOSS_W0 = 4.0f;
constexpr float CLAMP_LO_MIN_DOF = 8.0f;
constexpr double LOGM_LO = 1.0986122886681098, LOGM_HI = 3.4011973816621555;  // log 3, log 30

// offsets of the flat parameter vector (same order as the FP64 oracle)
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + DIN * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + H * DOUT;

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM of the training passes, C[M x N] = A[M x K] B[K x N],
// FP32 accumulation.  A(m, k) = transA ? A[k lda + m] : A[m lda + k];  B(k, n)
// likewise.  Tile 128 x 128, K in slices of 32 (kernel below).
// ---------------------------------------------------------------------------
// Operand layouts must keep the contiguous index 16-byte aligned: lda, ldb
// and the untransposed K multiples of 8 (every use here: 16 or 128).
struct Gemm {
  int M, N, K;
  const bf16 *A;
  int lda, transA;
  const bf16 *B;
  int ldb, transB;
  int k_chunk;          // split-K: blockIdx.z covers [z k_chunk, (z + 1) k_chunk)
  int mode;             // 0 split-K partial, 1 bias + GELU, 2 times GELU'(Zprev), 3 bias, fp32 out
  const float *bias;
  float *C;             // modes 0, 3
  int ldc;
  bf16 *Zout, *Hout;    // mode 1: Z and GELU(Z); mode 2: Hout receives the product
  int ldo;
  const bf16 *Zprev;    // mode 2
};

constexpr int BM = 128, BN = 128, BK = 32;

// GELU in its tanh form, the tanh from the hardware approximation
// (tanh.approx.f32, relative error about 2^-11, below the BF16 rounding of
// the activations); training and inference use the same function.
__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// GELU(z) = z/2 (1 + t), t = tanh(z (k + a k z^2)), k = sqrt(2/pi), a = 0.044715,
// evaluated in the same operation order in the scalar and the paired forms
// (so the GEMM path and the fused E-step produce the same activations).
constexpr float GELU_K = 0.7978845608028654f, GELU_AK = 0.044715f * 0.7978845608028654f;
__device__ __forceinline__ float gelu_f(float z) {
  const float arg = z * fmaf(z * z, GELU_AK, GELU_K);
  const float hz = 0.5f * z;
  return fmaf(hz, tanh_approx(arg), hz);
}
__device__ __forceinline__ float2 gelu_x2(float2 z) {
  const float2 arg = __fmul2_rn(z, __ffma2_rn(__fmul2_rn(z, z), make_float2(GELU_AK, GELU_AK),
                                              make_float2(GELU_K, GELU_K)));
  const float2 hz = __fmul2_rn(z, make_float2(0.5f, 0.5f));
  return __ffma2_rn(hz, make_float2(tanh_approx(arg.x), tanh_approx(arg.y)), hz);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float gelu_grad_f(float z) {
  const float t = tanh_approx(z * fmaf(z * z, GELU_AK, GELU_K));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * fmaf(3.0f * GELU_AK, z * z, GELU_K);
}

// The GEMM on the tcgen05 tensor cores.  A CTA of 256 threads owns one
// 128 x 128 output tile of one K range (split-K over blockIdx.z); K advances in
// slices of 32 staged in shared memory in the UMMA K-major layout (both
// operands K-major: A as [m][k], B as [n][k]), double-buffered so the loads of
// slice s + 1 overlap the MMAs of slice s; thread 0 issues two MMAs (K = 16)
// per slice into a 128 x 128 FP32 accumulator in tensor memory, each slice's
// completion arriving on its buffer's mbarrier.  The epilogue reads the
// accumulator with tcgen05.ld: warp w takes lanes 32 (w % 4) .. + 31 (rows) and
// columns 64 (w / 4) .. + 63.
constexpr uint32_t GT_TILE = BM * BK * 2;   // bytes of one operand slice
constexpr uint32_t GT_SBO = (BK / 8) * 128;
constexpr uint32_t GT_IDESC = tc::idesc_bf16_f32(BM, BN);

__device__ __forceinline__ void gemm_load_slice(const Gemm &g, unsigned char *As, unsigned char *Bs, int m0, int n0,
                                                int k0, int kb1, int tid) {
  const bf16 zero = __float2bfloat16(0.f);
  if (!g.transA) {
    for (int v = tid; v < BM * (BK / 8); v += 256) {
      const int mm = v / (BK / 8), kk = (v % (BK / 8)) * 8;
      const int m = m0 + mm, k = k0 + kk;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (m < g.M && k + 8 <= kb1) val = *reinterpret_cast<const uint4 *>(g.A + (int64_t)m * g.lda + k);
      *reinterpret_cast<uint4 *>(As + tc::kmajor_offset(mm, kk, BK)) = val;
    }
  } else {
    for (int v = tid; v < BK * (BM / 8); v += 256) {
      const int kk = v / (BM / 8), mm = (v % (BM / 8)) * 8;
      const int m = m0 + mm, k = k0 + kk;
      bf16 e[8];
      if (k < kb1 && m + 8 <= g.M) {
        *reinterpret_cast<uint4 *>(e) = *reinterpret_cast<const uint4 *>(g.A + (int64_t)k * g.lda + m);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) e[q] = (k < kb1 && m + q < g.M) ? g.A[(int64_t)k * g.lda + m + q] : zero;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) *reinterpret_cast<bf16 *>(As + tc::kmajor_offset(mm + q, kk, BK)) = e[q];
    }
  }
  if (!g.transB) {
    for (int v = tid; v < BK * (BN / 8); v += 256) {
      const int kk = v / (BN / 8), nn = (v % (BN / 8)) * 8;
      const int n = n0 + nn, k = k0 + kk;
      bf16 e[8];
      if (k < kb1 && n + 8 <= g.N) {
        *reinterpret_cast<uint4 *>(e) = *reinterpret_cast<const uint4 *>(g.B + (int64_t)k * g.ldb + n);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) e[q] = (k < kb1 && n + q < g.N) ? g.B[(int64_t)k * g.ldb + n + q] : zero;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) *reinterpret_cast<bf16 *>(Bs + tc::kmajor_offset(nn + q, kk, BK)) = e[q];
    }
  } else {
    for (int v = tid; v < BN * (BK / 8); v += 256) {
      const int nn = v / (BK / 8), kk = (v % (BK / 8)) * 8;
      const int n = n0 + nn, k = k0 + kk;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (n < g.N && k + 8 <= kb1) val = *reinterpret_cast<const uint4 *>(g.B + (int64_t)n * g.ldb + k);
      *reinterpret_cast<uint4 *>(Bs + tc::kmajor_offset(nn, kk, BK)) = val;
    }
  }
}

__global__ void __launch_bounds__(256) gemm_kernel(Gemm g, int *status) {
  // [stage][A | B] slices, then two mbarriers and the tensor-memory address
  __shared__ __align__(1024) unsigned char sm[2 * 2 * GT_TILE];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * g.k_chunk;
  const int kb1 = min(g.K, kb0 + g.k_chunk);
  if (tid < 2) tc::mbar_init1(bars + tid);
  if (warp == 0) {
    tc::tmem_alloc(&tslot, 128);
    tc::tmem_relinquish();
  }
  if (kb0 < kb1) gemm_load_slice(g, sm, sm + GT_TILE, m0, n0, kb0, kb1, tid);
  const uint32_t sbase = tc::smem_u32(sm);
  uint32_t ph[2] = {0u, 0u};
  bool bad = false;
  int it = 0;
  for (int k0 = kb0; k0 < kb1; k0 += BK, ++it) {
    const int s = it & 1;
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a = sbase + s * 2 * GT_TILE, b = a + GT_TILE;
#pragma unroll
      for (int ks = 0; ks < BK / 16; ++ks)
        tc::mma_bf16(tslot, tc::smem_desc(a + ks * 256, 128, GT_SBO), tc::smem_desc(b + ks * 256, 128, GT_SBO),
                     GT_IDESC, (k0 > kb0 || ks > 0) ? 1u : 0u);
      tc::mma_commit(bars + s);
    }
    if (k0 + BK < kb1) {
      // the other buffer was read by the previous slice's MMAs: wait for them
      if (it >= 1) {
        bad = !tc::mbar_wait(bars + (s ^ 1), ph[s ^ 1], 1 << 22) || bad;
        ph[s ^ 1] ^= 1u;
      }
      gemm_load_slice(g, sm + (s ^ 1) * 2 * GT_TILE, sm + (s ^ 1) * 2 * GT_TILE + GT_TILE, m0, n0, k0 + BK, kb1,
                      tid);
    }
  }
  // the last slice's MMAs (in order after every earlier one)
  if (it > 0) bad = !tc::mbar_wait(bars + ((it - 1) & 1), ph[(it - 1) & 1], 1 << 22) || bad;
  tc::fence_before_sync();
  __syncthreads();  // also publishes the tensor-memory address when K was empty
  tc::fence_after_sync();
  if (bad && status) atomicOr(status, ERR_TIMEOUT);
  // epilogue: this thread's row, 64 columns in two loads of 32, written 8
  // columns (16 bytes of BF16, 32 of FP32) at a time where the whole group
  // lies inside the matrix (every output here has rows of 16 or 128 values)
  const int row = (warp & 3) * 32 + lane, m = m0 + row;
  const uint32_t taddr = tslot + ((uint32_t)((warp & 3) * 32) << 16) + (warp >> 2) * 64;
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    uint32_t v[32];
    tc::tmem_ld32(taddr + half * 32, v);
    tc::tmem_wait_ld(v);
    if (m >= g.M) continue;
    const int nb = n0 + (warp >> 2) * 64 + half * 32;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = nb + 8 * q;
      if (n >= g.N) continue;
      float val[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) val[c] = it > 0 ? __uint_as_float(v[8 * q + c]) : 0.f;
      if (g.mode == 0 || g.mode == 3) {
        float *dst = g.C + (g.mode == 0 ? (int64_t)blockIdx.z * g.M * g.N : 0) + (int64_t)m * g.ldc + n;
        if (g.mode == 3)
#pragma unroll
          for (int c = 0; c < 8; ++c) val[c] += g.bias[n + c];
        reinterpret_cast<float4 *>(dst)[0] = make_float4(val[0], val[1], val[2], val[3]);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(val[4], val[5], val[6], val[7]);
      } else if (g.mode == 1) {
        uint32_t zw[4], hw[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float z0 = val[2 * c] + g.bias[n + 2 * c], z1 = val[2 * c + 1] + g.bias[n + 2 * c + 1];
          zw[c] = pack_bf16x2(z0, z1);
          hw[c] = pack_bf16x2(gelu_f(z0), gelu_f(z1));
        }
        *reinterpret_cast<uint4 *>(g.Zout + (int64_t)m * g.ldo + n) = make_uint4(zw[0], zw[1], zw[2], zw[3]);
        *reinterpret_cast<uint4 *>(g.Hout + (int64_t)m * g.ldo + n) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      } else {
        const uint4 zp4 = *reinterpret_cast<const uint4 *>(g.Zprev + (int64_t)m * g.ldo + n);
        const bf16 *zp = reinterpret_cast<const bf16 *>(&zp4);
        uint32_t hw[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          hw[c] = pack_bf16x2(val[2 * c] * gelu_grad_f(__bfloat162float(zp[2 * c])),
                              val[2 * c + 1] * gelu_grad_f(__bfloat162float(zp[2 * c + 1])));
        *reinterpret_cast<uint4 *>(g.Hout + (int64_t)m * g.ldo + n) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tslot, 128);
  }
}

cudaError_t gemm(const Gemm &g, int splits, cudaStream_t st, int *status) {
  // the epilogue writes groups of 8 columns: row lengths must be multiples of 8
  if (g.N % 8 != 0 || (g.mode == 0 || g.mode == 3 ? g.ldc : g.ldo) % 8 != 0) return cudaErrorInvalidValue;
  dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, splits);
  gemm_kernel<<<grid, 256, 0, st>>>(g, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small elementwise / reduction kernels
// ---------------------------------------------------------------------------

__device__ __forceinline__ void normalise_input(const float *x, float *u) {
  for (int t = 0; t < 3; ++t) u[t] = (2.f * x[t] - (C_LO + C_HI)) / (C_HI - C_LO);
  for (int t = 3; t < 6; ++t) u[t] = x[t] / RHO_MAX;
  u[6] = (float)((2.0 * x[6] - (LOGM_LO + LOGM_HI)) / (LOGM_HI - LOGM_LO));
}

// outputs -> network targets: log P becomes log(-log P) (relative precision
// for P near 1), second moments (upper order 00 01 02 11 12 22) become
// covariances E[X_a X_b] - E[X_a] E[X_b]
constexpr float NEGLOG_MIN = 1e-12f;
__host__ __device__ __forceinline__ void to_net(const float *y, float *t) {
  const int A[6] = {0, 0, 0, 1, 1, 2}, Bi[6] = {0, 1, 2, 1, 2, 2};
  t[0] = logf(fmaxf(-y[0], NEGLOG_MIN));
  for (int k = 1; k < 4; ++k) t[k] = y[k];
  for (int k = 0; k < 6; ++k) t[4 + k] = y[4 + k] - y[1 + A[k]] * y[1 + Bi[k]];
}
__host__ __device__ __forceinline__ void from_net(const float *t, float *y) {
  const int A[6] = {0, 0, 0, 1, 1, 2}, Bi[6] = {0, 1, 2, 1, 2, 2};
  y[0] = -expf(t[0]);
  for (int k = 1; k < 4; ++k) y[k] = t[k];
  for (int k = 0; k < 6; ++k) y[4 + k] = t[4 + k] + t[1 + A[k]] * t[1 + Bi[k]];
}

// raw inputs [B][7] -> padded normalised BF16 [B][16]
__global__ void prep_input_kernel(const float *x, bf16 *x0, int64_t B) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  float u[DIN];
  normalise_input(x + b * DIN, u);
  for (int t = 0; t < DINP; ++t) x0[b * DINP + t] = __float2bfloat16(t < DIN ? u[t] : 0.f);
}

// loss partial per block and dZ4 = 2 (out - t) / (B * 10), t normalised targets
__global__ void loss_kernel(const float *out, const float *y, const float *norm, bf16 *dz, double *loss_part,
                            int64_t B) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
    float t[DOUT];
    to_net(y + b * DOUT, t);
    for (int k = 0; k < DOUTP; ++k) {
      float d = 0.f;
      float wk = 0.f;
      if (k < DOUT) {
        const float tn = (t[k] - norm[k]) / norm[DOUT + k];
        d = out[b * DOUTP + k] - tn;
        wk = (k == 0) ? LOSS_W0 : 1.f;
        s += (double)wk * d * d;
      }
      dz[b * DOUTP + k] = __float2bfloat16(2.0f * wk * d / (float)(B * DOUT));
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// column sums of a BF16 [B][ld] matrix, columns < ncol, into grad[off + col]
__global__ void colsum_kernel(const bf16 *dz, int ld, int ncol, int64_t B, float *grad, int off) {
  const int col = blockIdx.x;
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t b = threadIdx.x; b < B; b += 256) s += __bfloat162float(dz[b * ld + col]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0 && col < ncol) grad[off + col] = red[0];
}

// sum split-K partials [S][M][Np] (rows < mrows, cols < ncols) into grad[off + m ncols + n]
__global__ void reduce_partials_kernel(const float *part, int S, int M, int Np, int mrows, int ncols, float *grad,
                                       int off) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mrows * ncols) return;
  const int m = idx / ncols, n = idx % ncols;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * M * Np + (int64_t)m * Np + n];
  grad[off + idx] = s;
}

__global__ void adam_kernel(float *theta, float *mom, float *vel, const float *grad, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = grad[k];
  const float mk = b1 * mom[k] + (1.f - b1) * gk;
  const float vk = b2 * vel[k] + (1.f - b2) * gk * gk;
  mom[k] = mk;
  vel[k] = vk;
  theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// flat FP32 parameters -> padded BF16 weights W1 [16][128], W2, W3 [128][128], W4 [128][16] and FP32 biases
__global__ void pack_weights_kernel(const float *theta, bf16 *W1, bf16 *W2, bf16 *W3, bf16 *W4, float *b1,
                                    float *b2, float *b3, float *b4) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < DINP * H) {
    const int i = k / H, o = k % H;
    W1[k] = __float2bfloat16(i < DIN ? theta[OFF_W1 + i * H + o] : 0.f);
  }
  if (k < H * H) {
    W2[k] = __float2bfloat16(theta[OFF_W2 + k]);
    W3[k] = __float2bfloat16(theta[OFF_W3 + k]);
  }
  if (k < H * DOUTP) {
    const int i = k / DOUTP, o = k % DOUTP;
    W4[k] = __float2bfloat16(o < DOUT ? theta[OFF_W4 + i * DOUT + o] : 0.f);
  }
  if (k < H) {
    b1[k] = theta[OFF_B1 + k];
    b2[k] = theta[OFF_B2 + k];
    b3[k] = theta[OFF_B3 + k];
  }
  if (k < DOUTP) b4[k] = (k < DOUT) ? theta[OFF_B4 + k] : 0.f;
}

// network output [B][16] (normalised covariance form) -> outputs [B][10]
__global__ void denorm_kernel(const float *out, const float *norm, float *y, int64_t B) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  float t[DOUT];
  for (int k = 0; k < DOUT; ++k) t[k] = fmaf(out[b * DOUTP + k], norm[DOUT + k], norm[k]);
  from_net(t, y + b * DOUT);
}

// chi-scale tables on the grid of m: [MGRID][N]
__global__ void chi_grid_kernel(LatticeDev lat, float *tab) {
  const int gidx = blockIdx.y;
  const double m = exp(LOGM_LO + gidx * (LOGM_HI - LOGM_LO) / (MGRID - 1));
  const int N = lat.n;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int64_t idx = ((int64_t)k * lat.z[0]) % N;
    double u = (double)idx / (double)N + lat.shift[0];
    if (u >= 1.0) u -= 1.0;
    u = 1.0 - fabs(2.0 * u - 1.0);
    u = fmin(fmax(u, 1.1102230246251565e-16), 1.0 - 1.1102230246251565e-16);
    tab[(int64_t)gidx * N + k] = (float)sqrt(2.0 * inc_gamma_inv(0.5 * m, u) / m);
  }
}

// One warp per sample: the lattice rule for P(X > c), E[X | X > c], E[X X^T | X > c]
// with X = L V, V ~ t_3(0, I, m), m snapped to the chi-table grid.
__global__ void __launch_bounds__(256) label_kernel(const float *x, float *y, int64_t B, LatticeDev lat,
                                                    const float *tab) {
  const int lane = threadIdx.x & 31;
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;
  const float *xb = x + b * DIN;
  const float c[3] = {xb[0], xb[1], xb[2]};
  const float r12 = xb[3], r13 = xb[4], r23 = xb[5];
  // Cholesky of the correlation matrix
  const float L00 = 1.f, L10 = r12, L20 = r13;
  const float L11 = sqrtf(fmaxf(1.f - r12 * r12, 1e-12f));
  const float L21 = (r23 - r13 * r12) / L11;
  const float L22 = sqrtf(fmaxf(1.f - r13 * r13 - L21 * L21, 1e-12f));
  const float Lm[3][3] = {{L00, 0.f, 0.f}, {L10, L11, 0.f}, {L20, L21, L22}};
  const float Li[3] = {1.f, 1.f / L11, 1.f / L22};
  // chi scale at this m: linear interpolation in log m between grid tables
  float gpos = (float)((xb[6] - LOGM_LO) / (LOGM_HI - LOGM_LO) * (MGRID - 1));
  gpos = fminf(fmaxf(gpos, 0.f), (float)(MGRID - 1));
  const int gi = min((int)gpos, MGRID - 2);
  const float gw = gpos - (float)gi;
  const int N = lat.n;
  const float *s_lo = tab + (int64_t)gi * N, *s_hi = s_lo + N;
  float fm[3], fstep[3], two_sf[3], sf[3];
  for (int t = 0; t < 3; ++t) {
    const int m0 = (int)(((int64_t)lane * lat.z[t + 1] + lat.sint[t + 1]) % N);
    fm[t] = (float)(2 * m0 - N);
    fstep[t] = (float)(2 * lat.step[t + 1]);
    two_sf[t] = (float)(2.0 * lat.sfrac[t + 1]);
    sf[t] = (float)lat.sfrac[t + 1];
  }
  const float fN = (float)N, invN = 1.f / fN;
  const float umin = 1.1102230246251565e-16f, umax = 1.f - 5.9604644775390625e-08f;
  float W = 0.f, Q = 0.f, M1[3] = {0.f, 0.f, 0.f}, M2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = lane; k < N; k += 32) {
    float um[3], uu[3];
    for (int t = 0; t < 3; ++t) {
      const float mm = 0.5f * (fm[t] + fN);
      um[t] = fminf(fmaxf(fabsf(fm[t] + two_sf[t]) * invN, umin), umax);
      uu[t] = fmaxf(2.f * fminf(mm + sf[t], (fN - mm) - sf[t]) * invN, umin);
      fm[t] += fstep[t];
      if (fm[t] >= fN) fm[t] -= 2.f * fN;
    }
    const float s = fmaf(gw, s_hi[k] - s_lo[k], s_lo[k]);
    // w = p_1 p_2 p_3 and 1 - w = q_1 + p_1 q_2 + p_1 p_2 q_3, both from the
    // small sides, so log P keeps its precision where P is near 1
    float w = 1.f, om = 0.f, z[3];
    for (int t = 0; t < 3; ++t) {
      float acc = c[t] * s;
      for (int h = 0; h < t; ++h) acc -= Lm[t][h] * z[h];
      float p, q;
      phi_upper_pq_f32(acc * Li[t], p, q);
      om = fmaf(w, q, om);
      w *= p;
      z[t] = neg_quantile_f32(um[t], uu[t], p, q);
    }
    Q += om;
    const float is = 1.f / s;
    float v[3];
    for (int t = 0; t < 3; ++t) v[t] = z[t] * is;
    W += w;
    int q6 = 0;
    for (int t = 0; t < 3; ++t) {
      M1[t] += w * v[t];
      for (int h = t; h < 3; ++h) M2[q6++] += w * v[t] * v[h];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    W += __shfl_xor_sync(0xffffffffu, W, o);
    Q += __shfl_xor_sync(0xffffffffu, Q, o);
    for (int t = 0; t < 3; ++t) M1[t] += __shfl_xor_sync(0xffffffffu, M1[t], o);
    for (int t = 0; t < 6; ++t) M2[t] += __shfl_xor_sync(0xffffffffu, M2[t], o);
  }
  if (lane != 0) return;
  // E[V], E[V V^T] (symmetric, from the upper triangle) -> E[L V], L E[V V^T] L^T
  const float iw = 1.f / W;
  float EV[3], EVV[3][3];
  int q6 = 0;
  for (int t = 0; t < 3; ++t) EV[t] = M1[t] * iw;
  for (int t = 0; t < 3; ++t)
    for (int h = t; h < 3; ++h) {
      EVV[t][h] = EVV[h][t] = M2[q6++] * iw;
    }
  float EX[3], EXX[3][3];
  for (int t = 0; t < 3; ++t) {
    EX[t] = 0.f;
    for (int h = 0; h <= t; ++h) EX[t] += Lm[t][h] * EV[h];
  }
  for (int t = 0; t < 3; ++t)
    for (int h = 0; h < 3; ++h) {
      float s2 = 0.f;
      for (int a = 0; a <= t; ++a)
        for (int bb = 0; bb <= h; ++bb) s2 += Lm[t][a] * EVV[a][bb] * Lm[h][bb];
      EXX[t][h] = s2;
    }
  float *yb = y + b * DOUT;
  if (!(W > 0.f)) {  // every point weight underflowed: no label
    for (int k = 0; k < DOUT; ++k) yb[k] = NAN;
    return;
  }
  const float qn = Q / fN;
  yb[0] = (qn < 0.5f) ? log1pf(-qn) : logf(W) - logf(fN);
  yb[1] = EX[0];
  yb[2] = EX[1];
  yb[3] = EX[2];
  yb[4] = EXX[0][0];
  yb[5] = EXX[0][1];
  yb[6] = EXX[0][2];
  yb[7] = EXX[1][1];
  yb[8] = EXX[1][2];
  yb[9] = EXX[2][2];
}

// Positive-definite repair of a predicted 3x3 covariance (upper order 00 01
// 02 11 12 22), keeping its diagonal: variances floored at PSD_FLOOR, each
// first-row correlation clamped to |rho| <= PSD_RHO, and the last factor of the
// LDL^T decomposition shrunk where needed so that every pivot keeps at least
// 1 - PSD_RHO^2 of its variance.  Every entry stays within the (floored)
// variances, a well-conditioned positive definite input comes back unchanged up
// to rounding, and e4 stays positive definite like the exact conditional
// moments.  Continuous in the prediction.
constexpr float PSD_FLOOR = 1e-6f, PSD_RHO = 0.999f;
__device__ __forceinline__ void psd_repair3(float *v) {
  const float d0 = fmaxf(v[0], PSD_FLOOR), d1 = fmaxf(v[3], PSD_FLOOR), d2 = fmaxf(v[5], PSD_FLOOR);
  const float m01 = PSD_RHO * sqrtf(d0 * d1), m02 = PSD_RHO * sqrtf(d0 * d2);
  const float c01 = fminf(fmaxf(v[1], -m01), m01), c02 = fminf(fmaxf(v[2], -m02), m02);
  const float l10 = c01 / d0, l20 = c02 / d0;
  const float p1 = d1 - l10 * c01;  // >= (1 - PSD_RHO^2) d1
  const float lmax = sqrtf(fmaxf(PSD_RHO * PSD_RHO * d2 - l20 * c02, 0.f) / p1);
  const float l21 = fminf(fmaxf((v[4] - l20 * c01) / p1, -lmax), lmax);
  v[0] = d0;
  v[1] = c01;
  v[2] = c02;
  v[3] = d1;
  v[4] = fmaf(l20, c01, l21 * p1);
  v[5] = d2;
}

// Standardised problem of one network row: pair (i, j), pass 0 (dof nu + p,
// limits a_A) or 1 (nu + p + 2, a_B).  X = L V with L = chol(Lambda) is
// t_3(0, Lambda, m); with D = diag(Lambda), X' = D^{-1/2} X is t_3(0, R, m)
// and L V > a holds exactly when X' > c = D^{-1/2} a.
struct RowProblem {
  float c[3], R[3], logm;  // network input (c clamped into the box)
  float logt, nud, q[3];
  float cmaxA;  // largest coordinate of pass A's point (unclamped)
  int kind;  // 2: the pair (both passes) lies in the training domain;
             // 1: only its truncation point leaves the box (log T is bounded
             //    through the clamped point); 0: R or the dof leave the domain
};

__device__ __forceinline__ RowProblem row_problem(const CompT<float> &c, const double *Y, int p, int64_t j,
                                                  int pass) {
  RowProblem rp;
  const double *yj = Y + j * (int64_t)p;
  float yc[PMAX];
#pragma unroll
  for (int k = 0; k < PMAX; ++k) yc[k] = (k < p) ? (float)yj[k] - c.fmu[k] : 0.f;
  float d = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f;
#pragma unroll
  for (int k = 0; k < PMAX; ++k) {
    if (k < p) {
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l <= k; ++l) acc = fmaf(c.fA[k * PMAX + l], yc[l], acc);
      d = fmaf(acc, acc, d);
      q0 = fmaf(c.fB[0 * PMAX + k], acc, q0);
      q1 = fmaf(c.fB[1 * PMAX + k], acc, q1);
      q2 = fmaf(c.fB[2 * PMAX + k], acc, q2);
    }
  }
  const float nu = c.fnu, mA = c.fmA, mB = c.fmB;
  rp.nud = nu + d;
  rp.logt = c.fc0 - 0.5f * mA * log1pf(d / nu);
  rp.q[0] = q0;
  rp.q[1] = q1;
  rp.q[2] = q2;
  // Lambda = L L^T: diagonal and correlations
  const float L00 = c.L[0], L10 = c.L[RMAX], L11 = c.L[RMAX + 1];
  const float L20 = c.L[2 * RMAX], L21 = c.L[2 * RMAX + 1], L22 = c.L[2 * RMAX + 2];
  const float D0 = L00 * L00, D1 = fmaf(L10, L10, L11 * L11), D2 = fmaf(L20, L20, fmaf(L21, L21, L22 * L22));
  const float i0 = rsqrtf(D0), i1 = rsqrtf(D1), i2 = rsqrtf(D2);
  rp.R[0] = L10 * L00 * i0 * i1;
  rp.R[1] = L20 * L00 * i0 * i2;
  rp.R[2] = fmaf(L20, L10, L21 * L11) * i1 * i2;
  const float p2 = 1.f - rp.R[0] * rp.R[0];
  const float l32 = (rp.R[2] - rp.R[1] * rp.R[0]) * rsqrtf(fmaxf(p2, 1e-30f));
  const float p3 = 1.f - rp.R[1] * rp.R[1] - l32 * l32;
  const bool comp_ok = fabsf(rp.R[0]) <= RHO_MAX && fabsf(rp.R[1]) <= RHO_MAX && fabsf(rp.R[2]) <= RHO_MAX &&
                       p2 >= PIVOT_MIN && p3 >= PIVOT_MIN && mA >= 3.f && mB <= 30.f;
  const float m = pass ? mB : mA;
  const float f = -sqrtf(m / rp.nud);
  const float cr[3] = {q0 * f * i0, q1 * f * i1, q2 * f * i2};
  const float fA = -sqrtf(mA / rp.nud);
  rp.cmaxA = fmaxf(q0 * fA * i0, fmaxf(q1 * fA * i1, q2 * fA * i2));
  // pass B has the larger limits (same signs): its box decides the pair
  const float fB = -sqrtf(mB / rp.nud);
  const float cB[3] = {q0 * fB * i0, q1 * fB * i1, q2 * fB * i2};
  // Below the box a coordinate is all but untruncated once the dof reach
  // CLAMP_LO_MIN_DOF: P(X_t < -8) <= 2.2e-5 for t_8 and less for more dof, the
  // most that clamping c_t up to -8 can move P; such pairs stay with the network.
  const float lo = (mA >= CLAMP_LO_MIN_DOF) ? -INFINITY : C_LO;
  bool inbox = true;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    inbox = inbox && cB[t] >= lo && cB[t] <= C_HI;
    rp.c[t] = fminf(fmaxf(cr[t], C_LO), C_HI);
  }
  rp.kind = comp_ok ? (inbox ? 2 : 1) : 0;
  rp.logm = logf(m);
  return rp;
}

// The network's normalised input of a row (the clamped point c and log m
// mapped from their ranges onto [-1, 1], R / 0.9), before its BF16 rounding.
__device__ __forceinline__ void network_input(const RowProblem &rp, float (&u)[DIN]) {
  const float logm_mid = (float)(LOGM_LO + LOGM_HI), logm_scale = (float)(2.0 / (LOGM_HI - LOGM_LO));
  const float cs = 2.f / (C_HI - C_LO), cm = C_LO + C_HI;
  u[0] = (2.f * rp.c[0] - cm) * 0.5f * cs;
  u[1] = (2.f * rp.c[1] - cm) * 0.5f * cs;
  u[2] = (2.f * rp.c[2] - cm) * 0.5f * cs;
  u[3] = rp.R[0] / RHO_MAX;
  u[4] = rp.R[1] / RHO_MAX;
  u[5] = rp.R[2] / RHO_MAX;
  u[6] = (2.f * rp.logm - logm_mid) * (0.5f * logm_scale);
}

// Every pair's two network inputs exactly as the surrogate E-step hands them
// to the tensor cores (BF16-rounded, returned as floats): x_out[(i n + j) 2 +
// pass][7], and the pair's domain class kind[i n + j] (2 in the domain, 1 the
// point clamped into the box, 0 outside).
__global__ void inputs_kernel(const double *Y, int64_t n, int g, int p, const CompT<float> *comp, float *x_out,
                              int *kind) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= 2 * (int64_t)g * n) return;
  const int64_t ij = k >> 1;
  const int pass = (int)(k & 1), i = (int)(ij / n);
  const int64_t j = ij % n;
  const RowProblem rp = row_problem(comp[i], Y, p, j, pass);
  float u[DIN];
  network_input(rp, u);
#pragma unroll
  for (int t = 0; t < DIN; ++t) x_out[k * DIN + t] = __bfloat162float(__float2bfloat16_rn(u[t]));
  if (pass == 0) kind[ij] = rp.kind;
}

// ---------------------------------------------------------------------------
// The network on the fifth-generation tensor cores (tcgen05).
//
// A CTA of four warpgroups (512 threads, one CTA per SM) holds the BF16
// weights in shared memory in the UMMA K-major layout (W_l as [out][in]: the
// B operand).  Each warpgroup owns a 32 KB activation tile (128 rows x 128
// BF16, the A operand) and 128 columns of tensor memory (its FP32
// accumulator, row t in lane t).  Thread t of a warpgroup is network row t
// throughout: it writes its input row, and after each layer's MMAs (issued by
// the warpgroup's first thread, completion signalled on the warpgroup's
// mbarrier) reads its accumulator row from tensor memory, adds the bias,
// applies GELU on FP32 pairs and writes the BF16 activations back into the
// tile as the next layer's A operand.  The four warpgroups run independently,
// so one's GELU epilogue overlaps the others' MMAs.
// ---------------------------------------------------------------------------
namespace tcn {
constexpr int WG = 4;                                    // warpgroups per CTA
constexpr int ROWS = 128;                                // rows per warpgroup tile (MMA M)
constexpr uint32_t OFF_W4 = 0;                           // [16 out][128 in]
constexpr uint32_t OFF_W1 = OFF_W4 + DOUTP * H * 2;      // [128 out][16 in]
constexpr uint32_t OFF_W2 = OFF_W1 + H * DINP * 2;       // [128 out][128 in]
constexpr uint32_t OFF_W3 = OFF_W2 + H * H * 2;
constexpr uint32_t OFF_ACT = OFF_W3 + H * H * 2;         // per-warpgroup activation tiles
constexpr uint32_t ACT_BYTES = ROWS * H * 2;
constexpr uint32_t OFF_BIAS = OFF_ACT + WG * ACT_BYTES;  // b1, b2, b3 [128], b4 [16]
constexpr uint32_t OFF_NORM = OFF_BIAS + (3 * H + DOUTP) * 4;
constexpr uint32_t OFF_BAR = OFF_NORM + 2 * DOUT * 4;    // one mbarrier per warpgroup
constexpr uint32_t OFF_TSLOT = OFF_BAR + WG * 8;         // tensor-memory address
constexpr uint32_t SMEM = OFF_TSLOT + 16;
constexpr uint32_t TMEM_COLS = WG * 128;
constexpr uint32_t SBO_K16 = (DINP / 8) * 128, SBO_K128 = (H / 8) * 128;
constexpr uint32_t IDESC_HID = tc::idesc_bf16_f32(ROWS, H), IDESC_OUT = tc::idesc_bf16_f32(ROWS, DOUTP);
constexpr int WAIT_POLLS = 1 << 22;
static_assert(OFF_BAR % 8 == 0, "mbarriers need 8-byte alignment");
static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
// every descriptor of a misread layout would still address this CTA's own
// shared memory: the largest reach of a 128 x 128 tile is 32 KB from its start
static_assert(OFF_W4 + ROWS * H * 2 <= SMEM && OFF_ACT + WG * ACT_BYTES <= SMEM, "operand reach");

struct Ctx {
  unsigned char *smem;
  uint32_t sbase;    // shared address of smem
  uint32_t act;      // shared address of this warpgroup's activation tile
  uint32_t tmem_d;   // this warpgroup's accumulator (lane 0, its first column)
  uint32_t tmem_t;   // the same with this thread's warp's lane quarter
  uint64_t *bar;
  uint32_t bar_id;   // named barrier of this warpgroup (1..4)
  int row;           // 0..127
};

// Copies the packed BF16 weights into the UMMA layout and the biases and
// target normalisation into shared memory (whole CTA).
// Two rewrites of the network for the tensor cores.  Layer 1's FP32 bias
// enters the MMA as three BF16 terms (b = hi + mid + lo to FP32 precision) in
// W1's input rows 7, 8, 9 (zero pads of the packed weights), fed by constant
// ones in the input: the accumulator equals the unfolded one up to FP32
// rounding.  The hidden activations are stored as 2 GELU(z) = z (1 + t) with
// W2, W3, W4 halved: scalings by powers of two are exact in BF16 and in the
// FP32 products, so this one changes nothing.
constexpr int BIAS_TERMS = 3;
static_assert(DIN + BIAS_TERMS <= DINP, "the bias terms need padded input columns");
__device__ __forceinline__ bf16 bias_term(float b, int k) {
  const bf16 hi = __float2bfloat16(b);
  const float r1 = b - __bfloat162float(hi);
  const bf16 mid = __float2bfloat16(r1);
  if (k == 0) return hi;
  if (k == 1) return mid;
  return __float2bfloat16(r1 - __bfloat162float(mid));
}
__device__ void stage_network(const SurrogateDev &sd, unsigned char *smem) {
  const bf16 *W1 = static_cast<const bf16 *>(sd.W1), *W2 = static_cast<const bf16 *>(sd.W2);
  const bf16 *W3 = static_cast<const bf16 *>(sd.W3), *W4 = static_cast<const bf16 *>(sd.W4);
  const bf16 half = __float2bfloat16(0.5f);
  for (int e = threadIdx.x; e < DINP * H; e += blockDim.x) {
    const int k = e / H, o = e % H;
    const bf16 w = (k >= DIN && k < DIN + BIAS_TERMS) ? bias_term(sd.b1[o], k - DIN) : W1[e];
    *reinterpret_cast<bf16 *>(smem + OFF_W1 + tc::kmajor_offset(o, k, DINP)) = w;
  }
  for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
    const int k = e / H, o = e % H;
    *reinterpret_cast<bf16 *>(smem + OFF_W2 + tc::kmajor_offset(o, k, H)) = __hmul(W2[e], half);
    *reinterpret_cast<bf16 *>(smem + OFF_W3 + tc::kmajor_offset(o, k, H)) = __hmul(W3[e], half);
  }
  for (int e = threadIdx.x; e < H * DOUTP; e += blockDim.x) {
    const int k = e / DOUTP, o = e % DOUTP;
    *reinterpret_cast<bf16 *>(smem + OFF_W4 + tc::kmajor_offset(o, k, H)) = __hmul(W4[e], half);
  }
  float *bias = reinterpret_cast<float *>(smem + OFF_BIAS);
  for (int e = threadIdx.x; e < H; e += blockDim.x) {
    bias[e] = sd.b1[e];
    bias[H + e] = sd.b2[e];
    bias[2 * H + e] = sd.b3[e];
  }
  if (threadIdx.x < DOUTP) bias[3 * H + threadIdx.x] = sd.b4[threadIdx.x];
  if (threadIdx.x < 2 * DOUT) reinterpret_cast<float *>(smem + OFF_NORM)[threadIdx.x] = sd.norm[threadIdx.x];
}

// CTA set-up: network staged, mbarriers initialised, 512 tensor-memory
// columns allocated by warp 0; returns this thread's view.
__device__ Ctx setup(const SurrogateDev &sd, unsigned char *smem) {
  stage_network(sd, smem);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
  uint32_t *slot = reinterpret_cast<uint32_t *>(smem + OFF_TSLOT);
  if (threadIdx.x < WG) tc::mbar_init1(bars + threadIdx.x);
  if (threadIdx.x < 32) {
    tc::tmem_alloc(slot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  Ctx c;
  const int wg = threadIdx.x >> 7;
  c.smem = smem;
  c.sbase = tc::smem_u32(smem);
  c.row = threadIdx.x & 127;
  c.act = c.sbase + OFF_ACT + wg * ACT_BYTES;
  c.tmem_d = *slot + wg * 128;
  c.tmem_t = c.tmem_d + ((uint32_t)((c.row >> 5) * 32) << 16);
  c.bar = bars + wg;
  c.bar_id = 1 + wg;
  return c;
}

// Barrier of the warpgroup that also ORs a flag over its threads (one
// instruction), so a give-up decision is the warpgroup's, never one thread's.
__device__ __forceinline__ bool sync_or(uint32_t id, bool flag) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, 128, pi;\n"
      " selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)flag), "r"(id)
      : "memory");
  return out != 0;
}

// This thread's input row (7 normalised values, zero padded to 16) as BF16
// into the activation tile, in the K = 16 layout of layer 1.
__device__ __forceinline__ void write_input(const Ctx &c, const float (&u)[DIN]) {
  uint32_t w[8];
  // columns DIN .. DIN + 2 are the constant ones that carry layer 1's bias
  const auto col = [&](int k) { return k < DIN ? u[k] : (k < DIN + BIAS_TERMS ? 1.f : 0.f); };
#pragma unroll
  for (int q = 0; q < 8; ++q) w[q] = pack_bf16x2(col(2 * q), col(2 * q + 1));
  tc::st_shared_v4(c.act + tc::kmajor_offset(c.row, 0, DINP), w[0], w[1], w[2], w[3]);
  tc::st_shared_v4(c.act + tc::kmajor_offset(c.row, 8, DINP), w[4], w[5], w[6], w[7]);
}

// One layer's MMAs by the warpgroup's first thread: D = A W^T over `ksteps`
// slices of 16, then a completion arrive on the warpgroup's mbarrier.
__device__ __forceinline__ void issue(const Ctx &c, uint32_t w_off, uint32_t a_sbo, uint32_t b_sbo, int ksteps,
                                      uint32_t idesc) {
  if (c.row != 0) return;
  tc::fence_after_sync();
  const uint32_t wb = c.sbase + w_off;
  for (int ks = 0; ks < ksteps; ++ks)
    tc::mma_bf16(c.tmem_d, tc::smem_desc(c.act + ks * 256, 128, a_sbo), tc::smem_desc(wb + ks * 256, 128, b_sbo),
                 idesc, ks > 0 ? 1u : 0u);
  tc::mma_commit(c.bar);
}

// Bounded wait for the layer's MMAs; false (this thread gave up) after the bound.
__device__ __forceinline__ bool wait_mma(const Ctx &c, uint32_t &phase) {
  const bool ok = tc::mbar_wait(c.bar, phase, WAIT_POLLS);
  phase ^= 1u;
  tc::fence_after_sync();
  return ok;
}

// z (1 + tanh(z (k + a k z^2))) = 2 GELU(z) on FP32 pairs, the same operations
// in the same order as gelu_x2 without its final halving (see stage_network).
__device__ __forceinline__ float2 gelu2_x2(float2 z) {
  const float2 arg = __fmul2_rn(z, __ffma2_rn(__fmul2_rn(z, z), make_float2(GELU_AK, GELU_AK),
                                              make_float2(GELU_K, GELU_K)));
  return __ffma2_rn(z, make_float2(tanh_approx(arg.x), tanh_approx(arg.y)), z);
}

// Hidden-layer epilogue of this thread's row: accumulator (+ bias for layers
// 2 and 3; layer 1's is in the MMA), 2 GELU, BF16, stored as the next layer's A
// operand (K = 128 layout).  16 columns at a time, the load of the next 16
// in flight while these are evaluated.
template <bool BIAS>
__device__ __forceinline__ void hidden_epilogue(const Ctx &c, const float *bias) {
  uint32_t va[16], vb[16];
  tc::tmem_ld16(c.tmem_t, va);
  tc::tmem_wait_ld(va);
#pragma unroll
  for (int cc = 0; cc < H / 16; ++cc) {
    uint32_t(&cur)[16] = (cc & 1) ? vb : va;
    uint32_t(&nxt)[16] = (cc & 1) ? va : vb;
    if (cc + 1 < H / 16) tc::tmem_ld16(c.tmem_t + (cc + 1) * 16, nxt);
    uint32_t w[8];
    const float2 *b2 = reinterpret_cast<const float2 *>(bias + cc * 16);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float2 z = make_float2(__uint_as_float(cur[2 * q]), __uint_as_float(cur[2 * q + 1]));
      if (BIAS) z = __fadd2_rn(z, b2[q]);
      const float2 gz = gelu2_x2(z);
      w[q] = pack_bf16x2(gz.x, gz.y);
    }
    tc::st_shared_v4(c.act + tc::kmajor_offset(c.row, cc * 16, H), w[0], w[1], w[2], w[3]);
    tc::st_shared_v4(c.act + tc::kmajor_offset(c.row, cc * 16 + 8, H), w[4], w[5], w[6], w[7]);
    if (cc + 1 < H / 16) tc::tmem_wait_ld(nxt);
  }
}

// The whole network for the warpgroup's tile (every thread's input row
// already written): o receives this thread's 16 output columns (10 used,
// bias added, still standardised).  Returns false, uniformly over the
// warpgroup, when a completion wait gave up (then *gave_up is set).
__device__ bool forward(const Ctx &c, uint32_t &phase, float (&o)[DOUTP], bool &gave_up) {
  const float *bias = reinterpret_cast<const float *>(c.smem + OFF_BIAS);
  bool bad = false;
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  // a wait given up in the previous tile ends the warpgroup's work here
  if (sync_or(c.bar_id, gave_up)) {
    gave_up = true;
    return false;
  }
  issue(c, OFF_W1, SBO_K16, SBO_K16, DINP / 16, IDESC_HID);
#pragma unroll 1
  for (int layer = 0; layer < 3; ++layer) {
    bad = !wait_mma(c, phase) || bad;
    if (layer == 0)
      hidden_epilogue<false>(c, bias);
    else
      hidden_epilogue<true>(c, bias + layer * H);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    if (sync_or(c.bar_id, bad)) {
      gave_up = true;
      return false;
    }
    if (layer < 2)
      issue(c, layer == 0 ? OFF_W2 : OFF_W3, SBO_K128, SBO_K128, H / 16, IDESC_HID);
    else
      issue(c, OFF_W4, SBO_K128, SBO_K128, H / 16, IDESC_OUT);
  }
  bad = !wait_mma(c, phase) || bad;
  uint32_t v[16];
  tc::tmem_ld16(c.tmem_t, v);
  tc::tmem_wait_ld(v);
#pragma unroll
  for (int k = 0; k < DOUTP; ++k) o[k] = __uint_as_float(v[k]) + bias[3 * H + k];
  // the next tile's first barrier orders these reads before its MMAs
  tc::fence_before_sync();
  if (bad) gave_up = true;
  return true;
}

// CTA tear-down: every warpgroup done with tensor memory, warp 0 frees it.
// A warpgroup that gave up first lets its last MMAs finish (bounded).
__device__ void teardown(const Ctx &c, uint32_t phase, bool gave_up, int *status) {
  if (sync_or(c.bar_id, gave_up) && c.row == 0) {
    tc::mbar_wait(c.bar, phase ^ 1u, WAIT_POLLS);
    if (status) atomicOr(status, ERR_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*reinterpret_cast<const uint32_t *>(c.smem + OFF_TSLOT) , TMEM_COLS);
  }
}

}  // namespace tcn

// Network prediction of raw problems x [B][7] -> outputs y [B][10]
// (de-normalised, moments form) on the tensor cores.
__global__ void __launch_bounds__(tcn::WG * 128, 1)
    predict_tc_kernel(SurrogateDev sd, const float *x, float *y, int64_t B, int *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const tcn::Ctx c = tcn::setup(sd, smem);
  const int wg = threadIdx.x >> 7;
  const float *norm = reinterpret_cast<const float *>(smem + tcn::OFF_NORM);
  const int64_t ntiles = (B + tcn::ROWS - 1) / tcn::ROWS;
  uint32_t phase = 0;
  bool gave_up = false;
  for (int64_t tile = (int64_t)blockIdx.x * tcn::WG + wg; tile < ntiles; tile += (int64_t)gridDim.x * tcn::WG) {
    const int64_t b = tile * tcn::ROWS + c.row;
    float u[DIN];
    if (b < B) {
      normalise_input(x + b * DIN, u);
    } else {
#pragma unroll
      for (int t = 0; t < DIN; ++t) u[t] = 0.f;
    }
    tcn::write_input(c, u);
    float o[DOUTP];
    if (!tcn::forward(c, phase, o, gave_up)) break;
    if (b < B) {
      float t[DOUT];
#pragma unroll
      for (int k = 0; k < DOUT; ++k) t[k] = fmaf(o[k], norm[DOUT + k], norm[k]);
      from_net(t, y + b * DOUT);
    }
  }
  tcn::teardown(c, phase, gave_up, status);
}

// Fused surrogate E-step on the tensor cores.  A warpgroup tile is 64 pairs
// of one component as 128 network rows: row 2k is pair k's pass A (dof
// nu + p), row 2k + 1 its pass B (nu + p + 2), so a pair's two rows sit in
// adjacent lanes of one warp; for the density alone a tile is 128 pairs, one
// row each (pass A).  Each thread prepares its row's standardised problem
// (FP32 prologue), runs the network, and the pair's two threads form log f
// and e1..e4 from the two output rows (the even thread log f, e1, e2, e3;
// the odd thread e4).  Pairs outside the training domain are appended to the
// lattice rule's list (one atomic per warp).
template <bool DENS>
__global__ void __launch_bounds__(tcn::WG * 128, 1)
    surrogate_estep_tc_kernel(SurrogateDev sd, const double *Y, int64_t n, int g, int p,
                              const CompT<float> *__restrict__ comp, EstepOut out, int *fb_list, unsigned *fb_count,
                              int *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const tcn::Ctx c = tcn::setup(sd, smem);
  const int wg = threadIdx.x >> 7, lane = threadIdx.x & 31;
  const float *mean = reinterpret_cast<const float *>(smem + tcn::OFF_NORM), *sdv = mean + DOUT;
  constexpr int PPT = DENS ? tcn::ROWS : tcn::ROWS / 2;  // pairs per tile
  const int64_t tpc = (n + PPT - 1) / PPT;
  const int64_t ntiles = tpc * g;
  const int pair = DENS ? c.row : c.row >> 1, pass = DENS ? 0 : (c.row & 1);
  uint32_t phase = 0;
  bool gave_up = false;
  // the tile's component i and its place tr among that component's tiles,
  // advanced by additions (one 64-bit division per thread, before the loop)
  const int64_t stride = (int64_t)gridDim.x * tcn::WG;
  const int64_t tile0 = (int64_t)blockIdx.x * tcn::WG + wg;
  int i = (int)(tile0 / tpc);
  int64_t tr = tile0 - (int64_t)i * tpc;
  const auto advance = [&](int &ci, int64_t &ct) {
    ct += stride;
    while (ct >= tpc) {
      ct -= tpc;
      ++ci;
    }
  };
  for (int64_t tile = tile0; tile < ntiles; tile += stride, advance(i, tr)) {
    const int64_t j = tr * PPT + pair;
    const CompT<float> &cp = comp[i];
    const bool valid = j < n;
    {
      // this row's observation in the warpgroup's next tile, brought into L1
      // while this tile runs through the network
      int in = i;
      int64_t trn = tr;
      advance(in, trn);
      const int64_t jn = trn * PPT + pair;
      if (tile + stride < ntiles && jn < n) tc::prefetch_l1(Y + jn * p);
    }
    RowProblem rp;
    float u[DIN];
    if (valid) {
      rp = row_problem(cp, Y, p, j, pass);
      network_input(rp, u);
    } else {
      rp.kind = -1;
#pragma unroll
      for (int t = 0; t < DIN; ++t) u[t] = 0.f;
    }
    tcn::write_input(c, u);
    // pairs outside the domain go to the lattice rule's list: one atomic per warp
    const bool push = valid && pass == 0 && rp.kind != 2;
    const unsigned pm = __ballot_sync(0xffffffffu, push);
    if (pm) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(fb_count + i, (unsigned)__popc(pm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (push) fb_list[(int64_t)i * n + base + __popc(pm & ((1u << lane) - 1u))] = (int)j;
    }
    float o[DOUTP];
    if (!tcn::forward(c, phase, o, gave_up)) break;

    const int64_t ij = (int64_t)i * n + j;
    // this row's log T (pass A: T_A, pass B: T_B) and standardised first moments
    const float logT = -__expf(fmaf(o[0], sdv[0], mean[0]));
    float EX[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) EX[t] = fmaf(o[1 + t], sdv[1 + t], mean[1 + t]);
    if (DENS) {
      if (valid) {
        float *lf = static_cast<float *>(out.logf);
        if (rp.kind == 2) lf[ij] = rp.logt + logT;
        if (rp.kind == 0) lf[ij] = INFINITY;
        if (rp.kind == 1) {
          // the lattice rule's triage bound: log T is decreasing in every c_t,
          // so the network at the box-clamped point plus a margin bounds it;
          // and P(X > c) <= P(X_t > c_t) <= (m + c_t^2) f_m(c_t) / ((m - 1) c_t)
          // for c_t > 0 (f_m the t_m density), tightest at pass A's largest coordinate
          float ub = logT + UB_MARGIN;
          const float cmx = rp.cmaxA, m = cp.fmA;
          if (cmx > 0.f && m > 1.f) {
            const float lnorm = lgammaf(0.5f * (m + 1.f)) - lgammaf(0.5f * m) - 0.5f * logf(m * 3.14159265f);
            const float lb =
                logf((m + cmx * cmx) / ((m - 1.f) * cmx)) + lnorm - 0.5f * (m + 1.f) * log1pf(cmx * cmx / m);
            ub = fminf(ub, lb + 1e-3f);
          }
          lf[ij] = rp.logt + ub;
        }
      }
      continue;
    }
    // the pair's other row: pass A's log T for the odd thread, pass B's log T
    // and first moments for the even one
    const float logT_o = __shfl_xor_sync(0xffffffffu, logT, 1);
    float EX_o[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) EX_o[t] = __shfl_xor_sync(0xffffffffu, EX[t], 1);
    if (!valid) continue;
    const float logTA = pass ? logT_o : logT, logTB = pass ? logT : logT_o;
    const float *EXB = pass ? EX : EX_o;
    if (pass == 0) {
      float *lf = static_cast<float *>(out.logf);
      if (rp.kind == 1) {
        float ub = logTA + UB_MARGIN;
        const float cmx = rp.cmaxA, m = cp.fmA;
        if (cmx > 0.f && m > 1.f) {
          const float lnorm = lgammaf(0.5f * (m + 1.f)) - lgammaf(0.5f * m) - 0.5f * logf(m * 3.14159265f);
          const float lb =
              logf((m + cmx * cmx) / ((m - 1.f) * cmx)) + lnorm - 0.5f * (m + 1.f) * log1pf(cmx * cmx / m);
          ub = fminf(ub, lb + 1e-3f);
        }
        lf[ij] = rp.logt + ub;
      }
      if (rp.kind == 0) lf[ij] = INFINITY;
    }
    if (rp.kind != 2) continue;
    const float nud = rp.nud, mA = cp.fmA, mB = cp.fmB;
    const float e1 = mA / nud * __expf(logTB - logTA);
    const float sig = sqrtf(nud / mB);
    // E[X] and E[X X^T] of pass B in the Lambda basis: D^{1/2} (.) D^{1/2}
    const float L00 = cp.L[0], L10 = cp.L[RMAX], L11 = cp.L[RMAX + 1];
    const float L20 = cp.L[2 * RMAX], L21 = cp.L[2 * RMAX + 1], L22 = cp.L[2 * RMAX + 2];
    const float sD[3] = {fabsf(L00), sqrtf(fmaf(L10, L10, L11 * L11)), sqrtf(fmaf(L20, L20, fmaf(L21, L21, L22 * L22)))};
    float LEV[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) LEV[t] = sD[t] * EXB[t];
    if (pass == 0) {
      static_cast<float *>(out.logf)[ij] = rp.logt + logTA;
      static_cast<float *>(out.e1)[ij] = e1;
      static_cast<float *>(out.e2)[ij] = e1 - (logf(0.5f * nud) + mA / nud - cp.fpsiA);
#pragma unroll
      for (int t = 0; t < 3; ++t)
        static_cast<float *>(out.e3)[((int64_t)i * 3 + t) * n + j] = e1 * fmaf(sig, LEV[t], rp.q[t]);
    } else {
      // e4 in lower-triangle order from the network's covariance (upper order
      // 00 01 02 11 12 22): E[X'_h X'_t] = cov + E[X'_h] E[X'_t]
      constexpr int UP[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
      float cv[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) cv[q] = fmaf(o[4 + q], sdv[4 + q], mean[4 + q]);
      psd_repair3(cv);
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int h = 0; h <= t; ++h) {
          const float Sth = sD[t] * sD[h] * fmaf(EXB[h], EXB[t], cv[UP[t][h]]);
          const float exx = rp.q[t] * rp.q[h] + sig * (rp.q[t] * LEV[h] + LEV[t] * rp.q[h]) + sig * sig * Sth;
          static_cast<float *>(out.e4)[((int64_t)i * 6 + t * (t + 1) / 2 + h) * n + j] = e1 * exx;
        }
    }
  }
  tcn::teardown(c, phase, gave_up, status);
}

// The standardised problems (network inputs of pass A and pass B) of every
// stride-th (i, j) pair in the network's domain, appended to x_out [max_rows][7]
// two rows per pair; *count receives the number of rows wanted.
__global__ void problems_kernel(const double *Y, int64_t n, int g, int p, const CompT<float> *comp, int64_t stride,
                                float *x_out, int64_t max_rows, unsigned long long *count) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * stride;
  if (k >= (int64_t)g * n) return;
  const int i = (int)(k / n);
  const int64_t j = k % n;
  const RowProblem ra = row_problem(comp[i], Y, p, j, 0);
  if (ra.kind != 2) return;
  const RowProblem rb = row_problem(comp[i], Y, p, j, 1);
  const unsigned long long slot = atomicAdd(count, 2ull);
  if ((int64_t)slot + 2 > max_rows) return;
  float *xa = x_out + (int64_t)slot * DIN;
  const RowProblem *rr[2] = {&ra, &rb};
  for (int q = 0; q < 2; ++q) {
    float *xr = xa + q * DIN;
    for (int t = 0; t < 3; ++t) xr[t] = rr[q]->c[t];
    for (int t = 0; t < 3; ++t) xr[3 + t] = rr[q]->R[t];
    xr[6] = rr[q]->logm;
  }
}

}  // namespace sg
}  // namespace cfust

namespace cfust {

cudaError_t launch_surrogate_problems(const double *Y, int64_t n, int g, int p, const CompT<float> *c32,
                                      int64_t stride, float *x_out, int64_t max_rows, unsigned long long *count,
                                      cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int64_t m = ((int64_t)g * n + stride - 1) / stride;
  if (m <= 0) return cudaSuccess;
  sg::problems_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(Y, n, g, p, c32, stride, x_out, max_rows, count);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_inputs(const double *Y, int64_t n, int g, int p, const CompT<float> *c32, float *x_out,
                                    int *kind, cudaStream_t st) {
  const int64_t m = 2 * (int64_t)g * n;
  if (m <= 0) return cudaSuccess;
  sg::inputs_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(Y, n, g, p, c32, x_out, kind);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_estep(const SurrogateDev &sd, const double *Y, int64_t n, int g, int p,
                                   const CompT<float> *c32, EstepOut out, bool density_only, int *fb_list,
                                   unsigned *fb_count, int *status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(fb_count, 0, sizeof(unsigned) * g, st);
  if (e != cudaSuccess || n <= 0) return e;
  const int smem = (int)sg::tcn::SMEM;
  const int64_t ppt = density_only ? sg::tcn::ROWS : sg::tcn::ROWS / 2;
  const int64_t ntiles = (n + ppt - 1) / ppt * g;
  const int sms = sm_count();
  int64_t blocks = (ntiles + sg::tcn::WG - 1) / sg::tcn::WG;
  if (blocks > sms) blocks = sms;
  if (density_only) {
    e = raise_smem_limit((const void *)sg::surrogate_estep_tc_kernel<true>, (size_t)(smem));
    if (e != cudaSuccess) return e;
    sg::surrogate_estep_tc_kernel<true><<<(unsigned)blocks, sg::tcn::WG * 128, smem, st>>>(sd, Y, n, g, p, c32, out,
                                                                                           fb_list, fb_count, status);
  } else {
    e = raise_smem_limit((const void *)sg::surrogate_estep_tc_kernel<false>, (size_t)(smem));
    if (e != cudaSuccess) return e;
    sg::surrogate_estep_tc_kernel<false><<<(unsigned)blocks, sg::tcn::WG * 128, smem, st>>>(
        sd, Y, n, g, p, c32, out, fb_list, fb_count, status);
  }
  return cudaGetLastError();
}

}  // namespace cfust

using namespace cfust;
using namespace cfust::sg;

struct cfust_surrogate {
  int device = 0;
  cudaStream_t stream = nullptr;
  LatticeDev lat{};
  std::string err;
  float *tab = nullptr;               // chi tables [MGRID][N]
  float *theta = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr;
  float *norm = nullptr;              // [20] target mean, std
  float host_norm[20];
  bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr;
  float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr, *b4 = nullptr;
  int64_t cap = 0;                    // rows the work buffers hold
  bf16 *x0 = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Z3 = nullptr, *H3 = nullptr;
  float *out = nullptr;
  bf16 *dz4 = nullptr, *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
  float *part = nullptr;
  int64_t part_len = 0;
  double *loss_part = nullptr;
  int *d_status = nullptr;            // error bits of the network kernels
  int adam_t = 0;
};

namespace cfust {
SurrogateDev surrogate_dev(const cfust_surrogate *s) {
  SurrogateDev d;
  d.W1 = s->W1;
  d.W2 = s->W2;
  d.W3 = s->W3;
  d.W4 = s->W4;
  d.b1 = s->b1;
  d.b2 = s->b2;
  d.b3 = s->b3;
  d.b4 = s->b4;
  d.norm = s->norm;
  return d;
}
}  // namespace cfust

namespace {

thread_local std::string g_sg_error;

cfust_status sg_fail(cfust_surrogate *s, cfust_status st, const std::string &m) {
  if (s) s->err = m; else g_sg_error = m;
  return st;
}

#define SG_CUDA(s, call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return sg_fail((s), CFUST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cfust_status ensure_rows(cfust_surrogate *s, int64_t B) {
  if (B <= s->cap) return CFUST_OK;
  void **bufs[] = {(void **)&s->x0, (void **)&s->Z1, (void **)&s->H1, (void **)&s->Z2,
                   (void **)&s->H2, (void **)&s->Z3, (void **)&s->H3, (void **)&s->out,
                   (void **)&s->dz4, (void **)&s->dz3, (void **)&s->dz2, (void **)&s->dz1};
  for (void **p : bufs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  s->cap = 0;
  SG_CUDA(s, cudaMalloc(&s->x0, sizeof(bf16) * B * DINP));
  SG_CUDA(s, cudaMalloc(&s->Z1, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->H1, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->Z2, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->H2, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->Z3, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->H3, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->out, sizeof(float) * B * DOUTP));
  SG_CUDA(s, cudaMalloc(&s->dz4, sizeof(bf16) * B * DOUTP));
  SG_CUDA(s, cudaMalloc(&s->dz3, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->dz2, sizeof(bf16) * B * H));
  SG_CUDA(s, cudaMalloc(&s->dz1, sizeof(bf16) * B * H));
  s->cap = B;
  return CFUST_OK;
}

Gemm fwd_layer(const bf16 *A, int K, const bf16 *W, int N, const float *bias, bf16 *Z, bf16 *Hh, int64_t B) {
  Gemm g{};
  g.M = (int)B;
  g.N = N;
  g.K = K;
  g.A = A;
  g.lda = K;
  g.transA = 0;
  g.B = W;
  g.ldb = N;
  g.transB = 0;
  g.k_chunk = K;
  g.mode = 1;
  g.bias = bias;
  g.Zout = Z;
  g.Hout = Hh;
  g.ldo = N;
  return g;
}

// forward pass of rows [0, B) from the packed inputs x0; network output in s->out
cfust_status forward(cfust_surrogate *s, int64_t B) {
  SG_CUDA(s, gemm(fwd_layer(s->x0, DINP, s->W1, H, s->b1, s->Z1, s->H1, B), 1, s->stream, s->d_status));
  SG_CUDA(s, gemm(fwd_layer(s->H1, H, s->W2, H, s->b2, s->Z2, s->H2, B), 1, s->stream, s->d_status));
  SG_CUDA(s, gemm(fwd_layer(s->H2, H, s->W3, H, s->b3, s->Z3, s->H3, B), 1, s->stream, s->d_status));
  Gemm g = fwd_layer(s->H3, H, s->W4, DOUTP, s->b4, nullptr, nullptr, B);
  g.mode = 3;
  g.C = s->out;
  g.ldc = DOUTP;
  SG_CUDA(s, gemm(g, 1, s->stream, s->d_status));
  return CFUST_OK;
}

// gradient of the weights: dW = Hin^T dZ (split-K over rows) into grad[off]
cfust_status weight_grad(cfust_surrogate *s, const bf16 *Hin, int kin, int kin_real, const bf16 *dZ, int nout,
                         int nout_real, int64_t B, int off) {
  const int chunk = 256;
  const int S = (int)((B + chunk - 1) / chunk);
  const int64_t need = (int64_t)S * kin * nout;
  if (need > s->part_len) {
    if (s->part) cudaFree(s->part);
    s->part = nullptr;
    s->part_len = 0;
    SG_CUDA(s, cudaMalloc(&s->part, sizeof(float) * need));
    s->part_len = need;
  }
  Gemm g{};
  g.M = kin;
  g.N = nout;
  g.K = (int)B;
  g.A = Hin;
  g.lda = kin;
  g.transA = 1;
  g.B = dZ;
  g.ldb = nout;
  g.transB = 0;
  g.k_chunk = chunk;
  g.mode = 0;
  g.C = s->part;
  g.ldc = nout;
  SG_CUDA(s, gemm(g, S, s->stream, s->d_status));
  const int cnt = kin_real * nout_real;
  reduce_partials_kernel<<<(cnt + 255) / 256, 256, 0, s->stream>>>(s->part, S, kin, nout, kin_real, nout_real,
                                                                   s->grad, off);
  SG_CUDA(s, cudaGetLastError());
  return CFUST_OK;
}

// input gradient through a layer: dZprev = (dZ W^T) * GELU'(Zprev)
cfust_status back_layer(cfust_surrogate *s, const bf16 *dZ, int nout, const bf16 *W, int kin, const bf16 *Zprev,
                        bf16 *dZprev, int64_t B) {
  Gemm g{};
  g.M = (int)B;
  g.N = kin;
  g.K = nout;
  g.A = dZ;
  g.lda = nout;
  g.transA = 0;
  g.B = W;
  g.ldb = nout;
  g.transB = 1;
  g.k_chunk = nout;
  g.mode = 2;
  g.Hout = dZprev;
  g.ldo = kin;
  g.Zprev = Zprev;
  return gemm(g, 1, s->stream, s->d_status) == cudaSuccess ? CFUST_OK : sg_fail(s, CFUST_ECUDA, "gemm (backward)");
}

// loss and full gradient (into s->grad) of rows [0, B) with raw targets y
cfust_status loss_grad(cfust_surrogate *s, const float *y, int64_t B, double *loss) {
  cfust_status st = forward(s, B);
  if (st != CFUST_OK) return st;
  const int nb = 256;
  loss_kernel<<<nb, 256, 0, s->stream>>>(s->out, y, s->norm, s->dz4, s->loss_part, B);
  SG_CUDA(s, cudaGetLastError());
  if ((st = weight_grad(s, s->H3, H, H, s->dz4, DOUTP, DOUT, B, OFF_W4)) != CFUST_OK) return st;
  colsum_kernel<<<DOUTP, 256, 0, s->stream>>>(s->dz4, DOUTP, DOUT, B, s->grad, OFF_B4);
  if ((st = back_layer(s, s->dz4, DOUTP, s->W4, H, s->Z3, s->dz3, B)) != CFUST_OK) return st;
  if ((st = weight_grad(s, s->H2, H, H, s->dz3, H, H, B, OFF_W3)) != CFUST_OK) return st;
  colsum_kernel<<<H, 256, 0, s->stream>>>(s->dz3, H, H, B, s->grad, OFF_B3);
  if ((st = back_layer(s, s->dz3, H, s->W3, H, s->Z2, s->dz2, B)) != CFUST_OK) return st;
  if ((st = weight_grad(s, s->H1, H, H, s->dz2, H, H, B, OFF_W2)) != CFUST_OK) return st;
  colsum_kernel<<<H, 256, 0, s->stream>>>(s->dz2, H, H, B, s->grad, OFF_B2);
  if ((st = back_layer(s, s->dz2, H, s->W2, H, s->Z1, s->dz1, B)) != CFUST_OK) return st;
  if ((st = weight_grad(s, s->x0, DINP, DIN, s->dz1, H, H, B, OFF_W1)) != CFUST_OK) return st;
  colsum_kernel<<<H, 256, 0, s->stream>>>(s->dz1, H, H, B, s->grad, OFF_B1);
  SG_CUDA(s, cudaGetLastError());
  if (loss) {
    std::vector<double> lp(nb);
    SG_CUDA(s, cudaMemcpyAsync(lp.data(), s->loss_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(s, cudaStreamSynchronize(s->stream));
    double t = 0.0;
    for (double v : lp) t += v;
    *loss = t / ((double)B * DOUT);
  }
  return CFUST_OK;
}

cfust_status pack(cfust_surrogate *s) {
  pack_weights_kernel<<<(H * H + 255) / 256, 256, 0, s->stream>>>(s->theta, s->W1, s->W2, s->W3, s->W4, s->b1, s->b2,
                                                                 s->b3, s->b4);
  SG_CUDA(s, cudaGetLastError());
  return CFUST_OK;
}

cfust_status prep(cfust_surrogate *s, const float *x, int64_t B) {
  cfust_status st = ensure_rows(s, B);
  if (st != CFUST_OK) return st;
  prep_input_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s->stream>>>(x, s->x0, B);
  SG_CUDA(s, cudaGetLastError());
  return CFUST_OK;
}

// Device buffer released when it goes out of scope (error paths included).
struct DevBuf {
  float *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Largest row count of one call: the GEMMs index rows with 32-bit integers.
constexpr int64_t MAX_ROWS = (int64_t)1 << 30;

// SplitMix64 for initial weights and training inputs (host)
struct SplitMix {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * 1.1102230246251565e-16; }
  double normal() {
    const double u1 = uniform() + 1e-300, u2 = uniform();
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
};

// Adam (beta 0.9, 0.999, eps 1e-8) on mini-batches of `batch` consecutive
// rows of (dx, dy), `epochs` passes, step size cosine-decayed from lr over the
// run; loss_trace[ep] = mean of the sampled batch losses of epoch ep.
cfust_status train_loop(cfust_surrogate *s, const float *dx, const float *dy, int64_t rows, int epochs, int batch,
                        float lr, float *loss_trace) {
  cfust_status st = CFUST_OK;
  const int64_t steps = rows / batch;
  for (int ep = 0; ep < epochs; ++ep) {
    double ep_loss = 0.0;
    for (int64_t k = 0; k < steps; ++k) {
      const int64_t off = k * batch;
      if ((st = prep(s, dx + off * DIN, batch)) != CFUST_OK) break;
      double l = 0.0;
      if ((st = loss_grad(s, dy + off * DOUT, batch, (k % 64 == 0) ? &l : nullptr)) != CFUST_OK) break;
      ep_loss += l;
      ++s->adam_t;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f - powf(b1, (float)s->adam_t), c2 = 1.f - powf(b2, (float)s->adam_t);
      const float frac = (float)(ep * steps + k) / (float)(epochs * steps);
      const float lr_t = lr * 0.5f * (1.f + cosf(3.14159265f * frac));
      adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s->stream>>>(s->theta, s->mom, s->vel, s->grad, NPARAM, lr_t, b1,
                                                               b2, 1e-8f, c1, c2);
      if (cudaGetLastError() != cudaSuccess) {
        st = sg_fail(s, CFUST_ECUDA, "adam_kernel launch");
        break;
      }
      if ((st = pack(s)) != CFUST_OK) break;
    }
    if (st != CFUST_OK) break;
    if (loss_trace) loss_trace[ep] = (float)(ep_loss / (double)((steps + 63) / 64));
  }
  if (st != CFUST_OK) return st;
  SG_CUDA(s, cudaStreamSynchronize(s->stream));
  return CFUST_OK;
}

}  // namespace

extern "C" {

cfust_status cfust_surrogate_create(cfust_surrogate **out, uint64_t seed, const cfust_lattice *L, void *stream) {
  if (!out || !L) return sg_fail(nullptr, CFUST_EINVAL, "out and lattice required");
  *out = nullptr;
  if (L->dim != 4 || L->n < 32 || L->n % 32 != 0 || L->n > CFUST_NMAX || !L->z || !L->shift)
    return sg_fail(nullptr, CFUST_EINVAL, "surrogate lattice must have dim 4 and a multiple of 32 points");
  cfust_surrogate *s = new cfust_surrogate();
  s->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&s->device);
  s->lat.n = L->n;
  for (int t = 0; t <= RMAX; ++t) {
    if (t < 4) {
      int64_t zz = L->z[t] % L->n;
      if (zz < 0) zz += L->n;
      s->lat.z[t] = (int)zz;
      s->lat.step[t] = (int)((32 * zz) % L->n);
      s->lat.shift[t] = L->shift[t];
      const double sn = L->shift[t] * (double)L->n;
      s->lat.sint[t] = (int)floor(sn);
      s->lat.sfrac[t] = sn - floor(sn);
    }
  }
  cfust_surrogate *S = s;
#define CR(call)                                   \
  do {                                             \
    if ((call) != cudaSuccess) {                   \
      g_sg_error = #call;                          \
      cfust_surrogate_destroy(S);                  \
      return CFUST_ECUDA;                          \
    }                                              \
  } while (0)
  CR(cudaMalloc(&s->tab, sizeof(float) * MGRID * (size_t)L->n));
  CR(cudaMalloc(&s->theta, sizeof(float) * NPARAM));
  CR(cudaMalloc(&s->mom, sizeof(float) * NPARAM));
  CR(cudaMalloc(&s->vel, sizeof(float) * NPARAM));
  CR(cudaMalloc(&s->grad, sizeof(float) * NPARAM));
  CR(cudaMalloc(&s->norm, sizeof(float) * 20));
  CR(cudaMalloc(&s->W1, sizeof(bf16) * DINP * H));
  CR(cudaMalloc(&s->W2, sizeof(bf16) * H * H));
  CR(cudaMalloc(&s->W3, sizeof(bf16) * H * H));
  CR(cudaMalloc(&s->W4, sizeof(bf16) * H * DOUTP));
  CR(cudaMalloc(&s->b1, sizeof(float) * H));
  CR(cudaMalloc(&s->b2, sizeof(float) * H));
  CR(cudaMalloc(&s->b3, sizeof(float) * H));
  CR(cudaMalloc(&s->b4, sizeof(float) * DOUTP));
  CR(cudaMalloc(&s->loss_part, sizeof(double) * 256));
  CR(cudaMalloc(&s->d_status, sizeof(int)));
  CR(cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream));
  CR(cudaMemsetAsync(s->mom, 0, sizeof(float) * NPARAM, s->stream));
  CR(cudaMemsetAsync(s->vel, 0, sizeof(float) * NPARAM, s->stream));
  // initial weights: N(0, 1/fan_in), zero biases; unit target normalisation
  SplitMix rng{seed};
  std::vector<float> th(NPARAM, 0.f);
  const int dims[5] = {DIN, H, H, H, DOUT};
  int off = 0;
  for (int k = 0; k < 4; ++k) {
    const double sd = 1.0 / sqrt((double)dims[k]);
    for (int e = 0; e < dims[k] * dims[k + 1]; ++e) th[off + e] = (float)(sd * rng.normal());
    off += dims[k] * dims[k + 1] + dims[k + 1];
  }
  for (int k = 0; k < 10; ++k) {
    s->host_norm[k] = 0.f;
    s->host_norm[10 + k] = 1.f;
  }
  CR(cudaMemcpy(s->theta, th.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
  CR(cudaMemcpy(s->norm, s->host_norm, sizeof(float) * 20, cudaMemcpyHostToDevice));
  chi_grid_kernel<<<dim3((L->n + 127) / 128, MGRID), 128, 0, s->stream>>>(s->lat, s->tab);
  CR(cudaGetLastError());
  if (pack(s) != CFUST_OK) {
    cfust_surrogate_destroy(s);
    return CFUST_ECUDA;
  }
  CR(cudaStreamSynchronize(s->stream));
#undef CR
  *out = s;
  return CFUST_OK;
}

cfust_status cfust_surrogate_destroy(cfust_surrogate *s) {
  if (!s) return CFUST_OK;
  void *bufs[] = {s->tab, s->theta, s->mom, s->vel, s->grad, s->norm, s->W1, s->W2, s->W3, s->W4, s->b1, s->b2, s->b3,
                  s->b4, s->x0, s->Z1, s->H1, s->Z2, s->H2, s->Z3, s->H3, s->out, s->dz4, s->dz3, s->dz2, s->dz1,
                  s->part, s->loss_part, s->d_status};
  for (void *p : bufs)
    if (p) cudaFree(p);
  delete s;
  return CFUST_OK;
}

const char *cfust_surrogate_last_error(cfust_surrogate *s) { return s ? s->err.c_str() : g_sg_error.c_str(); }

cfust_status cfust_surrogate_label(cfust_surrogate *s, const float *x, float *y, int64_t B) {
  if (!s || !x || !y || B < 0 || B > MAX_ROWS) return sg_fail(s, CFUST_EINVAL, "bad arguments (0 <= B <= 2^30)");
  if (B == 0) return CFUST_OK;
  const int64_t blocks = (B + 7) / 8;
  label_kernel<<<(unsigned)blocks, 256, 0, s->stream>>>(x, y, B, s->lat, s->tab);
  SG_CUDA(s, cudaGetLastError());
  SG_CUDA(s, cudaStreamSynchronize(s->stream));
  return CFUST_OK;
}

cfust_status cfust_surrogate_predict(cfust_surrogate *s, const float *x, float *y, int64_t B) {
  if (!s || !x || !y || B < 0 || B > MAX_ROWS) return sg_fail(s, CFUST_EINVAL, "bad arguments (0 <= B <= 2^30)");
  if (B == 0) return CFUST_OK;
  // the inference network on the tensor cores (tcgen05, accumulators in tensor memory)
  const int64_t ntiles = (B + tcn::ROWS - 1) / tcn::ROWS;
  int64_t blocks = (ntiles + tcn::WG - 1) / tcn::WG;
  if (blocks > sm_count()) blocks = sm_count();
  SG_CUDA(s, raise_smem_limit((const void *)predict_tc_kernel, (size_t)((int)tcn::SMEM)));
  SG_CUDA(s, cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream));
  predict_tc_kernel<<<(unsigned)blocks, tcn::WG * 128, tcn::SMEM, s->stream>>>(surrogate_dev(s), x, y, B,
                                                                               s->d_status);
  SG_CUDA(s, cudaGetLastError());
  int bits = 0;
  SG_CUDA(s, cudaMemcpyAsync(&bits, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  SG_CUDA(s, cudaStreamSynchronize(s->stream));
  if (bits & ERR_TIMEOUT) return sg_fail(s, CFUST_ETIMEOUT, "a bounded tensor-core completion wait ran out");
  return CFUST_OK;
}

cfust_status cfust_surrogate_set_params(cfust_surrogate *s, const float *theta, const float *norm) {
  if (!s || !theta) return sg_fail(s, CFUST_EINVAL, "bad arguments");
  SG_CUDA(s, cudaMemcpy(s->theta, theta, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
  if (norm) {
    memcpy(s->host_norm, norm, sizeof(float) * 20);
    SG_CUDA(s, cudaMemcpy(s->norm, norm, sizeof(float) * 20, cudaMemcpyHostToDevice));
  }
  cfust_status st = pack(s);
  if (st != CFUST_OK) return st;
  SG_CUDA(s, cudaStreamSynchronize(s->stream));
  return CFUST_OK;
}

cfust_status cfust_surrogate_get_params(cfust_surrogate *s, float *theta, float *norm) {
  if (!s) return sg_fail(s, CFUST_EINVAL, "bad arguments");
  SG_CUDA(s, cudaStreamSynchronize(s->stream));
  if (theta) SG_CUDA(s, cudaMemcpy(theta, s->theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
  if (norm) memcpy(norm, s->host_norm, sizeof(float) * 20);
  return CFUST_OK;
}

cfust_status cfust_surrogate_gradient(cfust_surrogate *s, const float *x, const float *y, int64_t B, double *loss,
                                      float *grad) {
  if (!s || !x || !y || B < 1 || B > MAX_ROWS) return sg_fail(s, CFUST_EINVAL, "bad arguments (1 <= B <= 2^30)");
  cfust_status st = prep(s, x, B);
  if (st != CFUST_OK) return st;
  if ((st = loss_grad(s, y, B, loss)) != CFUST_OK) return st;
  if (grad) {
    SG_CUDA(s, cudaMemcpyAsync(grad, s->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  return CFUST_OK;
}

cfust_status cfust_surrogate_train(cfust_surrogate *s, int64_t n_train, int epochs, int batch, float lr,
                                   uint64_t seed, float *loss_trace) {
  if (!s || n_train < batch || batch < 128 || epochs < 1 || !(lr > 0.f))
    return sg_fail(s, CFUST_EINVAL, "need n_train >= batch >= 128, epochs >= 1, lr > 0");
  if (n_train > MAX_ROWS) return sg_fail(s, CFUST_EINVAL, "n_train above 2^30");
  // training inputs drawn on the host over the domain (a box mixture, below),
  // labelled on the GPU
  SplitMix rng{seed};
  std::vector<float> hx(n_train * DIN);
  for (int64_t b = 0; b < n_train; ++b) {
    float *xb = hx.data() + b * DIN;
    for (;;) {
      // half uniform over the box, half c_t ~ N(-1.5, 2.5^2) clipped to it:
      // E-step pairs with weight crowd around moderate negative c
      const bool focus = rng.uniform() < 0.5;
      for (int t = 0; t < 3; ++t) {
        const double v = focus ? -1.5 + 2.5 * rng.normal() : C_LO + rng.uniform() * (C_HI - C_LO);
        xb[t] = (float)fmin(fmax(v, (double)C_LO), (double)C_HI);
      }
      for (int t = 3; t < 6; ++t) xb[t] = (float)((2.0 * rng.uniform() - 1.0) * RHO_MAX);
      xb[6] = (float)(LOGM_LO + rng.uniform() * (LOGM_HI - LOGM_LO));
      const double r12 = xb[3], r13 = xb[4], r23 = xb[5];
      const double p2 = 1.0 - r12 * r12;
      const double l32 = (r23 - r13 * r12) / sqrt(p2);
      const double p3 = 1.0 - r13 * r13 - l32 * l32;
      if (p2 >= PIVOT_MIN && p3 >= PIVOT_MIN) break;
    }
  }
  DevBuf bx, by;
  SG_CUDA(s, cudaMalloc(&bx.p, sizeof(float) * n_train * DIN));
  SG_CUDA(s, cudaMalloc(&by.p, sizeof(float) * n_train * DOUT));
  float *dx = bx.p, *dy = by.p;
  SG_CUDA(s, cudaMemcpy(dx, hx.data(), sizeof(float) * n_train * DIN, cudaMemcpyHostToDevice));
  cfust_status st = cfust_surrogate_label(s, dx, dy, n_train);
  if (st != CFUST_OK) return st;
  // keep the rows with finite labels (in the domain's far corner every point
  // weight can underflow), then set the target normalisation from them
  {
    std::vector<float> hy(n_train * DOUT);
    SG_CUDA(s, cudaMemcpy(hy.data(), dy, sizeof(float) * n_train * DOUT, cudaMemcpyDeviceToHost));
    int64_t kept = 0;
    for (int64_t b = 0; b < n_train; ++b) {
      bool fin = true;
      for (int k = 0; k < DOUT; ++k) fin = fin && std::isfinite(hy[b * DOUT + k]);
      if (!fin) continue;
      if (kept != b) {
        memmove(&hy[kept * DOUT], &hy[b * DOUT], sizeof(float) * DOUT);
        memmove(&hx[kept * DIN], &hx[b * DIN], sizeof(float) * DIN);
      }
      ++kept;
    }
    if (kept < batch) return sg_fail(s, CFUST_ENUMERIC, "too few finite training labels");
    n_train = kept;
    SG_CUDA(s, cudaMemcpy(dx, hx.data(), sizeof(float) * n_train * DIN, cudaMemcpyHostToDevice));
    SG_CUDA(s, cudaMemcpy(dy, hy.data(), sizeof(float) * n_train * DOUT, cudaMemcpyHostToDevice));
    std::vector<float> ht(n_train * DOUT);
    for (int64_t b = 0; b < n_train; ++b) to_net(&hy[b * DOUT], &ht[b * DOUT]);
    for (int k = 0; k < DOUT; ++k) {
      double m = 0, v = 0;
      for (int64_t b = 0; b < n_train; ++b) m += ht[b * DOUT + k];
      m /= (double)n_train;
      for (int64_t b = 0; b < n_train; ++b) v += (ht[b * DOUT + k] - m) * (ht[b * DOUT + k] - m);
      v = sqrt(v / (double)n_train);
      s->host_norm[k] = (float)m;
      s->host_norm[DOUT + k] = (float)(v > 1e-6 ? v : 1.0);
    }
    SG_CUDA(s, cudaMemcpy(s->norm, s->host_norm, sizeof(float) * 20, cudaMemcpyHostToDevice));
  }
  return train_loop(s, dx, dy, n_train, epochs, batch, lr, loss_trace);
}

cfust_status cfust_surrogate_finetune(cfust_surrogate *s, const float *x, int64_t rows, int epochs, int batch,
                                      float lr, uint64_t seed, float *loss_trace) {
  if (!s || !x || rows < batch || batch < 128 || epochs < 1 || !(lr > 0.f) || rows > MAX_ROWS)
    return sg_fail(s, CFUST_EINVAL, "need 128 <= batch <= rows <= 2^30, epochs >= 1, lr > 0");
  // label the given problems, drop rows without finite labels and shuffle
  // (callers pass problems grouped by component and observation)
  DevBuf by;
  SG_CUDA(s, cudaMalloc(&by.p, sizeof(float) * rows * DOUT));
  cfust_status st = cfust_surrogate_label(s, x, by.p, rows);
  if (st != CFUST_OK) return st;
  std::vector<float> hx(rows * DIN), hy(rows * DOUT);
  SG_CUDA(s, cudaMemcpy(hx.data(), x, sizeof(float) * rows * DIN, cudaMemcpyDeviceToHost));
  SG_CUDA(s, cudaMemcpy(hy.data(), by.p, sizeof(float) * rows * DOUT, cudaMemcpyDeviceToHost));
  std::vector<int64_t> keep;
  keep.reserve(rows);
  for (int64_t b = 0; b < rows; ++b) {
    bool fin = true;
    for (int k = 0; k < DOUT; ++k) fin = fin && std::isfinite(hy[b * DOUT + k]);
    if (fin) keep.push_back(b);
  }
  const int64_t kept = (int64_t)keep.size();
  if (kept < batch) return sg_fail(s, CFUST_ENUMERIC, "too few finite labels");
  SplitMix rng{seed};
  for (int64_t a = kept - 1; a > 0; --a) {
    const int64_t b = (int64_t)(rng.next() % (uint64_t)(a + 1));
    std::swap(keep[a], keep[b]);
  }
  std::vector<float> sx(kept * DIN), sy(kept * DOUT);
  for (int64_t a = 0; a < kept; ++a) {
    memcpy(&sx[a * DIN], &hx[keep[a] * DIN], sizeof(float) * DIN);
    memcpy(&sy[a * DOUT], &hy[keep[a] * DOUT], sizeof(float) * DOUT);
  }
  DevBuf bx, by2;
  SG_CUDA(s, cudaMalloc(&bx.p, sizeof(float) * kept * DIN));
  SG_CUDA(s, cudaMalloc(&by2.p, sizeof(float) * kept * DOUT));
  SG_CUDA(s, cudaMemcpy(bx.p, sx.data(), sizeof(float) * kept * DIN, cudaMemcpyHostToDevice));
  SG_CUDA(s, cudaMemcpy(by2.p, sy.data(), sizeof(float) * kept * DOUT, cudaMemcpyHostToDevice));
  // the target normalisation stays as trained
  return train_loop(s, bx.p, by2.p, kept, epochs, batch, lr, loss_trace);
}

}  // extern "C"

// Learned initialiser of FastFCA (not in the paper; its own initialisation is mask-based,
// Sec. VII).  Kernels and C ABI for: model-generated training mixtures (Philox4x32-10 on the
// GPU), per-frequency features, scale-free targets from converged FastFCA parameters, a
// 3-layer MLP (hidden 256, GELU) whose products run on the fifth-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulators in tensor memory), the 1-D conv over t that gives per-frame powers, the permutation-free loss
// with its gradient, Adam, and the prediction of (W, L, H) for Algorithm 1.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "../../include/fastfca.h"
#include "alloc.h"
#include "fastfca_em_sm.cuh"
#include "launch.cuh"
#include "learn.cuh"
#include "trace.h"

using namespace ffca;
using namespace ffca::learn;

namespace {

constexpr float kPi = 3.14159265358979f;
constexpr float kSound = 343.0f;
constexpr float kFs = 16000.0f;
constexpr size_t kHeadSmemMax = 200 * 1024;   // dynamic shared memory of the head kernel

// ------------------------------------------------------------------------------ generator
// x(f, t) = sum_n sqrt(v_n(f,t)) chol(R_n(f)) z_n(f,t), v_n = sum_k B_n(f,k) A_n(k,t) with
// B, A ~ Gamma(1,1) = Exp(1), R_n = a_n a_n^H + 0.01 I for a linear array of spacing d and a
// direction theta_n ~ U[0, pi), z ~ CN(0, I).  One thread per (mixture, f, t).
__global__ void gen_mixture_kernel(int B, int F, int T, int M, int N, int K, float d, uint32_t k0, uint32_t k1,
                                   float2* __restrict__ x) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)B * F * T) return;
  const int t = (int)(idx % T);
  const int f = (int)((idx / T) % F);
  const int b = (int)(idx / ((size_t)T * F));
  float2 acc[kMaxM];
  for (int m = 0; m < M; ++m) acc[m] = make_float2(0.f, 0.f);
  const float nu = (float)f * kFs / (2.0f * (float)(F > 1 ? F - 1 : 1));
  for (int n = 0; n < N; ++n) {
    const U4 th = philox4x32_10(U4{(uint32_t)b, (1u << 16) | (uint32_t)n, 0u, 0u}, k0, k1);
    const float theta = kPi * u01(th.x);
    // power v_n(f, t)
    float v = 0.f;
    for (int kk = 0; kk < K; kk += 4) {
      const U4 rb = philox4x32_10(U4{(uint32_t)b, (2u << 16) | (uint32_t)n, (uint32_t)f, (uint32_t)(kk / 4)}, k0, k1);
      const U4 ra = philox4x32_10(U4{(uint32_t)b, (3u << 16) | (uint32_t)n, (uint32_t)t, (uint32_t)(kk / 4)}, k0, k1);
      const uint32_t bb[4] = {rb.x, rb.y, rb.z, rb.w}, aa[4] = {ra.x, ra.y, ra.z, ra.w};
      for (int j = 0; j < 4 && kk + j < K; ++j) v += (-__logf(u01(bb[j]))) * (-__logf(u01(aa[j])));
    }
    // steering vector and Cholesky factor of a a^H + 0.01 I (lower, complex)
    float2 a[kMaxM];
    const float c = cosf(theta);
    for (int m = 0; m < M; ++m) {
      const float ph = -2.0f * kPi * nu * ((float)m * d * c) / kSound;
      a[m] = make_float2(cosf(ph), sinf(ph));
    }
    float2 Lc[kMaxM][kMaxM];
    for (int i = 0; i < M; ++i)
      for (int j = 0; j <= i; ++j) {
        // R_ij = a_i conj(a_j) + 0.01 delta_ij
        float2 s = make_float2(a[i].x * a[j].x + a[i].y * a[j].y, a[i].y * a[j].x - a[i].x * a[j].y);
        if (i == j) s.x += 0.01f;
        for (int q = 0; q < j; ++q) {   // s -= L_iq conj(L_jq)
          s.x -= Lc[i][q].x * Lc[j][q].x + Lc[i][q].y * Lc[j][q].y;
          s.y -= Lc[i][q].y * Lc[j][q].x - Lc[i][q].x * Lc[j][q].y;
        }
        if (i == j) {
          Lc[i][i] = make_float2(sqrtf(fmaxf(s.x, 1e-12f)), 0.f);
        } else {
          const float inv = 1.0f / Lc[j][j].x;
          Lc[i][j] = make_float2(s.x * inv, s.y * inv);
        }
      }
    // z ~ CN(0, I) by Box-Muller, two complex values per Philox call
    float2 z[kMaxM];
    for (int m = 0; m < M; m += 2) {
      const U4 rz = philox4x32_10(U4{(uint32_t)b, ((4u + (uint32_t)(m / 2)) << 16) | (uint32_t)n, (uint32_t)f,
                                     (uint32_t)t}, k0, k1);
      const float r0 = sqrtf(-__logf(u01(rz.x))), p0 = 2.0f * kPi * u01(rz.y);
      const float r1 = sqrtf(-__logf(u01(rz.z))), p1 = 2.0f * kPi * u01(rz.w);
      z[m] = make_float2(r0 * cosf(p0), r0 * sinf(p0));      // variance 1/2 per part
      if (m + 1 < M) z[m + 1] = make_float2(r1 * cosf(p1), r1 * sinf(p1));
    }
    const float sv = sqrtf(v);
    for (int i = 0; i < M; ++i) {
      float2 s = make_float2(0.f, 0.f);
      for (int j = 0; j <= i; ++j) {
        s.x += Lc[i][j].x * z[j].x - Lc[i][j].y * z[j].y;
        s.y += Lc[i][j].x * z[j].y + Lc[i][j].y * z[j].x;
      }
      acc[i].x += sv * s.x;
      acc[i].y += sv * s.y;
    }
  }
  for (int m = 0; m < M; ++m) x[idx * M + m] = acc[m];
}

// ------------------------------------------------------------------------------ features
// One CTA per (mixture, f): phi (16) and the centred log-power trace q (T).
__global__ void features_kernel(int F, int T, int M, const float2* __restrict__ x, float* __restrict__ feats,
                                float* __restrict__ q) {
  const int row = blockIdx.x;                  // (mixture, f)
  const int f = row % F;
  const float2* xf = x + (size_t)row * T * M;
  float* qf = q + (size_t)row * T;
  __shared__ float red[32][12];
  float acc[12];
  for (int i = 0; i < 12; ++i) acc[i] = 0.f;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    float2 xv[kMaxM];
    float pw = 0.f;
    for (int m = 0; m < M; ++m) {
      xv[m] = xf[(size_t)t * M + m];
      pw += xv[m].x * xv[m].x + xv[m].y * xv[m].y;
    }
    int e = 0;
    for (int a = 0; a < M; ++a) acc[e++] += xv[a].x * xv[a].x + xv[a].y * xv[a].y;
    for (int a = 0; a < M; ++a)
      for (int b2 = a + 1; b2 < M; ++b2) {   // R_ab = x_a conj(x_b)
        acc[e++] += xv[a].x * xv[b2].x + xv[a].y * xv[b2].y;
        acc[e++] += xv[a].y * xv[b2].x - xv[a].x * xv[b2].y;
      }
    const float p = logf(fmaxf(pw / (float)M, 1e-30f));
    qf[t] = p;
    acc[10] += p;
    acc[11] += p * p;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = 0; i < 12; ++i) {
    const float v = warp_sum(acc[i]);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  __shared__ float tot[12];
  if (threadIdx.x < 12) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
    tot[threadIdx.x] = s;
  }
  __syncthreads();
  const float mean = tot[10] / (float)T;
  if (threadIdx.x == 0) {
    float* ph = feats + (size_t)row * kDin;
    float tr = 0.f;
    for (int a = 0; a < M; ++a) tr += tot[a];
    const int ne = M + M * (M - 1);
    for (int e = 0; e < ne; ++e) ph[e] = tot[e] / tr;
    const float var = fmaxf(tot[11] / (float)T - mean * mean, 0.f);
    ph[ne] = logf(tr / (float)(T * M));
    ph[ne + 1] = mean;
    ph[ne + 2] = sqrtf(var);
    ph[ne + 3] = (float)f / (float)(F > 1 ? F - 1 : 1);
    ph[ne + 4] = 1.0f;
    for (int e = ne + 5; e < kDin; ++e) ph[e] = 0.f;
  }
  for (int t = threadIdx.x; t < T; t += blockDim.x) qf[t] -= mean;
}

// ------------------------------------------------------------------------------ targets
// Scale-free targets of one frequency from converged (W, L, H): unit-norm columns of W, with
// row m of L divided by ||w_m||^2 (same covariances), l = ln L - mean_m ln L,
// h = ln H + mean_m ln L.  One thread per (row, n, t) for h; the t == 0 threads also write lt,
// the (n, t) == (0, 0) thread wt.
__global__ void targets_kernel(int rows, int T, int M, int N, const double2* __restrict__ P,
                               const float* __restrict__ lam, const float* __restrict__ v, float* __restrict__ wt,
                               float* __restrict__ lt, float* __restrict__ ht) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * N * T) return;
  const int t = (int)(idx % T);
  const int n = (int)((idx / T) % N);
  const size_t r = idx / ((size_t)T * N);
  const float* L = lam + r * M * N;
  const double2* W = P + r * M * M;
  double lnorm2[kMaxM];            // ln ||w_m||^2
  for (int col = 0; col < M; ++col) {
    double s = 0.0;
    for (int a = 0; a < M; ++a) s += W[a * M + col].x * W[a * M + col].x + W[a * M + col].y * W[a * M + col].y;
    lnorm2[col] = log(s);
  }
  double mlog = 0.0;
  for (int m = 0; m < M; ++m) mlog += log((double)L[m * N + n]) - lnorm2[m];
  mlog /= (double)M;
  ht[idx] = (float)(log((double)v[idx]) + mlog);
  if (t == 0) {
    for (int m = 0; m < M; ++m) lt[r * M * N + m * N + n] = (float)(log((double)L[m * N + n]) - lnorm2[m] - mlog);
  }
  if (t == 0 && n == 0) {
    for (int col = 0; col < M; ++col) {
      const double inv = exp(-0.5 * lnorm2[col]);
      for (int a = 0; a < M; ++a) {
        wt[r * 2 * M * M + 2 * (a * M + col)] = (float)(W[a * M + col].x * inv);
        wt[r * 2 * M * M + 2 * (a * M + col) + 1] = (float)(W[a * M + col].y * inv);
      }
    }
  }
}

// ------------------------------------------------------------------------------ BF16 GEMM
// C[m][n] = sum_k A(m,k) B(n,k) (+ bias[n]), A(m,k) = A[m*sam + k*sak], B(n,k) = B[n*sbn + k*sbk],
// FP32 in memory (the master weights and FP32 activations, transposed in the backward
// products).  A CTA computes a 128 x 64 tile of C on the tensor cores with tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulation in 64 columns of tensor memory):
//  * per K block of 64, the 128 threads round their share of the A (128 x 64) and B (64 x 64)
//    tiles to BF16 into shared memory in the tensor cores' no-swizzle K-major layout: 8 x 8
//    core matrices of 128 contiguous bytes, K-neighbouring core matrices 128 bytes apart (the
//    leading-dimension offset), groups of 8 rows 1024 bytes apart (the stride offset);
//  * one thread issues the block's four K = 16 products and commits them to an mbarrier;
//    every thread waits on it (bounded) before the tiles are rewritten;
//  * the epilogue reads the accumulator (warp w: rows 32w..32w+31, one per lane) with
//    tcgen05.ld, adds the bias and stores C.
// The operands are rounded to BF16 while staged because they live in FP32; a TMA copy cannot
// convert, and BF16 copies of every operand would cost an extra pass for products of at most
// 2048 x 256 x 256.  A wait past its limit (the products never arrive) sets bit 1 of *status,
// waits once more (bounded) for the products in flight and skips the epilogue; the net's
// synchronising calls report it as ECUDA.
constexpr int GUM = 128, GUN = 64, GUK = 64;
constexpr int kGemmThreads = 128;
constexpr unsigned kGemmCols = 64;                   // TMEM columns of the FP32 accumulator
constexpr int kGemmSpin = 1 << 20;
constexpr int kGemmMaxSplit = 16;                    // K slices of a split product
constexpr size_t kGemmSmemA = GUM * GUK * 2, kGemmSmemB = GUN * GUK * 2;
// 29 KB of shared memory per CTA caps an SM at 7 CTAs: 7 x 64 <= 512 TMEM columns, so no CTA
// ever waits for tensor memory
constexpr size_t kGemmDynSmem = 29 * 1024;
static_assert(kGemmSmemA + kGemmSmemB + 16 <= kGemmDynSmem, "GEMM tiles exceed the CTA's shared memory");
static_assert((228 * 1024 / kGemmDynSmem) * kGemmCols <= 512, "GEMM CTAs per SM could exceed TMEM");

__device__ __forceinline__ uint32_t kmajor_offset(int row, int k) {
  return (uint32_t)((k >> 3) * 128 + (row >> 3) * (GUK / 8) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading-dimension offset 128 B and stride
// offset 1024 B (each in 16-byte units), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9
// and 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t kUmmaIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GUN >> 3) << 17) | ((uint32_t)(GUM >> 4) << 24);

__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(int Md, int Nd, int Kd, const float* __restrict__ A,
                                                                long long sam, long long sak, const float* __restrict__ B,
                                                                long long sbn, long long sbk,
                                                                const float* __restrict__ bias, float* __restrict__ C,
                                                                long long ldc, int kchunk, float* __restrict__ part,
                                                                int* status) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  unsigned char* sA = gsm;
  unsigned char* sB = gsm + kGemmSmemA;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(gsm + kGemmSmemA + kGemmSmemB);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(gsm + kGemmSmemA + kGemmSmemB + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GUM, n0 = blockIdx.x * GUN;
  if (warp == 0) tmem_alloc(tbase, kGemmCols);
  if (tid == 0) {
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t d_tmem = *tbase;
  const uint32_t aBase = (uint32_t)__cvta_generic_to_shared(sA), bBase = (uint32_t)__cvta_generic_to_shared(sB);
  unsigned phase = 0;
  bool failed = false;
  // split K (part != null): slice blockIdx.z takes K range [z kchunk, min(Kd, (z + 1) kchunk))
  const int kbeg = part ? (int)blockIdx.z * kchunk : 0;
  const int kend = part ? min(Kd, kbeg + kchunk) : Kd;
  const int nkb = (kend - kbeg + GUK - 1) / GUK;
  for (int kb = 0; kb < nkb; ++kb) {
    const int k0 = kbeg + kb * GUK;
    // stage the block's tiles as BF16 (coalesced along whichever stride is 1)
    for (int e = 0; e < GUM * GUK / kGemmThreads; ++e) {
      const int i = tid + e * kGemmThreads;
      int row, col;
      if (sak == 1) { row = i / GUK; col = i % GUK; } else { row = i % GUM; col = i / GUM; }
      const int m = m0 + row, k = k0 + col;
      const float val = (m < Md && k < kend) ? A[(long long)m * sam + (long long)k * sak] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(sA + kmajor_offset(row, col)) = __float2bfloat16(val);
    }
    for (int e = 0; e < GUN * GUK / kGemmThreads; ++e) {
      const int i = tid + e * kGemmThreads;
      int row, col;
      if (sbk == 1) { row = i / GUK; col = i % GUK; } else { row = i % GUN; col = i / GUN; }
      const int n = n0 + row, k = k0 + col;
      const float val = (n < Nd && k < kend) ? B[(long long)n * sbn + (long long)k * sbk] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(sB + kmajor_offset(row, col)) = __float2bfloat16(val);
    }
    // the tensor cores read shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tmem_fence_after_sync();
#pragma unroll
      for (int s = 0; s < GUK / 16; ++s) {
        const uint64_t ad = umma_smem_desc(aBase + s * 256), bd = umma_smem_desc(bBase + s * 256);
        const uint32_t accum = (kb > 0 || s > 0) ? 1u : 0u;      // the first product overwrites
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                d_tmem),
            "l"(ad), "l"(bd), "r"(kUmmaIdesc), "r"(accum)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(mbar))
                   : "memory");
    }
    int spins = 0;
    while (!mbar_try_wait(mbar, phase) && ++spins < kGemmSpin) {
    }
    if (__syncthreads_or(spins >= kGemmSpin)) {      // the same decision in every thread
      int drain = 0;
      while (!mbar_try_wait(mbar, phase) && ++drain < kGemmSpin) {
      }
      failed = true;
      break;
    }
    phase ^= 1;
    tmem_fence_after_sync();
  }
  if (failed) {
    if (tid == 0) atomicOr(status, 1);
  } else {
    const int m = m0 + warp * 32 + lane;
#pragma unroll
    for (int c4 = 0; c4 < GUN / 16; ++c4) {
      float a8[8], b8[8];
      tmem_ld16(d_tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c4 * 16), a8, b8);
      if (m < Md) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c4 * 16 + j;
          const float v = j < 8 ? a8[j] : b8[j - 8];
          if (n < Nd) {
            if (part) part[((size_t)blockIdx.z * Md + m) * Nd + n] = v;
            else C[(long long)m * ldc + n] = v + (bias ? bias[n] : 0.f);
          }
        }
      }
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(d_tmem, kGemmCols);
}

// C = sum over the split slices (fixed order) + bias
__global__ void gemm_split_sum_kernel(int Md, int Nd, int S, const float* __restrict__ part,
                                      const float* __restrict__ bias, float* __restrict__ C, long long ldc) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Md * Nd) return;
  const int m = (int)(i / Nd), n = (int)(i - (size_t)m * Nd);
  float acc = 0.f;
  for (int z = 0; z < S; ++z) acc += part[(size_t)z * Md * Nd + i];
  C[(long long)m * ldc + n] = acc + (bias ? bias[n] : 0.f);
}

// C[m][n] = sum_k A(m,k) B(n,k) (+ bias[n]).  When the output tiles are too few to fill the
// GPU and K is long (the weight gradients: K = the batch's rows), K is split over up to
// kGemmMaxSplit slices of the grid (workspace ws, ws_elems floats), each slice's product goes to
// its own part of ws, and a second kernel adds the slices in a fixed order: the result does not
// depend on scheduling.
cudaError_t gemm(int Md, int Nd, int Kd, const float* A, long long sam, long long sak, const float* B, long long sbn,
                 long long sbk, const float* bias, float* C, long long ldc, float* ws, size_t ws_elems, int* status,
                 cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmDynSmem);
  if (e != cudaSuccess) return e;
  const int gx = (Nd + GUN - 1) / GUN, gy = (Md + GUM - 1) / GUM;
  const int nkb = (Kd + GUK - 1) / GUK;
  int S = 1;
  if (ws && gx * gy < 76 && nkb >= 4) {
    S = std::min(std::min(kGemmMaxSplit, nkb / 2), std::max(1, 152 / (gx * gy)));
    while (S > 1 && (size_t)S * Md * Nd > ws_elems) --S;
  }
  if (S == 1) {
    gemm_bf16_kernel<<<dim3(gx, gy), kGemmThreads, kGemmDynSmem, s>>>(Md, Nd, Kd, A, sam, sak, B, sbn, sbk, bias, C, ldc,
                                                                      0, nullptr, status);
    return cudaGetLastError();
  }
  const int kchunk = ((nkb + S - 1) / S) * GUK;
  S = (Kd + kchunk - 1) / kchunk;
  gemm_bf16_kernel<<<dim3(gx, gy, S), kGemmThreads, kGemmDynSmem, s>>>(Md, Nd, Kd, A, sam, sak, B, sbn, sbk, nullptr,
                                                                       C, ldc, kchunk, ws, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)Md * Nd;
  gemm_split_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Md, Nd, S, ws, bias, C, ldc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ elementwise
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678f)); }
__device__ __forceinline__ float gelu_g(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678f)) + z * 0.39894228f * __expf(-0.5f * z * z);
}

__global__ void gelu_kernel(size_t n, const float* __restrict__ z, float* __restrict__ h) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) h[i] = gelu_f(z[i]);
}

__global__ void gelu_back_kernel(size_t n, const float* __restrict__ z, float* __restrict__ dh) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) dh[i] *= gelu_g(z[i]);
}

// Column sums of a rows x cols matrix (row stride ld) in a fixed order: block per 32 columns,
// 8 row-groups per column, each row-group sums its rows in order, then the 8 partials in order.
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ X, long long ld, float* __restrict__ out) {
  __shared__ float part[8][32];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int grp = threadIdx.x >> 5;
  float s = 0.f;
  if (col < cols)
    for (int r = grp; r < rows; r += 8) s += X[(long long)r * ld + col];
  part[grp][threadIdx.x & 31] = s;
  __syncthreads();
  if (grp == 0 && col < cols) {
    float t = 0.f;
    for (int g2 = 0; g2 < 8; ++g2) t += part[g2][threadIdx.x & 31];
    out[col] = t;
  }
}

// ------------------------------------------------------------------------------ head
// Permutation p of {0..n-1} with lexicographic rank `rank` (the order itertools yields).
__device__ void unrank_perm(int n, int rank, int* p) {
  int avail[kMaxN];
  for (int i = 0; i < n; ++i) avail[i] = i;
  int fact[kMaxN + 1];
  fact[0] = 1;
  for (int i = 1; i <= n; ++i) fact[i] = fact[i - 1] * i;
  int left = n;
  for (int i = 0; i < n; ++i) {
    const int fct = fact[left - 1];
    const int d = rank / fct;
    rank %= fct;
    p[i] = avail[d];
    for (int j = d; j < left - 1; ++j) avail[j] = avail[j + 1];
    --left;
  }
}

__device__ __forceinline__ int factorial(int n) {
  int f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

struct HeadArgs {
  int rows, T, M, N, mode;           // mode 0: loss + gradients; 1: prediction only
  float inv_rows;
  const float* o;                    // rows x kOutPad
  const float* q;                    // rows x T
  const float* kw;                   // N x kConvK
  const float* cb;                   // N
  const float* wt;                   // rows x 2M^2
  const float* lt;                   // rows x MN
  const float* ht;                   // rows x N x T
  float* loss;                       // rows
  float* dout;                       // rows x kOutPad
  float* dconv;                      // rows x (N*kConvK + N)
  double2* P;                        // prediction: rows x M x M
  float* lam;                        // prediction: rows x M x N
  float* v;                          // prediction: rows x N x T
};

// One CTA (128 threads) per frequency sample; ln v and its gradient live in shared memory.
__global__ void __launch_bounds__(128) head_kernel(HeadArgs a) {
  extern __shared__ float sm[];
  const int row = blockIdx.x;
  const int T = a.T, M = a.M, N = a.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* sq = sm;                    // T
  float* slv = sq + T;               // N x T  (ln v, later d ln v)
  __shared__ float s_red[4][2 * kMaxN + 2];
  __shared__ float s_mean[kMaxN], s_hbar[kMaxN], s_lnL[kMaxM * kMaxN], s_o[kOutPad];
  __shared__ int s_sigma[kMaxM], s_pi[kMaxN];
  __shared__ float s_loss_wl, s_dmean[kMaxN];
  const float* orow = a.o + (size_t)row * kOutPad;
  if (tid < kOutPad) s_o[tid] = orow[tid];
  for (int t = tid; t < T; t += 128) sq[t] = a.q[(size_t)row * T + t];
  __syncthreads();
  const int base = 2 * M * M;
  if (tid < N) {
    float mlog = 0.f;
    for (int m = 0; m < M; ++m) mlog += s_o[base + m * N + tid];
    s_mean[tid] = mlog / (float)M;
  }
  if (tid < M * N) s_lnL[tid] = s_o[base + tid];
  __syncthreads();
  // ln v = c_n + b_n + sum_j k_nj q_{t+j-4}
  constexpr int half = (kConvK - 1) / 2;
  float hsum[kMaxN];
  for (int n = 0; n < N; ++n) hsum[n] = 0.f;
  for (int t = tid; t < T; t += 128) {
    for (int n = 0; n < N; ++n) {
      float s = a.cb[n] + s_o[base + M * N + n];
      for (int j = 0; j < kConvK; ++j) {
        const int tt = t + j - half;
        if (tt >= 0 && tt < T) s = fmaf(a.kw[n * kConvK + j], sq[tt], s);
      }
      slv[n * T + t] = s;
      hsum[n] += s;
    }
  }
  if (a.mode == 1) {
    for (int t = tid; t < T; t += 128)
      for (int n = 0; n < N; ++n) a.v[((size_t)row * N + n) * T + t] = __expf(slv[n * T + t]);
    if (tid < M * M) {   // W with unit columns: the loss fixes only the columns' directions
      const int col = tid % M;
      float nrm = 0.f;
      for (int r = 0; r < M; ++r)
        nrm += s_o[2 * (r * M + col)] * s_o[2 * (r * M + col)] + s_o[2 * (r * M + col) + 1] * s_o[2 * (r * M + col) + 1];
      const float inv = rsqrtf(fmaxf(nrm, 1e-30f));
      a.P[(size_t)row * M * M + tid] = make_double2((double)(s_o[2 * tid] * inv), (double)(s_o[2 * tid + 1] * inv));
    }
    if (tid < M * N) a.lam[(size_t)row * M * N + tid] = __expf(s_o[base + tid]);
    return;
  }
  for (int n = 0; n < N; ++n) {
    const float v = warp_sum(hsum[n]);
    if (lane == 0) s_red[warp][n] = v;
  }
  __syncthreads();
  if (tid < N) {
    const float s = s_red[0][tid] + s_red[1][tid] + s_red[2][tid] + s_red[3][tid];
    s_hbar[tid] = s / (float)T + s_mean[tid];
  }
  __syncthreads();
  const float* wtr = a.wt + (size_t)row * 2 * M * M;
  const float* ltr = a.lt + (size_t)row * M * N;
  const float* htr = a.ht + (size_t)row * N * T;
  // permutations: sigma (channels, by the W term) then pi (sources), both on warp 0
  if (warp == 0) {
    // unit-norm predicted columns
    float ur[kMaxM][kMaxM], ui[kMaxM][kMaxM];
    for (int col = 0; col < M; ++col) {
      float s = 0.f;
      for (int r = 0; r < M; ++r) s += s_o[2 * (r * M + col)] * s_o[2 * (r * M + col)] + s_o[2 * (r * M + col) + 1] * s_o[2 * (r * M + col) + 1];
      const float inv = rsqrtf(fmaxf(s, 1e-30f));
      for (int r = 0; r < M; ++r) { ur[r][col] = s_o[2 * (r * M + col)] * inv; ui[r][col] = s_o[2 * (r * M + col) + 1] * inv; }
    }
    const int nsig = factorial(M);
    float best = 3.4e38f;
    int bestr = 0x7fffffff;
    for (int rk = lane; rk < nsig; rk += 32) {
      int p[kMaxN];
      unrank_perm(M, rk, p);
      float val = 0.f;
      for (int m = 0; m < M; ++m) {
        float sr = 0.f, si = 0.f;   // s = u^H t
        for (int r = 0; r < M; ++r) {
          const float tr = wtr[2 * (r * M + m)], ti = wtr[2 * (r * M + m) + 1];
          sr += ur[r][p[m]] * tr + ui[r][p[m]] * ti;
          si += ur[r][p[m]] * ti - ui[r][p[m]] * tr;
        }
        val += 1.0f - (sr * sr + si * si);
      }
      if (val < best) { best = val; bestr = rk; }
    }
    for (int off = 16; off >= 1; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int orr = __shfl_xor_sync(0xffffffffu, bestr, off);
      if (ob < best || (ob == best && orr < bestr)) { best = ob; bestr = orr; }
    }
    int sig[kMaxN];
    unrank_perm(M, bestr, sig);
    if (lane < M) s_sigma[lane] = sig[lane];
  }
  __syncthreads();
  // mean over t of the target h (per source) for the pi criterion
  float htsum[kMaxN];
  for (int n = 0; n < N; ++n) htsum[n] = 0.f;
  for (int t = tid; t < T; t += 128)
    for (int n = 0; n < N; ++n) htsum[n] += htr[n * T + t];
  for (int n = 0; n < N; ++n) {
    const float v = warp_sum(htsum[n]);
    if (lane == 0) s_red[warp][kMaxN + n] = v;
  }
  __syncthreads();
  if (warp == 0) {
    float htbar[kMaxN];
    for (int n = 0; n < N; ++n)
      htbar[n] = (s_red[0][kMaxN + n] + s_red[1][kMaxN + n] + s_red[2][kMaxN + n] + s_red[3][kMaxN + n]) / (float)T;
    const int npi = factorial(N);
    float best = 3.4e38f;
    int bestr = 0x7fffffff;
    for (int rk = lane; rk < npi; rk += 32) {
      int p[kMaxN];
      unrank_perm(N, rk, p);
      float val = 0.f;
      for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
          const float r = (s_lnL[s_sigma[m] * N + p[n]] - s_mean[p[n]]) - ltr[m * N + n];
          val += r * r;
        }
      for (int n = 0; n < N; ++n) {
        const float r = s_hbar[p[n]] - htbar[n];
        val += r * r;
      }
      if (val < best) { best = val; bestr = rk; }
    }
    for (int off = 16; off >= 1; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int orr = __shfl_xor_sync(0xffffffffu, bestr, off);
      if (ob < best || (ob == best && orr < bestr)) { best = ob; bestr = orr; }
    }
    int p[kMaxN];
    unrank_perm(N, bestr, p);
    if (lane < N) s_pi[lane] = p[lane];
    if (lane < N) s_dmean[lane] = 0.f;
  }
  __syncthreads();
  // H term: r = ln v[pi(n)] + mean[pi(n)] - h*[n]; loss += r^2/T; d ln v = 2r/T
  float lossh = 0.f;
  for (int t = tid; t < T; t += 128)
    for (int n = 0; n < N; ++n) {
      const int pn = s_pi[n];
      const float r = slv[pn * T + t] + s_mean[pn] - htr[n * T + t];
      lossh += r * r;
      slv[pn * T + t] = 2.0f * r / (float)T;       // each (pn, t) written once (pi is a bijection)
    }
  __syncthreads();
  // reductions of d ln v: per source sum (-> db and dmean) and conv-weight products
  const int NK = N * kConvK;
  float* dconv = a.dconv + (size_t)row * (NK + N);
  float dks[kMaxN * kConvK + kMaxN];
  for (int i = 0; i < NK + N; ++i) dks[i] = 0.f;
  for (int t = tid; t < T; t += 128)
    for (int n = 0; n < N; ++n) {
      const float g = slv[n * T + t];
      for (int j = 0; j < kConvK; ++j) {
        const int tt = t + j - half;
        if (tt >= 0 && tt < T) dks[n * kConvK + j] += g * sq[tt];
      }
      dks[NK + n] += g;
    }
  __shared__ float s_red2[4][kMaxN * kConvK + kMaxN + 1];
  for (int i = 0; i < NK + N; ++i) {
    const float v = warp_sum(dks[i]);
    if (lane == 0) s_red2[warp][i] = v;
  }
  {
    const float v = warp_sum(lossh);
    if (lane == 0) s_red2[warp][NK + N] = v;
  }
  __syncthreads();
  const float inv = a.inv_rows;
  if (tid < NK + N) {
    const float s = s_red2[0][tid] + s_red2[1][tid] + s_red2[2][tid] + s_red2[3][tid];
    dconv[tid] = s * inv;
  }
  if (warp == 0) {
    // W and L terms and d o (thread-serial on lane 0: tiny)
    if (lane == 0) {
      float* dout = a.dout + (size_t)row * kOutPad;
      for (int i = 0; i < kOutPad; ++i) dout[i] = 0.f;
      float loss = 0.f;
      for (int m = 0; m < M; ++m) {
        const int col = s_sigma[m];
        float nw2 = 0.f;
        for (int r = 0; r < M; ++r) nw2 += s_o[2 * (r * M + col)] * s_o[2 * (r * M + col)] + s_o[2 * (r * M + col) + 1] * s_o[2 * (r * M + col) + 1];
        const float nw = sqrtf(fmaxf(nw2, 1e-30f));
        float sr = 0.f, si = 0.f;
        for (int r = 0; r < M; ++r) {
          const float ur = s_o[2 * (r * M + col)] / nw, ui = s_o[2 * (r * M + col) + 1] / nw;
          const float tr = wtr[2 * (r * M + m)], ti = wtr[2 * (r * M + m) + 1];
          sr += ur * tr + ui * ti;
          si += ur * ti - ui * tr;
        }
        loss += 1.0f - (sr * sr + si * si);
        for (int r = 0; r < M; ++r) {
          const float ur = s_o[2 * (r * M + col)] / nw, ui = s_o[2 * (r * M + col) + 1] / nw;
          const float tr = wtr[2 * (r * M + m)], ti = wtr[2 * (r * M + m) + 1];
          // gz = -conj(s) (t_r - s u_r) / |w|
          const float dr = tr - (sr * ur - si * ui), di = ti - (sr * ui + si * ur);
          const float gzr = -(sr * dr + si * di) / nw, gzi = -(sr * di - si * dr) / nw;
          dout[2 * (r * M + col)] += 2.0f * gzr * inv;
          dout[2 * (r * M + col) + 1] += 2.0f * gzi * inv;
        }
      }
      float dlp[kMaxM * kMaxN];
      for (int i = 0; i < M * N; ++i) dlp[i] = 0.f;
      for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
          const int i = s_sigma[m] * N + s_pi[n];
          const float r = (s_lnL[i] - s_mean[s_pi[n]]) - ltr[m * N + n];
          loss += r * r;
          dlp[i] += 2.0f * r;
        }
      float dmean[kMaxN];
      for (int n = 0; n < N; ++n) {
        const float s = s_red2[0][NK + n] + s_red2[1][NK + n] + s_red2[2][NK + n] + s_red2[3][NK + n];
        dmean[n] = s;                              // sum_t d ln v for source n (= d mean)
      }
      for (int n = 0; n < N; ++n) {
        float colmean = 0.f;
        for (int m = 0; m < M; ++m) colmean += dlp[m * N + n];
        colmean /= (float)M;
        for (int m = 0; m < M; ++m) dout[base + m * N + n] += (dlp[m * N + n] - colmean + dmean[n] / (float)M) * inv;
        dout[base + M * N + n] += dmean[n] * inv;  // b_n enters ln v of every frame
      }
      const float lh = s_red2[0][NK + N] + s_red2[1][NK + N] + s_red2[2][NK + N] + s_red2[3][NK + N];
      a.loss[row] = loss + lh / (float)T;
    }
  }
}

__global__ void adam_kernel(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void init_weights_kernel(int n, float* __restrict__ p, float scale, float bias_id, int id_M, uint32_t k0,
                                    uint32_t k1, uint32_t tag, int is_bias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (is_bias) {
    // output bias: the identity W (real diagonal), zeros elsewhere; hidden biases zero
    float val = 0.f;
    if (id_M > 0 && i < 2 * id_M * id_M && (i % 2) == 0) {
      const int e = i / 2;
      if (e / id_M == e % id_M) val = bias_id;
    }
    p[i] = val;
    return;
  }
  const U4 r = philox4x32_10(U4{tag, (uint32_t)i, 7u, 11u}, k0, k1);
  p[i] = scale * (2.0f * u01(r.x) - 1.0f);
}

}  // namespace

// ================================================================================ C ABI
struct fastfca_net {
  int M = 0, N = 0, max_rows = 0, max_T = 0, out = 0;
  cudaStream_t stream = nullptr;
  float* params = nullptr;      // flat FP32 master weights
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long count = 0;
  long long off_W1, off_b1, off_W2, off_b2, off_W3, off_b3, off_k, off_c;
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *o = nullptr;
  float *dout = nullptr, *d2 = nullptr, *d1 = nullptr, *dconv = nullptr, *loss = nullptr, *scal = nullptr;
  int* gstat = nullptr;         // device status of the tensor-core products (bit 1: a wait ran out)
  float* gws = nullptr;         // split-K partial products (kGemmMaxSplit x the largest weight gradient)
  size_t gws_elems = 0;
  int step = 0;
  char msg[256] = "";
};

namespace {

fastfca_status nfail(fastfca_net* n, fastfca_status st, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (n) snprintf(n->msg, sizeof n->msg, "%s", buf);
  else ffca::set_thread_error(buf);
  return st;
}

#define NCK(n, expr, what)                                                      \
  do {                                                                          \
    cudaError_t e__ = (expr);                                                   \
    if (e__ != cudaSuccess) {                                                   \
      cudaGetLastError();                                                       \
      return nfail(n, FASTFCA_ECUDA, "%s: %s", what, cudaGetErrorString(e__)); \
    }                                                                           \
  } while (0)

unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

// After a synchronisation: the tensor-core products' status (a wait that ran out is ECUDA;
// the word is cleared).
fastfca_status net_status(fastfca_net* n) {
  int bits = 0;
  NCK(n, cudaMemcpyAsync(&bits, n->gstat, sizeof(int), cudaMemcpyDeviceToHost, n->stream), "status read");
  NCK(n, cudaStreamSynchronize(n->stream), "status sync");
  if (bits == 0) return FASTFCA_OK;
  NCK(n, cudaMemsetAsync(n->gstat, 0, sizeof(int), n->stream), "status clear");
  return nfail(n, FASTFCA_ECUDA, "a tensor-core product's completion wait ran out (bits 0x%x)", bits);
}

// forward for `rows` feature rows into net->o (and the activations)
fastfca_status net_forward(fastfca_net* n, int rows, const float* feats) {
  cudaStream_t s = n->stream;
  const float* P = n->params;
  NCK(n, gemm(rows, kHidden, kDin, feats, kDin, 1, P + n->off_W1, kDin, 1, P + n->off_b1, n->z1, kHidden, n->gws, n->gws_elems, n->gstat, s), "gemm 1");
  gelu_kernel<<<blocks((size_t)rows * kHidden, 256), 256, 0, s>>>((size_t)rows * kHidden, n->z1, n->h1);
  NCK(n, gemm(rows, kHidden, kHidden, n->h1, kHidden, 1, P + n->off_W2, kHidden, 1, P + n->off_b2, n->z2, kHidden, n->gws, n->gws_elems, n->gstat, s),
      "gemm 2");
  gelu_kernel<<<blocks((size_t)rows * kHidden, 256), 256, 0, s>>>((size_t)rows * kHidden, n->z2, n->h2);
  NCK(n, gemm(rows, kOutPad, kHidden, n->h2, kHidden, 1, P + n->off_W3, kHidden, 1, P + n->off_b3, n->o, kOutPad, n->gws, n->gws_elems, n->gstat, s),
      "gemm 3");
  return FASTFCA_OK;
}

// loss and gradients (into net->grads) for one batch; loss mean -> *loss (host) if not NULL
fastfca_status net_loss_grad(fastfca_net* n, int rows, int T, const float* feats, const float* q, const float* wt,
                             const float* lt, const float* ht, double* loss) {
  if (rows < 1 || rows > n->max_rows || T < 1 || T > n->max_T) return nfail(n, FASTFCA_EINVAL, "rows or T out of range");
  fastfca_status st = net_forward(n, rows, feats);
  if (st) return st;
  cudaStream_t s = n->stream;
  HeadArgs a{};
  a.rows = rows;
  a.T = T;
  a.M = n->M;
  a.N = n->N;
  a.mode = 0;
  a.inv_rows = 1.0f / (float)rows;
  a.o = n->o;
  a.q = q;
  a.kw = n->params + n->off_k;
  a.cb = n->params + n->off_c;
  a.wt = wt;
  a.lt = lt;
  a.ht = ht;
  a.loss = n->loss;
  a.dout = n->dout;
  a.dconv = n->dconv;
  const size_t hsm = sizeof(float) * (size_t)T * (1 + n->N);
  NCK(n, cudaFuncSetAttribute(head_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm), "head attr");
  head_kernel<<<rows, 128, hsm, s>>>(a);
  NCK(n, cudaGetLastError(), "head launch");
  float* G = n->grads;
  const int NKc = n->N * kConvK + n->N;
  colsum_kernel<<<blocks(NKc, 32), 256, 0, s>>>(rows, NKc, n->dconv, NKc, G + n->off_k);
  // backward through the MLP
  NCK(n, gemm(kOutPad, kHidden, rows, n->dout, 1, kOutPad, n->h2, 1, kHidden, nullptr, G + n->off_W3, kHidden, n->gws, n->gws_elems, n->gstat, s), "dW3");
  colsum_kernel<<<blocks(kOutPad, 32), 256, 0, s>>>(rows, kOutPad, n->dout, kOutPad, G + n->off_b3);
  NCK(n, gemm(rows, kHidden, kOutPad, n->dout, kOutPad, 1, n->params + n->off_W3, 1, kHidden, nullptr, n->d2, kHidden, n->gws, n->gws_elems, n->gstat, s),
      "dh2");
  gelu_back_kernel<<<blocks((size_t)rows * kHidden, 256), 256, 0, s>>>((size_t)rows * kHidden, n->z2, n->d2);
  NCK(n, gemm(kHidden, kHidden, rows, n->d2, 1, kHidden, n->h1, 1, kHidden, nullptr, G + n->off_W2, kHidden, n->gws, n->gws_elems, n->gstat, s), "dW2");
  colsum_kernel<<<blocks(kHidden, 32), 256, 0, s>>>(rows, kHidden, n->d2, kHidden, G + n->off_b2);
  NCK(n, gemm(rows, kHidden, kHidden, n->d2, kHidden, 1, n->params + n->off_W2, 1, kHidden, nullptr, n->d1, kHidden, n->gws, n->gws_elems, n->gstat, s),
      "dh1");
  gelu_back_kernel<<<blocks((size_t)rows * kHidden, 256), 256, 0, s>>>((size_t)rows * kHidden, n->z1, n->d1);
  NCK(n, gemm(kHidden, kDin, rows, n->d1, 1, kHidden, feats, 1, kDin, nullptr, G + n->off_W1, kDin, n->gws, n->gws_elems, n->gstat, s), "dW1");
  colsum_kernel<<<blocks(kHidden, 32), 256, 0, s>>>(rows, kHidden, n->d1, kHidden, G + n->off_b1);
  NCK(n, cudaGetLastError(), "backward launches");
  if (loss) {
    colsum_kernel<<<1, 256, 0, s>>>(rows, 1, n->loss, 1, n->scal);
    float lsum = 0.f;
    NCK(n, cudaMemcpyAsync(&lsum, n->scal, sizeof(float), cudaMemcpyDeviceToHost, s), "loss download");
    NCK(n, cudaStreamSynchronize(s), "loss sync");
    *loss = (double)lsum / rows;
    return net_status(n);
  }
  return FASTFCA_OK;
}

}  // namespace

extern "C" {

fastfca_status fastfca_generate_mixtures(int32_t B, int32_t F, int32_t T, int32_t M, int32_t N, int32_t K,
                                         double spacing, uint64_t seed, void* x, void* stream) {
  FFCA_TRACE("fastfca_generate_mixtures");
  if (B < 1 || F < 1 || T < 1 || M < 1 || M > kMaxM || N < 1 || N > kMaxN || K < 1 || !x)
    return nfail(nullptr, FASTFCA_EINVAL, "generate: sizes out of range (M <= %d, N <= %d)", kMaxM, kMaxN);
  const size_t n = (size_t)B * F * T;
  gen_mixture_kernel<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(B, F, T, M, N, K, (float)spacing,
                                                                      (uint32_t)seed, (uint32_t)(seed >> 32),
                                                                      static_cast<float2*>(x));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FASTFCA_OK : nfail(nullptr, FASTFCA_ECUDA, "generate: %s", cudaGetErrorString(e));
}

fastfca_status fastfca_net_features(int32_t rows, int32_t F, int32_t T, int32_t M, const void* x, float* feats, float* q,
                                    void* stream) {
  FFCA_TRACE("fastfca_net_features");
  if (rows < 1 || F < 1 || T < 1 || M < 1 || M > kMaxM || !x || !feats || !q)
    return nfail(nullptr, FASTFCA_EINVAL, "features: bad arguments (M <= %d)", kMaxM);
  features_kernel<<<rows, 128, 0, (cudaStream_t)stream>>>(F, T, M, static_cast<const float2*>(x), feats, q);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FASTFCA_OK : nfail(nullptr, FASTFCA_ECUDA, "features: %s", cudaGetErrorString(e));
}

fastfca_status fastfca_net_targets(int32_t rows, int32_t T, int32_t M, int32_t N, const void* P, const float* lam,
                                   const float* v, float* wt, float* lt, float* ht, void* stream) {
  FFCA_TRACE("fastfca_net_targets");
  if (rows < 1 || T < 1 || M < 1 || M > kMaxM || N < 1 || N > kMaxN || !P || !lam || !v || !wt || !lt || !ht)
    return nfail(nullptr, FASTFCA_EINVAL, "targets: bad arguments");
  const size_t n = (size_t)rows * N * T;
  targets_kernel<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(rows, T, M, N, static_cast<const double2*>(P), lam,
                                                                  v, wt, lt, ht);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FASTFCA_OK : nfail(nullptr, FASTFCA_ECUDA, "targets: %s", cudaGetErrorString(e));
}

fastfca_status fastfca_net_create(int32_t M, int32_t N, int32_t max_rows, int32_t max_T, uint64_t seed, void* stream,
                                  fastfca_net** out) {
  if (!out) return nfail(nullptr, FASTFCA_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_rows < 1 || max_T < 1 || (size_t)max_T * (N + 1) * sizeof(float) > kHeadSmemMax)
    return nfail(nullptr, FASTFCA_EINVAL, "net: max_rows >= 1 and 1 <= max_T, max_T (N+1) 4 B <= %zu", kHeadSmemMax);
  if (M < 2 || M > kMaxM || N < 1 || N > kMaxN || 2 * M * M + M * N + N > kOutPad)
    return nfail(nullptr, FASTFCA_EUNSUPPORTED, "net: M in 2..%d, N in 1..%d, 2M^2+MN+N <= %d", kMaxM, kMaxN, kOutPad);
  fastfca_net* n = new (std::nothrow) fastfca_net();
  if (!n) return nfail(nullptr, FASTFCA_ENOMEM, "host allocation failed");
  n->M = M;
  n->N = N;
  n->max_rows = max_rows;
  n->max_T = max_T;
  n->out = 2 * M * M + M * N + N;
  n->stream = (cudaStream_t)stream;
  long long c = 0;
  n->off_W1 = c; c += (long long)kHidden * kDin;
  n->off_b1 = c; c += kHidden;
  n->off_W2 = c; c += (long long)kHidden * kHidden;
  n->off_b2 = c; c += kHidden;
  n->off_W3 = c; c += (long long)kOutPad * kHidden;
  n->off_b3 = c; c += kOutPad;
  n->off_k = c; c += (long long)N * kConvK;
  n->off_c = c; c += N;
  n->count = c;
  auto bail = [&](const char* what, cudaError_t e) {
    snprintf(n->msg, sizeof n->msg, "%s: %s", what, cudaGetErrorString(e));
    ffca::set_thread_error(n->msg);
    fastfca_net_destroy(n);
    return e == cudaErrorMemoryAllocation ? FASTFCA_ENOMEM : FASTFCA_ECUDA;
  };
  cudaError_t e;
  const size_t act = sizeof(float) * (size_t)max_rows * kHidden;
  if ((e = ffca::dev_malloc(&n->params, sizeof(float) * c)) != cudaSuccess) return bail("params", e);
  if ((e = ffca::dev_malloc(&n->grads, sizeof(float) * c)) != cudaSuccess) return bail("grads", e);
  if ((e = ffca::dev_malloc(&n->adam_m, sizeof(float) * c)) != cudaSuccess) return bail("adam", e);
  if ((e = ffca::dev_malloc(&n->adam_v, sizeof(float) * c)) != cudaSuccess) return bail("adam", e);
  for (float** p : {&n->z1, &n->h1, &n->z2, &n->h2, &n->d2, &n->d1})
    if ((e = ffca::dev_malloc(p, act)) != cudaSuccess) return bail("activations", e);
  if ((e = ffca::dev_malloc(&n->o, sizeof(float) * (size_t)max_rows * kOutPad)) != cudaSuccess) return bail("out", e);
  if ((e = ffca::dev_malloc(&n->dout, sizeof(float) * (size_t)max_rows * kOutPad)) != cudaSuccess) return bail("dout", e);
  if ((e = ffca::dev_malloc(&n->dconv, sizeof(float) * (size_t)max_rows * (N * kConvK + N))) != cudaSuccess) return bail("dconv", e);
  if ((e = ffca::dev_malloc(&n->loss, sizeof(float) * (size_t)max_rows)) != cudaSuccess) return bail("loss", e);
  if ((e = ffca::dev_malloc(&n->scal, sizeof(float) * 4)) != cudaSuccess) return bail("scalar", e);
  if ((e = ffca::dev_malloc(&n->gstat, sizeof(int))) != cudaSuccess) return bail("status", e);
  n->gws_elems = (size_t)kGemmMaxSplit * kHidden * kHidden;
  if ((e = ffca::dev_malloc(&n->gws, sizeof(float) * n->gws_elems)) != cudaSuccess) return bail("GEMM workspace", e);
  cudaMemsetAsync(n->gstat, 0, sizeof(int), n->stream);
  cudaMemsetAsync(n->adam_m, 0, sizeof(float) * c, n->stream);
  cudaMemsetAsync(n->adam_v, 0, sizeof(float) * c, n->stream);
  cudaMemsetAsync(n->grads, 0, sizeof(float) * c, n->stream);
  // initial weights: uniform(-a, a), a = sqrt(3 / fan_in) (unit-variance activations); the last
  // layer 100x smaller with the identity W in its bias, so the untrained net starts at W = I
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  auto init = [&](long long off, int cnt, float scale, int tag, int is_bias, int idM, float bid) {
    init_weights_kernel<<<blocks(cnt, 256), 256, 0, n->stream>>>(cnt, n->params + off, scale, bid, idM, k0, k1,
                                                                (uint32_t)tag, is_bias);
  };
  init(n->off_W1, kHidden * kDin, sqrtf(3.0f / kDin), 1, 0, 0, 0.f);
  init(n->off_b1, kHidden, 0.f, 2, 1, 0, 0.f);
  init(n->off_W2, kHidden * kHidden, sqrtf(3.0f / kHidden), 3, 0, 0, 0.f);
  init(n->off_b2, kHidden, 0.f, 4, 1, 0, 0.f);
  init(n->off_W3, kOutPad * kHidden, 0.01f * sqrtf(3.0f / kHidden), 5, 0, 0, 0.f);
  init(n->off_b3, kOutPad, 0.f, 6, 1, M, 1.0f);
  init(n->off_k, N * kConvK, 0.1f, 7, 0, 0, 0.f);
  init(n->off_c, N, 0.f, 8, 1, 0, 0.f);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail("init", e);
  if ((e = cudaStreamSynchronize(n->stream)) != cudaSuccess) return bail("init sync", e);
  *out = n;
  return FASTFCA_OK;
}

void fastfca_net_destroy(fastfca_net* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  for (float* p : {n->params, n->grads, n->adam_m, n->adam_v, n->z1, n->h1, n->z2, n->h2, n->o, n->dout, n->d2, n->d1,
                   n->dconv, n->loss, n->scal})
    ffca::dev_free(p);
  ffca::dev_free(n->gstat);
  ffca::dev_free(n->gws);
  delete n;
}

const char* fastfca_net_last_error(const fastfca_net* n) { return n ? n->msg : fastfca_last_error(nullptr); }

int64_t fastfca_net_param_count(const fastfca_net* n) { return n ? n->count : 0; }

fastfca_status fastfca_net_get_params(fastfca_net* n, float* out) {
  if (!n || !out) return FASTFCA_EINVAL;
  NCK(n, cudaMemcpyAsync(out, n->params, sizeof(float) * n->count, cudaMemcpyDefault, n->stream), "get params");
  NCK(n, cudaStreamSynchronize(n->stream), "get params sync");
  return net_status(n);
}

fastfca_status fastfca_net_set_params(fastfca_net* n, const float* in) {
  if (!n || !in) return FASTFCA_EINVAL;
  NCK(n, cudaMemcpyAsync(n->params, in, sizeof(float) * n->count, cudaMemcpyDefault, n->stream), "set params");
  NCK(n, cudaStreamSynchronize(n->stream), "set params sync");
  return FASTFCA_OK;
}

fastfca_status fastfca_net_forward(fastfca_net* n, int32_t rows, const float* feats, float* out) {
  FFCA_TRACE("fastfca_net_forward");
  if (!n || !feats || !out || rows < 1 || rows > n->max_rows) return FASTFCA_EINVAL;
  fastfca_status st = net_forward(n, rows, feats);
  if (st) return st;
  NCK(n, cudaMemcpyAsync(out, n->o, sizeof(float) * (size_t)rows * kOutPad, cudaMemcpyDefault, n->stream), "out copy");
  NCK(n, cudaStreamSynchronize(n->stream), "forward sync");
  return net_status(n);
}

fastfca_status fastfca_net_loss_grad(fastfca_net* n, int32_t rows, int32_t T, const float* feats, const float* q,
                                     const float* wt, const float* lt, const float* ht, double* loss, float* grads) {
  FFCA_TRACE("fastfca_net_loss_grad");
  if (!n || !feats || !q || !wt || !lt || !ht) return FASTFCA_EINVAL;
  fastfca_status st = net_loss_grad(n, rows, T, feats, q, wt, lt, ht, loss);
  if (st) return st;
  if (grads) {
    NCK(n, cudaMemcpyAsync(grads, n->grads, sizeof(float) * n->count, cudaMemcpyDefault, n->stream), "grad copy");
    NCK(n, cudaStreamSynchronize(n->stream), "grad sync");
    return net_status(n);
  }
  return FASTFCA_OK;
}

fastfca_status fastfca_net_train_step(fastfca_net* n, int32_t rows, int32_t T, const float* feats, const float* q,
                                      const float* wt, const float* lt, const float* ht, float lr, double* loss) {
  FFCA_TRACE("fastfca_net_train_step");
  if (!n || !feats || !q || !wt || !lt || !ht || !(lr > 0.f)) return FASTFCA_EINVAL;
  fastfca_status st = net_loss_grad(n, rows, T, feats, q, wt, lt, ht, loss);
  if (st) return st;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)n->step), c2 = 1.0f - powf(b2, (float)n->step);
  adam_kernel<<<blocks(n->count, 256), 256, 0, n->stream>>>((int)n->count, n->params, n->grads, n->adam_m, n->adam_v,
                                                           lr, b1, b2, 1e-8f, c1, c2);
  NCK(n, cudaGetLastError(), "adam launch");
  return FASTFCA_OK;
}

fastfca_status fastfca_net_predict(fastfca_net* n, int32_t rows, int32_t T, const float* feats, const float* q, void* P,
                                   float* lam, float* v) {
  FFCA_TRACE("fastfca_net_predict");
  if (!n || !feats || !q || !P || !lam || !v || rows < 1 || rows > n->max_rows || T < 1 || T > n->max_T)
    return FASTFCA_EINVAL;
  fastfca_status st = net_forward(n, rows, feats);
  if (st) return st;
  HeadArgs a{};
  a.rows = rows;
  a.T = T;
  a.M = n->M;
  a.N = n->N;
  a.mode = 1;
  a.o = n->o;
  a.q = q;
  a.kw = n->params + n->off_k;
  a.cb = n->params + n->off_c;
  a.P = static_cast<double2*>(P);
  a.lam = lam;
  a.v = v;
  const size_t hsm = sizeof(float) * (size_t)T * (1 + n->N);
  NCK(n, cudaFuncSetAttribute(head_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm), "head attr");
  head_kernel<<<rows, 128, hsm, n->stream>>>(a);
  NCK(n, cudaGetLastError(), "predict launch");
  return FASTFCA_OK;
}

}  // extern "C"

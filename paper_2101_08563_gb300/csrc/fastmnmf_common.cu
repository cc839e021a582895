// FastMNMF kernels shared by every (M, N): the cross-frequency activation update, h for the
// Wiener filter, and the default start (declared in fastmnmf.cuh).
#include "fastmnmf.cuh"
#include "philox.cuh"

namespace ffca {

// v_jkn <- v_jkn (sum_i t_ikn a_ijn / sum_i t_ikn b_ijn)^1/2.  Grid (ceil(T/32), N), 512
// threads: lane = frame within the CTA's 32, warp w sums frequencies i = w, w + 16, ... (eight
// at a time, so each warp keeps 16 loads in flight); the 16 partial sums meet in shared
// memory (two CTAs per SM, so the N x ceil(T/32) CTAs of the bench shape fit in one wave).
// Then h_ijn = sum_k t_ikn v_jkn of the new v for every frequency (the next
// iteration's h, and the Wiener filter's), written to h (F x N x T).  Dynamic shared memory:
// F*K floats (t[:, n, :]) plus 16 x 32 x 2K floats (partial sums, then the new v of the tile).
constexpr int kMnmfVWarps = 16;

__global__ void __launch_bounds__(kMnmfVWarps * 32, 2) fastmnmf_v_kernel(const float* __restrict__ tb,
                                                                     const float* __restrict__ ab,
                                                                     float* __restrict__ va,
                                                                     float* __restrict__ h, int F, int N, int K,
                                                                     int T) {
  extern __shared__ __align__(16) float smv[];
  const int n = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float* sTn = smv;                          // F x K
  float* sP = smv + (size_t)F * K;           // [w][lane][2K]
  for (int e = threadIdx.x; e < F * K; e += blockDim.x) {
    const int i = e / K, k = e - (e / K) * K;
    sTn[e] = tb[((size_t)i * N + n) * K + k];
  }
  __syncthreads();
  float num[kMnmfMaxK], den[kMnmfMaxK];
#pragma unroll
  for (int k = 0; k < kMnmfMaxK; ++k) { num[k] = 0.f; den[k] = 0.f; }
  if (j < T) {
    const float* ap = ab + (size_t)n * T + j;
    const float* bp = ab + (size_t)F * N * T + (size_t)n * T + j;
    const size_t fs = (size_t)N * T;
#pragma unroll 8
    for (int i = w; i < F; i += kMnmfVWarps) {
      const float a = __ldg(ap + (size_t)i * fs);
      const float b = __ldg(bp + (size_t)i * fs);
      const float* tr = sTn + (size_t)i * K;
#pragma unroll
      for (int k = 0; k < kMnmfMaxK; ++k) {
        if (k < K) {
          num[k] = fmaf(tr[k], a, num[k]);
          den[k] = fmaf(tr[k], b, den[k]);
        }
      }
    }
  }
  float* mine = sP + ((size_t)w * 32 + lane) * 2 * K;
#pragma unroll
  for (int k = 0; k < kMnmfMaxK; ++k) {
    if (k < K) {
      mine[k] = num[k];
      mine[K + k] = den[k];
    }
  }
  __syncthreads();
  float vnew[kMnmfMaxK / kMnmfVWarps > 0 ? kMnmfMaxK / kMnmfVWarps : 1];
  int c = 0;
  for (int k = w; k < K; k += kMnmfVWarps, ++c) {
    float nm = 0.f, dn = 0.f;
    for (int q = 0; q < kMnmfVWarps; ++q) {
      const float* o = sP + ((size_t)q * 32 + lane) * 2 * K;
      nm += o[k];
      dn += o[K + k];
    }
    float val = 0.f;
    if (j < T) {
      float* vp = va + ((size_t)n * K + k) * T + j;
      val = *vp * ((dn > 0.f) ? sqrtf(nm / dn) : 1.0f);
      *vp = val;
    }
    vnew[c] = val;
  }
  __syncthreads();                           // the partial sums are consumed: reuse sP
  float* sV = sP;                            // [k][lane], the new v of the tile
  c = 0;
  for (int k = w; k < K; k += kMnmfVWarps, ++c) sV[k * 32 + lane] = vnew[c];
  __syncthreads();
  if (j < T) {
    const size_t fs = (size_t)N * T;
    float* hp = h + (size_t)n * T + j;
    float vk[kMnmfMaxK];
#pragma unroll
    for (int k = 0; k < kMnmfMaxK; ++k) vk[k] = (k < K) ? sV[k * 32 + lane] : 0.f;
#pragma unroll 4
    for (int i = w; i < F; i += kMnmfVWarps) {
      const float* tr = sTn + (size_t)i * K;
      float hv = 0.f;
#pragma unroll
      for (int k = 0; k < kMnmfMaxK; ++k)
        if (k < K) hv = fmaf(tr[k], vk[k], hv);
      hp[(size_t)i * fs] = hv;
    }
  }
}

// h_ijn = sum_k t_ikn v_jkn (Eq. 52) as F x N x T, the layout of the FastFCA filter's H.
__global__ void fastmnmf_h_kernel(const float* __restrict__ tb, const float* __restrict__ va, float* __restrict__ h,
                                  int F, int N, int K, int T) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)F * N * T) return;
  const size_t t = e % T, fn = e / T, n = fn % N;
  const float* tr = tb + fn * K;
  float s = 0.f;
  for (int k = 0; k < K; ++k) s = fmaf(tr[k], va[(n * K + k) * T + t], s);
  h[e] = s;
}

static size_t mnmf_v_smem(int F, int K) {
  return sizeof(float) * ((size_t)F * K + (size_t)kMnmfVWarps * 32 * 2 * K);
}

cudaError_t launch_mnmf_v(const float* tb, const float* ab, float* va, float* h, int F, int N, int K, int T,
                          cudaStream_t s) {
  const size_t smem = mnmf_v_smem(F, K);
  cudaError_t e = cudaFuncSetAttribute(fastmnmf_v_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((T + 31) / 32, N);
  fastmnmf_v_kernel<<<grid, kMnmfVWarps * 32, smem, s>>>(tb, ab, va, h, F, N, K, T);
  return cudaGetLastError();
}

cudaError_t launch_mnmf_h(const float* tb, const float* va, float* h, int F, int N, int K, int T, cudaStream_t s) {
  const size_t n = (size_t)F * N * T;
  fastmnmf_h_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tb, va, h, F, N, K, T);
  return cudaGetLastError();
}

namespace {
// pf[i] = mean_j ||x_ij||^2 / (M N): one CTA per frequency, fixed summation order.
__global__ void mnmf_pf_kernel(const float2* __restrict__ x, float* __restrict__ pf, int T, int M, int N) {
  __shared__ float red[256];
  const int i = blockIdx.x;
  float s = 0.f;
  for (int j = threadIdx.x; j < T; j += blockDim.x) {
    const float2* xv = x + ((size_t)i * T + j) * M;
    for (int a = 0; a < M; ++a) s = fmaf(xv[a].x, xv[a].x, fmaf(xv[a].y, xv[a].y, s));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) pf[i] = red[0] / ((float)T * (float)(M * N));
}

// pt[j] = mean_i ||x_ij||^2 / (M N): a CTA of 32 x 32 threads per 32 frames; thread (lane, y)
// sums frequencies i = y, y + 32, ..., then the 32 partial sums are added in a fixed order.
__global__ void mnmf_pt_kernel(const float2* __restrict__ x, float* __restrict__ pt, int F, int T, int M, int N) {
  __shared__ float part[32][33];
  const int lane = threadIdx.x, y = threadIdx.y;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < T) {
    for (int i = y; i < F; i += 32) {
      const float2* xv = x + ((size_t)i * T + j) * M;
      for (int a = 0; a < M; ++a) s = fmaf(xv[a].x, xv[a].x, fmaf(xv[a].y, xv[a].y, s));
    }
  }
  part[y][lane] = s;
  __syncthreads();
  if (y == 0 && j < T) {
    float tot = 0.f;
    for (int q = 0; q < 32; ++q) tot += part[q][lane];
    pt[j] = tot / ((float)F * (float)(M * N));
  }
}

// mean of pf (= mean_ij p_ij), one CTA.
__global__ void mnmf_mean_kernel(const float* __restrict__ pf, float* __restrict__ out, int F) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < F; i += blockDim.x) s += pf[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / (float)F;
}

__global__ void mnmf_fill_kernel(const float* __restrict__ scratch, double2* __restrict__ P, float* __restrict__ lam,
                                 float* __restrict__ tb, float* __restrict__ va, int F, int T, int M, int N, int K,
                                 uint32_t seed) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const float* pf = scratch;
  const float* pt = scratch + F;
  const float mean = scratch[F + T];
  if (e < (size_t)F * M * M) {
    const size_t r = e % ((size_t)M * M);
    P[e] = make_double2((r / M == r % M) ? 1.0 : 0.0, 0.0);
  }
  if (e < (size_t)F * M * N) lam[e] = 1.0f;
  if (e < (size_t)F * N * K) {
    const size_t i = e / ((size_t)N * K), n = (e / K) % N, k = e % K;
    const U4 r = philox4x32_10(U4{(uint32_t)i, (uint32_t)n, (uint32_t)k, 0x7a11u}, seed, 0u);
    tb[e] = fmaxf(pf[i] / (float)K * (0.5f + u01(r.x)), 1e-30f);
  }
  if (e < (size_t)N * K * T) {
    const size_t j = e % T, nk = e / T, n = nk / K, k = nk % K;
    const U4 r = philox4x32_10(U4{(uint32_t)j, (uint32_t)n, (uint32_t)k, 0x7a12u}, seed, 0u);
    va[e] = fmaxf(pt[j] / fmaxf(mean, 1e-30f) * (0.5f + u01(r.x)), 1e-30f);
  }
}
}  // namespace

cudaError_t launch_mnmf_default(const float2* x, double2* P, float* lam, float* tb, float* va, float* scratch, int F,
                                int T, int M, int N, int K, uint32_t seed, cudaStream_t s) {
  mnmf_pf_kernel<<<F, 256, 0, s>>>(x, scratch, T, M, N);
  mnmf_pt_kernel<<<(T + 31) / 32, dim3(32, 32), 0, s>>>(x, scratch + F, F, T, M, N);
  mnmf_mean_kernel<<<1, 256, 0, s>>>(scratch, scratch + F + T, F);
  size_t n = (size_t)F * M * M;
  if ((size_t)F * M * N > n) n = (size_t)F * M * N;
  if ((size_t)F * N * K > n) n = (size_t)F * N * K;
  if ((size_t)N * K * T > n) n = (size_t)N * K * T;
  mnmf_fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scratch, P, lam, tb, va, F, T, M, N, K, seed);
  return cudaGetLastError();
}

}  // namespace ffca

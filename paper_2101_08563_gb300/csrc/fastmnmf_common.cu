// FastMNMF kernels shared by every (M, N): the cross-frequency activation update, h for the
// Wiener filter, and the default start (declared in fastmnmf.cuh).
#include "fastmnmf.cuh"
#include "philox.cuh"

namespace ffca {

// v_jkn <- v_jkn (sum_i t_ikn a_ijn / sum_i t_ikn b_ijn)^1/2.  Grid (ceil(T/32), N), 512
// threads: lane = frame within the CTA's 32, warp w sums frequencies i = w, w + 16, ... (eight
// at a time, so each warp keeps 16 loads in flight); the 16 partial sums meet in shared
// memory, laid out [warp][2K][lane] so that a warp's accesses fall on distinct banks (two
// CTAs per SM, so the N x ceil(T/32) CTAs of the bench shape fit in one wave).  Then
// h_ijn = sum_k t_ikn v_jkn of the new v for every frequency (the next iteration's h, and the
// Wiener filter's), written to h (F x N x T).  K is a template parameter so that no lane
// issues work for absent bases.  Dynamic shared memory: F*K floats (t[:, n, :]) plus
// 16 x 2K x 32 floats (partial sums, then the new v of the tile).
constexpr int kMnmfVWarps = 16;

template <int K>
__device__ __forceinline__ void load_row(const float* p, float (&r)[K]) {
  if constexpr (K % 4 == 0) {
#pragma unroll
    for (int k = 0; k < K; k += 4) {
      const float4 q = *reinterpret_cast<const float4*>(p + k);
      r[k] = q.x; r[k + 1] = q.y; r[k + 2] = q.z; r[k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) r[k] = p[k];
  }
}

template <int K>
__global__ void __launch_bounds__(kMnmfVWarps * 32, 2) fastmnmf_v_kernel(const float* __restrict__ tb,
                                                                     const float* __restrict__ ab,
                                                                     float* __restrict__ va,
                                                                     float* __restrict__ h, int F, int N, int T) {
  extern __shared__ __align__(16) float smv[];
  const int n = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float* sTn = smv;                          // F x K
  float* sP = smv + (size_t)F * K;           // [w][2K][lane]
  for (int e = threadIdx.x; e < F * K; e += blockDim.x) {
    const int i = e / K, k = e - (e / K) * K;
    sTn[e] = tb[((size_t)i * N + n) * K + k];
  }
  __syncthreads();
  float num[K], den[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { num[k] = 0.f; den[k] = 0.f; }
  if (j < T) {
    const float* ap = ab + (size_t)n * T + j;
    const float* bp = ab + (size_t)F * N * T + (size_t)n * T + j;
    const size_t fs = (size_t)N * T;
#pragma unroll 8
    for (int i = w; i < F; i += kMnmfVWarps) {
      const float a = __ldg(ap + (size_t)i * fs);
      const float b = __ldg(bp + (size_t)i * fs);
      float tr[K];
      load_row<K>(sTn + (size_t)i * K, tr);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        num[k] = fmaf(tr[k], a, num[k]);
        den[k] = fmaf(tr[k], b, den[k]);
      }
    }
  }
  float* mine = sP + (size_t)w * 2 * K * 32 + lane;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    mine[k * 32] = num[k];
    mine[(K + k) * 32] = den[k];
  }
  __syncthreads();
  float vnew = 0.f;                          // K <= 16 = warps: warp w owns basis w
  if (w < K) {
    float nm = 0.f, dn = 0.f;
    for (int q = 0; q < kMnmfVWarps; ++q) {
      const float* o = sP + (size_t)q * 2 * K * 32 + lane;
      nm += o[w * 32];
      dn += o[(K + w) * 32];
    }
    if (j < T) {
      float* vp = va + ((size_t)n * K + w) * T + j;
      vnew = *vp * ((dn > 0.f) ? sqrtf(nm / dn) : 1.0f);
      *vp = vnew;
    }
  }
  __syncthreads();                           // the partial sums are consumed: reuse sP
  float* sV = sP;                            // [k][lane], the new v of the tile
  if (w < K) sV[w * 32 + lane] = vnew;
  __syncthreads();
  if (j < T) {
    const size_t fs = (size_t)N * T;
    float* hp = h + (size_t)n * T + j;
    float vk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vk[k] = sV[k * 32 + lane];
#pragma unroll 4
    for (int i = w; i < F; i += kMnmfVWarps) {
      float tr[K];
      load_row<K>(sTn + (size_t)i * K, tr);
      float hv = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) hv = fmaf(tr[k], vk[k], hv);
      hp[(size_t)i * fs] = hv;
    }
  }
}
static_assert(kMnmfMaxK <= kMnmfVWarps, "one warp per basis in the v update");

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

// t_ikn <- t_ikn (sum_j v_jkn a_ijn / sum_j v_jkn b_ijn)^1/2.  Grid (ceil(F / 16), N), 512
// threads: warp w takes frequency i = 16 blockIdx.x + w, lanes stride over frames.  The
// CTA's source row block v[n][:][chunk] is staged in shared memory chunk by chunk and serves
// all 16 frequencies; each lane keeps 2K partial sums, one warp reduction at the end.
constexpr int kMnmfTFreqs = 16;
constexpr int kMnmfTChunk = 256;

template <int K>
__global__ void __launch_bounds__(kMnmfTFreqs * 32, 2) fastmnmf_t_kernel(float* __restrict__ tb,
                                                                        const float* __restrict__ va,
                                                                        const float* __restrict__ ab, int F, int N,
                                                                        int T) {
  constexpr int VP = pow2_ceil(2 * K);
  __shared__ float sV[K * kMnmfTChunk];
  const int n = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kMnmfTFreqs + w;
  const bool live = i < F;
  const float* ap = ab + ((size_t)(live ? i : 0) * N + n) * T;
  const float* bp = ap + (size_t)F * N * T;
  float acc[VP];
#pragma unroll
  for (int k = 0; k < VP; ++k) acc[k] = 0.f;
  for (int c0 = 0; c0 < T; c0 += kMnmfTChunk) {
    __syncthreads();                          // the previous chunk is consumed
    for (int e = threadIdx.x; e < K * kMnmfTChunk; e += blockDim.x) {
      const int k = e / kMnmfTChunk, jj = e - k * kMnmfTChunk;
      sV[e] = (c0 + jj < T) ? __ldg(va + ((size_t)n * K + k) * T + c0 + jj) : 0.f;
    }
    __syncthreads();
    if (live) {
      const int cn = (T - c0 < kMnmfTChunk) ? T - c0 : kMnmfTChunk;
#pragma unroll 8
      for (int jj = lane; jj < cn; jj += 32) {
        const float a = __ldg(ap + c0 + jj);
        const float b = __ldg(bp + c0 + jj);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float vk = sV[k * kMnmfTChunk + jj];
          acc[k] = fmaf(vk, a, acc[k]);
          acc[K + k] = fmaf(vk, b, acc[K + k]);
        }
      }
    }
  }
  warp_reduce_scatter<VP>(acc, lane);       // lane l holds the total of element (l VP) / 32
  const int kk = lane < K ? lane : 0;
  const float num = __shfl_sync(0xffffffffu, acc[0], (kk * 32) / VP);
  const float den = __shfl_sync(0xffffffffu, acc[0], ((K + kk) * 32) / VP);
  if (live && lane < K) {
    // a basis whose activations have all underflowed to zero gives 0/0: it has no effect on
    // the model and is left as it is (the lambda update treats a source the same way)
    float* tp = tb + ((size_t)i * N + n) * K + lane;
    *tp *= (den > 0.f) ? sqrtf(num / den) : 1.0f;
  }
}

namespace {
template <template <int> class Fn, typename... Args>
cudaError_t dispatch_k(int K, Args... args) {
  switch (K) {
    case 1: return Fn<1>::run(args...);
    case 2: return Fn<2>::run(args...);
    case 3: return Fn<3>::run(args...);
    case 4: return Fn<4>::run(args...);
    case 5: return Fn<5>::run(args...);
    case 6: return Fn<6>::run(args...);
    case 7: return Fn<7>::run(args...);
    case 8: return Fn<8>::run(args...);
    case 9: return Fn<9>::run(args...);
    case 10: return Fn<10>::run(args...);
    case 11: return Fn<11>::run(args...);
    case 12: return Fn<12>::run(args...);
    case 13: return Fn<13>::run(args...);
    case 14: return Fn<14>::run(args...);
    case 15: return Fn<15>::run(args...);
    case 16: return Fn<16>::run(args...);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
struct RunT {
  static cudaError_t run(float* tb, const float* va, const float* ab, int F, int N, int T, cudaStream_t s) {
    dim3 grid((F + kMnmfTFreqs - 1) / kMnmfTFreqs, N);
    fastmnmf_t_kernel<K><<<grid, kMnmfTFreqs * 32, 0, s>>>(tb, va, ab, F, N, T);
    return cudaGetLastError();
  }
};

template <int K>
struct RunV {
  static cudaError_t run(const float* tb, const float* ab, float* va, float* h, int F, int N, int T, cudaStream_t s) {
    const size_t smem = sizeof(float) * ((size_t)F * K + (size_t)kMnmfVWarps * 32 * 2 * K);
    cudaError_t e = cudaFuncSetAttribute(fastmnmf_v_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((T + 31) / 32, N);
    fastmnmf_v_kernel<K><<<grid, kMnmfVWarps * 32, smem, s>>>(tb, ab, va, h, F, N, T);
    return cudaGetLastError();
  }
};
}  // namespace

cudaError_t launch_mnmf_t(float* tb, const float* va, const float* ab, int F, int N, int K, int T, cudaStream_t s) {
  return dispatch_k<RunT>(K, tb, va, ab, F, N, T, s);
}

cudaError_t launch_mnmf_v(const float* tb, const float* ab, float* va, float* h, int F, int N, int K, int T,
                          cudaStream_t s) {
  return dispatch_k<RunV>(K, tb, ab, va, h, F, N, T, s);
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

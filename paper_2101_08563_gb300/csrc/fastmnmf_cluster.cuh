// FastMNMF's per-frequency step for large bins: the FastFCA cluster kernel with its MN flag
// (Q, FP64 IP, U and lambda's MM update on a thread-block cluster per frequency), and the
// v update's per-bin terms with N taken at run time.
#pragma once
#include "fastmnmf.cuh"
#include "launch.cuh"

namespace ffca {

template <int M>
cudaError_t launch_mnmf_cluster(const MnmfArgs& m, cudaStream_t s) {
  EmArgs a{};
  a.x = m.x;
  a.xh = nullptr;
  a.P = m.P;
  a.lam = m.lam;
  a.v = const_cast<float*>(m.hin);       // read only in the MN form
  a.ll_hist = m.ll_out;
  a.ll_last = m.iterate ? nullptr : m.ll_last;
  a.Bst = m.Bst;
  a.detst = m.detst;
  a.b_valid = m.b_valid;
  a.err = m.err;
  a.F = m.F;
  a.T = m.T;
  a.n_iter = m.iterate ? 1 : 0;
  a.ll_stride = m.ll_stride;
  a.N = m.N;
  a.clocks = nullptr;
  ClusterArgs ca{a, m.u, m.ab, cluster_wait_limit()};
  int C = 0;
  size_t smem = 0;
  if (!cluster_shape<M>(a.T, a.N, &C, &smem)) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(fastfca_em_cluster_kernel<M, true, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.F * C), 1, 1);
  cfg.blockDim = dim3(kCThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, fastfca_em_cluster_kernel<M, true, false, true>, ca);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// fastmnmf_ab_kernel with N at run time (N <= kCMaxN): the same layout and staging.
template <int M>
__global__ void __launch_bounds__(kMnmfAbFrames) fastmnmf_ab_rt_kernel(const float* __restrict__ lam,
                                                                       const float* __restrict__ tb,
                                                                       const float* __restrict__ va,
                                                                       const float* __restrict__ u,
                                                                       float* __restrict__ ab, int F, int N, int K,
                                                                       int T, int* err) {
  extern __shared__ __align__(16) float sab[];
  const int NK = N * K;
  float* sV = sab;                                       // [n K + k][jj]
  float* sTt = sV + (size_t)NK * kMnmfAbFrames;          // [ii][n K + k]
  float* sLm = sTt + (size_t)kMnmfAbFreqs * NK;          // [ii][m N + n]
  const int jj = threadIdx.x;
  const int j = blockIdx.x * kMnmfAbFrames + jj;
  const int i0 = blockIdx.y * kMnmfAbFreqs;
  for (int e = jj; e < NK * kMnmfAbFrames; e += kMnmfAbFrames) {
    const int row = e / kMnmfAbFrames, c = e - row * kMnmfAbFrames;
    const int jc = blockIdx.x * kMnmfAbFrames + c;
    sV[e] = (jc < T) ? __ldg(va + (size_t)row * T + jc) : 0.f;
  }
  for (int e = jj; e < kMnmfAbFreqs * NK; e += kMnmfAbFrames) {
    const int ii = e / NK;
    sTt[e] = (i0 + ii < F) ? __ldg(tb + (size_t)(i0 + ii) * NK + (e - ii * NK)) : 0.f;
  }
  for (int e = jj; e < kMnmfAbFreqs * M * N; e += kMnmfAbFrames) {
    const int ii = e / (M * N);
    sLm[e] = (i0 + ii < F) ? __ldg(lam + (size_t)(i0 + ii) * M * N + (e - ii * M * N)) : 0.f;
  }
  __syncthreads();
  if (j >= T) return;
  bool bad = false;
  const size_t plane = (size_t)F * N * T;
  for (int ii = 0; ii < kMnmfAbFreqs && i0 + ii < F; ++ii) {
    const int i = i0 + ii;
    const float* tr = sTt + ii * NK;
    const float* lr = sLm + ii * M * N;
    float h[kCMaxN];
#pragma unroll
    for (int n = 0; n < kCMaxN; ++n) {
      float s = 0.f;
      if (n < N)
        for (int k = 0; k < K; ++k) s = fmaf(tr[n * K + k], sV[(n * K + k) * kMnmfAbFrames + jj], s);
      h[n] = s;
    }
    float e[M], r[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float s2 = 0.f;
#pragma unroll
      for (int n = 0; n < kCMaxN; ++n)
        if (n < N) s2 = fmaf(lr[m * N + n], h[n], s2);
      bad |= !(s2 > 0.f && s2 < INFINITY);
      r[m] = fast_rcp(s2);
      e[m] = __ldg(u + ((size_t)i * M + m) * T + j) * r[m] * r[m];
    }
#pragma unroll
    for (int n = 0; n < kCMaxN; ++n) {
      if (n < N) {
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          a = fmaf(lr[m * N + n], e[m], a);
          b = fmaf(lr[m * N + n], r[m], b);
        }
        ab[((size_t)i * N + n) * T + j] = a;
        ab[plane + ((size_t)i * N + n) * T + j] = b;
      }
    }
  }
  if (bad) atomicOr(err, kErrSigma);
}

template <int M>
cudaError_t launch_mnmf_ab_rt(const float* lam, const float* tb, const float* va, const float* u, float* ab, int F,
                              int N, int K, int T, int* err, cudaStream_t s) {
  if (N < 1 || N > kCMaxN) return cudaErrorInvalidValue;
  const size_t smem = mnmf_ab_smem(M, N, K);
  cudaError_t e =
      cudaFuncSetAttribute(fastmnmf_ab_rt_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((T + kMnmfAbFrames - 1) / kMnmfAbFrames, (F + kMnmfAbFreqs - 1) / kMnmfAbFreqs);
  fastmnmf_ab_rt_kernel<M><<<grid, kMnmfAbFrames, smem, s>>>(lam, tb, va, u, ab, F, N, K, T, err);
  return cudaGetLastError();
}

template <int M>
bool mnmf_cluster_ops_m(int N, int T, MnmfOps* o) {
  int C = 0;
  size_t smem = 0;
  if (!cluster_shape<M>(T, N, &C, &smem)) return false;
  o->freq = &launch_mnmf_cluster<M>;
  o->ab = &launch_mnmf_ab_rt<M>;
  o->max_T = T;
  return true;
}

}  // namespace ffca

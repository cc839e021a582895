// Default starting point of Algorithm 1 for a context or a batch mixture.  The paper's own
// initialisation is mask-based (Sec. VII); this one needs no side information:
//   W = I, L = 1, v[n][t] = ||x_t||^2 / (M N) * u[n][t],
//   u ~ U[0.5, 1.5) from Philox4x32-10 with key (seed, 0) and counter (f, n, t, 0x1d17).
// The random factor matters: with equal L and v the updates of Algorithm 1 treat all sources
// alike, and they stay identical forever.
#pragma once
#include "common.cuh"
#include "philox.cuh"

namespace ffca {

static __global__ void default_params_kernel(const float2* __restrict__ x, double2* __restrict__ P,
                                      float* __restrict__ lam, float* __restrict__ v, int F, int T,
                                      int M, int N, uint32_t seed) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < (size_t)F * M * M) {
    const size_t r = i % ((size_t)M * M);
    P[i] = make_double2((r / M == r % M) ? 1.0 : 0.0, 0.0);
  }
  if (i < (size_t)F * M * N) lam[i] = 1.0f;
  if (i < (size_t)F * N * T) {
    const size_t f = i / ((size_t)N * T), n = (i / T) % N, t = i % T;
    float pw = 0.f;
    for (int m = 0; m < M; ++m) {
      const float2 a = x[(f * T + t) * M + m];
      pw += a.x * a.x + a.y * a.y;
    }
    const U4 r = philox4x32_10(U4{(uint32_t)f, (uint32_t)n, (uint32_t)t, 0x1d17u}, seed, 0u);
    v[i] = fmaxf(pw / (float)(M * N) * (0.5f + u01(r.x)), 1e-30f);
  }
}

// Elements the kernel above must cover: max(F N T, F M M, F M N).
inline size_t default_params_elems(int F, int T, int M, int N) {
  size_t n = (size_t)F * N * T;
  if ((size_t)F * M * M > n) n = (size_t)F * M * M;
  if ((size_t)F * M * N > n) n = (size_t)F * M * N;
  return n;
}

}  // namespace ffca

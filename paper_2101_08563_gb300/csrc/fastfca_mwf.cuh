// FastFCA multichannel Wiener filter (Sec. IV-F, Eq. 39):
//   c_tn = W^{-H} diag(g_n(t)) W^H x_t,   g_{mn}(t) = L[m,n] H[n,t] / sigma^2_{mt}.
// Decorrelate, scale each decorrelated channel by its single-channel Wiener gain, project
// back.  The gains of one frame sum to one over n, so the images add up to x_t (Eq. 2).
#pragma once
#include "common.cuh"
#include "fastfca_em.cuh"

namespace ffca {

// W^{-H} for every frequency in FP64 (one warp per frequency, pivoted Gauss-Jordan on W^H),
// written as complex64 row-major for the filter kernel.
template <int M>
__global__ void __launch_bounds__(32) winv_kernel(const double2* __restrict__ P, float2* __restrict__ WmH,
                                                  int F, int* err) {
  __shared__ double2 s[4 * M * M];
  const int f = blockIdx.x, lane = threadIdx.x;
  if (f >= F) return;
  double2* src = s;
  double2* work = s + M * M;
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, j = e - (e / M) * M;
    const double2 w = P[(size_t)f * M * M + j * M + i];
    src[e] = make_double2(w.x, -w.y);          // W^H
  }
  __syncwarp();
  double mant, expo;
  __shared__ double2 dst[M * M];
  warp_inverse_pivot<M>(src, work, dst, mant, expo, lane, err);
  for (int e = lane; e < M * M; e += 32)
    WmH[(size_t)f * M * M + e] = make_float2((float)dst[e].x, (float)dst[e].y);
}

constexpr int kMwfThreads = 128;
constexpr int kMwfBatches = 2;        // frame batches of kMwfThreads per CTA

// One thread per frame of each batch; grid (F, ceil(T / (kMwfThreads kMwfBatches))).  With
// piecewise-stationary parameters (Sec. VI-B) frame t uses the powers of its block t / B.
// The N x M images of a batch are staged in shared memory so that each warp writes its
// frames' output as one contiguous span; a CTA runs kMwfBatches batches, so the parameter
// prologue is paid once and one batch's stores overlap the next batch's arithmetic.
template <int M, int N>
__global__ void __launch_bounds__(kMwfThreads) fastfca_mwf_kernel(
    const float2* __restrict__ x, const double2* __restrict__ P, const float2* __restrict__ WmH,
    const float* __restrict__ lam, const float* __restrict__ v, float2* __restrict__ c, int F, int T, int B) {
  __shared__ float2 sWc[M * M];       // conj(W[a][m]) at [m*M + a]
  __shared__ float2 sWi[M * M];       // W^{-H}[a][m] at [a*M + m]
  __shared__ float sL[M * N];
  __shared__ float4 sOut[kMwfThreads * N * M / 2 + 1];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  for (int e = tid; e < M * M; e += kMwfThreads) {
    const int a = e / M, m = e - (e / M) * M;
    const double2 w = P[(size_t)f * M * M + e];
    sWc[m * M + a] = make_float2((float)w.x, (float)-w.y);
    sWi[e] = WmH[(size_t)f * M * M + e];
  }
  for (int e = tid; e < M * N; e += kMwfThreads) sL[e] = lam[(size_t)f * M * N + e];
  const int J = T / B;                 // v holds one column per block of B frames
  float2* out = reinterpret_cast<float2*>(sOut);
#pragma unroll 1
  for (int bt = 0; bt < kMwfBatches; ++bt) {
    const int t0 = (blockIdx.y * kMwfBatches + bt) * kMwfThreads;
    if (t0 >= T) break;                                    // uniform over the CTA
    const int t = t0 + tid;
    __syncthreads();                   // parameters loaded; the previous batch's sOut consumed
    if (t < T) {
      float2 xv[M];
      const float2* xt = x + ((size_t)f * T + t) * M;
      if constexpr (M % 2 == 0) {
#pragma unroll
        for (int a = 0; a < M; a += 2) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(xt + a));
          xv[a] = make_float2(q.x, q.y);
          xv[a + 1] = make_float2(q.z, q.w);
        }
      } else {
#pragma unroll
        for (int a = 0; a < M; ++a) xv[a] = __ldg(xt + a);
      }
      float h[N];
#pragma unroll
      for (int n = 0; n < N; ++n) h[n] = __ldg(v + ((size_t)f * N + n) * J + t / B);
      float2 y[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < M; ++a) acc = cfmaf(sWc[m * M + a], xv[a], acc);
        y[m] = acc;
      }
      float rs[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        float s2 = 0.f;
#pragma unroll
        for (int n = 0; n < N; ++n) s2 = fmaf(sL[m * N + n], h[n], s2);
        rs[m] = 1.0f / s2;
      }
#pragma unroll
      for (int n = 0; n < N; ++n) {
        float2 z[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float g = sL[m * N + n] * h[n] * rs[m];
          z[m] = make_float2(g * y[m].x, g * y[m].y);
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int m = 0; m < M; ++m) acc = cfmaf(sWi[a * M + m], z[m], acc);
          out[(tid * N + n) * M + a] = acc;
        }
      }
    }
    __syncthreads();
    // contiguous write-out of the batch's frames: (nt * N * M) complex64 values
    const int nt = min(kMwfThreads, T - t0);
    const int total = nt * N * M;                     // float2 count
    float2* dst = c + ((size_t)f * T + t0) * N * M;
    if (((reinterpret_cast<uintptr_t>(dst) & 15) == 0) && (total % 2 == 0)) {
      float4* d4 = reinterpret_cast<float4*>(dst);
      for (int i = tid; i < total / 2; i += kMwfThreads) d4[i] = sOut[i];
    } else {
      for (int i = tid; i < total; i += kMwfThreads) dst[i] = out[i];
    }
  }
}

// Wide form of the filter for large bins (any M <= 8, runtime N <= kMwfWMaxN).  A CTA of
// M x 32 threads takes kMwfWBatches batches of kMwfWFrames frames, so that the parameter
// prologue (W, W^{-H}, lambda) is paid once per 256 frames; one batch's stores overlap the
// next batch's loads.  Per batch, phase 1 (thread per (frame, m)) forms
// z_nm(t) = g_nm(t) y_m(t) for every source in shared memory.  Phase 2 gives thread
// (task slot s, row a) = (tid / M, tid % M) the fixed row a of W^{-H}, held in registers, and
// walks the tasks (frame, n) s, s + 32, ...: each output c_tn[a] = sum_m W^{-H}[a][m] z_nm(t)
// reads only the M values of z of its task (shared by the M threads of the task), and
// consecutive threads write consecutive complex values of the output span (coalesced).
// Rows of sZ are padded to M + 1 values so that the tasks of a warp fall in distinct banks;
// sZ is dynamic shared memory of kMwfWFrames N (M + 1) complex values (mwf_wide_smem).
// With blocks of B frames (Sec. VI-B) v has J = T / B columns and frame t takes column t / B.
constexpr int kMwfWFrames = 32;
constexpr int kMwfWBatches = 8;
constexpr int kMwfWMaxN = 16;

constexpr size_t mwf_wide_smem(int M, int N) { return sizeof(float2) * kMwfWFrames * N * (M + 1); }

template <int M>
__global__ void __launch_bounds__(M * 32) fastfca_mwf_wide_kernel(
    const float2* __restrict__ x, const double2* __restrict__ P, const float2* __restrict__ WmH,
    const float* __restrict__ lam, const float* __restrict__ v, float2* __restrict__ c, int F, int T, int N,
    int B) {
  constexpr int kThreads = M * 32;
  const int J = T / B;
  __shared__ float2 sWc[M * M];                                   // conj(W[a][m]) at [m*M + a]
  __shared__ float sL[M * kMwfWMaxN];
  extern __shared__ float2 sZ[];                                  // [(tl*N + n)][m], padded
  const int f = blockIdx.x, tid = threadIdx.x;
  if (f >= F || N > kMwfWMaxN) return;
  for (int e = tid; e < M * M; e += kThreads) {
    const int a = e / M, m = e - (e / M) * M;
    const double2 w = P[(size_t)f * M * M + e];
    sWc[m * M + a] = make_float2((float)w.x, (float)-w.y);
  }
  for (int e = tid; e < M * N; e += kThreads) sL[e] = lam[(size_t)f * M * N + e];
  // this thread's row of W^{-H}
  const int a_row = tid % M, slot = tid / M;
  float2 wi[M];
#pragma unroll
  for (int m = 0; m < M; ++m) wi[m] = WmH[(size_t)f * M * M + a_row * M + m];
#pragma unroll 1
  for (int bt = 0; bt < kMwfWBatches; ++bt) {
  const int t0 = (blockIdx.y * kMwfWBatches + bt) * kMwfWFrames;
  if (t0 >= T) break;                                             // uniform over the CTA
  const int nt = min(kMwfWFrames, T - t0);
  __syncthreads();                     // parameters loaded; the previous batch's sZ consumed
  // phase 1: thread (tl, m) for tl < nt (32 frames x M rows = the CTA)
  {
    const int tl = tid / M, m = tid - (tid / M) * M;
    if (tl < nt) {
      const int t = t0 + tl;
      const int tb = t / B;
      const float2* xt = x + ((size_t)f * T + t) * M;
      float2 y = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < M; ++a) y = cfmaf(sWc[m * M + a], xt[a], y);
      float h[kMwfWMaxN];
      float s2 = 0.f;
#pragma unroll
      for (int n = 0; n < kMwfWMaxN; ++n) {
        const int nn = (n < N) ? n : 0;                  // index kept inside the arrays
        const float hv = v[((size_t)f * N + nn) * J + tb], lv = sL[m * N + nn];
        h[n] = (n < N) ? hv : 0.f;
        s2 = fmaf((n < N) ? lv : 0.f, h[n], s2);
      }
      const float rs = 1.0f / s2;
#pragma unroll
      for (int n = 0; n < kMwfWMaxN; ++n)
        if (n < N) {
          const float g = sL[m * N + n] * h[n] * rs;
          sZ[(tl * N + n) * (M + 1) + m] = make_float2(g * y.x, g * y.y);
        }
    }
  }
  __syncthreads();
  // phase 2: outputs in memory order, task-major (task = tl*N + n), row a minor
  const int tasks = nt * N;
  float2* dst = c + ((size_t)f * T + t0) * N * M;
  for (int task = slot; task < tasks; task += 32) {
    const float2* z = sZ + task * (M + 1);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < M; ++m) acc = cfmaf(wi[m], z[m], acc);
    dst[(size_t)task * M + a_row] = acc;
  }
  }
}

}  // namespace ffca

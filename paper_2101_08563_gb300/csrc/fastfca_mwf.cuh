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

// Stride of one frame's N x M images in the staging buffer, in complex values: N M rounded so
// that it is 2 (mod 4).  Frames then start on 16 bytes when N M is even, and the 8-byte stores
// of a half-warp (16 frames) meet at most 2 to a bank instead of 8 (N M = 24: 48 words apart).
__host__ __device__ constexpr int mwf_frame_stride(int N, int M) { return (N * M) % 2 ? N * M : (N * M) % 4 ? N * M : N * M + 2; }

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
  constexpr int FSn = mwf_frame_stride(N, M);
  __shared__ float4 sOut[(kMwfThreads * FSn + 1) / 2];
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
          out[tid * FSn + n * M + a] = acc;
        }
      }
    }
    __syncthreads();
    // contiguous write-out of the batch's frames: (nt * N * M) complex64 values
    const int nt = min(kMwfThreads, T - t0);
    const int total = nt * N * M;                     // float2 count
    float2* dst = c + ((size_t)f * T + t0) * N * M;
    if constexpr ((N * M) % 2 == 0) {
      if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        constexpr int Q = N * M / 2;                  // float4 per frame
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int i = tid; i < total / 2; i += kMwfThreads) {
          const int fr = i / Q;
          d4[i] = sOut[fr * (FSn / 2) + (i - fr * Q)];
        }
        continue;
      }
    }
    for (int i = tid; i < total; i += kMwfThreads) {
      const int fr = i / (N * M);
      dst[i] = out[fr * FSn + (i - fr * (N * M))];
    }
  }
}

// Wide form of the filter for large bins (any M <= 8, runtime N <= kMwfWMaxN).  A CTA of
// M x 32 threads takes kMwfWBatches batches of kMwfWFrames frames, so that the parameter
// prologue (W, W^{-H}, lambda) is paid once per 256 frames.  Per batch:
//  0. the batch's x (contiguous) and h values (one column of v per frame or block) are
//     staged in shared memory with coalesced loads, double-buffered: the next batch's loads
//     are issued before this batch's phase 2 and stored after it;
//  1. thread (frame, m) forms y_m = w_m^H x, sigma^2_m and z_nm = g_nm y_m for every
//     source, g_nm = L[m,n] h_n / sigma^2_m, into shared memory;
//  2. thread (task slot s, row a) = (tid / M, tid % M), holding row a of W^{-H} in registers,
//     walks the tasks (frame, n) s, s + 32, ...: c_tn[a] = sum_m W^{-H}[a][m] z_nm, so that
//     consecutive threads write consecutive complex values of the output span (coalesced).
// Layout of z: one row of kMwfWRow(M) complex values per task (frame, n), at task * row, the
// row even so that it starts on 16 bytes and phase 2 reads it as float4 pairs (one broadcast
// per quarter-warp) with no division by N.  conj(W) rows are padded to M + 1 so that the M
// threads of a frame read distinct banks.
// With blocks of B frames (Sec. VI-B) v has J = T / B columns and frame t takes column t / B.
constexpr int kMwfWFrames = 32;
constexpr int kMwfWBatches = 8;
constexpr int kMwfWMaxN = 16;

__host__ __device__ constexpr int kMwfWRow(int M) { return (M + 2) & ~1; }
constexpr size_t mwf_wide_smem(int M, int N) { return sizeof(float2) * kMwfWFrames * N * kMwfWRow(M); }

// Staging of one batch (t0, nt frames) for the wide filter: thread tid loads x value tid and
// h values tid + j M 32 of the N x kMwfWFrames block into registers (mwf_wide_load), and later
// stores them to one of the two shared buffers (mwf_wide_store).
template <int M, int HPER>
__device__ __forceinline__ void mwf_wide_load(const float2* __restrict__ x, const float* __restrict__ v, int f,
                                              int T, int N, int J, int B, int t0, int nt, int tid, float2& xr,
                                              float (&hr)[HPER]) {
  if (tid < nt * M) xr = __ldg(x + ((size_t)f * T + t0) * M + tid);
#pragma unroll
  for (int j = 0; j < HPER; ++j) {
    const int i = tid + j * M * 32;
    const int n = i / kMwfWFrames, tl = i - (i / kMwfWFrames) * kMwfWFrames;
    hr[j] = (n < N && tl < nt) ? __ldg(v + ((size_t)f * N + n) * J + (t0 + tl) / B) : 0.f;
  }
}

template <int M, int HPER>
__device__ __forceinline__ void mwf_wide_store(float2* sXb, float* sHb, int N, int nt, int tid, float2 xr,
                                               const float (&hr)[HPER]) {
  if (tid < nt * M) sXb[tid] = xr;
#pragma unroll
  for (int j = 0; j < HPER; ++j) {
    const int i = tid + j * M * 32;
    if (i < N * kMwfWFrames) sHb[i] = hr[j];
  }
}

template <int M>
__global__ void __launch_bounds__(M * 32) fastfca_mwf_wide_kernel(
    const float2* __restrict__ x, const double2* __restrict__ P, const float2* __restrict__ WmH,
    const float* __restrict__ lam, const float* __restrict__ v, float2* __restrict__ c, int F, int T, int N,
    int B) {
  constexpr int kThreads = M * 32;
  constexpr int RS = kMwfWRow(M);
  const int J = T / B;
  __shared__ float2 sWc[M * (M + 1)];                             // conj(W[a][m]) at [m*(M+1) + a]
  __shared__ float sL[M * kMwfWMaxN];
  __shared__ __align__(16) float2 sX[2][kMwfWFrames * M];         // a batch's x, frame-major
  __shared__ float sH[2][kMwfWMaxN * kMwfWFrames];                // a batch's h_n, [n][tl]
  extern __shared__ __align__(16) float2 sZ[];                    // [(tl*N + n)*RS + m]
  const int f = blockIdx.x, tid = threadIdx.x;
  if (f >= F || N > kMwfWMaxN) return;
  for (int e = tid; e < M * M; e += kThreads) {
    const int a = e / M, m = e - (e / M) * M;
    const double2 w = P[(size_t)f * M * M + e];
    sWc[m * (M + 1) + a] = make_float2((float)w.x, (float)-w.y);
  }
  for (int e = tid; e < M * N; e += kThreads) sL[e] = lam[(size_t)f * M * N + e];
  // this thread's row of W^{-H} (phase 2) and (frame, m) (phase 1)
  const int a_row = tid % M, slot = tid / M;
  float2 wi[M];
#pragma unroll
  for (int m = 0; m < M; ++m) wi[m] = WmH[(size_t)f * M * M + a_row * M + m];
  const int tl1 = tid / M, m1 = tid - (tid / M) * M;
  // staging of a batch: thread tid takes x value tid (kThreads = kMwfWFrames M of them) and h
  // values tid + j kThreads of the N x kMwfWFrames block; loads go to registers first, so that
  // the next batch's loads are in flight while this batch is computed
  constexpr int kHPer = (kMwfWMaxN * kMwfWFrames + kThreads - 1) / kThreads;
  float2 xr = make_float2(0.f, 0.f);
  float hr[kHPer];
  {
    const int t0 = blockIdx.y * kMwfWBatches * kMwfWFrames;
    if (t0 < T) {
      const int nt = min(kMwfWFrames, T - t0);
      mwf_wide_load<M, kHPer>(x, v, f, T, N, J, B, t0, nt, tid, xr, hr);
      mwf_wide_store<M, kHPer>(sX[0], sH[0], N, nt, tid, xr, hr);
    }
  }
#pragma unroll 1
  for (int bt = 0; bt < kMwfWBatches; ++bt) {
    const int t0 = (blockIdx.y * kMwfWBatches + bt) * kMwfWFrames;
    if (t0 >= T) break;                                           // uniform over the CTA
    const int nt = min(kMwfWFrames, T - t0);
    const int buf = bt & 1;
    const float2* sXb = sX[buf];
    const float* sHb = sH[buf];
    // parameters and this batch's inputs stored; the previous batch's sZ consumed
    __syncthreads();
    // 1. thread (tl1, m1): y, sigma^2, z for every source
    if (tl1 < nt) {
      float2 y = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < M; ++a) y = cfmaf(sWc[m1 * (M + 1) + a], sXb[tl1 * M + a], y);
      float s2 = 0.f;
      for (int n = 0; n < N; ++n) s2 = fmaf(sL[m1 * N + n], sHb[n * kMwfWFrames + tl1], s2);
      const float rs = 1.0f / s2;
      float2* zt = sZ + tl1 * N * RS + m1;
      for (int n = 0; n < N; ++n) {
        const float g = sL[m1 * N + n] * sHb[n * kMwfWFrames + tl1] * rs;
        zt[n * RS] = make_float2(g * y.x, g * y.y);
      }
    }
    // the next batch's loads, in flight during the barrier and phase 2
    const int t1 = t0 + kMwfWFrames;
    const bool more = bt + 1 < kMwfWBatches && t1 < T;
    if (more) mwf_wide_load<M, kHPer>(x, v, f, T, N, J, B, t1, min(kMwfWFrames, T - t1), tid, xr, hr);
    __syncthreads();
    // 2. outputs in memory order, task-major (task = tl*N + n), row a minor
    const int tasks = nt * N;
    float2* dst = c + ((size_t)f * T + t0) * N * M;
    for (int task = slot; task < tasks; task += 32) {
      const float4* z4 = reinterpret_cast<const float4*>(sZ + task * RS);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int mm = 0; mm < M / 2; ++mm) {
        const float4 q = z4[mm];
        acc = cfmaf(wi[2 * mm], make_float2(q.x, q.y), acc);
        acc = cfmaf(wi[2 * mm + 1], make_float2(q.z, q.w), acc);
      }
      if constexpr (M % 2 == 1) acc = cfmaf(wi[M - 1], sZ[task * RS + M - 1], acc);
      dst[(size_t)task * M + a_row] = acc;
    }
    // the other buffer was last read by the previous batch's phase 1, before this batch's
    // first barrier; the next iteration's first barrier publishes these stores
    if (more) mwf_wide_store<M, kHPer>(sX[buf ^ 1], sH[buf ^ 1], N, min(kMwfWFrames, T - t1), tid, xr, hr);
  }
}

}  // namespace ffca

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
// Tiled form of the filter for large bins (M <= 8, runtime N <= kMwfWMaxN).  Each warp owns a
// contiguous range of (frequency, tile) groups, so every warp gets the same number of frames,
// and runs them one after another with no CTA barrier:
//  - P = 2 threads per frame, a tile of 32 / P = 16 frames per warp: thread (q, i) of the warp
//    (q = lane / 16) takes frame i of the tile and the R = ceil(M / P) channels / rows
//    q R .. q R + R - 1;
//  - y_m = w_m^H x_t, sigma^2_m = sum_n L[m,n] h_n(t) and y_m / sigma^2_m for its channels, then
//    shuffles among the frame's P threads give each all M of them;
//  - c_tn[a] = h_n(t) sum_m K_n[a][m] y_m / sigma^2_m for its rows a, K_n = W^{-H} diag(L[:,n])
//    precomputed per frequency: M complex FMAs per output, K read as 16-byte broadcasts;
//  - the tile's images are staged frame by frame in shared memory, and each frame's N x M
//    values (contiguous in c) leave with one bulk copy (cp.async.bulk) issued by one of its
//    threads, overlapping the next tile's arithmetic; the staging buffer is reused once those
//    copies have read it.
// The next tile's x and h are loaded into registers while the current one is computed.  Per
// warp shared memory is 20 KB at M = 8, N = 12 (two CTAs of four warps per SM).
// With blocks of B frames (Sec. VI-B) v has J = T / B columns and frame t takes column t / B.
constexpr int kMwfWMaxN = 16;
constexpr int kMwfTThreads = 128;
constexpr int kMwfTWarps = kMwfTThreads / 32;

// Threads per frame, rows per thread and frames per warp tile for M channels.  Two threads
// per frame (16-frame tiles, 8 warps per SM at M = 8, N = 12) measured faster than four (8-frame
// tiles, 16 warps per SM): 0.999 against 1.053 ms for the large instance's filter.
__host__ __device__ constexpr int mwf_tile_p(int /*M*/) { return 2; }
__host__ __device__ constexpr int mwf_tile_r(int M) { return (M + mwf_tile_p(M) - 1) / mwf_tile_p(M); }
__host__ __device__ constexpr int mwf_tile_frames(int M) { return 32 / mwf_tile_p(M); }

__host__ __device__ constexpr int mwf_align16(int b) { return (b + 15) & ~15; }

// Bytes of one staged frame: N M complex64 values rounded up to 16 bytes, plus 16 when that is
// an even number of 16-byte units.  Eight consecutive frames then start in distinct 16-byte
// bank groups (a quarter-warp's 16-byte stores meet no conflict), and every frame starts on
// 16 bytes, as its bulk copy requires.
__host__ __device__ constexpr int mwf_tile_frame_bytes(int N, int M) {
  return (mwf_align16(N * M * 8) / 16) % 2 ? mwf_align16(N * M * 8) : mwf_align16(N * M * 8) + 16;
}

// Byte offsets of one warp's region of dynamic shared memory.
struct MwfTileLayout {
  int k, wc, lt, h, out, total;
};
__host__ __device__ inline MwfTileLayout mwf_tile_layout(int M, int N) {
  MwfTileLayout L{};
  L.k = 0;                                                    // K_n[a][m] at [n][m][a]
  L.wc = L.k + mwf_align16(N * M * M * 8);                    // conj(W[a][m]) at [a][m]
  L.lt = L.wc + mwf_align16(M * M * 8);                       // L[m,n] at [n][m]
  L.h = L.lt + mwf_align16(kMwfWMaxN * M * 4);                // h_n(t) at [n][frame]
  L.out = L.h + mwf_align16(kMwfWMaxN * mwf_tile_frames(M) * 4);
  L.total = L.out + mwf_tile_frames(M) * mwf_tile_frame_bytes(N, M);   // staged images
  return L;
}
inline size_t mwf_tile_smem(int M, int N) { return (size_t)kMwfTWarps * mwf_tile_layout(M, N).total; }

// Whether a thread's R rows are read and written as 16-byte vectors: R and M even, so that
// every row segment (index a M + q R, or (n M + m) M + q R) starts on 16 bytes.
__host__ __device__ constexpr bool mwf_tile_vec(int M) { return mwf_tile_r(M) % 2 == 0 && M % 2 == 0; }

// The R complex values row[0 .. R) of a thread's rows (cnt of them valid), as 16-byte loads
// where mwf_tile_vec(M).
template <int M, int R>
__device__ __forceinline__ void mwf_tile_row(const float2* row, int cnt, bool all, float2 (&w)[R]) {
  if constexpr (mwf_tile_vec(M)) {
#pragma unroll
    for (int j = 0; j < R; j += 2) {
      const float4 q = *reinterpret_cast<const float4*>(row + j);
      w[j] = make_float2(q.x, q.y);
      w[j + 1] = make_float2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) w[j] = (all || j < cnt) ? row[j] : make_float2(0.f, 0.f);
  }
}

template <int M>
__global__ void __launch_bounds__(kMwfTThreads) fastfca_mwf_tile_kernel(
    const float2* __restrict__ x, const double2* __restrict__ P, const float2* __restrict__ WmH,
    const float* __restrict__ lam, const float* __restrict__ v, float2* __restrict__ c, int F, int T, int N,
    int B) {
  constexpr int PT = mwf_tile_p(M), R = mwf_tile_r(M), FT = mwf_tile_frames(M);
  constexpr bool kFull = PT * R == M;               // every thread holds R valid rows
  constexpr int kHPer = kMwfWMaxN / PT;
  extern __shared__ __align__(16) unsigned char mwf_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = lane / FT, fi = lane % FT;
  const int lo = q * R, cnt = min(R, M - q * R);
  const MwfTileLayout Ly = mwf_tile_layout(M, N);
  unsigned char* base = mwf_smem + (size_t)warp * Ly.total;
  float2* sK = reinterpret_cast<float2*>(base + Ly.k);       // K_n[a][m] at [n][m][a]
  float2* sWc = reinterpret_cast<float2*>(base + Ly.wc);     // conj(W[a][m]) at [a][m]
  float* sLt = reinterpret_cast<float*>(base + Ly.lt);       // L[m,n] at [n][m]
  float* sH = reinterpret_cast<float*>(base + Ly.h);         // h_n(t) at [n][frame]
  unsigned char* sOut = base + Ly.out;
  const int FB = mwf_tile_frame_bytes(N, M);
  const int NM = N * M;
  const int J = T / B;
  const int tiles = (T + FT - 1) / FT;
  const long long G = (long long)F * tiles;
  const long long nw = (long long)gridDim.x * kMwfTWarps;
  const long long gw = (long long)blockIdx.x * kMwfTWarps + warp;
  const long long g0 = gw * G / nw, g1 = (gw + 1) * G / nw;
  if (g0 >= g1) return;                                          // uniform over the warp
  const bool bulk = NM % 2 == 0 && (reinterpret_cast<uintptr_t>(c) & 15) == 0;

  // this thread's frame of tile (f, t0): all M channels of x, and h_n for n = q, q + PT, ...
  float2 xr[M];
  float hr[kHPer];
  auto load = [&](int f, int t0) {
    const int t = t0 + fi;
    if (t >= T) return;
    const float2* xt = x + ((size_t)f * T + t) * M;
    if constexpr (M % 2 == 0) {
#pragma unroll
      for (int a = 0; a < M; a += 2) {
        const float4 u = __ldg(reinterpret_cast<const float4*>(xt + a));
        xr[a] = make_float2(u.x, u.y);
        xr[a + 1] = make_float2(u.z, u.w);
      }
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) xr[a] = __ldg(xt + a);
    }
#pragma unroll
    for (int j = 0; j < kHPer; ++j) {
      const int n = PT * j + q;
      hr[j] = n < N ? __ldg(v + ((size_t)f * N + n) * J + t / B) : 0.f;
    }
  };

  int f = (int)(g0 / tiles), tile = (int)(g0 - (long long)f * tiles);
  load(f, tile * FT);
  int fcur = -1;
#pragma unroll 1
  for (long long g = g0; g < g1; ++g) {
    const int t0 = tile * FT;
    const int nt = min(FT, T - t0);
    if (f != fcur) {                    // parameters of frequency f; the last reads of the old
      const double2* Pf = P + (size_t)f * M * M;      // ones ended before the last __syncwarp
      for (int e = lane; e < M * M; e += 32) {
        const double2 w = Pf[e];
        sWc[e] = make_float2((float)w.x, (float)-w.y);
      }
      const float* lf = lam + (size_t)f * M * N;
      for (int e = lane; e < NM; e += 32) {
        const int n = e / M, m = e - (e / M) * M;
        sLt[e] = lf[m * N + n];
      }
      const float2* wf = WmH + (size_t)f * M * M;
      for (int e = lane; e < N * M * M; e += 32) {
        const int n = e / (M * M), r = e - (e / (M * M)) * (M * M);
        const int m = r / M, a = r - (r / M) * M;
        const float2 w = wf[a * M + m];
        const float l = lf[m * N + n];
        sK[e] = make_float2(w.x * l, w.y * l);
      }
      fcur = f;
    }
    float2 xa[M];
#pragma unroll
    for (int a = 0; a < M; ++a) xa[a] = xr[a];
#pragma unroll
    for (int j = 0; j < kHPer; ++j) {
      const int n = PT * j + q;
      if (n < N) sH[n * FT + fi] = hr[j];
    }
    __syncwarp();
    // the next tile's loads, in flight during this tile's arithmetic
    const int fn = tile + 1 == tiles ? f + 1 : f, tn = tile + 1 == tiles ? 0 : tile + 1;
    if (g + 1 < g1) load(fn, tn * FT);

    // sigma^2_m, y_m = sum_a conj(W[a][m]) x_a and y_m / sigma^2_m for channels lo + j
    float s2[R];
#pragma unroll
    for (int j = 0; j < R; ++j) s2[j] = 0.f;
    for (int n = 0; n < N; ++n) {
      const float hn = sH[n * FT + fi];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (kFull || j < cnt) s2[j] = fmaf(sLt[n * M + lo + j], hn, s2[j]);
    }
    float yr[R], yi[R];
#pragma unroll
    for (int j = 0; j < R; ++j) yr[j] = yi[j] = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) {                 // a outer: the R rows' chains interleave
      float2 w[R];
      mwf_tile_row<M, R>(sWc + a * M + lo, cnt, kFull, w);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        yr[j] = fmaf(w[j].x, xa[a].x, yr[j]);
        yi[j] = fmaf(w[j].x, xa[a].y, yi[j]);
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        yr[j] = fmaf(-w[j].y, xa[a].y, yr[j]);
        yi[j] = fmaf(w[j].y, xa[a].x, yi[j]);
      }
    }
    float2 yt[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float rs = 1.0f / s2[j];
      yt[j] = make_float2(yr[j] * rs, yi[j] * rs);
    }
    // every thread of the frame holds all M values y_m / sigma^2_m
    float2 ya[M];
#pragma unroll
    for (int p = 0; p < PT; ++p)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float2 o = make_float2(__shfl_sync(0xffffffffu, yt[j].x, p * FT + fi),
                                     __shfl_sync(0xffffffffu, yt[j].y, p * FT + fi));
        if (p * R + j < M) ya[p * R + j] = o;
      }
    // the previous tile's bulk copies have read the staging buffer
    if (bulk && q == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncwarp();

    float2* my = reinterpret_cast<float2*>(sOut + fi * FB);
#pragma unroll 2
    for (int n = 0; n < N; ++n) {
      const float hn = sH[n * FT + fi];
      float cr[R], ci[R];
#pragma unroll
      for (int r = 0; r < R; ++r) cr[r] = ci[r] = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) {               // m outer: the R rows' chains interleave
        float2 k[R];
        mwf_tile_row<M, R>(sK + (n * M + m) * M + lo, cnt, kFull, k);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          cr[r] = fmaf(k[r].x, ya[m].x, cr[r]);
          ci[r] = fmaf(k[r].x, ya[m].y, ci[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          cr[r] = fmaf(-k[r].y, ya[m].y, cr[r]);
          ci[r] = fmaf(k[r].y, ya[m].x, ci[r]);
        }
      }
      float2* dst = my + n * M + lo;
      if constexpr (mwf_tile_vec(M)) {
#pragma unroll
        for (int r = 0; r < R; r += 2)
          *reinterpret_cast<float4*>(dst + r) = make_float4(cr[r] * hn, ci[r] * hn, cr[r + 1] * hn, ci[r + 1] * hn);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (kFull || r < cnt) dst[r] = make_float2(cr[r] * hn, ci[r] * hn);
      }
    }
    // write-out of the tile: frames t0 .. t0 + nt - 1, each N M values contiguous in c
    if (bulk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (q == 0 && fi < nt) {
        const float2* gdst = c + ((size_t)f * T + t0 + fi) * NM;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                     "r"((uint32_t)__cvta_generic_to_shared(my)), "r"(NM * 8)
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    } else {
      __syncwarp();
      float2* gdst = c + ((size_t)f * T + t0) * NM;
      for (int e = lane; e < nt * NM; e += 32) {
        const int fr = e / NM;
        gdst[e] = reinterpret_cast<const float2*>(sOut + fr * FB)[e - fr * NM];
      }
      __syncwarp();                   // staging consumed before the next tile's stores
    }
    tile = tn;
    f = fn;
  }
  // shared memory stays valid until the last bulk copies have read it
  if (bulk && q == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

}  // namespace ffca

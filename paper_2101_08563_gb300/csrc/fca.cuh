// Full-rank spatial covariance analysis (FCA), the comparison model (Sec. III).
//
// EM per iteration and frequency (Eq. 12-13, App. A), one CTA per frequency:
//   X_t = sum_n h_nt R_n, and its explicit inverse (one M x M inverse per bin, Sec. III-D)
//   B_nt = R_n X_t^{-1},  mu_nt = h_nt B_nt x_t  (posterior mean, Eq. 7)
//   Psi_nt = mu mu^H + h_nt R_n - h_nt^2 R_n X_t^{-1} R_n                (Eq. 12)
//   h_nt <- tr(R_n^{-1} Psi_nt) / M
//         = (mu^H R_n^{-1} mu + h_nt M - h_nt^2 tr(B_nt)) / M           (Eq. 13, old R_n)
//   R_n  <- (1/T) sum_t Psi_nt / h_nt                                     (Eq. 13, new h)
//   log-likelihood -sum_t (ln det X_t + x_t^H X_t^{-1} x_t) - M T ln(pi)  (Eq. 10)
// Per-bin work in FP32 complex; R_n, R_n^{-1} and the reductions' final combine in FP64.
// X_t^{-1} (packed Hermitian, M*M floats per frame) and h stay in shared memory.
#pragma once
#include "common.cuh"

namespace ffca {

struct FcaArgs {
  const float2* x;      // F x T x M
  double2* R;           // F x N x M x M
  float* h;             // F x N x T
  double* ll_hist;      // F x ll_stride or null
  double* ll_last;      // F or null
  int* err;
  int F, T, n_iter, ll_stride;
};

struct FcaWork {
  float2* dummy;
};

inline cudaError_t fca_work_alloc(FcaWork* w, int, int, int, int) {
  w->dummy = nullptr;
  return cudaSuccess;
}
inline void fca_work_free(FcaWork* w) { w->dummy = nullptr; }

struct FcaOps {
  cudaError_t (*em)(const FcaArgs& a, FcaWork* w, cudaStream_t s);
  cudaError_t (*mwf)(const float2* x, const double2* R, const float* h, float2* c, int F, int T, int* err,
                     cudaStream_t s);
  int max_T;
};

bool fca_ops(int M, int N, FcaOps* o);

constexpr int kFcaSlots = 4;
constexpr int kFcaMaxThreads = 512;
constexpr int kFcaMaxWarps = kFcaMaxThreads / 32;

// Packed Hermitian M x M (e < M: real diagonal; then pairs a < b row-major: re, im).
template <int M>
__device__ __forceinline__ void unpack_herm(const float* p, float2 (&A)[M][M]) {
#pragma unroll
  for (int a = 0; a < M; ++a) A[a][a] = make_float2(p[a], 0.f);
  int k = M;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = a + 1; b < M; ++b) {
      A[a][b] = make_float2(p[k], p[k + 1]);
      A[b][a] = make_float2(p[k], -p[k + 1]);
      k += 2;
    }
}

// In-register inverse of an HPD matrix by Gauss-Jordan without pivoting; returns
// ln det A = sum ln(pivots) and whether every pivot was positive.
template <int M>
__device__ __forceinline__ float herm_inverse_f32(float2 (&A)[M][M], bool& ok) {
  float logdet = 0.f;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const float d = A[k][k].x;
    ok &= (d > 0.f) && (d < INFINITY);
    logdet += __logf(d);
    const float rd = 1.0f / d;
    float2 rowk[M];
#pragma unroll
    for (int j = 0; j < M; ++j) rowk[j] = A[k][j];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      if (i == k) continue;
      const float2 aik = A[i][k];
#pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j == k) {
          A[i][j] = make_float2(-aik.x * rd, -aik.y * rd);
        } else {
          const float2 pr = cmulf(aik, rowk[j]);
          A[i][j] = make_float2(fmaf(-pr.x, rd, A[i][j].x), fmaf(-pr.y, rd, A[i][j].y));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
      A[k][j] = (j == k) ? make_float2(rd, 0.f) : make_float2(rowk[j].x * rd, rowk[j].y * rd);
  }
  return logdet;
}

template <int M, int N>
struct FcaSmem {
  static constexpr int NE = M * M;
  static constexpr int VP = pow2_ceil(NE);
  static size_t bytes(int threads) {
    const size_t Tp = (size_t)threads * kFcaSlots;
    size_t b = 0;
    b += sizeof(double2) * N * M * M * 3;          // sRd (FP64 R), sRid (FP64 R^{-1}), scratch
    b += sizeof(float2) * N * M * M * 2;           // sRf, sRif (FP32 copies)
    b += sizeof(float) * 2 * kFcaMaxWarps * 32;    // reduction rows
    b += sizeof(float) * kFcaMaxWarps;             // LL partials
    b += sizeof(float) * NE * Tp;                  // X^{-1} packed, [e][t]
    b += sizeof(float) * N * Tp;                   // h, [n][t]
    return b;
  }
};

template <int M, int N>
__global__ void __launch_bounds__(kFcaMaxThreads) fca_em_kernel(FcaArgs p) {
  using SMM = FcaSmem<M, N>;
  constexpr int NE = SMM::NE, VP = SMM::VP;
  const int f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bd = blockDim.x, nw = bd >> 5;
  const int T = p.T;
  const int Tp = bd * kFcaSlots;
  if (f >= p.F) return;
  if (Tp < T || nw > kFcaMaxWarps) {
    if (tid == 0) atomicOr(p.err, kErrConfig);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sRd = reinterpret_cast<double2*>(smem_raw);
  double2* sRid = sRd + N * M * M;
  double2* sScr = sRid + N * M * M;
  float2* sRf = reinterpret_cast<float2*>(sScr + N * M * M);
  float2* sRif = sRf + N * M * M;
  float* sRed = reinterpret_cast<float*>(sRif + N * M * M);
  float* sLL = sRed + 2 * kFcaMaxWarps * 32;
  float* sXi = sLL + kFcaMaxWarps;
  float* sh = sXi + NE * Tp;

  const float2* xf = p.x + (size_t)f * T * M;
  const double invT = 1.0 / (double)T;

  for (int i = tid; i < N * M * M; i += bd) sRd[i] = p.R[(size_t)f * N * M * M + i];
  for (int n = 0; n < N; ++n) {
    const float* hf = p.h + ((size_t)f * N + n) * T;
#pragma unroll
    for (int k = 0; k < kFcaSlots; ++k) {
      const int t = tid + k * bd;
      sh[n * Tp + t] = (t < T) ? hf[t] : 1.0f;
    }
  }
  __syncthreads();

  // R_n^{-1} in FP64 (warp n), FP32 copies of R_n and R_n^{-1}
  auto refresh_inverses = [&]() {
    for (int n = warp; n < N; n += nw) {
      double2* A = sScr + n * M * M;
      for (int e = lane; e < M * M; e += 32) A[e] = sRd[n * M * M + e];
      __syncwarp();
      // in-place HPD inverse (Gauss-Jordan without pivoting)
      for (int k = 0; k < M; ++k) {
        const double d = A[k * M + k].x;
        const bool bad = !(d > 0.0) || !isfinite(d);
        const double rd = rcp_pos_f64(bad ? 1.0 : d);
        double2 nv[(M * M + 31) / 32];
#pragma unroll
        for (int q = 0; q < (M * M + 31) / 32; ++q) {
          const int e = lane + 32 * q;
          if (e < M * M) {
            const int i = e / M, j = e - (e / M) * M;
            const double2 aij = A[e], aik = A[i * M + k], akj = A[k * M + j];
            nv[q] = (i == k) ? ((j == k) ? make_double2(rd, 0.0) : cscale(akj, rd))
                             : ((j == k) ? cscale(aik, -rd) : csub(aij, cscale(cmul(aik, akj), rd)));
          }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < (M * M + 31) / 32; ++q) {
          const int e = lane + 32 * q;
          if (e < M * M) A[e] = nv[q];
        }
        __syncwarp();
        if (bad && lane == 0) atomicOr(p.err, kErrFcaPivot);
      }
      for (int e = lane; e < M * M; e += 32) {
        sRid[n * M * M + e] = A[e];
        sRif[n * M * M + e] = make_float2((float)A[e].x, (float)A[e].y);
        sRf[n * M * M + e] = make_float2((float)sRd[n * M * M + e].x, (float)sRd[n * M * M + e].y);
      }
    }
  };
  refresh_inverses();
  __syncthreads();

  int par = 0;
  for (int it = 0;; ++it) {
    const bool have_ll = (it > 0) || (p.n_iter == 0);
    const bool do_iter = it < p.n_iter;
    // ---- X_t, X_t^{-1} (stored packed), log-likelihood of the current parameters
    {
      float llp = 0.f;
      bool ok = true;
#pragma unroll 1
      for (int k = 0; k < kFcaSlots; ++k) {
        const int t = tid + k * bd;
        if (t < T) {
          float2 X[M][M];
#pragma unroll
          for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) X[a][b] = make_float2(0.f, 0.f);
#pragma unroll
          for (int n = 0; n < N; ++n) {
            const float hn = sh[n * Tp + t];
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
              for (int b = 0; b < M; ++b) {
                const float2 r = sRf[(n * M + a) * M + b];
                X[a][b] = make_float2(fmaf(hn, r.x, X[a][b].x), fmaf(hn, r.y, X[a][b].y));
              }
          }
          const float logdet = herm_inverse_f32<M>(X, ok);
          float2 xv[M];
#pragma unroll
          for (int a = 0; a < M; ++a) xv[a] = __ldg(xf + (size_t)t * M + a);
          float quad = 0.f;
#pragma unroll
          for (int a = 0; a < M; ++a) {
            float2 z = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < M; ++b) z = cfmaf(X[a][b], xv[b], z);
            quad = fmaf(xv[a].x, z.x, fmaf(xv[a].y, z.y, quad));
          }
          llp += logdet + quad;
          // pack X^{-1} (Hermitian) into [e][t]
#pragma unroll
          for (int a = 0; a < M; ++a) sXi[a * Tp + t] = X[a][a].x;
          int e = M;
#pragma unroll
          for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a + 1; b < M; ++b) {
              sXi[e * Tp + t] = 0.5f * (X[a][b].x + X[b][a].x);
              sXi[(e + 1) * Tp + t] = 0.5f * (X[a][b].y - X[b][a].y);
              e += 2;
            }
        }
      }
      if (!ok) atomicOr(p.err, kErrFcaPivot);
      llp = warp_sum(llp);
      if (lane == 0) sLL[warp] = llp;
      __syncthreads();
      if (tid == 0 && have_ll) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += (double)sLL[w];
        const double ll = -s - (double)M * (double)T * kLnPi;
        if (it > 0 && p.ll_hist) p.ll_hist[(size_t)f * p.ll_stride + it - 1] = ll;
        if (!do_iter && p.ll_last) p.ll_last[f] = ll;
      }
    }
    if (!do_iter) break;

    // ---- per source: posterior statistics, h update, R accumulation (Eq. 12-13)
#pragma unroll 1
    for (int n = 0; n < N; ++n) {
      float2 Rn[M][M];
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) Rn[a][b] = sRf[(n * M + a) * M + b];
      float acc[VP];
#pragma unroll
      for (int i = 0; i < VP; ++i) acc[i] = 0.f;
      bool ok = true;
#pragma unroll 1
      for (int k = 0; k < kFcaSlots; ++k) {
        const int t = tid + k * bd;
        if (t < T) {
          float Xp[NE];
#pragma unroll
          for (int e = 0; e < NE; ++e) Xp[e] = sXi[e * Tp + t];
          float2 Xi[M][M];
          unpack_herm<M>(Xp, Xi);
          float2 xv[M];
#pragma unroll
          for (int a = 0; a < M; ++a) xv[a] = __ldg(xf + (size_t)t * M + a);
          const float hn = sh[n * Tp + t];
          // B = R_n X^{-1}
          float2 B[M][M];
#pragma unroll
          for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int c = 0; c < M; ++c) s = cfmaf(Rn[a][c], Xi[c][b], s);
              B[a][b] = s;
            }
          // mu = h B x ; trB = tr(B)
          float2 mu[M];
          float trB = 0.f;
#pragma unroll
          for (int a = 0; a < M; ++a) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < M; ++b) s = cfmaf(B[a][b], xv[b], s);
            mu[a] = make_float2(hn * s.x, hn * s.y);
            trB += B[a][a].x;
          }
          // mu^H R^{-1} mu
          float q = 0.f;
#pragma unroll
          for (int a = 0; a < M; ++a) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < M; ++b) s = cfmaf(sRif[(n * M + a) * M + b], mu[b], s);
            q = fmaf(mu[a].x, s.x, fmaf(mu[a].y, s.y, q));
          }
          const float hnew = (q + hn * (float)M - hn * hn * trB) * (1.0f / (float)M);
          ok &= (hnew > 0.f) && (hnew < INFINITY);
          sh[n * Tp + t] = hnew;
          const float ih = 1.0f / hnew;
          // Psi / hnew, packed: mu mu^H + h R - h^2 B R  (Hermitian)
          int e = 0;
#pragma unroll
          for (int a = 0; a < M; ++a) {
            // diagonal
            float2 br = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < M; ++c) br = cfmaf(B[a][c], Rn[c][a], br);
            const float psi = fmaf(mu[a].x, mu[a].x, mu[a].y * mu[a].y) + hn * Rn[a][a].x - hn * hn * br.x;
            acc[a] = fmaf(psi, ih, acc[a]);
          }
          e = M;
#pragma unroll
          for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a + 1; b < M; ++b) {
              float2 br = make_float2(0.f, 0.f);
#pragma unroll
              for (int c = 0; c < M; ++c) br = cfmaf(B[a][c], Rn[c][b], br);
              // mu_a conj(mu_b)
              const float mre = fmaf(mu[a].x, mu[b].x, mu[a].y * mu[b].y);
              const float mim = fmaf(mu[a].y, mu[b].x, -mu[a].x * mu[b].y);
              const float pre = mre + hn * Rn[a][b].x - hn * hn * br.x;
              const float pim = mim + hn * Rn[a][b].y - hn * hn * br.y;
              acc[e] = fmaf(pre, ih, acc[e]);
              acc[e + 1] = fmaf(pim, ih, acc[e + 1]);
              e += 2;
            }
        }
      }
      if (!ok) atomicOr(p.err, kErrFcaPivot);
      warp_reduce_scatter<VP>(acc, lane);
      {
        float* red = sRed + par * kFcaMaxWarps * 32 + warp * 32;
        if (VP >= 32) {
#pragma unroll
          for (int i = 0; i < VP / 32; ++i) red[lane * (VP / 32) + i] = acc[i];
        } else if ((lane * VP) % 32 == 0) {
          red[(lane * VP) / 32] = acc[0];
        }
      }
      __syncthreads();
      if (tid < NE) {
        const float* red = sRed + par * kFcaMaxWarps * 32;
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += red[w * 32 + tid];
        const double val = (double)s * invT;
        double2* Rd = sRd + n * M * M;
        const int e = tid;
        if (e < M) {
          Rd[e * M + e] = make_double2(val, 0.0);
        } else {
          int idx = (e - M) >> 1;
          const bool im = ((e - M) & 1) != 0;
          int a = 0;
          while (idx >= M - 1 - a) { idx -= M - 1 - a; ++a; }
          const int b = a + 1 + idx;
          if (!im) { Rd[a * M + b].x = val; Rd[b * M + a].x = val; }
          else { Rd[a * M + b].y = val; Rd[b * M + a].y = -val; }
        }
      }
      par ^= 1;
    }
    __syncthreads();
    refresh_inverses();
    __syncthreads();
  }
  __syncthreads();
  for (int i = tid; i < N * M * M; i += bd) p.R[(size_t)f * N * M * M + i] = sRd[i];
  for (int n = 0; n < N; ++n) {
    float* hf = p.h + ((size_t)f * N + n) * T;
#pragma unroll
    for (int k = 0; k < kFcaSlots; ++k) {
      const int t = tid + k * bd;
      if (t < T) hf[t] = sh[n * Tp + t];
    }
  }
}

// FCA Wiener filter (Eq. 7): c_tn = h_nt R_n X_t^{-1} x_t.  One thread per frame.
template <int M, int N>
__global__ void __launch_bounds__(128) fca_mwf_kernel(const float2* __restrict__ x, const double2* __restrict__ R,
                                                      const float* __restrict__ h, float2* __restrict__ c,
                                                      int F, int T, int* err) {
  __shared__ float2 sR[N * M * M];
  const int f = blockIdx.x;
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  for (int e = threadIdx.x; e < N * M * M; e += blockDim.x) {
    const double2 r = R[(size_t)f * N * M * M + e];
    sR[e] = make_float2((float)r.x, (float)r.y);
  }
  __syncthreads();
  if (t >= T) return;
  float hv[N];
#pragma unroll
  for (int n = 0; n < N; ++n) hv[n] = h[((size_t)f * N + n) * T + t];
  float2 X[M][M];
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < M; ++b) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int n = 0; n < N; ++n) {
        const float2 r = sR[(n * M + a) * M + b];
        s = make_float2(fmaf(hv[n], r.x, s.x), fmaf(hv[n], r.y, s.y));
      }
      X[a][b] = s;
    }
  bool ok = true;
  herm_inverse_f32<M>(X, ok);
  if (!ok) atomicOr(err, kErrFcaPivot);
  float2 xv[M];
#pragma unroll
  for (int a = 0; a < M; ++a) xv[a] = x[((size_t)f * T + t) * M + a];
  float2 z[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < M; ++b) s = cfmaf(X[a][b], xv[b], s);
    z[a] = s;
  }
  float2* out = c + ((size_t)f * T + t) * N * M;
#pragma unroll
  for (int n = 0; n < N; ++n) {
#pragma unroll
    for (int a = 0; a < M; ++a) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < M; ++b) s = cfmaf(sR[(n * M + a) * M + b], z[b], s);
      out[n * M + a] = make_float2(hv[n] * s.x, hv[n] * s.y);
    }
  }
}

inline int fca_threads(int T) {
  const int warps = (T + 32 * kFcaSlots - 1) / (32 * kFcaSlots);
  return (warps < 1 ? 1 : warps) * 32;
}

template <int M, int N>
cudaError_t launch_fca_em(const FcaArgs& a, FcaWork*, cudaStream_t s) {
  const int threads = fca_threads(a.T);
  if (threads > kFcaMaxThreads) return cudaErrorInvalidConfiguration;
  const size_t smem = FcaSmem<M, N>::bytes(threads);
  cudaError_t e = cudaFuncSetAttribute(fca_em_kernel<M, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fca_em_kernel<M, N><<<a.F, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int M, int N>
cudaError_t launch_fca_mwf(const float2* x, const double2* R, const float* h, float2* c, int F, int T, int* err,
                           cudaStream_t s) {
  dim3 grid(F, (T + 127) / 128);
  fca_mwf_kernel<M, N><<<grid, 128, 0, s>>>(x, R, h, c, F, T, err);
  return cudaGetLastError();
}

template <int M, int N>
FcaOps make_fca_ops() {
  FcaOps o;
  o.em = &launch_fca_em<M, N>;
  o.mwf = &launch_fca_mwf<M, N>;
  o.max_T = kFcaMaxThreads * kFcaSlots;
  return o;
}

}  // namespace ffca

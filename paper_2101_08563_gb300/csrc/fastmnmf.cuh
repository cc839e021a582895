// FastMNMF (Sec. IV-H, App. C): the FastFCA model with the source powers factored across
// frequencies by NMF, h_ijn = sum_k t_ikn v_jkn (Eq. 52), fitted by minimising Eq. 53.
//
// One iteration (IP for W, then the exponent-1/2 MM rules of IS-NMF for lambda, t, v in that
// order, sigma^2 recomputed before each) is four launches, each shaped for its work:
//   fastmnmf_freq_kernel, one CTA per frequency i (frames owned as in fastfca_em_kernel):
//     h_ijn = sum_k t_ikn v_jkn (read: the previous activation update wrote it)   Eq. 52
//     sigma^2 = Lambda_i h, log-likelihood of the incoming parameters       Eq. 28, Eq. 53
//     Q_m, IP (FP64), U = |W^H x|^2                                           Eq. 33-35, 37
//     lambda_imn *= (sum_j h U/sigma^4 / sum_j h/sigma^2)^1/2
//     then, with sigma^2 from the new lambda: a_ijn = sum_m lambda_imn U_mij/sigma^4_mij and
//     b_ijn = sum_m lambda_imn/sigma^2_mij, written with U
//   fastmnmf_t_kernel: t_ikn *= (sum_j v_jkn a_ijn / sum_j v_jkn b_ijn)^1/2 -- a contraction
//     over frames with v staged once per CTA in shared memory for 16 frequencies
//   fastmnmf_ab_kernel: a, b again with sigma^2 from the new t (h = t v recomputed per bin,
//     each thread's v column in registers across a tile of frequencies)
//   fastmnmf_v_kernel: v_jkn *= (sum_i t_ikn a_ijn / sum_i t_ikn b_ijn)^1/2, the sum over
//     every frequency (the step that couples the bins), then h = t v of the new t and v for
//     the next iteration and for the Wiener filter.
// The per-frequency kernel holds the latency-bound part (reductions, FP64 IP); the three
// contractions over v run in kernels that read v once per tile instead of once per frequency.
//
// Layouts: t (bases) F x N x K, t_ikn at tb[(i N + n) K + k]; v (activations) N x K x T,
// v_jkn at va[(n K + k) T + j] (frames contiguous, so a warp's reads of one v row coalesce);
// a and b: two planes F x N x T; U: F x M x T.  W, W^{-H} and |det W|^2 are carried between
// launches as in the FastFCA kernels.
#pragma once
#include "fastfca_em.cuh"

namespace ffca {

constexpr int kMnmfMaxK = 16;      // bases per source
static_assert(2 * kMnmfMaxK == 32, "the t update reduces num and den of one source as one 32-wide row");
constexpr int kMnmfMaxFK = 36864;  // the activation update stages t[:, n, :] (F*K floats) on chip

struct MnmfArgs {
  const float2* x;     // F x T x M
  double2* P;          // F x M x M, W[a][m]
  double2* Bst;        // F x M x M, W^{-H}
  double* detst;       // F x 2, |det W|^2 as (mantissa, exponent)
  int b_valid;         // Bst/detst are current
  float* lam;          // F x M x N
  const float* hin;    // F x N x T: h = t v of the incoming t and v (Eq. 52)
  float* ab;           // 2 x F x N x T (a plane, then b plane); written when iterating
  float* u;            // F x M x T: U = |W^H x|^2 of the new W; written when iterating
  double* ll_out;      // log-likelihood of the incoming parameters at ll_out[f * ll_stride], or null
  double* ll_last;     // F or null: the same value, when only the log-likelihood is asked for
  int* err;
  int F, T, ll_stride;
  int iterate;         // 1: one iteration; 0: log-likelihood only
  int N;               // sources (the cluster form takes N at run time)
};

template <int M, int N>
struct MnSmem {
  using E = EmSmem<M, N>;
  static size_t bytes(int threads) {
    size_t b = 0;
    b += sizeof(double2) * M * M * 2;        // sW, sB
    b += sizeof(double2) * E::kQsz;          // sQ
    b += sizeof(double) * 4;                 // sDet
    b += sizeof(float2) * E::kWcPad;         // sWc
    b += sizeof(float) * ((M * N + 3) & ~3); // sL
    b += sizeof(float) * 2 * kMaxWarps * 32; // reduction rows
    b += sizeof(float) * kMaxWarps;          // sLL
    b += sizeof(float) * (size_t)threads * (kSlots * N + 1);   // sH, thread-major
    b += sizeof(float) * (size_t)threads * (kSlots * M + 1);   // sU, thread-major
    return b;
  }
};

template <int M, int N>
__global__ void __maxnreg__(kEmMaxRegs) fastmnmf_freq_kernel(MnmfArgs p) {
  using SM = EmSmem<M, N>;
  constexpr int QCH = SM::kQCH, MC = SM::kMC, V = SM::kV, VP = SM::kVP;
  constexpr int NE = M * M;
  const int f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bd = blockDim.x, nw = bd >> 5;
  const int T = p.T;
  if (f >= p.F) return;
  if (bd * kSlots < T || bd > kMaxThreads) {    // uniform
    if (tid == 0) atomicOr(p.err, kErrConfig);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sW = reinterpret_cast<double2*>(smem_raw);
  double2* sB = sW + M * M;
  double2* sQ = sB + M * M;
  double* sDet = reinterpret_cast<double*>(sQ + SM::kQsz);
  float2* sWc = reinterpret_cast<float2*>(sDet + 4);
  float* sL = reinterpret_cast<float*>(sWc + SM::kWcPad);
  float* sRed = sL + ((M * N + 3) & ~3);
  float* sLL = sRed + 2 * kMaxWarps * 32;
  float* sH = sLL + kMaxWarps;
  constexpr int SH = kSlots * N + 1, SU = kSlots * M + 1;
  float* sU = sH + bd * SH;
  float* pH = sH + tid * SH;
  float* pU = sU + tid * SU;

  const float2* xf = p.x + (size_t)f * T * M;
  const double invT = 1.0 / (double)T;
  const bool need_ll = !p.iterate || p.ll_out != nullptr;

  // ---- parameters of frequency f; B = W^{-H} and |det W|^2 carried over or formed once
  for (int i = tid; i < M * N; i += bd) sL[i] = p.lam[(size_t)f * M * N + i];
  for (int i = tid; i < M * M; i += bd) sW[i] = p.P[(size_t)f * M * M + i];
  __syncthreads();
  if (warp == 0) {
    if (p.b_valid) {
      for (int e = lane; e < M * M; e += 32) sB[e] = p.Bst[(size_t)f * M * M + e];
      if (lane == 0) { sDet[0] = p.detst[2 * f]; sDet[1] = p.detst[2 * f + 1]; }
    } else {
      for (int e = lane; e < M * M; e += 32) {
        const int i = e / M, j = e - (e / M) * M;
        const double2 w = sW[j * M + i];
        sQ[e] = make_double2(w.x, -w.y);
      }
      __syncwarp();
      double mant, expo;
      warp_inverse_pivot<M>(sQ, sQ + M * M, sB, mant, expo, lane, p.err);
      if (lane == 0) { sDet[0] = mant; sDet[1] = expo; }
    }
    for (int e = lane; e < M * M; e += 32) {
      const int a = e / M, m = e - (e / M) * M;
      const double2 w = sW[a * M + m];
      sWc[m * M + a] = make_float2((float)w.x, (float)-w.y);
    }
  }

  auto load_x = [&](int t, float2 (&xv)[M]) {
    const float2* src = xf + (size_t)t * M;
    if constexpr (M % 2 == 0) {
#pragma unroll
      for (int a = 0; a < M; a += 2) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(src + a));
        xv[a] = make_float2(q.x, q.y);
        xv[a + 1] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) xv[a] = __ldg(src + a);
    }
  };
  auto pass_U = [&]() {
    float2 wc[M * M];
#pragma unroll
    for (int i = 0; i < M * M; ++i) wc[i] = sWc[i];
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int t = tid + k * bd;
      if (t < T) {
        float2 xv[M];
        load_x(t, xv);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float2 y = make_float2(0.f, 0.f);
#pragma unroll
          for (int a = 0; a < M; ++a) y = cfmaf(wc[m * M + a], xv[a], y);
          pU[k * M + m] = fmaf(y.x, y.x, y.y * y.y);
        }
      }
    }
  };
  // r[k][m] = 1/sigma^2 of the current lambda and h; optionally the log-likelihood terms
  float r[kSlots][M];
  auto pass_sigma = [&](bool ll, float& llp) -> bool {
    float Lr[M][N];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int n = 0; n < N; ++n) Lr[m][n] = sL[m * N + n];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int t = tid + k * bd;
      if (t < T) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float s2 = 0.f;
#pragma unroll
          for (int n = 0; n < N; ++n) s2 = fmaf(Lr[m][n], pH[k * N + n], s2);
          bad |= !(s2 > 0.f && s2 < INFINITY);
          const float rs = fast_rcp(s2);
          r[k][m] = rs;
          if (ll) llp += fmaf(pU[k * M + m], rs, __logf(s2));
        }
      }
    }
    return bad;
  };

  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSlots; ++k) {
    const int t = tid + k * bd;
    if (t < T) {
#pragma unroll
      for (int n = 0; n < N; ++n) pH[k * N + n] = __ldg(p.hin + ((size_t)f * N + n) * T + t);
    }
  }
  if (need_ll) pass_U();
  int par = 0;
  {
    float llp = 0.f;
    if (pass_sigma(need_ll, llp)) atomicOr(p.err, kErrSigma);
    if (need_ll) {
      llp = warp_sum(llp);
      if (lane == 0) sLL[warp] = llp;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += (double)sLL[w];
        const double logdet = (double)__logf((float)sDet[0]) + sDet[1] * kLn2;
        const double ll = (double)T * logdet - s - (double)M * (double)T * kLnPi;
        if (p.ll_out) p.ll_out[(size_t)f * p.ll_stride] = ll;
        if (!p.iterate && p.ll_last) p.ll_last[f] = ll;
      }
    }
  }
  if (!p.iterate) {
    __syncthreads();
    if (!p.b_valid) {
      for (int i = tid; i < M * M; i += bd) p.Bst[(size_t)f * M * M + i] = sB[i];
      if (tid == 0) { p.detst[2 * f] = sDet[0]; p.detst[2 * f + 1] = sDet[1]; }
    }
    return;
  }

  // ---- Q_m = (1/T) sum_t x x^H / sigma^2_m (Eq. 33), chunk by chunk over m
#pragma unroll 1
  for (int c = 0; c < QCH; ++c) {
    float acc[VP];
#pragma unroll
    for (int i = 0; i < VP; ++i) acc[i] = 0.f;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int t = tid + k * bd;
      if (t < T) {
        float2 xv[M];
        load_x(t, xv);
        float e[NE];
        xxh_packed<M>(xv, e);
#pragma unroll
        for (int mm = 0; mm < MC; ++mm) {
          float w = r[k][mm];
#pragma unroll
          for (int cc = 1; cc < QCH; ++cc)
            if (cc == c) w = r[k][cc * MC + mm];
#pragma unroll
          for (int q = 0; q < NE; ++q) acc[mm * NE + q] = fmaf(w, e[q], acc[mm * NE + q]);
        }
      }
    }
    warp_reduce_scatter<VP>(acc, lane);
    {
      float* red = sRed + par * kMaxWarps * 32 + warp * 32;
      if (VP >= 32) {
#pragma unroll
        for (int i = 0; i < VP / 32; ++i) red[lane * (VP / 32) + i] = acc[i];
      } else if ((lane * VP) % 32 == 0) {
        red[(lane * VP) / 32] = acc[0];
      }
    }
    __syncthreads();
    if (tid < V) {
      const float* red = sRed + par * kMaxWarps * 32;
      float q = 0.f;
      for (int w = 0; w < nw; ++w) q += red[w * 32 + tid];
      const int mm = tid / NE, e = tid - mm * NE;
      const int m = c * MC + mm;
      double2* Qm = sQ + m * M * M;
      const double qd = (double)q * invT;
      if (e < M) {
        Qm[e * M + e] = make_double2(qd, 0.0);
      } else {
        int idx = (e - M) >> 1;
        const bool im = ((e - M) & 1) != 0;
        int a = 0;
        while (idx >= M - 1 - a) { idx -= M - 1 - a; ++a; }
        const int b = a + 1 + idx;
        if (!im) { Qm[a * M + b].x = qd; Qm[b * M + a].x = qd; }
        else { Qm[a * M + b].y = qd; Qm[b * M + a].y = -qd; }
      }
    }
    par ^= 1;
  }
  __syncthreads();

  // ---- IP in FP64 (Eq. 34-35), then U = |W^H x|^2 (Eq. 37)
  if (warp == 0) warp_hpd_inverse_all<M>(sQ, lane, p.err);
  __syncwarp();
  if (warp == 0) ip_columns<M>(sQ, sW, sB, sWc, sDet, lane, p.err);
  __syncthreads();
  pass_U();

  // ---- lambda <- lambda (.) {[U (.) sigma^-4] h^T / sigma^-2 h^T}^1/2 (r: 1/sigma^2 of the
  // incoming lambda and h, unchanged since), sources in chunks of NC
  {
    constexpr int NC = (N < 16 / M) ? N : 16 / M;
    constexpr int VLP = pow2_ceil(2 * M * NC);
#pragma unroll 1
    for (int n0 = 0; n0 < N; n0 += NC) {
      float acc[VLP];
#pragma unroll
      for (int i = 0; i < VLP; ++i) acc[i] = 0.f;
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const int t = tid + k * bd;
        if (t < T) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float rs = r[k][m];
            const float a = pU[k * M + m] * rs * rs;
#pragma unroll
            for (int nc = 0; nc < NC; ++nc) {
              const int n = n0 + nc < N ? n0 + nc : N - 1;    // a partial last chunk's extra sums are unused
              const float h = pH[k * N + n];
              acc[m * NC + nc] = fmaf(a, h, acc[m * NC + nc]);
              acc[M * NC + m * NC + nc] = fmaf(rs, h, acc[M * NC + m * NC + nc]);
            }
          }
        }
      }
      warp_reduce_scatter<VLP>(acc, lane);
      {
        float* red = sRed + par * kMaxWarps * 32 + warp * 32;
        if ((lane * VLP) % 32 == 0) red[(lane * VLP) / 32] = acc[0];
      }
      __syncthreads();
      if (tid < M * NC) {
        const int m = tid / NC, nc = tid - (tid / NC) * NC;
        if (n0 + nc < N) {
          const float* red = sRed + par * kMaxWarps * 32;
          float num = 0.f, den = 0.f;
          for (int w = 0; w < nw; ++w) {
            num += red[w * 32 + m * NC + nc];
            den += red[w * 32 + M * NC + m * NC + nc];
          }
          sL[m * N + n0 + nc] *= (den > 0.f) ? sqrtf(num / den) : 1.0f;
        }
      }
      par ^= 1;
    }
  }
  __syncthreads();

  // ---- the t update's per-bin terms with sigma^2 from the new lambda and the incoming h:
  // a_jn = sum_m lambda_mn U_mj / sigma^4_mj, b_jn = sum_m lambda_mn / sigma^2_mj, written with
  // U for the kernels that finish the iteration
  {
    float dummy = 0.f;
    if (pass_sigma(false, dummy)) atomicOr(p.err, kErrSigma);
    float Lr[M][N];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int n = 0; n < N; ++n) Lr[m][n] = sL[m * N + n];
    float* ap = p.ab + (size_t)f * N * T;
    float* bp = p.ab + (size_t)p.F * N * T + (size_t)f * N * T;
    float* up = p.u + (size_t)f * M * T;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int t = tid + k * bd;
      if (t < T) {
        float e[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float u = pU[k * M + m];
          e[m] = u * r[k][m] * r[k][m];
          up[(size_t)m * T + t] = u;
        }
#pragma unroll
        for (int n = 0; n < N; ++n) {
          float av = 0.f, bv = 0.f;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            av = fmaf(Lr[m][n], e[m], av);
            bv = fmaf(Lr[m][n], r[k][m], bv);
          }
          ap[(size_t)n * T + t] = av;
          bp[(size_t)n * T + t] = bv;
        }
      }
    }
  }

  // ---- write back
  __syncthreads();
  for (int i = tid; i < M * N; i += bd) p.lam[(size_t)f * M * N + i] = sL[i];
  for (int i = tid; i < M * M; i += bd) {
    p.P[(size_t)f * M * M + i] = sW[i];
    p.Bst[(size_t)f * M * M + i] = sB[i];
  }
  if (tid == 0) {
    p.detst[2 * f] = sDet[0];
    p.detst[2 * f + 1] = sDet[1];
  }
}

// The cross-frequency v update, h for the filter, and the default start (fastmnmf_common.cu).
// v_jkn <- v_jkn (sum_i t_ikn a_ijn / sum_i t_ikn b_ijn)^1/2 over every frequency i, then
// h = t v (Eq. 52) of the new v into h (F x N x T).
cudaError_t launch_mnmf_v(const float* tb, const float* ab, float* va, float* h, int F, int N, int K, int T,
                          cudaStream_t s);
// t_ikn *= (sum_j v_jkn a_ijn / sum_j v_jkn b_ijn)^1/2 for every frequency.
cudaError_t launch_mnmf_t(float* tb, const float* va, const float* ab, int F, int N, int K, int T, cudaStream_t s);
// h_ijn = sum_k t_ikn v_jkn (Eq. 52) as F x N x T (the FastFCA filter's H layout).
cudaError_t launch_mnmf_h(const float* tb, const float* va, float* h, int F, int N, int K, int T, cudaStream_t s);
// Default start: W = I, lambda = 1; with p_ij = ||x_ij||^2 / (M N),
// t_ikn = (mean_j p_ij / K) u and v_jkn = (mean_i p_ij / mean_ij p_ij) u', u and u' ~ U[0.5, 1.5)
// from Philox4x32-10 keyed by `seed` (counters (i, n, k, 0x7a11) and (j, n, k, 0x7a12)).
// `scratch` holds F + T + 1 floats.
cudaError_t launch_mnmf_default(const float2* x, double2* P, float* lam, float* tb, float* va, float* scratch, int F,
                                int T, int M, int N, int K, uint32_t seed, cudaStream_t s);

// a_ijn = sum_m lambda_imn U_mij / sigma^4_mij and b_ijn = sum_m lambda_imn / sigma^2_mij with
// sigma^2_mij = sum_n lambda_imn h_ijn, h_ijn = sum_k t_ikn v_jkn (the current t and v).
// Grid (ceil(T / 128), ceil(F / kMnmfAbFreqs)), 128 threads, one frame each; the CTA's
// v[:, :, frames] (N K x 128 floats) is staged once in shared memory and serves every
// frequency of the tile; t and lambda of the tile are staged too.
constexpr int kMnmfAbFreqs = 8;
constexpr int kMnmfAbFrames = 128;

template <int M, int N>
__global__ void __launch_bounds__(kMnmfAbFrames) fastmnmf_ab_kernel(const float* __restrict__ lam,
                                                                    const float* __restrict__ tb,
                                                                    const float* __restrict__ va,
                                                                    const float* __restrict__ u,
                                                                    float* __restrict__ ab, int F, int K, int T,
                                                                    int* err) {
  extern __shared__ __align__(16) float sab[];
  float* sV = sab;                                       // [n K + k][jj]
  float* sTt = sV + (size_t)N * K * kMnmfAbFrames;       // [ii][n K + k]
  float* sLm = sTt + (size_t)kMnmfAbFreqs * N * K;       // [ii][m N + n]
  const int jj = threadIdx.x;
  const int j = blockIdx.x * kMnmfAbFrames + jj;
  const int i0 = blockIdx.y * kMnmfAbFreqs;
  const int NK = N * K;
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
    float h[N];
#pragma unroll
    for (int n = 0; n < N; ++n) {
      float s = 0.f;
#pragma unroll 4
      for (int k = 0; k < K; ++k) s = fmaf(tr[n * K + k], sV[(n * K + k) * kMnmfAbFrames + jj], s);
      h[n] = s;
    }
    float e[M], r[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float s2 = 0.f;
#pragma unroll
      for (int n = 0; n < N; ++n) s2 = fmaf(lr[m * N + n], h[n], s2);
      bad |= !(s2 > 0.f && s2 < INFINITY);
      r[m] = fast_rcp(s2);
      e[m] = __ldg(u + ((size_t)i * M + m) * T + j) * r[m] * r[m];
    }
#pragma unroll
    for (int n = 0; n < N; ++n) {
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
  if (bad) atomicOr(err, kErrSigma);
}

inline size_t mnmf_ab_smem(int M, int N, int K) {
  return sizeof(float) * ((size_t)N * K * kMnmfAbFrames + (size_t)kMnmfAbFreqs * N * K + (size_t)kMnmfAbFreqs * M * N);
}

template <int M, int N>
cudaError_t launch_mnmf_ab_mn(const float* lam, const float* tb, const float* va, const float* u, float* ab, int F,
                              int /*N, a template parameter here*/, int K, int T, int* err, cudaStream_t s) {
  const size_t smem = mnmf_ab_smem(M, N, K);
  cudaError_t e = cudaFuncSetAttribute(fastmnmf_ab_kernel<M, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((T + kMnmfAbFrames - 1) / kMnmfAbFrames, (F + kMnmfAbFreqs - 1) / kMnmfAbFreqs);
  fastmnmf_ab_kernel<M, N><<<grid, kMnmfAbFrames, smem, s>>>(lam, tb, va, u, ab, F, K, T, err);
  return cudaGetLastError();
}

struct MnmfOps {
  cudaError_t (*freq)(const MnmfArgs& a, cudaStream_t s);
  cudaError_t (*ab)(const float* lam, const float* tb, const float* va, const float* u, float* ab, int F, int N,
                    int K, int T, int* err, cudaStream_t s);
  int max_T;
};

bool mnmf_ops_m2(int N, MnmfOps* o);
bool mnmf_ops_m3(int N, MnmfOps* o);
bool mnmf_ops_m4(int N, MnmfOps* o);
inline bool mnmf_ops(int M, int N, MnmfOps* o) {
  switch (M) {
    case 2: return mnmf_ops_m2(N, o);
    case 3: return mnmf_ops_m3(N, o);
    case 4: return mnmf_ops_m4(N, o);
    default: return false;
  }
}
// The per-frequency step on thread-block clusters (the FastFCA cluster kernel's MN form) for
// shapes the frequency-resident kernel does not take: M <= 8, N <= 16, T as the cluster
// kernel fits (fastmnmf_cluster.cuh; defined with the cluster kernels).
bool mnmf_cluster_ops(int M, int N, int T, MnmfOps* o);

template <int M, int N>
cudaError_t launch_mnmf_freq(const MnmfArgs& a, cudaStream_t s) {
  int warps = (a.T + 32 * kSlots - 1) / (32 * kSlots);
  if (warps < 1) warps = 1;
  const int threads = warps * 32;
  if (threads > kMaxThreads) return cudaErrorInvalidConfiguration;
  const size_t smem = MnSmem<M, N>::bytes(threads);
  cudaError_t e =
      cudaFuncSetAttribute(fastmnmf_freq_kernel<M, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fastmnmf_freq_kernel<M, N><<<a.F, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int M, int N>
MnmfOps make_mnmf_ops() {
  MnmfOps o;
  o.freq = &launch_mnmf_freq<M, N>;
  o.ab = &launch_mnmf_ab_mn<M, N>;
  o.max_T = kMaxThreads * kSlots;
  return o;
}

// Instantiations of one M (one translation unit per M).
template <int M>
bool mnmf_ops_for_m(int N, MnmfOps* o) {
  switch (N) {
    case 2: *o = make_mnmf_ops<M, 2>(); return true;
    case 3: *o = make_mnmf_ops<M, 3>(); return true;
    case 4: *o = make_mnmf_ops<M, 4>(); return true;
    case 5: *o = make_mnmf_ops<M, 5>(); return true;
    case 6: *o = make_mnmf_ops<M, 6>(); return true;
    case 7: *o = make_mnmf_ops<M, 7>(); return true;
    case 8: *o = make_mnmf_ops<M, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffca

// FastMNMF (Sec. IV-H, App. C): the FastFCA model with the source powers factored across
// frequencies by NMF, h_ijn = sum_k t_ikn v_jkn (Eq. 52), fitted by minimising Eq. 53.
//
// One iteration (IP for W, then the exponent-1/2 MM rules of IS-NMF for lambda, t, v in that
// order, sigma^2 recomputed before each):
//   fastmnmf_freq_kernel, one CTA per frequency i (frames owned as in fastfca_em_kernel):
//     h_ijn = sum_k t_ikn v_jkn  (read: the previous activation update wrote it)  Eq. 52
//     sigma^2 = Lambda_i h, log-likelihood of the incoming parameters    Eq. 28, Eq. 53
//     Q_m, IP (FP64), U = |W^H x|^2                                        Eq. 33-35, 37
//     lambda_imn *= (sum_j h U/sigma^4 / sum_j h/sigma^2)^1/2
//     t_ikn *= (sum_j v_jkn a_ijn / sum_j v_jkn b_ijn)^1/2, with sigma^2 from the new lambda,
//        a_ijn = sum_m lambda_imn U_mij/sigma^4_mij, b_ijn = sum_m lambda_imn/sigma^2_mij
//     a_ijn, b_ijn again with sigma^2 from the new t, written to memory for the v update
//   fastmnmf_v_kernel: v_jkn *= (sum_i t_ikn a_ijn / sum_i t_ikn b_ijn)^1/2, the sum over
//     every frequency (the step that couples the bins), then h = t v of the new t and v for
//     the next iteration and for the Wiener filter.
//
// Layouts: t (bases) F x N x K, t_ikn at tb[(i N + n) K + k]; v (activations) N x K x T,
// v_jkn at va[(n K + k) T + j] (frames contiguous, so a warp's reads of one v row coalesce);
// a and b: two planes F x N x T.  W, W^{-H} and |det W|^2 are carried between launches as in
// the FastFCA kernels.
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
  float* tb;           // F x N x K
  const float* va;     // N x K x T
  const float* hin;    // F x N x T: h = t v of the incoming t and v (Eq. 52)
  float* ab;           // 2 x F x N x T (a plane, then b plane); written when iterating
  double* ll_out;      // log-likelihood of the incoming parameters at ll_out[f * ll_stride], or null
  double* ll_last;     // F or null: the same value, when only the log-likelihood is asked for
  int* err;
  int F, T, K, ll_stride;
  int iterate;         // 1: one iteration; 0: log-likelihood only
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
    b += sizeof(float) * N * kMnmfMaxK;      // sT
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
  const int T = p.T, K = p.K;
  if (f >= p.F) return;
  if (bd * kSlots < T || bd > kMaxThreads || K < 1 || K > kMnmfMaxK) {    // uniform
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
  float* sT = sL + ((M * N + 3) & ~3);
  float* sRed = sT + N * kMnmfMaxK;
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
  for (int i = tid; i < N * K; i += bd) sT[i] = p.tb[(size_t)f * N * K + i];
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
  // h_n = sum_k t_nk v_nk(t) for this thread's frames (Eq. 52), into pH.  The frame slots
  // are the inner loop, so each basis issues kSlots independent coalesced loads of v.
  auto pass_h = [&]() {
#pragma unroll 1
    for (int n = 0; n < N; ++n) {
      float hs[kSlots];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) hs[k] = 0.f;
      const float* vr = p.va + (size_t)n * K * T + tid;
#pragma unroll 2
      for (int kk = 0; kk < K; ++kk) {
        const float tv = sT[n * K + kk];
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
          if (tid + k * bd < T) hs[k] = fmaf(tv, __ldg(vr + (size_t)kk * T + k * bd), hs[k]);
      }
#pragma unroll
      for (int k = 0; k < kSlots; ++k)
        if (tid + k * bd < T) pH[k * N + n] = hs[k];
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

  // ---- t_nk <- t_nk (sum_j v_nk a_n / sum_j v_nk b_n)^1/2, a and b with sigma^2 from the new
  // lambda and the incoming t (pH); one source per pass: a_n, b_n of the thread's frames in
  // registers, then every basis's v row with the frame slots as the inner loop
  {
    float dummy = 0.f;
    if (pass_sigma(false, dummy)) atomicOr(p.err, kErrSigma);     // r = 1/sigma^2, new lambda
#pragma unroll 1
    for (int n = 0; n < N; ++n) {
      float av[kSlots], bv[kSlots];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        av[k] = 0.f;
        bv[k] = 0.f;
        if (tid + k * bd < T) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float rs = r[k][m];
            const float l = sL[m * N + n];
            av[k] = fmaf(l, pU[k * M + m] * rs * rs, av[k]);
            bv[k] = fmaf(l, rs, bv[k]);
          }
        }
      }
      float acc[2 * kMnmfMaxK];
      const float* vr = p.va + (size_t)n * K * T + tid;
#pragma unroll
      for (int kk = 0; kk < kMnmfMaxK; ++kk) {
        float sn = 0.f, sd = 0.f;
        if (kk < K) {
#pragma unroll
          for (int k = 0; k < kSlots; ++k) {
            if (tid + k * bd < T) {
              const float vv = __ldg(vr + (size_t)kk * T + k * bd);
              sn = fmaf(vv, av[k], sn);
              sd = fmaf(vv, bv[k], sd);
            }
          }
        }
        acc[kk] = sn;
        acc[kMnmfMaxK + kk] = sd;
      }
      warp_reduce_scatter<2 * kMnmfMaxK>(acc, lane);
      sRed[par * kMaxWarps * 32 + warp * 32 + lane] = acc[0];
      __syncthreads();
      if (tid < K) {
        const float* red = sRed + par * kMaxWarps * 32;
        float num = 0.f, den = 0.f;
        for (int w = 0; w < nw; ++w) {
          num += red[w * 32 + tid];
          den += red[w * 32 + kMnmfMaxK + tid];
        }
        sT[n * K + tid] *= (den > 0.f) ? sqrtf(num / den) : 1.0f;
      }
      par ^= 1;
    }
  }
  __syncthreads();

  // ---- a, b with sigma^2 from the new t, for the v update over all frequencies
  pass_h();
  {
    float Lr[M][N];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int n = 0; n < N; ++n) Lr[m][n] = sL[m * N + n];
    float* ap = p.ab + (size_t)f * N * T;
    float* bp = p.ab + (size_t)p.F * N * T + (size_t)f * N * T;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int t = tid + k * bd;
      if (t < T) {
        float e[M], s[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float s2 = 0.f;
#pragma unroll
          for (int n = 0; n < N; ++n) s2 = fmaf(Lr[m][n], pH[k * N + n], s2);
          bad |= !(s2 > 0.f && s2 < INFINITY);
          s[m] = fast_rcp(s2);
          e[m] = pU[k * M + m] * s[m] * s[m];
        }
#pragma unroll
        for (int n = 0; n < N; ++n) {
          float a = 0.f, b = 0.f;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            a = fmaf(Lr[m][n], e[m], a);
            b = fmaf(Lr[m][n], s[m], b);
          }
          ap[(size_t)n * T + t] = a;
          bp[(size_t)n * T + t] = b;
        }
      }
    }
    if (bad) atomicOr(p.err, kErrSigma);
  }

  // ---- write back
  __syncthreads();
  for (int i = tid; i < M * N; i += bd) p.lam[(size_t)f * M * N + i] = sL[i];
  for (int i = tid; i < N * K; i += bd) p.tb[(size_t)f * N * K + i] = sT[i];
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
// h_ijn = sum_k t_ikn v_jkn (Eq. 52) as F x N x T (the FastFCA filter's H layout).
cudaError_t launch_mnmf_h(const float* tb, const float* va, float* h, int F, int N, int K, int T, cudaStream_t s);
// Default start: W = I, lambda = 1; with p_ij = ||x_ij||^2 / (M N),
// t_ikn = (mean_j p_ij / K) u and v_jkn = (mean_i p_ij / mean_ij p_ij) u', u and u' ~ U[0.5, 1.5)
// from Philox4x32-10 keyed by `seed` (counters (i, n, k, 0x7a11) and (j, n, k, 0x7a12)).
// `scratch` holds F + T + 1 floats.
cudaError_t launch_mnmf_default(const float2* x, double2* P, float* lam, float* tb, float* va, float* scratch, int F,
                                int T, int M, int N, int K, uint32_t seed, cudaStream_t s);

struct MnmfOps {
  cudaError_t (*freq)(const MnmfArgs& a, cudaStream_t s);
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

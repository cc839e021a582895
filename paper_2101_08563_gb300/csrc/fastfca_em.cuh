// FastFCA IP+EM (Algorithm 1), frequency-resident: one CTA owns one frequency bin f and runs
// every iteration on it without leaving the SM.
//
// Per iteration and frequency (Sec. IV-E, Algorithm 1):
//   sigma^2 = L H                                   Eq. 28, Eq. 38
//   Q_m = (1/T) sum_t x_t x_t^H / sigma^2_{mt}       Eq. 33   (all m in one pass over t)
//   for m: w_m <- (W^H Q_m)^{-1} e_m, normalise      Eq. 34-35 (FP64, see ip_sweep below)
//   U_{mt} = |w_m^H x_t|^2                           Eq. 37
//   for n: G_n, Phi_n, L[:,n], H[n,:]                Algorithm 1 n-loop (Gauss-Seidel)
//   log-likelihood of the updated parameters        Eq. 31 (+ constant)
//
// Layout and ownership.  Thread `tid` of the CTA owns frames t = tid + k*blockDim,
// k < kSlots.  H (N x T) and U (M x T) live in shared memory for the whole run; every thread
// holds its own copy of L (M x N) in registers and applies the same updates to it; x is
// re-read from global memory (it stays in L2 for the workload sizes this kernel takes).
// The per-frame quantities r_{mt} (see below) stay in registers of the owning thread.
// Phase 2 of source n (the H[n,:] update) and phase 1 of source n+1 run in one pass over
// the frames, so each source costs one CTA barrier; the last phase 2 shares its pass with
// the next iteration's sigma^2 / log-likelihood pass.  The single-mixture launch (the TM
// flag, IP+EM) keeps sigma^2 of every frame in tensor memory: pass A forms it as L H, and
// after each source's update the n-loop changes it by that source's term (never below the
// new term) instead of forming L H again from all N sources.
//
// NMF update in factored form.  With S = L[:,n] H[n,:], G = S / sigma^2 and
// Phi = G^2 U + (1 - G) S, one has Phi = S * r with r = 1 + G (U / sigma^2 - 1).  Hence
//   L[m,n] <- (1/T) sum_t Phi/H[n,t]  = L[m,n] * mean_t r_{mt}
//   H[n,t] <- (1/M) sum_m Phi/L'[m,n] = H[n,t] * (1/M) sum_m r_{mt} / mean_t r_{mt}
// (the same numbers as Algorithm 1 with one reciprocal per (m,t) instead of three).
//
// Piecewise-stationary input (Sec. VI-B, the BL template flag): the "frames" are blocks j of
// B frames and the input is X^_j = (1/B) sum_b x x^H, packed as in xxh_packed (M^2 floats
// per block, built by block_stats_kernel).  The Q pass reads the packed entries instead of
// forming them from x, and U_mj = w_m^H X^_j w_m is the real quadratic form; Algorithms 1
// and 2 are otherwise unchanged.
//
// IP+MM (Algorithm 2, the MM template flag): the same IP and U, then L and H by the
// multiplicative MM updates of IS-NMF with exponent 1/2, all sources at once: one pass over
// the frames accumulates [U (.) (LH)^-2] H^T and (LH)^-1 H^T (in chunks of sources, reduced
// over the CTA) for L; a second pass forms, per frame, sigma^2 from the new L and updates
// every H[n, t].  Two barriers per iteration instead of one per source.
//
// IP in FP64 (Eq. 34-35).  With B = W^{-H} (columns b_m), (W^H Q_m)^{-1} e_m = Q_m^{-1} b_m,
// so Eq. 34 is w = Q_m^{-1} b_m and Eq. 35 divides by sqrt(s), s = b_m^H Q_m^{-1} b_m.  The
// M inverses Q_m^{-1} do not depend on W and are formed in parallel (one warp each); the
// column loop then only needs matrix-vector products.  After w_m changes, B is kept equal to
// W^{-H} by the rank-one update b_k <- b_k - (w_m^H b_k)/(w_m^H b_m) b_m (k != m),
// b_m <- b_m / (w_m^H b_m), where w_m^H b_m = sqrt(s); and |det W|^2 is multiplied by s.
#pragma once
#include "common.cuh"
#include "tmem.cuh"

namespace ffca {

constexpr int kSlots = 8;          // frames per thread
constexpr int kMaxThreads = 256;   // so at most kSlots * 256 = 2048 frames per frequency
constexpr int kMaxWarps = kMaxThreads / 32;
// Register cap: 4 CTAs of 160 threads (T <= 1280) or 2 of 256 fit an SM's 64K registers.
constexpr int kEmMaxRegs = 96;

struct EmArgs {
  const float2* x;      // F x T x M complex64, m fastest
  const float* xh;      // blocks mode: F x T x M^2 packed X^_j (T counts blocks); else null
  double2* P;           // F x M x M complex128, W[a][m] at P[(f*M + a)*M + m]
  float* lam;           // F x M x N, L[m][n]
  float* v;             // F x N x T, H[n][t]
  double* ll_hist;      // F x ll_stride or null: log-likelihood after iteration it
  double* ll_last;      // F or null: log-likelihood of the parameters on exit
  double2* Bst;         // F x M x M: W^{-H} carried between launches (row-major)
  double* detst;        // F x 2: |det W|^2 as (mantissa, exponent)
  int b_valid;          // Bst/detst hold W^{-H} and |det W|^2 of the current P
  int* err;             // status bits (ErrBits)
  int F, T, n_iter, ll_stride;
  int N;                // sources (read by the cluster kernel; the others take N as a template)
  long long* clocks;    // phase timestamps of frequency 0 (only with FFCA_PHASE_CLOCKS)
};

// Phase timestamps (clock64) of frequency 0, thread 0, for the first 8 iterations; compiled
// in only with -DFFCA_PHASE_CLOCKS (profiling builds), otherwise empty.
#ifdef FFCA_PHASE_CLOCKS
#define FFCA_MARK(it, slot)                                                       \
  do {                                                                            \
    if (q.clocks && tid == 0 && (it) < 8) q.clocks[(it) * 16 + (slot)] = clock64(); \
  } while (0)
#else
#define FFCA_MARK(it, slot) \
  do {                      \
  } while (0)
#endif

// Packed Hermitian entries of x x^H: e < M -> diagonal |x_a|^2; then for each pair a < b
// (row-major) two entries: Re(x_a conj x_b), Im(x_a conj x_b).
template <int M>
__device__ __forceinline__ void xxh_packed(const float2 (&xv)[M], float (&e)[M * M]) {
#pragma unroll
  for (int a = 0; a < M; ++a) e[a] = fmaf(xv[a].x, xv[a].x, xv[a].y * xv[a].y);
  int k = M;
#pragma unroll
  for (int a = 0; a < M; ++a) {
#pragma unroll
    for (int b = a + 1; b < M; ++b) {
      e[k] = fmaf(xv[a].x, xv[b].x, xv[a].y * xv[b].y);
      e[k + 1] = fmaf(xv[a].y, xv[b].x, -xv[a].x * xv[b].y);
      k += 2;
    }
  }
}

// Host-visible shared-memory size for a CTA of `threads` threads.
template <int M, int N>
struct EmSmem {
  static constexpr int kQCH = (M <= 3) ? 1 : (M / 2);     // chunks of the Q accumulation
  static constexpr int kMC = M / kQCH;                     // m values per chunk
  static constexpr int kV = kMC * M * M;                   // values reduced per chunk
  static constexpr int kVP = pow2_ceil(kV);
  static_assert(kVP <= 32, "Q chunk must fit one reduction row");
  static constexpr int kRedW = 32;                         // floats per warp per buffer
  // sQ holds the M matrices Q_m; once per launch it is also the scratch of the pivoted
  // inverse of W^H (M*M source + M*2M augmented work).
  static constexpr int kQsz = (M * M * M > 3 * M * M) ? M * M * M : 3 * M * M;
  // sWc holds M*M float2; rounded up to an even count so that sL (read as float4) starts on a
  // 16-byte boundary for every M.
  static constexpr int kWcPad = (M * M + 1) & ~1;
  static size_t bytes(int threads) {
    size_t b = 0;
    b += sizeof(double2) * M * M * 3;        // sW, sB, sWork
    b += sizeof(double2) * kQsz;             // sQ
    b += sizeof(double) * 4;                 // sDet (mantissa, exponent), spare
    b += sizeof(float2) * kWcPad;            // sWc (padded to 16 bytes)
    b += sizeof(float) * ((M * N + 3) & ~3); // sL
    b += sizeof(float) * 2 * kMaxWarps * kRedW;
    b += sizeof(float) * kMaxWarps;          // sLL
    b += sizeof(float) * (size_t)threads * (kSlots * N + 1);   // sH, thread-major
    b += sizeof(float) * (size_t)threads * (kSlots * M + 1);   // sU, thread-major
    return b;
  }
};

// ---------------------------------------------------------------------------------------
// FP64 helpers executed by one warp.

// In-place inverses of the M matrices Q_0..Q_{M-1} (each M x M Hermitian positive definite,
// row-major, consecutive in smem) by Gauss-Jordan without pivoting (the pivots of an HPD
// matrix are its positive Schur complements), all by one warp.  On this part every FP64
// warp instruction occupies the sub-partition's FP64 unit for ~70 cycles whatever its lane
// mask, so the M matrices share the warp's lanes: lane l works on matrix l / kLPM, entries
// (l % kLPM) + q * kLPM.
template <int M>
struct HpdPack {
  static constexpr int kE = M * M;
  static constexpr int kLPM = (32 / M < kE) ? 32 / M : kE;   // lanes per matrix
  static constexpr int kEPL = (kE + kLPM - 1) / kLPM;         // entries per lane
};

template <int M>
__device__ void warp_hpd_inverse_all(double2* Q, int lane, int* err) {
  using PK = HpdPack<M>;
  constexpr int E = PK::kE, LPM = PK::kLPM, EPL = PK::kEPL;
  const int mat = lane / LPM;
  const bool act = mat < M;
  double2* A = Q + (act ? mat : 0) * E;
  const int l0 = lane - mat * LPM;
  for (int k = 0; k < M; ++k) {
    const double d = A[k * M + k].x;
    const float df = (float)d;
    const bool bad = act && !(df > 0.f && df < INFINITY);
    const double rd = rcp_pos_f64(bad ? 1.0 : d);
    double2 nv[EPL];
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      const int e = l0 + q * LPM;
      if (act && e < E) {
        const int i = e / M, j = e - (e / M) * M;
        // new = base - (c1 rd) c2 with base = a_ij (i,j != k) else 0, c1 = a_ik (i != k)
        // else -1, c2 = a_kj (j != k) else 1: covers the four Gauss-Jordan cases at once.
        const double2 aij = A[e], aik = A[i * M + k], akj = A[k * M + j];
        const double2 base = (i != k && j != k) ? aij : make_double2(0.0, 0.0);
        const double2 c1 = (i != k) ? aik : make_double2(-1.0, 0.0);
        const double2 c2 = (j != k) ? akj : make_double2(1.0, 0.0);
        const double2 t = make_double2(c1.x * rd, c1.y * rd);
        nv[q] = make_double2(fma(t.y, c2.y, fma(-t.x, c2.x, base.x)), fma(-t.y, c2.x, fma(-t.x, c2.y, base.y)));
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      const int e = l0 + q * LPM;
      if (act && e < E) A[e] = nv[q];
    }
    __syncwarp();
    if (bad) atomicOr(err, kErrQPivot);
  }
}

// Gauss-Jordan with partial pivoting on the M x (2M) matrix [A | I] (row-major in work,
// A given in `src` row-major): leaves A^{-1} in `dst` (row-major) and returns
// |det A|^2 as mantissa * 2^expo.  One warp; used once per launch.
template <int M>
__device__ void warp_inverse_pivot(const double2* src, double2* work, double2* dst, double& mant,
                                   double& expo, int lane, int* err) {
  constexpr int C = 2 * M;
  for (int e = lane; e < M * C; e += 32) {
    const int i = e / C, j = e - (e / C) * C;
    work[e] = (j < M) ? src[i * M + j] : make_double2((j - M == i) ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  mant = 1.0;
  expo = 0.0;
  for (int k = 0; k < M; ++k) {
    float mag = -1.f;
    int piv = lane;
    if (lane >= k && lane < M) {
      const double2 a = work[lane * C + k];
      mag = (float)(a.x * a.x + a.y * a.y);
      // NaN compares false both ways: ranked as 0 so that the argmax is a total order, every
      // lane agrees on piv and piv stays in [k, M); a NaN pivot is then flagged below.
      if (!(mag >= 0.f)) mag = 0.f;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float om = __shfl_xor_sync(0xffffffffu, mag, off);
      const int op = __shfl_xor_sync(0xffffffffu, piv, off);
      if (om > mag || (om == mag && op < piv)) { mag = om; piv = op; }
    }
    if (piv != k) {
      for (int j = lane; j < C; j += 32) {
        const double2 t = work[k * C + j];
        work[k * C + j] = work[piv * C + j];
        work[piv * C + j] = t;
      }
    }
    __syncwarp();
    const double2 p = work[k * C + k];
    const double pm = p.x * p.x + p.y * p.y;
    if (!(pm > 0.0) || !isfinite(pm)) {
      if (lane == 0) atomicOr(err, kErrWSingular);
    }
    mant *= pm;
    renorm(mant, expo);
    const double rp = rcp_pos_f64(pm > 0.0 ? pm : 1.0);
    const double2 ip = make_double2(p.x * rp, -p.y * rp);     // 1/p
    __syncwarp();
    for (int j = lane; j < C; j += 32) {
      if (j > k) work[k * C + j] = cmul(work[k * C + j], ip);
      else if (j == k) work[k * C + k] = make_double2(1.0, 0.0);
    }
    __syncwarp();
    for (int e = lane; e < M * C; e += 32) {
      const int i = e / C, j = e - (e / C) * C;
      if (i != k && j > k) {
        const double2 f = work[i * C + k];
        work[e] = csub(work[e], cmul(f, work[k * C + j]));
      }
    }
    __syncwarp();
  }
  for (int e = lane; e < M * M; e += 32) {
    const int i = e / M, j = e - (e / M) * M;
    dst[e] = work[i * C + M + j];
  }
  __syncwarp();
}

// The IP column loop (warp 0).  Q holds Q_m^{-1} (row-major per m).  Updates W (sW, row-major
// W[a][m]), B = W^{-H} (sB), the float copy conj(W[a][m]) at sWc[m*M + a], and |det W|^2.
// Every product is split into its real and imaginary part on two lanes: lane
// l = (r * MP + c) * 2 + part, so that each FP64 instruction does 2*M*M lanes of work.
template <int M>
__device__ void ip_columns(const double2* Qi, double2* sW, double2* sB, float2* sWc, double* sDet,
                           int lane, int* err) {
  constexpr int MP = pow2_ceil(M);
  static_assert(2 * MP * MP <= 32 || M > 4, "lane split needs 2 M^2 <= 32");
  const int part = lane & 1;
  const int r = (lane >> 1) / MP, c = (lane >> 1) - ((lane >> 1) / MP) * MP;
  const bool act = r < M && c < M;
  double mant = sDet[0], expo = sDet[1];
  for (int m = 0; m < M; ++m) {
    const double2* Q = Qi + m * M * M;
    // w_raw[r] = sum_c Qinv[r][c] b_m[c]          (lane (r, c, part))
    double pw = 0.0;
    if (act) {
      const double2 q = Q[r * M + c];
      const double2 bb = sB[c * M + m];
      const double x1 = part ? bb.y : bb.x;
      const double x2 = part ? bb.x : -bb.y;
      pw = fma(q.x, x1, q.y * x2);
    }
#pragma unroll
    for (int off = 2; off < 2 * MP; off <<= 1) pw += __shfl_xor_sync(0xffffffffu, pw, off);
    // beta_k = sum_i conj(w_raw[i]) B[i][k]           (lane (k, i, part) with k = r, i = c)
    const double wre = __shfl_sync(0xffffffffu, pw, (c * MP) * 2 + 0);
    const double wim = __shfl_sync(0xffffffffu, pw, (c * MP) * 2 + 1);
    double pb = 0.0;
    if (act) {
      const double2 bk = sB[c * M + r];
      pb = part ? fma(wre, bk.y, -wim * bk.x) : fma(wre, bk.x, wim * bk.y);
    }
#pragma unroll
    for (int off = 2; off < 2 * MP; off <<= 1) pb += __shfl_xor_sync(0xffffffffu, pb, off);
    // s = Re(beta_m) = b_m^H Q_m^{-1} b_m; scale 1/sqrt(s)
    const double s = __shfl_sync(0xffffffffu, pb, (m * MP) * 2 + 0);
    const float sf = (float)s;
    const bool ok = sf > 0.f && sf < INFINITY;
    const double sc = rsqrt_pos_f64(ok ? s : 1.0);
    const double sc2 = sc * sc;
    // B update (lane (i, k, part) with i = r, k = c):
    //   b_k <- b_k - (beta_k / s) b_m  (k != m),   b_m <- b_m / sqrt(s)
    const double bre = __shfl_sync(0xffffffffu, pb, (c * MP) * 2 + 0);
    const double bim = __shfl_sync(0xffffffffu, pb, (c * MP) * 2 + 1);
    double nb = 0.0;
    if (act) {
      const double2 bki = sB[r * M + c];
      const double2 bmi = sB[r * M + m];
      if (c == m) {
        nb = (part ? bmi.y : bmi.x) * sc;
      } else {
        const double cr = bre * sc2, ci = bim * sc2;
        nb = part ? fma(-ci, bmi.x, fma(-cr, bmi.y, bki.y)) : fma(ci, bmi.y, fma(-cr, bmi.x, bki.x));
      }
    }
    // w_m = w_raw / sqrt(s) on lanes (i, 0, part)
    const double wv = pw * sc;
    __syncwarp();
    if (act) reinterpret_cast<double*>(sB)[2 * (r * M + c) + part] = nb;
    if (act && c == 0) {
      reinterpret_cast<double*>(sW)[2 * (r * M + m) + part] = wv;
      reinterpret_cast<float*>(sWc)[2 * (m * M + r) + part] = part ? (float)-wv : (float)wv;
    }
    if (!ok && lane == 0) atomicOr(err, kErrIpNorm);
    mant *= ok ? s : 1.0;
    renorm(mant, expo);
    __syncwarp();
  }
  if (lane == 0) { sDet[0] = mant; sDet[1] = expo; }
  __syncwarp();
}

// Sum over the warps of a CTA of the per-warp rows red[w][0..MP) written before the barrier;
// every lane of every warp returns the same M totals (same order everywhere).
template <int M, int MP>
__device__ __forceinline__ void cta_rows_sum(const float* red, int nw, int lane, float (&tot)[M]) {
  // lane l = w*MP + m reads warp w's value m; butterfly over the warp index bits
  const int w = lane / MP, m = lane - (lane / MP) * MP;
  float v = (w < nw && m < M) ? red[w * 32 + m] : 0.f;
#pragma unroll
  for (int off = MP; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
#pragma unroll
  for (int i = 0; i < M; ++i) tot[i] = __shfl_sync(0xffffffffu, v, i);
}

// One frequency of one mixture: everything em_frequency needs, as per-frequency pointers.
struct EmItem {
  const float2* x;      // T x M
  const float* xh;      // blocks mode: T x M^2 packed X^_j; else null
  double2* P;           // M x M (W[a][m] at a*M + m)
  float* lam;           // M x N
  float* v;             // N rows of T frames
  double2* Bst;         // M x M, W^{-H} carried between launches
  double* detst;        // 2: |det W|^2 as (mantissa, exponent)
  double* ll_hist;      // n_iter entries or null
  double* ll_last;      // 1 entry or null
  long long* clocks;    // phase timestamps (profiling builds) or null
  int* valid_flag;      // if set: 1 when Bst/detst are current (read at start, set at end)
  unsigned long long* stamp;   // if set: start and end %globaltimer of this item
  int T, n_iter, b_valid;
};

// The whole IP+EM run of one frequency by one CTA (see the file comment).  `smem_raw` is the
// CTA's dynamic shared memory (EmSmem<M, N>::bytes(blockDim.x)); T <= blockDim.x * kSlots.
// TM (IP+EM only): sigma^2 of every frame kept in tensor memory, 4 columns per frame slot
// (32 columns per four warps), and updated by each source's change in the n-loop instead of
// recomputed as L H from all sources; pass A still forms it from L H once per iteration.
// tmem_slot: one 32-bit word of shared memory for the allocation's address.
template <int M, int N, bool MM = false, bool BL = false, bool TM = false>
__device__ __forceinline__ void em_frequency(const EmItem& q, int* err, unsigned char* smem_raw,
                                             uint32_t* tmem_slot = nullptr) {
  using SM = EmSmem<M, N>;
  constexpr int QCH = SM::kQCH, MC = SM::kMC, V = SM::kV, VP = SM::kVP;
  constexpr int MP = pow2_ceil(M);
  constexpr int NE = M * M;                   // packed Hermitian entries per Q_m
  static_assert(MP * (kMaxWarps) <= 32, "n-step reduction rows must fit one warp");

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bd = blockDim.x, nw = bd >> 5;
  const int T = q.T;
  const int Tp = bd * kSlots;

  double2* sW = reinterpret_cast<double2*>(smem_raw);
  double2* sB = sW + M * M;
  double2* sWork = sB + M * M;
  double2* sQ = sWork + M * M;
  double* sDet = reinterpret_cast<double*>(sQ + SM::kQsz);
  float2* sWc = reinterpret_cast<float2*>(sDet + 4);
  float* sL = reinterpret_cast<float*>(sWc + SM::kWcPad);
  float* sRed = sL + ((M * N + 3) & ~3);
  float* sLL = sRed + 2 * kMaxWarps * SM::kRedW;
  float* sH = sLL + kMaxWarps;
  // H and U are stored thread-major: thread tid's frames (slot k) at sH[tid*SH + k*N + n]
  // and sU[tid*SU + k*M + m].  The odd strides SH, SU keep a warp's accesses on distinct
  // banks, and every access in the passes is a compile-time offset from one base pointer.
  constexpr int SH = kSlots * N + 1, SU = kSlots * M + 1;
  float* sU = sH + bd * SH;
  float* pH = sH + tid * SH;
  float* pU = sU + tid * SU;

  const float2* xf = q.x;
  const float* xhf = q.xh;
  const double invT = 1.0 / (double)T;
  const float invTf = 1.0f / (float)T;

  // ---- tensor memory for sigma^2 (TM): warp 0 allocates; warps w and w + 4 share a lane
  // quarter and take column groups 0 and 1; slot k of a thread at columns 4k of its group
  static_assert(!TM || (!MM && M <= 4), "sigma^2 in tensor memory: IP+EM, M <= 4");
  const unsigned tm_cols = nw > 4 ? 64u : 32u;
  uint32_t tm_base = 0;
  if constexpr (TM) {
    if (warp == 0) tmem_alloc(tmem_slot, tm_cols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    tm_base = *tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
  }

  // ---- load the parameters of frequency f
  for (int i = tid; i < M * N; i += bd) sL[i] = q.lam[i];
  for (int i = tid; i < M * M; i += bd) sW[i] = q.P[i];
  for (int n = 0; n < N; ++n) {
    const float* vf = q.v + (size_t)n * T;
    for (int t = tid; t < Tp; t += bd) {
      const int owner = t % bd, k = t / bd;
      sH[owner * SH + k * N + n] = (t < T) ? vf[t] : 1.0f;
    }
  }
  __syncthreads();
  // ---- B = W^{-H}, |det W|^2: carried over from the previous launch when valid, else
  // formed once by pivoted Gauss-Jordan on W^H (warp 0)
  const int b_valid = q.valid_flag ? *reinterpret_cast<volatile int*>(q.valid_flag) : q.b_valid;
  if (warp == 0) {
    if (b_valid) {
      for (int e = lane; e < M * M; e += 32) sB[e] = q.Bst[e];
      if (lane == 0) { sDet[0] = q.detst[0]; sDet[1] = q.detst[1]; }
    } else {
      for (int e = lane; e < M * M; e += 32) {
        const int i = e / M, j = e - (e / M) * M;
        const double2 w = sW[j * M + i];
        sQ[e] = make_double2(w.x, -w.y);
      }
      __syncwarp();
      double mant, expo;
      warp_inverse_pivot<M>(sQ, sQ + M * M, sB, mant, expo, lane, err);
      if (lane == 0) { sDet[0] = mant; sDet[1] = expo; }
    }
    for (int e = lane; e < M * M; e += 32) {
      const int a = e / M, m = e - (e / M) * M;
      const double2 w = sW[a * M + m];
      sWc[m * M + a] = make_float2((float)w.x, (float)-w.y);
    }
  }
  __syncthreads();

  // L (M x N) lives in shared memory and every thread reads it into registers at the start
  // of each pass.  After a source's reduction every thread stores the same new column
  // (identical values), so each thread's later reads see the new column through its own
  // store, without another barrier.
  auto load_L = [&](float (&Lr)[M][N]) {
    constexpr int Q4 = (M * N) / 4;
    float tmp[M * N];
    const float4* s4 = reinterpret_cast<const float4*>(sL);
#pragma unroll
    for (int i = 0; i < Q4; ++i) {
      const float4 v4 = s4[i];
      tmp[4 * i] = v4.x; tmp[4 * i + 1] = v4.y; tmp[4 * i + 2] = v4.z; tmp[4 * i + 3] = v4.w;
    }
#pragma unroll
    for (int i = 4 * Q4; i < M * N; ++i) tmp[i] = sL[i];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int n = 0; n < N; ++n) Lr[m][n] = tmp[m * N + n];
  };

  // per-slot registers: r[k][m] holds 1/sigma^2 during the Q pass and r_{mt} in the sweep
  float r[kSlots][M];
  int par = 0;

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

  // packed X^_j of block t (blocks mode)
  auto load_xh = [&](int t, float (&e)[NE]) {
    const float* src = xhf + (size_t)t * NE;
    if constexpr (NE % 4 == 0) {
#pragma unroll
      for (int i = 0; i < NE; i += 4) {
        const float4 q4 = __ldg(reinterpret_cast<const float4*>(src + i));
        e[i] = q4.x; e[i + 1] = q4.y; e[i + 2] = q4.z; e[i + 3] = q4.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < NE; ++i) e[i] = __ldg(src + i);
    }
  };

  // U = |W^H x|^2 for the current W (blocks: U = w^H X^ w = sum_a |w_a|^2 X_aa
  // + 2 sum_{a<b} Re(conj(w_a) w_b X_ab), with conj(w_a) = wc[a])
  auto pass_U = [&]() {
    if constexpr (BL) {
      float2 wc[M * M];
#pragma unroll
      for (int i = 0; i < M * M; ++i) wc[i] = sWc[i];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const int t = tid + k * bd;
        if (t < T) {
          float e[NE];
          load_xh(t, e);
#pragma unroll
          for (int m = 0; m < M; ++m) {
            float u = 0.f;
#pragma unroll
            for (int a = 0; a < M; ++a) u = fmaf(fmaf(wc[m * M + a].x, wc[m * M + a].x, wc[m * M + a].y * wc[m * M + a].y), e[a], u);
            int idx = M;
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
              for (int b = a + 1; b < M; ++b) {
                const float2 wa = wc[m * M + a], wb = wc[m * M + b];
                const float pr = fmaf(wa.x, wb.x, wa.y * wb.y);       // wa conj(wb)
                const float pi = fmaf(wa.y, wb.x, -wa.x * wb.y);
                u = fmaf(2.f, fmaf(pr, e[idx], -pi * e[idx + 1]), u);
                idx += 2;
              }
            pU[k * M + m] = u;
          }
        }
      }
    } else {
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
    }
  };

  auto ll_from_sum = [&](double s) {
    const double logdet = (double)__logf((float)sDet[0]) + sDet[1] * kLn2;
    return (double)T * logdet - s - (double)M * (double)T * kLnPi;
  };

  float coef[M];
#pragma unroll
  for (int m = 0; m < M; ++m) coef[m] = 0.f;

  if (q.n_iter == 0) pass_U();

  // The loop body is written once (n and the Q chunks are runtime loops) so that the
  // kernel's code stays small enough for the instruction cache; register arrays are indexed
  // with compile-time indices only, through selects.
#pragma unroll 1
  for (int it = 0;; ++it) {
    const bool have_ll = (it > 0) || (q.n_iter == 0);
    const bool do_iter = it < q.n_iter;
    FFCA_MARK(it, 0);

    // ---- pass A: the pending H[N-1,:] update of the last sweep (it > 0), then
    // sigma^2 = LH, 1/sigma^2 -> r, and the log-likelihood terms of the current parameters
    {
      float Lr[M][N];
      load_L(Lr);
      float llp = 0.f;
      bool bad = false;
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const int t = tid + k * bd;
        float s2v[4] = {1.f, 1.f, 1.f, 1.f};
        if (t < T) {
          if (!MM && it > 0) {
            float g = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) g = fmaf(r[k][m], coef[m], g);
            pH[k * N + N - 1] *= g;
          }
          float h[N];
#pragma unroll
          for (int n = 0; n < N; ++n) h[n] = pH[k * N + n];
#pragma unroll
          for (int m = 0; m < M; ++m) {
            float s2 = 0.f;
#pragma unroll
            for (int n = 0; n < N; ++n) s2 = fmaf(Lr[m][n], h[n], s2);
            bad |= !(s2 > 0.f && s2 < INFINITY);
            const float rs = fast_rcp(s2);
            r[k][m] = rs;
            if constexpr (TM) s2v[m] = s2;
            if (have_ll) llp += fmaf(pU[k * M + m], rs, __logf(s2));
          }
        }
        if constexpr (TM) {
          if (k * bd < T) tmem_st4(tm_base + 4 * k, s2v);         // uniform over the CTA
        }
      }
      if constexpr (TM) tmem_wait_st();
      if (bad) atomicOr(err, kErrSigma);
      if (have_ll) {
        llp = warp_sum(llp);
        if (lane == 0) sLL[warp] = llp;
      }
    }
    if (!do_iter) {
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += (double)sLL[w];
        const double ll = ll_from_sum(s);
        if (it > 0 && q.ll_hist) q.ll_hist[it - 1] = ll;
        if (q.ll_last) q.ll_last[0] = ll;
      }
      break;
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
          float e[NE];
          if constexpr (BL) {
            load_xh(t, e);
          } else {
            float2 xv[M];
            load_x(t, xv);
            xxh_packed<M>(xv, e);
          }
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
        float* red = sRed + par * kMaxWarps * SM::kRedW + warp * SM::kRedW;
        if (VP >= 32) {
#pragma unroll
          for (int i = 0; i < VP / 32; ++i) red[lane * (VP / 32) + i] = acc[i];
        } else if ((lane * VP) % 32 == 0) {
          red[(lane * VP) / 32] = acc[0];
        }
      }
      __syncthreads();
      if (tid < V) {
        const float* red = sRed + par * kMaxWarps * SM::kRedW;
        float q = 0.f;
        for (int w = 0; w < nw; ++w) q += red[w * SM::kRedW + tid];
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
      if (c == 0 && have_ll && tid == 32 % bd) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += (double)sLL[w];
        if (q.ll_hist) q.ll_hist[it - 1] = ll_from_sum(s);
      }
      par ^= 1;
    }
    __syncthreads();
    FFCA_MARK(it, 1);

    // ---- IP (FP64): Q_m^{-1} for all m packed on warp 0's lanes, then the column loop.
    // (One matrix per warp shortens the chain but issues ~2.5x the FP64 warp instructions,
    // which the other CTAs on the SM then wait for: measured slower.)
    if (warp == 0) warp_hpd_inverse_all<M>(sQ, lane, err);
    __syncwarp();
    FFCA_MARK(it, 2);
    if (warp == 0) ip_columns<M>(sQ, sW, sB, sWc, sDet, lane, err);
    __syncthreads();
    FFCA_MARK(it, 3);

    // ---- U = |W^H x|^2 (Eq. 37)
    pass_U();
    FFCA_MARK(it, 4);

    if constexpr (MM) {
      // ---- Algorithm 2: L <- L (.) {[U (.) (LH)^-2] H^T / (LH)^-1 H^T}^1/2, sources in chunks
      // of NC; r[k][m] still holds 1/sigma^2 of pass A (L and H are unchanged since)
      constexpr int NC = (N < 16 / M) ? N : 16 / M;            // 2 M NC <= 32 values per chunk
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
                const int n = n0 + nc < N ? n0 + nc : N - 1;   // a partial last chunk repeats a source; its sums are not used
                const float h = pH[k * N + n];
                acc[m * NC + nc] = fmaf(a, h, acc[m * NC + nc]);
                acc[M * NC + m * NC + nc] = fmaf(rs, h, acc[M * NC + m * NC + nc]);
              }
            }
          }
        }
        warp_reduce_scatter<VLP>(acc, lane);
        {
          float* red = sRed + par * kMaxWarps * SM::kRedW + warp * SM::kRedW;
          if ((lane * VLP) % 32 == 0) red[(lane * VLP) / 32] = acc[0];
        }
        __syncthreads();
        if (tid < M * NC) {
          const int m = tid / NC, nc = tid - (tid / NC) * NC;
          if (n0 + nc < N) {
            const float* red = sRed + par * kMaxWarps * SM::kRedW;
            float num = 0.f, den = 0.f;
            for (int w = 0; w < nw; ++w) {
              num += red[w * SM::kRedW + m * NC + nc];
              den += red[w * SM::kRedW + M * NC + m * NC + nc];
            }
            // a source whose H row has underflowed to zero in FP32 gives 0/0 here; L[:, n] then
            // has no effect on the model and is left as it is
            sL[m * N + n0 + nc] *= (den > 0.f) ? sqrtf(num / den) : 1.0f;
          }
        }
        par ^= 1;
      }
      __syncthreads();
      // ---- H <- H (.) {L^T [U (.) (LH)^-2] / L^T (LH)^-1}^1/2 with sigma^2 from the new L
      {
        float Lr[M][N];
        load_L(Lr);
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
          const int t = tid + k * bd;
          if (t < T) {
            float h[N];
#pragma unroll
            for (int n = 0; n < N; ++n) h[n] = pH[k * N + n];
            float a[M], b[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
              float s2 = 0.f;
#pragma unroll
              for (int n = 0; n < N; ++n) s2 = fmaf(Lr[m][n], h[n], s2);
              const float rs = fast_rcp(s2);
              b[m] = rs;
              a[m] = pU[k * M + m] * rs * rs;
            }
#pragma unroll
            for (int n = 0; n < N; ++n) {
              float num = 0.f, den = 0.f;
#pragma unroll
              for (int m = 0; m < M; ++m) {
                num = fmaf(Lr[m][n], a[m], num);
                den = fmaf(Lr[m][n], b[m], den);
              }
              pH[k * N + n] = (den > 0.f) ? h[n] * sqrtf(num * fast_rcp(den)) : h[n];
            }
          }
        }
      }
      __syncthreads();           // the next pass A reads L and the new H
    } else {
      // ---- NMF EM sweep over sources (Algorithm 1 n-loop, Gauss-Seidel).  Pass n applies
      // the H[n-1,:] update of the previous source, then forms r for source n.
      // L[:, n-1] before and after its update (TM: the change of sigma^2 it makes)
      float Lold[M], Lnew[M];
#pragma unroll
      for (int m = 0; m < M; ++m) Lold[m] = Lnew[m] = 0.f;
#pragma unroll 1
      for (int n = 0; n < N; ++n) {
        float* pHn = pH + n;                   // this thread's H[n, .] (slot k at k*N)
        float Lr[M][N];
        if constexpr (!TM) load_L(Lr);
        float Ln[M];
#pragma unroll
        for (int m = 0; m < M; ++m) Ln[m] = sL[m * N + n];
        float acc[MP];
#pragma unroll
        for (int m = 0; m < MP; ++m) acc[m] = 0.f;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
          const int t = tid + k * bd;
          float s2v[4] = {1.f, 1.f, 1.f, 1.f};
          if constexpr (TM) {
            if (k * bd < T) tmem_ld4(tm_base + 4 * k, s2v);       // uniform over the CTA
          }
          if (t < T) {
            if (n > 0) {
              float g = 0.f;
#pragma unroll
              for (int m = 0; m < M; ++m) g = fmaf(r[k][m], coef[m], g);
              const float hold = pHn[k * N - 1];
              const float hnew = hold * g;
              pHn[k * N - 1] = hnew;
              if constexpr (TM) {
#pragma unroll
                for (int m = 0; m < M; ++m) {
                  // sigma^2 <- sigma^2 - L H + L' H', never below the new term: the rest of
                  // the sum, clamped at zero, plus the new term in one fma
                  const float rest = fmaxf(fmaf(-Lold[m], hold, s2v[m]), 0.f);
                  s2v[m] = fmaf(Lnew[m], hnew, rest);
                }
              }
            }
            const float hn = pHn[k * N];
            float h[N];
            if constexpr (!TM) {
#pragma unroll
              for (int n2 = 0; n2 < N; ++n2) h[n2] = pH[k * N + n2];
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
              float s2 = 0.f;
              if constexpr (TM) {
                s2 = s2v[m];
              } else {
#pragma unroll
                for (int n2 = 0; n2 < N; ++n2) s2 = fmaf(Lr[m][n2], h[n2], s2);
              }
              const float rs = fast_rcp(s2);
              const float G = Ln[m] * hn * rs;
              const float rr = fmaf(G, fmaf(pU[k * M + m], rs, -1.f), 1.f);
              r[k][m] = rr;
              acc[m] += rr;
            }
          }
          if constexpr (TM) {
            if (n > 0 && k * bd < T) tmem_st4(tm_base + 4 * k, s2v);
          }
        }
        if constexpr (TM) tmem_wait_st();
        warp_reduce_scatter<MP>(acc, lane);
        {
          float* red = sRed + par * kMaxWarps * SM::kRedW + warp * SM::kRedW;
          if ((lane * MP) % 32 == 0) red[(lane * MP) / 32] = acc[0];
        }
        __syncthreads();
        float tot[M];
        cta_rows_sum<M, MP>(sRed + par * kMaxWarps * SM::kRedW, nw, lane, tot);
        par ^= 1;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float mean = tot[m] * invTf;
          sL[m * N + n] = Ln[m] * mean;       // same value from every thread
          coef[m] = fast_rcp(mean) * (1.0f / (float)M);
          Lold[m] = Ln[m];
          Lnew[m] = Ln[m] * mean;
        }
        FFCA_MARK(it, 5 + (n < 9 ? n : 9));
      }
    }
    FFCA_MARK(it, 15);
  }

  // ---- write back
  __syncthreads();
  for (int i = tid; i < M * N; i += bd) q.lam[i] = sL[i];
  for (int i = tid; i < M * M; i += bd) {
    q.P[i] = sW[i];
    q.Bst[i] = sB[i];
  }
  if (tid == 0) {
    q.detst[0] = sDet[0];
    q.detst[1] = sDet[1];
    if (q.valid_flag) *q.valid_flag = 1;
  }
  for (int n = 0; n < N; ++n) {
    float* vf = q.v + (size_t)n * T;
    for (int t = tid; t < T; t += bd) vf[t] = sH[(t % bd) * SH + (t / bd) * N + n];
  }
  // ---- release the tensor memory once every thread's accesses are complete
  if constexpr (TM) {
    tmem_wait_st();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc(*tmem_slot, tm_cols);
  }
}


template <int M, int N, bool MM = false, bool BL = false, bool TM = false>
__global__ void __maxnreg__(kEmMaxRegs) fastfca_em_kernel(EmArgs p) {
  const int f = blockIdx.x;
  if (f >= p.F) return;
  if (blockDim.x * kSlots < (unsigned)p.T || blockDim.x > (unsigned)kMaxThreads) {   // uniform
    if (threadIdx.x == 0) atomicOr(p.err, kErrConfig);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EmItem q;
  q.x = p.x + (size_t)f * p.T * M;
  q.xh = BL ? p.xh + (size_t)f * p.T * M * M : nullptr;
  q.P = p.P + (size_t)f * M * M;
  q.lam = p.lam + (size_t)f * M * N;
  q.v = p.v + (size_t)f * N * p.T;
  q.Bst = p.Bst + (size_t)f * M * M;
  q.detst = p.detst + 2 * (size_t)f;
  q.ll_hist = p.ll_hist ? p.ll_hist + (size_t)f * p.ll_stride : nullptr;
  q.ll_last = p.ll_last ? p.ll_last + f : nullptr;
  q.clocks = (p.clocks && f == 0) ? p.clocks : nullptr;
  q.valid_flag = nullptr;
  q.stamp = nullptr;
  q.T = p.T;
  q.n_iter = p.n_iter;
  q.b_valid = p.b_valid;
  __shared__ uint32_t tmem_slot;
  em_frequency<M, N, MM, BL, TM>(q, p.err, smem_raw, &tmem_slot);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Persistent form for batches of mixtures: each CTA takes items (one frequency of one mixture
// each, all of this kernel's (M, N) and algorithm: IP+EM, or IP+MM with MM) from an atomic counter, in the order they are listed
// (the host lists them longest-first), until the list is exhausted.  blockDim.x * kSlots must
// cover every item's T.  No CTA waits on another.
template <int M, int N, bool MM = false>
__global__ void __maxnreg__(kEmMaxRegs) fastfca_em_persistent_kernel(const EmItem* __restrict__ items,
                                                                    int n_items, int n_iter,
                                                                    int* counter, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  for (;;) {
    __syncthreads();                               // previous item's smem reads are done
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int i = s_next;
    if (i >= n_items) return;
    EmItem q = items[i];
    q.n_iter = n_iter;
    if (blockDim.x * kSlots < (unsigned)q.T) {    // uniform over the CTA
      if (threadIdx.x == 0) atomicOr(err, kErrConfig);
      continue;
    }
    const unsigned long long t0 = global_ns();
    em_frequency<M, N, MM>(q, err, smem_raw);
    __syncthreads();
    if (threadIdx.x == 0 && q.stamp) {
      q.stamp[0] = t0;
      q.stamp[1] = global_ns();
    }
  }
}

// X^_j = (1/B) sum_b x x^H of the blocks j of B consecutive frames (Sec. VI-B), packed as in
// xxh_packed; one thread per (frequency, block).  x: F x (J B) x M; xh: F x J x M^2.
template <int M>
__global__ void block_stats_kernel(const float2* __restrict__ x, float* __restrict__ xh, int F, int J, int B) {
  constexpr int NE = M * M;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)F * J) return;
  const size_t f = i / J, j = i - (i / J) * J;
  const float2* src = x + (f * J * B + j * B) * M;
  float acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e] = 0.f;
  for (int b = 0; b < B; ++b) {
    float2 xv[M];
#pragma unroll
    for (int a = 0; a < M; ++a) xv[a] = src[(size_t)b * M + a];
    float e[NE];
    xxh_packed<M>(xv, e);
#pragma unroll
    for (int q = 0; q < NE; ++q) acc[q] += e[q];
  }
  const float invB = 1.0f / (float)B;
#pragma unroll
  for (int q = 0; q < NE; ++q) xh[i * NE + q] = acc[q] * invB;
}

}  // namespace ffca

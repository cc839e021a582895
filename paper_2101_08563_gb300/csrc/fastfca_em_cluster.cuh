// FastFCA IP+EM (Algorithm 1) for large bins: one thread-block cluster owns one frequency.
//
// The frequency-resident kernel (fastfca_em.cuh) keeps a frequency's per-frame state in one
// CTA and its per-frame ratios in registers; that stops at M = 4, N = 8, T = 2048.  Here the
// T frames of a frequency are split over the C CTAs of a cluster (C in {1, 2, 4, 8}, CTA rank
// c owns frames [c Tc, min((c+1) Tc, T)), Tc = ceil(T / C)), and every per-frame array lives
// in that CTA's shared memory: H (N x Tc), U = |W^H x|^2, sigma^2 and r (M x Tc each).  M is a
// template parameter (M <= 8); N is a runtime parameter (N <= 16).  The steps and their
// order are those of the frequency-resident kernel (see its file comment for the equations):
//
//   pass A   pending H[N-1,:] update, sigma^2 = L H, 1/sigma^2, log-likelihood terms
//   Q pass   Q_m = (1/T) sum_t x x^H / sigma^2_m  (Eq. 33): lanes own Hermitian entries,
//            warps own frames, so no warp reduction is needed
//   IP       Q_m^{-1} (HPD Gauss-Jordan, FP64), the CTAs of the cluster splitting the M
//            matrices; then the column loop of Eq. 34-35 on B = W^{-H} by four warps (FP64)
//   U pass   U = |W^H x|^2 (Eq. 37)
//   n-loop   for each source: r = 1 + G (U / sigma^2 - 1), L[:,n] *= mean_t r, then
//            H[n,:] *= (1/M) sum_m r / mean_t r in the next pass (Gauss-Seidel), with sigma^2
//            updated by the change of that source's term: sigma^2_m += L'H' - LH
//   (BL)     piecewise-stationary input (Sec. VI-B, the BL template flag): the "frames" are
//            blocks j with packed X^_j (M^2 floats each, as block_stats_kernel writes them);
//            the Q pass reads them instead of forming x x^H, and U = w_m^H X^_j w_m
//   (MN)     FastMNMF's per-frequency step (App. C, the MN template flag): H holds the given
//            h = t v; one iteration of Q, IP, U and lambda's MM update (the L line below),
//            then U and a = sum_m lambda U / sigma^4, b = sum_m lambda / sigma^2 (new lambda)
//            are written for the kernels that update the bases and activations; the
//            log-likelihood is that of the incoming parameters
//   (MM)     IP+MM (Algorithm 2, the MM template flag) replaces the n-loop: one pass forms
//            sum_t U sigma^-4 H_n and sum_t sigma^-2 H_n for every (m, n), one cluster
//            exchange sums them and every CTA updates all of L; then each frame's H column
//            is updated with sigma^2 from the new L.  One cluster barrier for all sources.
//
// Every reduction over t (Q, log-likelihood, the n-loop means) is summed per warp, then per
// CTA in warp order, then over the cluster in rank order through distributed shared memory,
// so all CTAs of a cluster hold bit-identical W, B, L and agree on every decision.  Exchange
// buffers are double-buffered, so one cluster barrier per reduction suffices (a buffer is
// rewritten only after every CTA has passed the following barrier, i.e. finished reading).
#pragma once
#include "fastfca_em.cuh"

namespace ffca {

constexpr int kCThreads = 256;               // threads per CTA
constexpr int kCWarps = kCThreads / 32;
constexpr int kCMaxN = 16;                   // sources
constexpr int kCMaxCluster = 8;              // portable cluster size
constexpr int kCIpThreads = 128;             // the four FP64 warps of the IP (one per SMSP)

// ------------------------------------------------------------------ cluster primitives
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned dyn_smem_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// Barrier over every thread of every CTA of the cluster; release/acquire order the shared
// memory accesses (local and distributed) made before it against those made after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of `p` (this CTA's shared memory) in the shared memory of CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, unsigned rank) {
  const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  return remote;
}

__device__ __forceinline__ double ld_dsmem_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ float ld_dsmem_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ double2 ld_dsmem_f64x2(uint32_t addr) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr) : "memory");
  return v;
}

// mbarrier + st.async: a CTA pushes values into a peer's shared memory and the peer's
// transaction barrier counts the bytes; the peer waits on its own barrier only.
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(m)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(m)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"((uint32_t)__cvta_generic_to_shared(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The non-blocking form: true if the phase of this parity has completed, at once.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* m, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"((uint32_t)__cvta_generic_to_shared(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void st_async_f32(uint32_t remote_addr, float v, uint32_t remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(remote_addr),
               "r"(__float_as_uint(v)), "r"(remote_mbar)
               : "memory");
}

// Status bit: a cluster exchange waited longer than its limit (the kernel continues; the
// host reports the launch as failed).  kMbarSpinLimit is the default limit; a launch may pass
// a smaller one (ClusterArgs::wait_limit) to make the time-out path run in a test.
constexpr int kErrClusterWait = 64;
constexpr int kMbarSpinLimit = 1 << 20;

// Barrier of the four IP warps (threads 0..127) only.
__device__ __forceinline__ void ip_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// ------------------------------------------------------------------ shared-memory layout
template <int M>
struct ClusterSmem {
  static constexpr int NE = M * M;                        // packed Hermitian entries of Q_m
  static constexpr int V = M * NE;                        // reals of all Q_m
  static constexpr int kXV0 = (V > kCWarps * 8 ? V : kCWarps * 8);
  static constexpr int kXV = (kXV0 > 2 * M * kCMaxN ? kXV0 : 2 * M * kCMaxN) + 4;   // float exchange row
  static constexpr int kQsz = (M * M * M > 3 * M * M) ? M * M * M : 3 * M * M;
  static constexpr int kWcPad = (M * M + 1) & ~1;
  // byte offsets (all multiples of 16)
  static constexpr size_t oW = 0;                                         // double2 M*M
  static constexpr size_t oB = oW + 16 * M * M;                           // double2 M*M
  static constexpr size_t oQ = oB + 16 * M * M;                           // double2 kQsz
  static constexpr size_t oV = oQ + 16 * (size_t)kQsz;                    // double2 8 (w_raw)
  static constexpr size_t oBeta = oV + 16 * 8;                            // double2 8
  static constexpr size_t oDet = oBeta + 16 * 8;                          // double 4
  static constexpr size_t oXll = oDet + 32;                               // double 2 (log-lik)
  static constexpr size_t oX = oXll + 16;                                 // float 2 x kXV
  static constexpr size_t oWc = oX + ((4 * 2 * (size_t)kXV + 15) & ~(size_t)15);   // float2 kWcPad
  static constexpr size_t oL = oWc + 8 * (size_t)kWcPad;                  // float M*kCMaxN
  static constexpr size_t oRed = oL + 4 * (size_t)M * kCMaxN;             // float kCWarps*8
  static constexpr size_t oLL = oRed + 4 * kCWarps * 8;                   // float kCWarps
  static constexpr size_t oQw = oLL + 4 * kCWarps;                        // float kCWarps*V
  static constexpr size_t oPush = oQw + 4 * (size_t)kCWarps * V;         // float 2 x C x kCWarps x 8
  static constexpr size_t oMbar = oPush + 4 * 2 * kCMaxCluster * kCWarps * 8;   // uint64 2
  static constexpr size_t oFrames = oMbar + 16;                           // per-frame arrays
  // per-frame arrays, each row padded to Tcp = Tc rounded up to 4 floats
  __host__ __device__ static int tcp(int Tc) { return (Tc + 3) & ~3; }
  __host__ __device__ static size_t bytes(int N, int Tc) { return oFrames + 4 * (size_t)tcp(Tc) * (N + 3 * M); }
};

// ------------------------------------------------------------------ FP64 pieces of the IP
// In-place inverses of the Q_m (HPD, row-major, M*M each, at Q + m*M*M) for the m with
// m % C == crank, by the four IP warps.  Entry i of the owned entries goes to warp i % 4,
// lane (i / 4) % 32, slot i / 128: the four warps sit on the four sub-partitions, and an FP64
// warp instruction costs the same whatever its lane count, so spreading the entries over the
// warps shortens each step.  Gauss-Jordan without pivoting (the pivots of an HPD matrix are
// positive Schur complements); a non-positive pivot sets kErrQPivot.
template <int M>
__device__ void cluster_hpd_inverses(double2* Q, int crank, int C, int tid, int* err) {
  constexpr int E = M * M;
  constexpr int kMaxSlots = (M * E + kCIpThreads - 1) / kCIpThreads;   // all M matrices when C = 1
  const int owned = (crank < M) ? (M - 1 - crank) / C + 1 : 0;
  const int total = owned * E;
  const int me = (tid & 31) * 4 + (tid >> 5);        // this thread's entry within a slot
  for (int k = 0; k < M; ++k) {
    double2 nv[kMaxSlots];
    bool bad = false;
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      const int i = me + s * kCIpThreads;
      if (i < total) {
        const int mo = i / E, e = i - mo * E;
        double2* A = Q + (crank + mo * C) * E;
        const int r = e / M, cc = e - r * M;
        const double d = A[k * M + k].x;
        const float df = (float)d;
        bad |= !(df > 0.f && df < INFINITY);
        const double rd = rcp_pos_f64((df > 0.f && df < INFINITY) ? d : 1.0);
        const double2 aij = A[e], aik = A[r * M + k], akj = A[k * M + cc];
        const double2 base = (r != k && cc != k) ? aij : make_double2(0.0, 0.0);
        const double2 c1 = (r != k) ? aik : make_double2(-1.0, 0.0);
        const double2 c2 = (cc != k) ? akj : make_double2(1.0, 0.0);
        const double2 t = make_double2(c1.x * rd, c1.y * rd);
        nv[s] = make_double2(fma(t.y, c2.y, fma(-t.x, c2.x, base.x)), fma(-t.y, c2.x, fma(-t.x, c2.y, base.y)));
      }
    }
    ip_bar();
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      const int i = me + s * kCIpThreads;
      if (i < total) {
        const int mo = i / E, e = i - mo * E;
        Q[(crank + mo * C) * E + e] = nv[s];
      }
    }
    ip_bar();
    if (bad) atomicOr(err, kErrQPivot);
  }
}

// The IP column loop (Eq. 34-35) by the four IP warps, for any M <= 8.  Qi holds Q_m^{-1}.
// Thread (w, lane) with lane = (rl * 8 + c) * 2 + part covers row r = 2 w + rl, column c,
// real (part 0) or imaginary (part 1) part; sums over c are xor-shuffles over lane bits 1-3.
// Per column m:  w_raw = Q_m^{-1} b_m;  beta = w_raw^H B;  s = Re beta_m;  w_m = w_raw/sqrt(s);
// b_k -= (beta_k / s) b_m (k != m), b_m /= sqrt(s);  |det W|^2 *= s.  Updates sW, sB, sWc
// and sDet; all four warps leave with the results visible to each other.
template <int M>
__device__ void cluster_ip_columns(const double2* Qi, double2* sW, double2* sB, float2* sWc, double* sDet,
                                   double2* sV, double2* sBeta, int tid, int* err) {
  const int w = tid >> 5, lane = tid & 31;
  const int part = lane & 1, c = (lane >> 1) & 7, rl = lane >> 4;
  const int r = 2 * w + rl;
  const bool act = r < M && c < M;
  double mant = sDet[0], expo = sDet[1];
  for (int m = 0; m < M; ++m) {
    const double2* Q = Qi + m * M * M;
    // w_raw[r] = sum_c Qinv[r][c] b_m[c]
    double pw = 0.0;
    if (act) {
      const double2 q = Q[r * M + c];
      const double2 bb = sB[c * M + m];
      pw = fma(q.x, part ? bb.y : bb.x, q.y * (part ? bb.x : -bb.y));
    }
#pragma unroll
    for (int off = 2; off <= 8; off <<= 1) pw += __shfl_xor_sync(0xffffffffu, pw, off);
    if (act && c == 0) reinterpret_cast<double*>(sV)[2 * r + part] = pw;
    ip_bar();
    // beta_k = sum_i conj(w_raw[i]) B[i][k]     (row index r plays k, c plays i)
    double pb = 0.0;
    if (act) {
      const double2 wi = sV[c];
      const double2 bk = sB[c * M + r];
      pb = part ? fma(wi.x, bk.y, -wi.y * bk.x) : fma(wi.x, bk.x, wi.y * bk.y);
    }
#pragma unroll
    for (int off = 2; off <= 8; off <<= 1) pb += __shfl_xor_sync(0xffffffffu, pb, off);
    if (act && c == 0) reinterpret_cast<double*>(sBeta)[2 * r + part] = pb;
    ip_bar();
    const double s = sBeta[m].x;
    const float sf = (float)s;
    const bool ok = sf > 0.f && sf < INFINITY;
    const double sc = rsqrt_pos_f64(ok ? s : 1.0);
    const double sc2 = sc * sc;
    // B update on row i = r, column k = c; w_m[i] = w_raw[i] sqrt(s)^-1
    double nb = 0.0;
    if (act) {
      const double2 bki = sB[r * M + c];
      const double2 bmi = sB[r * M + m];
      if (c == m) {
        nb = (part ? bmi.y : bmi.x) * sc;
      } else {
        const double2 be = sBeta[c];
        const double cr = be.x * sc2, ci = be.y * sc2;
        nb = part ? fma(-ci, bmi.x, fma(-cr, bmi.y, bki.y)) : fma(ci, bmi.y, fma(-cr, bmi.x, bki.x));
      }
    }
    const double wv = act ? reinterpret_cast<const double*>(sV)[2 * r + part] * sc : 0.0;
    __syncwarp();                         // row r's reads above precede its writes below
    if (act) reinterpret_cast<double*>(sB)[2 * (r * M + c) + part] = nb;
    if (act && c == 0) {
      reinterpret_cast<double*>(sW)[2 * (r * M + m) + part] = wv;
      reinterpret_cast<float*>(sWc)[2 * (m * M + r) + part] = part ? (float)-wv : (float)wv;
    }
    if (!ok && tid == 0) atomicOr(err, kErrIpNorm);
    mant *= ok ? s : 1.0;
    renorm(mant, expo);
    ip_bar();
  }
  if (tid == 0) { sDet[0] = mant; sDet[1] = expo; }
}

// Phase timestamps (clock64) of frequency 0, rank 0, thread 0, for the first 8 iterations,
// 32 slots each; compiled in only with -DFFCA_PHASE_CLOCKS (profiling builds).
#ifdef FFCA_PHASE_CLOCKS
#define FFCA_CMARK(it, slot)                                                                   \
  do {                                                                                         \
    if (p.clocks && f == 0 && crank == 0 && tid == 0 && (it) < 8) p.clocks[(it) * 32 + (slot)] = clock64(); \
  } while (0)
#else
#define FFCA_CMARK(it, slot) \
  do {                       \
  } while (0)
#endif

// Packed Hermitian entry e of x x^H (the order of xxh_packed): e < M is |x_e|^2, then for
// each pair a < b (row-major) Re(x_a conj x_b) and Im(x_a conj x_b).  kind 0 diagonal,
// 1 real part, 2 imaginary part.
template <int M>
__device__ __forceinline__ void decode_entry(int e, int& a, int& b, int& kind) {
  if (e < M) { a = e; b = e; kind = 0; return; }
  int idx = (e - M) >> 1;
  kind = 1 + ((e - M) & 1);
  a = 0;
  while (idx >= M - 1 - a) { idx -= M - 1 - a; ++a; }
  b = a + 1 + idx;
}

// ------------------------------------------------------------------ the kernel
// Grid: F * C CTAs of kCThreads threads in clusters of C (rank c of cluster f owns frames
// [c Tc, ...) of frequency f); dynamic shared memory ClusterSmem<M>::bytes(N, Tc).
// The cluster kernel's arguments: the FastFCA ones, and the FastMNMF outputs of the MN form
// (U, F x M x T, and the bases' update terms a, b, two planes F x N x T; null otherwise).
// They stay out of EmArgs, which the frequency-resident kernels take at their register cap.
struct ClusterArgs {
  EmArgs e;
  float* mn_u;
  float* mn_ab;
  int wait_limit;       // spins of a cluster exchange before it is reported as timed out
};

template <int M, bool MM = false, bool BL = false, bool MN = false>
__global__ void __launch_bounds__(kCThreads, 2) fastfca_em_cluster_kernel(ClusterArgs ca) {
  static_assert(!(MN && BL), "FastMNMF takes frames");
  const EmArgs& p = ca.e;
  using SM = ClusterSmem<M>;
  constexpr int NE = SM::NE, V = SM::V, XV = SM::kXV;
  constexpr int EPL = (NE + 31) / 32;
  constexpr int MP = pow2_ceil(M);
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = (int)cluster_size(), crank = (int)cluster_rank();
  const int f = blockIdx.x / C;
  const int T = p.T, N = p.N;
  const int Tc = (T + C - 1) / C;
  const int Tcp = SM::tcp(Tc);
  // the same outcome in every CTA: no CTA is left waiting at a cluster barrier
  if (N < 1 || N > kCMaxN || blockDim.x != kCThreads || f >= p.F || (C - 1) * Tc >= T ||
      dyn_smem_size() < SM::bytes(N, Tc)) {
    if (tid == 0) atomicOr(p.err, kErrConfig);
    return;
  }
  double2* sW = reinterpret_cast<double2*>(smem + SM::oW);
  double2* sB = reinterpret_cast<double2*>(smem + SM::oB);
  double2* sQ = reinterpret_cast<double2*>(smem + SM::oQ);
  double2* sV = reinterpret_cast<double2*>(smem + SM::oV);
  double2* sBeta = reinterpret_cast<double2*>(smem + SM::oBeta);
  double* sDet = reinterpret_cast<double*>(smem + SM::oDet);
  double* sXll = reinterpret_cast<double*>(smem + SM::oXll);
  float* sX = reinterpret_cast<float*>(smem + SM::oX);
  float2* sWc = reinterpret_cast<float2*>(smem + SM::oWc);
  float* sL = reinterpret_cast<float*>(smem + SM::oL);
  float* sRed = reinterpret_cast<float*>(smem + SM::oRed);
  float* sLL = reinterpret_cast<float*>(smem + SM::oLL);
  float* sQw = reinterpret_cast<float*>(smem + SM::oQw);
  float* sPush = reinterpret_cast<float*>(smem + SM::oPush);       // [parity][rank][warp][8]
  uint64_t* sMbar = reinterpret_cast<uint64_t*>(smem + SM::oMbar);  // [parity]
  float* sH = reinterpret_cast<float*>(smem + SM::oFrames);   // [n][j]
  float* sU = sH + (size_t)N * Tcp;                             // [m][j]
  float* sS = sU + (size_t)M * Tcp;                             // sigma^2 [m][j]
  float* sR = sS + (size_t)M * Tcp;                             // 1/sigma^2 or r [m][j]

  const int t0 = crank * Tc;
  const int Tl = min(Tc, T - t0);
  const float2* xf = BL ? nullptr : p.x + ((size_t)f * T + t0) * M;
  const float* xhf = BL ? p.xh + ((size_t)f * T + t0) * NE : nullptr;     // blocks: packed X^_j
  double2* Pf = p.P + (size_t)f * M * M;
  float* lamf = p.lam + (size_t)f * M * N;
  float* vf = p.v + (size_t)f * N * T;
  const double invT = 1.0 / (double)T;
  const float invTf = 1.0f / (float)T;

  // transaction barriers of the n-loop exchange: each phase expects one value per (CTA, warp,
  // m); armed here for the first two uses, re-armed after each use
  const unsigned push_bytes = (unsigned)(C * kCWarps * M * sizeof(float));
  if (!MM && !MN && tid == 0) {
    mbar_init(&sMbar[0], 1);
    mbar_init(&sMbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&sMbar[0], push_bytes);
    mbar_expect_tx(&sMbar[1], push_bytes);
  }

  // ---- load the parameters (L and W replicated, H for this CTA's frames)
  for (int i = tid; i < M * N; i += kCThreads) sL[i] = lamf[i];
  for (int i = tid; i < M * M; i += kCThreads) sW[i] = Pf[i];
  for (int n = 0; n < N; ++n)
    for (int j = tid; j < Tl; j += kCThreads) sH[n * Tcp + j] = vf[(size_t)n * T + t0 + j];
  __syncthreads();
  if (warp == 0) {
    if (p.b_valid) {
      for (int e = lane; e < M * M; e += 32) sB[e] = p.Bst[(size_t)f * M * M + e];
      if (lane == 0) { sDet[0] = p.detst[2 * f]; sDet[1] = p.detst[2 * f + 1]; }
    } else {
      for (int e = lane; e < M * M; e += 32) {
        const int i = e / M, j = e - (e / M) * M;
        const double2 w = sW[j * M + i];
        sQ[e] = make_double2(w.x, -w.y);                        // W^H
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
  __syncthreads();

  auto load_x = [&](int j, float2 (&xv)[M]) {
    const float2* src = xf + (size_t)j * M;
    if constexpr (M % 2 == 0) {
#pragma unroll
      for (int a = 0; a < M; a += 2) {
        const float4 q4 = __ldg(reinterpret_cast<const float4*>(src + a));
        xv[a] = make_float2(q4.x, q4.y);
        xv[a + 1] = make_float2(q4.z, q4.w);
      }
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) xv[a] = __ldg(src + a);
    }
  };

  // U = |W^H x|^2 for this CTA's frames, two frames per thread at a time (loads overlap);
  // blocks: U = w^H X^ w = sum_a |w_a|^2 X_aa + 2 sum_{a<b} Re(conj(w_a) w_b X_ab), with
  // conj(w_a) = sWc[m M + a] (same frames per thread as for x)
  auto pass_U = [&]() {
    if constexpr (BL) {
      for (int j = tid; j < Tl; j += kCThreads) {
        const float* e = xhf + (size_t)j * NE;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float u = 0.f;
#pragma unroll
          for (int a = 0; a < M; ++a) {
            const float2 wa = sWc[m * M + a];
            u = fmaf(fmaf(wa.x, wa.x, wa.y * wa.y), __ldg(e + a), u);
          }
          int idx = M;
#pragma unroll
          for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a + 1; b < M; ++b) {
              const float2 wa = sWc[m * M + a], wb = sWc[m * M + b];
              const float pr = fmaf(wa.x, wb.x, wa.y * wb.y);       // wa conj(wb)
              const float pi = fmaf(wa.y, wb.x, -wa.x * wb.y);
              u = fmaf(2.f, fmaf(pr, __ldg(e + idx), -pi * __ldg(e + idx + 1)), u);
              idx += 2;
            }
          sU[m * Tcp + j] = u;
        }
      }
    } else {
      for (int j = tid; j < Tl; j += 2 * kCThreads) {
        const int j2 = j + kCThreads;
        float2 xv[M], xw[M];
        load_x(j, xv);
        if (j2 < Tl) load_x(j2, xw);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float2 y = make_float2(0.f, 0.f), z = make_float2(0.f, 0.f);
#pragma unroll
          for (int a = 0; a < M; ++a) {
            const float2 wc = sWc[m * M + a];
            y = cfmaf(wc, xv[a], y);
            z = cfmaf(wc, xw[a], z);
          }
          sU[m * Tcp + j] = fmaf(y.x, y.x, y.y * y.y);
          if (j2 < Tl) sU[m * Tcp + j2] = fmaf(z.x, z.x, z.y * z.y);
        }
      }
    }
  };

  auto ll_from_sum = [&](double s) {
    const double logdet = (double)__logf((float)sDet[0]) + sDet[1] * kLn2;
    return (double)T * logdet - s - (double)M * (double)T * kLnPi;
  };

  // sums over the cluster, in rank order, of the value at this CTA's shared address `local`
  auto cluster_sum = [&](const double* local) {
    double s = 0.0;
    for (int c = 0; c < C; ++c) s += ld_dsmem_f64(dsmem_addr(local, (unsigned)c));
    return s;
  };
  auto cluster_sum_f = [&](const float* local) {
    float s = 0.f;
    for (int c = 0; c < C; ++c) s += ld_dsmem_f32(dsmem_addr(local, (unsigned)c));
    return s;
  };

  // lane -> Hermitian entries of the Q pass
  int ea[EPL], eb[EPL], ek[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int e = lane + 32 * q;
    if (e < NE) decode_entry<M>(e, ea[q], eb[q], ek[q]);
    else { ea[q] = 0; eb[q] = 0; ek[q] = 3; }
  }

  unsigned nphase[2] = {0u, 0u};
  int npar = 0;
  float coef[M], Lold[M], Lnew[M];
#pragma unroll
  for (int m = 0; m < M; ++m) { coef[m] = 0.f; Lold[m] = 0.f; Lnew[m] = 0.f; }
  int par = 0;

  if (p.n_iter == 0 || (MN && p.ll_hist)) {     // the log-likelihood of the incoming W needs its U
    pass_U();
    __syncthreads();
  }

#pragma unroll 1
  for (int it = 0;; ++it) {
    // MN: the launch's one iteration reports the log-likelihood of the incoming parameters,
    // into slot `it` (0); otherwise slot it - 1 holds the value after iteration it - 1
    const bool have_ll = MN ? (p.ll_hist != nullptr || p.n_iter == 0) : ((it > 0) || (p.n_iter == 0));
    const bool do_iter = it < p.n_iter;
    const int ll_slot = MN ? it : it - 1;
    FFCA_CMARK(it, 0);

    // ---- pass A: pending H[N-1,:] update, sigma^2 = L H, 1/sigma^2, log-likelihood terms
    {
      float llp = 0.f;
      bool bad = false;
      for (int j = tid; j < Tl; j += kCThreads) {
        if (!MM && !MN && it > 0) {
          float g = 0.f;
#pragma unroll
          for (int m = 0; m < M; ++m) g = fmaf(sR[m * Tcp + j], coef[m], g);
          sH[(N - 1) * Tcp + j] *= g;
        }
        float h[kCMaxN];
#pragma unroll
        for (int n = 0; n < kCMaxN; ++n) {
          const float hv = sH[(n < N ? n : 0) * Tcp + j];     // index kept inside the array
          h[n] = (n < N) ? hv : 0.f;
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float s2 = 0.f;
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n)
            if (n < N) s2 = fmaf(sL[m * N + (n < N ? n : 0)], h[n], s2);
          bad |= !(s2 > 0.f && s2 < INFINITY);
          const float rs = fast_rcp(s2);
          sS[m * Tcp + j] = s2;
          sR[m * Tcp + j] = rs;
          if (have_ll) llp += fmaf(sU[m * Tcp + j], rs, __logf(s2));
        }
      }
      if (bad) atomicOr(p.err, kErrSigma);
      llp = warp_sum(llp);
      if (lane == 0) sLL[warp] = llp;
    }
    __syncthreads();          // the Q pass reads 1/sigma^2 of frames other threads wrote
    FFCA_CMARK(it, 1);
    float* xb = sX + par * XV;
    double* xll = sXll + par;
    if (!do_iter) {
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < kCWarps; ++w) s += (double)sLL[w];
        *xll = s;
      }
      cluster_sync();
      if (crank == 0 && tid == 0) {
        const double ll = ll_from_sum(cluster_sum(xll));
        if ((MN || it > 0) && p.ll_hist) p.ll_hist[(size_t)f * p.ll_stride + ll_slot] = ll;
        if (p.ll_last) p.ll_last[f] = ll;
      }
      break;
    }

    // ---- Q_m = (1/T) sum_t x x^H / sigma^2_m (Eq. 33).  Warp w takes a contiguous block of
    // frames; one load instruction brings 4 frames x 8 channels (lane 8 f + a holds x_a of
    // frame f), a batch of 32 frames is loaded before any of it is used, and lane l forms
    // the Hermitian entries l + 32 q of every frame from shuffled channels, for every m
    {
      float acc[M][EPL];
#pragma unroll
      for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < EPL; ++q) acc[m][q] = 0.f;
      const int per = (Tl + kCWarps - 1) / kCWarps;
      const int fb = warp * per, fe = min(fb + per, Tl);
      const int lf = lane >> 3, la = lane & 7;
      if constexpr (BL) {
        // lane l reads entries l + 32 q of each block's packed X^ (coalesced per block)
#pragma unroll 4
        for (int fr = fb; fr < fe; ++fr) {
          float ev[EPL];
#pragma unroll
          for (int q = 0; q < EPL; ++q) {
            const int e = lane + 32 * q;
            ev[q] = (e < NE) ? __ldg(xhf + (size_t)fr * NE + e) : 0.f;
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float w = sR[m * Tcp + fr];
#pragma unroll
            for (int q = 0; q < EPL; ++q) acc[m][q] = fmaf(w, ev[q], acc[m][q]);
          }
        }
      }
      if constexpr (!BL) {
        for (int base = fb; base < fe; base += 32) {
          float2 xr[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int fr = base + 4 * k + lf;
            xr[k] = (fr < fe && la < M) ? __ldg(xf + (size_t)fr * M + la) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int fi = 0; fi < 4; ++fi) {
              const int fr = base + 4 * k + fi;          // warp-uniform
              if (fr >= fe) break;
              float ev[EPL];
#pragma unroll
              for (int q = 0; q < EPL; ++q) {
                const float ax = __shfl_sync(0xffffffffu, xr[k].x, fi * 8 + ea[q]);
                const float ay = __shfl_sync(0xffffffffu, xr[k].y, fi * 8 + ea[q]);
                const float bx = __shfl_sync(0xffffffffu, xr[k].x, fi * 8 + eb[q]);
                const float by = __shfl_sync(0xffffffffu, xr[k].y, fi * 8 + eb[q]);
                ev[q] = (ek[q] == 3) ? 0.f
                        : (ek[q] == 0) ? fmaf(ax, ax, ay * ay)
                        : (ek[q] == 1) ? fmaf(ax, bx, ay * by) : fmaf(ay, bx, -ax * by);
              }
#pragma unroll
              for (int m = 0; m < M; ++m) {
                const float w = sR[m * Tcp + fr];
#pragma unroll
                for (int q = 0; q < EPL; ++q) acc[m][q] = fmaf(w, ev[q], acc[m][q]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < EPL; ++q)
          if (lane + 32 * q < NE) sQw[warp * V + m * NE + lane + 32 * q] = acc[m][q];
    }
    __syncthreads();
    // FP32 sums over warps (in warp order) and CTAs (in rank order), one conversion per entry
    for (int i = tid; i < V; i += kCThreads) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kCWarps; ++w) s += sQw[w * V + i];
      xb[i] = s;
    }
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kCWarps; ++w) s += (double)sLL[w];
      *xll = s;
    }
    cluster_sync();
    // only the Q_m this CTA inverts are combined here (rank c owns m = c mod C)
    for (int i = tid; i < V; i += kCThreads) {
      const int m = i / NE, e = i - m * NE;
      if (m % C != crank) continue;
      const double qd = (double)cluster_sum_f(xb + i) * invT;
      int a, b, kind;
      decode_entry<M>(e, a, b, kind);
      double2* Qm = sQ + m * M * M;
      if (kind == 0) Qm[a * M + a] = make_double2(qd, 0.0);
      else if (kind == 1) { Qm[a * M + b].x = qd; Qm[b * M + a].x = qd; }
      else { Qm[a * M + b].y = qd; Qm[b * M + a].y = -qd; }
    }
    if (have_ll && crank == 0 && tid == 0 && p.ll_hist)
      p.ll_hist[(size_t)f * p.ll_stride + ll_slot] = ll_from_sum(cluster_sum(xll));
    par ^= 1;
    __syncthreads();
    FFCA_CMARK(it, 2);

    // ---- IP (FP64): this CTA's share of the Q_m^{-1}, gathered over the cluster, then the
    // column loop (every CTA, identical inputs, identical results)
    // ---- IP (FP64): each CTA inverts its share of the Q_m; rank 0 gathers them and runs
    // the column loop; the other CTAs then copy W, B = W^{-H}, conj(W)^T and |det W|^2
    if (tid < kCIpThreads) cluster_hpd_inverses<M>(sQ, crank, C, tid, p.err);
    cluster_sync();
    FFCA_CMARK(it, 3);
    if (crank == 0) {
      if (C > 1) {
        for (int i = tid; i < M * M * M; i += kCThreads) {
          const int owner = (i / (M * M)) % C;
          if (owner != 0) sQ[i] = ld_dsmem_f64x2(dsmem_addr(sQ + i, (unsigned)owner));
        }
        __syncthreads();
      }
      if (tid < kCIpThreads) cluster_ip_columns<M>(sQ, sW, sB, sWc, sDet, sV, sBeta, tid, p.err);
    }
    if (C > 1) {
      cluster_sync();
      if (crank != 0) {
        for (int i = tid; i < M * M; i += kCThreads) {
          sW[i] = ld_dsmem_f64x2(dsmem_addr(sW + i, 0u));
          sB[i] = ld_dsmem_f64x2(dsmem_addr(sB + i, 0u));
        }
        double2* wc2 = reinterpret_cast<double2*>(sWc);       // kWcPad float2 = kWcPad/2 x 16 B
        for (int i = tid; i < SM::kWcPad / 2; i += kCThreads) wc2[i] = ld_dsmem_f64x2(dsmem_addr(wc2 + i, 0u));
        if (tid == 0) {
          sDet[0] = ld_dsmem_f64(dsmem_addr(sDet, 0u));
          sDet[1] = ld_dsmem_f64(dsmem_addr(sDet + 1, 0u));
        }
      }
    }
    __syncthreads();

    FFCA_CMARK(it, 4);
    // ---- U = |W^H x|^2 (Eq. 37); each thread later reads only its own frames
    pass_U();
    FFCA_CMARK(it, 5);

    if constexpr (MM || MN) {
      // ---- Algorithm 2, the L line: num_mn = sum_t U sigma^-4 H_nt, den_mn = sum_t sigma^-2
      // H_nt with sigma^2 of pass A (L and H unchanged since).  Warp w takes m = w % M and
      // frame phase w / M (kCWarps / M phases; warps past them idle); each lane keeps the 2N
      // sums of its frames, one warp reduction, then the phases and the cluster are summed in
      // a fixed order, so every CTA computes the same L.
      constexpr int NPH = kCWarps / M;
      __syncthreads();        // U of frames other threads wrote (the EM loop reads only its own)
      float acc[2 * kCMaxN];
#pragma unroll
      for (int i = 0; i < 2 * kCMaxN; ++i) acc[i] = 0.f;
      const int m = warp % M, ph = warp / M;
      if (ph < NPH) {
        for (int j = ph * 32 + lane; j < Tl; j += NPH * 32) {
          const float rs = sR[m * Tcp + j];
          const float a = sU[m * Tcp + j] * rs * rs;
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) {
            if (n < N) {
              const float hv = sH[n * Tcp + j];
              acc[n] = fmaf(a, hv, acc[n]);
              acc[kCMaxN + n] = fmaf(rs, hv, acc[kCMaxN + n]);
            }
          }
        }
      }
      warp_reduce_scatter<2 * kCMaxN>(acc, lane);          // lane l: total of element l
      float* scr = sPush;                                   // the EM exchange rows, unused here
      scr[warp * 32 + lane] = acc[0];
      __syncthreads();
      float* xm = sX + par * XV;                            // [num (M N)][den (M N)]
      for (int i = tid; i < 2 * M * N; i += kCThreads) {
        const int half = i / (M * N), mn = i - half * (M * N);
        const int mm = mn / N, n = mn - mm * N;
        float s2 = 0.f;
        for (int q = 0; q < NPH; ++q) s2 += scr[(q * M + mm) * 32 + half * kCMaxN + n];
        xm[i] = s2;
      }
      cluster_sync();
      for (int i = tid; i < M * N; i += kCThreads) {
        const float num = cluster_sum_f(xm + i);
        const float den = cluster_sum_f(xm + M * N + i);
        // a source whose H row has underflowed to zero gives 0/0: it has no effect on the
        // model, and L[:, n] is left as it is
        sL[i] *= (den > 0.f) ? sqrtf(num / den) : 1.0f;
      }
      par ^= 1;
      __syncthreads();
      if constexpr (MN) {
        // ---- FastMNMF: U and the bases' update terms with sigma^2 from the new lambda and
        // the given h, for this CTA's frames; then the launch's one iteration is done
        const size_t plane = (size_t)p.F * N * T;
        for (int j = tid; j < Tl; j += kCThreads) {
          float h[kCMaxN];
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) h[n] = (n < N) ? sH[n * Tcp + j] : 0.f;
          float e[M], r[M];
          bool bad = false;
#pragma unroll
          for (int m2 = 0; m2 < M; ++m2) {
            float s2 = 0.f;
#pragma unroll
            for (int n = 0; n < kCMaxN; ++n)
              if (n < N) s2 = fmaf(sL[m2 * N + n], h[n], s2);
            bad |= !(s2 > 0.f && s2 < INFINITY);
            r[m2] = fast_rcp(s2);
            const float u = sU[m2 * Tcp + j];
            e[m2] = u * r[m2] * r[m2];
            ca.mn_u[((size_t)f * M + m2) * T + t0 + j] = u;
          }
          if (bad) atomicOr(p.err, kErrSigma);
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) {
            if (n < N) {
              float a = 0.f, b = 0.f;
#pragma unroll
              for (int m2 = 0; m2 < M; ++m2) {
                a = fmaf(sL[m2 * N + n], e[m2], a);
                b = fmaf(sL[m2 * N + n], r[m2], b);
              }
              ca.mn_ab[((size_t)f * N + n) * T + t0 + j] = a;
              ca.mn_ab[plane + ((size_t)f * N + n) * T + t0 + j] = b;
            }
          }
        }
        break;                 // uniform over the cluster: every CTA leaves after one iteration
      } else {
        // ---- the H line: H <- H (.) {L^T [U (.) sigma^-4] / L^T sigma^-2}^1/2, sigma^2 from
        // the new L, frame by frame (this CTA's frames only)
        for (int j = tid; j < Tl; j += kCThreads) {
          float h[kCMaxN];
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) h[n] = (n < N) ? sH[n * Tcp + j] : 0.f;
          float a[M], b[M];
#pragma unroll
          for (int m2 = 0; m2 < M; ++m2) {
            float s2 = 0.f;
#pragma unroll
            for (int n = 0; n < kCMaxN; ++n)
              if (n < N) s2 = fmaf(sL[m2 * N + n], h[n], s2);
            const float rs = fast_rcp(s2);
            b[m2] = rs;
            a[m2] = sU[m2 * Tcp + j] * rs * rs;
          }
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) {
            if (n < N) {
              float num = 0.f, den = 0.f;
#pragma unroll
              for (int m2 = 0; m2 < M; ++m2) {
                num = fmaf(sL[m2 * N + n], a[m2], num);
                den = fmaf(sL[m2 * N + n], b[m2], den);
              }
              sH[n * Tcp + j] = (den > 0.f) ? h[n] * sqrtf(num * fast_rcp(den)) : h[n];
            }
          }
        }
        __syncthreads();
      }
    } else {
      // ---- NMF EM sweep over sources (Gauss-Seidel); pass n first applies source n-1's
      // H update and its change of sigma^2
#pragma unroll 1
      for (int n = 0; n < N; ++n) {
        float Ln[M];
#pragma unroll
        for (int m = 0; m < M; ++m) Ln[m] = sL[m * N + n];
        float acc[MP];
#pragma unroll
        for (int m = 0; m < MP; ++m) acc[m] = 0.f;
        for (int j = tid; j < Tl; j += kCThreads) {
          if (n > 0) {
            float g = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) g = fmaf(sR[m * Tcp + j], coef[m], g);
            const float hold = sH[(n - 1) * Tcp + j];
            const float hnew = hold * g;
            sH[(n - 1) * Tcp + j] = hnew;
#pragma unroll
            for (int m = 0; m < M; ++m) {
              // sigma^2 <- sigma^2 - L H + L' H' (one rounding: fma), never below the new term
              const float s2 = fmaf(Lnew[m], hnew, fmaf(-Lold[m], hold, sS[m * Tcp + j]));
              sS[m * Tcp + j] = fmaxf(s2, Lnew[m] * hnew);
            }
          }
          const float hn = sH[n * Tcp + j];
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float s2 = sS[m * Tcp + j];
            const float rs = fast_rcp(s2);
            const float G = Ln[m] * hn * rs;
            const float rr = fmaf(G, fmaf(sU[m * Tcp + j], rs, -1.f), 1.f);
            sR[m * Tcp + j] = rr;
            acc[m] += rr;
          }
        }
        // per-warp sums are pushed (st.async) into every CTA's receive row [rank][warp][m] of
        // this parity, counted by that CTA's transaction barrier; each CTA waits on its own
        // barrier, then lane (m, q) adds warps 2q, 2q+1 of every rank in rank order and two
        // shuffles finish: the same order in every warp of every CTA.  A parity's row is
        // rewritten only after every warp here has pushed the next exchange, i.e. read this one.
        warp_reduce_scatter<MP>(acc, lane);
        float* rb = sPush + npar * (kCMaxCluster * kCWarps * 8);
        if ((lane * MP) % 32 == 0 && (lane * MP) / 32 < M) {
          float* slot = rb + (crank * kCWarps + warp) * 8 + (lane * MP) / 32;
          for (int c = 0; c < C; ++c)
            st_async_f32(dsmem_addr(slot, (unsigned)c), acc[0], dsmem_addr(&sMbar[npar], (unsigned)c));
        }
        if (ca.wait_limit <= 0) {
          int spins = 0;
          while (!mbar_try_wait(&sMbar[npar], nphase[npar]) && ++spins < kMbarSpinLimit) {
          }
          if (spins >= kMbarSpinLimit && lane == 0) atomicOr(p.err, kErrClusterWait);
        } else {
          // an injected limit (failure tests): wait_limit non-blocking polls, then the exchange
          // is reported as timed out and the wait continues, bounded by the default limit, so
          // the peers' pushes still land in this phase (the barrier's phase count stays in
          // step and nothing is written into this CTA's shared memory after it moves on)
          int spins = 0;
          bool done = false;
          while (!(done = mbar_test_wait(&sMbar[npar], nphase[npar])) && ++spins < ca.wait_limit) {
          }
          if (!done) {
            if (lane == 0) atomicOr(p.err, kErrClusterWait);
            int drain = 0;
            while (!mbar_try_wait(&sMbar[npar], nphase[npar]) && ++drain < kMbarSpinLimit) {
            }
          }
        }
        nphase[npar] ^= 1u;
        float tot_l = 0.f;
        {
          const int m = lane >> 2, q = lane & 3;
          if (m < M) {
            for (int c = 0; c < C; ++c) {
              tot_l += rb[(c * kCWarps + 2 * q) * 8 + m];
              tot_l += rb[(c * kCWarps + 2 * q + 1) * 8 + m];
            }
          }
          tot_l += __shfl_xor_sync(0xffffffffu, tot_l, 1);
          tot_l += __shfl_xor_sync(0xffffffffu, tot_l, 2);
        }
        if (tid == 0) mbar_expect_tx(&sMbar[npar], push_bytes);   // arm this parity's next use
        npar ^= 1;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float mean = __shfl_sync(0xffffffffu, tot_l, 4 * m) * invTf;
          Lold[m] = Ln[m];
          Lnew[m] = Ln[m] * mean;
          sL[m * N + n] = Lnew[m];           // the same value from every thread
          coef[m] = fast_rcp(mean) * (1.0f / (float)M);
        }
        FFCA_CMARK(it, 6 + (n < 25 ? n : 25));
      }
    }
  }

  // ---- write back: this CTA's frames of H (FastMNMF: H is an input); rank 0 the
  // per-frequency parameters
  __syncthreads();
  if (!MN)
    for (int n = 0; n < N; ++n)
      for (int j = tid; j < Tl; j += kCThreads) vf[(size_t)n * T + t0 + j] = sH[n * Tcp + j];
  if (crank == 0) {
    for (int i = tid; i < M * N; i += kCThreads) lamf[i] = sL[i];
    for (int i = tid; i < M * M; i += kCThreads) {
      Pf[i] = sW[i];
      p.Bst[(size_t)f * M * M + i] = sB[i];
    }
    if (tid == 0) { p.detst[2 * f] = sDet[0]; p.detst[2 * f + 1] = sDet[1]; }
  }
  cluster_sync();          // no CTA exits while a peer may still read its shared memory
}

}  // namespace ffca

// FastFCA IP+EM (Algorithm 1) for large bins, one SM per frequency, the per-frame state in
// tensor memory.
//
// The cluster kernel (fastfca_em_cluster.cuh) spreads a frequency's frames over up to eight
// CTAs because one SM's shared memory cannot hold H, U, sigma^2 and r for thousands of frames.
// Every Q reduction, the IP hand-off and each of the N source means then cross SMs, and each
// crossing waits for the slowest of the cluster's CTAs.  This kernel keeps a whole frequency
// (T <= 4096 frames, M <= 8) on one SM instead, with the SM's 256 KB of tensor memory (TMEM,
// reached with tcgen05.ld / tcgen05.st) as the per-frame store:
//
//   TMEM (all 512 columns, 128 lanes)   sigma^2 and U of every frame (16 32-bit columns per
//                                       frame: sigma^2_m at 0..7, U_m at 8..15)
//   shared memory                       r_mt (the n-loop's per-frame ratios) and 1/sigma^2,
//                                       in two planes [frame][4] (m < 4, m >= 4), so a warp's
//                                       float4 accesses of consecutive frames are conflict-free;
//                                       the last source row of H per frame slot; Q partials;
//                                       W, B, Q_m in FP64
//   global memory (L2)                  H = v[f], updated in place row by row; x
//
// Thread `tid` of the 512 owns frames t = tid + k * 512, k < 8, and reaches its frames' TMEM
// columns in its warp's lane quarter (lane 32 (warp % 4) + lane, columns 128 (warp / 4) +
// 16 k ...).  Every reduction is CTA-local, so no step waits on another SM.
//
// The steps, their order and their arithmetic are those of the cluster kernel (see its file
// comment and fastfca_em.cuh for the equations): pass A (pending H[N-1,:] update, sigma^2 =
// L H, 1/sigma^2, log-likelihood terms), the Q pass (Eq. 33), the IP (Eq. 34-35, FP64), the
// U pass (Eq. 37) and the n-loop (Gauss-Seidel over sources, sigma^2 updated by the change of
// each source's term), with reductions over t in a fixed order.
#pragma once
#include "fastfca_em_cluster.cuh"

namespace ffca {

constexpr int kSThreads = 512;               // threads per CTA (one CTA per SM: 512 x 128 registers)
constexpr int kSWarps = kSThreads / 32;
constexpr int kSSlots = 8;                   // frames per thread
constexpr int kSMaxT = kSThreads * kSSlots;  // 4096 frames
constexpr int kSMaxM = 8;
constexpr unsigned kSCols = 512;             // TMEM columns allocated: all of them
constexpr int kSColsPerSlot = 16;            // sigma^2 (8 columns), then U (8 columns)


// ------------------------------------------------------------------ shared-memory layout
template <int M>
struct SmSmem {
  static constexpr int NE = M * M;                        // packed Hermitian entries of Q_m
  static constexpr int V = M * NE;                        // reals of all Q_m
  static constexpr int kQsz = (M * M * M > 3 * M * M) ? M * M * M : 3 * M * M;
  static constexpr int kWcPad = (M * M + 1) & ~1;
  // byte offsets (all multiples of 16)
  static constexpr size_t oR = 0;                                          // float [2][kSMaxT][4]
  static constexpr size_t oHp = oR + 4 * (size_t)kSMaxT * 8;               // float [kSSlots][kSThreads]
  static constexpr size_t oQw = oHp + 4 * (size_t)kSSlots * kSThreads;     // float [kSWarps/2][V]
  static constexpr size_t oW = oQw + 4 * (size_t)(kSWarps / 2) * V;       // double2 M*M
  static constexpr size_t oB = oW + 16 * M * M;                            // double2 M*M
  static constexpr size_t oQ = oB + 16 * M * M;                            // double2 kQsz
  static constexpr size_t oV = oQ + 16 * (size_t)kQsz;                     // double2 8 (w_raw)
  static constexpr size_t oBeta = oV + 16 * 8;                             // double2 8
  static constexpr size_t oDet = oBeta + 16 * 8;                           // double 4
  static constexpr size_t oPiv = oDet + 32;                                // double 8 (pivot reciprocals)
  static constexpr size_t oWc = oPiv + 64;                                 // float2 kWcPad
  static constexpr size_t oL = oWc + ((8 * (size_t)kWcPad + 15) & ~(size_t)15);   // float M*kCMaxN
  static constexpr size_t oLt = oL + 4 * (size_t)M * kCMaxN;              // float [kCMaxN][8]: L transposed
  static constexpr size_t oRed = oLt + 4 * (size_t)kCMaxN * 8;            // float 2 x kSWarps x 8
  static constexpr size_t oLL = oRed + 4 * 2 * kSWarps * 8;                // float kSWarps
  static constexpr size_t oTmem = oLL + 4 * kSWarps;                       // uint32 TMEM base (+ pad)
  static constexpr size_t bytes = oTmem + 16;
};

// Lane jobs of the Q pass: each lane forms two packed entries of x x^H per frame from four
// shuffled values.  Lanes 0 .. P-1 take the pairs a < b (row-major, P = M(M-1)/2) and give
// Re and Im of x_a conj(x_b); the next ceil(M/2) lanes take two diagonal entries |x_a|^2,
// |x_{a+1}|^2 (one when a + 1 = M); the rest are idle.  For M = 8 that is 28 + 4 = 32 lanes.
template <int M>
__device__ __forceinline__ void sm_lane_job(int lane, int& a, int& b, int& kind, int& e0, int& e1) {
  constexpr int P = M * (M - 1) / 2;
  if (lane < P) {
    int idx = lane;
    a = 0;
    while (idx >= M - 1 - a) { idx -= M - 1 - a; ++a; }
    b = a + 1 + idx;
    kind = 0;
    e0 = M + 2 * lane;
    e1 = e0 + 1;
  } else if (lane < P + (M + 1) / 2) {
    a = 2 * (lane - P);
    b = (a + 1 < M) ? a + 1 : a;
    kind = 1;
    e0 = a;
    e1 = (a + 1 < M) ? a + 1 : -1;
  } else {
    a = 0; b = 0; kind = 2; e0 = -1; e1 = -1;
  }
}

// -x with an integer operation on the sign bit (no FP64 instruction).
__device__ __forceinline__ double neg_f64(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// In-place inverses of the M matrices Q_m (HPD, row-major, consecutive) by the four FP64 warps
// (threads 0..127), by the Hermitian sweep: step k, with d = a_kk > 0,
//   a_ij <- a_ij - a_ik a_kj / d  (i, j != k),   a_kj <- a_kj / d,   a_ik <- a_ik / d,
//   a_kk <- -1 / d,
// keeps the matrix Hermitian and leaves -Q^{-1} after the M steps.  Only the upper triangle
// is updated (entries below the diagonal are read as conj(a_ji)), which is 36 of the 64
// entries at M = 8; the off-diagonal entries take two slots of the 128 threads and the real
// diagonal entries one, three FP64 instructions each instead of six.  On this part every FP64
// warp instruction holds its sub-partition's FP64 unit for ~68 cycles, so the instruction count
// per warp sets the time.  The reciprocal of each step's pivot is formed once per matrix, by
// the thread that wrote that pivot in the step before (or by thread m for step 0), and read
// from shared memory.  A final pass writes -a (upper) and -conj(a) (lower) so that Q holds the
// full Q^{-1}.  A non-positive pivot sets kErrQPivot.
template <int M>
__device__ void sm_hpd_inverses(double2* Q, double* sPiv, int tid, int* err) {
  constexpr int E = M * M;
  constexpr int P = M * (M - 1) / 2;                                  // upper pairs per matrix
  constexpr int kOff = (M * P + kCIpThreads - 1) / kCIpThreads;       // slots of pairs
  constexpr int kDia = (M * M + kCIpThreads - 1) / kCIpThreads;       // slots of diagonal entries
  auto pivot_rcp = [&](double d, int m) {
    const float df = (float)d;
    const bool ok = df > 0.f && df < INFINITY;
    if (!ok) atomicOr(err, kErrQPivot);
    sPiv[m] = rcp_pos_f64(ok ? d : 1.0);
  };
  // this thread's pairs (matrix, r < c) and diagonal entries (matrix, r), -1 when idle
  int om[kOff], orr[kOff], oc[kOff], dm[kDia], dr[kDia];
#pragma unroll
  for (int s = 0; s < kOff; ++s) {
    const int i = tid + s * kCIpThreads;
    om[s] = -1; orr[s] = 0; oc[s] = 1;
    if (i < M * P) {
      om[s] = i / P;
      int idx = i - om[s] * P, a = 0;
      while (idx >= M - 1 - a) { idx -= M - 1 - a; ++a; }
      orr[s] = a;
      oc[s] = a + 1 + idx;
    }
  }
#pragma unroll
  for (int s = 0; s < kDia; ++s) {
    const int i = tid + s * kCIpThreads;
    dm[s] = i < M * M ? i / M : -1;
    dr[s] = i < M * M ? i - (i / M) * M : 0;
  }
  // a_ij of matrix A read from the upper triangle
  auto get = [&](const double2* A, int i, int j) {
    if (i <= j) return A[i * M + j];
    const double2 v = A[j * M + i];
    return make_double2(v.x, neg_f64(v.y));
  };
  if (tid < M) pivot_rcp(Q[tid * E].x, tid);
  ip_bar();
  for (int k = 0; k < M; ++k) {
    double2 nv[kOff];
    double nd[kDia];
#pragma unroll
    for (int s = 0; s < kOff; ++s) {
      nv[s] = make_double2(0.0, 0.0);
      if (om[s] >= 0) {
        const double2* A = Q + om[s] * E;
        const int r = orr[s], c = oc[s];
        const double rd = sPiv[om[s]];
        double2 base = make_double2(0.0, 0.0), c1, c2;
        if (r != k && c != k) {
          base = A[r * M + c];
          c1 = get(A, r, k);
          c2 = get(A, k, c);
        } else if (r == k) {                        // row k: a_kc / d
          c1 = make_double2(-1.0, 0.0);
          c2 = A[k * M + c];
        } else {                                    // column k: a_rk / d
          c1 = A[r * M + k];
          c2 = make_double2(-1.0, 0.0);
        }
        const double2 u = make_double2(c2.x * rd, c2.y * rd);
        nv[s] = make_double2(fma(c1.y, u.y, fma(-c1.x, u.x, base.x)), fma(-c1.y, u.x, fma(-c1.x, u.y, base.y)));
      }
    }
#pragma unroll
    for (int s = 0; s < kDia; ++s) {
      nd[s] = 0.0;
      if (dm[s] >= 0) {
        const double2* A = Q + dm[s] * E;
        const int r = dr[s];
        const double rd = sPiv[dm[s]];
        const double2 g = (r != k) ? get(A, r, k) : make_double2(1.0, 0.0);
        const double base = (r != k) ? A[r * M + r].x : 0.0;
        nd[s] = fma(-fma(g.x, g.x, g.y * g.y), rd, base);
      }
    }
    ip_bar();
#pragma unroll
    for (int s = 0; s < kOff; ++s)
      if (om[s] >= 0) Q[om[s] * E + orr[s] * M + oc[s]] = nv[s];
#pragma unroll
    for (int s = 0; s < kDia; ++s)
      if (dm[s] >= 0) {
        Q[dm[s] * E + dr[s] * (M + 1)] = make_double2(nd[s], 0.0);
        if (k + 1 < M && dr[s] == k + 1) pivot_rcp(nd[s], dm[s]);
      }
    ip_bar();
  }
  // Q <- -(the swept matrix), upper triangle in place and lower triangle by conjugation
  constexpr int kAll = (M * E + kCIpThreads - 1) / kCIpThreads;
  double2 fin[kAll];
#pragma unroll
  for (int s = 0; s < kAll; ++s) {
    const int i = tid + s * kCIpThreads;
    if (i < M * E) {
      const int mo = i / E, e = i - mo * E, r = e / M, c = e - (e / M) * M;
      const double2 v = get(Q + mo * E, r, c);
      fin[s] = make_double2(neg_f64(v.x), neg_f64(v.y));
    }
  }
  ip_bar();
#pragma unroll
  for (int s = 0; s < kAll; ++s) {
    const int i = tid + s * kCIpThreads;
    if (i < M * E) Q[i] = fin[s];
  }
  ip_bar();
}

#ifdef FFCA_PHASE_CLOCKS
#define FFCA_SMARK(it, slot)                                                                   \
  do {                                                                                         \
    if (p.clocks && f == 0 && tid == 0 && (it) < 8) p.clocks[(it) * 32 + (slot)] = clock64();  \
  } while (0)
#else
#define FFCA_SMARK(it, slot) \
  do {                       \
  } while (0)
#endif

// ------------------------------------------------------------------ the kernel
// Grid: F CTAs of kSThreads threads, one frequency each; dynamic shared memory
// SmSmem<M>::bytes.  Requires T <= kSMaxT, N <= kCMaxN.
template <int M>
__global__ void __launch_bounds__(kSThreads, 1) fastfca_em_sm_kernel(EmArgs p) {
  static_assert(M >= 2 && M <= kSMaxM, "M out of range");
  using SM = SmSmem<M>;
  constexpr int NE = SM::NE, V = SM::V;
  constexpr int MP = pow2_ceil(M);
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int f = blockIdx.x;
  const int T = p.T, N = p.N;
  if (N < 1 || N > kCMaxN || blockDim.x != kSThreads || f >= p.F || T < 1 || T > kSMaxT ||
      dyn_smem_size() < SM::bytes) {
    if (tid == 0) atomicOr(p.err, kErrConfig);
    return;
  }
  float* sRr = reinterpret_cast<float*>(smem + SM::oR);          // [2][t][4]: 1/sigma^2 or r
  float* sHp = reinterpret_cast<float*>(smem + SM::oHp);         // [k][tid]: H of the last source done
  float* sQw = reinterpret_cast<float*>(smem + SM::oQw);
  double2* sW = reinterpret_cast<double2*>(smem + SM::oW);
  double2* sB = reinterpret_cast<double2*>(smem + SM::oB);
  double2* sQ = reinterpret_cast<double2*>(smem + SM::oQ);
  double2* sV = reinterpret_cast<double2*>(smem + SM::oV);
  double2* sBeta = reinterpret_cast<double2*>(smem + SM::oBeta);
  double* sDet = reinterpret_cast<double*>(smem + SM::oDet);
  double* sPiv = reinterpret_cast<double*>(smem + SM::oPiv);
  float2* sWc = reinterpret_cast<float2*>(smem + SM::oWc);
  float* sL = reinterpret_cast<float*>(smem + SM::oL);
  float* sLt = reinterpret_cast<float*>(smem + SM::oLt);         // [n][8] = L[m][n], zero for m >= M
  float* sRed = reinterpret_cast<float*>(smem + SM::oRed);       // [parity][warp][8]
  float* sLL = reinterpret_cast<float*>(smem + SM::oLL);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + SM::oTmem);

  const float2* xf = p.x + (size_t)f * T * M;
  double2* Pf = p.P + (size_t)f * M * M;
  float* lamf = p.lam + (size_t)f * M * N;
  float* vf = p.v + (size_t)f * N * T;
  const double invT = 1.0 / (double)T;
  const float invTf = 1.0f / (float)T;
  const int KF = (T + kSThreads - 1) / kSThreads;          // frame slots in use, the same for every thread

  // ---- tensor memory: warp 0 allocates all 512 columns; the address reaches every thread
  if (warp == 0) tmem_alloc(sTmem, kSCols);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = *sTmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));
  auto tm_s2 = [&](int k) { return tmem + (uint32_t)(kSColsPerSlot * k); };

  // ---- parameters: L and W in shared memory, B = W^{-H} and |det W|^2 (carried or formed)
  for (int i = tid; i < M * N; i += kSThreads) sL[i] = lamf[i];
  for (int i = tid; i < kCMaxN * 8; i += kSThreads) {
    const int n = i >> 3, m = i & 7;
    sLt[i] = (n < N && m < M) ? lamf[m * N + n] : 0.f;
  }
  for (int i = tid; i < M * M; i += kSThreads) sW[i] = Pf[i];
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

  // U = |W^H x|^2 of this thread's frames into TMEM (columns 8..15 of each frame slot)
  auto load_x = [&](int t, float2 (&xv)[M]) {
    const float2* src = xf + (size_t)t * M;
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
  auto pass_U = [&]() {
#pragma unroll
    for (int k = 0; k < kSSlots; ++k) {
      if (k >= KF) break;                                  // uniform over the CTA
      const int t = tid + k * kSThreads;
      float u[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) u[m] = 0.f;
      if (t < T) {
        float2 xv[M];
        load_x(t, xv);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float2 y = make_float2(0.f, 0.f);
          if constexpr (M % 2 == 0) {           // row m starts on a 16-byte boundary
            const float4* row = reinterpret_cast<const float4*>(sWc + m * M);
#pragma unroll
            for (int a = 0; a < M; a += 2) {
              const float4 w2 = row[a / 2];
              y = cfmaf(make_float2(w2.x, w2.y), xv[a], y);
              y = cfmaf(make_float2(w2.z, w2.w), xv[a + 1], y);
            }
          } else {
#pragma unroll
            for (int a = 0; a < M; ++a) y = cfmaf(sWc[m * M + a], xv[a], y);
          }
          u[m] = fmaf(y.x, y.x, y.y * y.y);
        }
      }
      tmem_st8(tm_s2(k) + 8, u);
    }
    tmem_wait_st();
  };

  auto ll_from_sum = [&](double s) {
    const double logdet = (double)__logf((float)sDet[0]) + sDet[1] * kLn2;
    return (double)T * logdet - s - (double)M * (double)T * kLnPi;
  };

  // lane job of the Q pass
  int ja, jb, jkind, je0, je1;
  sm_lane_job<M>(lane, ja, jb, jkind, je0, je1);

  float coef[M], Lold[M], Lnew[M];
#pragma unroll
  for (int m = 0; m < M; ++m) { coef[m] = 0.f; Lold[m] = 0.f; Lnew[m] = 0.f; }
  // the eight ratios of frame t (two conflict-free float4) and the H of a thread's slot k
  auto r_load = [&](int t, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(sRr + 4 * t);
    const float4 b = *reinterpret_cast<const float4*>(sRr + 4 * kSMaxT + 4 * t);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  };
  auto r_store = [&](int t, const float (&v)[8]) {
    *reinterpret_cast<float4*>(sRr + 4 * t) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(sRr + 4 * kSMaxT + 4 * t) = make_float4(v[4], v[5], v[6], v[7]);
  };
  float* hprev = sHp + tid;                                      // hprev[k * kSThreads]
  int rpar = 0;

  if (p.n_iter == 0) {          // the log-likelihood of the incoming W needs its U
    pass_U();
    __syncthreads();
  }

#pragma unroll 1
  for (int it = 0;; ++it) {
    const bool have_ll = (it > 0) || (p.n_iter == 0);
    const bool do_iter = it < p.n_iter;
    FFCA_SMARK(it, 0);

    // ---- pass A: pending H[N-1,:] update, sigma^2 = L H into TMEM, 1/sigma^2 into sRr,
    // log-likelihood terms
    {
      float llp = 0.f;
      bool bad = false;
      if (it > 0) {                      // the last source's H update, for every slot first
#pragma unroll
        for (int k = 0; k < kSSlots; ++k) {
          const int t = tid + k * kSThreads;
          if (k < KF && t < T) {
            float rv[8];
            r_load(t, rv);
            float g = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) g = fmaf(rv[m], coef[m], g);
            const float hn = hprev[k * kSThreads] * g;
            hprev[k * kSThreads] = hn;
            vf[(size_t)(N - 1) * T + t] = hn;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kSSlots; ++k) {
        if (k >= KF) break;                                // uniform over the CTA
        const int t = tid + k * kSThreads;
        float u[8], s2v[8];
        if (have_ll) tmem_ld8(tm_s2(k) + 8, u);
#pragma unroll
        for (int m = 0; m < 8; ++m) s2v[m] = 1.f;
        if (t < T) {
          // H[n][t] for every source (the pending row from the register), all loads in flight
          // together; then sigma^2_m = sum_n L[m][n] H[n][t] source by source against rows of
          // L^T (two float4 per source, eight independent accumulations)
          float h[kCMaxN];
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) {
            if (n < N) h[n] = (it > 0 && n == N - 1) ? hprev[k * kSThreads] : vf[(size_t)n * T + t];
            else h[n] = 0.f;
          }
          float acc2[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) acc2[m] = 0.f;
#pragma unroll
          for (int n = 0; n < kCMaxN; ++n) {
            if (n < N) {
              const float4 l0 = *reinterpret_cast<const float4*>(sLt + n * 8);
              const float4 l1 = *reinterpret_cast<const float4*>(sLt + n * 8 + 4);
              const float lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
              for (int m = 0; m < M; ++m) acc2[m] = fmaf(lv[m], h[n], acc2[m]);
            }
          }
          float rs[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) rs[m] = 0.f;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float s2 = acc2[m];
            bad |= !(s2 > 0.f && s2 < INFINITY);
            rs[m] = fast_rcp(s2);
            s2v[m] = s2;
            if (have_ll) llp += fmaf(u[m], rs[m], __logf(s2));
          }
          r_store(t, rs);
        }
        tmem_st8(tm_s2(k), s2v);
      }
      tmem_wait_st();
      if (bad) atomicOr(p.err, kErrSigma);
      llp = warp_sum(llp);
      if (lane == 0) sLL[warp] = llp;
    }
    __syncthreads();          // the Q pass reads 1/sigma^2 of frames other threads wrote
    FFCA_SMARK(it, 1);
    if (have_ll && tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kSWarps; ++w) s += (double)sLL[w];
      const double ll = ll_from_sum(s);
      if (it > 0 && p.ll_hist) p.ll_hist[(size_t)f * p.ll_stride + it - 1] = ll;
      if (!do_iter && p.ll_last) p.ll_last[f] = ll;
    }
    if (!do_iter) break;

    // ---- Q_m = (1/T) sum_t x x^H / sigma^2_m (Eq. 33).  Warp w takes a contiguous block of
    // frames; one load instruction brings 4 frames x 8 channels (lane 8 f + a loads x_a of
    // frame f) into shared memory; each lane forms its two entries from two values read there
    // and accumulates them for every m with the weights 1/sigma^2 read as two broadcast float4.
    {
      float acc[M][2];
#pragma unroll
      for (int m = 0; m < M; ++m) { acc[m][0] = 0.f; acc[m][1] = 0.f; }
      const int per = (T + kSWarps - 1) / kSWarps;
      const int fb = warp * per, fe = min(fb + per, T);
      const int lf = lane >> 3, la = lane & 7;
      // the block's x staged in this warp's 1 KB of the last-source H buffer (dead from pass A
      // until the n-loop's first source): 16 frames x 8 channels
      float2* sX = reinterpret_cast<float2*>(sHp) + warp * 128;
      // the next block's x is loaded into registers while this block is accumulated
      float2 xn[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int fr = fb + 4 * k + lf;
        xn[k] = (fr < fe && la < M) ? __ldg(xf + (size_t)fr * M + la) : make_float2(0.f, 0.f);
      }
#pragma unroll 1
      for (int base = fb; base < fe; base += 16) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sX[(4 * k + lf) * 8 + la] = xn[k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int fr = base + 16 + 4 * k + lf;
          xn[k] = (fr < fe && la < M) ? __ldg(xf + (size_t)fr * M + la) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int fi = 0; fi < 16; ++fi) {
          const int fr = base + fi;                    // warp-uniform
          if (fr >= fe) break;
          const float2 xa = sX[fi * 8 + ja], xb = sX[fi * 8 + jb];
          const float ax = xa.x, ay = xa.y, bx = xb.x, by = xb.y;
          const float v0 = (jkind == 0) ? fmaf(ax, bx, ay * by) : fmaf(ax, ax, ay * ay);
          const float v1 = (jkind == 0) ? fmaf(ay, bx, -ax * by) : fmaf(bx, bx, by * by);
          const float4 w0 = *reinterpret_cast<const float4*>(sRr + 4 * fr);
          const float4 w1 = *reinterpret_cast<const float4*>(sRr + 4 * kSMaxT + 4 * fr);
          const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
          for (int m = 0; m < M; ++m) {
            acc[m][0] = fmaf(wv[m], v0, acc[m][0]);
            acc[m][1] = fmaf(wv[m], v1, acc[m][1]);
          }
        }
        __syncwarp();                                  // the block's reads before the next stores
      }
      // per-warp partials, summed in a fixed order: warp w + 8 onto warp w, then warps 0..7
      if (warp >= kSWarps / 2) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if (je0 >= 0) sQw[(warp - kSWarps / 2) * V + m * NE + je0] = acc[m][0];
          if (je1 >= 0) sQw[(warp - kSWarps / 2) * V + m * NE + je1] = acc[m][1];
        }
      }
      __syncthreads();
      if (warp < kSWarps / 2) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if (je0 >= 0) sQw[warp * V + m * NE + je0] = acc[m][0] + sQw[warp * V + m * NE + je0];
          if (je1 >= 0) sQw[warp * V + m * NE + je1] = acc[m][1] + sQw[warp * V + m * NE + je1];
        }
      }
      __syncthreads();
      for (int i = tid; i < V; i += kSThreads) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kSWarps / 2; ++w) s += sQw[w * V + i];
        const double qd = (double)s * invT;
        const int m = i / NE, e = i - m * NE;
        int a, b, kind;
        decode_entry<M>(e, a, b, kind);
        double2* Qm = sQ + m * M * M;
        if (kind == 0) Qm[a * M + a] = make_double2(qd, 0.0);
        else if (kind == 1) { Qm[a * M + b].x = qd; Qm[b * M + a].x = qd; }
        else { Qm[a * M + b].y = qd; Qm[b * M + a].y = -qd; }
      }
      __syncthreads();
    }
    FFCA_SMARK(it, 2);

    // ---- IP (FP64): the M inverses Q_m^{-1}, then the column loop of Eq. 34-35, on the four
    // FP64 warps (one per sub-partition); the other warps wait at the barrier below
    if (tid < kCIpThreads) {
      sm_hpd_inverses<M>(sQ, sPiv, tid, p.err);
      FFCA_SMARK(it, 3);
      cluster_ip_columns<M>(sQ, sW, sB, sWc, sDet, sV, sBeta, tid, p.err);
    }
    __syncthreads();
    FFCA_SMARK(it, 4);

    // ---- U = |W^H x|^2 (Eq. 37) into TMEM; each thread later reads only its own frames
    pass_U();
    FFCA_SMARK(it, 5);

    // ---- NMF EM sweep over sources (Gauss-Seidel); pass n first applies source n-1's H
    // update and its change of sigma^2
#pragma unroll 1
    for (int n = 0; n < N; ++n) {
      float Ln[M];
#pragma unroll
      for (int m = 0; m < M; ++m) Ln[m] = sL[m * N + n];
      float acc[MP];
#pragma unroll
      for (int m = 0; m < MP; ++m) acc[m] = 0.f;
      // this source's H row for all of the thread's frames, loads in flight together
      float hrow[kSSlots];
#pragma unroll
      for (int k = 0; k < kSSlots; ++k) {
        const int t = tid + k * kSThreads;
        hrow[k] = (k < KF && t < T) ? vf[(size_t)n * T + t] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < kSSlots; ++k) {
        if (k >= KF) break;                                // uniform over the CTA
        const int t = tid + k * kSThreads;
        const float hn = hrow[k];
        float s2v[8], u[8];
        tmem_ld16(tm_s2(k), s2v, u);
        if (t < T) {
          if (n > 0) {
            float rv[8];
            r_load(t, rv);
            float g = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) g = fmaf(rv[m], coef[m], g);
            const float hold = hprev[k * kSThreads];
            const float hnew = hold * g;
            vf[(size_t)(n - 1) * T + t] = hnew;
#pragma unroll
            for (int m = 0; m < M; ++m) {
              // sigma^2 <- sigma^2 - L H + L' H', never below the new term: the rest of the sum,
              // clamped at zero, plus the new term in one fma (rounding is monotone, so this is
              // max(fma(L', H', rest), L' H') bit for bit)
              const float rest = fmaxf(fmaf(-Lold[m], hold, s2v[m]), 0.f);
              s2v[m] = fmaf(Lnew[m], hnew, rest);
            }
          }
          hprev[k * kSThreads] = hn;
          float rv[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) rv[m] = 0.f;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const float rs = fast_rcp(s2v[m]);
            const float G = Ln[m] * hn * rs;
            const float rr_ = fmaf(G, fmaf(u[m], rs, -1.f), 1.f);
            rv[m] = rr_;
            acc[m] += rr_;
          }
          r_store(t, rv);
        }
        if (n > 0) tmem_st8(tm_s2(k), s2v);
      }
      tmem_wait_st();
      // per-warp sums of r, then every warp adds the 16 warps' sums in the same order: lane
      // (m, q) adds warps q, q + 4, q + 8, q + 12, and two shuffles finish
      warp_reduce_scatter<MP>(acc, lane);
      float* rb = sRed + rpar * (kSWarps * 8);
      if ((lane * MP) % 32 == 0 && (lane * MP) / 32 < M) rb[warp * 8 + (lane * MP) / 32] = acc[0];
      __syncthreads();
      float tot_l = 0.f;
      {
        const int m = lane >> 2, q = lane & 3;
        if (m < M) {
#pragma unroll
          for (int w = q; w < kSWarps; w += 4) tot_l += rb[w * 8 + m];
        }
        tot_l += __shfl_xor_sync(0xffffffffu, tot_l, 1);
        tot_l += __shfl_xor_sync(0xffffffffu, tot_l, 2);
      }
      rpar ^= 1;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const float mean = __shfl_sync(0xffffffffu, tot_l, 4 * m) * invTf;
        Lold[m] = Ln[m];
        Lnew[m] = Ln[m] * mean;
        coef[m] = fast_rcp(mean) * (1.0f / (float)M);
      }
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (tid == m) {
          sL[m * N + n] = Lnew[m];
          sLt[n * 8 + m] = Lnew[m];
        }
      FFCA_SMARK(it, 6 + (n < 25 ? n : 25));
    }
    __syncthreads();          // sL of the last source before pass A reads it
  }

  // ---- write back the per-frequency parameters (H is already in global memory)
  __syncthreads();
  for (int i = tid; i < M * N; i += kSThreads) lamf[i] = sL[i];
  for (int i = tid; i < M * M; i += kSThreads) {
    Pf[i] = sW[i];
    p.Bst[(size_t)f * M * M + i] = sB[i];
  }
  if (tid == 0) { p.detst[2 * f] = sDet[0]; p.detst[2 * f + 1] = sDet[1]; }

  // ---- release the tensor memory once every thread's accesses are complete
  tmem_wait_st();
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(*sTmem, kSCols);
}

}  // namespace ffca

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
// MM per iteration (Eq. 15-17, App. B), the same CTA layout, both right-hand sides at the
// current parameters:
//   z_t = X_t^{-1} x_t,  h_nt <- h_nt sqrt(z^H R_n z / tr(X_t^{-1} R_n))               (Eq. 16)
//   A_n = sum_t h_nt X_t^{-1},  S_n = sum_t h_nt z z^H (old h, packed FP32 sums)
//   R_n <- A_n^{-1} # (R_n S_n R_n)   (geometric mean, one warp per source, FP64)     (Eq. 17)
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
  cudaError_t (*em)(const FcaArgs& a, FcaWork* w, cudaStream_t s);     // EM (Eq. 12-13)
  cudaError_t (*em_mm)(const FcaArgs& a, FcaWork* w, cudaStream_t s);  // MM (Eq. 15-17)
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
      // a_ik / d first: it is O(1) whatever the matrix's scale, whereas a_ik a_kj would
      // underflow for entries below ~1e-19 (a frame whose power is near zero)
      const float2 g = make_float2(A[i][k].x * rd, A[i][k].y * rd);
#pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j == k) {
          A[i][j] = make_float2(-g.x, -g.y);
        } else {
          const float2 pr = cmulf(g, rowk[j]);
          A[i][j] = make_float2(A[i][j].x - pr.x, A[i][j].y - pr.y);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
      A[k][j] = (j == k) ? make_float2(rd, 0.f) : make_float2(rowk[j].x * rd, rowk[j].y * rd);
  }
  return logdet;
}

// ---------------------------------------------------------------- FP64 M x M on one warp
// Matrices are row-major double2 in shared memory; lane e < M*M owns entry (e / M, e % M).

// C = A B (C may alias neither A nor B).
static_assert(kFcaMaxWarps <= 32, "one reduction row per warp");

// Packed Hermitian sums (FP64, the layout of unpack_herm) to a full row-major M x M matrix.
template <int M>
__device__ __forceinline__ void wm_unpack(const double* p, double2* A, int lane) {
  if (lane < M * M) {
    const int i = lane / M, j = lane - (lane / M) * M;
    if (i == j) {
      A[lane] = make_double2(p[i], 0.0);
    } else {
      const int a = i < j ? i : j, b = i < j ? j : i;
      const int k = a * M - (a * (a + 1)) / 2 + (b - a - 1);
      const double im = p[M + 2 * k + 1];
      A[lane] = make_double2(p[M + 2 * k], i < j ? im : -im);
    }
  }
  __syncwarp();
}

template <int M>
__device__ __forceinline__ void wm_mul(const double2* A, const double2* B, double2* C, int lane) {
  if (lane < M * M) {
    const int i = lane / M, j = lane - (lane / M) * M;
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < M; ++k) s = cadd(s, cmul(A[i * M + k], B[k * M + j]));
    C[lane] = s;
  }
  __syncwarp();
}

// C = A B^H.
template <int M>
__device__ __forceinline__ void wm_mul_h(const double2* A, const double2* B, double2* C, int lane) {
  if (lane < M * M) {
    const int i = lane / M, j = lane - (lane / M) * M;
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < M; ++k) s = cadd(s, cmul(A[i * M + k], make_double2(B[j * M + k].x, -B[j * M + k].y)));
    C[lane] = s;
  }
  __syncwarp();
}

// In-place inverse of an HPD matrix (Gauss-Jordan without pivoting); false if a pivot is not
// positive.
template <int M>
__device__ __forceinline__ bool wm_hpd_inverse(double2* A, int lane) {
  bool ok = true;
  for (int k = 0; k < M; ++k) {
    const double d = A[k * M + k].x;
    ok &= (d > 0.0) && isfinite(d);
    const double rd = rcp_pos_f64((d > 0.0 && isfinite(d)) ? d : 1.0);
    double2 nv = make_double2(0.0, 0.0);
    if (lane < M * M) {
      const int i = lane / M, j = lane - (lane / M) * M;
      const double2 aij = A[lane], aik = A[i * M + k], akj = A[k * M + j];
      nv = (i == k) ? ((j == k) ? make_double2(rd, 0.0) : cscale(akj, rd))
                    : ((j == k) ? cscale(aik, -rd) : csub(aij, cscale(cmul(aik, akj), rd)));
    }
    __syncwarp();
    if (lane < M * M) A[lane] = nv;
    __syncwarp();
  }
  return ok;
}

// ln d for a positive normal double: exponent field plus the FP32 log of the mantissa in
// [1, 2) (only the step size of the iteration below depends on it).
__device__ __forceinline__ float log_pos_f64(double d) {
  const long long b = __double_as_longlong(d);
  const long long e = ((b >> 52) & 0x7ff) - 1023;
  const double m = __longlong_as_double(b - e * kExpUnit);
  return (float)e * 0.693147181f + logf((float)m);
}

// In-place inverses of two HPD matrices at once: lanes [0, E) eliminate A, lanes [E, 2E) B
// (Gauss-Jordan without pivoting, E = M * M).  ldA, ldB receive ln det A, ln det B (sums of
// the pivots' logs, FP32).  False if a pivot of either is not positive.
template <int M>
__device__ __forceinline__ bool wm_hpd_inverse2(double2* A, double2* B, int lane, float& ldA, float& ldB) {
  constexpr int E = M * M;
  static_assert(2 * E <= 32, "two matrices on one warp");
  const bool act = lane < 2 * E;
  double2* X = lane < E ? A : B;
  const int l = lane < E ? lane : lane - E;
  bool ok = true;
  float ld = 0.f;
  for (int k = 0; k < M; ++k) {
    const double d = act ? X[k * M + k].x : 1.0;
    const bool good = (d > 0.0) && isfinite(d);
    ok &= good;
    const double dd = good ? d : 1.0;
    ld += log_pos_f64(dd);
    const double rd = rcp_pos_f64(dd);
    double2 nv = make_double2(0.0, 0.0);
    if (act) {
      const int i = l / M, j = l - (l / M) * M;
      const double2 aij = X[l], aik = X[i * M + k], akj = X[k * M + j];
      nv = (i == k) ? ((j == k) ? make_double2(rd, 0.0) : cscale(akj, rd))
                    : ((j == k) ? cscale(aik, -rd) : csub(aij, cscale(cmul(aik, akj), rd)));
    }
    __syncwarp();
    if (act) X[l] = nv;
    __syncwarp();
  }
  ldA = __shfl_sync(0xffffffffu, ld, 0);
  ldB = __shfl_sync(0xffffffffu, ld, E);
  return __all_sync(0xffffffffu, ok);
}

// The geometric mean G = Om1 # Om2 (after Eq. 17) of HPD matrices, by congruence:
// Om1 = L L^H (Cholesky, lane 0), C = L^-1 Om2 L^-H, G = L C^1/2 L^H, the Hermitian square
// root C^1/2 by the Denman-Beavers iteration Y <- (Y + Z^-1)/2, Z <- (Z + Y^-1)/2 from
// Y = C, Z = I (Y -> C^1/2, Z -> C^-1/2).  While det(Y) det(Z) is far from 1 the step is
// taken on (mu Y, mu Z), mu = |det Y det Z|^(-1/(2M)) (determinant scaling, Higham 1997),
// which shortens the slow first phase on ill-conditioned C; once mu is within 1e-3 of 1 the
// plain step runs, so the fixed point is exact.  Stopped once a step changes Y by less than
// 1e-11 of its largest entry (at most 40 steps).
// W holds 6 M x M scratch matrices.  Returns false on a non-positive pivot.
template <int M>
__device__ bool wm_gmean(const double2* Om1, const double2* Om2, double2* G, double2* W, int lane) {
  constexpr int E = M * M;
  double2* Lm = W;            // Cholesky factor, then its inverse
  double2* Li = W + E;
  double2* Y = W + 2 * E;
  double2* Z = W + 3 * E;
  double2* Yi = W + 4 * E;
  double2* Zi = W + 5 * E;
  bool ok = true;
  if (lane == 0) {
    for (int e = 0; e < E; ++e) { Lm[e] = make_double2(0.0, 0.0); Li[e] = make_double2(0.0, 0.0); }
    for (int k = 0; k < M; ++k) {
      double d = Om1[k * M + k].x;
      for (int q = 0; q < k; ++q) d -= Lm[k * M + q].x * Lm[k * M + q].x + Lm[k * M + q].y * Lm[k * M + q].y;
      ok &= d > 0.0 && isfinite(d);
      const double l = sqrt(d > 0.0 ? d : 1.0);
      Lm[k * M + k] = make_double2(l, 0.0);
      for (int i = k + 1; i < M; ++i) {
        double2 s = Om1[i * M + k];
        for (int q = 0; q < k; ++q)
          s = csub(s, cmul(Lm[i * M + q], make_double2(Lm[k * M + q].x, -Lm[k * M + q].y)));
        Lm[i * M + k] = cscale(s, 1.0 / l);
      }
    }
    // Li = L^-1 (lower triangular, forward substitution per column)
    for (int j = 0; j < M; ++j) {
      Li[j * M + j] = make_double2(1.0 / Lm[j * M + j].x, 0.0);
      for (int i = j + 1; i < M; ++i) {
        double2 s = make_double2(0.0, 0.0);
        for (int q = j; q < i; ++q) s = cadd(s, cmul(Lm[i * M + q], Li[q * M + j]));
        Li[i * M + j] = cscale(s, -1.0 / Lm[i * M + i].x);
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
  __syncwarp();
  wm_mul<M>(Li, Om2, Yi, lane);          // Yi = L^-1 Om2
  wm_mul_h<M>(Yi, Li, Y, lane);          // Y = L^-1 Om2 L^-H = C
  if (lane < E) {
    const int i = lane / M, j = lane - (lane / M) * M;
    Y[lane] = (i == j) ? make_double2(Y[lane].x, 0.0) : Y[lane];
    Z[lane] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  for (int it = 0; it < 40; ++it) {
    if (lane < E) { Yi[lane] = Y[lane]; Zi[lane] = Z[lane]; }
    __syncwarp();
    float ldY, ldZ;
    ok &= wm_hpd_inverse2<M>(Yi, Zi, lane, ldY, ldZ);
    const float lmu = -(ldY + ldZ) * (0.5f / (float)M);
    const double mu = fabsf(lmu) > 1e-3f ? (double)expf(lmu) : 1.0;     // warp-uniform
    const double imu = 1.0 / mu;
    double change = 0.0, size = 0.0;
    if (lane < E) {
      const double2 yn = cadd(cscale(Y[lane], 0.5 * mu), cscale(Zi[lane], 0.5 * imu));
      const double2 zn = cadd(cscale(Z[lane], 0.5 * mu), cscale(Yi[lane], 0.5 * imu));
      change = fabs(yn.x - Y[lane].x) + fabs(yn.y - Y[lane].y);
      size = fabs(yn.x) + fabs(yn.y);
      Y[lane] = yn;
      Z[lane] = zn;
    }
    __syncwarp();
    for (int off = 16; off >= 1; off >>= 1) {
      change = fmax(change, __shfl_xor_sync(0xffffffffu, change, off));
      size = fmax(size, __shfl_xor_sync(0xffffffffu, size, off));
    }
    if (!(change > 1e-11 * size)) break;             // warp-uniform
  }
  wm_mul<M>(Lm, Y, Yi, lane);            // Yi = L C^1/2
  wm_mul_h<M>(Yi, Lm, G, lane);          // G = L C^1/2 L^H
  if (lane < E) {                        // exact Hermitian symmetry
    const int i = lane / M, j = lane - (lane / M) * M;
    const double2 a = G[i * M + j], b = G[j * M + i];
    Zi[lane] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
  __syncwarp();
  if (lane < E) G[lane] = Zi[lane];
  __syncwarp();
  return ok;
}

template <int M, int N, bool MM = false>
struct FcaSmem {
  static constexpr int NE = M * M;
  static constexpr int VP = pow2_ceil(MM ? 2 * NE : NE);   // floats a frame adds to the sums
  static constexpr int kGmMats = 9;                         // M x M FP64 matrices per source
  // The X^{-1} region (floats); MM reuses it after the source loop as the geometric-mean
  // scratch, so it is at least that large.
  __host__ __device__ static size_t xi_floats(int Tp) {
    const size_t a = (size_t)NE * Tp;
    const size_t g = MM ? (size_t)N * kGmMats * NE * 4 : 0;
    return a > g ? a : g;
  }
  static size_t bytes(int threads) {
    const size_t Tp = (size_t)threads * kFcaSlots;
    size_t b = 0;
    b += sizeof(double2) * N * M * M * 3;          // sRd (FP64 R), sRid (FP64 R^{-1}), scratch
    b += sizeof(float2) * N * M * M * 2;           // sRf, sRif (FP32 copies)
    b += sizeof(float) * 2 * kFcaMaxWarps * 32;    // reduction rows
    b += sizeof(float) * kFcaMaxWarps;             // LL partials
    b += sizeof(float) * xi_floats((int)Tp);       // X^{-1} packed, [e][t]
    b += sizeof(float) * N * Tp;                   // h, [n][t]
    return b;
  }
};

template <int M, int N, bool MM>
__global__ void __launch_bounds__(kFcaMaxThreads) fca_em_kernel(FcaArgs p) {
  static_assert(M * M <= 32, "the FP64 M x M warp helpers give one entry per lane");
  using SMM = FcaSmem<M, N, MM>;
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
  float* sh = sXi + SMM::xi_floats(Tp);

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
          if constexpr (MM) {
            // z = X^{-1} x; Eq. 16 with num = z^H R z, den = tr(X^{-1} R) (R_n read from shared
            // memory: the sums below hold the registers)
            const float2* Rs = sRf + n * M * M;
            float2 z[M];
#pragma unroll
            for (int a = 0; a < M; ++a) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int b = 0; b < M; ++b) s = cfmaf(Xi[a][b], xv[b], s);
              z[a] = s;
            }
            float num = 0.f, den = 0.f;
#pragma unroll
            for (int a = 0; a < M; ++a) {
              float2 s = make_float2(0.f, 0.f);
#pragma unroll
              for (int b = 0; b < M; ++b) {
                s = cfmaf(Rs[a * M + b], z[b], s);
                den = fmaf(Xi[a][b].x, Rs[b * M + a].x, fmaf(-Xi[a][b].y, Rs[b * M + a].y, den));
              }
              num = fmaf(z[a].x, s.x, fmaf(z[a].y, s.y, num));
            }
            const float hnew = hn * sqrtf(num / den);
            ok &= (den > 0.f) && (hnew > 0.f) && (hnew < INFINITY);
            sh[n * Tp + t] = hnew;
            // A_n += h X^{-1}, S_n += h z z^H (packed, old h: Eq. 17)
#pragma unroll
            for (int e = 0; e < NE; ++e) acc[e] = fmaf(hn, Xp[e], acc[e]);
#pragma unroll
            for (int a = 0; a < M; ++a) acc[NE + a] = fmaf(hn, fmaf(z[a].x, z[a].x, z[a].y * z[a].y), acc[NE + a]);
            int e = NE + M;
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
              for (int b = a + 1; b < M; ++b) {
                acc[e] = fmaf(hn, fmaf(z[a].x, z[b].x, z[a].y * z[b].y), acc[e]);
                acc[e + 1] = fmaf(hn, fmaf(z[a].y, z[b].x, -z[a].x * z[b].y), acc[e + 1]);
                e += 2;
              }
          } else {
          // EM: B = R_n X^{-1}
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
          // h (h tr B), not h^2 tr B: h tr B is O(1) while h^2 underflows for h below ~1e-19
          const float hnew = (q + hn * (float)M - hn * (hn * trB)) * (1.0f / (float)M);
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
            const float psi = fmaf(mu[a].x, mu[a].x, mu[a].y * mu[a].y) + hn * Rn[a][a].x - hn * (hn * br.x);
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
              const float pre = mre + hn * Rn[a][b].x - hn * (hn * br.x);
              const float pim = mim + hn * Rn[a][b].y - hn * (hn * br.y);
              acc[e] = fmaf(pre, ih, acc[e]);
              acc[e + 1] = fmaf(pim, ih, acc[e + 1]);
              e += 2;
            }
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
      if (MM && tid < 2 * NE) {
        const float* red = sRed + par * kFcaMaxWarps * 32;
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += red[w * 32 + tid];
        reinterpret_cast<double*>(sScr)[n * 2 * NE + tid] = (double)s * invT;
      } else if (!MM && tid < NE) {
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
    if constexpr (MM) {
      // Eq. 17 for each source on its own warp: R_n <- A_n^{-1} # (R_n S_n R_n), the scratch
      // in the X^{-1} region (rewritten by the next iteration's first pass).
      for (int n = warp; n < N; n += nw) {
        const double* sums = reinterpret_cast<const double*>(sScr) + n * 2 * NE;
        double2* g = reinterpret_cast<double2*>(sXi) + (size_t)n * SMM::kGmMats * NE;
        double2* Om1 = g;
        double2* Om2 = g + NE;
        double2* G = g + 2 * NE;
        double2* W = g + 3 * NE;
        double2* Rd = sRd + n * NE;
        wm_unpack<M>(sums, Om1, lane);                 // A_n
        bool ok = wm_hpd_inverse<M>(Om1, lane);        // A_n^{-1}
        wm_unpack<M>(sums + NE, G, lane);              // S_n
        wm_mul<M>(Rd, G, W, lane);                     // R S
        wm_mul<M>(W, Rd, Om2, lane);                   // R S R
        ok &= wm_gmean<M>(Om1, Om2, G, W, lane);
        if (lane < NE) Rd[lane] = G[lane];
        __syncwarp();
        if (!ok && lane == 0) atomicOr(p.err, kErrFcaPivot);
      }
      __syncthreads();
    }
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

// Threads per CTA: about two frames per thread, up to kFcaMaxThreads (512 x 128 registers is
// the register file).  Shared memory (X^{-1} per frame) holds the kernel to one CTA per SM,
// so the CTA takes as many warps as fit to hide latency; kFcaSlots frames per thread still
// bound T.
inline int fca_threads(int T) {
  const int need = (T + 32 * kFcaSlots - 1) / (32 * kFcaSlots);     // warps for kFcaSlots frames each
  int warps = (T + 63) / 64;                                         // warps for two frames each
  if (warps > kFcaMaxThreads / 32) warps = kFcaMaxThreads / 32;
  if (warps < need) warps = need;
  return (warps < 1 ? 1 : warps) * 32;
}

template <int M, int N, bool MM>
cudaError_t launch_fca_em(const FcaArgs& a, FcaWork*, cudaStream_t s) {
  const int threads = fca_threads(a.T);
  if (threads > kFcaMaxThreads) return cudaErrorInvalidConfiguration;
  const size_t smem = FcaSmem<M, N, MM>::bytes(threads);
  cudaError_t e =
      cudaFuncSetAttribute(fca_em_kernel<M, N, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fca_em_kernel<M, N, MM><<<a.F, threads, smem, s>>>(a);
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
  o.em = &launch_fca_em<M, N, false>;
  o.em_mm = &launch_fca_em<M, N, true>;
  o.mwf = &launch_fca_mwf<M, N>;
  o.max_T = kFcaMaxThreads * kFcaSlots;
  return o;
}

}  // namespace ffca

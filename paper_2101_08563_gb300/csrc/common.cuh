// Shared device helpers for the FastFCA / FCA kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ffca {

// Error bits written (atomicOr) into the context's device status word.
enum ErrBits : int {
  kErrSigma = 1,       // a sigma^2 = [LH]_mt that is not finite and positive
  kErrIpNorm = 2,      // w^H Q_m w not finite and positive in the IP normalisation
  kErrQPivot = 4,      // Q_m not numerically positive definite (non-positive pivot)
  kErrWSingular = 8,   // W singular when forming W^{-H}
  kErrFcaPivot = 16,   // FCA: X_t or R_n not numerically positive definite
  kErrConfig = 32,     // launch configuration inconsistent with the problem size
};

constexpr double kLnPi = 1.1447298858494002;   // ln(pi)
constexpr double kLn2 = 0.6931471805599453;

__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float fast_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP64 reciprocal and reciprocal square root of a positive normal number.  FP64 has a
// ~70-cycle dependent latency on this part, so the seed comes from the FP32 approximation
// and one Newton-Raphson step squares its relative error (about 2^-22 -> 2^-44), far below
// the FP32 error of the sums the IP works on.  The argument is first scaled by a power of two
// into [1, 2) (reciprocal) or [1, 4) (reciprocal square root) with integer operations on its
// exponent field, so the FP32 seed is always in range and no slow path exists; the result
// is scaled back the same way.  Callers pass positive normal values only.
constexpr long long kExpUnit = 1LL << 52;                          // one step of the exponent field

__device__ __forceinline__ double rcp_pos_f64(double d) {
  const long long b = __double_as_longlong(d);
  const long long e = ((b >> 52) & 0x7ff) - 1023;                 // d = m * 2^e, m in [1, 2)
  const long long shift = e * kExpUnit;
  const double m = __longlong_as_double(b - shift);
  const double r0 = (double)fast_rcp((float)m);
  const double r1 = fma(r0, fma(-m, r0, 1.0), r0);                 // 1/m in (0.5, 1]
  return __longlong_as_double(__double_as_longlong(r1) - shift);
}

__device__ __forceinline__ double rsqrt_pos_f64(double s) {
  const long long b = __double_as_longlong(s);
  const long long e = ((b >> 52) & 0x7ff) - 1023;
  const long long k = e >> 1;                                      // s = m * 4^k, m in [1, 4)
  const double m = __longlong_as_double(b - 2 * k * kExpUnit);
  const double y0 = (double)fast_rsqrt((float)m);
  const double y1 = fma(0.5 * y0, fma(-m * y0, y0, 1.0), y0);      // 1/sqrt(m) in (0.5, 1]
  return __longlong_as_double(__double_as_longlong(y1) - k * kExpUnit);
}

// ---------------------------------------------------------------------- complex helpers
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + conj(a) * b
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfmaf(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

// ---------------------------------------------------------------------- reductions
__host__ __device__ constexpr int pow2_ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Butterfly reduce-scatter of VP (a power of two) per-lane values over a warp.  On return
// lane l holds in v[i], i < max(VP/32, 1), the warp total of value index (l*VP)/32 + i.
// Costs VP-1 shuffles (VP <= 32) instead of 5*VP for VP separate all-reductions.
template <int VP>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[VP], int lane) {
  static_assert((VP & (VP - 1)) == 0, "VP must be a power of two");
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int off = 16 >> lvl;
    const int cnt = (VP >> lvl) > 1 ? (VP >> lvl) : 1;
    if (cnt > 1) {
      const int half = cnt / 2;
      const bool upper = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const float send = upper ? v[i] : v[i + half];
        const float keep = upper ? v[i + half] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Keeps a positive double product as mantissa * 2^exponent (mantissa in [0.5, 1)) so that
// M updates per iteration over many iterations can neither overflow nor underflow.  Integer
// operations on the bit pattern only (normal numbers; others are left unchanged).
__device__ __forceinline__ void renorm(double& mant, double& expo) {
  const long long b = __double_as_longlong(mant);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0 || e == 0x7ff) return;
  expo += (double)(e - 1022);
  mant = __longlong_as_double((b & ~(0x7ffLL << 52)) | (1022LL << 52));
}

}  // namespace ffca

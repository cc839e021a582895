// Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11,
// "Parallel random numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64-bit
// multiplications with Weyl key bumps.  Callable on the host and the device so that the
// published known-answer vectors can be checked on the CPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ffca {

struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = mulhi32(M1, c.z), lo1 = M1 * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// Uniform in (0, 1) from 32 random bits (never 0, so ln() is finite): 23 bits plus a half
// step, so the largest value, 1 - 2^-24, is still below 1 in FP32.
__host__ __device__ __forceinline__ float u01(uint32_t b) { return ((float)(b >> 9) + 0.5f) * (1.0f / 8388608.0f); }

}  // namespace ffca

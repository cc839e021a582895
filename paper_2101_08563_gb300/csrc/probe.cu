// Entry points that measure or check the machine rather than run the method: the FP32 FMA
// rate of the GPU (the denominator of the arithmetic roofline the benchmark reports) and the
// library's FP64 reciprocal helpers used by the IP (so a test can hold them against CUDA's
// own division and square root).
#include <cuda_runtime.h>

#include "../../include/fastfca.h"
#include "alloc.h"
#include "common.cuh"
#include "launch.cuh"

namespace {

// Eight independent FMA chains per thread; the result is written so nothing is removed.
__global__ void __launch_bounds__(512) fp32_fma_kernel(float* out, int iters) {
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1.0f + 1e-3f * (float)(threadIdx.x + j);
  const float b = 0.999999f, c = 1e-7f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void f64_reciprocals_kernel(const double* __restrict__ x, double* __restrict__ rcp,
                                       double* __restrict__ rsq, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    rcp[i] = ffca::rcp_pos_f64(x[i]);
    rsq[i] = ffca::rsqrt_pos_f64(x[i]);
  }
}

}  // namespace

extern "C" fastfca_status fastfca_measure_fp32_fma(int32_t iters, double* tflops, void* stream) {
  if (iters < 1 || !tflops) {
    ffca::set_thread_error("iters must be positive and tflops non-null");
    return FASTFCA_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    ffca::set_thread_error("device query failed");
    return FASTFCA_ECUDA;
  }
  const int threads = 512, blocks = 4 * sms;        // 2048 resident threads per SM
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = ffca::dev_malloc(&out, sizeof(float) * (size_t)threads * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    fp32_fma_kernel<<<blocks, threads, 0, s>>>(out, iters);            // warm-up
    cudaEventRecord(e0, s);
    fp32_fma_kernel<<<blocks, threads, 0, s>>>(out, iters);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) ffca::dev_free(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ffca::set_thread_error(cudaGetErrorString(e));
    return FASTFCA_ECUDA;
  }
  const double flops = 2.0 * 8 * 16 * (double)iters * threads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return FASTFCA_OK;
}

extern "C" fastfca_status fastfca_debug_f64_reciprocals(int32_t n, const double* x, double* rcp, double* rsqrt,
                                                        void* stream) {
  if (n < 1 || !x || !rcp || !rsqrt) {
    ffca::set_thread_error("n must be positive and x, rcp, rsqrt non-null");
    return FASTFCA_EINVAL;
  }
  f64_reciprocals_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, rcp, rsqrt, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ffca::set_thread_error(cudaGetErrorString(e));
    return FASTFCA_ECUDA;
  }
  return FASTFCA_OK;
}

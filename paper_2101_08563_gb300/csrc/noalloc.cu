// fastfca_separate_noalloc: the Wiener-filter separation for callers that must not allocate.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where they separate a
// block of audio: a real-time audio callback, for one, has a fixed deadline, and an
// allocation may block the thread or synchronise the whole device.  This entry point runs
// the same two kernels as fastfca_separate (W^{-H} per frequency, then the filter) with
// every input and output supplied by the caller, and keeps the one intermediate it needs
// (W^{-H} as complex64, F*M*M values) in a fixed-size array compiled into the library.
//
// The array lives in device memory of every GPU that loads the library, until the process
// exits.  Its address is looked up once per device (cudaGetSymbolAddress, with that device
// current) on the first call made on that device: make that first call before any stream
// capture.  The address is kept for the life of the process, so the entry point must not be
// used on a device after cudaDeviceReset (the reset destroys the array with the context).
// The filter is chosen by (M, N) alone: it has no frame limit, whatever the EM kernels'.
// All calls share the array and it keeps the last call's contents, so calls that overlap on
// the GPU (on different streams, or from different host threads) race on it.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/fastfca.h"
#include "launch.cuh"
#include "trace.h"

namespace {

// 256 bytes of status word (error bits of the W^{-H} kernel), then the W^{-H} values.
constexpr int kStatusSlots = 32;                       // float2 slots reserved for the status
constexpr int kNoAllocMaxWinv = FASTFCA_NOALLOC_MAX_FMM;
static __device__ __align__(256) float2 g_noalloc_scratch[kStatusSlots + kNoAllocMaxWinv];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float2* g_scratch_addr[kMaxDevices] = {};

// Messages go where fastfca_last_error(NULL) reads them (the calling thread's slot).
fastfca_status noalloc_fail(fastfca_status st, const char* msg) {
  ffca::set_thread_error(msg);
  return st;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" fastfca_status fastfca_separate_noalloc(int32_t F, int32_t T, int32_t M, int32_t N,
                                                   const void* x, const void* P, const float* lam,
                                                   const float* v, void* c, void* stream) {
  FFCA_TRACE("fastfca_separate_noalloc");
  if (F < 1 || T < 1 || M < 1 || N < 1) return noalloc_fail(FASTFCA_EINVAL, "F, T, M, N must be positive");
  ffca::FastOps ops{};
  if (!ffca::filter_ops(M, N, &ops)) return noalloc_fail(FASTFCA_EUNSUPPORTED, "no kernel for this (M, N)");
  if ((long long)F * M * M > kNoAllocMaxWinv) {
    char msg[256];
    snprintf(msg, sizeof msg, "F*M*M = %lld exceeds the %d complex values of the static scratch",
             (long long)F * M * M, kNoAllocMaxWinv);
    return noalloc_fail(FASTFCA_EINVAL, msg);
  }
  if (!x || !P || !lam || !v || !c) return noalloc_fail(FASTFCA_EINVAL, "x, P, lam, v and c are required");
  // the kernels load x and P as 16-byte vectors, store c as 8-byte complex values and read
  // lam and v as floats: checked before anything touches the GPU
  if (reinterpret_cast<uintptr_t>(x) % 16 != 0 || reinterpret_cast<uintptr_t>(P) % 16 != 0)
    return noalloc_fail(FASTFCA_EINVAL, "x and P must start on a 16-byte boundary");
  if (reinterpret_cast<uintptr_t>(c) % 8 != 0)
    return noalloc_fail(FASTFCA_EINVAL, "c must start on an 8-byte boundary");
  if (reinterpret_cast<uintptr_t>(lam) % 4 != 0 || reinterpret_cast<uintptr_t>(v) % 4 != 0)
    return noalloc_fail(FASTFCA_EINVAL, "lam and v must start on a 4-byte boundary");
  if (!device_pointer(x) || !device_pointer(P) || !device_pointer(lam) || !device_pointer(v) || !device_pointer(c))
    return noalloc_fail(FASTFCA_EINVAL, "x, P, lam, v and c must be device pointers");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(FASTFCA_ECUDA, "cudaGetDevice failed or device index out of range");
  float2* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) {
        cudaGetLastError();
        return noalloc_fail(FASTFCA_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      g_scratch_addr[dev] = static_cast<float2*>(addr);
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(base);
  float2* winv = base + kStatusSlots;
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(FASTFCA_ECUDA, "status clear failed");
  }
  cudaError_t e = ops.winv(static_cast<const double2*>(P), winv, F, status, s);
  if (e == cudaSuccess)
    e = ops.mwf(static_cast<const float2*>(x), static_cast<const double2*>(P), winv, lam, v,
                static_cast<float2*>(c), F, T, N, 1, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(FASTFCA_ECUDA, cudaGetErrorString(e));
  }
  return FASTFCA_OK;
}

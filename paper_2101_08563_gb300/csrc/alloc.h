// Device memory of contexts, batches and networks.  Every allocation the library makes goes
// through dev_malloc / dev_malloc_async and is released by dev_free / dev_free_async, which
// keep a count of the live allocations.  A host-side countdown (fastfca_debug_fail_alloc) can
// make one chosen allocation fail as an out-of-memory would: fault injection for the error
// paths, decided on the host before anything reaches the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace ffca {

cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p);                          // no-op for nullptr
void dev_free_async(void* p, cudaStream_t s);    // no-op for nullptr

template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

template <class T>
inline cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t s) {
  return dev_malloc_async_raw(reinterpret_cast<void**>(p), bytes, s);
}

}  // namespace ffca

// Host-side launchers for one (M, N) specialisation of the FastFCA kernels.
#pragma once
#include "fastfca_em.cuh"
#include "fastfca_mwf.cuh"

namespace ffca {

struct FastOps {
  cudaError_t (*em)(const EmArgs& a, cudaStream_t s);
  cudaError_t (*winv)(const double2* P, float2* WmH, int F, int* err, cudaStream_t s);
  cudaError_t (*mwf)(const float2* x, const double2* P, const float2* WmH, const float* lam,
                     const float* v, float2* c, int F, int T, cudaStream_t s);
  // persistent batch form: items in device memory, `bd` threads per CTA, `grid` CTAs
  cudaError_t (*em_persistent)(const EmItem* items, int n_items, int n_iter, int* counter, int* err, int bd,
                               int grid, cudaStream_t s);
  size_t (*em_smem)(int bd);
  int (*em_blocks_per_sm)(int bd);
  int max_T;
};

// Threads for a frequency of T frames: whole warps, kSlots frames each.
inline int em_threads(int T) {
  const int warps = (T + 32 * kSlots - 1) / (32 * kSlots);
  return (warps < 1 ? 1 : warps) * 32;
}

template <int M, int N>
cudaError_t launch_em(const EmArgs& a, cudaStream_t s) {
  const int threads = em_threads(a.T);
  if (threads > kMaxThreads) return cudaErrorInvalidConfiguration;
  const size_t smem = EmSmem<M, N>::bytes(threads);
  cudaError_t e = cudaFuncSetAttribute(fastfca_em_kernel<M, N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fastfca_em_kernel<M, N><<<a.F, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int M, int N>
cudaError_t launch_em_persistent(const EmItem* items, int n_items, int n_iter, int* counter, int* err, int bd,
                                 int grid, cudaStream_t s) {
  if (bd > kMaxThreads || bd % 32 != 0) return cudaErrorInvalidConfiguration;
  const size_t smem = EmSmem<M, N>::bytes(bd);
  cudaError_t e = cudaFuncSetAttribute(fastfca_em_persistent_kernel<M, N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fastfca_em_persistent_kernel<M, N><<<grid, bd, smem, s>>>(items, n_items, n_iter, counter, err);
  return cudaGetLastError();
}

template <int M, int N>
size_t em_smem_bytes(int bd) {
  return EmSmem<M, N>::bytes(bd);
}

template <int M, int N>
int em_blocks_per_sm(int bd) {
  const size_t smem = EmSmem<M, N>::bytes(bd);
  if (cudaFuncSetAttribute(fastfca_em_persistent_kernel<M, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fastfca_em_persistent_kernel<M, N>, bd, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

template <int M>
cudaError_t launch_winv(const double2* P, float2* WmH, int F, int* err, cudaStream_t s) {
  winv_kernel<M><<<F, 32, 0, s>>>(P, WmH, F, err);
  return cudaGetLastError();
}

template <int M, int N>
cudaError_t launch_mwf(const float2* x, const double2* P, const float2* WmH, const float* lam,
                       const float* v, float2* c, int F, int T, cudaStream_t s) {
  dim3 grid(F, (T + kMwfThreads - 1) / kMwfThreads);
  fastfca_mwf_kernel<M, N><<<grid, kMwfThreads, 0, s>>>(x, P, WmH, lam, v, c, F, T);
  return cudaGetLastError();
}

template <int M, int N>
FastOps make_fast_ops() {
  FastOps o;
  o.em = &launch_em<M, N>;
  o.winv = &launch_winv<M>;
  o.mwf = &launch_mwf<M, N>;
  o.em_persistent = &launch_em_persistent<M, N>;
  o.em_smem = &em_smem_bytes<M, N>;
  o.em_blocks_per_sm = &em_blocks_per_sm<M, N>;
  o.max_T = kMaxThreads * kSlots;
  return o;
}

// Records a message for fastfca_last_error(NULL) on the calling thread (api.cu).
void set_thread_error(const char* msg);

// Defined in the per-M translation units.
bool fast_ops_m2(int N, FastOps* o);
bool fast_ops_m3(int N, FastOps* o);
bool fast_ops_m4(int N, FastOps* o);

inline bool fast_ops(int M, int N, FastOps* o) {
  switch (M) {
    case 2: return fast_ops_m2(N, o);
    case 3: return fast_ops_m3(N, o);
    case 4: return fast_ops_m4(N, o);
    default: return false;
  }
}

}  // namespace ffca

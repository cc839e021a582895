// Host-side launchers for one (M, N) specialisation of the FastFCA kernels.
#pragma once
#include "fastfca_em.cuh"
#include "fastfca_em_cluster.cuh"
#include "fastfca_em_sm.cuh"
#include "fastfca_mwf.cuh"

namespace ffca {

struct FastOps {
  cudaError_t (*em)(const EmArgs& a, cudaStream_t s);
  cudaError_t (*em_mm)(const EmArgs& a, cudaStream_t s);   // IP+MM (Algorithm 2); null if none
  // piecewise-stationary input (Sec. VI-B): a.xh holds the packed block statistics, a.T counts
  // blocks; null if none
  cudaError_t (*em_blk)(const EmArgs& a, cudaStream_t s);
  cudaError_t (*em_mm_blk)(const EmArgs& a, cudaStream_t s);
  cudaError_t (*block_stats)(const float2* x, float* xh, int F, int J, int B, cudaStream_t s);
  cudaError_t (*winv)(const double2* P, float2* WmH, int F, int* err, cudaStream_t s);
  // B: frames per block of v (1 = per frame; frame t reads v column t / B)
  cudaError_t (*mwf)(const float2* x, const double2* P, const float2* WmH, const float* lam,
                     const float* v, float2* c, int F, int T, int N, int B, cudaStream_t s);
  // persistent batch form: items in device memory, `bd` threads per CTA, `grid` CTAs; [0] IP+EM
  // (Algorithm 1), [1] IP+MM (Algorithm 2)
  cudaError_t (*em_persistent[2])(const EmItem* items, int n_items, int n_iter, int* counter, int* err, int bd,
                                  int grid, cudaStream_t s);
  size_t (*em_smem)(int bd);
  int (*em_blocks_per_sm[2])(int bd);
  int max_T;
  bool cluster;          // the cluster kernel (any T it fits, runtime N); no batch form
  int cluster_c;         // the cluster kernel's CTAs per frequency for this shape (0: not cluster)
};

// Threads for a frequency of T frames: whole warps, kSlots frames each.
inline int em_threads(int T) {
  const int warps = (T + 32 * kSlots - 1) / (32 * kSlots);
  return (warps < 1 ? 1 : warps) * 32;
}

// Dynamic shared memory for the IP+EM kernel with sigma^2 in tensor memory: at least its
// layout's, and enough more that the CTAs one SM holds at once never ask for more than the
// SM's 512 TMEM columns together (32 columns per CTA up to four warps, 64 above), so no
// allocation ever waits.  0 when that cannot be arranged.
// The kernel's dynamic shared memory limit is set once to the device's opt-in maximum (a
// permission, not a reservation: occupancy follows the size each launch asks for), so that
// launches of one instantiation with different sizes, captured in one graph, never see a
// lower limit than they were made with.
template <typename Kernel>
size_t em_tm_smem(Kernel kernel, int threads, size_t smem) {
  const int cap = 512 / (threads > 128 ? 64 : 32);
  int dev = 0, per_sm_smem = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || fa.sharedSizeBytes >= (size_t)optin) return 0;
  const int max_dyn = optin - (int)fa.sharedSizeBytes;      // the limit counts dynamic bytes only
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn) != cudaSuccess) return 0;
  for (size_t dyn = smem; dyn <= (size_t)std::min(per_sm_smem, max_dyn); dyn += 1024) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, dyn) != cudaSuccess) return 0;
    if (nb >= 1 && nb <= cap) return dyn;
  }
  return 0;
}

template <int M, int N, bool MM = false, bool BL = false>
cudaError_t launch_em(const EmArgs& a, cudaStream_t s) {
  const int threads = em_threads(a.T);
  if (threads > kMaxThreads) return cudaErrorInvalidConfiguration;
  if (BL && !a.xh) return cudaErrorInvalidValue;
  const size_t smem = EmSmem<M, N>::bytes(threads);
  if constexpr (!MM) {
    // IP+EM keeps sigma^2 in tensor memory (the n-loop then updates it by each source's change)
    const size_t dyn = em_tm_smem(fastfca_em_kernel<M, N, false, BL, true>, threads, smem);
    if (dyn == 0) return cudaErrorInvalidConfiguration;
    fastfca_em_kernel<M, N, false, BL, true><<<a.F, threads, dyn, s>>>(a);
    return cudaGetLastError();
  } else {
    cudaError_t e = cudaFuncSetAttribute(fastfca_em_kernel<M, N, MM, BL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fastfca_em_kernel<M, N, MM, BL><<<a.F, threads, smem, s>>>(a);
    return cudaGetLastError();
  }
}

template <int M>
cudaError_t launch_block_stats(const float2* x, float* xh, int F, int J, int B, cudaStream_t s) {
  const size_t n = (size_t)F * J;
  block_stats_kernel<M><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, xh, F, J, B);
  return cudaGetLastError();
}

template <int M, int N, bool MM>
cudaError_t launch_em_persistent(const EmItem* items, int n_items, int n_iter, int* counter, int* err, int bd,
                                 int grid, cudaStream_t s) {
  if (bd > kMaxThreads || bd % 32 != 0) return cudaErrorInvalidConfiguration;
  const size_t smem = EmSmem<M, N>::bytes(bd);
  cudaError_t e = cudaFuncSetAttribute(fastfca_em_persistent_kernel<M, N, MM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fastfca_em_persistent_kernel<M, N, MM><<<grid, bd, smem, s>>>(items, n_items, n_iter, counter, err);
  return cudaGetLastError();
}

template <int M, int N>
size_t em_smem_bytes(int bd) {
  return EmSmem<M, N>::bytes(bd);
}

template <int M, int N, bool MM>
int em_blocks_per_sm(int bd) {
  const size_t smem = EmSmem<M, N>::bytes(bd);
  if (cudaFuncSetAttribute(fastfca_em_persistent_kernel<M, N, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fastfca_em_persistent_kernel<M, N, MM>, bd, smem) !=
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
                       const float* v, float2* c, int F, int T, int /*N*/, int B, cudaStream_t s) {
  if (B < 1 || T % B != 0) return cudaErrorInvalidValue;
  dim3 grid(F, (T + kMwfThreads * kMwfBatches - 1) / (kMwfThreads * kMwfBatches));
  fastfca_mwf_kernel<M, N><<<grid, kMwfThreads, 0, s>>>(x, P, WmH, lam, v, c, F, T, B);
  return cudaGetLastError();
}

template <int M, int N>
FastOps make_fast_ops() {
  FastOps o;
  o.em = &launch_em<M, N>;
  o.em_mm = &launch_em<M, N, true>;
  o.em_blk = &launch_em<M, N, false, true>;
  o.em_mm_blk = &launch_em<M, N, true, true>;
  o.block_stats = &launch_block_stats<M>;
  o.winv = &launch_winv<M>;
  o.mwf = &launch_mwf<M, N>;
  o.em_persistent[0] = &launch_em_persistent<M, N, false>;
  o.em_persistent[1] = &launch_em_persistent<M, N, true>;
  o.em_smem = &em_smem_bytes<M, N>;
  o.em_blocks_per_sm[0] = &em_blocks_per_sm<M, N, false>;
  o.em_blocks_per_sm[1] = &em_blocks_per_sm<M, N, true>;
  o.max_T = kMaxThreads * kSlots;
  o.cluster = false;
  o.cluster_c = 0;
  return o;
}

// ---------------------------------------------------------------- cluster kernel (large bins)
// Spins a cluster exchange of the cluster kernel waits before it reports a time-out (0: the
// kernel's default).  Host state, set by fastfca_debug_cluster_wait_limit (fastfca_sm.cu).
int cluster_wait_limit();

// Shared memory available to one CTA, alone on an SM or as one of two.
constexpr size_t kSmemOnePerSm = 227 * 1024;
constexpr size_t kSmemTwoPerSm = 113 * 1024;

// Cluster size C for T frames and N sources: the smallest C in {1, 2, 4, 8} (with C <= T)
// whose CTAs fit two per SM, else the smallest that fits one per SM.  False if none fits.
template <int M>
bool cluster_shape(int T, int N, int* C, size_t* smem) {
  if (N < 1 || N > kCMaxN || T < 1) return false;
  for (size_t cap : {kSmemTwoPerSm, kSmemOnePerSm}) {
    for (int c = 1; c <= kCMaxCluster; c *= 2) {
      const int Tc = (T + c - 1) / c;
      if ((c - 1) * Tc >= T) break;                  // every CTA must own a frame
      const size_t b = ClusterSmem<M>::bytes(N, Tc);
      if (b <= cap) { *C = c; *smem = b; return true; }
    }
  }
  return false;
}

template <int M, bool MM = false, bool BL = false>
cudaError_t launch_em_cluster(const EmArgs& a, cudaStream_t s) {
  int C = 0;
  size_t smem = 0;
  if (!cluster_shape<M>(a.T, a.N, &C, &smem)) return cudaErrorInvalidConfiguration;
  if (BL && !a.xh) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fastfca_em_cluster_kernel<M, MM, BL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.F * C), 1, 1);
  cfg.blockDim = dim3(kCThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ClusterArgs ca{a, nullptr, nullptr, cluster_wait_limit()};
  e = cudaLaunchKernelEx(&cfg, fastfca_em_cluster_kernel<M, MM, BL>, ca);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The one-SM IP+EM kernel (fastfca_em_sm.cuh): one CTA of kSThreads per frequency.
template <int M>
cudaError_t launch_em_sm(const EmArgs& a, cudaStream_t s) {
  if (a.T < 1 || a.T > kSMaxT || a.N < 1 || a.N > kCMaxN) return cudaErrorInvalidConfiguration;
  const size_t smem = SmSmem<M>::bytes;
  cudaError_t e = cudaFuncSetAttribute(fastfca_em_sm_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fastfca_em_sm_kernel<M><<<a.F, kSThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Which kernel takes IP+EM for the large-bin shapes: 0 picks by shape (below), 1 forces the
// cluster kernel, 2 the one-SM kernel where it fits.  Host state, set by
// fastfca_debug_large_bin_kernel (for tests that cover both kernels on one shape).
int large_bin_kernel_choice();

// The one-SM IP+EM launcher for M (null if not built for that M) (fastfca_sm.cu).
using EmLaunch = cudaError_t (*)(const EmArgs&, cudaStream_t);
EmLaunch sm_em_launcher(int M);

// Gives IP+EM on a large-bin shape to the one-SM kernel where it fits (T <= kSMaxT) and the
// cluster kernel would spread a frequency over two or more CTAs (at fewer frames two cluster
// CTAs share an SM, i.e. two frequencies per SM, against one for the one-SM kernel).  The
// other models and the block input stay on the cluster kernel.
inline void prefer_sm_kernel(int M, int N, int T, FastOps* o) {
  const int choice = large_bin_kernel_choice();
  if (choice == 1 || T > kSMaxT || N < 1 || N > kCMaxN) return;
  const EmLaunch fn = sm_em_launcher(M);
  if (!fn) return;
  if (choice == 2 || o->cluster_c >= 2) o->em = fn;
}

// One persistent wave: as many CTAs as fit on every SM at once, so that each warp's range of
// tiles is the same length.
template <int M>
cudaError_t launch_mwf_wide(const float2* x, const double2* P, const float2* WmH, const float* lam, const float* v,
                            float2* c, int F, int T, int N, int B, cudaStream_t s) {
  if (N < 1 || N > kMwfWMaxN || B < 1 || T % B != 0) return cudaErrorInvalidValue;
  if (F < 1 || T < 1) return cudaSuccess;
  const size_t smem = mwf_tile_smem(M, N);
  cudaError_t e = cudaFuncSetAttribute(fastfca_mwf_tile_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fastfca_mwf_tile_kernel<M>, kMwfTThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long tiles = (long long)F * ((T + mwf_tile_frames(M) - 1) / mwf_tile_frames(M));
  const long long ctas = std::min<long long>((long long)sms * per_sm, (tiles + kMwfTWarps - 1) / kMwfTWarps);
  fastfca_mwf_tile_kernel<M><<<(unsigned)ctas, kMwfTThreads, smem, s>>>(x, P, WmH, lam, v, c, F, T, N, B);
  return cudaGetLastError();
}

template <int M>
FastOps make_cluster_ops() {
  FastOps o{};
  o.em = &launch_em_cluster<M, false, false>;
  o.em_mm = &launch_em_cluster<M, true, false>;
  o.em_blk = &launch_em_cluster<M, false, true>;
  o.em_mm_blk = &launch_em_cluster<M, true, true>;
  o.block_stats = &launch_block_stats<M>;
  o.winv = &launch_winv<M>;
  o.mwf = &launch_mwf_wide<M>;
  o.em_persistent[0] = nullptr;
  o.em_persistent[1] = nullptr;
  o.em_smem = nullptr;
  o.em_blocks_per_sm[0] = nullptr;
  o.em_blocks_per_sm[1] = nullptr;
  o.max_T = 0;                     // set by cluster_ops for the N at hand
  o.cluster = true;
  o.cluster_c = 0;                 // set by cluster_ops
  return o;
}

// Records a message for fastfca_last_error(NULL) on the calling thread (api.cu).
void set_thread_error(const char* msg);

// Defined in the per-M translation units.
bool fast_ops_m2(int N, FastOps* o);
bool fast_ops_m3(int N, FastOps* o);
bool fast_ops_m4(int N, FastOps* o);
// Cluster-kernel ops for M in 2..8 and N in 1..kCMaxN when T frames fit (fastfca_cluster_*.cu).
bool cluster_ops(int M, int N, int T, FastOps* o);

inline bool fast_ops(int M, int N, FastOps* o) {
  switch (M) {
    case 2: return fast_ops_m2(N, o);
    case 3: return fast_ops_m3(N, o);
    case 4: return fast_ops_m4(N, o);
    default: return false;
  }
}

// The Wiener-filter kernels (winv, mwf) for (M, N): the frequency-resident filter where the
// frequency-resident kernels exist, else the wide filter.  Neither filter limits T, so the
// wide filter's ops are taken for a one-frame shape, which every cluster shape holds.
inline bool filter_ops(int M, int N, FastOps* o) {
  if (fast_ops(M, N, o)) return true;
  return cluster_ops(M, N, 1, o);
}

// The kernels for one FastFCA problem: the frequency-resident kernel where it applies
// (M <= 4, N <= 8, T <= 2048), else the cluster kernel (M <= 8, N <= 16, T up to what eight
// CTAs hold).
inline bool fast_ops_for(int M, int N, int T, FastOps* o) {
  if (fast_ops(M, N, o) && T <= o->max_T) return true;
  return cluster_ops(M, N, T, o);
}

}  // namespace ffca

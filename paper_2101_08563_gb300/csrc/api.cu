// C ABI of libfastfca.so (declared in include/fastfca.h): argument checking, buffer
// ownership, host/device transfers and kernel dispatch.  All arithmetic of the method runs in
// the kernels; this file only moves data and launches.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fastfca.h"
#include "alloc.h"
#include "fca.cuh"
#include "fastmnmf.cuh"
#include "init.cuh"
#include "launch.cuh"
#include "trace.h"

namespace {

constexpr int kMaxM = 8;
constexpr int kMaxN = 16;

thread_local char g_create_error[512] = "";

}  // namespace

namespace ffca {
void set_thread_error(const char* msg) { snprintf(g_create_error, sizeof g_create_error, "%s", msg); }

std::atomic<long long> g_fail_countdown{-1};   // allocations left before the injected failure
std::atomic<long long> g_live_allocs{0};

namespace {
// True for the one allocation the armed countdown selects (and disarms it).
bool injected_failure() {
  long long c = g_fail_countdown.load();
  while (c >= 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}
}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  g_live_allocs.fetch_sub(1);
}

void dev_free_async(void* p, cudaStream_t s) {
  if (!p) return;
  cudaFreeAsync(p, s);
  g_live_allocs.fetch_sub(1);
}
}  // namespace ffca

struct fastfca_ctx {
  fastfca_config cfg{};          // cfg.T counts the parameter columns: frames, or blocks
  int Tf = 0;                    // frames of the mixture
  int B = 1;                     // frames per block (Sec. VI-B); 1 = frame-wise model
  cudaStream_t stream = nullptr;
  const float2* x = nullptr;     // device mixture (borrowed or owned), F x Tf x M
  float2* x_owned = nullptr;
  float* xh = nullptr;           // blocks: packed X^_j, F x cfg.T x M^2
  // FastFCA parameters
  double2* P = nullptr;
  float* lam = nullptr;
  float* v = nullptr;
  float2* winv = nullptr;        // W^{-H} complex64 scratch for the filter
  float2* c_stage = nullptr;     // device staging of a separation into a host c (made on first use)
  double2* Bst = nullptr;        // W^{-H} (FP64) carried between FastFCA launches
  double* detst = nullptr;       // |det W|^2 as (mantissa, exponent) per frequency
  int b_valid = 0;               // Bst/detst match the current P
  // FastMNMF parameters (P, lam, Bst, detst, winv as above; v holds h = t v for the filter)
  int K = 0;
  float* tb = nullptr;           // F x N x K bases
  float* va = nullptr;           // N x K x T activations
  float* ab = nullptr;           // 2 x F x N x T per-bin terms of the t and v updates
  float* ubuf = nullptr;         // F x M x T: U of the current W
  float* mscratch = nullptr;     // F + T + 1 floats (default start)
  int h_valid = 0;               // v (the h buffer) holds t va of the current t and va
  ffca::MnmfOps mops{};
  // FCA parameters
  double2* R = nullptr;
  float* h = nullptr;
  ffca::FcaWork fca{};
  // log-likelihood
  double* ll_hist = nullptr;     // F x ll_cap
  int ll_cap = 0;
  double* ll_last = nullptr;     // F
  double* ll_sum = nullptr;      // ll_cap totals (device)
  int* err = nullptr;
  ffca::FastOps ops{};
  ffca::FcaOps fops{};
  fastfca_status sticky = FASTFCA_OK;
  char msg[512] = "";
};

namespace {

fastfca_status fail(fastfca_ctx* c, fastfca_status st, const char* fmt, ...) {
  char* dst = c ? c->msg : g_create_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  if (c && st == FASTFCA_ECUDA) c->sticky = st;
  return st;
}

fastfca_status cuda_fail(fastfca_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, FASTFCA_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(c, FASTFCA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(c, expr, what)                               \
  do {                                                  \
    cudaError_t e__ = (expr);                           \
    if (e__ != cudaSuccess) return cuda_fail(c, e__, what); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from src (host or device) to device dst on the stream.
cudaError_t to_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (is_device_ptr(src)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);   // the host buffer may be reused after return
}

cudaError_t from_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (is_device_ptr(dst)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

size_t FT(const fastfca_config& c) { return (size_t)c.F * c.T; }

// The FastFCA model, fitted by IP+EM (Algorithm 1) or IP+MM (Algorithm 2): the same parameters.
bool fastfca_family(int model) { return model == FASTFCA_MODEL_FASTFCA || model == FASTFCA_MODEL_FASTFCA_MM; }
// The full-rank FCA model, fitted by EM (Eq. 12-13) or MM (Eq. 15-17).
bool fca_family(int model) { return model == FASTFCA_MODEL_FCA || model == FASTFCA_MODEL_FCA_MM; }

fastfca_status check_ready(fastfca_ctx* c) {
  if (!c) return FASTFCA_EINVAL;
  if (c->sticky == FASTFCA_ECUDA) return c->sticky;
  return FASTFCA_OK;
}

// check_ready for the calls that run the model: after a numerical failure the parameters
// may hold NaN or Inf, so no kernel starts from them until set_params replaces them.
fastfca_status check_params_usable(fastfca_ctx* c) {
  fastfca_status st = check_ready(c);
  if (st) return st;
  if (c->sticky == FASTFCA_ENUMERIC)
    return fail(c, FASTFCA_ENUMERIC,
                "the parameters are unusable after a numerical failure; set_params replaces them");
  return FASTFCA_OK;
}

// Reads and clears the device status word; maps set bits to ENUMERIC.
fastfca_status collect_device_status(fastfca_ctx* c) {
  int bits = 0;
  CK(c, cudaMemcpyAsync(&bits, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
  CK(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  if (bits == 0) return FASTFCA_OK;
  CK(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "status clear");
  if (bits & (ffca::kErrConfig | ffca::kErrClusterWait))
    return fail(c, FASTFCA_ECUDA, "kernel launch configuration rejected or a cluster exchange timed out (bits 0x%x)", bits);
  c->sticky = FASTFCA_ENUMERIC;
  return fail(c, FASTFCA_ENUMERIC,
              "numerical failure in a kernel (bits 0x%x: 1 sigma^2, 2 IP norm, 4 Q not PD, 8 W singular, 16 FCA not PD)",
              bits);
}

// W^{-H} for the filter from the FP64 inverse the IP keeps (B = W^{-H}, maintained by
// rank-one updates), rounded to complex64: replaces a fresh pivoted inversion when B is current.
__global__ void bst_to_winv_kernel(const double2* __restrict__ B, float2* __restrict__ WmH, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) WmH[i] = make_float2((float)B[i].x, (float)B[i].y);
}

// Default start of the piecewise-stationary model: W = I, L = 1, v[n][j] = tr(X^_j)/(M N) u,
// u ~ U[0.5, 1.5) from Philox4x32-10 (the frame-wise default with tr(X^_j) for ||x_t||^2).
__global__ void default_params_blocks_kernel(const float* __restrict__ xh, double2* __restrict__ P,
                                             float* __restrict__ lam, float* __restrict__ v, int F, int J, int M,
                                             int N, uint32_t seed) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < (size_t)F * M * M) {
    const size_t r = i % ((size_t)M * M);
    P[i] = make_double2((r / M == r % M) ? 1.0 : 0.0, 0.0);
  }
  if (i < (size_t)F * M * N) lam[i] = 1.0f;
  if (i < (size_t)F * N * J) {
    const size_t f = i / ((size_t)N * J), n = (i / J) % N, j = i % J;
    const float* e = xh + (f * J + j) * (size_t)M * M;
    float tr = 0.f;
    for (int a = 0; a < M; ++a) tr += e[a];
    const ffca::U4 r = ffca::philox4x32_10(ffca::U4{(uint32_t)f, (uint32_t)n, (uint32_t)j, 0x1d17u}, seed, 0u);
    v[i] = fmaxf(tr / (float)(M * N) * (0.5f + ffca::u01(r.x)), 1e-30f);
  }
}

// out[it] = sum_f hist[f * stride + it] for it < n: one CTA of kSumThreads per column, each
// thread summing f = tid, tid + kSumThreads, ... in order, then a fixed-shape tree over the
// threads, so that the total is the same bits on every call.
constexpr int kSumThreads = 256;

__global__ void __launch_bounds__(kSumThreads) sum_over_f_kernel(const double* __restrict__ hist, int F, int stride,
                                                                 int n, double* __restrict__ out) {
  __shared__ double red[kSumThreads];
  const int it = blockIdx.x, tid = threadIdx.x;
  if (it >= n) return;                                  // uniform over the CTA
  double s = 0.0;
  for (int f = tid; f < F; f += kSumThreads) s += hist[(size_t)f * stride + it];
  red[tid] = s;
#pragma unroll
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    __syncthreads();
    if (tid < w) red[tid] += red[tid + w];
  }
  if (tid == 0) out[it] = red[0];
}

__global__ void init_fca_params_kernel(double2* __restrict__ R, int F, int N, int M) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < (size_t)F * N * M * M) {
    const size_t r = i % ((size_t)M * M);
    R[i] = make_double2((r / M == r % M) ? 1.0 : 0.0, 0.0);
  }
}

void free_all(fastfca_ctx* c) {
  ffca::dev_free(c->x_owned);
  ffca::dev_free(c->xh);
  ffca::dev_free(c->P);
  ffca::dev_free(c->lam);
  ffca::dev_free(c->v);
  ffca::dev_free(c->winv);
  ffca::dev_free(c->c_stage);
  ffca::dev_free(c->Bst);
  ffca::dev_free(c->detst);
  ffca::dev_free(c->tb);
  ffca::dev_free(c->va);
  ffca::dev_free(c->ab);
  ffca::dev_free(c->ubuf);
  ffca::dev_free(c->mscratch);
  ffca::dev_free(c->R);
  ffca::dev_free(c->h);
  ffca::fca_work_free(&c->fca);
  ffca::dev_free(c->ll_hist);
  ffca::dev_free(c->ll_last);
  ffca::dev_free(c->ll_sum);
  ffca::dev_free(c->err);
}

fastfca_status ensure_ll_capacity(fastfca_ctx* c, int n) {
  if (n <= c->ll_cap) return FASTFCA_OK;
  ffca::dev_free(c->ll_hist);
  ffca::dev_free(c->ll_sum);
  c->ll_hist = nullptr;
  c->ll_sum = nullptr;
  c->ll_cap = 0;
  CK(c, ffca::dev_malloc(&c->ll_hist, sizeof(double) * (size_t)c->cfg.F * n), "ll history alloc");
  CK(c, ffca::dev_malloc(&c->ll_sum, sizeof(double) * n), "ll sum alloc");
  c->ll_cap = n;
  return FASTFCA_OK;
}

}  // namespace

extern "C" {

const char* fastfca_version(void) { return "fastfca-gb300 0.1 (sm_103a)"; }

const char* fastfca_last_error(const fastfca_ctx* ctx) { return ctx ? ctx->msg : g_create_error; }

void fastfca_debug_fail_alloc(int64_t n) { ffca::g_fail_countdown.store(n < 0 ? -1 : (long long)n); }

int64_t fastfca_debug_live_allocs(void) { return ffca::g_live_allocs.load(); }

static fastfca_status create_impl(const fastfca_config* cfg, int B, int K, const void* x, void* stream,
                                  fastfca_ctx** out) {
  if (!out) return fail(nullptr, FASTFCA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || !x) return fail(nullptr, FASTFCA_EINVAL, "cfg and x are required");
  fastfca_config c = *cfg;
  if (c.F < 1 || c.T < 1 || c.M < 1 || c.N < 1)
    return fail(nullptr, FASTFCA_EINVAL, "F, T, M, N must be positive (got %d %d %d %d)", c.F, c.T, c.M, c.N);
  const bool mnmf = c.model == FASTFCA_MODEL_FASTMNMF;
  if (!fastfca_family(c.model) && !fca_family(c.model) && !mnmf)
    return fail(nullptr, FASTFCA_EINVAL, "unknown model %d", c.model);
  if (mnmf != (K > 0))
    return fail(nullptr, FASTFCA_EINVAL, mnmf ? "FastMNMF contexts are created by fastfca_create_mnmf"
                                              : "fastfca_create_mnmf needs cfg->model = FASTFCA_MODEL_FASTMNMF");
  if (mnmf && K > ffca::kMnmfMaxK)
    return fail(nullptr, FASTFCA_EINVAL, "K=%d bases per source is outside 1..%d", K, ffca::kMnmfMaxK);
  if (B < 1 || c.T % B != 0)
    return fail(nullptr, FASTFCA_EINVAL, "the block size B=%d must be >= 1 and divide T=%d", B, c.T);
  const int Tf = c.T;
  c.T = Tf / B;                                   // parameter columns: blocks
  ffca::FastOps ops{};
  ffca::FcaOps fops{};
  ffca::MnmfOps mops{};
  if (mnmf) {
    // the frequency-resident per-frequency step where it fits, else the cluster form
    const bool resident = ffca::mnmf_ops(c.M, c.N, &mops) && c.T <= mops.max_T;
    if (!resident && !ffca::mnmf_cluster_ops(c.M, c.N, c.T, &mops))
      return fail(nullptr, FASTFCA_EUNSUPPORTED, "no FastMNMF kernel for M=%d N=%d T=%d (M in 2..%d, N in 1..%d)",
                  c.M, c.N, c.T, kMaxM, kMaxN);
    if (!ffca::fast_ops_for(c.M, c.N, c.T, &ops))
      return fail(nullptr, FASTFCA_EUNSUPPORTED, "no Wiener filter for M=%d N=%d T=%d", c.M, c.N, c.T);
    if ((long long)c.F * K > ffca::kMnmfMaxFK)
      return fail(nullptr, FASTFCA_EUNSUPPORTED, "FastMNMF holds F*K <= %d bases of one source on chip (F=%d, K=%d)",
                  ffca::kMnmfMaxFK, c.F, K);
  } else if (B > 1) {
    if (!fastfca_family(c.model))
      return fail(nullptr, FASTFCA_EINVAL, "the piecewise-stationary input serves the FastFCA models only");
    if (!ffca::fast_ops_for(c.M, c.N, c.T, &ops) || !ops.em_blk)
      return fail(nullptr, FASTFCA_EUNSUPPORTED,
                  "no FastFCA kernel for M=%d N=%d and %d blocks (M in 2..%d, N in 1..%d)", c.M, c.N, c.T, kMaxM,
                  kMaxN);
  } else if (fastfca_family(c.model)) {
    if (!ffca::fast_ops_for(c.M, c.N, c.T, &ops))
      return fail(nullptr, FASTFCA_EUNSUPPORTED,
                  "no FastFCA kernel for M=%d N=%d T=%d (M in 2..%d, N in 1..%d, T within eight CTAs' "
                  "shared memory)", c.M, c.N, c.T, kMaxM, kMaxN);
    if (c.model == FASTFCA_MODEL_FASTFCA_MM && !ops.em_mm)
      return fail(nullptr, FASTFCA_EUNSUPPORTED, "no IP+MM (Algorithm 2) kernel for M=%d N=%d T=%d", c.M, c.N, c.T);
  } else {
    if (!ffca::fca_ops(c.M, c.N, &fops))
      return fail(nullptr, FASTFCA_EUNSUPPORTED, "no FCA kernel for M=%d N=%d", c.M, c.N);
    if (c.T > fops.max_T)
      return fail(nullptr, FASTFCA_EUNSUPPORTED, "T=%d exceeds the %d frames one FCA CTA holds", c.T, fops.max_T);
  }
  fastfca_ctx* ctx = new (std::nothrow) fastfca_ctx();
  if (!ctx) return fail(nullptr, FASTFCA_ENOMEM, "host allocation failed");
  ctx->cfg = c;
  ctx->Tf = Tf;
  ctx->B = B;
  ctx->stream = (cudaStream_t)stream;
  ctx->ops = ops;
  ctx->fops = fops;
  ctx->mops = mops;
  ctx->K = K;
  const size_t nx = (size_t)c.F * Tf * c.M;
  auto bail = [&](fastfca_status st) {
    snprintf(g_create_error, sizeof g_create_error, "%s", ctx->msg);
    free_all(ctx);
    delete ctx;
    return st;
  };
#define CKC(expr, what)                                              \
  do {                                                               \
    cudaError_t e__ = (expr);                                        \
    if (e__ != cudaSuccess) return bail(cuda_fail(ctx, e__, what));  \
  } while (0)
  if (is_device_ptr(x)) {
    // the kernels load frames as 16-byte vectors
    if (reinterpret_cast<uintptr_t>(x) % 16 != 0)
      return bail(fail(ctx, FASTFCA_EINVAL, "a device x must start on a 16-byte boundary"));
    ctx->x = static_cast<const float2*>(x);
  } else {
    CKC(ffca::dev_malloc(&ctx->x_owned, sizeof(float2) * nx), "x alloc");
    CKC(cudaMemcpyAsync(ctx->x_owned, x, sizeof(float2) * nx, cudaMemcpyHostToDevice, ctx->stream), "x upload");
    ctx->x = ctx->x_owned;
  }
  CKC(ffca::dev_malloc(&ctx->err, sizeof(int)), "status alloc");
  CKC(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream), "status clear");
  CKC(ffca::dev_malloc(&ctx->ll_last, sizeof(double) * c.F), "ll alloc");
  const int threads = 256;
  if (mnmf) {
    CKC(ffca::dev_malloc(&ctx->P, sizeof(double2) * (size_t)c.F * c.M * c.M), "W alloc");
    CKC(ffca::dev_malloc(&ctx->lam, sizeof(float) * (size_t)c.F * c.M * c.N), "lam alloc");
    CKC(ffca::dev_malloc(&ctx->v, sizeof(float) * FT(c) * c.N), "h alloc");
    CKC(ffca::dev_malloc(&ctx->winv, sizeof(float2) * (size_t)c.F * c.M * c.M), "winv alloc");
    CKC(ffca::dev_malloc(&ctx->Bst, sizeof(double2) * (size_t)c.F * c.M * c.M), "B alloc");
    CKC(ffca::dev_malloc(&ctx->detst, sizeof(double) * 2 * (size_t)c.F), "det alloc");
    CKC(ffca::dev_malloc(&ctx->tb, sizeof(float) * (size_t)c.F * c.N * K), "t alloc");
    CKC(ffca::dev_malloc(&ctx->va, sizeof(float) * (size_t)c.N * K * c.T), "v alloc");
    CKC(ffca::dev_malloc(&ctx->ab, sizeof(float) * 2 * FT(c) * c.N), "update terms alloc");
    CKC(ffca::dev_malloc(&ctx->ubuf, sizeof(float) * FT(c) * c.M), "U alloc");
    CKC(ffca::dev_malloc(&ctx->mscratch, sizeof(float) * ((size_t)c.F + c.T + 1)), "scratch alloc");
    CKC(ffca::launch_mnmf_default(ctx->x, ctx->P, ctx->lam, ctx->tb, ctx->va, ctx->mscratch, c.F, c.T, c.M, c.N, K,
                                  (uint32_t)c.seed, ctx->stream),
        "init launch");
  } else if (fastfca_family(c.model)) {
    CKC(ffca::dev_malloc(&ctx->P, sizeof(double2) * (size_t)c.F * c.M * c.M), "P alloc");
    CKC(ffca::dev_malloc(&ctx->lam, sizeof(float) * (size_t)c.F * c.M * c.N), "lam alloc");
    CKC(ffca::dev_malloc(&ctx->v, sizeof(float) * FT(c) * c.N), "v alloc");
    CKC(ffca::dev_malloc(&ctx->winv, sizeof(float2) * (size_t)c.F * c.M * c.M), "winv alloc");
    CKC(ffca::dev_malloc(&ctx->Bst, sizeof(double2) * (size_t)c.F * c.M * c.M), "B alloc");
    CKC(ffca::dev_malloc(&ctx->detst, sizeof(double) * 2 * (size_t)c.F), "det alloc");
    const size_t n = ffca::default_params_elems(c.F, c.T, c.M, c.N);
    if (B > 1) {
      CKC(ffca::dev_malloc(&ctx->xh, sizeof(float) * FT(c) * c.M * c.M), "block statistics alloc");
      CKC(ctx->ops.block_stats(ctx->x, ctx->xh, c.F, c.T, B, ctx->stream), "block statistics launch");
      default_params_blocks_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, ctx->stream>>>(
          ctx->xh, ctx->P, ctx->lam, ctx->v, c.F, c.T, c.M, c.N, (uint32_t)c.seed);
    } else {
      ffca::default_params_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, ctx->stream>>>(
          ctx->x, ctx->P, ctx->lam, ctx->v, c.F, c.T, c.M, c.N, (uint32_t)c.seed);
    }
    CKC(cudaGetLastError(), "init launch");
  } else {
    CKC(ffca::dev_malloc(&ctx->R, sizeof(double2) * (size_t)c.F * c.N * c.M * c.M), "R alloc");
    CKC(ffca::dev_malloc(&ctx->h, sizeof(float) * FT(c) * c.N), "h alloc");
    // FastFCA's initial v is also FCA's initial h
    double2* Ptmp = nullptr;
    float* lamtmp = nullptr;
    cudaError_t e = ffca::dev_malloc(&Ptmp, sizeof(double2) * (size_t)c.F * c.M * c.M);
    if (e == cudaSuccess) e = ffca::dev_malloc(&lamtmp, sizeof(float) * (size_t)c.F * c.M * c.N);
    if (e == cudaSuccess) {
      const size_t n = ffca::default_params_elems(c.F, c.T, c.M, c.N);
      ffca::default_params_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, ctx->stream>>>(
          ctx->x, Ptmp, lamtmp, ctx->h, c.F, c.T, c.M, c.N, (uint32_t)c.seed);
      const size_t nr = (size_t)c.F * c.N * c.M * c.M;
      init_fca_params_kernel<<<(unsigned)((nr + threads - 1) / threads), threads, 0, ctx->stream>>>(ctx->R, c.F, c.N, c.M);
      e = cudaGetLastError();
      cudaStreamSynchronize(ctx->stream);
    }
    ffca::dev_free(Ptmp);     // both temporaries, whichever step failed
    ffca::dev_free(lamtmp);
    CKC(e, "FCA start");
    CKC(ffca::fca_work_alloc(&ctx->fca, c.F, c.T, c.M, c.N), "FCA workspace alloc");
  }
  CKC(cudaStreamSynchronize(ctx->stream), "create synchronize");
#undef CKC
  *out = ctx;
  return FASTFCA_OK;
}

fastfca_status fastfca_create(const fastfca_config* cfg, const void* x, void* stream, fastfca_ctx** out) {
  FFCA_TRACE("fastfca_create");
  return create_impl(cfg, 1, 0, x, stream, out);
}

fastfca_status fastfca_create_blocks(const fastfca_config* cfg, int32_t B, const void* x, void* stream,
                                     fastfca_ctx** out) {
  FFCA_TRACE("fastfca_create_blocks");
  return create_impl(cfg, B, 0, x, stream, out);
}

fastfca_status fastfca_create_mnmf(const fastfca_config* cfg, int32_t K, const void* x, void* stream,
                                   fastfca_ctx** out) {
  FFCA_TRACE("fastfca_create_mnmf");
  if (K < 1) {
    if (out) *out = nullptr;
    return fail(nullptr, FASTFCA_EINVAL, "K=%d bases per source is outside 1..%d", K, ffca::kMnmfMaxK);
  }
  return create_impl(cfg, 1, K, x, stream, out);
}

fastfca_status fastfca_set_params_mnmf(fastfca_ctx* ctx, const void* W, const float* lam, const float* t,
                                       const float* v) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (ctx->cfg.model != FASTFCA_MODEL_FASTMNMF) return fail(ctx, FASTFCA_EINVAL, "context does not hold FastMNMF");
  if (!W || !lam || !t || !v) return fail(ctx, FASTFCA_EINVAL, "W, lam, t and v are required");
  const fastfca_config& c = ctx->cfg;
  CK(ctx, to_device(ctx->P, W, sizeof(double2) * (size_t)c.F * c.M * c.M, ctx->stream), "W upload");
  CK(ctx, to_device(ctx->lam, lam, sizeof(float) * (size_t)c.F * c.M * c.N, ctx->stream), "lam upload");
  CK(ctx, to_device(ctx->tb, t, sizeof(float) * (size_t)c.F * c.N * ctx->K, ctx->stream), "t upload");
  CK(ctx, to_device(ctx->va, v, sizeof(float) * (size_t)c.N * ctx->K * c.T, ctx->stream), "v upload");
  ctx->b_valid = 0;
  ctx->h_valid = 0;
  if (ctx->sticky == FASTFCA_ENUMERIC) ctx->sticky = FASTFCA_OK;
  return FASTFCA_OK;
}

fastfca_status fastfca_get_params_mnmf(fastfca_ctx* ctx, void* W, float* lam, float* t, float* v) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (ctx->cfg.model != FASTFCA_MODEL_FASTMNMF) return fail(ctx, FASTFCA_EINVAL, "context does not hold FastMNMF");
  const fastfca_config& c = ctx->cfg;
  if (W) CK(ctx, from_device(W, ctx->P, sizeof(double2) * (size_t)c.F * c.M * c.M, ctx->stream), "W download");
  if (lam) CK(ctx, from_device(lam, ctx->lam, sizeof(float) * (size_t)c.F * c.M * c.N, ctx->stream), "lam download");
  if (t) CK(ctx, from_device(t, ctx->tb, sizeof(float) * (size_t)c.F * c.N * ctx->K, ctx->stream), "t download");
  if (v) CK(ctx, from_device(v, ctx->va, sizeof(float) * (size_t)c.N * ctx->K * c.T, ctx->stream), "v download");
  return collect_device_status(ctx);
}

}  // extern "C"

namespace {
// h = t v (Eq. 52) into the h buffer unless it already holds it.
fastfca_status mnmf_ensure_h(fastfca_ctx* ctx) {
  if (ctx->h_valid) return FASTFCA_OK;
  const fastfca_config& c = ctx->cfg;
  CK(ctx, ffca::launch_mnmf_h(ctx->tb, ctx->va, ctx->v, c.F, c.N, ctx->K, c.T, ctx->stream), "FastMNMF h launch");
  ctx->h_valid = 1;
  return FASTFCA_OK;
}

// One FastMNMF launch of the per-frequency kernel (iterate = 1: one iteration; 0: the
// log-likelihood of the current parameters only).
fastfca_status mnmf_freq(fastfca_ctx* ctx, int iterate, double* ll_out, int ll_stride, double* ll_last) {
  const fastfca_config& c = ctx->cfg;
  fastfca_status st = mnmf_ensure_h(ctx);
  if (st) return st;
  ffca::MnmfArgs a{};
  a.x = ctx->x;
  a.P = ctx->P;
  a.Bst = ctx->Bst;
  a.detst = ctx->detst;
  a.b_valid = ctx->b_valid;
  a.lam = ctx->lam;
  a.hin = ctx->v;
  a.ab = ctx->ab;
  a.u = ctx->ubuf;
  a.ll_out = ll_out;
  a.ll_last = ll_last;
  a.err = ctx->err;
  a.F = c.F;
  a.T = c.T;
  a.N = c.N;
  a.ll_stride = ll_stride;
  a.iterate = iterate;
  CK(ctx, ctx->mops.freq(a, ctx->stream), "FastMNMF frequency launch");
  ctx->b_valid = 1;
  return FASTFCA_OK;
}
}  // namespace

extern "C" {

void fastfca_destroy(fastfca_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
}

fastfca_status fastfca_set_params(fastfca_ctx* ctx, const void* P, const float* lam, const float* v) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (!fastfca_family(ctx->cfg.model)) return fail(ctx, FASTFCA_EINVAL, "context does not hold the FastFCA model");
  if (!P || !lam || !v) return fail(ctx, FASTFCA_EINVAL, "P, lam and v are required");
  const fastfca_config& c = ctx->cfg;
  CK(ctx, to_device(ctx->P, P, sizeof(double2) * (size_t)c.F * c.M * c.M, ctx->stream), "P upload");
  CK(ctx, to_device(ctx->lam, lam, sizeof(float) * (size_t)c.F * c.M * c.N, ctx->stream), "lam upload");
  CK(ctx, to_device(ctx->v, v, sizeof(float) * FT(c) * c.N, ctx->stream), "v upload");
  ctx->b_valid = 0;
  if (ctx->sticky == FASTFCA_ENUMERIC) ctx->sticky = FASTFCA_OK;
  return FASTFCA_OK;
}

fastfca_status fastfca_get_params(fastfca_ctx* ctx, void* P, float* lam, float* v) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (!fastfca_family(ctx->cfg.model)) return fail(ctx, FASTFCA_EINVAL, "context does not hold the FastFCA model");
  const fastfca_config& c = ctx->cfg;
  if (P) CK(ctx, from_device(P, ctx->P, sizeof(double2) * (size_t)c.F * c.M * c.M, ctx->stream), "P download");
  if (lam) CK(ctx, from_device(lam, ctx->lam, sizeof(float) * (size_t)c.F * c.M * c.N, ctx->stream), "lam download");
  if (v) CK(ctx, from_device(v, ctx->v, sizeof(float) * FT(c) * c.N, ctx->stream), "v download");
  return collect_device_status(ctx);
}

fastfca_status fastfca_set_params_fca(fastfca_ctx* ctx, const void* R, const float* h) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (!fca_family(ctx->cfg.model)) return fail(ctx, FASTFCA_EINVAL, "context does not hold the FCA model");
  if (!R || !h) return fail(ctx, FASTFCA_EINVAL, "R and h are required");
  const fastfca_config& c = ctx->cfg;
  CK(ctx, to_device(ctx->R, R, sizeof(double2) * (size_t)c.F * c.N * c.M * c.M, ctx->stream), "R upload");
  CK(ctx, to_device(ctx->h, h, sizeof(float) * FT(c) * c.N, ctx->stream), "h upload");
  if (ctx->sticky == FASTFCA_ENUMERIC) ctx->sticky = FASTFCA_OK;
  return FASTFCA_OK;
}

fastfca_status fastfca_get_params_fca(fastfca_ctx* ctx, void* R, float* h) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (!fca_family(ctx->cfg.model)) return fail(ctx, FASTFCA_EINVAL, "context does not hold the FCA model");
  const fastfca_config& c = ctx->cfg;
  if (R) CK(ctx, from_device(R, ctx->R, sizeof(double2) * (size_t)c.F * c.N * c.M * c.M, ctx->stream), "R download");
  if (h) CK(ctx, from_device(h, ctx->h, sizeof(float) * FT(c) * c.N, ctx->stream), "h download");
  return collect_device_status(ctx);
}

fastfca_status fastfca_iterate(fastfca_ctx* ctx, int32_t n_iter, double* ll_per_iter) {
  FFCA_TRACE("fastfca_iterate");
  fastfca_status st = check_params_usable(ctx);
  if (st) return st;
  if (n_iter < 1) return fail(ctx, FASTFCA_EINVAL, "n_iter must be >= 1 (got %d)", n_iter);
  const fastfca_config& c = ctx->cfg;
  double* hist = nullptr;
  if (ll_per_iter) {
    st = ensure_ll_capacity(ctx, n_iter);
    if (st) return st;
    hist = ctx->ll_hist;
  }
  if (c.model == FASTFCA_MODEL_FASTMNMF) {
    // launch it of the per-frequency kernel also gives the log-likelihood after iteration it-1
    for (int it = 0; it < n_iter; ++it) {
      // IP and lambda (per frequency), then t, then the v update's terms with the new t, then v
      st = mnmf_freq(ctx, 1, (hist && it > 0) ? hist + (it - 1) : nullptr, n_iter, nullptr);
      if (st) return st;
      CK(ctx, ffca::launch_mnmf_t(ctx->tb, ctx->va, ctx->ab, c.F, c.N, ctx->K, c.T, ctx->stream),
         "FastMNMF basis update launch");
      CK(ctx, ctx->mops.ab(ctx->lam, ctx->tb, ctx->va, ctx->ubuf, ctx->ab, c.F, c.N, ctx->K, c.T, ctx->err, ctx->stream),
         "FastMNMF activation-update terms launch");
      CK(ctx, ffca::launch_mnmf_v(ctx->tb, ctx->ab, ctx->va, ctx->v, c.F, c.N, ctx->K, c.T, ctx->stream),
         "FastMNMF activation update launch");
    }
    if (hist) {
      st = mnmf_freq(ctx, 0, hist + (n_iter - 1), n_iter, ctx->ll_last);
      if (st) return st;
    }
  } else if (fastfca_family(c.model)) {
    ffca::EmArgs a{};
    a.x = ctx->x;
    a.xh = ctx->xh;
    a.P = ctx->P;
    a.lam = ctx->lam;
    a.v = ctx->v;
    a.ll_hist = hist;
    a.ll_last = ctx->ll_last;
    a.Bst = ctx->Bst;
    a.detst = ctx->detst;
    a.b_valid = ctx->b_valid;
    a.err = ctx->err;
    a.F = c.F;
    a.T = c.T;
    a.N = c.N;
    a.n_iter = n_iter;
    a.ll_stride = n_iter;
    const bool mm = c.model == FASTFCA_MODEL_FASTFCA_MM;
    auto launch = ctx->B > 1 ? (mm ? ctx->ops.em_mm_blk : ctx->ops.em_blk) : (mm ? ctx->ops.em_mm : ctx->ops.em);
    CK(ctx, launch(a, ctx->stream), "FastFCA IP+EM/IP+MM launch");
    ctx->b_valid = 1;
  } else {
    ffca::FcaArgs a{};
    a.x = ctx->x;
    a.R = ctx->R;
    a.h = ctx->h;
    a.ll_hist = hist;
    a.ll_last = ctx->ll_last;
    a.err = ctx->err;
    a.F = c.F;
    a.T = c.T;
    a.n_iter = n_iter;
    a.ll_stride = n_iter;
    auto launch = c.model == FASTFCA_MODEL_FCA_MM ? ctx->fops.em_mm : ctx->fops.em;
    CK(ctx, launch(a, &ctx->fca, ctx->stream), "FCA EM/MM launch");
  }
  if (!ll_per_iter) return FASTFCA_OK;
  sum_over_f_kernel<<<n_iter, kSumThreads, 0, ctx->stream>>>(ctx->ll_hist, c.F, n_iter, n_iter, ctx->ll_sum);
  CK(ctx, cudaGetLastError(), "ll sum launch");
  // stream-ordered download; kernel status is collected by the next synchronising call
  CK(ctx, cudaMemcpyAsync(ll_per_iter, ctx->ll_sum, sizeof(double) * n_iter, cudaMemcpyDefault, ctx->stream),
     "ll download");
  return FASTFCA_OK;
}

fastfca_status fastfca_loglik(fastfca_ctx* ctx, double* ll_total, double* ll_per_f) {
  FFCA_TRACE("fastfca_loglik");
  fastfca_status st = check_params_usable(ctx);
  if (st) return st;
  const fastfca_config& c = ctx->cfg;
  if (c.model == FASTFCA_MODEL_FASTMNMF) {
    st = mnmf_freq(ctx, 0, nullptr, 0, ctx->ll_last);
    if (st) return st;
  } else if (fastfca_family(c.model)) {
    ffca::EmArgs a{};
    a.x = ctx->x;
    a.xh = ctx->xh;
    a.P = ctx->P;
    a.lam = ctx->lam;
    a.v = ctx->v;
    a.ll_hist = nullptr;
    a.ll_last = ctx->ll_last;
    a.Bst = ctx->Bst;
    a.detst = ctx->detst;
    a.b_valid = ctx->b_valid;
    a.err = ctx->err;
    a.F = c.F;
    a.T = c.T;
    a.N = c.N;
    a.n_iter = 0;
    a.ll_stride = 0;
    CK(ctx, (ctx->B > 1 ? ctx->ops.em_blk : ctx->ops.em)(a, ctx->stream), "FastFCA log-likelihood launch");
    ctx->b_valid = 1;
  } else {
    ffca::FcaArgs a{};
    a.x = ctx->x;
    a.R = ctx->R;
    a.h = ctx->h;
    a.ll_last = ctx->ll_last;
    a.err = ctx->err;
    a.F = c.F;
    a.T = c.T;
    a.n_iter = 0;
    CK(ctx, ctx->fops.em(a, &ctx->fca, ctx->stream), "FCA log-likelihood launch");
  }
  if (ll_total) {
    st = ensure_ll_capacity(ctx, 1);
    if (st) return st;
    sum_over_f_kernel<<<1, kSumThreads, 0, ctx->stream>>>(ctx->ll_last, c.F, 1, 1, ctx->ll_sum);
    CK(ctx, cudaGetLastError(), "ll sum launch");
    CK(ctx, cudaMemcpyAsync(ll_total, ctx->ll_sum, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "ll download");
  }
  if (ll_per_f) CK(ctx, from_device(ll_per_f, ctx->ll_last, sizeof(double) * c.F, ctx->stream), "ll per f download");
  return collect_device_status(ctx);
}

fastfca_status fastfca_separate(fastfca_ctx* ctx, void* c_out) {
  FFCA_TRACE("fastfca_separate");
  fastfca_status st = check_params_usable(ctx);
  if (st) return st;
  if (!c_out) return fail(ctx, FASTFCA_EINVAL, "c is required");
  if (reinterpret_cast<uintptr_t>(c_out) % 8 != 0)
    return fail(ctx, FASTFCA_EINVAL, "c must start on an 8-byte boundary (complex64 stores)");
  const fastfca_config& c = ctx->cfg;
  const size_t bytes = sizeof(float2) * (size_t)c.F * ctx->Tf * c.N * c.M;
  const bool dev = is_device_ptr(c_out);
  float2* dst = static_cast<float2*>(c_out);
  if (!dev) {
    // the staging buffer is made on the first separation into host memory and kept: a
    // stream of host separations then allocates nothing per call
    if (!ctx->c_stage) CK(ctx, ffca::dev_malloc(&ctx->c_stage, bytes), "c staging alloc");
    dst = ctx->c_stage;
  }
  cudaError_t e = cudaSuccess;
  if (fastfca_family(c.model) || c.model == FASTFCA_MODEL_FASTMNMF) {
    // FastMNMF: h = t v (Eq. 52) in the FastFCA filter's H layout, then the same filter (Eq. 39)
    if (c.model == FASTFCA_MODEL_FASTMNMF && !ctx->h_valid) {
      e = ffca::launch_mnmf_h(ctx->tb, ctx->va, ctx->v, c.F, c.N, ctx->K, c.T, ctx->stream);
      if (e == cudaSuccess) ctx->h_valid = 1;
    }
    if (e == cudaSuccess && ctx->b_valid) {
      const size_t n = (size_t)c.F * c.M * c.M;
      bst_to_winv_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->Bst, ctx->winv, n);
      e = cudaGetLastError();
    } else if (e == cudaSuccess) {
      e = ctx->ops.winv(ctx->P, ctx->winv, c.F, ctx->err, ctx->stream);
    }
    if (e == cudaSuccess)
      e = ctx->ops.mwf(ctx->x, ctx->P, ctx->winv, ctx->lam, ctx->v, dst, c.F, ctx->Tf, c.N, ctx->B, ctx->stream);
  } else {
    e = ctx->fops.mwf(ctx->x, ctx->R, ctx->h, dst, c.F, c.T, ctx->err, ctx->stream);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "separate launch");
  if (!dev) {
    // stream-ordered download: no synchronisation here, kernel status is collected by the
    // next synchronising call
    e = cudaMemcpyAsync(c_out, ctx->c_stage, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "c download");
  }
  return FASTFCA_OK;
}

fastfca_status fastfca_set_mixture(fastfca_ctx* ctx, const void* x) {
  FFCA_TRACE("fastfca_set_mixture");
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  if (!x) return fail(ctx, FASTFCA_EINVAL, "x is required");
  const size_t bytes = sizeof(float2) * (size_t)ctx->cfg.F * ctx->Tf * ctx->cfg.M;
  if (!ctx->x_owned) CK(ctx, ffca::dev_malloc(&ctx->x_owned, bytes), "x alloc");
  CK(ctx, cudaMemcpyAsync(ctx->x_owned, x, bytes, cudaMemcpyDefault, ctx->stream), "x upload");
  ctx->x = ctx->x_owned;
  if (ctx->B > 1)
    CK(ctx, ctx->ops.block_stats(ctx->x, ctx->xh, ctx->cfg.F, ctx->cfg.T, ctx->B, ctx->stream), "block statistics launch");
  return FASTFCA_OK;
}

fastfca_status fastfca_sync(fastfca_ctx* ctx) {
  fastfca_status st = check_ready(ctx);
  if (st) return st;
  return collect_device_status(ctx);
}

}  // extern "C"

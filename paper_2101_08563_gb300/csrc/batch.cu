// Batched FastFCA: many mixtures with mixed (M, N, T) in one CUDA-graph launch.
//
// Work unit: one frequency of one mixture (an EmItem), run start to finish by one CTA with the
// same per-frequency code as the single-mixture path (em_frequency).  Items are grouped into
// classes by (M, N) and a frame bucket that fixes the CTA size; every class runs as one
// persistent launch whose CTAs take items from an atomic counter, longest first.  All class
// launches sit on forked streams inside one captured CUDA graph, so one graph launch runs the
// whole batch.  The schedule (bucketing of T into CTA sizes, CTAs per class) is chosen by a
// small autotuner that times each candidate on the batch itself (fastfca_batch_tune).
// %globaltimer stamps per item give each mixture's wall time inside the launch.
//
// One more schedule runs each mixture as one launch of the single-mixture kernel (one CTA per
// frequency, all of them in one wave), the mixtures spread longest-first over a few concurrent
// branches of the graph so that one launch's tail overlaps the next launch's start.  Measured
// on the 64-mixture batch (M in {2,3,4}, T in [200, 2000], 20 iterations), the per-class
// persistent launches took 44.5 ms and the same 64 single-mixture launches in a row 35.9 ms:
// co-resident CTAs of many classes, each running items of its own size, used the SMs worse
// than one mixture's uniform wave.  The tuner measures this schedule beside the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "../../include/fastfca.h"
#include "alloc.h"
#include "init.cuh"
#include "launch.cuh"
#include "trace.h"

namespace {

struct Mix {
  fastfca_config cfg{};
  const float2* x = nullptr;
  float2* x_owned = nullptr;
  double2* P = nullptr;
  float* lam = nullptr;
  float* v = nullptr;
  double2* Bst = nullptr;
  double* detst = nullptr;
  double* ll_last = nullptr;
  int* flags = nullptr;
  float2* winv = nullptr;
  size_t item0 = 0;          // global index of this mixture's frequency 0
  ffca::FastOps ops{};
};

struct Class {
  int M = 0, N = 0, mm = 0, bd = 0, grid = 0;   // mm: 0 IP+EM (Algorithm 1), 1 IP+MM (Algorithm 2)
  std::vector<size_t> items;          // global item indices, longest first
  ffca::EmItem* d_items = nullptr;
  int* d_counter = nullptr;
  ffca::FastOps ops{};
};

// Frame-bucket schemes the tuner chooses between.
// kMixture: one single-mixture launch per mixture, on 2 x factor concurrent graph branches.
enum Scheme { kFine = 0, kCoarse = 1, kSingle = 2, kMixture = 3, kNumSchemes = 4 };

int bucket_threads(int scheme, int T, int group_max_T) {
  auto warps_for = [](int t) { return std::max(1, (t + 32 * ffca::kSlots - 1) / (32 * ffca::kSlots)); };
  switch (scheme) {
    case kFine: return 32 * warps_for(T);
    case kCoarse: return T <= 1024 ? 128 : 256;
    default: return 32 * warps_for(group_max_T);
  }
}

}  // namespace

struct fastfca_batch {
  std::vector<Mix> mix;
  std::vector<ffca::EmItem> items;     // host mirror, global order (mixture-major)
  std::vector<Class> classes;
  unsigned long long* d_stamps = nullptr;
  int* d_err = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;       // one join event per side stream
  cudaEvent_t fork = nullptr;
  cudaStream_t capture = nullptr;    // graphs are captured here (never the legacy stream)
  std::map<int, cudaGraphExec_t> graphs;
  int scheme = kFine;
  double grid_factor = 1.0;
  bool have_schedule = false;
  std::vector<std::vector<int>> branch_mix;   // kMixture: the mixtures of each branch, in order
  std::vector<cudaEvent_t> tev;              // kMixture: start / end events per mixture (timing)
  int sms = 0;
  fastfca_status sticky = FASTFCA_OK;
  char msg[512] = "";
};

namespace {

fastfca_status bfail(fastfca_batch* b, fastfca_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) {
    snprintf(b->msg, sizeof b->msg, "%s", buf);
    if (st == FASTFCA_ECUDA) b->sticky = st;
  } else {
    ffca::set_thread_error(buf);
  }
  return st;
}

#define BCK(b, expr, what)                                                             \
  do {                                                                                 \
    cudaError_t e__ = (expr);                                                          \
    if (e__ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                              \
      return bfail(b, e__ == cudaErrorMemoryAllocation ? FASTFCA_ENOMEM : FASTFCA_ECUDA, \
                   "%s: %s", what, cudaGetErrorString(e__));                           \
    }                                                                                  \
  } while (0)

// The status BCK would return for e, without returning: for paths that must clean up.
fastfca_status bcheck(fastfca_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FASTFCA_OK;
  cudaGetLastError();
  return bfail(b, e == cudaErrorMemoryAllocation ? FASTFCA_ENOMEM : FASTFCA_ECUDA, "%s: %s", what,
               cudaGetErrorString(e));
}

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (is_dev(src)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  return e != cudaSuccess ? e : cudaStreamSynchronize(s);
}

cudaError_t copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (is_dev(dst)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
  return e != cudaSuccess ? e : cudaStreamSynchronize(s);
}

void free_graphs(fastfca_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

void free_classes(fastfca_batch* b) {
  for (auto& c : b->classes) {
    ffca::dev_free(c.d_items);
    ffca::dev_free(c.d_counter);
  }
  b->classes.clear();
}

void free_batch(fastfca_batch* b) {
  free_graphs(b);
  free_classes(b);
  for (auto& m : b->mix) {
    ffca::dev_free(m.x_owned);
    ffca::dev_free(m.P);
    ffca::dev_free(m.lam);
    ffca::dev_free(m.v);
    ffca::dev_free(m.Bst);
    ffca::dev_free(m.detst);
    ffca::dev_free(m.ll_last);
    ffca::dev_free(m.flags);
    ffca::dev_free(m.winv);
  }
  ffca::dev_free(b->d_stamps);
  ffca::dev_free(b->d_err);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->ev) cudaEventDestroy(e);
  for (auto e : b->tev) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->capture) cudaStreamDestroy(b->capture);
}

double item_cost(const ffca::EmItem& it, int M, int N) { return (double)it.T * (double)(M * M + M * N + 8); }

fastfca_status ensure_side_streams(fastfca_batch* b, size_t n) {
  while (b->side.size() < n) {
    cudaStream_t s;
    cudaEvent_t e;
    BCK(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "side stream");
    BCK(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "side event");
    b->side.push_back(s);
    b->ev.push_back(e);
  }
  if (!b->fork) BCK(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "fork event");
  return FASTFCA_OK;
}

// The kMixture schedule: 2 x factor branches; mixtures longest-first, each to the branch with
// the least work so far.
fastfca_status build_mixture_schedule(fastfca_batch* b, double grid_factor) {
  const int nb = std::max(1, std::min<int>((int)std::lround(2.0 * grid_factor), (int)b->mix.size()));
  std::vector<std::pair<double, int>> order;
  for (size_t i = 0; i < b->mix.size(); ++i) {
    const fastfca_config& c = b->mix[i].cfg;
    order.push_back({(double)c.F * c.T * (double)(c.M * c.M + c.M * c.N + 8), (int)i});
  }
  std::stable_sort(order.begin(), order.end(), [](const auto& a, const auto& z) { return a.first > z.first; });
  b->branch_mix.assign(nb, {});
  std::vector<double> load(nb, 0.0);
  for (const auto& w : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->branch_mix[j].push_back(w.second);
    load[j] += w.first;
  }
  const fastfca_status st = ensure_side_streams(b, (size_t)nb);
  if (st) return st;
  b->scheme = kMixture;
  b->grid_factor = grid_factor;
  b->have_schedule = true;
  return FASTFCA_OK;
}

// Builds the classes of a schedule: bucket the items, order each class longest first, size
// each class's persistent grid by its share of the work and the occupancy of its kernel.
fastfca_status build_classes_once(fastfca_batch* b, int scheme, double grid_factor) {
  free_graphs(b);
  free_classes(b);
  b->have_schedule = false;
  b->branch_mix.clear();
  if (scheme == kMixture) return build_mixture_schedule(b, grid_factor);
  std::map<std::pair<int, int>, int> group_max_T;
  for (const auto& m : b->mix) {
    auto key = std::make_pair(m.cfg.M, m.cfg.N);
    group_max_T[key] = std::max(group_max_T[key], m.cfg.T);
  }
  std::map<std::tuple<int, int, int, int>, size_t> index;
  for (size_t mi = 0; mi < b->mix.size(); ++mi) {
    const Mix& m = b->mix[mi];
    const int bd = bucket_threads(scheme, m.cfg.T, group_max_T[std::make_pair(m.cfg.M, m.cfg.N)]);
    const int mm = m.cfg.model == FASTFCA_MODEL_FASTFCA_MM ? 1 : 0;
    auto key = std::make_tuple(m.cfg.M, m.cfg.N, mm, bd);
    auto it = index.find(key);
    if (it == index.end()) {
      Class c;
      c.M = m.cfg.M;
      c.N = m.cfg.N;
      c.mm = mm;
      c.bd = bd;
      c.ops = m.ops;
      index[key] = b->classes.size();
      b->classes.push_back(c);
      it = index.find(key);
    }
    Class& c = b->classes[it->second];
    for (int f = 0; f < m.cfg.F; ++f) c.items.push_back(m.item0 + f);
  }
  double total = 0.0;
  std::vector<double> work(b->classes.size(), 0.0);
  for (size_t ci = 0; ci < b->classes.size(); ++ci) {
    Class& c = b->classes[ci];
    std::stable_sort(c.items.begin(), c.items.end(),
                     [&](size_t a, size_t z) { return b->items[a].T > b->items[z].T; });
    for (size_t id : c.items) work[ci] += item_cost(b->items[id], c.M, c.N);
    total += work[ci];
  }
  for (size_t ci = 0; ci < b->classes.size(); ++ci) {
    Class& c = b->classes[ci];
    const int per_sm = std::max(1, c.ops.em_blocks_per_sm[c.mm](c.bd));
    const double share = total > 0 ? work[ci] / total : 1.0;
    int grid = (int)std::lround(grid_factor * share * per_sm * b->sms);
    grid = std::max(1, std::min<int>(grid, (int)c.items.size()));
    c.grid = grid;
    std::vector<ffca::EmItem> h;
    h.reserve(c.items.size());
    for (size_t id : c.items) h.push_back(b->items[id]);
    BCK(b, ffca::dev_malloc(&c.d_items, sizeof(ffca::EmItem) * h.size()), "batch item alloc");
    BCK(b, cudaMemcpyAsync(c.d_items, h.data(), sizeof(ffca::EmItem) * h.size(), cudaMemcpyHostToDevice, b->stream),
        "batch item upload");
    BCK(b, ffca::dev_malloc(&c.d_counter, sizeof(int)), "batch counter alloc");
  }
  const fastfca_status st = ensure_side_streams(b, b->classes.size());
  if (st) return st;
  b->scheme = scheme;
  b->grid_factor = grid_factor;
  BCK(b, cudaStreamSynchronize(b->stream), "batch schedule upload");
  b->have_schedule = true;
  return FASTFCA_OK;
}

// Builds the schedule (scheme, grid_factor).  On failure the schedule (fallback_scheme,
// fallback_factor) is rebuilt when fallback_scheme >= 0; if that fails too, or there is none,
// the batch is left with no classes and fastfca_batch_iterate refuses it.  The first
// failure's status and message are returned.
fastfca_status build_classes(fastfca_batch* b, int scheme, double grid_factor, int fallback_scheme,
                             double fallback_factor) {
  const fastfca_status st = build_classes_once(b, scheme, grid_factor);
  if (st == FASTFCA_OK) return st;
  char msg[sizeof b->msg];
  snprintf(msg, sizeof msg, "%s", b->msg);
  free_graphs(b);
  free_classes(b);
  if (fallback_scheme >= 0 && build_classes_once(b, fallback_scheme, fallback_factor) != FASTFCA_OK) {
    free_graphs(b);
    free_classes(b);
  }
  snprintf(b->msg, sizeof b->msg, "%s", msg);
  return st;
}

// kMixture: each branch's mixtures, one single-mixture launch each (B = W^{-H} formed at the
// start of every launch), between start / end events of each mixture when `timed`.
fastfca_status enqueue_mixtures(fastfca_batch* b, int n_iter, cudaStream_t origin, bool timed) {
  BCK(b, cudaEventRecord(b->fork, origin), "fork record");
  for (size_t j = 0; j < b->branch_mix.size(); ++j) {
    cudaStream_t s = b->side[j];
    BCK(b, cudaStreamWaitEvent(s, b->fork, 0), "fork wait");
    for (int i : b->branch_mix[j]) {
      Mix& m = b->mix[i];
      ffca::EmArgs a{};
      a.x = m.x;
      a.xh = nullptr;
      a.P = m.P;
      a.lam = m.lam;
      a.v = m.v;
      a.ll_hist = nullptr;
      a.ll_last = m.ll_last;
      a.Bst = m.Bst;
      a.detst = m.detst;
      a.b_valid = 0;
      a.err = b->d_err;
      a.F = m.cfg.F;
      a.T = m.cfg.T;
      a.n_iter = n_iter;
      a.ll_stride = 0;
      a.N = m.cfg.N;
      a.clocks = nullptr;
      if (timed) BCK(b, cudaEventRecord(b->tev[2 * i], s), "mixture start record");
      const bool mm = m.cfg.model == FASTFCA_MODEL_FASTFCA_MM;
      BCK(b, mm ? m.ops.em_mm(a, s) : m.ops.em(a, s), "mixture launch");
      if (timed) BCK(b, cudaEventRecord(b->tev[2 * i + 1], s), "mixture end record");
    }
    BCK(b, cudaEventRecord(b->ev[j], s), "join record");
    BCK(b, cudaStreamWaitEvent(origin, b->ev[j], 0), "join wait");
  }
  return FASTFCA_OK;
}

// Enqueues every class launch: fork from `origin` onto side streams, join back onto it.
fastfca_status enqueue_all(fastfca_batch* b, int n_iter, cudaStream_t origin) {
  if (b->scheme == kMixture) return enqueue_mixtures(b, n_iter, origin, false);
  cudaEvent_t fork = b->fork;
  BCK(b, cudaEventRecord(fork, origin), "fork record");
  for (size_t ci = 0; ci < b->classes.size(); ++ci) {
    Class& c = b->classes[ci];
    cudaStream_t s = b->side[ci];
    BCK(b, cudaStreamWaitEvent(s, fork, 0), "fork wait");
    BCK(b, cudaMemsetAsync(c.d_counter, 0, sizeof(int), s), "counter reset");
    BCK(b, c.ops.em_persistent[c.mm](c.d_items, (int)c.items.size(), n_iter, c.d_counter, b->d_err, c.bd, c.grid, s),
        "persistent launch");
    BCK(b, cudaEventRecord(b->ev[ci], s), "join record");
    BCK(b, cudaStreamWaitEvent(origin, b->ev[ci], 0), "join wait");
  }
  return FASTFCA_OK;
}

fastfca_status graph_for(fastfca_batch* b, int n_iter, cudaGraphExec_t* out) {
  auto it = b->graphs.find(n_iter);
  if (it != b->graphs.end()) {
    *out = it->second;
    return FASTFCA_OK;
  }
  cudaGraph_t g = nullptr;
  if (!b->capture) BCK(b, cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
  BCK(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeRelaxed), "begin capture");
  fastfca_status st = enqueue_all(b, n_iter, b->capture);
  cudaError_t e = cudaStreamEndCapture(b->capture, &g);
  if (st != FASTFCA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BCK(b, e, "end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  BCK(b, e, "graph instantiate");
  b->graphs[n_iter] = exec;
  *out = exec;
  return FASTFCA_OK;
}

fastfca_status check_err(fastfca_batch* b) {
  int bits = 0;
  BCK(b, cudaMemcpyAsync(&bits, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "status read");
  BCK(b, cudaStreamSynchronize(b->stream), "batch synchronize");
  if (!bits) return FASTFCA_OK;
  BCK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "status clear");
  if (bits & ffca::kErrConfig) return bfail(b, FASTFCA_ECUDA, "batch launch configuration rejected (0x%x)", bits);
  return bfail(b, FASTFCA_ENUMERIC, "numerical failure in a batch kernel (bits 0x%x)", bits);
}

}  // namespace

extern "C" {

fastfca_status fastfca_batch_create(int32_t B, const fastfca_config* cfgs, const void* const* xs, void* stream,
                                    fastfca_batch** out) {
  FFCA_TRACE("fastfca_batch_create");
  if (!out) return bfail(nullptr, FASTFCA_EINVAL, "out is NULL");
  *out = nullptr;
  if (B < 1 || !cfgs || !xs) return bfail(nullptr, FASTFCA_EINVAL, "B >= 1, cfgs and xs are required");
  fastfca_batch* b = new (std::nothrow) fastfca_batch();
  if (!b) return bfail(nullptr, FASTFCA_ENOMEM, "host allocation failed");
  b->stream = (cudaStream_t)stream;
  auto bail = [&](fastfca_status st) {
    ffca::set_thread_error(b->msg);
    free_batch(b);
    delete b;
    return st;
  };
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  size_t n_items = 0;
  b->mix.resize(B);
  for (int i = 0; i < B; ++i) {
    const fastfca_config c = cfgs[i];
    Mix& m = b->mix[i];
    m.cfg = c;
    if (c.F < 1 || c.T < 1 || (c.model != FASTFCA_MODEL_FASTFCA && c.model != FASTFCA_MODEL_FASTFCA_MM) || !xs[i]) {
      bfail(b, FASTFCA_EINVAL, "mixture %d: bad config or NULL x", i);
      return bail(FASTFCA_EINVAL);
    }
    if (!ffca::fast_ops(c.M, c.N, &m.ops) || c.T > m.ops.max_T) {
      bfail(b, FASTFCA_EUNSUPPORTED, "mixture %d: no kernel for M=%d N=%d T=%d", i, c.M, c.N, c.T);
      return bail(FASTFCA_EUNSUPPORTED);
    }
    m.item0 = n_items;
    n_items += c.F;
  }
  fastfca_status st;
#define BCKC(expr, what)                                  \
  do {                                                    \
    cudaError_t e__ = (expr);                             \
    if (e__ != cudaSuccess) {                             \
      cudaGetLastError();                                 \
      bfail(b, FASTFCA_ECUDA, "%s: %s", what, cudaGetErrorString(e__)); \
      return bail(e__ == cudaErrorMemoryAllocation ? FASTFCA_ENOMEM : FASTFCA_ECUDA); \
    }                                                     \
  } while (0)
  BCKC(ffca::dev_malloc(&b->d_stamps, sizeof(unsigned long long) * 2 * n_items), "stamps alloc");
  BCKC(cudaMemsetAsync(b->d_stamps, 0, sizeof(unsigned long long) * 2 * n_items, b->stream), "stamps clear");
  BCKC(ffca::dev_malloc(&b->d_err, sizeof(int)), "status alloc");
  BCKC(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "status clear");
  b->items.resize(n_items);
  for (int i = 0; i < B; ++i) {
    Mix& m = b->mix[i];
    const fastfca_config& c = m.cfg;
    const size_t FT = (size_t)c.F * c.T;
    if (is_dev(xs[i])) {
      if (reinterpret_cast<uintptr_t>(xs[i]) % 16 != 0) {       // frames are loaded as 16-byte vectors
        bfail(b, FASTFCA_EINVAL, "mixture %d: a device x must start on a 16-byte boundary", i);
        return bail(FASTFCA_EINVAL);
      }
      m.x = static_cast<const float2*>(xs[i]);
    } else {
      BCKC(ffca::dev_malloc(&m.x_owned, sizeof(float2) * FT * c.M), "x alloc");
      BCKC(cudaMemcpyAsync(m.x_owned, xs[i], sizeof(float2) * FT * c.M, cudaMemcpyHostToDevice, b->stream), "x upload");
      m.x = m.x_owned;
    }
    BCKC(ffca::dev_malloc(&m.P, sizeof(double2) * (size_t)c.F * c.M * c.M), "P alloc");
    BCKC(ffca::dev_malloc(&m.lam, sizeof(float) * (size_t)c.F * c.M * c.N), "lam alloc");
    BCKC(ffca::dev_malloc(&m.v, sizeof(float) * FT * c.N), "v alloc");
    BCKC(ffca::dev_malloc(&m.Bst, sizeof(double2) * (size_t)c.F * c.M * c.M), "B alloc");
    BCKC(ffca::dev_malloc(&m.detst, sizeof(double) * 2 * (size_t)c.F), "det alloc");
    BCKC(ffca::dev_malloc(&m.ll_last, sizeof(double) * (size_t)c.F), "ll alloc");
    BCKC(ffca::dev_malloc(&m.flags, sizeof(int) * (size_t)c.F), "flag alloc");
    BCKC(ffca::dev_malloc(&m.winv, sizeof(float2) * (size_t)c.F * c.M * c.M), "winv alloc");
    BCKC(cudaMemsetAsync(m.flags, 0, sizeof(int) * (size_t)c.F, b->stream), "flag clear");
    const size_t n = ffca::default_params_elems(c.F, c.T, c.M, c.N);
    ffca::default_params_kernel<<<(unsigned)((n + 255) / 256), 256, 0, b->stream>>>(m.x, m.P, m.lam, m.v, c.F, c.T,
                                                                                     c.M, c.N, (uint32_t)c.seed);
    BCKC(cudaGetLastError(), "init launch");
    for (int f = 0; f < c.F; ++f) {
      ffca::EmItem& it = b->items[m.item0 + f];
      it.x = m.x + (size_t)f * c.T * c.M;
      it.P = m.P + (size_t)f * c.M * c.M;
      it.lam = m.lam + (size_t)f * c.M * c.N;
      it.v = m.v + (size_t)f * c.N * c.T;
      it.Bst = m.Bst + (size_t)f * c.M * c.M;
      it.detst = m.detst + 2 * (size_t)f;
      it.ll_hist = nullptr;
      it.ll_last = m.ll_last + f;
      it.clocks = nullptr;
      it.valid_flag = m.flags + f;
      it.stamp = b->d_stamps + 2 * (m.item0 + f);
      it.T = c.T;
      it.n_iter = 1;
      it.b_valid = 0;
    }
  }
  BCKC(cudaStreamSynchronize(b->stream), "create synchronize");
#undef BCKC
  st = build_classes(b, kFine, 1.0, -1, 0.0);
  if (st != FASTFCA_OK) return bail(st);
  *out = b;
  return FASTFCA_OK;
}

void fastfca_batch_destroy(fastfca_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  free_batch(b);
  delete b;
}

const char* fastfca_batch_last_error(const fastfca_batch* b) { return b ? b->msg : fastfca_last_error(nullptr); }

fastfca_status fastfca_batch_set_params(fastfca_batch* b, int32_t i, const void* P, const float* lam, const float* v) {
  if (!b) return FASTFCA_EINVAL;
  if (b->sticky == FASTFCA_ECUDA) return b->sticky;
  if (i < 0 || i >= (int)b->mix.size() || !P || !lam || !v) return bfail(b, FASTFCA_EINVAL, "bad mixture index or NULL");
  Mix& m = b->mix[i];
  const fastfca_config& c = m.cfg;
  BCK(b, copy_in(m.P, P, sizeof(double2) * (size_t)c.F * c.M * c.M, b->stream), "P upload");
  BCK(b, copy_in(m.lam, lam, sizeof(float) * (size_t)c.F * c.M * c.N, b->stream), "lam upload");
  BCK(b, copy_in(m.v, v, sizeof(float) * (size_t)c.F * c.T * c.N, b->stream), "v upload");
  BCK(b, cudaMemsetAsync(m.flags, 0, sizeof(int) * (size_t)c.F, b->stream), "flag clear");
  return FASTFCA_OK;
}

fastfca_status fastfca_batch_get_params(fastfca_batch* b, int32_t i, void* P, float* lam, float* v) {
  if (!b) return FASTFCA_EINVAL;
  if (b->sticky == FASTFCA_ECUDA) return b->sticky;
  if (i < 0 || i >= (int)b->mix.size()) return bfail(b, FASTFCA_EINVAL, "bad mixture index");
  Mix& m = b->mix[i];
  const fastfca_config& c = m.cfg;
  if (P) BCK(b, copy_out(P, m.P, sizeof(double2) * (size_t)c.F * c.M * c.M, b->stream), "P download");
  if (lam) BCK(b, copy_out(lam, m.lam, sizeof(float) * (size_t)c.F * c.M * c.N, b->stream), "lam download");
  if (v) BCK(b, copy_out(v, m.v, sizeof(float) * (size_t)c.F * c.T * c.N, b->stream), "v download");
  return check_err(b);
}

fastfca_status fastfca_batch_iterate(fastfca_batch* b, int32_t n_iter, double* ll_per_mixture,
                                     double* seconds_per_mixture) {
  FFCA_TRACE("fastfca_batch_iterate");
  if (!b) return FASTFCA_EINVAL;
  if (b->sticky == FASTFCA_ECUDA) return b->sticky;
  if (n_iter < 1) return bfail(b, FASTFCA_EINVAL, "n_iter must be >= 1");
  if (!b->have_schedule)
    return bfail(b, FASTFCA_EINVAL, "the batch has no schedule (building one failed); call fastfca_batch_schedule");
  const bool timed_mix = seconds_per_mixture && b->scheme == kMixture;
  if (timed_mix) {
    // per-mixture spans from events around each launch: the launches go out directly
    // (the same launches as the graph's), not through the graph
    while (b->tev.size() < 2 * b->mix.size()) {
      cudaEvent_t e;
      BCK(b, cudaEventCreate(&e), "timing event");
      b->tev.push_back(e);
    }
    const fastfca_status st = enqueue_mixtures(b, n_iter, b->stream, true);
    if (st) return st;
  } else {
    cudaGraphExec_t exec = nullptr;
    fastfca_status st = graph_for(b, n_iter, &exec);
    if (st) return st;
    BCK(b, cudaGraphLaunch(exec, b->stream), "graph launch");
  }
  if (!ll_per_mixture && !seconds_per_mixture) return FASTFCA_OK;
  // ENUMERIC still fills the outputs: mixtures are independent, the failed ones read
  // non-finite there and the others are valid.
  const fastfca_status num = check_err(b);
  if (num && num != FASTFCA_ENUMERIC) return num;
  if (ll_per_mixture) {
    for (size_t i = 0; i < b->mix.size(); ++i) {
      const Mix& m = b->mix[i];
      std::vector<double> ll(m.cfg.F);
      BCK(b, cudaMemcpy(ll.data(), m.ll_last, sizeof(double) * m.cfg.F, cudaMemcpyDeviceToHost), "ll download");
      double s = 0.0;
      for (double x : ll) s += x;
      ll_per_mixture[i] = s;
    }
  }
  if (timed_mix) {
    for (size_t i = 0; i < b->mix.size(); ++i) {
      float ms = 0.f;
      BCK(b, cudaEventElapsedTime(&ms, b->tev[2 * i], b->tev[2 * i + 1]), "mixture span");
      seconds_per_mixture[i] = (double)ms * 1e-3;
    }
  } else if (seconds_per_mixture) {
    std::vector<unsigned long long> st2(2 * b->items.size());
    BCK(b, cudaMemcpy(st2.data(), b->d_stamps, sizeof(unsigned long long) * st2.size(), cudaMemcpyDeviceToHost),
        "stamp download");
    for (size_t i = 0; i < b->mix.size(); ++i) {
      const Mix& m = b->mix[i];
      unsigned long long lo = ~0ULL, hi = 0;
      for (int f = 0; f < m.cfg.F; ++f) {
        lo = std::min(lo, st2[2 * (m.item0 + f)]);
        hi = std::max(hi, st2[2 * (m.item0 + f) + 1]);
      }
      seconds_per_mixture[i] = hi > lo ? (double)(hi - lo) * 1e-9 : 0.0;
    }
  }
  return num;
}

fastfca_status fastfca_batch_tune(fastfca_batch* b, int32_t n_iter, int32_t* chosen_scheme, double* chosen_factor) {
  FFCA_TRACE("fastfca_batch_tune");
  if (!b) return FASTFCA_EINVAL;
  if (b->sticky == FASTFCA_ECUDA) return b->sticky;
  if (n_iter < 1) return bfail(b, FASTFCA_EINVAL, "n_iter must be >= 1");
  const int orig_scheme = b->have_schedule ? b->scheme : -1;
  const double orig_factor = b->grid_factor;
  // snapshot the parameters: the probes iterate on them.  Every exit below frees the
  // snapshot and the events, and puts the parameters back once the snapshot is complete.
  struct Saved { double2* P = nullptr; float* lam = nullptr; float* v = nullptr; };
  std::vector<Saved> saved(b->mix.size());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fastfca_status st = FASTFCA_OK;
  bool snapped = false;
  for (size_t i = 0; i < b->mix.size() && !st; ++i) {
    const fastfca_config& c = b->mix[i].cfg;
    st = bcheck(b, ffca::dev_malloc(&saved[i].P, sizeof(double2) * (size_t)c.F * c.M * c.M), "tune snapshot");
    if (!st) st = bcheck(b, ffca::dev_malloc(&saved[i].lam, sizeof(float) * (size_t)c.F * c.M * c.N), "tune snapshot");
    if (!st) st = bcheck(b, ffca::dev_malloc(&saved[i].v, sizeof(float) * (size_t)c.F * c.T * c.N), "tune snapshot");
  }
  for (size_t i = 0; i < b->mix.size() && !st; ++i) {
    const Mix& m = b->mix[i];
    const fastfca_config& c = m.cfg;
    st = bcheck(b, cudaMemcpyAsync(saved[i].P, m.P, sizeof(double2) * (size_t)c.F * c.M * c.M, cudaMemcpyDeviceToDevice, b->stream), "snapshot");
    if (!st) st = bcheck(b, cudaMemcpyAsync(saved[i].lam, m.lam, sizeof(float) * (size_t)c.F * c.M * c.N, cudaMemcpyDeviceToDevice, b->stream), "snapshot");
    if (!st) st = bcheck(b, cudaMemcpyAsync(saved[i].v, m.v, sizeof(float) * (size_t)c.F * c.T * c.N, cudaMemcpyDeviceToDevice, b->stream), "snapshot");
  }
  snapped = !st;
  auto restore = [&]() -> fastfca_status {
    fastfca_status r = FASTFCA_OK;
    for (size_t i = 0; i < b->mix.size() && !r; ++i) {
      Mix& m = b->mix[i];
      const fastfca_config& c = m.cfg;
      r = bcheck(b, cudaMemcpyAsync(m.P, saved[i].P, sizeof(double2) * (size_t)c.F * c.M * c.M, cudaMemcpyDeviceToDevice, b->stream), "restore");
      if (!r) r = bcheck(b, cudaMemcpyAsync(m.lam, saved[i].lam, sizeof(float) * (size_t)c.F * c.M * c.N, cudaMemcpyDeviceToDevice, b->stream), "restore");
      if (!r) r = bcheck(b, cudaMemcpyAsync(m.v, saved[i].v, sizeof(float) * (size_t)c.F * c.T * c.N, cudaMemcpyDeviceToDevice, b->stream), "restore");
      if (!r) r = bcheck(b, cudaMemsetAsync(m.flags, 0, sizeof(int) * (size_t)c.F, b->stream), "restore");
    }
    return r;
  };
  if (!st) st = bcheck(b, cudaEventCreate(&e0), "tune event");
  if (!st) st = bcheck(b, cudaEventCreate(&e1), "tune event");
  const double factors[] = {1.0, 2.0, 4.0, 8.0};     // 8: the per-mixture schedule only (16 branches)
  float best_ms = 1e30f;
  int best_scheme = kFine;
  double best_factor = 1.0;
  for (int scheme = 0; scheme < kNumSchemes && !st; ++scheme) {
    for (double fac : factors) {
      if (fac > 4.0 && scheme != kMixture) continue;
      st = build_classes(b, scheme, fac, -1, 0.0);
      if (st) break;
      st = restore();
      if (st) break;
      cudaEventRecord(e0, b->stream);
      st = enqueue_all(b, n_iter, b->stream);
      if (st) break;
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = bfail(b, FASTFCA_ECUDA, "tune probe failed"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best_scheme = scheme; best_factor = fac; }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (snapped) {
    const fastfca_status r = restore();
    if (!st) st = r;
    if (!st) st = bcheck(b, cudaStreamSynchronize(b->stream), "restore synchronize");
    else cudaStreamSynchronize(b->stream);     // the snapshot is read until here
  }
  for (auto& sv : saved) {
    ffca::dev_free(sv.P);
    ffca::dev_free(sv.lam);
    ffca::dev_free(sv.v);
  }
  if (st) {
    // back to the schedule the batch had before tuning (a failed probe may have replaced it)
    char msg[sizeof b->msg];
    snprintf(msg, sizeof msg, "%s", b->msg);
    if (orig_scheme >= 0) build_classes(b, orig_scheme, orig_factor, -1, 0.0);
    snprintf(b->msg, sizeof b->msg, "%s", msg);
    return st;
  }
  st = build_classes(b, best_scheme, best_factor, orig_scheme, orig_factor);
  if (st) return st;
  if (chosen_scheme) *chosen_scheme = best_scheme;
  if (chosen_factor) *chosen_factor = best_factor;
  return check_err(b);
}

fastfca_status fastfca_batch_schedule(fastfca_batch* b, int32_t scheme, double grid_factor) {
  FFCA_TRACE("fastfca_batch_schedule");
  if (!b) return FASTFCA_EINVAL;
  if (b->sticky == FASTFCA_ECUDA) return b->sticky;
  if (scheme < 0 || scheme >= kNumSchemes || !(grid_factor > 0.0)) return bfail(b, FASTFCA_EINVAL, "bad schedule");
  return build_classes(b, scheme, grid_factor, b->have_schedule ? b->scheme : -1, b->grid_factor);
}

fastfca_status fastfca_batch_separate(fastfca_batch* b, int32_t i, void* c) {
  FFCA_TRACE("fastfca_batch_separate");
  if (!b) return FASTFCA_EINVAL;
  if (b->sticky == FASTFCA_ECUDA) return b->sticky;
  if (i < 0 || i >= (int)b->mix.size() || !c) return bfail(b, FASTFCA_EINVAL, "bad mixture index or NULL c");
  Mix& m = b->mix[i];
  const fastfca_config& cf = m.cfg;
  if (!is_dev(c)) return bfail(b, FASTFCA_EINVAL, "c must be a device pointer");
  BCK(b, m.ops.winv(m.P, m.winv, cf.F, b->d_err, b->stream), "winv launch");
  BCK(b, m.ops.mwf(m.x, m.P, m.winv, m.lam, m.v, static_cast<float2*>(c), cf.F, cf.T, cf.N, 1, b->stream), "filter launch");
  return FASTFCA_OK;
}

}  // extern "C"

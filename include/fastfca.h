/*
 * fastfca.h -- C ABI of the GB300 FastFCA library (libfastfca.so).
 *
 * FastFCA (Ito, Ikeshita, Sawada, Nakatani, "A Joint Diagonalization Based Efficient
 * Approach to Underdetermined Blind Audio Source Separation Using the Multichannel Wiener
 * Filter") separates N sources from an M-channel STFT mixture x(t, f).  Every source n has
 * the spatial covariance R_n(f) = W_f^{-H} diag(lambda_n(f)) W_f^{-1} (Sec. IV-B, Eq. 19)
 * with one joint diagonaliser W_f per frequency, and power v_n(t, f) (Sec. III-A, Eq. 4).
 * The library estimates (W, lambda, v) by the IP+EM algorithm (Sec. IV-E, Algorithm 1),
 * evaluates the log-likelihood (Eq. 31), and separates the sources with the multichannel
 * Wiener filter (Sec. IV-F, Eq. 39).  The plain full-rank FCA model (Sec. III, EM of
 * Eq. 12-13, one explicit M x M inverse per time-frequency bin) is available as the
 * comparison model.
 *
 * Names: the paper's W (the joint diagonaliser, "P_f" elsewhere), L ([L]_{mn} = lambda_n,m)
 * and H ([H]_{nt} = v_n(t)); frames are t = 0..T-1 (the paper's j), frequencies f = 0..F-1
 * (the paper's i), microphones m = 0..M-1, sources n = 0..N-1.
 *
 * Layouts (all row-major, C order, interleaved complex (re, im)):
 *   x      complex64  [F][T][M]        the mixture, m fastest
 *   P      complex128 [F][M][M]        P[f][a][m] = W_f[a, m]; column m is w_m
 *   lam    float32    [F][M][N]        lam[f][m][n] = [L_f]_{mn}
 *   v      float32    [F][N][T]        v[f][n][t] = [H_f]_{nt}
 *   c      complex64  [F][T][N][M]     separated source images
 *   R      complex128 [F][N][M][M]     FCA spatial covariances (FCA model only)
 *   h      float32    [F][N][T]        FCA source powers (FCA model only)
 *
 * Pointers: every array argument may be a host pointer or a device pointer of the current
 * device; the library tells them apart with cudaPointerGetAttributes.  Host arrays are
 * copied on the context's stream inside the call (the call then synchronises that stream).
 * Device arrays are used in place, asynchronously on the stream, except where a call says it
 * synchronises.
 *
 * Ownership: a device x given to fastfca_create is borrowed, not copied: the caller keeps it
 * alive and unchanged until fastfca_destroy.  A host x is copied into a device buffer the
 * context owns.  The context owns its parameter and workspace buffers; output buffers (c,
 * parameter copies) belong to the caller.
 *
 * Errors: every call returns a fastfca_status.  No C++ exception crosses the ABI.  A
 * FASTFCA_ECUDA status is sticky (later calls on the context return it).  A FASTFCA_ENUMERIC
 * status stays until fastfca_set_params (or set_params_fca / set_params_mnmf) replaces the
 * parameters: meanwhile fastfca_iterate, fastfca_loglik and fastfca_separate return it
 * without launching, and the get_params calls still work.  fastfca_last_error gives a
 * one-line message.  Numerical trouble found by a kernel (a non-finite or non-positive
 * sigma^2, a Q_m that is not numerically positive definite, a singular W) is recorded on the
 * device and reported by the next call that synchronises.
 *
 * Input that makes the model degenerate: a non-finite x (NaN or Inf) gives FASTFCA_ENUMERIC
 * within the first iterations.  An x_ft that is exactly zero (digital silence) has no
 * maximum-likelihood variance, since sigma^2 -> 0 raises the likelihood without bound.  IP+EM
 * and FCA by EM shrink that bin's power geometrically and stay finite for many iterations.
 * IP+MM and FCA by MM set it to exactly zero in their first update, and FastMNMF does the
 * same for a frame that is zero at every frequency (its v is shared across frequencies); all
 * three then report FASTFCA_ENUMERIC in the next iteration.  Drop such frames or add dither at
 * the noise floor.
 *
 * Threads: a context may be used by one host thread at a time.
 */
#ifndef FASTFCA_H
#define FASTFCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FASTFCA_OK = 0,
  FASTFCA_EINVAL = 1,        /* invalid argument (null pointer, size out of range, ...) */
  FASTFCA_ENOMEM = 2,        /* a device allocation failed */
  FASTFCA_ECUDA = 3,         /* a CUDA call or kernel launch failed */
  FASTFCA_ENUMERIC = 4,      /* non-finite or non-positive quantity met by a kernel */
  FASTFCA_EUNSUPPORTED = 5   /* valid request for which the library has no kernel */
} fastfca_status;

typedef enum {
  FASTFCA_MODEL_FASTFCA = 0,    /* joint-diagonalisation model, Sec. IV, IP+EM (Algorithm 1) */
  FASTFCA_MODEL_FCA = 1,        /* full-rank FCA, Sec. III (comparison model) */
  FASTFCA_MODEL_FASTFCA_MM = 2, /* the FastFCA model fitted by IP+MM (Algorithm 2); same
                                   parameters, calls and shapes as FASTFCA */
  FASTFCA_MODEL_FCA_MM = 3,     /* full-rank FCA fitted by MM (Eq. 15-17, geometric-mean R
                                   update); same parameters and calls as FCA */
  FASTFCA_MODEL_FASTMNMF = 4    /* FastMNMF (Sec. IV-H, App. C): FastFCA with the source powers
                                   factored across frequencies, h_ijn = sum_k t_ikn v_jkn
                                   (Eq. 52); created by fastfca_create_mnmf */
} fastfca_model;

typedef struct {
  int32_t F;      /* frequency bins, >= 1 */
  int32_t T;      /* frames, >= 1 (FastFCA: up to what eight CTAs' shared memory holds, ~11k at M=8, N=12) */
  int32_t M;      /* microphones: FastFCA and FastMNMF 2..8, FCA 2..4 */
  int32_t N;      /* sources: FastFCA and FastMNMF 1..16, FCA 2..8 */
  int32_t model;  /* fastfca_model */
  int32_t seed;   /* seed of the default initial v (Philox4x32-10); any value */
} fastfca_config;

typedef struct fastfca_ctx fastfca_ctx;

/* Creates a context for the mixture x (complex64 [F][T][M], host or device; a device x is
 * borrowed and must start on a 16-byte boundary, EINVAL otherwise) on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The parameters start at W = I,
 * lambda = 1 and v[n][t] = ||x_t||^2 / (M N) * u, u ~ U[0.5, 1.5) drawn from Philox4x32-10
 * keyed by cfg->seed with counter (f, n, t, 0x1d17) (FCA: R_n = I, h = the same v).  The random
 * factor breaks the symmetry between sources that equal starting values would keep forever.
 * Callers may overwrite the start with fastfca_set_params.  Sec. II defines the problem: estimate the source
 * images c given x and N.  Returns EINVAL for sizes out of range, EUNSUPPORTED for an (M, N)
 * without a kernel, ENOMEM/ECUDA on allocation or copy failure; *out is NULL then. */
fastfca_status fastfca_create(const fastfca_config* cfg, const void* x, void* stream,
                              fastfca_ctx** out);

/* Piecewise-stationary FastFCA (Sec. VI-B): the T frames of x (complex64 [F][T][M], host or
 * device, as for fastfca_create) are partitioned into J = T / B blocks of B consecutive
 * frames, and the model is fitted to X^_j = (1/B) sum_b x x^H (the paper's Eq. 44 cost) by
 * Algorithm 1 or 2 (cfg->model FASTFCA or FASTFCA_MM).  Every parameter call then has J
 * columns where fastfca_create's contexts have T: v float32 [F][N][J], the log-likelihood
 * is Eq. 44's (per block).  fastfca_separate filters every frame with the powers of its
 * block (c complex64 [F][T][N][M]).  B = 1 is fastfca_create.  EINVAL unless B divides T,
 * or for a model other than FASTFCA and FASTFCA_MM; EUNSUPPORTED for the (M, N, J) that
 * fastfca_create would reject with J frames. */
fastfca_status fastfca_create_blocks(const fastfca_config* cfg, int32_t B, const void* x, void* stream,
                                     fastfca_ctx** out);

/* Replaces the FastFCA parameters: P complex128 [F][M][M], lam float32 [F][M][N],
 * v float32 [F][N][T] (each host or device).  All three are required.  Clears a sticky
 * ENUMERIC and the log-likelihood history. */
fastfca_status fastfca_set_params(fastfca_ctx* ctx, const void* P, const float* lam, const float* v);

/* Copies the current FastFCA parameters into caller buffers (host or device, any may be
 * NULL to skip).  Synchronises the stream. */
fastfca_status fastfca_get_params(fastfca_ctx* ctx, void* P, float* lam, float* v);

/* FastMNMF (App. C): the FastFCA model in every frequency i (demixing W_i, weights
 * lambda_imn) with the source powers h_ijn = sum_k t_ikn v_jkn (Eq. 52) shared across
 * frequencies through the activations v, fitted by minimising Eq. 53.  One fastfca_iterate
 * iteration runs IP (Eq. 33-35) in every frequency, then the exponent-1/2 multiplicative MM
 * updates of lambda, t and v in that order (the rules Algorithm 2 gives for L and H, applied to
 * each factor; sigma^2 recomputed before each); the v update sums over all frequencies.
 * cfg->model must be FASTFCA_MODEL_FASTMNMF; K is the number of bases per source, 1..16;
 * the shapes fastfca_create takes (M 2..8, N 1..16, T as the kernels fit), F*K <= 36864.
 * x as for fastfca_create.  The default start is W = I,
 * lambda = 1, t_ikn = (mean_j p_ij / K) u, v_jkn = (mean_i p_ij / mean p) u', p_ij =
 * ||x_ij||^2 / (M N), u and u' ~ U[0.5, 1.5) from Philox4x32-10 keyed by cfg->seed.
 * fastfca_iterate, fastfca_loglik (Eq. 53 negated, with -M T ln(pi) per frequency),
 * fastfca_separate (Eq. 39 with h from Eq. 52), fastfca_set_mixture, fastfca_sync and
 * fastfca_destroy take the context.  Errors as for fastfca_create, EINVAL for K out of range. */
fastfca_status fastfca_create_mnmf(const fastfca_config* cfg, int32_t K, const void* x, void* stream,
                                   fastfca_ctx** out);

/* FastMNMF parameters (host or device): W complex128 [F][M][M] (W[a][m] at (f*M + a)*M + m),
 * lam float32 [F][M][N], t float32 [F][N][K] (t_ikn at (i*N + n)*K + k), v float32 [N][K][T]
 * (v_jkn at (n*K + k)*T + j).  set: all four required; get: NULL skips, synchronises. */
fastfca_status fastfca_set_params_mnmf(fastfca_ctx* ctx, const void* W, const float* lam, const float* t,
                                       const float* v);
fastfca_status fastfca_get_params_mnmf(fastfca_ctx* ctx, void* W, float* lam, float* t, float* v);

/* FCA models (FCA, FCA_MM): replaces R complex128 [F][N][M][M] and h float32 [F][N][T]. */
fastfca_status fastfca_set_params_fca(fastfca_ctx* ctx, const void* R, const float* h);

/* FCA models: copies R and h out (host or device; NULL skips).  Synchronises. */
fastfca_status fastfca_get_params_fca(fastfca_ctx* ctx, void* R, float* h);

/* Runs n_iter iterations of the model's algorithm on every frequency: FastFCA IP+EM
 * (Algorithm 1, Sec. IV-E), FastFCA IP+MM (Algorithm 2), FCA EM (Eq. 12-13), FCA MM
 * (Eq. 15-17) or FastMNMF (App. C; see fastfca_create_mnmf).  n_iter >= 1.  If ll_per_iter is not
 * NULL (host or device, n_iter doubles) it receives the total log-likelihood sum_f l_f
 * after each iteration,
 * l_f = T ln|det W_f|^2 - sum_{m,t} (|y_mt|^2 / sigma^2_mt + ln sigma^2_mt) - M T ln(pi)
 * (Eq. 31 negated, with its constant).  Stream-ordered and asynchronous: a host
 * ll_per_iter (pinned for a truly asynchronous copy) is complete once the context's stream
 * has passed the call, e.g. after fastfca_sync, which also reports the kernels' numerical
 * status (ENUMERIC). */
fastfca_status fastfca_iterate(fastfca_ctx* ctx, int32_t n_iter, double* ll_per_iter);

/* Log-likelihood of the current parameters: *ll_total (host, may be NULL) = sum_f l_f and
 * ll_per_f (host or device, may be NULL) = l_f for each f.  Synchronises. */
fastfca_status fastfca_loglik(fastfca_ctx* ctx, double* ll_total, double* ll_per_f);

/* Source images by the multichannel Wiener filter of the current parameters: FastFCA
 * Eq. 39 (c = W^{-H} diag(g_n) W^H x), FCA (both fits) Eq. 7 (c = h_n R_n X^{-1} x).  c is complex64
 * [F][T][N][M], host or device, caller-allocated.  Stream-ordered and asynchronous for both:
 * a host c (pinned for a truly asynchronous copy) holds the images once the context's
 * stream has passed the call, e.g. after fastfca_sync, which also reports any kernel
 * status of the filter.  c must start on an 8-byte boundary (EINVAL otherwise).  For a host c
 * the images pass through a device staging buffer of the same size, which the context makes
 * on the first such call (ENOMEM if that fails) and keeps until fastfca_destroy. */
fastfca_status fastfca_separate(fastfca_ctx* ctx, void* c);

/* Replaces the mixture of a context with another of the same shape (complex64 [F][T][M],
 * host or device), for running many mixtures through one context without reallocating.
 * The data is copied, stream-ordered, into a buffer the context owns (allocated on the
 * first call when the context was created on a borrowed device mixture); the caller may
 * reuse x once the stream has passed the copy.  The parameters are left as they are.
 * Sec. II: the input of the method is the mixture x and N. */
fastfca_status fastfca_set_mixture(fastfca_ctx* ctx, const void* x);

/* Waits for the context's stream and reports kernel-side numerical errors. */
fastfca_status fastfca_sync(fastfca_ctx* ctx);

/* One-line description of the last error on ctx (or of the last failed create when ctx is
 * NULL).  The string lives until the next call on the same context. */
const char* fastfca_last_error(const fastfca_ctx* ctx);

/* Frees everything the context owns (never the borrowed device x).  NULL is a no-op. */
void fastfca_destroy(fastfca_ctx* ctx);

/* Library version string. */
const char* fastfca_version(void);

/* Fault injection for the error paths, decided on the host (nothing reaches the GPU).  After
 * n further device allocations by the library succeed, the next one fails as an out of memory
 * would: the call that made it returns FASTFCA_ENOMEM and frees what it had allocated, and a
 * context or batch it was called on stays usable.  One-shot; n < 0 disarms.  Process-wide. */
void fastfca_debug_fail_alloc(int64_t n);

/* Device allocations the library holds now, over all contexts, batches and networks of the
 * process (with fastfca_debug_fail_alloc: a failed call leaves this count where it was). */
int64_t fastfca_debug_live_allocs(void);

/* Kernel choice for IP+EM (Algorithm 1) on the large-bin shapes (M > 4, or N > 8, or T > 2048),
 * for tests that run both kernels on one shape: 0 (the default) picks by shape, 1 takes the
 * thread-block-cluster kernel, 2 the one-SM kernel wherever it fits (T <= 4096).  Read when a
 * context is created; host state, process-wide; any other value is ignored.  Both kernels
 * compute the same steps in the same order; their results differ by FP32 rounding. */
void fastfca_debug_large_bin_kernel(int32_t which);

/* Failure injection for the cluster kernel's bounded waits (the wait of each source's exchange
 * between the CTAs of a cluster, Algorithm 1's n-loop): spins > 0 sets the number of polls
 * after which an exchange is reported as timed out, 0 restores the kernel's default (2^20).
 * A timed-out exchange sets a status bit, so the next synchronising call returns ECUDA and the
 * context stays failed; the kernel keeps waiting, bounded by the default, for the bytes
 * already on their way, so no memory is written after the wait.  Read at each launch; host
 * state, process-wide. */
void fastfca_debug_cluster_wait_limit(int32_t spins);

/* Measurement, not part of the method: the FP32 FMA rate of the current GPU in TFLOP/s (2 flops
 * per FMA), from one timed launch of iters x 128 dependent-free FMAs per thread on every SM at
 * full occupancy, after one untimed launch.  The denominator of the arithmetic roofline the
 * benchmark reports beside the one from unit counts.  Synchronises; allocates a small buffer.
 * EINVAL for iters < 1 or a null tflops; ECUDA on a failed launch. */
fastfca_status fastfca_measure_fp32_fma(int32_t iters, double* tflops, void* stream);

/* Check, not part of the method: the library's FP64 reciprocal and reciprocal square root of a
 * positive normal number (an FP32 hardware approximation refined by one Newton-Raphson step,
 * used by the IP of Eq. 34-35) applied to n device doubles x into device rcp and rsqrt, so a
 * test can compare them with CUDA's correctly rounded 1/x and 1/sqrt(x).  Asynchronous on the
 * stream; EINVAL for n < 1 or a null pointer. */
fastfca_status fastfca_debug_f64_reciprocals(int32_t n, const double* x, double* rcp, double* rsqrt, void* stream);

/* ------------------------------------------------------------------------------------------
 * Batches: many independent mixtures (mixed M, N, T) iterated together in one CUDA-graph
 * launch.  Each (mixture, frequency) pair is one work item run by one CTA with the same code
 * as the single-mixture path.  Two kinds of schedule: (a) items grouped into classes by
 * (M, N) and a frame bucket, each class one persistent launch whose CTAs take items
 * longest-first from an atomic counter, all classes concurrent on forked streams; (b) one
 * single-mixture launch per mixture (one CTA per frequency), the mixtures spread
 * longest-first over concurrent branches.  Either is captured once per n_iter in one graph.
 * (Not in the paper: FastFCA processes frequencies independently, Sec. IV-G, so independent
 * mixtures batch naturally.)
 */
typedef struct fastfca_batch fastfca_batch;

/* Creates a batch of B FastFCA mixtures: cfgs[b] (model FASTFCA for IP+EM, Algorithm 1, or
 * FASTFCA_MM for IP+MM, Algorithm 2; mixtures may differ) and xs[b] (complex64 [F][T][M],
 * host or device; device arrays are borrowed and must start on a 16-byte boundary, EINVAL
 * otherwise).  Parameters start as in
 * fastfca_create.  The initial schedule is the finest bucketing with one grid share per
 * class; fastfca_batch_tune picks a measured one. */
fastfca_status fastfca_batch_create(int32_t B, const fastfca_config* cfgs, const void* const* xs, void* stream,
                                    fastfca_batch** out);

/* Replaces mixture b's parameters (layouts as fastfca_set_params; host or device). */
fastfca_status fastfca_batch_set_params(fastfca_batch* batch, int32_t b, const void* P, const float* lam,
                                        const float* v);

/* Copies mixture b's parameters out (host or device; NULL skips).  Synchronises. */
fastfca_status fastfca_batch_get_params(fastfca_batch* batch, int32_t b, void* P, float* lam, float* v);

/* Runs n_iter iterations (IP+EM, Algorithm 1, or IP+MM, Algorithm 2, as each mixture's
 * config.model says) on every frequency of every mixture with one graph launch (the graph is
 * captured on first use of each n_iter and reused).  Optional host outputs: ll_per_mixture[b]
 * = sum_f l_f after the last iteration; seconds_per_mixture[b] = the span between the first
 * start and the last end of mixture b's items inside the launch (%globaltimer; under schedule
 * 3 the time between CUDA events around mixture b's launch, which then goes out directly
 * rather than through the graph).  With either
 * output the call synchronises; otherwise it is asynchronous.  Mixtures are independent: on
 * FASTFCA_ENUMERIC the outputs are still filled, ll_per_mixture[b] is non-finite for each
 * mixture that failed, and the others' results are valid.  A failed mixture keeps reporting
 * ENUMERIC until fastfca_batch_set_params replaces its parameters. */
fastfca_status fastfca_batch_iterate(fastfca_batch* batch, int32_t n_iter, double* ll_per_mixture,
                                     double* seconds_per_mixture);

/* Autotuner: times every candidate schedule (frame bucketing: fine / coarse / one per (M, N),
 * with grid share factor 1, 2 or 4; or one launch per mixture on 2, 4, 8 or 16 branches) on this
 * batch with n_iter iterations, restores the parameters, and keeps the fastest.  *scheme and
 * *factor (may be NULL) receive the choice. */
fastfca_status fastfca_batch_tune(fastfca_batch* batch, int32_t n_iter, int32_t* scheme, double* factor);

/* Sets a schedule directly (scheme 0 fine, 1 coarse, 2 one per (M, N): factor > 0 scales each
 * class's persistent grid; scheme 3 one launch per mixture: round(2 factor) branches). */
fastfca_status fastfca_batch_schedule(fastfca_batch* batch, int32_t scheme, double factor);

/* Wiener-filter separation of mixture b into c (complex64 [F][T][N][M], device). */
fastfca_status fastfca_batch_separate(fastfca_batch* batch, int32_t b, void* c);

/* Last error message of the batch (or of the last failed batch create when NULL). */
const char* fastfca_batch_last_error(const fastfca_batch* batch);

/* Frees everything the batch owns (never borrowed device mixtures). */
void fastfca_batch_destroy(fastfca_batch* batch);

/* Largest F*M*M that fastfca_separate_noalloc accepts (complex64 values of its static
 * scratch: 512 KiB of device memory). */
#define FASTFCA_NOALLOC_MAX_FMM 65536

/* The Wiener-filter separation of fastfca_separate (Eq. 39), for callers that must not
 * allocate device memory, with no context.  The paper has no counterpart: this is a
 * deployment variant.  Who needs it: code that separates audio inside a real-time callback
 * (or another section where an allocation may block the thread or synchronise the device
 * and so miss a deadline) cannot call cudaMalloc there.  This call allocates nothing: the
 * caller supplies every input and the output, and the one intermediate (W^{-H}, F*M*M
 * complex64 values) lives in a fixed array compiled into the library, present in the
 * memory of every GPU that loads it until the process exits.
 *
 *   x    complex64  [F][T][M]  device     P    complex128 [F][M][M]  device
 *   lam  float32    [F][M][N]  device     v    float32    [F][N][T]  device
 *   c    complex64  [F][T][N][M] device (output, caller-allocated)
 * x and P must start on a 16-byte boundary, c on an 8-byte and lam and v on a 4-byte boundary
 * (EINVAL otherwise, checked before any device work).  Any T is accepted.
 *   stream  cudaStream_t (NULL = legacy default stream)
 *
 * Returns EINVAL when F*M*M > FASTFCA_NOALLOC_MAX_FMM, a size is not positive, a pointer is
 * NULL or not a device pointer; EUNSUPPORTED for an (M, N) without a kernel; ECUDA when a
 * launch fails.  The message is in fastfca_last_error(NULL).  Asynchronous on the stream;
 * it reports no kernel-side numerical status.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress): make that call before any stream capture.
 * All calls share the array, which keeps the last call's contents: calls that overlap on
 * the GPU (other streams, other host threads) race on it and must be serialised.  The
 * looked-up address is kept for the process: do not call this on a device after
 * cudaDeviceReset. */
fastfca_status fastfca_separate_noalloc(int32_t F, int32_t T, int32_t M, int32_t N, const void* x,
                                        const void* P, const float* lam, const float* v, void* c,
                                        void* stream);

/* ---------------------------------------------------------------------------------------
 * Learned initialiser (not in the paper: its initialisation is mask-based, Sec. VII, and it
 * leaves the choice of a better starting point open).  A small network maps statistics of
 * each frequency of a mixture to a starting point (W, L, H) of Algorithm 1:
 *
 *   features phi (16 floats per frequency): the upper triangle of R / tr R, R = (1/T) sum_t
 *     x_t x_t^H (the M diagonal reals, then (re, im) of each a < b pair), ln(tr R / M), the mean
 *     and standard deviation over t of p_t = ln(||x_t||^2 / M), f / (F - 1), 1, zeros to 16;
 *     q_t = p_t - mean_t p (T floats per frequency).
 *   network: h1 = gelu(W1 phi + b1), h2 = gelu(W2 h1 + b2), o = W3 h2 + b3; hidden 256,
 *     gelu(z) = z Phi(z).  o holds W (2M^2 reals, row-major complex), ln L (M N, m-major) and a
 *     per-source bias b_n; o is padded to 40 columns.
 *   per-frame powers: ln v[n][t] = c_n + b_n + sum_{j<9} k[n][j] q_{t+j-4} (zero outside [0, T)).
 *   loss of one frequency against a converged (W*, L*, H*): W's columns to unit norm (row m
 *     of L divided by ||w_m||^2, the same covariances), l = ln L - mean_m ln L,
 *     h = ln v + mean_m ln L; the channel permutation sigma that best matches the unit
 *     columns, then the source permutation pi that best matches l and mean_t h (first in
 *     lexicographic order on ties);  loss = sum_m (1 - |u_sigma(m)^H u*_m|^2)
 *     + sum_{m,n} (l[sigma(m)][pi(n)] - l*[m][n])^2 + (1/T) sum_{n,t} (h[pi(n)][t] - h*[n][t])^2,
 *     averaged over the rows of a batch.
 * Products run on the tensor cores (tcgen05.mma: operands rounded to BF16, FP32 accumulators in
 * tensor memory; a product whose completion wait runs out makes the net's next synchronising
 * call return ECUDA); the rest in
 * FP32.  Parameters are one flat FP32 vector: W1 [256][16], b1 [256], W2 [256][256], b2 [256],
 * W3 [40][256], b3 [40], k [N][9], c [N].  The network supports M in {2, 3}, N <= 5 and
 * 2 M^2 + M N + N <= 40.  A "row" is one frequency of one mixture.  Unless stated otherwise
 * arrays are device memory and calls are asynchronous on the given stream.
 * --------------------------------------------------------------------------------------- */
typedef struct fastfca_net fastfca_net;

/* Synthetic training mixtures from the model of Sec. IV (the same recipe as the tests' data):
 * x[b][f][t] = sum_n sqrt(v_n(f,t)) chol(a_n a_n^H + 0.01 I) z, v_n(f,t) = sum_{k<K} B A with
 * B, A ~ Exp(1), a_n the steering vector of a linear array (spacing metres, 16 kHz, 343 m/s)
 * for a direction uniform in [0, pi), z ~ CN(0, I); all draws from Philox4x32-10 keyed by
 * seed.  x: complex64 [B][F][T][M], device.  M <= 3, N <= 5. */
fastfca_status fastfca_generate_mixtures(int32_t B, int32_t F, int32_t T, int32_t M, int32_t N, int32_t K,
                                         double spacing, uint64_t seed, void* x, void* stream);

/* Features of `rows` frequencies: x complex64 [rows][T][M] (row r is frequency r % F of its
 * mixture) -> feats float32 [rows][16], q float32 [rows][T].  Device arrays. */
fastfca_status fastfca_net_features(int32_t rows, int32_t F, int32_t T, int32_t M, const void* x, float* feats,
                                    float* q, void* stream);

/* Training targets from converged parameters (layouts of fastfca_set_params with F = rows):
 * wt float32 [rows][M][M][2] (unit columns), lt float32 [rows][M][N], ht float32 [rows][N][T].
 * Device arrays. */
fastfca_status fastfca_net_targets(int32_t rows, int32_t T, int32_t M, int32_t N, const void* P, const float* lam,
                                   const float* v, float* wt, float* lt, float* ht, void* stream);

/* Creates a network for (M, N) with workspace for batches of up to max_rows rows of up to
 * max_T frames (max_T (N + 1) 4 bytes <= 200 KiB).  Weights start uniform in +-sqrt(3/fan_in)
 * (Philox4x32-10, seed), the last layer 100x smaller, with b3 holding W = I.  Adam moments
 * start at zero.  EUNSUPPORTED outside the supported (M, N). */
fastfca_status fastfca_net_create(int32_t M, int32_t N, int32_t max_rows, int32_t max_T, uint64_t seed, void* stream,
                                  fastfca_net** out);

/* Number of FP32 parameters of the flat vector. */
int64_t fastfca_net_param_count(const fastfca_net* net);

/* Copies the parameter vector out / in (host or device; synchronises). */
fastfca_status fastfca_net_get_params(fastfca_net* net, float* out);
fastfca_status fastfca_net_set_params(fastfca_net* net, const float* in);

/* Network output o float32 [rows][40] (host or device; synchronises) for feats [rows][16]. */
fastfca_status fastfca_net_forward(fastfca_net* net, int32_t rows, const float* feats, float* out);

/* Batch loss and gradients: the mean loss goes to *loss (host; synchronises when not NULL),
 * the gradient of every parameter (the flat layout) to grads (host or device; NULL keeps it
 * in the network only). */
fastfca_status fastfca_net_loss_grad(fastfca_net* net, int32_t rows, int32_t T, const float* feats, const float* q,
                                     const float* wt, const float* lt, const float* ht, double* loss, float* grads);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) at learning rate lr on one batch; the mean loss
 * before the step goes to *loss when not NULL (synchronises). */
fastfca_status fastfca_net_train_step(fastfca_net* net, int32_t rows, int32_t T, const float* feats, const float* q,
                                      const float* wt, const float* lt, const float* ht, float lr, double* loss);

/* Starting point of Algorithm 1 for `rows` frequencies: P complex128 [rows][M][M],
 * lam float32 [rows][M][N], v float32 [rows][N][T] (device; the layouts of
 * fastfca_set_params with F = rows). */
fastfca_status fastfca_net_predict(fastfca_net* net, int32_t rows, int32_t T, const float* feats, const float* q,
                                   void* P, float* lam, float* v);

/* Last error message of the network (or of the last failed call without one when NULL). */
const char* fastfca_net_last_error(const fastfca_net* net);

/* Frees the network. */
void fastfca_net_destroy(fastfca_net* net);

#ifdef __cplusplus
}
#endif

#endif /* FASTFCA_H */

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
 * FASTFCA_ECUDA status is sticky (later calls on the context return it); a FASTFCA_ENUMERIC
 * status is cleared by fastfca_set_params.  fastfca_last_error gives a one-line message.
 * Numerical trouble found by a kernel (a non-positive sigma^2, a non-positive-definite Q_m)
 * is recorded on the device and reported by the next call that synchronises.
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
  FASTFCA_EUNSUPPORTED = 5   /* valid request for which this build has no kernel */
} fastfca_status;

typedef enum {
  FASTFCA_MODEL_FASTFCA = 0, /* joint-diagonalisation model, Sec. IV */
  FASTFCA_MODEL_FCA = 1      /* full-rank FCA, Sec. III (comparison model) */
} fastfca_model;

typedef struct {
  int32_t F;      /* frequency bins, >= 1 */
  int32_t T;      /* frames, >= 1 (FastFCA: <= 2048 in this build) */
  int32_t M;      /* microphones: 2, 3 or 4 in this build */
  int32_t N;      /* sources: 2..8 in this build */
  int32_t model;  /* fastfca_model */
  int32_t reserved;
} fastfca_config;

typedef struct fastfca_ctx fastfca_ctx;

/* Creates a context for the mixture x (complex64 [F][T][M], host or device) on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The parameters start at W = I,
 * lambda = 1 and v = ||x_t||^2 / (M N) (FCA: R_n = I, h = the same v); callers normally
 * overwrite them with fastfca_set_params.  Sec. II defines the problem: estimate the source
 * images c given x and N.  Returns EINVAL for sizes out of range, EUNSUPPORTED for an (M, N)
 * without a kernel, ENOMEM/ECUDA on allocation or copy failure; *out is NULL then. */
fastfca_status fastfca_create(const fastfca_config* cfg, const void* x, void* stream,
                              fastfca_ctx** out);

/* Replaces the FastFCA parameters: P complex128 [F][M][M], lam float32 [F][M][N],
 * v float32 [F][N][T] (each host or device).  All three are required.  Clears a sticky
 * ENUMERIC and the log-likelihood history. */
fastfca_status fastfca_set_params(fastfca_ctx* ctx, const void* P, const float* lam, const float* v);

/* Copies the current FastFCA parameters into caller buffers (host or device, any may be
 * NULL to skip).  Synchronises the stream. */
fastfca_status fastfca_get_params(fastfca_ctx* ctx, void* P, float* lam, float* v);

/* FCA model: replaces R complex128 [F][N][M][M] and h float32 [F][N][T]. */
fastfca_status fastfca_set_params_fca(fastfca_ctx* ctx, const void* R, const float* h);

/* FCA model: copies R and h out (host or device; NULL skips).  Synchronises. */
fastfca_status fastfca_get_params_fca(fastfca_ctx* ctx, void* R, float* h);

/* Runs n_iter iterations of the model's algorithm on every frequency: FastFCA IP+EM
 * (Algorithm 1, Sec. IV-E) or FCA EM (Eq. 12-13).  n_iter >= 1.  If ll_per_iter is not
 * NULL it receives (host) the total log-likelihood sum_f l_f after each iteration,
 * l_f = T ln|det W_f|^2 - sum_{m,t} (|y_mt|^2 / sigma^2_mt + ln sigma^2_mt) - M T ln(pi)
 * (Eq. 31 negated, with its constant); the call then synchronises.  Otherwise it is
 * asynchronous. */
fastfca_status fastfca_iterate(fastfca_ctx* ctx, int32_t n_iter, double* ll_per_iter);

/* Log-likelihood of the current parameters: *ll_total (host, may be NULL) = sum_f l_f and
 * ll_per_f (host or device, may be NULL) = l_f for each f.  Synchronises. */
fastfca_status fastfca_loglik(fastfca_ctx* ctx, double* ll_total, double* ll_per_f);

/* Source images by the multichannel Wiener filter of the current parameters: FastFCA
 * Eq. 39 (c = W^{-H} diag(g_n) W^H x), FCA Eq. 7 (c = h_n R_n X^{-1} x).  c is complex64
 * [F][T][N][M], host or device, caller-allocated.  Asynchronous for a device c. */
fastfca_status fastfca_separate(fastfca_ctx* ctx, void* c);

/* Waits for the context's stream and reports kernel-side numerical errors. */
fastfca_status fastfca_sync(fastfca_ctx* ctx);

/* One-line description of the last error on ctx (or of the last failed create when ctx is
 * NULL).  The string lives until the next call on the same context. */
const char* fastfca_last_error(const fastfca_ctx* ctx);

/* Frees everything the context owns (never the borrowed device x).  NULL is a no-op. */
void fastfca_destroy(fastfca_ctx* ctx);

/* Library version string. */
const char* fastfca_version(void);

/* ------------------------------------------------------------------------------------------
 * Batches: many independent mixtures (mixed M, N, T) iterated together in one CUDA-graph
 * launch.  Each (mixture, frequency) pair is one work item run by one CTA with the same code
 * as the single-mixture path; items are grouped into classes by (M, N) and a frame bucket,
 * each class is one persistent launch whose CTAs take items longest-first from an atomic
 * counter, and all classes run concurrently on forked streams inside one captured graph.
 * (Not in the paper: FastFCA processes frequencies independently, Sec. IV-G, so independent
 * mixtures batch naturally.)
 */
typedef struct fastfca_batch fastfca_batch;

/* Creates a batch of B FastFCA mixtures: cfgs[b] (model must be FASTFCA) and xs[b] (complex64
 * [F][T][M], host or device; device arrays are borrowed).  Parameters start as in
 * fastfca_create.  The initial schedule is the finest bucketing with one grid share per
 * class; fastfca_batch_tune picks a measured one. */
fastfca_status fastfca_batch_create(int32_t B, const fastfca_config* cfgs, const void* const* xs, void* stream,
                                    fastfca_batch** out);

/* Replaces mixture b's parameters (layouts as fastfca_set_params; host or device). */
fastfca_status fastfca_batch_set_params(fastfca_batch* batch, int32_t b, const void* P, const float* lam,
                                        const float* v);

/* Copies mixture b's parameters out (host or device; NULL skips).  Synchronises. */
fastfca_status fastfca_batch_get_params(fastfca_batch* batch, int32_t b, void* P, float* lam, float* v);

/* Runs n_iter IP+EM iterations (Algorithm 1) on every frequency of every mixture with one
 * graph launch (the graph is captured on first use of each n_iter and reused).  Optional host
 * outputs: ll_per_mixture[b] = sum_f l_f after the last iteration; seconds_per_mixture[b] =
 * the span between the first start and the last end of mixture b's items inside the launch
 * (%globaltimer).  With either output the call synchronises; otherwise it is asynchronous. */
fastfca_status fastfca_batch_iterate(fastfca_batch* batch, int32_t n_iter, double* ll_per_mixture,
                                     double* seconds_per_mixture);

/* Autotuner: times every candidate schedule (frame bucketing: fine / coarse / one per (M, N);
 * grid share factor 1, 2 or 4) on this batch with n_iter iterations, restores the parameters,
 * and keeps the fastest.  *scheme and *factor (may be NULL) receive the choice. */
fastfca_status fastfca_batch_tune(fastfca_batch* batch, int32_t n_iter, int32_t* scheme, double* factor);

/* Sets a schedule directly (scheme 0 fine, 1 coarse, 2 one per (M, N); factor > 0). */
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
 *   stream  cudaStream_t (NULL = legacy default stream)
 *
 * Returns EINVAL when F*M*M > FASTFCA_NOALLOC_MAX_FMM, a size is not positive, a pointer is
 * NULL or not a device pointer; EUNSUPPORTED for an (M, N) without a kernel; ECUDA when a
 * launch fails.  The message is in fastfca_last_error(NULL).  Asynchronous on the stream;
 * it reports no kernel-side numerical status.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress): make that call before any stream capture.
 * All calls share the array, which keeps the last call's contents: calls that overlap on
 * the GPU (other streams, other host threads) race on it and must be serialised. */
fastfca_status fastfca_separate_noalloc(int32_t F, int32_t T, int32_t M, int32_t N, const void* x,
                                        const void* P, const float* lam, const float* v, void* c,
                                        void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTFCA_H */

/*
 * fpw.h -- C ABI of the GB300 FPW periodogram library (libfpw_gb300.so).
 *
 * Fast Periodicity Weighting (Finkbeiner, Prince & Whitebook,
 * arXiv:2502.00243). For a light curve with observation times t_i, fluxes x_i
 * and errors sigma_i, and a trial frequency f, the library evaluates Eq. 1
 * (Section 2, eq:phasesum):
 *
 *     w_i  = 1 / sigma_i^2,                 a_i = x_i w_i
 *     m_i  = floor(M * frac(t_i f))         (Appendix A.1 phase bin, t_ref = 0,
 *                                            zero-indexed 0..M-1)
 *     A_m  = sum_{i: m_i = m} a_i,          B_m = sum_{i: m_i = m} w_i
 *     S(f) = sum_m A_m^2 / (B_m + 1/alpha^2)
 *
 * for every (light curve, trial frequency) pair, and the post-processing step
 * of Section 3.5 (the highest peaks of each periodogram).
 *
 * Conventions shared by every entry point:
 *  - Arrays are caller-owned. Unless an entry point says "host", every pointer
 *    is a DEVICE pointer on the context's device (e.g. a torch CUDA tensor's
 *    data_ptr()). The library never frees caller memory.
 *  - Times are used as given (t_ref = 0): subtract a reference epoch first if
 *    |t f| would exceed about 2^40 cycles. Fluxes are used as given: the
 *    library does not subtract the mean (Section 3.5 calls that
 *    pre-processing, not part of FPW).
 *  - A bin whose denominator B_m + 1/alpha^2 is 0 (an empty bin with
 *    1/alpha^2 = 0) contributes 0. Bins are half-open [m/M, (m+1)/M).
 *  - A peak is a local maximum S_k > S_{k-1} and S_k >= S_{k+1}, with
 *    out-of-range neighbours taken as -infinity; peaks are ranked by S
 *    descending, ties to the lower frequency index. Missing peaks are reported
 *    as index -1 and S = NaN.
 *  - Return value: FPW_OK (0) or one of the FPW_E* codes below. No C++
 *    exception crosses this ABI. Entry points without the _ex suffix are
 *    synchronous and report data errors directly; _ex entry points are
 *    stream-ordered and latch device-detected data errors in the context,
 *    reported by fpw_ctx_status().
 */
#ifndef FPW_GB300_H
#define FPW_GB300_H

#include <stdint.h>

#if defined(__GNUC__) || defined(__clang__)
#define FPW_API __attribute__((visibility("default")))
#else
#define FPW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define FPW_OK 0
#define FPW_EINVAL 1   /* bad argument: null pointer, M < 1, negative size, bad offsets, k out of range */
#define FPW_EDATA 2    /* sigma <= 0 or a non-finite t, x, sigma or frequency (found on the device) */
#define FPW_ENOMEM 3   /* device or host allocation failed */
#define FPW_ECUDA 4    /* a CUDA runtime call failed */
#define FPW_ETIMEOUT 5 /* a bounded device-side wait gave up */
#define FPW_ENOTSUP 6  /* combination of options not supported */

/* Phase arithmetic (how frac(t f) is formed on the device). */
#define FPW_PHASE_FIXED64 0 /* default: exact integer product of the binary64 significands of t and the
                               anchor frequency, then 64-bit fixed-point stepping across the grid */
#define FPW_PHASE_FP64 1    /* plain form: fl(t f) - floor(fl(t f)) in binary64 per evaluation,
                               binary64 bin sums, one launch per curve */
#define FPW_PHASE_FP32 2    /* FP32 phase: anchor rounded to FP32 every K frequencies, FP32 steps */

#define FPW_ACCUM_FP32 0      /* bin sums A_m, B_m in FP32 (default) */
#define FPW_ACCUM_FP64 1      /* bin sums in binary64 */
#define FPW_ACCUM_FP32_COMP 2 /* compensated FP32 bin sums: each term enters as an FP32 hi + lo pair and
                                 every addition's rounding error is carried in a second FP32 sum
                                 (about 48 significant bits; batched and single-curve calls) */

#define FPW_PEAK_LOCALMAX 0 /* top-k over local maxima of S (default) */
#define FPW_PEAK_RAW 1      /* top-k over every frequency */

#define FPW_MAX_TOPK 64 /* largest k accepted by the batched calls */

typedef struct fpw_ctx fpw_ctx; /* opaque: device, scratch buffers, plan and graph caches */

typedef struct fpw_params {
  double inv_alpha2;    /* 1/alpha^2 >= 0 in Eq. 1's denominator (default 0: the prior is neglected) */
  int phase_mode;       /* FPW_PHASE_* (default FPW_PHASE_FIXED64) */
  int accum;            /* FPW_ACCUM_* (default FPW_ACCUM_FP32) */
  int K;                /* FPW_PHASE_FP32 only: re-anchor interval in frequencies (default 256) */
  int peak_mode;        /* FPW_PEAK_* (default FPW_PEAK_LOCALMAX) */
  int threads;          /* 0 = tuned; else threads per block (multiple of 32, 32..512) */
  int freqs_per_thread; /* 0 = tuned; else 1, 2, 4 or 8, or 3, 5 or 6 with FPW_ACCUM_FP32 on a call of one M
                           (FPW_ENOTSUP on the other calls) */
  int obs_chunk;        /* 0 = tuned; else observations staged in shared memory per pass (>= 32) */
  int use_graph;        /* 1 = capture the launch sequence in a CUDA graph and replay it on identical calls */
  int items_per_slot;   /* 0 = tuned (default 8); else the persistent schedule's work items per resident block:
                           each curve's frequency range is cut into segments of about total cost /
                           (items_per_slot x resident blocks), longest first (>= 1) */
} fpw_params;

/* Fill *p with the defaults listed above. */
FPW_API void fpw_params_default(fpw_params* p);

/* Create a context on CUDA device `device` (>= 0). *ctx receives the handle.
 * Errors: FPW_EINVAL (null ctx, bad device), FPW_ECUDA, FPW_ENOMEM. */
FPW_API int fpw_ctx_create(fpw_ctx** ctx, int device);

/* Synchronize the context's work, free its scratch memory and graphs. NULL is a no-op. */
FPW_API int fpw_ctx_destroy(fpw_ctx* ctx);

/* Synchronize the stream of the context's last call and return, then clear,
 * the status latched by device-side checks (FPW_OK, FPW_EDATA or FPW_ETIMEOUT). */
FPW_API int fpw_ctx_status(fpw_ctx* ctx);

/* Single light curve, Eq. 1 at every frequency (Section 2; the frequency sweep of Section 4).
 *   t, x, sigma: device float64[n] (times in days, fluxes, errors > 0), any order
 *   freqs:       device float64[nfreq] trial frequencies (any values; linear grids take the fast path)
 *   M:           number of phase bins, >= 1
 *   S_out:       device float64[nfreq], receives S(f_k)
 * Uses an internal per-device context, the legacy default stream and default
 * parameters, and synchronizes before returning.
 * Errors: FPW_EINVAL, FPW_EDATA (S_out then holds NaN), FPW_ECUDA, FPW_ENOMEM. */
FPW_API int fpw_periodogram(const double* t, const double* x, const double* sigma, int64_t n, const double* freqs,
                    int64_t nfreq, int M, double* S_out);

/* As fpw_periodogram, on context `ctx`, stream `stream` (a cudaStream_t, NULL =
 * legacy default stream) and parameters `params` (NULL = defaults).
 * Stream-ordered: returns after enqueueing; data errors are latched in ctx. */
FPW_API int fpw_periodogram_ex(fpw_ctx* ctx, void* stream, const fpw_params* params, const double* t, const double* x,
                       const double* sigma, int64_t n, const double* freqs, int64_t nfreq, int M, double* S_out);

/* Ragged batch of independent light curves with per-curve top-k peaks
 * (Eq. 1 per curve and frequency; Section 3.5 post-processing).
 *   offsets:       device int64[ncurves + 1], CSR offsets into t/x/sigma; offsets[0] = 0,
 *                  non-decreasing (empty curves allowed: S = 0 everywhere)
 *   t, x, sigma:   device float64[offsets[ncurves]]
 *   freqs:         device float64[nfreq], one grid shared by all curves
 *   M:             phase bins (>= 1);  k: peaks per curve (0 <= k <= min(FPW_MAX_TOPK, ...))
 *   topk_idx:      device int32[ncurves * k], frequency indices of the peaks (row per curve)
 *   topk_S:        device float32[ncurves * k], their S values
 * Synchronous, internal context, default parameters.
 * Errors: FPW_EINVAL, FPW_EDATA (bad curves get -1 / NaN), FPW_ECUDA, FPW_ENOMEM. */
FPW_API int fpw_periodogram_batch(const int64_t* offsets, int64_t ncurves, const double* t, const double* x,
                          const double* sigma, const double* freqs, int64_t nfreq, int M, int k, int32_t* topk_idx,
                          float* topk_S);

/* As fpw_periodogram_batch on ctx/stream/params.
 *   offsets_host: optional HOST copy of offsets (NULL: the library copies the
 *                 device offsets to the host, which synchronizes `stream`)
 *   S_out:        optional device float64[ncurves * nfreq] dense periodograms (NULL: not written)
 *   topk_idx/topk_S may be NULL when k == 0.
 * With params->phase_mode == FPW_PHASE_FP64 the plain binary64 form runs:
 * one launch per curve, binary64 phases and sums (M <= 100, else FPW_ENOTSUP). */
FPW_API int fpw_periodogram_batch_ex(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                             const int64_t* offsets_host, int64_t ncurves, const double* t, const double* x,
                             const double* sigma, const double* freqs, int64_t nfreq, int M, int k,
                             int32_t* topk_idx, float* topk_S, double* S_out);

/* Several bin counts from one pass (Section 3.4): the bin sums at M_max bins
 * are combined into M = M_max / g bins for each requested group g, with each
 * of the g bin offsets o (combined bin j holds the M_max-bins (j g + o + u) mod
 * M_max, u < g; the offset shifts every bin edge by o / M_max of a cycle).
 * For each curve and group the periodogram reported is S_g(f) = the largest S
 * over the g offsets (ties to the lower offset), and its peaks are ranked as
 * in fpw_periodogram_batch.
 *   groups:      HOST int[ngroups], 1 <= ngroups <= 8, each g in [1, 64] dividing M_max
 *   topk_idx:    device int32[ncurves * ngroups * k], row (c * ngroups + q) per curve and group
 *   topk_offset: device int32[ncurves * ngroups * k], the offset o of each peak (-1 if none)
 *   topk_S:      device float32[ncurves * ngroups * k]
 *   S_out:       optional device float64[ncurves * ngroups * nfreq], S_g(f) per curve and group
 * Other arguments as fpw_periodogram_batch_ex. FP32 sums only and at most 256
 * threads per block (FPW_ENOTSUP otherwise); nfreq < 2^25 when k > 0.
 * (M_max; groups) = (60; 3, 6, 15), (40; 2, 4, 10) and (20; 1, 2, 4), listed in
 * that order, run a combination compiled for them (same results bit for bit,
 * 7-14 % faster at the default shapes). Stream-ordered. */
FPW_API int fpw_periodogram_batch_multi(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                                        const int64_t* offsets_host, int64_t ncurves, const double* t,
                                        const double* x, const double* sigma, const double* freqs, int64_t nfreq,
                                        int M_max, const int* groups, int ngroups, int k, int32_t* topk_idx,
                                        int32_t* topk_offset, float* topk_S, double* S_out);

/* Curves that share one set of observation times (Section 4 and the batch
 * routine of Appendix D: many light curves of one field observed in the same
 * exposures). Eq. 1 per curve with the bins computed once per (observation,
 * frequency); on GB300 the bin sums of 64 curves at a time are one tensor-core
 * product of the fp16 hi/lo split of (x w, w) with the one-hot bin matrix
 * (FP32 accumulation), so the result matches FP32 bin sums of the batched call.
 *   t:        device float64[n], the shared times (finite)
 *   x, sigma: device float64[ncurves * n], curve c's values at [c * n + i]
 *   freqs:    device float64[nfreq] (any grid; phases are exact per frequency)
 *   M:        1 <= M <= 256
 *   k, topk_idx, topk_S, S_out: as fpw_periodogram_batch_ex (S_out optional,
 *             float64[ncurves * nfreq], the FP32 statistic widened)
 * params: FPW_PHASE_FIXED64 and FPW_ACCUM_FP32 only (FPW_ENOTSUP otherwise);
 * inv_alpha2 and peak_mode apply. A curve with sigma <= 0 or a non-finite value
 * gets S = NaN and no peaks (status FPW_EDATA). Scratch held by the context:
 * 8 n bytes per curve (rounded up to 64 curves x 32 observations) and, when
 * k > 0, a dense FP32 periodogram of 4 ncurves nfreq bytes.
 * Stream-ordered. Errors: FPW_EINVAL, FPW_ENOTSUP, FPW_ENOMEM, FPW_ECUDA. */
FPW_API int fpw_periodogram_shared(fpw_ctx* ctx, void* stream, const fpw_params* params, const double* t, int64_t n,
                                   int64_t ncurves, const double* x, const double* sigma, const double* freqs,
                                   int64_t nfreq, int M, int k, int32_t* topk_idx, float* topk_S, double* S_out);

/* FPW with a polynomial baseline drift marginalised instead of subtracted
 * (Appendix A.1-A.2: the general form the paper derives before neglecting the
 * baseline). Data covariance C_B + C_sigma with C_B = B B^T, B[i, k] =
 * beta T_k(tau_i) for k < K (Chebyshev polynomials of the first kind in the
 * curve's times mapped to [-1, 1] over its span), and
 *   S = u^T (I / alpha^2 + E^T W E)^-1 u,  u = E^T W x,  W = (C_B + C_sigma)^-1,
 * E the one-hot bin matrix; with 1/alpha^2 = 0 empty bins are dropped. K = 0
 * (or beta = 0) gives Eq. 1. Bin sums are FP32, the per-frequency K x K solve
 * binary64.
 *   offsets, t, x, sigma, freqs, k, topk_idx, topk_S, S_out: as
 *       fpw_periodogram_batch_ex (device pointers; ncurves <= 65535)
 *   K: 0..4 basis functions; beta >= 0: prior standard deviation of each
 *       basis coefficient, in flux units
 *   M: 1 <= M, with 32 M b + 128 * 36 bytes within the device's shared
 *       memory per block, b = 8 (K <= 1), 16 (K = 2, 3) or 20 (K = 4) bytes
 *       per bin (FPW_ENOTSUP beyond)
 * params: FPW_PHASE_FIXED64 and FPW_ACCUM_FP32 only; inv_alpha2 and
 * peak_mode apply; threads (32..128) and freqs_per_thread (1 or 2) set the
 * block shape (0 = 128 threads, fewer where M needs it, and two frequencies
 * per thread for K <= 1 where they fit); a shape whose bins do not fit (R
 * times the bound on M above) or any other value gives FPW_ENOTSUP.
 * Scratch held by the context: 32 bytes per observation,
 * 168 bytes per curve and,
 * when k > 0, a dense FP32 periodogram of 4 ncurves nfreq bytes. Reads
 * offsets[ncurves] back to the host (synchronizes `stream` once).
 * Errors: FPW_EINVAL, FPW_ENOTSUP, FPW_ENOMEM, FPW_ECUDA; invalid data in a
 * curve gives S = NaN and no peaks for it (status FPW_EDATA). */
FPW_API int fpw_periodogram_drift(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                                  int64_t ncurves, const double* t, const double* x, const double* sigma,
                                  const double* freqs, int64_t nfreq, int M, int K, double beta, int k,
                                  int32_t* topk_idx, float* topk_S, double* S_out);

/* Phase entropy (Appendix C) of one set of observation times at every trial
 * frequency: H(f) = -sum_m (N_m/N) log(N_m/N), N_m the observations in phase bin
 * m (bins as the periodogram kernels assign them), natural logarithm, FP32.
 * The paper computes it once per field (it depends on the times only) to flag
 * periods whose phase coverage is uneven.
 *   t: device float64[n] (finite); freqs: device float64[nfreq]; 1 <= M <= 256;
 *   H_out: device float32[nfreq]. Stream-ordered. Errors: FPW_EINVAL, FPW_ECUDA. */
FPW_API int fpw_phase_entropy(fpw_ctx* ctx, void* stream, const double* t, int64_t n, const double* freqs,
                              int64_t nfreq, int M, float* H_out);

/* Phase entropy at each reported peak of a batch (Appendix C, the paper's ZTF
 * practice) and its z-score against Hutcheson's approximations for equally
 * likely bins: E(H) = log M - (M-1)/(2N) - (M-1)(M+1)/(12N^2),
 * Var(H) = (M-1)/(2N^2) + (M^2-1)/(6N^3), z = (H - E)/sqrt(Var).
 *   offsets, t, freqs: as for the batch call (device); topk_idx: device
 *   int32[ncurves * k] (e.g. fpw_periodogram_batch's output; -1 or out-of-range
 *   entries give NaN); H_out, z_out: device float32[ncurves * k]; 1 <= M <= 4096.
 * Stream-ordered. Errors: FPW_EINVAL, FPW_ECUDA. */
FPW_API int fpw_phase_entropy_peaks(fpw_ctx* ctx, void* stream, const int64_t* offsets, int64_t ncurves,
                                    const double* t, const double* freqs, int64_t nfreq, int M, int k,
                                    const int32_t* topk_idx, float* H_out, float* z_out);

/* End-to-end form with HOST buffers: copies the inputs to context-owned device
 * memory, runs fpw_periodogram_batch_ex, copies the top-k back and
 * synchronizes. All pointers are host pointers (pinned memory copies fastest).
 * Same arguments and errors as fpw_periodogram_batch_ex, minus S_out. */
FPW_API int fpw_periodogram_batch_host(fpw_ctx* ctx, const fpw_params* params, const int64_t* offsets, int64_t ncurves,
                               const double* t, const double* x, const double* sigma, const double* freqs,
                               int64_t nfreq, int M, int k, int32_t* topk_idx, float* topk_S);

/* The batched call with a bin dump: runs exactly the kernels that
 * fpw_periodogram_batch_ex runs for the same arguments and params (same kernel
 * shape, tiles, phase anchors and stepping; params->use_graph is ignored), with
 * no peaks, and additionally writes the phase bin (Appendix A.1, 0..M-1) that
 * the periodogram kernel gave every observation at every frequency k with
 * k0 <= k < k1, from the same arithmetic that forms the bin sums:
 *   bins_out: device int32[(k1 - k0) * offsets[ncurves]], entry
 *             [(k - k0) * offsets[ncurves] + i] for observation i (CSR index)
 *   S_out:    optional device float64[ncurves * nfreq] dense periodograms
 * Entries of curves with invalid data (status FPW_EDATA) are left unwritten.
 * 0 <= k0 <= k1 <= nfreq. Other arguments as fpw_periodogram_batch_ex.
 * Stream-ordered. Errors: FPW_EINVAL, FPW_ENOTSUP, FPW_ENOMEM, FPW_ECUDA. */
FPW_API int fpw_periodogram_batch_bins(fpw_ctx* ctx, void* stream, const fpw_params* params, const int64_t* offsets,
                                       const int64_t* offsets_host, int64_t ncurves, const double* t,
                                       const double* x, const double* sigma, const double* freqs, int64_t nfreq,
                                       int M, int64_t k0, int64_t k1, int32_t* bins_out, double* S_out);

/* fpw_periodogram_batch without any device allocation. (The paper has no
 * counterpart: this is a deployment variant of the batched call.)
 * For callers that cannot call cudaMalloc: code that runs inside another
 * framework's memory pool, plugins whose host forbids device allocation after
 * start-up, and real-time pipelines that must not risk an allocation failure or
 * an implicit device synchronization mid-run. All scratch memory lives in one
 * file-scope device array of 32 MiB that every GPU loading the library holds
 * until the process exits; inputs and outputs are still the caller's.
 *   Arguments as fpw_periodogram_batch_ex (device pointers; offsets_host is an
 *   optional host copy of offsets, else the offsets are read back to host
 *   memory and checked there: offsets[0] = 0, non-decreasing, offsets[ncurves]
 *   <= 2^40, FPW_EINVAL otherwise), minus S_out. One work item per curve,
 *   largest curves first. phase_mode FPW_PHASE_FP64 is not supported.
 *   Limit: 320 + 16*C + 4*(C+1) + C + 12*C*k + 8*(nobs+2) bytes (16*(nobs+2)
 *   with FPW_ACCUM_FP64 or FPW_ACCUM_FP32_COMP), each term rounded up to 256,
 *   must fit in 32 MiB (about 4 million observations); larger inputs return
 *   FPW_EINVAL.
 *   The first call on a device (with that device current) looks up the
 *   array's device address; make it before any stream capture. Every call
 *   shares the array and clears what must start at zero; calls that overlap
 *   on the GPU race. Synchronizes `stream` before returning.
 * Errors: FPW_EINVAL, FPW_EDATA, FPW_ENOTSUP, FPW_ECUDA, FPW_ETIMEOUT. */
FPW_API int fpw_periodogram_batch_noalloc(void* stream, const fpw_params* params, const int64_t* offsets,
                                          const int64_t* offsets_host, int64_t ncurves, const double* t,
                                          const double* x, const double* sigma, const double* freqs, int64_t nfreq,
                                          int M, int k, int32_t* topk_idx, float* topk_S);

/* Tuned kernel shapes. Adds a shape -- threads per block (multiple of 32,
 * 32..512), frequencies per thread (1, 2, 3, 4, 5, 6 or 8), observations per
 * pass (0 = largest that keeps two blocks per SM) and work items per resident
 * block (0 = 8; see fpw_params.items_per_slot) -- used for batched and single
 * calls whose bin count lies in [M_lo, M_hi] and whose observation-weighted
 * mean curve size lies in [n_lo, n_hi). Later entries take precedence; explicit
 * fpw_params fields override the table. An entry's 3, 5 or 6 frequencies per
 * thread apply to calls of one M with FP32 sums; the other calls in its range
 * take 2 or 4 instead. The autotuner
 * (paper_2502_00243_gb300/autotune.py) measures candidates and fills it.
 * Errors: FPW_EINVAL for an empty range or an invalid shape. */
FPW_API int fpw_ctx_set_shape(fpw_ctx* ctx, int M_lo, int M_hi, int64_t n_lo, int64_t n_hi, int threads,
                              int freqs_per_thread, int obs_chunk, int items_per_slot);
FPW_API int fpw_ctx_clear_shapes(fpw_ctx* ctx);

/* The tile-kernel shape of the context's most recent batched or single-curve
 * call that ran the tile kernel: threads per block, frequencies per thread,
 * observations staged per pass and the persistent grid (blocks). All zero
 * before the first such call. Pass the first three as fpw_params threads /
 * freqs_per_thread / obs_chunk to launch another call with the same tiles.
 * Errors: FPW_EINVAL (null pointer). */
FPW_API int fpw_ctx_last_shape(fpw_ctx* ctx, int* threads, int* freqs_per_thread, int* obs_chunk, int* grid);

/* Limit, in SM clock cycles, of each wait inside the pipeline of the
 * shared-timestamp kernel (fpw_periodogram_shared: its builder, copy and
 * tensor-core roles wait on each other through mbarriers). 0 restores the
 * default of 4e9 cycles (about 2 s). A wait that runs out makes the kernel
 * stop its work, wait (with the default limit) for its own bulk copies and
 * tensor-core operations in flight, free its tensor memory and return; the
 * call's status is then FPW_ETIMEOUT (fpw_ctx_status), and the context stays
 * usable. Errors: FPW_EINVAL (null ctx, clocks < 0). */
FPW_API int fpw_ctx_set_wait_limit(fpw_ctx* ctx, int64_t clocks);

/* Profiling hook. While enabled, the context records a pair of CUDA events on
 * the caller's stream around every launch of the periodogram kernel (the
 * persistent tile kernel; not in calls that use a CUDA graph).
 * fpw_ctx_kernel_time waits for those events, returns in *ms the summed
 * kernel time and in *launches the number of launches since the previous
 * query, then resets both. */
FPW_API int fpw_ctx_set_timing(fpw_ctx* ctx, int enable);
FPW_API int fpw_ctx_kernel_time(fpw_ctx* ctx, double* ms, int64_t* launches);

/* Human-readable text for a status code (static storage). */
FPW_API const char* fpw_strerror(int status);

/* Library ABI version (increments on incompatible changes; 2: fpw_debug_bins
 * replaced by fpw_periodogram_batch_bins, fpw_params.items_per_slot added,
 * fpw_ctx_set_shape takes items_per_slot). */
FPW_API int fpw_version(void);

/* Text of the last CUDA runtime error seen by the calling thread (static,
 * thread-local storage; empty if none). */
FPW_API const char* fpw_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FPW_GB300_H */

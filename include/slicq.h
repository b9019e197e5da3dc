/*
 * slicq.h — C ABI of the GB300 sliCQ library (libslicq.so).
 *
 * The sliced constant-Q nonstationary Gabor transform (sliCQ) of Holighaus,
 * Doerfler, Velasco and Grill, "A framework for invertible, real-time
 * constant-Q transforms" (arXiv:1210.0084):
 *   forward  = Algorithm 3 (sliCQ analysis), each slice by Algorithm 1,
 *   inverse  = Algorithm 4 (sliCQ synthesis), each slice by Algorithm 2 with
 *              the canonical dual of Proposition 2 (eq. painlessframe2),
 *   adjoint  = the adjoint of the forward map (frame synthesis with the
 *              analysis windows, Sec. 2.1 eq. frameop), used as its gradient.
 *
 * Conventions shared by every entry point
 *   - Signals are real float32, channel-major: d_f[b * n_samples + t],
 *     b < batch, t < n_samples.
 *   - Coefficients are complex float32 stored as interleaved (re, im) pairs,
 *     slice-major: coefficient n of channel k of slice m of signal b is the
 *     pair at index ((b * S + m) * C_s + off_k + n), with S =
 *     slicq_num_slices(), C_s = coefs_per_slice, off_k = sum_{i<k} M_i,
 *     n < M_k, k = 0..K+1 (the channels that a real signal needs, Table 1;
 *     channels K+2..2K+1 are the complex conjugates of K..1).  The paper's
 *     2-layer array s^l (Sec. 4.1) is the index map l = m mod 2,
 *     n_layer = (n + (m-1) M_k / 2) mod (S M_k / 2).
 *   - Coefficients are the frame coefficients c_{n,k} = <f^m, phi_{n,k}>
 *     with the unitary DFT of Sec. 2.1 (eq. CQ_coeff).
 *   - All pointers named d_* are device pointers on the plan's device and are
 *     owned by the caller.  Host pointers are named h_*.
 *   - Calls that take a stream are asynchronous on that stream.  They return
 *     argument errors before launching anything and launch errors at once;
 *     faults inside a kernel surface at the next synchronising call.
 *   - No entry point allocates device memory except slicq_plan_create,
 *     slicq_batch_create and slicq_stream_create (the objects they create
 *     own it until destroyed) and slicq_selftest_wait (one int, freed
 *     before it returns).  A plan's creation also allocates and frees
 *     scratch for its own calibration runs.
 *   - Nothing throws across the ABI; every call returns a slicq_status.
 */
#ifndef SLICQ_H
#define SLICQ_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLICQ_ABI_VERSION 2

#if defined(__GNUC__)
#define SLICQ_API __attribute__((visibility("default")))
#else
#define SLICQ_API
#endif

typedef enum {
  SLICQ_OK = 0,
  SLICQ_EINVAL = 1,       /* invalid parameter or null pointer */
  SLICQ_ENOMEM = 2,       /* device or host allocation failed (plan only) */
  SLICQ_ECUDA = 3,        /* a CUDA runtime call or launch failed */
  SLICQ_ESIZE = 4,        /* a caller buffer is too small */
  SLICQ_ETIMEOUT = 5,     /* a bounded device wait gave up */
  SLICQ_EUNSUPPORTED = 6  /* valid parameters outside what this build runs */
} slicq_status;

typedef enum {                                             /* H of Sec. 3 */
  SLICQ_WIN_HANN = 0,             /* cos^2(pi t) on |t| < 1/2 */
  SLICQ_WIN_BLACKMAN_HARRIS = 1   /* 4-term Blackman-Harris (Harris 1978), centred, |t| < 1/2 */
} slicq_window;
typedef enum {                                             /* M_k choice */
  SLICQ_MK_POW2 = 0,   /* M_k = max(16, next power of two >= |J_k|) */
  SLICQ_MK_MULT4 = 1,  /* smallest multiple of 4 >= |J_k|: not built (EUNSUPPORTED) */
  SLICQ_MK_CONST = 2   /* one M for every channel: the rectangular representation */
} slicq_mk_policy;
typedef enum {                                             /* band-transform arithmetic */
  SLICQ_PREC_FP32 = 0,        /* every DFT stage in FP32 on the CUDA cores */
  SLICQ_PREC_SPLIT_FP16 = 1,  /* radix-8/16/32 stages of the band DFTs on the tensor cores: FP16 hi + lo */
  SLICQ_PREC_SPLIT_BF16 = 2   /* the same with BF16 hi + lo */
} slicq_precision;

/*
 * Parameters of one sliCQ system (Sec. 3 and Sec. 4).
 *   fs, fmin, fmax   xi_s, xi_min, xi_max in Hz (Table 1); 0 < fmin < fmax.
 *                    fmax at or above fs/2 selects the largest K with
 *                    xi_K < fs/2.
 *   bins_per_octave  B >= 1.
 *   slice_len        2N, the FFT length of one slice, a power of two in
 *                    [2048, 131072].
 *   trans_len        M, the Tukey transition length, even, 2 <= M < N.
 *   min_filter_len   lower bound on the support of g_k in samples (Sec. 5.2;
 *                    16 is the paper's recommendation). >= 1.
 *   window           SLICQ_WIN_HANN or SLICQ_WIN_BLACKMAN_HARRIS (same
 *                    supports J_k, different values; plateaus stay flat).
 *   mk_policy        SLICQ_MK_POW2: M_k = max(16, next power of two >= |J_k|).
 *                    SLICQ_MK_CONST: every M_k is the largest of those, so
 *                    each slice's coefficients form a (K+2) x M array (the
 *                    rectangular representation, L/a_k constant, Sec. 4.1).
 *   slice_cluster    CTAs per slice FFT (thread-block cluster size); 0 picks
 *                    the default.  Must be a power of two <= 8 if given.
 *   precision        arithmetic of the band DFTs of length M_k (Algorithm 1's
 *                    IFFT_{M_k}, Algorithm 2's FFT_{M_k}) for M_k <= 1024:
 *                    SLICQ_PREC_FP32, or a split-precision tensor-core form
 *                    in which each radix-8/16/32 stage is a product of
 *                    (hi + lo) operands in FP16 or BF16 with FP32
 *                    accumulation (three of the four partial products;
 *                    rows scaled by powers of two first).  FP16 pairs keep
 *                    22 significant bits (about FP32's accuracy), BF16 pairs
 *                    16.  Slice FFTs, windows and M_k = 2048, 4096 stay FP32.
 *                    Plan tables (duals, twiddles) are FP64-computed either way.
 */
typedef struct {
  double fs;
  double fmin;
  double fmax;
  int32_t bins_per_octave;
  int32_t min_filter_len;
  int64_t slice_len;
  int64_t trans_len;
  int32_t window;
  int32_t mk_policy;
  int32_t slice_cluster;
  int32_t precision;
} slicq_params;

typedef struct slicq_plan slicq_plan;

/* Human-readable name of a status code (static storage, never NULL). */
SLICQ_API const char* slicq_status_string(slicq_status s);

/* ABI version of the loaded library (SLICQ_ABI_VERSION). */
SLICQ_API int32_t slicq_abi_version(void);

/*
 * Host-only layout query (no device needed).  Computes K and the channel
 * layout of Table 1 with the supports J_k of Sec. 3.
 *   n_channels       out: K + 2 (the kept channels 0..K+1).
 *   coefs_per_slice  out: sum_k M_k.
 * Returns SLICQ_EINVAL for invalid parameters, SLICQ_EUNSUPPORTED for valid
 * ones this build does not run (e.g. an M_k above 1024).
 */
SLICQ_API slicq_status slicq_layout(const slicq_params* p, int32_t* n_channels,
                          int64_t* coefs_per_slice);

/*
 * Host-only per-channel tables, each an array of n_channels entries owned by
 * the caller (any may be NULL):
 *   h_M       M_k                      h_off    off_k (coefficient offset)
 *   h_j0      first support sample of g_k on Z_{2N} (0 <= j0 < 2N)
 *   h_len     |J_k|                    h_xi, h_omega   xi_k, Omega_k in Hz
 */
SLICQ_API slicq_status slicq_layout_tables(const slicq_params* p, int32_t n_channels,
                                 int32_t* h_M, int64_t* h_off, int64_t* h_j0,
                                 int32_t* h_len, double* h_xi, double* h_omega);

/*
 * Build a plan on `device`: integer layout on the host, window, dual-window
 * (reciprocal of sum_k M_k g_k^2, Prop. 2), slicing-window and twiddle
 * tables in FP64 on the device, stored as float32.  Synchronous.  The plan
 * owns its device tables; free with slicq_plan_destroy.
 */
SLICQ_API slicq_status slicq_plan_create(const slicq_params* p, int device,
                               slicq_plan** out);
SLICQ_API void slicq_plan_destroy(slicq_plan* plan);

/*
 * Device-side status of a plan's launches so far.  Synchronises the plan's
 * device, then returns SLICQ_ETIMEOUT (and clears it) if a band kernel of
 * a split-precision plan gave up waiting for its tensor-core products
 * (each wait is bounded, about one second; the kernel then stops and frees
 * its tensor memory, and its outputs are incomplete), SLICQ_ECUDA if the
 * device reports an error, SLICQ_OK otherwise.  FP32 plans never time out.
 */
SLICQ_API slicq_status slicq_plan_check(const slicq_plan* plan);

/*
 * What the plan chose by measurement at creation: the slice kernels'
 * cluster size (CTAs per slice; with slice_cluster = 0 in the parameters the
 * plan times every valid size on its device and keeps the fastest) and the
 * number of persistent CTAs of the band analysis and synthesis kernels
 * (their lanes per band group come from measured per-group costs).  Any
 * pointer may be NULL.
 */
SLICQ_API slicq_status slicq_plan_tuning(const slicq_plan* plan, int32_t* slice_cluster,
                                         int32_t* band_ctas_analysis, int32_t* band_ctas_synthesis);

/*
 * Self-test of the bounded device waits (the paper has no counterpart).
 * One CTA on `device` waits, with the wait the split-precision band kernels
 * use for their tensor-core products, on an mbarrier that nothing
 * completes; after limit_cycles SM clocks it gives up.  Returns
 * SLICQ_ETIMEOUT when the wait gave up (the expected result), SLICQ_OK if it
 * completed, SLICQ_EINVAL for limit_cycles < 1, SLICQ_ECUDA on a CUDA
 * error.  Synchronous; allocates one int; the context stays usable.
 */
SLICQ_API slicq_status slicq_selftest_wait(int device, int64_t limit_cycles);

/* K + 2 and sum_k M_k of a plan. */
SLICQ_API slicq_status slicq_plan_info(const slicq_plan* plan, int32_t* n_channels,
                             int64_t* coefs_per_slice);

/* Number of slices L/N for n_samples (L = 2N ceil(n/2N), Sec. 4.1); 0 on error. */
SLICQ_API int64_t slicq_num_slices(const slicq_plan* plan, int64_t n_samples);

/*
 * Device workspace (bytes) that forward / inverse / adjoint need for
 * `batch` signals of n_samples.  The workspace holds slice spectra and the
 * partial sums (band bins several groups share, transition samples two
 * slices share) that make the overlap-adds deterministic.  It needs no
 * initialisation: every call writes each value before reading it.  Calls
 * that share a workspace must not overlap in time.
 */
SLICQ_API slicq_status slicq_workspace_size(const slicq_plan* plan, int64_t n_samples,
                                  int64_t batch, size_t* bytes);

/*
 * Forward sliCQ (Algorithm 3 with Algorithm 1 per slice) of `batch` real
 * signals.  d_coef receives batch * S * coefs_per_slice complex values;
 * coef_capacity is its size in complex values (SLICQ_ESIZE if too small).
 */
SLICQ_API slicq_status slicq_forward(const slicq_plan* plan, const float* d_f,
                           int64_t n_samples, int64_t batch, float* d_coef,
                           int64_t coef_capacity, void* d_work,
                           size_t work_bytes, cudaStream_t stream);

/*
 * Inverse sliCQ (Algorithm 4 with Algorithm 2 per slice, canonical dual,
 * dual slicing window = indicator of the support of h_0), real output of
 * n_samples per signal.  For coefficients of a real signal this is its
 * perfect reconstruction (Prop. 3); for other coefficients it is the real
 * part of the synthesis with the conjugate channels restored.
 */
SLICQ_API slicq_status slicq_inverse(const slicq_plan* plan, const float* d_coef,
                           int64_t n_samples, int64_t batch, float* d_out,
                           void* d_work, size_t work_bytes,
                           cudaStream_t stream);

/*
 * Adjoint of the forward map for real input: d_out = Re(A^H c), i.e. the
 * synthesis of Algorithm 2 with the analysis windows g_k over channels
 * 0..K+1 and overlap-add with h_0.  This is the gradient of a real loss with
 * respect to the signal given the conjugate-Wirtinger gradient d_coef.
 */
SLICQ_API slicq_status slicq_adjoint(const slicq_plan* plan, const float* d_coef,
                           int64_t n_samples, int64_t batch, float* d_out,
                           void* d_work, size_t work_bytes,
                           cudaStream_t stream);

/*
 * Copy a plan table to host memory (tests and diagnostics; synchronous).
 *   which = 0  analysis windows g_k / sqrt(2N), channels 0..K+1 concatenated
 *          1  synthesis windows w_k g~_k / sqrt(2N) (w_k = 1/2 for k = 0, K+1)
 *          2  adjoint windows g_k / (2 sqrt(2N))
 *          3  Tukey transition h_0 at |j - N| = (N-M)/2 + o, o = 0..M
 *   count  capacity of h_out in floats; SLICQ_ESIZE if too small.
 *   n_out  out: number of floats written.
 */
SLICQ_API slicq_status slicq_plan_table(const slicq_plan* plan, int32_t which,
                              float* h_out, int64_t count, int64_t* n_out);

/*
 * Ragged batches (not in the paper, whose slices are independent, Sec. 4):
 * many clips of different lengths, sample rates and bins per octave in one
 * call.  Every plan of a batch must have the same slice_len and trans_len
 * and live on the same device (SLICQ_EUNSUPPORTED otherwise).
 *   plans[p]          p < n_plans, owned by the caller, alive while the
 *                     batch is used
 *   clip_plan[c]      plan of clip c, clip_samples[c] its length (>= 1)
 * slicq_batch_create allocates the batch's row tables on the device and
 * creates one stream per plan; each call forks the plans' kernel chains from
 * the caller's stream and joins them back, so capturing one call in a CUDA
 * graph records the whole batch (plans as parallel branches).
 * Layouts (queried with slicq_batch_layout, host arrays of n_clips entries):
 *   signals       one float buffer; clip c at h_sig_off[c] (multiple of 4
 *                 samples), sig_total floats in all, 16-byte aligned base
 *   coefficients  one interleaved complex buffer; clip c's slices
 *                 (h_slices[c] of them, its plan's coefs_per_slice each) at
 *                 h_coef_off[c] complex values; coef_total in all
 *   workspace     work_bytes, 256-byte aligned (no initialisation needed)
 */
typedef struct slicq_batch slicq_batch;
SLICQ_API slicq_status slicq_batch_create(const slicq_plan* const* plans, int32_t n_plans,
                                          const int32_t* clip_plan, const int64_t* clip_samples,
                                          int32_t n_clips, slicq_batch** out);
SLICQ_API void slicq_batch_destroy(slicq_batch* batch);
SLICQ_API slicq_status slicq_batch_layout(const slicq_batch* batch, int64_t* h_sig_off,
                                          int64_t* h_coef_off, int64_t* h_slices,
                                          int64_t* sig_total, int64_t* coef_total,
                                          size_t* work_bytes);
/* Forward (Algorithm 3) of every clip of the batch. */
SLICQ_API slicq_status slicq_batch_forward(const slicq_batch* batch, const float* d_sig,
                                           float* d_coef, void* d_work, size_t work_bytes,
                                           cudaStream_t stream);
/* Inverse (Algorithm 4) of every clip; writes each clip's samples at its offset. */
SLICQ_API slicq_status slicq_batch_inverse(const slicq_batch* batch, const float* d_coef,
                                           float* d_sig_out, void* d_work, size_t work_bytes,
                                           cudaStream_t stream);

/*
 * slicq_inverse with modified coefficients, for transposition and masking
 * (Sec. 6; the modification is applied as the synthesis reads them):
 *   channel_shift  s: channel k = 1..K is synthesised from channel k - s
 *                  (zero where k - s is outside 1..K), modulated by the
 *                  centre-bin difference exp(2 pi i (jc_k - jc_{k-s}) t / 2N),
 *                  jc_k = round(xi_k 2N / xi_s), t = (m-1)N + n 2N/M the
 *                  time of coefficient n of slice m (the coefficients of a
 *                  channel keep its absolute frequency, so a translation
 *                  along the channels needs this modulation).  s = 8 at
 *                  B = 48 transposes by 2 semitones.  The plateau channels
 *                  0 and K+1 keep their own.  s != 0 needs SLICQ_MK_CONST
 *                  (one time grid for all channels), SLICQ_EINVAL otherwise.
 *   d_mask         null, or device float [batch][S][coefs_per_slice]: gains
 *                  multiplying the (shifted) coefficients; 4-byte aligned.
 * Other arguments, layouts and errors as slicq_inverse.
 */
SLICQ_API slicq_status slicq_inverse_modified(const slicq_plan* plan, const float* d_coef,
                                              int64_t n_samples, int64_t batch, int32_t channel_shift,
                                              const float* d_mask, float* d_out, void* d_work,
                                              size_t work_bytes, cudaStream_t stream);

/*
 * Streaming sliCQ (real-time mode with bounded delay; the paper's framework
 * is built for it, Sec. 4): one slice per call, N = slice_len / 2 samples
 * per call in either direction (slicq_stream_hop).
 *   slicq_stream_create   device state for one stream of `plan` (input and
 *                         output rings of 2N samples, one slice's
 *                         workspace); allocates; the plan must outlive it.
 *   slicq_stream_forward  d_in: device, N new float samples (the block
 *                         [mN, (m+1)N) of call m); d_coef: device, complex64
 *                         [coefs_per_slice], 8-byte aligned, receives slice
 *                         m, which covers [(m-1)N, (m+1)N) (Algorithm 3;
 *                         samples before the first block are zero).  Equals
 *                         slice m of slicq_forward of the whole signal when
 *                         that signal ends with at least N zeros.
 *   slicq_stream_inverse  d_coef: one slice's coefficients (call m: slice
 *                         m); d_out: device, N floats, receives output
 *                         samples (m-1)N + a0 + 1 .. mN + a0,
 *                         a0 = (N - trans_len)/2 (Algorithm 4; the first
 *                         call's samples before time 0 lack slice -1).
 *   slicq_stream_reset    back to the start (zero history), asynchronous.
 * A stream's calls are asynchronous on `stream` and must not overlap in time
 * (each call's state is the previous call's result).  The forward and the
 * inverse directions of one stream are independent.
 * Errors: SLICQ_EINVAL (null pointers, misaligned d_coef), SLICQ_ENOMEM,
 * SLICQ_ECUDA.
 */
typedef struct slicq_stream slicq_stream;
SLICQ_API slicq_status slicq_stream_create(const slicq_plan* plan, slicq_stream** out);
SLICQ_API void slicq_stream_destroy(slicq_stream* stream_state);
SLICQ_API int64_t slicq_stream_hop(const slicq_plan* plan);
SLICQ_API slicq_status slicq_stream_forward(slicq_stream* stream_state, const float* d_in, float* d_coef,
                                            cudaStream_t stream);
SLICQ_API slicq_status slicq_stream_inverse(slicq_stream* stream_state, const float* d_coef, float* d_out,
                                            cudaStream_t stream);
SLICQ_API slicq_status slicq_stream_reset(slicq_stream* stream_state, cudaStream_t stream);

/*
 * sliCQ spectrogram (Sec. 4.1): |s^0 + s^1|^2, where the 2-layer array s^l
 * holds slice m's coefficient n of channel k in layer l = m mod 2 at time
 * index t = n + (m-1) M_k / 2 (circular in S M_k / 2), i.e. at time
 * t a_k, a_k = 2N / M_k.  Each t is covered by one even and one odd slice.
 *   d_coef        device, complex64 [batch][S][coefs_per_slice] as written
 *                 by slicq_forward for (n_samples, batch); 8-byte aligned.
 *   d_out         device, float32 [batch][S * coefs_per_slice / 2]: channel
 *                 k's S M_k / 2 values (t = 0, 1, ...) start at S off_k / 2
 *                 (off_k as returned by slicq_layout_tables).
 *   out_capacity  floats available at d_out.
 * Asynchronous on `stream`; allocates nothing, needs no workspace.
 * Errors: SLICQ_EINVAL (null pointers, n_samples or batch < 1, misaligned
 * d_coef), SLICQ_ESIZE (out_capacity too small), SLICQ_ECUDA.
 */
SLICQ_API slicq_status slicq_spectrogram(const slicq_plan* plan, const float* d_coef, int64_t n_samples,
                                         int64_t batch, float* d_out, int64_t out_capacity,
                                         cudaStream_t stream);

/*
 * Forward sliCQ without a caller workspace and without allocating (the paper
 * has no counterpart: this serves callers that may not allocate device
 * memory, such as real-time audio callbacks that must not block on an
 * allocator, or plug-in hosts that own all device memory).
 *   Same arguments and result as slicq_forward, minus the workspace.  The
 *   slice spectra go to a fixed 32 MiB array compiled into the library,
 *   which every GPU that loads the library holds until the process exits.
 *   Returns SLICQ_ESIZE when batch * slicq_num_slices(n_samples) * (N + 2)
 *   complex values (8 bytes each) exceed 32 MiB, and the usual errors
 *   otherwise.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   The first call on a device looks up the array's device address (once per
 *   device, with the plan's device current); make that first call before
 *   any stream capture.  All calls share the array and it keeps the last
 *   call's contents, so calls that overlap on the GPU (other streams, other
 *   threads, other plans) race and must be serialised by the caller.
 */
SLICQ_API slicq_status slicq_forward_noalloc(const slicq_plan* plan, const float* d_f,
                                             int64_t n_samples, int64_t batch,
                                             float* d_coef, int64_t coef_capacity,
                                             cudaStream_t stream);

/*
 * Kernel timing trace (diagnostics and benchmarking; not part of the
 * paper's method).  With enable != 0 every later forward / inverse /
 * adjoint call on this plan records a CUDA event on its stream before and
 * after each kernel launch (up to 4096 launches; later ones are not traced).
 * Kernel ids: 0 slice forward (slicing + real FFT), 1 band analysis,
 * 2 band synthesis, 3 slice inverse (real inverse FFT + overlap-add).
 * slicq_trace_read waits for the recorded events, writes up to `cap`
 * (kernel id, milliseconds) pairs to host arrays and clears the trace.
 * enable = 0 releases the events.  Not thread-safe with concurrent calls
 * on the same plan.
 */
SLICQ_API slicq_status slicq_trace_enable(const slicq_plan* plan, int32_t enable);
SLICQ_API slicq_status slicq_trace_read(const slicq_plan* plan, int32_t* h_kernel,
                                        float* h_ms, int32_t cap, int32_t* n_out);

#ifdef __cplusplus
}
#endif
#endif /* SLICQ_H */

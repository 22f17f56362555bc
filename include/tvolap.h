/*
 * tvolap.h -- C ABI of the GB300 (sm_103a) TVOLAP library.
 *
 * Time-variant overlap-add in partitions (arxiv 2310.00319, Section 2): each
 * input channel is cut into 2L-sample blocks every L samples (Eq. 1), weighted
 * by a periodic Hann window (Eq. "w_hann"; this library uses the amplitude 1/2
 * under which hop-L windows sum to one), zero padded to 4L (Eq. 3) and
 * transformed (Eq. 5). Impulse responses are cut into M partitions of 2L taps
 * (Eq. 2), padded (Eq. 4) and transformed (Eq. 6). Output block l is
 *     Y(k, l) = sum_{m<M} H_l(k, m) X(k, l - 2m)                       (Eq. 7)
 * with H_l the filter current at block l (all partitions exchanged at once,
 * Section 2), followed by the inverse transform (Eq. 8) and the two-step
 * overlap-add (Eqs. 9-12, read with the same-parity predecessor l - 2).
 *
 * Spectra in this library are taken on the half-bin grid (k + 1/2) / 4L rather
 * than the paper's k / 4L. Because every product in Eq. 7 is the transform of
 * a linear convolution shorter than 4L, both grids give the same time-domain
 * output; the half-bin grid has exactly 2L independent complex bins per real
 * block (no separate DC/Nyquist bins), stored as interleaved float pairs
 * (re, im). A spectrum is P = 2L complex values, 8*P bytes.
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device pointers; the caller owns them and keeps
 *    them valid until the handle's CUDA stream has passed the call.
 *  - Every call is enqueued on the stream given to tvolap_create and returns
 *    without waiting for the GPU, unless stated otherwise.
 *  - Every call returns TVOLAP_OK or a negative tvolap_status. A call that
 *    returns TVOLAP_ERR_ARG has enqueued nothing and changed nothing.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Schedules index output blocks by t = l + 1: block l = -1 (L zeros of
 *    history followed by the first L input samples) is entry 0. Output
 *    samples [0, out_len) need n_blocks = floor((out_len - 1) / L) + 2 entries.
 *  - A slot index outside [0, tvolap_slot_count) in a schedule or selection
 *    is replaced on the device by an all-zero filter and recorded; the next
 *    tvolap_check returns TVOLAP_ERR_ARG.
 */
#ifndef TVOLAP_H
#define TVOLAP_H

#include <stdint.h>

#if defined(__GNUC__)
#define TVOLAP_API __attribute__((visibility("default")))
#else
#define TVOLAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tvolap_plan *tvolap_t;

typedef enum tvolap_status {
    TVOLAP_OK = 0,
    TVOLAP_ERR_ARG = -1,      /* invalid argument (nothing enqueued) */
    TVOLAP_ERR_OOM = -2,      /* a device allocation failed */
    TVOLAP_ERR_CUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    TVOLAP_ERR_STATE = -4,    /* handle is NULL or unusable */
    TVOLAP_ERR_CAPACITY = -5, /* request exceeds a stated capacity */
    TVOLAP_ERR_TIMEOUT = -6   /* a bounded device wait gave up */
} tvolap_status;

/* Human-readable name of a status code (static string, never NULL). */
TVOLAP_API const char *tvolap_strerror(int status);

/* Library version, major * 10000 + minor * 100 + patch. */
TVOLAP_API int tvolap_version(void);

/*
 * Create a plan (Section 2: hop L, M partitions of 2L taps, transform length
 * 4L, c channels processed side by side).
 *   out         receives the handle
 *   L           hop; a power of two in [16, 1024]
 *   partitions  M >= 1; impulse responses may have up to 2*L*M taps
 *   fft_len     must be 4*L (Eq. 3: double-length zero padding), or 0 for 4*L
 *   n_in        input channels >= 1
 *   n_out       output channels >= 1
 *   out_to_in   host array [n_out]: input channel feeding each output
 *               (several outputs may share one input, e.g. binaural pairs);
 *               NULL means identity and requires n_in == n_out
 *   n_slots     stored filter slots >= 1 shared by all outputs (filled by
 *               tvolap_load_bank); the plan also keeps one private slot per
 *               output for tvolap_set_filter, so tvolap_slot_count(h) is
 *               n_slots + n_out
 *   stream      cudaStream_t for every call on this handle (NULL = legacy
 *               default stream)
 * Allocates device memory for the filter bank, the frequency-domain delay
 * line and the overlap state; synchronises the stream before returning.
 * Errors: TVOLAP_ERR_ARG, TVOLAP_ERR_OOM, TVOLAP_ERR_CUDA.
 */
TVOLAP_API int tvolap_create(tvolap_t *out, int L, int partitions, int fft_len, int n_in, int n_out,
                  const int32_t *out_to_in, int n_slots, void *stream);

/* Synchronise the stream and free everything the handle owns. NULL is a no-op. */
TVOLAP_API int tvolap_destroy(tvolap_t h);

/* Plan geometry: L, M, P = 2L (complex bins per spectrum), channels, slots. */
TVOLAP_API int tvolap_get_dims(tvolap_t h, int *L, int *M, int *P, int *n_in, int *n_out, int *n_slots);

/* Total addressable filter slots: n_slots + n_out (private set_filter slots). */
TVOLAP_API int tvolap_slot_count(tvolap_t h);

/*
 * Zero the streaming state (delay line, input history, overlap state, block
 * counter) and reset every output's selection to its private slot. The bank
 * keeps its contents.
 */
TVOLAP_API int tvolap_reset(tvolap_t h);

/*
 * Transform impulse responses into filter slots [first_slot, first_slot+count)
 * (Eqs. 2, 4, 6): partition m of slot s holds taps [2mL, 2mL + 2L) of
 * ir_dev[s - first_slot]. Taps at or beyond ir_len are zero.
 *   ir_dev     device float [count][ir_stride]
 *   ir_len     taps per response, 1 <= ir_len <= 2*L*M
 *   ir_stride  floats between consecutive responses, >= ir_len
 * first_slot + count must not exceed n_slots (the private slots are written
 * only by tvolap_set_filter).
 */
TVOLAP_API int tvolap_load_bank(tvolap_t h, int first_slot, int count, const float *ir_dev, int ir_len,
                     int64_t ir_stride);

/*
 * Exchange the filter of one output (Section 2: all partitions at once): the
 * response is transformed into the output's private slot and selected alone.
 * Takes effect from the next tvolap_process_block on this handle.
 */
TVOLAP_API int tvolap_set_filter(tvolap_t h, int out_ch, const float *ir_dev, int ir_len);

/*
 * Select the filter of one output for the following streamed blocks:
 * H = (1 - alpha) * H[slot_a] + alpha * H[slot_b]. A mix of transfer functions
 * equals the transfer function of the mixed taps (linearity of Eq. 6).
 */
TVOLAP_API int tvolap_select(tvolap_t h, int out_ch, int slot_a, int slot_b, float alpha);

/*
 * Stream one hop (one streaming tick): consume L new samples per input,
 * emit L samples per output. Tick t processes block l = t - 1 (the previous
 * L samples of history and the L new ones), so the emitted samples are the
 * offline output delayed by exactly L samples (block latency 2L in total,
 * Table 1).
 *   in_dev    device float [n_in][L]
 *   out_dev   device float [n_out][L]
 *   sel_a, sel_b, sel_alpha   optional device arrays [n_out] giving this
 *             tick's selection (and keeping it for later ticks); NULL keeps
 *             the current selection. sel_b / sel_alpha may be NULL on their
 *             own (then b = a, alpha = 0).
 */
TVOLAP_API int tvolap_process_block(tvolap_t h, const float *in_dev, float *out_dev, const int32_t *sel_a,
                         const int32_t *sel_b, const float *sel_alpha);

/*
 * Whole-signal (offline) TVOLAP; the streaming state is not touched. Every
 * block of every channel is independent (Eq. 7 has no recurrence), so all run
 * in parallel: forward transforms, partition MAC, inverse transforms with the
 * overlap-add.
 *   x_dev        device float [n_in][x_stride], N valid samples per channel
 *   sched_a      device int32 [n_out][sched_stride] slot per block (t = l+1)
 *   sched_b      device int32 [n_out][sched_stride] or NULL (b = a)
 *   sched_alpha  device float [n_out][sched_stride] or NULL (alpha = 0)
 *   sched_stride >= n_blocks = floor((out_len - 1) / L) + 2
 *   y_dev        device float [n_out][y_stride]; samples [0, out_len) written,
 *                aligned with x (no delay); out_len may exceed N (tail)
 * Uses a device workspace owned by the handle of
 * 8 * P * n_blocks * (n_in + n_out) bytes, grown (cudaMalloc) when needed.
 */
TVOLAP_API int tvolap_process_signal(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                          const int32_t *sched_a, const int32_t *sched_b,
                          const float *sched_alpha, int64_t sched_stride, float *y_dev,
                          int64_t out_len, int64_t y_stride);

/*
 * tvolap_process_signal for a batch whose channels differ in length and in
 * the number of partitions they use (many independent sources of one hop L in
 * one call; Section 2: c channels side by side). Channel c is input c and
 * output c (the plan must have identity routing). Per channel, device arrays:
 *   n_dev        int64 [n_in]   input samples of channel c (<= x_stride)
 *   out_len_dev  int64 [n_out]  output samples to write (<= max_out_len)
 *   parts_dev    int32 [n_out]  partitions its filters use (1 .. M): its
 *                impulse responses have at most 2 * L * parts taps
 * Grids cover max_out_len; each channel does only its own blocks and
 * partitions. Values are clamped on the device to the bounds above. Schedules
 * as in tvolap_process_signal (sched_stride >= blocks of max_out_len); samples
 * of y_dev past a channel's out_len are not written.
 */
TVOLAP_API int tvolap_process_ragged(tvolap_t h, const float *x_dev, int64_t x_stride,
                                     const int64_t *n_dev, const int64_t *out_len_dev,
                                     const int32_t *parts_dev, int64_t max_out_len,
                                     const int32_t *sched_a, const int32_t *sched_b,
                                     const float *sched_alpha, int64_t sched_stride, float *y_dev,
                                     int64_t y_stride);

/* Bytes of workspace tvolap_process_signal needs for out_len samples. */
TVOLAP_API int64_t tvolap_signal_workspace_bytes(tvolap_t h, int64_t out_len);

/*
 * Stage 1 of tvolap_process_signal on its own (Eqs. 1, 3, 5): the spectra of
 * input blocks l = -1 .. n_blocks - 2 of every input channel.
 *   X_dev  device float2 [n_in][n_blocks][P]
 */
TVOLAP_API int tvolap_forward_spectra(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                           int n_blocks, float *X_dev);

/*
 * Stage 2 on its own (Eq. 7 with the block's filter): for every output o and
 * block t < n_blocks, Y[o][t] = sum_{m < M, t - 2m >= 0} H_t(m) X[in(o)][t - 2m].
 *   X_dev  device float2 [n_in][n_blocks][P];  Y_dev device float2 [n_out][n_blocks][P]
 */
TVOLAP_API int tvolap_mac(tvolap_t h, const float *X_dev, int n_blocks, const int32_t *sched_a,
               const int32_t *sched_b, const float *sched_alpha, int64_t sched_stride,
               float *Y_dev);

/*
 * Stage 3 on its own (Eqs. 8-12): inverse transform of every block's Y and
 * overlap-add into y[o][0 .. out_len); n_blocks must equal
 * floor((out_len - 1) / L) + 2.
 */
TVOLAP_API int tvolap_inverse_ola(tvolap_t h, const float *Y_dev, int n_blocks, float *y_dev,
                       int64_t out_len, int64_t y_stride);

/*
 * ---- Differentiable TVOLAP (free per-block partition spectra) -------------
 * A model in which the filter partitions of Eq. 7 are free spectra
 * P[o][t][m][k] (t < p_blocks output blocks, m < M, k < P; the same half-bin
 * grid and storage as every spectrum here) instead of transforms of impulse
 * responses: Y(t) = sum_{m, t-2m >= 0} P(t, m) X(t - 2m), followed by Eqs. 8-12
 * (tvolap_inverse_ola). Gradients use the convention dL/dRe + i dL/dIm for
 * complex values. All buffers of these calls must be 16-byte aligned; block
 * ranges let a caller recompute input spectra segment by segment.
 */

/* Spectra of input blocks t_first .. t_first + t_count - 1 (Eqs. 1, 3, 5):
   X_dev float2 [n_in][t_count][P]. */
TVOLAP_API int tvolap_block_spectra(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                                    int64_t t_first, int t_count, float *X_dev);

/*
 * Y[o][i] = sum_{m < M, t - 2m >= 0} P[o][t][m] * X[in(o)][t - 2m - x_first],
 * t = t_first + i, i < t_count (Eq. 7 with the parameters as filter).
 *   X_dev  float2 [n_in][x_count][P], rows x_first .. x_first + x_count - 1;
 *          must hold every row needed: x_first <= max(0, t_first - 2(M-1)) and
 *          x_first + x_count >= t_first + t_count
 *   P_dev  float2 [n_out][p_blocks][M][P]; t_first + t_count <= p_blocks
 *   Y_dev  float2 [n_out][y_rows][P], rows 0 .. t_count - 1 written
 *          (y_rows >= t_count: a segment can land inside a larger buffer)
 */
TVOLAP_API int tvolap_mac_params(tvolap_t h, const float *X_dev, int64_t x_first, int x_count,
                                 const float *P_dev, int64_t p_blocks, int64_t t_first,
                                 int t_count, float *Y_dev, int64_t y_rows);

/*
 * Adjoint of Eq. 8 (with the overlap-add of Eqs. 9-12) for g = dL/dy:
 * G[o][i] = dL/dY(t) = (1/2L) sum_{n<4L} g[o][(t-1)L + n] e^{-i pi n (2k+1)/4L},
 * t = t_first + i; samples outside [0, g_len) count as zero.
 *   g_dev float [n_out][g_stride];  G_dev float2 [n_out][t_count][P]
 */
TVOLAP_API int tvolap_adjoint_output(tvolap_t h, const float *g_dev, int64_t g_len,
                                     int64_t g_stride, int64_t t_first, int t_count,
                                     float *G_dev);

/*
 * Adjoint of Eq. 7, for input blocks q = q_first .. q_first + q_count - 1:
 *   dX[o][q - q_first] = sum_{m, q+2m < p_blocks} G(q + 2m) conj P(q + 2m, m)
 *   dP(t, m) = G(t) conj X(q)   for every t, m with t - 2m = q
 * and, when q_first == 0, dP(t, m) = 0 for t < 2m. Called over ranges that
 * cover 0 .. p_blocks - 1, this writes all of dP.
 *   G_dev  float2 [n_out][g_count][P], rows g_first ..; needs g_first <= q_first
 *          and g_first + g_count >= min(p_blocks, q_first + q_count + 2(M-1))
 *   X_dev  float2 [n_in][x_count][P], rows x_first ..; must cover the q range
 *   P_dev, dP_dev  float2 [n_out][p_blocks][M][P]
 *   dX_dev float2 [n_out][dx_rows][P], rows 0 .. q_count - 1 written (dx_rows >=
 *          q_count: segments can land inside one buffer)
 * Requires identity routing (n_in == n_out, output o reads input o).
 */
TVOLAP_API int tvolap_adjoint_mac(tvolap_t h, const float *G_dev, int64_t g_first, int g_count,
                                  const float *X_dev, int64_t x_first, int x_count,
                                  const float *P_dev, int64_t p_blocks, int64_t q_first,
                                  int q_count, float *dP_dev, float *dX_dev, int64_t dx_rows);

/*
 * tvolap_adjoint_mac with the input spectra recomputed inside the kernel
 * instead of read: each CTA transforms the blocks q it handles from x_dev
 * (Eqs. 1, 3, 5, the same arithmetic as tvolap_block_spectra) and uses them at
 * once, so no input spectra are stored between forward and backward (the
 * limit of recomputing per segment, segment length 1). Results equal those of
 * tvolap_block_spectra followed by tvolap_adjoint_mac.
 *   x_dev  device float [n_in][x_stride], N valid samples per channel
 * Other arguments and requirements as tvolap_adjoint_mac.
 */
TVOLAP_API int tvolap_adjoint_mac_x(tvolap_t h, const float *G_dev, int64_t g_first, int g_count,
                                    const float *x_dev, int64_t N, int64_t x_stride,
                                    const float *P_dev, int64_t p_blocks, int64_t q_first,
                                    int q_count, float *dP_dev, float *dX_dev, int64_t dx_rows);

/*
 * Adjoint of Eqs. 1, 3, 5: for each block q of the range,
 *   dx[c][(q-1)L + n] += w(n) Re sum_{k<P} dX[c][q - q_first](k) e^{+i pi n (2k+1)/4L},
 * 0 <= n < 2L, samples outside [0, N) dropped. Adds to what dx_dev holds, so
 * ranges can be processed one after another (zero dx_dev first).
 *   dX_dev float2 [n_in][q_count][P];  dx_dev float [n_in][x_stride]
 * Requires identity routing.
 */
TVOLAP_API int tvolap_adjoint_input(tvolap_t h, const float *dX_dev, int64_t q_first, int q_count,
                                    float *dx_dev, int64_t N, int64_t x_stride);

/* Copy the M partition spectra of one slot to out_dev (device float2 [M][P]). */
TVOLAP_API int tvolap_bank_spectra(tvolap_t h, int slot, float *out_dev);

/* Size of the fixed device scratch array used by tvolap_process_signal_static. */
#define TVOLAP_STATIC_SCRATCH_BYTES (32u << 20)

/*
 * tvolap_process_signal without any device allocation. The paper has no
 * counterpart; this serves callers that must not allocate device memory once
 * they are running (a real-time audio callback with a hard deadline, a process
 * under a device-memory budget fixed at start-up). tvolap_process_signal grows
 * a workspace with cudaMalloc; this call instead keeps its scratch (the block
 * spectra X and Y) in one file-scope device array of TVOLAP_STATIC_SCRATCH_BYTES
 * bytes, which every GPU that loads the library holds until the process exits.
 * Arguments, results and stream ordering are those of tvolap_process_signal,
 * and the caller still passes every input and output buffer.
 *  - Returns TVOLAP_ERR_CAPACITY when 8 * P * n_blocks * (n_in + n_out) exceeds
 *    TVOLAP_STATIC_SCRATCH_BYTES, with nothing enqueued.
 *  - The device that is current at the call must be the plan's (its
 *    stream's) device; otherwise TVOLAP_ERR_ARG, with nothing enqueued.
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress, with that device current). Under lazy module
 *    loading that first lookup is also when the device reserves the
 *    TVOLAP_STATIC_SCRATCH_BYTES of the array, so make the first call at
 *    start-up, before any stream capture and before the device-memory budget
 *    is fixed; later calls take no device memory.
 *  - All calls, from every handle on a device, share the one array; calls that
 *    overlap on the GPU (other streams, other threads) race on it and give
 *    undefined results. Each call writes all the scratch it reads, so nothing
 *    left by an earlier call is used.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine. The
 *    multiply-accumulate runs the cp.async kernel, which needs no scratch.
 */
TVOLAP_API int tvolap_process_signal_static(tvolap_t h, const float *x_dev, int64_t N,
                                            int64_t x_stride, const int32_t *sched_a,
                                            const int32_t *sched_b, const float *sched_alpha,
                                            int64_t sched_stride, float *y_dev, int64_t out_len,
                                            int64_t y_stride);

/* ========================================================================
 * Frequency-domain mixdown of several outputs (an extension of Section 2's
 * c parallel channels for multi-channel binaural rendering, Section 5): the
 * inverse transform (Eq. 8) and the overlap-add (Eqs. 9-12) are linear, so
 * the sum of several outputs equals one inverse transform of the sum of
 * their spectra Y. A renderer with S sources and E ears makes S*E plan
 * outputs (output o reads source out_to_in[o] through its own filters) and
 * E mix outputs, and runs E inverse transforms per block instead of S*E.
 * ======================================================================== */

/*
 * Define the mixdown: n_mix mix outputs, 1 <= n_mix <= n_out; mix_of_out
 * (host int32 [n_out]) gives each plan output's mix output in [0, n_mix);
 * a mix output with no member is silent. n_mix = 0 removes the mixdown.
 * Synchronises the plan's stream (allocates), clears the mix outputs'
 * streaming overlap-add state; the plan's own streaming state is kept.
 * Returns TVOLAP_ERR_ARG for an invalid map.
 */
TVOLAP_API int tvolap_set_mix(tvolap_t h, int n_mix, const int32_t *mix_of_out);

/*
 * Mixdown stage: Ymix[e][t][k] = sum of Y[o][t][k] over the outputs o of mix
 * output e, added in increasing o (a single member is copied exactly).
 *   Y_dev     device complex64 [n_out][n_blocks][2L] (tvolap_mac's layout)
 *   Ymix_dev  device complex64 [n_mix][n_blocks][2L]
 * Both 16-byte aligned. TVOLAP_ERR_ARG without a mixdown.
 */
TVOLAP_API int tvolap_mix(tvolap_t h, const void *Y_dev, int n_blocks, void *Ymix_dev);

/*
 * tvolap_process_signal with the mixdown: forward transforms, the partition
 * MAC of every plan output, the mixdown, then n_mix inverse transforms with
 * the overlap-add.
 *   y_dev   device float [n_mix][y_stride]; samples [0, out_len) of each
 *           mix output written
 * Other arguments as tvolap_process_signal; the workspace grows by
 * 8 * P * n_blocks * n_mix bytes.
 */
TVOLAP_API int tvolap_process_signal_mix(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                                         const int32_t *sched_a, const int32_t *sched_b,
                                         const float *sched_alpha, int64_t sched_stride,
                                         float *y_dev, int64_t out_len, int64_t y_stride);

/*
 * tvolap_process_block with the mixdown: out_dev is device float [n_mix][L],
 * delayed by L samples like tvolap_process_block. The mix outputs keep their
 * own overlap-add state, so a stream is run with one of the two calls (after
 * tvolap_reset or tvolap_set_mix).
 */
TVOLAP_API int tvolap_process_block_mix(tvolap_t h, const float *in_dev, float *out_dev,
                                        const int32_t *sel_a, const int32_t *sel_b,
                                        const float *sel_alpha);

/* ========================================================================
 * Streaming-state snapshot (serving resilience: checkpoint a stream, resume
 * it later or on another plan of the same shape). The state is what
 * tvolap_process_block / tvolap_process_block_mix carry from tick to tick:
 * the frequency-domain delay line, the input history, the pending
 * overlap-add sums (of the outputs and of the mix outputs), the current
 * selection and the block counter. The filter bank is not part of it.
 * ======================================================================== */

/* Bytes of a snapshot of this plan (a 256-byte aligned layout: a header
   with the plan's shape and block counter, then the arrays). */
TVOLAP_API int64_t tvolap_state_bytes(tvolap_t h);

/*
 * Copy the streaming state into buf (host or device memory, cap bytes >=
 * tvolap_state_bytes), ordered after the work already on the plan's stream;
 * returns when the copy is complete (synchronises the stream).
 */
TVOLAP_API int tvolap_get_state(tvolap_t h, void *buf, int64_t cap);

/*
 * Restore a snapshot (host or device memory) taken from a plan with the same
 * L, M, n_in, n_out and number of mix outputs; TVOLAP_ERR_ARG if the shape
 * or the format differs (the plan is then unchanged). Synchronises the
 * stream. The next tick continues exactly where the snapshot was taken.
 */
TVOLAP_API int tvolap_set_state(tvolap_t h, const void *buf, int64_t bytes);

/* ========================================================================
 * Two-level non-uniform partitions (small first partitions, larger later
 * ones: the partitioned-convolution lineage the paper builds on, Section 1).
 * A head plan (hop La, Ma partitions) convolves with taps [0, D), D = 2 La Ma,
 * at the small hop's latency; a tail plan (hop Lb = ratio * La, Mb
 * partitions) convolves with taps [D, D + 2 Lb Mb) at a fraction of the cost
 * per sample, and its aligned output is added D samples later. A fixed
 * response gives exactly its full convolution (linearity and time invariance
 * of each level); a switch crossfades in each level at that level's block
 * boundaries. The tail's schedule entry tb is the head's entry
 * (tb + 1) * ratio - 1 (in streaming: the head's selection when the tail's
 * hop completes). Streaming needs Ma >= ratio - 1, so that every tail sample
 * has been produced when the head output that adds it is emitted.
 * ======================================================================== */
typedef struct tvolap_nu *tvolap_nu_t;

/* ratio: a power of two in [2, 64] with La * ratio <= 1024; Ma >= ratio - 1;
   other arguments as tvolap_create (the same for both levels). */
TVOLAP_API int tvolap_nu_create(tvolap_nu_t *out, int La, int Ma, int ratio, int Mb, int n_in,
                                int n_out, const int32_t *out_to_in, int n_slots, void *stream);
TVOLAP_API int tvolap_nu_destroy(tvolap_nu_t h);
/* Zero both levels' streaming state and the tail's delay line of outputs. */
TVOLAP_API int tvolap_nu_reset(tvolap_nu_t h);
/* Hops, head taps D and the longest response (D + 2 Lb Mb). */
TVOLAP_API int tvolap_nu_dims(tvolap_nu_t h, int *La, int *Lb, int64_t *head_taps,
                              int64_t *max_taps);
/* Stored responses of up to D + 2 Lb Mb taps: taps [0, D) go to the head's
   slots, the rest to the tail's (as tvolap_load_bank). */
TVOLAP_API int tvolap_nu_load_bank(tvolap_nu_t h, int first_slot, int count, const float *ir_dev,
                                   int ir_len, int64_t ir_stride);
/* Offline, as tvolap_process_signal; schedules are per head block (hop La). */
TVOLAP_API int tvolap_nu_process_signal(tvolap_nu_t h, const float *x_dev, int64_t N,
                                        int64_t x_stride, const int32_t *sched_a,
                                        const int32_t *sched_b, const float *sched_alpha,
                                        int64_t sched_stride, float *y_dev, int64_t out_len,
                                        int64_t y_stride);
/* One head hop, as tvolap_process_block (La samples in and out, output
   delayed by La); every ratio-th call also runs the tail's hop. */
TVOLAP_API int tvolap_nu_process_block(tvolap_nu_t h, const float *in_dev, float *out_dev,
                                       const int32_t *sel_a, const int32_t *sel_b,
                                       const float *sel_alpha);
/* tvolap_set_option for the head (level 0), the tail (1) or both (-1): the
   tail's filters change by larger steps per block, so another MAC staging
   may suit it better. */
TVOLAP_API int tvolap_nu_set_option(tvolap_nu_t h, int level, int option, int value);
/* Deferred device errors of both levels (as tvolap_check). */
TVOLAP_API int tvolap_nu_check(tvolap_nu_t h);

/* Options of tvolap_set_option. */
typedef enum tvolap_option {
    /* Staging of the offline multiply-accumulate: 0 = tiled bulk tensor copies
       (TMA) when the buffers allow it, else cp.async (default): resident CTAs
       take groups of 64 consecutive blocks from a work counter, staging up to
       four distinct filters per group, a run (8 blocks of one parity)
       mixing at most three (groups with more go to a per-warp kernel that
       splits their runs); 1 = always cp.async; 2 = TMA, one group per CTA, up to four
       distinct filters per group and per run (for schedules that cycle four
       filters); 3 = TMA, one group per CTA, up to three filters; 4 = as 3
       with two adjacent bins per thread when 2L is a multiple of 64; 5 = as 0
       with runs of up to four filters.
       0, 1, 3 and 4 give identical results, and so do 2 and 5; 2 and 5 differ
       from the others only in the rounding of runs that mix four filters. */
    TVOLAP_OPT_MAC_STAGING = 1,
    /* 1: tvolap_process_block records CUDA events around its three stages
       (forward transform, multiply-accumulate, inverse + overlap-add) and
       each call first waits for the previous call's events, adding their
       times up for tvolap_stage_times; 0 (default): off. Setting it (either
       value) clears the sums. */
    TVOLAP_OPT_STAGE_TIMING = 2,
    /* Threads per CTA of the offline transform kernels (forward transforms,
       partition bank, inverse + overlap-add): 0 (default) or 256, 128, 64
       (never fewer than one transform's 2L / 16 threads). Each transform runs
       on 2L / 16 threads, so this sets how many transforms share a CTA and
       its shared memory. Results do not depend on it. */
    TVOLAP_OPT_XFORM_THREADS = 3
} tvolap_option;

/* Set a plan option (takes effect for the following calls). */
TVOLAP_API int tvolap_set_option(tvolap_t h, int option, int value);

/* Stage times of the streaming ticks timed since TVOLAP_OPT_STAGE_TIMING was
   set: stage_ms[0..2] = forward transform, multiply-accumulate (Eq. 7),
   inverse transform + overlap-add, in milliseconds summed over *ticks ticks
   (may be NULL). Waits for the last timed tick. */
TVOLAP_API int tvolap_stage_times(tvolap_t h, double *stage_ms, int64_t *ticks);

/*
 * Synchronise the stream and report deferred device-side errors: returns
 * TVOLAP_ERR_ARG if any kernel since the previous check met an invalid slot
 * index, TVOLAP_ERR_TIMEOUT if a bounded wait for an asynchronous copy gave
 * up (the affected outputs are not written), TVOLAP_ERR_CUDA on a CUDA error,
 * otherwise TVOLAP_OK. The error record is cleared.
 */
TVOLAP_API int tvolap_check(tvolap_t h);

/* ========================================================================
 * Batched sources: many independent sources with different hops, partition
 * counts, numbers of stored filters and signal lengths, run together. The
 * sources are grouped by hop; each group is one plan whose channels are the
 * group's sources (tvolap_process_ragged). Every call is ordered on the
 * batch's stream; inside a run (and a load of filters, and the autotuner)
 * each group works on a stream of its own, forked from the batch's stream and
 * joined back into it, so the groups' kernels overlap on the GPU. The whole
 * batch can be captured once as a CUDA graph (one branch per group) and
 * replayed. The
 * multiply-accumulate staging (TVOLAP_OPT_MAC_STAGING) can be chosen per
 * group by timing the variants on the batch itself.
 * ======================================================================== */
typedef struct tvolap_batch *tvolap_batch_t;

/* One source of a batch. */
typedef struct tvolap_batch_source {
    int L;             /* hop, a power of two in [16, 1024] */
    int M;             /* partitions: responses of up to 2*L*M taps */
    int n_filters;     /* stored filters (responses) >= 1 */
    int64_t N;         /* input samples >= 0 */
    int64_t out_len;   /* output samples >= 0 */
} tvolap_batch_source;

/*
 * Create a batch of n_src sources (host array src). Allocates, per hop group,
 * a plan, the inputs [sources][max N], schedules [sources][max blocks] and
 * outputs [sources][max out_len] in device memory (all zero), and the
 * per-source lengths and partition counts. stream: cudaStream_t of every call
 * (NULL = the batch creates its own; graphs cannot be captured on the legacy
 * stream). Synchronises before returning.
 */
TVOLAP_API int tvolap_batch_create(tvolap_batch_t *out, const tvolap_batch_source *src, int n_src,
                                   void *stream);
TVOLAP_API int tvolap_batch_destroy(tvolap_batch_t b);

/*
 * Where source i lives (device pointers, valid for the batch's life):
 *   x     float [N]            its input (write it before running)
 *   sched int32 [n_blocks]     filter of each block, t = l + 1, as slot_base +
 *                              the source's own filter index (0 .. n_filters-1)
 *   y     float [out_len]      its output after a run
 * n_blocks = floor((out_len - 1) / L) + 2. Any pointer argument may be NULL.
 */
TVOLAP_API int tvolap_batch_source_view(tvolap_batch_t b, int i, float **x, int32_t **sched,
                                        float **y, int *slot_base, int64_t *n_blocks);

/*
 * Copy source i's input (device float [N]) and schedule (device int32
 * [n_blocks], the source's own filter indices 0 .. n_filters - 1) into the
 * batch, on the batch's stream. A schedule entry outside that range selects an
 * all-zero filter and makes tvolap_batch_check return TVOLAP_ERR_ARG.
 */
TVOLAP_API int tvolap_batch_set_source(tvolap_batch_t b, int i, const float *x_dev,
                                       const int32_t *sched_dev);

/* Copy source i's output (out_len floats) to y_dev, on the batch's stream. */
TVOLAP_API int tvolap_batch_get_output(tvolap_batch_t b, int i, float *y_dev);

/* Transform source i's n_filters responses (device float [n_filters][ir_stride],
   ir_len <= 2*L*M taps) into its filter slots (Eqs. 2, 4, 6). */
TVOLAP_API int tvolap_batch_load_filters(tvolap_batch_t b, int i, const float *ir_dev,
                                         int ir_len, int64_t ir_stride);

/* Enqueue one run of every source: the captured graph if there is one, else
   the groups' calls directly. */
TVOLAP_API int tvolap_batch_run(tvolap_batch_t b);

/* Record one run of the whole batch as a CUDA graph (after one direct run,
   so every workspace has its size); later runs replay it. */
TVOLAP_API int tvolap_batch_capture(tvolap_batch_t b);

/*
 * For every hop group, time each multiply-accumulate staging (0 .. 5) over
 * reps runs on the batch itself and keep the fastest, then, with it, each
 * CTA size of the transform kernels (TVOLAP_OPT_XFORM_THREADS 256, 128, 64:
 * how many transforms share a CTA) and keep the fastest; drops a captured
 * graph. chosen (may be NULL): host int [number of groups], the staging per
 * group in increasing hop order (tvolap_batch_group_tiling gives both
 * choices). Synchronises.
 */
TVOLAP_API int tvolap_batch_autotune(tvolap_batch_t b, int reps, int *chosen);

/* Set the multiply-accumulate staging of group g (-1: every group); drops a
   captured graph. */
TVOLAP_API int tvolap_batch_set_staging(tvolap_batch_t b, int g, int staging);

/* Group g's multiply-accumulate staging and transform CTA size (0 = default). */
TVOLAP_API int tvolap_batch_group_tiling(tvolap_batch_t b, int g, int *mac_staging,
                                         int *xform_threads);

/* Number of hop groups, and group g's hop, sources and staging. */
TVOLAP_API int tvolap_batch_groups(tvolap_batch_t b, int *n_groups);
TVOLAP_API int tvolap_batch_group_info(tvolap_batch_t b, int g, int *L, int *n_sources,
                                       int *staging);

/* Synchronise the batch's stream and report deferred errors of every group
   (as tvolap_check). */
TVOLAP_API int tvolap_batch_check(tvolap_batch_t b);

/* ========================================================================
 * Streaming server: many independent streams, each with its own hop L,
 * partition count M, outputs (1 or 2, e.g. a binaural pair fed by one input)
 * and a bank of stored filters, processed block by block as in
 * tvolap_process_block (Section 2: all partitions switch at once, output
 * delayed by L), admitted and retired while the server runs.
 *
 * Time advances in base ticks of base_hop samples. A stream of hop L =
 * r * base_hop is due once every r base ticks, at ticks T with T mod r equal
 * to its phase; the phase is picked at admission to even out the bytes read
 * per tick. One tick processes every due stream: forward transforms into each
 * stream's delay line, the Eq. 7 multiply-accumulate against the filter
 * selected for that block, inverse transforms and overlap-add. A tick is one
 * CUDA-graph replay (or the same launches issued directly).
 *
 * Device memory: one arena of arena_bytes, allocated at creation, holds every
 * stream's filter bank, delay line and overlap state; admission takes a
 * contiguous piece (first fit, 256-byte aligned) and fails with
 * TVOLAP_ERR_CAPACITY when no free slot or no piece of the stream's footprint
 * is left. Retiring returns the piece at once; the server orders any later
 * writes into it after the ticks already enqueued.
 *
 * Input and output blocks pass through two sets of pinned host staging arrays
 * that the kernels read and write directly (mapped host memory); tick k
 * (k = 1, 2, ...) uses set (k - 1) mod 2, so the caller can fill one set
 * while the previous tick runs on the other. tvolap_server_due names the set
 * of the next tick after waiting for the tick that used it before: write, for
 * every stream it lists, the L new samples into in[id][0..L) of that set and
 * the filter index of the block into sel[id]; once that tick has finished
 * (the next tvolap_server_due naming the same set, or tvolap_server_wait) the
 * output block of output o is in out[id][o][0..L) of the set.
 *
 * A server is not thread-safe, except tvolap_server_post (any thread).
 * ======================================================================== */
typedef struct tvolap_server *tvolap_server_t;

/*
 * Create a server.
 *   base_hop     smallest hop; a power of two in [16, 1024]
 *   max_hop      largest hop; a power of two in [base_hop, 1024], at most
 *                8 * base_hop (hops base_hop, 2 base_hop, ... max_hop)
 *   capacity     maximum number of streams admitted at once, 1 .. 65536
 *   max_out      outputs per stream, 1 or 2
 *   arena_bytes  device memory for the streams' state and banks
 *   stream       cudaStream_t of the ticks (NULL = legacy default stream)
 * Allocates the arena, the per-slot tables, the host staging (pinned) and a
 * second stream for admissions. Returns TVOLAP_ERR_OOM when an allocation
 * fails.
 */
TVOLAP_API int tvolap_server_create(tvolap_server_t *out, int base_hop, int max_hop, int capacity,
                                    int max_out, int64_t arena_bytes, void *stream);

/* Wait for outstanding work and release everything. NULL is accepted. */
TVOLAP_API int tvolap_server_destroy(tvolap_server_t s);

/*
 * Device bytes a stream of hop L, M partitions, n_out outputs and n_filters
 * stored filters takes from the arena: its bank (n_filters * n_out * M spectra),
 * its delay line (2M spectra), its overlap state (3L floats per output) and
 * its input history (L floats), each rounded up to 256 bytes.
 */
TVOLAP_API int tvolap_server_footprint(tvolap_server_t s, int L, int M, int n_out, int n_filters,
                                       int64_t *bytes);

/*
 * Admit a stream.
 *   L          hop: base_hop * 2^k <= max_hop
 *   M          partitions (responses of up to 2*L*M taps), >= 1
 *   n_out      1 .. max_out outputs, all fed by the stream's one input
 *   n_filters  stored filters, >= 1; filter f has one response per output
 *   ir_dev     device float [n_filters * n_out][ir_stride]: response of
 *              output o of filter f in row f * n_out + o, ir_len taps
 *              (<= 2*L*M, zero beyond); kept valid by the caller until the
 *              stream is live (tvolap_server_state) or the server is waited on
 *   id         receives the stream id, in [0, capacity)
 * The bank transform (Eqs. 2, 4, 6) and the zeroing of the stream's state run
 * on the admission stream, overlapping ticks in flight; the stream becomes
 * live, and starts to be listed as due, at the first tick planned after that
 * work has finished. Returns TVOLAP_ERR_CAPACITY (nothing changed) when no
 * slot or no arena piece is free.
 */
TVOLAP_API int tvolap_server_admit(tvolap_server_t s, int L, int M, int n_out, int n_filters,
                                   const float *ir_dev, int ir_len, int64_t ir_stride, int *id);

/*
 * Admission queue (continuous batching, Section 2's c channels served block by
 * block as they come and go). A request that finds no free slot or arena
 * piece waits instead of being refused; waiting requests are admitted in
 * arrival order, oldest first, as retired streams free their slots and
 * memory: at tvolap_server_submit itself and at every tvolap_server_due, so
 * at most one base tick after the room appears. Nothing overtakes the oldest
 * request (a large request at the head holds back smaller ones behind it).
 * tvolap_server_admit does not look at the queue.
 *
 * tvolap_server_submit
 *   arguments as tvolap_server_admit, except ticket, which receives the
 *   request's number (1, 2, 3, ... in submission order). ir_dev stays valid
 *   until the request has been admitted and its stream is live, or it is
 *   cancelled, or the server is destroyed. Returns TVOLAP_ERR_ARG for
 *   invalid arguments and TVOLAP_ERR_CAPACITY only when the stream's
 *   footprint is larger than the whole arena (it could never be admitted);
 *   otherwise TVOLAP_OK, whether the request was admitted at once or queued.
 * tvolap_server_admitted
 *   moves out up to cap records of requests admitted from the queue since the
 *   last call, oldest first: tickets[k] received stream id ids[k] after
 *   waiting wait_ticks[k] base ticks (wait_ticks may be NULL); *count
 *   receives the number written. Records not taken stay for the next call.
 * tvolap_server_cancel
 *   removes a still-waiting request (TVOLAP_ERR_ARG when ticket is not
 *   waiting: unknown, admitted or cancelled).
 * tvolap_server_queue
 *   requests waiting, the base ticks the oldest has waited, requests admitted
 *   from the queue so far and the longest wait of those (any pointer may be
 *   NULL).
 */
TVOLAP_API int tvolap_server_submit(tvolap_server_t s, int L, int M, int n_out, int n_filters,
                                    const float *ir_dev, int ir_len, int64_t ir_stride,
                                    int64_t *ticket);
TVOLAP_API int tvolap_server_admitted(tvolap_server_t s, int64_t *tickets, int32_t *ids,
                                      int64_t *wait_ticks, int cap, int *count);
TVOLAP_API int tvolap_server_cancel(tvolap_server_t s, int64_t ticket);
TVOLAP_API int tvolap_server_queue(tvolap_server_t s, int *waiting, int64_t *oldest_wait_ticks,
                                   int64_t *admitted_total, int64_t *max_wait_ticks);

/*
 * Stream snapshots (serving resilience, migration between slots or servers):
 * tvolap_server_stream_bytes gives the bytes of stream id's snapshot (a
 * 256-byte header, then its arena piece: transformed filters, delay line,
 * pending overlap-add sums, input history). tvolap_server_snapshot completes
 * the ticks in flight (as tvolap_server_wait, whose status it returns) and
 * copies the stream into buf (host or device memory, cap bytes).
 * tvolap_server_restore admits a new stream from a snapshot taken on a
 * server with the same hop range: a new slot and piece (TVOLAP_ERR_CAPACITY
 * when none is free), the piece copied on the admission stream (buf stays
 * valid until the stream is live or the server is waited on, as an
 * admission's responses), the block counter and the selected filter
 * restored; it becomes live like an admitted stream and continues exactly
 * where the snapshot was taken. Migrating a stream: snapshot, retire,
 * restore.
 */
TVOLAP_API int tvolap_server_stream_bytes(tvolap_server_t s, int id, int64_t *bytes);
TVOLAP_API int tvolap_server_snapshot(tvolap_server_t s, int id, void *buf, int64_t cap);
TVOLAP_API int tvolap_server_restore(tvolap_server_t s, const void *buf, int64_t bytes, int *id);

/* Retire a stream: it is never due again and its slot and memory are free. */
TVOLAP_API int tvolap_server_retire(tvolap_server_t s, int id);

/*
 * State of stream id: 0 free, 1 admitted (bank transform pending), 2 live.
 * blocks (may be NULL) receives the number of blocks the stream has been
 * given so far, phase (may be NULL) its phase in base ticks.
 */
TVOLAP_API int tvolap_server_state(tvolap_server_t s, int id, int *state, int64_t *blocks,
                                   int *phase);

/*
 * Host staging arrays of set `buffer` (0 or 1; pinned, valid for the
 * server's life):
 *   in   float [capacity][in_stride]          in_stride = max_hop
 *   sel  int32 [capacity]                     (one array, read by tick)
 *   out  float [capacity][max_out][out_stride] out_stride = max_hop
 * Any pointer argument may be NULL.
 */
TVOLAP_API int tvolap_server_staging(tvolap_server_t s, int buffer, float **in,
                                     int64_t *in_stride, int32_t **sel, float **out,
                                     int64_t *out_stride);

/*
 * Streams due at the next tick, in increasing id order (live streams whose
 * phase matches; streams whose admission work has finished turn live here).
 * Admits waiting requests of the admission queue that now fit (they turn
 * live at a later tick, once their bank transform has finished).
 * First waits for the tick that last used the next tick's staging set, whose
 * index goes to *buffer (may be NULL). Writes up to cap ids to ids_host and
 * the total to count.
 */
TVOLAP_API int tvolap_server_due(tvolap_server_t s, int32_t *ids_host, int cap, int *count,
                                 int *buffer);

/*
 * Run the next tick on the due streams (the list tvolap_server_due returned,
 * or would return). Reads sel[id] now and in[id] of its staging set when the
 * tick executes. Returns TVOLAP_ERR_ARG, with nothing enqueued, when a due
 * stream's sel is outside [0, n_filters). Returns without waiting; at most two
 * ticks are in flight (a third waits for the first).
 */
TVOLAP_API int tvolap_server_tick(tvolap_server_t s);

/*
 * Wait until every enqueued tick and admission has finished; afterwards the
 * out arrays of both staging sets hold the outputs of their last ticks. Returns TVOLAP_ERR_TIMEOUT when the input
 * wait of TVOLAP_SERVER_OPT_WAIT_US ran out for a tick: that tick processed
 * nothing, the due streams' block counts are rolled back (the same blocks
 * are due again), and the server stays usable. TVOLAP_ERR_CUDA on a CUDA
 * error.
 */
TVOLAP_API int tvolap_server_wait(tvolap_server_t s);

/*
 * Producer hand-off for TVOLAP_SERVER_OPT_WAIT_US: declare that the staging
 * for tick number seq (1 for the first tick, then 2, 3, ...) is written. Any
 * thread may call it.
 */
TVOLAP_API int tvolap_server_post(tvolap_server_t s, uint64_t seq);

/* Options of tvolap_server_set_option. */
typedef enum tvolap_server_option {
    /* 1 (default): each tick is a CUDA-graph replay; 0: direct launches. */
    TVOLAP_SERVER_OPT_GRAPH = 1,
    /* 0 (default): ticks start at once. > 0: each tick first waits on the GPU,
       for at most this many microseconds (<= 2000000), until
       tvolap_server_post has declared its staging written; one tick is in
       flight at a time. */
    TVOLAP_SERVER_OPT_WAIT_US = 2,
    /* 1: direct launches with CUDA events around the three stages; their
       times accumulate into tvolap_server_stats. 0 (default): off. */
    TVOLAP_SERVER_OPT_TIMING = 3,
    /* Fault injection on the host: the next `value` admissions (admit and
       restore) with valid arguments return TVOLAP_ERR_CAPACITY as if no arena
       piece were free, and change nothing. 0 (default): none. */
    TVOLAP_SERVER_OPT_FAIL_ADMITS = 4
} tvolap_server_option;

TVOLAP_API int tvolap_server_set_option(tvolap_server_t s, int option, int64_t value);

/* Counters of a server. */
typedef struct tvolap_server_stats {
    int64_t ticks;             /* ticks enqueued */
    int64_t stream_blocks;     /* (stream, block) pairs processed */
    int64_t channel_samples;   /* output samples produced, all outputs */
    int64_t mac_bytes;         /* algorithmic bytes of Eq. 7: spectra read + written */
    int32_t live, pending;     /* streams live / admitted but not yet live */
    int32_t last_due, last_items;
    int64_t arena_bytes, arena_used;
    double stage_ms[3];        /* forward, multiply-accumulate, inverse (timing option) */
    int64_t timed_ticks;       /* ticks that stage_ms covers */
} tvolap_server_stats;

TVOLAP_API int tvolap_server_stats_get(tvolap_server_t s, tvolap_server_stats *st);

/* ------------------------------------------------------------------------
 * The server's host-side scheduler on its own (no device memory, no GPU):
 * slot allocation, arena placement, phase choice and due lists, exactly as
 * the server uses them. Offsets are byte offsets into an arena of
 * arena_bytes. Arguments and errors are those of the server calls above.
 * ------------------------------------------------------------------------ */
typedef struct tvolap_sched *tvolap_sched_t;

TVOLAP_API int tvolap_sched_create(tvolap_sched_t *out, int base_hop, int max_hop, int capacity,
                                   int max_out, int64_t arena_bytes);
TVOLAP_API int tvolap_sched_destroy(tvolap_sched_t s);
/* Footprint of a stream (as tvolap_server_footprint). */
TVOLAP_API int tvolap_sched_footprint(int L, int M, int n_out, int n_filters, int64_t *bytes);
/* Admit: receives the id, the arena offset and the phase. */
TVOLAP_API int tvolap_sched_admit(tvolap_sched_t s, int L, int M, int n_out, int n_filters,
                                  int *id, int64_t *offset, int *phase);
/* Fault injection (as TVOLAP_SERVER_OPT_FAIL_ADMITS): the next n admissions
   with valid arguments return TVOLAP_ERR_CAPACITY and change nothing. */
TVOLAP_API int tvolap_sched_fail_admits(tvolap_sched_t s, int64_t n);
/* Admission queue (as tvolap_server_submit / _admitted / _cancel / _queue):
   submit queues a request and admits from the queue at once; pump admits
   waiting requests, oldest first, while they fit (*admitted may be NULL). */
TVOLAP_API int tvolap_sched_submit(tvolap_sched_t s, int L, int M, int n_out, int n_filters,
                                   int64_t *ticket);
TVOLAP_API int tvolap_sched_pump(tvolap_sched_t s, int *admitted);
TVOLAP_API int tvolap_sched_cancel(tvolap_sched_t s, int64_t ticket);
TVOLAP_API int tvolap_sched_admitted(tvolap_sched_t s, int64_t *tickets, int32_t *ids,
                                     int64_t *wait_ticks, int cap, int *count);
TVOLAP_API int tvolap_sched_queue(tvolap_sched_t s, int *waiting, int64_t *oldest_wait_ticks);
TVOLAP_API int tvolap_sched_activate(tvolap_sched_t s, int id);
TVOLAP_API int tvolap_sched_retire(tvolap_sched_t s, int id);
/* Due ids at the next tick (live streams only), as tvolap_server_due. */
TVOLAP_API int tvolap_sched_due(tvolap_sched_t s, int32_t *ids_host, int cap, int *count);
/* Advance one tick: the due streams' block counts grow by one. */
TVOLAP_API int tvolap_sched_advance(tvolap_sched_t s);
/* Bytes of Eq. 7 read per base tick by the streams due at each phase
   (loads[q] for q in [0, max_hop / base_hop)); *n receives that count. */
TVOLAP_API int tvolap_sched_phase_loads(tvolap_sched_t s, int64_t *loads, int cap, int *n);
/* Arena bytes in use, and the largest free piece. */
TVOLAP_API int tvolap_sched_arena(tvolap_sched_t s, int64_t *used, int64_t *largest_free);

#ifdef __cplusplus
}
#endif

#endif /* TVOLAP_H */

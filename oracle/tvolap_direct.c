/*
 * FP64 CPU oracle for time-variant overlap-add in partitions (TVOLAP).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code, header or table with the CUDA library.
 *
 * What it computes (arxiv 2310.00319, Section 2, Eqs. 1-12, restated in the
 * time domain without any FFT):
 *
 *   window   w(i) = 1/2 * (1 - cos(2*pi*i / 2L)),  0 <= i < 2L
 *            (Eq. "w_hann" with the 1/2 that makes the 50%-overlap sum equal 1)
 *   blocks   block l covers input samples [l*L, l*L + 2L); l = -1, 0, 1, ...
 *            (Eq. 1; x(n) = 0 outside [0, N))
 *   filter   h_l = (1 - alpha) * ir[a] + alpha * ir[b], the filter current at
 *            output block l, used for ALL partitions m (Section 2, the exchange
 *            of all transfer-function partitions at once; Eq. 7)
 *   output   y(n) = sum_l sum_{m<M} sum_{i<2L} sum_{j<2L}
 *                     w(i) x(l*L - 2mL + i) h_l(2mL + j) [n == l*L + i + j]
 *
 * Eqs. 5-8 evaluate, per block l, sum_m (block l-2m windowed) (*) (partition m of
 * h_l) by 4L-point DFTs; the zero padding of Eqs. 3-4 makes that product a linear
 * convolution of length 4L-1, which is exactly the double sum over i, j above.
 * Eqs. 9-12 then add every such length-4L result at offset l*L (the two-step
 * overlap-add with the preceding block of the same parity, l-2).
 *
 * Schedules are indexed by t = l + 1 (block l = -1 is schedule entry 0).
 * The caller supplies the number of schedule entries per output channel;
 * output samples [0, out_len) need t < floor((out_len - 1) / L) + 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static double hann_half(int i, int L)
{
    /* periodic Hann of length 2L, scaled by 1/2 (Eq. "w_hann", reading: the
       50%-overlapped windows then sum to exactly one) */
    const double pi = 3.14159265358979323846264338327950288;
    return 0.5 * (1.0 - cos(2.0 * pi * (double)i / (double)(2 * L)));
}

/* One output sample y_o(n) in the gather form: the (at most four) blocks l with
   0 <= n - l*L < 4L - 1, every partition m, every window position i. */
static double one_sample(int L, int M, int64_t N, const double *xc,
                         int ir_len, const double *irs,
                         int n_blocks, const int *sa, const int *sb, const double *sal,
                         const double *w, int64_t n)
{
    double acc = 0.0;
    int64_t l_hi = n / L;                      /* n - l*L >= 0 */
    int64_t l_lo = (n - (4 * (int64_t)L - 2) + L - 1);
    l_lo = (l_lo >= 0) ? l_lo / L : -((-l_lo + L - 1) / L);   /* ceil((n-4L+2)/L) */
    if (l_lo < -1) l_lo = -1;
    for (int64_t l = l_lo; l <= l_hi; ++l) {
        int64_t t = l + 1;
        if (t >= n_blocks) continue;          /* caller gave too few entries */
        const double *ha = irs + (int64_t)sa[t] * ir_len;
        const double *hb = irs + (int64_t)sb[t] * ir_len;
        const double alpha = sal[t];
        const int64_t d = n - l * L;           /* 0 .. 4L-2 */
        int i0 = (int)(d - (2 * L - 1));
        if (i0 < 0) i0 = 0;
        int i1 = (int)d;
        if (i1 > 2 * L - 1) i1 = 2 * L - 1;
        for (int m = 0; m < M; ++m) {
            for (int i = i0; i <= i1; ++i) {
                const int64_t s = l * L - 2 * (int64_t)m * L + i;   /* input index */
                if (s < 0 || s >= N) continue;
                const int64_t tap = 2 * (int64_t)m * L + (d - i); /* partition m, j = d - i */
                if (tap >= ir_len) continue;
                const double h = (1.0 - alpha) * ha[tap] + alpha * hb[tap];
                acc += w[i] * xc[s] * h;
            }
        }
    }
    return acc;
}

/*
 * Full output: y[o][n] for 0 <= n < out_len, every output channel o.
 *   x          [n_in][N]
 *   irs        [n_slots][ir_len]   stored impulse responses (taps)
 *   out_to_in  [n_out]             input channel feeding output o
 *   sched_*    [n_out][n_blocks]   a, b, alpha per output block (t = l + 1)
 *   y          [n_out][out_len]
 */
void oracle_tvolap_direct(int L, int M, int n_in, int64_t N, const double *x,
                          int n_slots, int ir_len, const double *irs,
                          int n_out, const int *out_to_in, int n_blocks,
                          const int *sched_a, const int *sched_b, const double *sched_alpha,
                          int64_t out_len, double *y)
{
    (void)n_in;
    (void)n_slots;
    double *w = (double *)malloc(sizeof(double) * 2 * L);
    for (int i = 0; i < 2 * L; ++i) w[i] = hann_half(i, L);
    for (int o = 0; o < n_out; ++o) {
        const double *xc = x + (int64_t)out_to_in[o] * N;
        const int *sa = sched_a + (int64_t)o * n_blocks;
        const int *sb = sched_b + (int64_t)o * n_blocks;
        const double *sal = sched_alpha + (int64_t)o * n_blocks;
        double *yo = y + (int64_t)o * out_len;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t n = 0; n < out_len; ++n)
            yo[n] = one_sample(L, M, N, xc, ir_len, irs, n_blocks, sa, sb, sal, w, n);
    }
    free(w);
}

/*
 * Sampled output: y_out[k] = y[out_ch[k]][n_idx[k]] for k < count. Same
 * arithmetic as oracle_tvolap_direct, for full-size checks on a sample.
 */
void oracle_tvolap_samples(int L, int M, int n_in, int64_t N, const double *x,
                           int n_slots, int ir_len, const double *irs,
                           int n_out, const int *out_to_in, int n_blocks,
                           const int *sched_a, const int *sched_b, const double *sched_alpha,
                           int count, const int *out_ch, const int64_t *n_idx, double *y_out)
{
    (void)n_in;
    (void)n_slots;
    (void)n_out;
    double *w = (double *)malloc(sizeof(double) * 2 * L);
    for (int i = 0; i < 2 * L; ++i) w[i] = hann_half(i, L);
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < count; ++k) {
        const int o = out_ch[k];
        y_out[k] = one_sample(L, M, N, x + (int64_t)out_to_in[o] * N, ir_len, irs, n_blocks,
                              sched_a + (int64_t)o * n_blocks, sched_b + (int64_t)o * n_blocks,
                              sched_alpha + (int64_t)o * n_blocks, w, n_idx[k]);
    }
    free(w);
}

/* Threads the OpenMP runtime will use (for reporting the CPU baseline). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

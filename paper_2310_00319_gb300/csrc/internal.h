// Internal plan layout and kernel launchers of the TVOLAP library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tvolap.h"

struct tvolap_plan {
    int L, M, P;                  // hop, partitions, complex bins per spectrum (2L)
    int lgP;                      // log2(P)
    int n_in, n_out;
    int identity_routing;         // n_in == n_out and output o reads input o
    int n_user_slots;             // slots written by tvolap_load_bank
    int n_slots_total;            // user + one private slot per output
    int null_slot;                // all-zero slot that replaces invalid indices
    cudaStream_t stream;

    // transform tables (FP32, generated in FP64 on the device)
    float2 *tw;                   // [2P]  FFT twiddles, stage by stage (tw_offset in fft_core.cuh)
    float2 *rot;                  // [P]   e^{-i pi r / P}
    float2 *post;                 // [P/2] e^{-i pi (2k+1) / 2P}
    float *win;                   // [2L]  (1 - cos(pi n / L)) / 2

    float2 *bank;                 // [n_slots_total + 1][M][P]
    int32_t *out_to_in;           // [n_out]
    int32_t *sel_a, *sel_b;       // [n_out] current selection (streaming)
    float *sel_alpha;             // [n_out]
    unsigned int *err;            // [1] device error record (bit 0: invalid slot)

    // streaming state
    float2 *ring;                 // [n_in][2M][P] frequency-domain delay line
    float *hist;                  // [n_in][L] previous L input samples
    float *ola;                   // [n_out][3L] pending overlap-add sums
    float2 *Ystream;              // [n_out][P] this tick's output spectra
    int64_t tick;

    int mac_variant;              // 0: TMA staging, persistent groups of <= 3 slots (when
                                  // the buffers allow TMA), 1: cp.async staging, 2: TMA,
                                  // groups of <= 4 slots, 3: TMA, one group of <= 3 slots
                                  // per CTA, 4: as 3 with two bins per thread,
                                  // 5: as 0 with groups of <= 4 slots
    int xform_threads;            // CTA size of the offline transform kernels (0: 256)
    int4 *ovf_list;               // groups the group kernel hands to the per-warp kernel
    int *ovf_count;
    int64_t ovf_cap;

    // process_signal workspace
    void *ws;
    size_t ws_bytes;

    // frequency-domain mixdown (tvolap_set_mix): mix output e sums the spectra
    // of plan outputs mix_members[mix_off[e] .. mix_off[e + 1]), in increasing order
    int n_mix;
    int32_t *mix_off;             // [n_mix + 1]
    int32_t *mix_members;         // [n_out]
    float *mix_ola;               // [n_mix][3L] pending overlap-add sums (streaming)
    float2 *Ymix_stream;          // [n_mix][P] this tick's mixed spectra

    // stage timing of streaming ticks (TVOLAP_OPT_STAGE_TIMING): events around
    // the forward transform, the multiply-accumulate and the inverse of the
    // last tick, and the times of the earlier timed ticks
    int timing;
    cudaEvent_t tev[4];
    int tev_pending;
    double stage_ms[3];
    int64_t timed_ticks;
};

namespace tvolap {

// Per-channel sizes of a ragged batch: device arrays, all null for a uniform
// batch. Channel c is input c and output c (identity routing). Kernels clamp
// every value to the plan and the launch (0 <= n <= x_stride, 0 <= out_len <=
// the launch's output length, 1 <= parts <= M).
struct Ragged {
    const int64_t *n;          // [n_in]  input samples
    const int64_t *out_len;    // [n_out] output samples
    const int32_t *parts;      // [n_out] partitions used
};

__host__ __device__ inline int64_t blocks_of(int64_t out_len, int L)
{
    return out_len <= 0 ? 0 : (out_len - 1) / L + 2;
}

// kernels_fft.cu
cudaError_t launch_tables(tvolap_plan *h);
cudaError_t launch_forward_signal(tvolap_plan *h, const float *x, int64_t N, int64_t x_stride,
                                  int n_blocks, float2 *X);
cudaError_t launch_block_spectra(tvolap_plan *h, const float *x, int64_t N, int64_t x_stride,
                                 int64_t t_first, int n_blocks, float2 *X, Ragged rg = Ragged{});
cudaError_t launch_adjoint_output(tvolap_plan *h, const float *g, int64_t g_len, int64_t g_stride,
                                  int64_t t_first, int n_blocks, float2 *G);
cudaError_t launch_adjoint_input(tvolap_plan *h, const float2 *dX, int64_t q_first, int q_count,
                                 float *dx, int64_t N, int64_t x_stride);
cudaError_t launch_bank(tvolap_plan *h, int first_slot, int count, const float *ir, int ir_len,
                        int64_t ir_stride);
// n_outputs: spectra rows of Y and output rows of y (-1: the plan's n_out)
cudaError_t launch_inverse_ola(tvolap_plan *h, const float2 *Y, int n_blocks, float *y,
                               int64_t out_len, int64_t y_stride, Ragged rg = Ragged{},
                               int n_outputs = -1);
cudaError_t launch_forward_stream(tvolap_plan *h, const float *in);
// Ys, ola, n_outputs: this tick's spectra and pending sums (null, -1: the plan's outputs)
cudaError_t launch_inverse_stream(tvolap_plan *h, float *out, const float2 *Ys = nullptr,
                                  float *ola = nullptr, int n_outputs = -1);
// Ymix[e][t] = sum over the members of mix output e of Y[o][t], t < n_blocks
cudaError_t launch_mix_spectra(tvolap_plan *h, const float2 *Y, int n_blocks, float2 *Ymix);
// tables and bank transform for a hop L (P = 2L = 1 << lgP) outside a plan
cudaError_t launch_tables_raw(float2 *tw, float2 *rot, float2 *post, float *win, int L,
                              cudaStream_t st);
cudaError_t launch_bank_raw(int lgP, int L, int M, int64_t count, const float *ir, int ir_len,
                            int64_t ir_stride, const float2 *rot, const float2 *post,
                            const float2 *tw, float2 *dst, cudaStream_t st);

// kernels_mac_tma.cu (falls back to the cp.async kernel of kernels_mac.cu)
cudaError_t launch_mac_signal(tvolap_plan *h, const float2 *X, int n_blocks, const int32_t *sa,
                              const int32_t *sb, const float *sal, int64_t sched_stride,
                              float2 *Y, Ragged rg = Ragged{});
// api.cu: grow the overflow list of the offline multiply-accumulate
cudaError_t ensure_overflow(tvolap_plan *h, int64_t entries);

// kernels_adjoint.cu
cudaError_t launch_mac_params(tvolap_plan *h, const float2 *X, int64_t x_first, int x_count,
                              const float2 *Pm, int64_t p_blocks, int64_t t_first, int t_count,
                              float2 *Y, int64_t y_rows);
cudaError_t launch_adjoint_mac(tvolap_plan *h, const float2 *G, int64_t g_first, int g_count,
                               const float2 *X, int64_t x_first, int x_count, const float2 *Pm,
                               int64_t p_blocks, int64_t q_first, int q_count, float2 *dP,
                               float2 *dX, int64_t dx_rows);
cudaError_t launch_adjoint_mac_x(tvolap_plan *h, const float2 *G, int64_t g_first, int g_count,
                                 const float *x, int64_t N, int64_t x_stride, const float2 *Pm,
                                 int64_t p_blocks, int64_t q_first, int q_count, float2 *dP,
                                 float2 *dX, int64_t dx_rows);

// kernels_mac.cu
cudaError_t launch_mac_signal_lsu(tvolap_plan *h, const float2 *X, int n_blocks,
                                  const int32_t *sa, const int32_t *sb, const float *sal,
                                  int64_t sched_stride, float2 *Y, Ragged rg = Ragged{});
cudaError_t launch_mac_stream(tvolap_plan *h, const int32_t *sa, const int32_t *sb,
                              const float *sal);
cudaError_t launch_select(tvolap_plan *h, int out_ch, int a, int b, float alpha);

}  // namespace tvolap

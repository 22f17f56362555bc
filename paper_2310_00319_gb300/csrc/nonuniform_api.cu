// Two-level non-uniform partitioning built from two TVOLAP plans (C ABI
// tvolap_nu_*). The head plan (hop La, Ma partitions) convolves with taps
// [0, D), D = 2 La Ma, at the latency of the small hop; the tail plan (hop
// Lb = r La, Mb partitions) convolves with taps [D, D + 2 Lb Mb) and its
// aligned output is added D samples later. By linearity and time invariance
// of each level, a fixed response gives exactly its full convolution; under
// switching each level crossfades at its own block boundaries (Section 2's
// exchange of all partitions at once, per level). The tail's filter for its
// schedule entry tb is the head's entry (tb + 1) r - 1: in streaming that is
// the selection given with the head tick that completes the tail's hop.
#include <new>

#include "internal.h"
#include "trace.h"

struct tvolap_nu {
    tvolap_t head = nullptr, tail = nullptr;
    int La = 0, Ma = 0, r = 1, Lb = 0, Mb = 0, n_in = 0, n_out = 0;
    int64_t D = 0;
    cudaStream_t stream = nullptr;
    // offline workspace: tail schedules and tail output
    int32_t *ta = nullptr, *tb = nullptr;
    float *tal = nullptr, *yt = nullptr;
    int64_t ws_sched = 0, ws_y = 0;
    // streaming: tail input accumulator [n_in][Lb], tail output block
    // [n_out][Lb], delay ring [n_out][ring] of aligned tail output samples
    float *acc = nullptr, *tout = nullptr, *ring = nullptr;
    int64_t ring_len = 0, tick = 0;
};

namespace {

// sched_tail[o][t] = sched_head[o][min((t + 1) r - 1, nb_head - 1)], t < nb_tail
__global__ void k_nu_tail_sched(const int32_t *__restrict__ sa, const int32_t *__restrict__ sb,
                                const float *__restrict__ sal, int64_t stride, int nb_head, int r,
                                int n_out, int nb_tail, int32_t *ta, int32_t *tb, float *tal)
{
    const int64_t total = (int64_t)n_out * nb_tail;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i / nb_tail), t = (int)(i % nb_tail);
        int64_t th = (int64_t)(t + 1) * r - 1;
        if (th > nb_head - 1) th = nb_head - 1;
        const int64_t src = (int64_t)o * stride + th;
        ta[i] = sa[src];
        tb[i] = sb ? sb[src] : sa[src];
        tal[i] = sal ? sal[src] : 0.f;
    }
}

// y[o][n] += yt[o][n - D], D <= n < out_len
__global__ void k_nu_add_shifted(float *y, int64_t y_stride, const float *__restrict__ yt,
                                 int64_t yt_len, int64_t D, int64_t out_len, int n_out)
{
    const int64_t span = out_len - D;
    const int64_t total = (int64_t)n_out * span;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i / span);
        const int64_t m = i % span;
        y[(int64_t)o * y_stride + D + m] += yt[(int64_t)o * yt_len + m];
    }
}

// streaming: this head tick's input into the tail accumulator at column off
__global__ void k_nu_stage_in(const float *__restrict__ in, int La, int n_in, float *acc, int Lb,
                              int off)
{
    const int total = n_in * La;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        acc[(i / La) * Lb + off + i % La] = in[i];
}

// streaming: the tail tick's output block (aligned samples [m0, m0 + Lb)) into the ring
__global__ void k_nu_ring_write(const float *__restrict__ tout, int Lb, int n_out, float *ring,
                                int64_t ring_len, int64_t m0)
{
    const int total = n_out * Lb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int64_t m = m0 + i % Lb;
        if (m >= 0) ring[(int64_t)(i / Lb) * ring_len + m % ring_len] = tout[i];
    }
}

// streaming: head output samples [n0, n0 + La) += aligned tail samples n - D
__global__ void k_nu_add_ring(float *out, int La, int n_out, const float *__restrict__ ring,
                              int64_t ring_len, int64_t n0, int64_t D)
{
    const int total = n_out * La;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int64_t m = n0 + i % La - D;
        if (m >= 0) out[i] += ring[(int64_t)(i / La) * ring_len + m % ring_len];
    }
}

unsigned grid_for(int64_t total)
{
    int64_t g = (total + 255) / 256;
    if (g > 4096) g = 4096;
    return (unsigned)(g < 1 ? 1 : g);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? TVOLAP_OK : TVOLAP_ERR_CUDA; }

void free_nu(tvolap_nu *h)
{
    if (!h) return;
    if (h->head) tvolap_destroy(h->head);
    if (h->tail) tvolap_destroy(h->tail);
    void *ptrs[] = {h->ta, h->tb, h->tal, h->yt, h->acc, h->tout, h->ring};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete h;
}

}  // namespace

extern "C" {

int tvolap_nu_create(tvolap_nu_t *out, int La, int Ma, int ratio, int Mb, int n_in, int n_out,
                     const int32_t *out_to_in, int n_slots, void *stream)
{
    if (!out) return TVOLAP_ERR_ARG;
    *out = nullptr;
    if (ratio < 2 || ratio > 64 || (ratio & (ratio - 1)) || Ma < ratio - 1 || Ma < 1 || Mb < 1 ||
        (int64_t)La * ratio > 1024)
        return TVOLAP_ERR_ARG;
    tvolap_nu *h = new (std::nothrow) tvolap_nu;
    if (!h) return TVOLAP_ERR_OOM;
    h->La = La;
    h->Ma = Ma;
    h->r = ratio;
    h->Lb = La * ratio;
    h->Mb = Mb;
    h->n_in = n_in;
    h->n_out = n_out;
    h->D = 2LL * La * Ma;
    h->stream = (cudaStream_t)stream;
    int st = tvolap_create(&h->head, La, Ma, 4 * La, n_in, n_out, out_to_in, n_slots, stream);
    if (st == TVOLAP_OK)
        st = tvolap_create(&h->tail, h->Lb, Mb, 4 * h->Lb, n_in, n_out, out_to_in, n_slots, stream);
    if (st != TVOLAP_OK) {
        free_nu(h);
        return st;
    }
    // the ring outlives a tail sample from its tick to its last use: D + 2 Lb covers it
    h->ring_len = h->D + 2LL * h->Lb;
    cudaError_t e = cudaMalloc(&h->acc, sizeof(float) * (size_t)n_in * h->Lb);
    if (e == cudaSuccess) e = cudaMalloc(&h->tout, sizeof(float) * (size_t)n_out * h->Lb);
    if (e == cudaSuccess) e = cudaMalloc(&h->ring, sizeof(float) * (size_t)n_out * h->ring_len);
    if (e != cudaSuccess) {
        free_nu(h);
        return TVOLAP_ERR_OOM;
    }
    st = tvolap_nu_reset(h);
    if (st != TVOLAP_OK) {
        free_nu(h);
        return st;
    }
    *out = h;
    return TVOLAP_OK;
}

int tvolap_nu_destroy(tvolap_nu_t h)
{
    if (!h) return TVOLAP_OK;
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    free_nu(h);
    return status_of(e);
}

int tvolap_nu_reset(tvolap_nu_t h)
{
    if (!h) return TVOLAP_ERR_STATE;
    int st = tvolap_reset(h->head);
    if (st == TVOLAP_OK) st = tvolap_reset(h->tail);
    if (st != TVOLAP_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->ring, 0, sizeof(float) * (size_t)h->n_out * h->ring_len, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->acc, 0, sizeof(float) * (size_t)h->n_in * h->Lb, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->tick = 0;
    return status_of(e);
}

int tvolap_nu_dims(tvolap_nu_t h, int *La, int *Lb, int64_t *head_taps, int64_t *max_taps)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (La) *La = h->La;
    if (Lb) *Lb = h->Lb;
    if (head_taps) *head_taps = h->D;
    if (max_taps) *max_taps = h->D + 2LL * h->Lb * h->Mb;
    return TVOLAP_OK;
}

int tvolap_nu_load_bank(tvolap_nu_t h, int first_slot, int count, const float *ir_dev, int ir_len,
                        int64_t ir_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (count < 0 || ir_len < 1 || ir_stride < ir_len || (count > 0 && !ir_dev) ||
        (int64_t)ir_len > h->D + 2LL * h->Lb * h->Mb)
        return TVOLAP_ERR_ARG;
    if (count == 0) return TVOLAP_OK;
    const int head_len = (int)(ir_len < h->D ? ir_len : h->D);
    int st = tvolap_load_bank(h->head, first_slot, count, ir_dev, head_len, ir_stride);
    if (st != TVOLAP_OK) return st;
    if (ir_len > h->D) {
        st = tvolap_load_bank(h->tail, first_slot, count, ir_dev + h->D, (int)(ir_len - h->D),
                              ir_stride);
    } else {
        // no tail taps: the tail slots hold zero responses
        float *zero = nullptr;
        cudaError_t e = cudaMalloc(&zero, sizeof(float) * (size_t)count);
        if (e != cudaSuccess) return TVOLAP_ERR_OOM;
        e = cudaMemsetAsync(zero, 0, sizeof(float) * (size_t)count, h->stream);
        st = e == cudaSuccess ? tvolap_load_bank(h->tail, first_slot, count, zero, 1, 1) : TVOLAP_ERR_CUDA;
        cudaStreamSynchronize(h->stream);
        cudaFree(zero);
    }
    return st;
}

int tvolap_nu_process_signal(tvolap_nu_t h, const float *x_dev, int64_t N, int64_t x_stride,
                             const int32_t *sched_a, const int32_t *sched_b, const float *sched_alpha,
                             int64_t sched_stride, float *y_dev, int64_t out_len, int64_t y_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    int st = tvolap_process_signal(h->head, x_dev, N, x_stride, sched_a, sched_b, sched_alpha,
                                   sched_stride, y_dev, out_len, y_stride);
    if (st != TVOLAP_OK || out_len <= h->D) return st;
    const int64_t tail_len = out_len - h->D;
    const int64_t nb_head = (out_len - 1) / h->La + 2, nb_tail = (tail_len - 1) / h->Lb + 2;
    const int64_t need_s = (int64_t)h->n_out * nb_tail, need_y = (int64_t)h->n_out * tail_len;
    cudaError_t e = cudaSuccess;
    if (need_s > h->ws_sched || need_y > h->ws_y) {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return TVOLAP_ERR_CUDA;
    }
    if (need_s > h->ws_sched) {
        cudaFree(h->ta);
        cudaFree(h->tb);
        cudaFree(h->tal);
        h->ta = h->tb = nullptr;
        h->tal = nullptr;
        h->ws_sched = 0;
        if (cudaMalloc(&h->ta, sizeof(int32_t) * need_s) != cudaSuccess ||
            cudaMalloc(&h->tb, sizeof(int32_t) * need_s) != cudaSuccess ||
            cudaMalloc(&h->tal, sizeof(float) * need_s) != cudaSuccess)
            return TVOLAP_ERR_OOM;
        h->ws_sched = need_s;
    }
    if (need_y > h->ws_y) {
        cudaFree(h->yt);
        h->yt = nullptr;
        h->ws_y = 0;
        if (cudaMalloc(&h->yt, sizeof(float) * need_y) != cudaSuccess) return TVOLAP_ERR_OOM;
        h->ws_y = need_y;
    }
    k_nu_tail_sched<<<grid_for(need_s), 256, 0, h->stream>>>(sched_a, sched_b, sched_alpha,
                                                            sched_stride, (int)nb_head, h->r,
                                                            h->n_out, (int)nb_tail, h->ta, h->tb,
                                                            h->tal);
    if ((e = cudaGetLastError()) != cudaSuccess) return TVOLAP_ERR_CUDA;
    st = tvolap_process_signal(h->tail, x_dev, N, x_stride, h->ta, h->tb, h->tal, nb_tail, h->yt,
                               tail_len, tail_len);
    if (st != TVOLAP_OK) return st;
    k_nu_add_shifted<<<grid_for(need_y), 256, 0, h->stream>>>(y_dev, y_stride, h->yt, tail_len, h->D,
                                                             out_len, h->n_out);
    return status_of(cudaGetLastError());
}

int tvolap_nu_process_block(tvolap_nu_t h, const float *in_dev, float *out_dev, const int32_t *sel_a,
                            const int32_t *sel_b, const float *sel_alpha)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!in_dev || !out_dev) return TVOLAP_ERR_ARG;
    int st = tvolap_process_block(h->head, in_dev, out_dev, sel_a, sel_b, sel_alpha);
    if (st != TVOLAP_OK) return st;
    const int off = (int)(h->tick % h->r) * h->La;
    k_nu_stage_in<<<grid_for((int64_t)h->n_in * h->La), 256, 0, h->stream>>>(in_dev, h->La, h->n_in,
                                                                              h->acc, h->Lb, off);
    if (cudaGetLastError() != cudaSuccess) return TVOLAP_ERR_CUDA;
    if ((h->tick + 1) % h->r == 0) {
        // tail tick k consumes input [k Lb, (k + 1) Lb) and emits aligned [(k - 1) Lb, k Lb)
        const int64_t k = (h->tick + 1) / h->r - 1;
        // the tail takes the head's current selection (set by this or an earlier tick)
        st = tvolap_process_block(h->tail, h->acc, h->tout, h->head->sel_a, h->head->sel_b,
                                  h->head->sel_alpha);
        if (st != TVOLAP_OK) return st;
        k_nu_ring_write<<<grid_for((int64_t)h->n_out * h->Lb), 256, 0, h->stream>>>(
            h->tout, h->Lb, h->n_out, h->ring, h->ring_len, (k - 1) * h->Lb);
        if (cudaGetLastError() != cudaSuccess) return TVOLAP_ERR_CUDA;
    }
    // head tick t emits aligned samples [(t - 1) La, t La)
    k_nu_add_ring<<<grid_for((int64_t)h->n_out * h->La), 256, 0, h->stream>>>(
        out_dev, h->La, h->n_out, h->ring, h->ring_len, (h->tick - 1) * h->La, h->D);
    if (cudaGetLastError() != cudaSuccess) return TVOLAP_ERR_CUDA;
    h->tick += 1;
    return TVOLAP_OK;
}

int tvolap_nu_set_option(tvolap_nu_t h, int level, int option, int value)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (level < -1 || level > 1) return TVOLAP_ERR_ARG;
    int st = TVOLAP_OK;
    if (level != 1) st = tvolap_set_option(h->head, option, value);
    if (st == TVOLAP_OK && level != 0) st = tvolap_set_option(h->tail, option, value);
    return st;
}

int tvolap_nu_check(tvolap_nu_t h)
{
    if (!h) return TVOLAP_ERR_STATE;
    int st = tvolap_check(h->head);
    const int st2 = tvolap_check(h->tail);
    return st != TVOLAP_OK ? st : st2;
}

}  // extern "C"

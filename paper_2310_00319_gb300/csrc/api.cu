// C ABI of the TVOLAP library: argument checks, device state, launches.
// Declarations and the contract of every entry point are in include/tvolap.h.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.h"
#include "trace.h"

using namespace tvolap;

namespace {

int ilog2_exact(int v)
{
    int lg = 0;
    while ((1 << lg) < v) ++lg;
    return ((1 << lg) == v) ? lg : -1;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return TVOLAP_OK;
    if (e == cudaErrorMemoryAllocation) return TVOLAP_ERR_OOM;
    return TVOLAP_ERR_CUDA;
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

void free_plan(tvolap_plan *h)
{
    if (!h) return;
    void *ptrs[] = {h->tw,   h->rot,  h->post, h->win,     h->bank, h->out_to_in,
                    h->sel_a, h->sel_b, h->sel_alpha, h->err, h->ring, h->hist,
                    h->ola,  h->Ystream, h->ws,  h->ovf_list, h->ovf_count,
                    h->mix_off, h->mix_members, h->mix_ola, h->Ymix_stream};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : h->tev)
        if (e) cudaEventDestroy(e);
    delete h;
}

// Adds the stage times of the last timed tick (waits for it).
cudaError_t timing_collect(tvolap_plan *h)
{
    if (!h->tev_pending) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(h->tev[3]);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->tev[i], h->tev[i + 1]);
        h->stage_ms[i] += ms;
    }
    h->tev_pending = 0;
    if (e == cudaSuccess) h->timed_ticks += 1;
    return e;
}

// Event i of a timed tick (i = 0 before the forward transform, 1 before the
// multiply-accumulate, 2 before the inverse, 3 after it); nothing when off.
cudaError_t timing_mark(tvolap_plan *h, int i)
{
    if (!h->timing) return cudaSuccess;
    if (i == 0) {
        const cudaError_t e = timing_collect(h);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = cudaEventRecord(h->tev[i], h->stream);
    if (i == 3 && e == cudaSuccess) h->tev_pending = 1;
    return e;
}

int64_t blocks_for(const tvolap_plan *h, int64_t out_len)
{
    return out_len <= 0 ? 0 : (out_len - 1) / h->L + 2;
}

// Device memory for process_signal: X [n_in][nb][P], Y [n_out][nb][P], then
// (with a mixdown) Ymix [n_mix][nb][P].
int64_t workspace_bytes(const tvolap_plan *h, int64_t nb)
{
    return (int64_t)sizeof(float2) * h->P * nb * (h->n_in + h->n_out + h->n_mix);
}

int ensure_workspace(tvolap_plan *h, size_t bytes)
{
    if (bytes <= h->ws_bytes) return TVOLAP_OK;
    if (h->ws) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return TVOLAP_ERR_OOM;
    }
    h->ws_bytes = bytes;
    return TVOLAP_OK;
}

int reset_state(tvolap_plan *h)
{
    cudaError_t e;
    const size_t P = h->P;
    if ((e = cudaMemsetAsync(h->ring, 0, sizeof(float2) * h->n_in * 2 * h->M * P, h->stream)) ||
        (e = cudaMemsetAsync(h->hist, 0, sizeof(float) * h->n_in * h->L, h->stream)) ||
        (e = cudaMemsetAsync(h->ola, 0, sizeof(float) * h->n_out * 3 * h->L, h->stream)) ||
        (h->n_mix > 0 &&
         (e = cudaMemsetAsync(h->mix_ola, 0, sizeof(float) * h->n_mix * 3 * h->L, h->stream))) ||
        (e = cudaMemsetAsync(h->sel_alpha, 0, sizeof(float) * h->n_out, h->stream)))
        return cuda_status(e);
    // every output starts on its private (zero) slot
    int32_t *init = (int32_t *)malloc(sizeof(int32_t) * h->n_out);
    if (!init) return TVOLAP_ERR_OOM;
    for (int o = 0; o < h->n_out; ++o) init[o] = h->n_user_slots + o;
    e = cudaMemcpyAsync(h->sel_a, init, sizeof(int32_t) * h->n_out, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->sel_b, init, sizeof(int32_t) * h->n_out, cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // init is pageable and freed below
    free(init);
    h->tick = 0;
    return cuda_status(e);
}

}  // namespace

namespace tvolap {

cudaError_t ensure_overflow(tvolap_plan *h, int64_t entries)
{
    if (!h->ovf_count) {
        cudaError_t e = cudaMalloc(&h->ovf_count, 2 * sizeof(int));
        if (e != cudaSuccess) return e;
    }
    if (entries <= h->ovf_cap) return cudaSuccess;
    if (h->ovf_list) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return e;
        cudaFree(h->ovf_list);
        h->ovf_list = nullptr;
        h->ovf_cap = 0;
    }
    cudaError_t e = cudaMalloc(&h->ovf_list, sizeof(int4) * (size_t)entries);
    if (e != cudaSuccess) return e;
    h->ovf_cap = entries;
    return cudaSuccess;
}

}  // namespace tvolap

// Streaming-state snapshot: a header, then each array at a 256-byte aligned
// offset (delay line, input history, pending sums, selection, mix pending sums).
namespace {

struct StateHeader {
    uint32_t magic, version;
    int32_t L, M, n_in, n_out, n_mix, pad;
    int64_t tick;
};
constexpr uint32_t STATE_MAGIC = 0x54535654u;   // "TVST"
constexpr uint32_t STATE_VERSION = 1;

struct StatePart {
    void *dev;
    int64_t bytes;
};

int state_parts(tvolap_plan *h, StatePart (&p)[7])
{
    const int64_t P = h->P, L = h->L;
    p[0] = {h->ring, (int64_t)sizeof(float2) * h->n_in * 2 * h->M * P};
    p[1] = {h->hist, (int64_t)sizeof(float) * h->n_in * L};
    p[2] = {h->ola, (int64_t)sizeof(float) * h->n_out * 3 * L};
    p[3] = {h->sel_a, (int64_t)sizeof(int32_t) * h->n_out};
    p[4] = {h->sel_b, (int64_t)sizeof(int32_t) * h->n_out};
    p[5] = {h->sel_alpha, (int64_t)sizeof(float) * h->n_out};
    p[6] = {h->mix_ola, (int64_t)sizeof(float) * h->n_mix * 3 * L};
    return 7;
}

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

int64_t state_bytes(tvolap_plan *h)
{
    StatePart p[7];
    int64_t off = align256(sizeof(StateHeader));
    for (int i = 0, n = state_parts(h, p); i < n; ++i) off += align256(p[i].bytes);
    return off;
}

}  // namespace

extern "C" {

const char *tvolap_strerror(int status)
{
    switch (status) {
    case TVOLAP_OK: return "TVOLAP_OK";
    case TVOLAP_ERR_ARG: return "TVOLAP_ERR_ARG: invalid argument";
    case TVOLAP_ERR_OOM: return "TVOLAP_ERR_OOM: device allocation failed";
    case TVOLAP_ERR_CUDA: return "TVOLAP_ERR_CUDA: CUDA runtime or launch failure";
    case TVOLAP_ERR_STATE: return "TVOLAP_ERR_STATE: invalid handle";
    case TVOLAP_ERR_CAPACITY: return "TVOLAP_ERR_CAPACITY: capacity exceeded";
    case TVOLAP_ERR_TIMEOUT: return "TVOLAP_ERR_TIMEOUT: bounded device wait gave up";
    default: return "TVOLAP: unknown status";
    }
}

int tvolap_version(void) { return 10000; }

int tvolap_create(tvolap_t *out, int L, int partitions, int fft_len, int n_in, int n_out,
                  const int32_t *out_to_in, int n_slots, void *stream)
{
    if (!out) return TVOLAP_ERR_ARG;
    *out = nullptr;
    const int lgL = ilog2_exact(L);
    if (lgL < 4 || lgL > 10) return TVOLAP_ERR_ARG;              // L in 16 .. 1024
    if (partitions < 1 || (fft_len != 0 && fft_len != 4 * L)) return TVOLAP_ERR_ARG;
    if (n_in < 1 || n_out < 1 || n_slots < 1) return TVOLAP_ERR_ARG;
    if (!out_to_in && n_in != n_out) return TVOLAP_ERR_ARG;
    if (out_to_in)
        for (int o = 0; o < n_out; ++o)
            if (out_to_in[o] < 0 || out_to_in[o] >= n_in) return TVOLAP_ERR_ARG;
    if ((int64_t)n_slots + n_out + 1 > (1 << 30)) return TVOLAP_ERR_ARG;

    tvolap_plan *h = new (std::nothrow) tvolap_plan;
    if (!h) return TVOLAP_ERR_OOM;
    memset(h, 0, sizeof(*h));
    h->L = L;
    h->M = partitions;
    h->P = 2 * L;
    h->lgP = lgL + 1;
    h->n_in = n_in;
    h->n_out = n_out;
    h->n_user_slots = n_slots;
    h->n_slots_total = n_slots + n_out;
    h->null_slot = n_slots + n_out;
    h->stream = (cudaStream_t)stream;

    const size_t P = h->P, M = h->M;
    cudaError_t e;
    if ((e = dalloc(&h->tw, 2 * P)) || (e = dalloc(&h->rot, P)) || (e = dalloc(&h->post, P / 2)) ||
        (e = dalloc(&h->win, 2 * (size_t)L)) ||
        (e = dalloc(&h->bank, (size_t)(h->n_slots_total + 1) * M * P)) ||
        (e = dalloc(&h->out_to_in, (size_t)n_out)) || (e = dalloc(&h->sel_a, (size_t)n_out)) ||
        (e = dalloc(&h->sel_b, (size_t)n_out)) || (e = dalloc(&h->sel_alpha, (size_t)n_out)) ||
        (e = dalloc(&h->err, 1)) || (e = dalloc(&h->ring, (size_t)n_in * 2 * M * P)) ||
        (e = dalloc(&h->hist, (size_t)n_in * L)) || (e = dalloc(&h->ola, (size_t)n_out * 3 * L)) ||
        (e = dalloc(&h->Ystream, (size_t)n_out * P))) {
        cudaGetLastError();
        free_plan(h);
        return cuda_status(e);
    }
    int32_t *o2i = (int32_t *)malloc(sizeof(int32_t) * n_out);
    if (!o2i) {
        free_plan(h);
        return TVOLAP_ERR_OOM;
    }
    h->identity_routing = (n_in == n_out);
    for (int o = 0; o < n_out; ++o) {
        o2i[o] = out_to_in ? out_to_in[o] : o;
        if (o2i[o] != o) h->identity_routing = 0;
    }
    e = cudaMemcpyAsync(h->out_to_in, o2i, sizeof(int32_t) * n_out, cudaMemcpyHostToDevice,
                        h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->bank, 0, sizeof(float2) * (h->n_slots_total + 1) * M * P, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = launch_tables(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    free(o2i);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(h);
        return cuda_status(e);
    }
    int st = reset_state(h);
    if (st != TVOLAP_OK) {
        free_plan(h);
        return st;
    }
    *out = h;
    return TVOLAP_OK;
}

int tvolap_destroy(tvolap_t h)
{
    if (!h) return TVOLAP_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    free_plan(h);
    return cuda_status(e);
}

int tvolap_get_dims(tvolap_t h, int *L, int *M, int *P, int *n_in, int *n_out, int *n_slots)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (L) *L = h->L;
    if (M) *M = h->M;
    if (P) *P = h->P;
    if (n_in) *n_in = h->n_in;
    if (n_out) *n_out = h->n_out;
    if (n_slots) *n_slots = h->n_user_slots;
    return TVOLAP_OK;
}

int tvolap_slot_count(tvolap_t h)
{
    if (!h) return TVOLAP_ERR_STATE;
    return h->n_slots_total;
}

int tvolap_reset(tvolap_t h)
{
    if (!h) return TVOLAP_ERR_STATE;
    return reset_state(h);
}

int tvolap_load_bank(tvolap_t h, int first_slot, int count, const float *ir_dev, int ir_len,
                     int64_t ir_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (first_slot < 0 || count < 0 || (int64_t)first_slot + count > h->n_user_slots)
        return TVOLAP_ERR_ARG;
    if (count == 0) return TVOLAP_OK;
    if (!ir_dev || ir_len < 1 || (int64_t)ir_len > 2LL * h->L * h->M || ir_stride < ir_len)
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_bank(h, first_slot, count, ir_dev, ir_len, ir_stride));
}

int tvolap_set_filter(tvolap_t h, int out_ch, const float *ir_dev, int ir_len)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (out_ch < 0 || out_ch >= h->n_out || !ir_dev || ir_len < 1 ||
        (int64_t)ir_len > 2LL * h->L * h->M)
        return TVOLAP_ERR_ARG;
    const int slot = h->n_user_slots + out_ch;
    cudaError_t e = launch_bank(h, slot, 1, ir_dev, ir_len, ir_len);
    if (e == cudaSuccess) e = launch_select(h, out_ch, slot, slot, 0.f);
    return cuda_status(e);
}

int tvolap_select(tvolap_t h, int out_ch, int slot_a, int slot_b, float alpha)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (out_ch < 0 || out_ch >= h->n_out || slot_a < 0 || slot_a >= h->n_slots_total ||
        slot_b < 0 || slot_b >= h->n_slots_total)
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_select(h, out_ch, slot_a, slot_b, alpha));
}

int tvolap_process_block(tvolap_t h, const float *in_dev, float *out_dev, const int32_t *sel_a,
                         const int32_t *sel_b, const float *sel_alpha)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!in_dev || !out_dev) return TVOLAP_ERR_ARG;
    if (!sel_a && (sel_b || sel_alpha)) return TVOLAP_ERR_ARG;
    cudaError_t e = timing_mark(h, 0);
    if (e == cudaSuccess) e = launch_forward_stream(h, in_dev);
    if (e == cudaSuccess) e = timing_mark(h, 1);
    if (e == cudaSuccess) e = launch_mac_stream(h, sel_a, sel_b, sel_alpha);
    if (e == cudaSuccess) e = timing_mark(h, 2);
    if (e == cudaSuccess) e = launch_inverse_stream(h, out_dev);
    if (e == cudaSuccess) e = timing_mark(h, 3);
    if (e != cudaSuccess) return cuda_status(e);
    h->tick += 1;
    return TVOLAP_OK;
}

int64_t tvolap_signal_workspace_bytes(tvolap_t h, int64_t out_len)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (out_len < 0) return TVOLAP_ERR_ARG;
    return workspace_bytes(h, blocks_for(h, out_len));
}

int tvolap_process_signal(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                          const int32_t *sched_a, const int32_t *sched_b,
                          const float *sched_alpha, int64_t sched_stride, float *y_dev,
                          int64_t out_len, int64_t y_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (N < 0 || out_len < 0 || x_stride < N || y_stride < out_len) return TVOLAP_ERR_ARG;
    if (out_len == 0) return TVOLAP_OK;
    if ((N > 0 && !x_dev) || !y_dev || !sched_a) return TVOLAP_ERR_ARG;
    const int64_t nb = blocks_for(h, out_len);
    if (nb > (int64_t)0x7fffffff / 2 || sched_stride < nb) return TVOLAP_ERR_ARG;
    int st = ensure_workspace(h, (size_t)workspace_bytes(h, nb));
    if (st != TVOLAP_OK) return st;
    float2 *X = reinterpret_cast<float2 *>(h->ws);
    float2 *Y = X + (int64_t)h->n_in * nb * h->P;
    cudaError_t e = launch_forward_signal(h, x_dev, N, x_stride, (int)nb, X);
    if (e == cudaSuccess)
        e = launch_mac_signal(h, X, (int)nb, sched_a, sched_b, sched_alpha, sched_stride, Y);
    if (e == cudaSuccess) e = launch_inverse_ola(h, Y, (int)nb, y_dev, out_len, y_stride);
    return cuda_status(e);
}

int tvolap_process_ragged(tvolap_t h, const float *x_dev, int64_t x_stride, const int64_t *n_dev,
                          const int64_t *out_len_dev, const int32_t *parts_dev, int64_t max_out_len,
                          const int32_t *sched_a, const int32_t *sched_b, const float *sched_alpha,
                          int64_t sched_stride, float *y_dev, int64_t y_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!h->identity_routing) return TVOLAP_ERR_ARG;
    if (max_out_len < 0 || x_stride < 0 || y_stride < max_out_len) return TVOLAP_ERR_ARG;
    if (max_out_len == 0) return TVOLAP_OK;
    if (!x_dev || !y_dev || !sched_a || !n_dev || !out_len_dev || !parts_dev) return TVOLAP_ERR_ARG;
    const int64_t nb = blocks_for(h, max_out_len);
    if (nb > (int64_t)0x7fffffff / 2 || sched_stride < nb) return TVOLAP_ERR_ARG;
    int st = ensure_workspace(h, (size_t)workspace_bytes(h, nb));
    if (st != TVOLAP_OK) return st;
    float2 *X = reinterpret_cast<float2 *>(h->ws);
    float2 *Y = X + (int64_t)h->n_in * nb * h->P;
    const Ragged rg{n_dev, out_len_dev, parts_dev};
    cudaError_t e = launch_block_spectra(h, x_dev, x_stride, x_stride, 0, (int)nb, X, rg);
    if (e == cudaSuccess)
        e = launch_mac_signal(h, X, (int)nb, sched_a, sched_b, sched_alpha, sched_stride, Y, rg);
    if (e == cudaSuccess) e = launch_inverse_ola(h, Y, (int)nb, y_dev, max_out_len, y_stride, rg);
    return cuda_status(e);
}

int tvolap_forward_spectra(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                           int n_blocks, float *X_dev)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (N < 0 || x_stride < N || n_blocks < 0 || (N > 0 && !x_dev) || (n_blocks > 0 && !X_dev))
        return TVOLAP_ERR_ARG;
    return cuda_status(
        launch_forward_signal(h, x_dev, N, x_stride, n_blocks, reinterpret_cast<float2 *>(X_dev)));
}

int tvolap_mac(tvolap_t h, const float *X_dev, int n_blocks, const int32_t *sched_a,
               const int32_t *sched_b, const float *sched_alpha, int64_t sched_stride,
               float *Y_dev)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (n_blocks < 0 || sched_stride < n_blocks) return TVOLAP_ERR_ARG;
    if (n_blocks == 0) return TVOLAP_OK;
    if (!X_dev || !Y_dev || !sched_a) return TVOLAP_ERR_ARG;
    return cuda_status(launch_mac_signal(h, reinterpret_cast<const float2 *>(X_dev), n_blocks,
                                         sched_a, sched_b, sched_alpha, sched_stride,
                                         reinterpret_cast<float2 *>(Y_dev)));
}

int tvolap_inverse_ola(tvolap_t h, const float *Y_dev, int n_blocks, float *y_dev,
                       int64_t out_len, int64_t y_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (out_len < 0 || y_stride < out_len || n_blocks != blocks_for(h, out_len))
        return TVOLAP_ERR_ARG;
    if (out_len == 0) return TVOLAP_OK;
    if (!Y_dev || !y_dev) return TVOLAP_ERR_ARG;
    return cuda_status(launch_inverse_ola(h, reinterpret_cast<const float2 *>(Y_dev), n_blocks,
                                          y_dev, out_len, y_stride));
}

int tvolap_bank_spectra(tvolap_t h, int slot, float *out_dev)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (slot < 0 || slot >= h->n_slots_total || !out_dev) return TVOLAP_ERR_ARG;
    const size_t bytes = sizeof(float2) * (size_t)h->M * h->P;
    return cuda_status(cudaMemcpyAsync(out_dev, h->bank + (int64_t)slot * h->M * h->P, bytes,
                                       cudaMemcpyDeviceToDevice, h->stream));
}

int tvolap_check(tvolap_t h)
{
    if (!h) return TVOLAP_ERR_STATE;
    unsigned err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (err) {
        e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_status(e);
        return (err & 2u) ? TVOLAP_ERR_TIMEOUT : TVOLAP_ERR_ARG;
    }
    return TVOLAP_OK;
}

static bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int tvolap_block_spectra(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                         int64_t t_first, int t_count, float *X_dev)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (N < 0 || x_stride < N || t_first < 0 || t_count < 0 || (N > 0 && !x_dev) ||
        (t_count > 0 && !X_dev))
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_block_spectra(h, x_dev, N, x_stride, t_first, t_count,
                                            reinterpret_cast<float2 *>(X_dev)));
}

int tvolap_mac_params(tvolap_t h, const float *X_dev, int64_t x_first, int x_count,
                      const float *P_dev, int64_t p_blocks, int64_t t_first, int t_count,
                      float *Y_dev, int64_t y_rows)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (t_count < 0 || t_first < 0 || x_first < 0 || x_count < 0) return TVOLAP_ERR_ARG;
    if (t_count == 0) return TVOLAP_OK;
    if (!X_dev || !P_dev || !Y_dev || !a16(X_dev) || !a16(P_dev) || !a16(Y_dev)) return TVOLAP_ERR_ARG;
    const int64_t need_lo = t_first - 2 * (int64_t)(h->M - 1) > 0 ? t_first - 2 * (int64_t)(h->M - 1) : 0;
    if (t_first + t_count > p_blocks || x_first > need_lo || x_first + x_count < t_first + t_count ||
        y_rows < t_count)
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_mac_params(h, reinterpret_cast<const float2 *>(X_dev), x_first, x_count,
                                         reinterpret_cast<const float2 *>(P_dev), p_blocks, t_first,
                                         t_count, reinterpret_cast<float2 *>(Y_dev), y_rows));
}

int tvolap_adjoint_output(tvolap_t h, const float *g_dev, int64_t g_len, int64_t g_stride,
                          int64_t t_first, int t_count, float *G_dev)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (g_len < 0 || g_stride < g_len || t_first < 0 || t_count < 0 || (g_len > 0 && !g_dev) ||
        (t_count > 0 && !G_dev))
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_adjoint_output(h, g_dev, g_len, g_stride, t_first, t_count,
                                             reinterpret_cast<float2 *>(G_dev)));
}

int tvolap_adjoint_mac(tvolap_t h, const float *G_dev, int64_t g_first, int g_count,
                       const float *X_dev, int64_t x_first, int x_count, const float *P_dev,
                       int64_t p_blocks, int64_t q_first, int q_count, float *dP_dev, float *dX_dev,
                       int64_t dx_rows)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!h->identity_routing) return TVOLAP_ERR_ARG;
    if (q_count < 0 || q_first < 0 || g_first < 0 || x_first < 0 || g_count < 0 || x_count < 0)
        return TVOLAP_ERR_ARG;
    if (q_count == 0) return TVOLAP_OK;
    if (!G_dev || !X_dev || !P_dev || !dP_dev || !dX_dev || !a16(G_dev) || !a16(X_dev) ||
        !a16(P_dev) || !a16(dP_dev) || !a16(dX_dev))
        return TVOLAP_ERR_ARG;
    int64_t g_need = q_first + q_count + 2 * (int64_t)(h->M - 1);
    if (g_need > p_blocks) g_need = p_blocks;
    if (q_first + q_count > p_blocks || x_first > q_first || x_first + x_count < q_first + q_count ||
        g_first > q_first || g_first + g_count < g_need || dx_rows < q_count)
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_adjoint_mac(
        h, reinterpret_cast<const float2 *>(G_dev), g_first, g_count,
        reinterpret_cast<const float2 *>(X_dev), x_first, x_count,
        reinterpret_cast<const float2 *>(P_dev), p_blocks, q_first, q_count,
        reinterpret_cast<float2 *>(dP_dev), reinterpret_cast<float2 *>(dX_dev), dx_rows));
}

int tvolap_adjoint_mac_x(tvolap_t h, const float *G_dev, int64_t g_first, int g_count,
                         const float *x_dev, int64_t N, int64_t x_stride, const float *P_dev,
                         int64_t p_blocks, int64_t q_first, int q_count, float *dP_dev,
                         float *dX_dev, int64_t dx_rows)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!h->identity_routing) return TVOLAP_ERR_ARG;
    if (q_count < 0 || q_first < 0 || g_first < 0 || g_count < 0 || N < 0 || x_stride < N)
        return TVOLAP_ERR_ARG;
    if (q_count == 0) return TVOLAP_OK;
    if (!G_dev || (!x_dev && N > 0) || !P_dev || !dP_dev || !dX_dev || !a16(G_dev) ||
        !a16(P_dev) || !a16(dP_dev) || !a16(dX_dev))
        return TVOLAP_ERR_ARG;
    int64_t g_need = q_first + q_count + 2 * (int64_t)(h->M - 1);
    if (g_need > p_blocks) g_need = p_blocks;
    if (q_first + q_count > p_blocks || g_first > q_first || g_first + g_count < g_need ||
        dx_rows < q_count)
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_adjoint_mac_x(
        h, reinterpret_cast<const float2 *>(G_dev), g_first, g_count, x_dev, N, x_stride,
        reinterpret_cast<const float2 *>(P_dev), p_blocks, q_first, q_count,
        reinterpret_cast<float2 *>(dP_dev), reinterpret_cast<float2 *>(dX_dev), dx_rows));
}

int tvolap_adjoint_input(tvolap_t h, const float *dX_dev, int64_t q_first, int q_count,
                         float *dx_dev, int64_t N, int64_t x_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!h->identity_routing) return TVOLAP_ERR_ARG;
    if (q_first < 0 || q_count < 0 || N < 0 || x_stride < N) return TVOLAP_ERR_ARG;
    if (q_count == 0 || N == 0) return TVOLAP_OK;
    if (!dX_dev || !dx_dev) return TVOLAP_ERR_ARG;
    return cuda_status(launch_adjoint_input(h, reinterpret_cast<const float2 *>(dX_dev), q_first,
                                            q_count, dx_dev, N, x_stride));
}

int tvolap_set_mix(tvolap_t h, int n_mix, const int32_t *mix_of_out)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (n_mix < 0 || n_mix > h->n_out || (n_mix > 0 && !mix_of_out)) return TVOLAP_ERR_ARG;
    for (int o = 0; n_mix > 0 && o < h->n_out; ++o)
        if (mix_of_out[o] < 0 || mix_of_out[o] >= n_mix) return TVOLAP_ERR_ARG;
    // members of each mix output in increasing output order (CSR)
    std::vector<int32_t> off(n_mix + 1, 0), members(n_mix > 0 ? h->n_out : 0);
    for (int o = 0; n_mix > 0 && o < h->n_out; ++o) ++off[mix_of_out[o] + 1];
    for (int e = 0; e < n_mix; ++e) off[e + 1] += off[e];
    {
        std::vector<int32_t> fill(off.begin(), off.end() - (n_mix > 0 ? 1 : 0));
        for (int o = 0; n_mix > 0 && o < h->n_out; ++o) members[fill[mix_of_out[o]]++] = o;
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);          // the old arrays may be in use
    if (e != cudaSuccess) return cuda_status(e);
    void *old[] = {h->mix_off, h->mix_members, h->mix_ola, h->Ymix_stream};
    for (void *p : old)
        if (p) cudaFree(p);
    h->mix_off = h->mix_members = nullptr;
    h->mix_ola = nullptr;
    h->Ymix_stream = nullptr;
    h->n_mix = 0;
    if (n_mix == 0) return TVOLAP_OK;
    if ((e = dalloc(&h->mix_off, (size_t)n_mix + 1)) || (e = dalloc(&h->mix_members, (size_t)h->n_out)) ||
        (e = dalloc(&h->mix_ola, (size_t)n_mix * 3 * h->L)) ||
        (e = dalloc(&h->Ymix_stream, (size_t)n_mix * h->P)))
        return cuda_status(e);
    if ((e = cudaMemcpy(h->mix_off, off.data(), sizeof(int32_t) * (n_mix + 1), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->mix_members, members.data(), sizeof(int32_t) * h->n_out,
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemsetAsync(h->mix_ola, 0, sizeof(float) * n_mix * 3 * h->L, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
        return cuda_status(e);
    h->n_mix = n_mix;
    return TVOLAP_OK;
}

int tvolap_mix(tvolap_t h, const void *Y_dev, int n_blocks, void *Ymix_dev)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (h->n_mix == 0 || n_blocks < 0) return TVOLAP_ERR_ARG;
    if (n_blocks == 0) return TVOLAP_OK;
    if (!Y_dev || !Ymix_dev || (reinterpret_cast<uintptr_t>(Y_dev) & 15u) ||
        (reinterpret_cast<uintptr_t>(Ymix_dev) & 15u))
        return TVOLAP_ERR_ARG;
    return cuda_status(launch_mix_spectra(h, reinterpret_cast<const float2 *>(Y_dev), n_blocks,
                                          reinterpret_cast<float2 *>(Ymix_dev)));
}

int tvolap_process_signal_mix(tvolap_t h, const float *x_dev, int64_t N, int64_t x_stride,
                              const int32_t *sched_a, const int32_t *sched_b,
                              const float *sched_alpha, int64_t sched_stride, float *y_dev,
                              int64_t out_len, int64_t y_stride)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (h->n_mix == 0) return TVOLAP_ERR_ARG;
    if (N < 0 || out_len < 0 || x_stride < N || y_stride < out_len) return TVOLAP_ERR_ARG;
    if (out_len == 0) return TVOLAP_OK;
    if ((N > 0 && !x_dev) || !y_dev || !sched_a) return TVOLAP_ERR_ARG;
    const int64_t nb = blocks_for(h, out_len);
    if (nb > (int64_t)0x7fffffff / 2 || sched_stride < nb) return TVOLAP_ERR_ARG;
    int st = ensure_workspace(h, (size_t)workspace_bytes(h, nb));
    if (st != TVOLAP_OK) return st;
    float2 *X = reinterpret_cast<float2 *>(h->ws);
    float2 *Y = X + (int64_t)h->n_in * nb * h->P;
    float2 *Ym = Y + (int64_t)h->n_out * nb * h->P;
    cudaError_t e = launch_forward_signal(h, x_dev, N, x_stride, (int)nb, X);
    if (e == cudaSuccess)
        e = launch_mac_signal(h, X, (int)nb, sched_a, sched_b, sched_alpha, sched_stride, Y);
    if (e == cudaSuccess) e = launch_mix_spectra(h, Y, (int)nb, Ym);
    if (e == cudaSuccess)
        e = launch_inverse_ola(h, Ym, (int)nb, y_dev, out_len, y_stride, Ragged{}, h->n_mix);
    return cuda_status(e);
}

int tvolap_process_block_mix(tvolap_t h, const float *in_dev, float *out_dev, const int32_t *sel_a,
                             const int32_t *sel_b, const float *sel_alpha)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (h->n_mix == 0 || !in_dev || !out_dev) return TVOLAP_ERR_ARG;
    if (!sel_a && (sel_b || sel_alpha)) return TVOLAP_ERR_ARG;
    cudaError_t e = launch_forward_stream(h, in_dev);
    if (e == cudaSuccess) e = launch_mac_stream(h, sel_a, sel_b, sel_alpha);
    if (e == cudaSuccess) e = launch_mix_spectra(h, h->Ystream, 1, h->Ymix_stream);
    if (e == cudaSuccess) e = launch_inverse_stream(h, out_dev, h->Ymix_stream, h->mix_ola, h->n_mix);
    if (e != cudaSuccess) return cuda_status(e);
    h->tick += 1;
    return TVOLAP_OK;
}

int64_t tvolap_state_bytes(tvolap_t h)
{
    if (!h) return TVOLAP_ERR_STATE;
    return state_bytes(h);
}

int tvolap_get_state(tvolap_t h, void *buf, int64_t cap)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!buf || cap < state_bytes(h)) return TVOLAP_ERR_ARG;
    const StateHeader hd{STATE_MAGIC, STATE_VERSION, h->L, h->M, h->n_in, h->n_out, h->n_mix, 0,
                         h->tick};
    char *dst = static_cast<char *>(buf);
    cudaError_t e = cudaMemcpyAsync(dst, &hd, sizeof(hd), cudaMemcpyDefault, h->stream);
    StatePart p[7];
    int64_t off = align256(sizeof(StateHeader));
    for (int i = 0, n = state_parts(h, p); i < n && e == cudaSuccess; ++i) {
        if (p[i].bytes)
            e = cudaMemcpyAsync(dst + off, p[i].dev, (size_t)p[i].bytes, cudaMemcpyDefault, h->stream);
        off += align256(p[i].bytes);
    }
    // the header is read from this stack frame: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

int tvolap_set_state(tvolap_t h, const void *buf, int64_t bytes)
{
    TVOLAP_TRACE();
    if (!h) return TVOLAP_ERR_STATE;
    if (!buf || bytes < state_bytes(h)) return TVOLAP_ERR_ARG;
    StateHeader hd;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&hd, buf, sizeof(hd), cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_status(e);
    if (hd.magic != STATE_MAGIC || hd.version != STATE_VERSION || hd.L != h->L || hd.M != h->M ||
        hd.n_in != h->n_in || hd.n_out != h->n_out || hd.n_mix != h->n_mix || hd.tick < 0)
        return TVOLAP_ERR_ARG;
    const char *src = static_cast<const char *>(buf);
    StatePart p[7];
    int64_t off = align256(sizeof(StateHeader));
    for (int i = 0, n = state_parts(h, p); i < n && e == cudaSuccess; ++i) {
        if (p[i].bytes)
            e = cudaMemcpyAsync(p[i].dev, src + off, (size_t)p[i].bytes, cudaMemcpyDefault, h->stream);
        off += align256(p[i].bytes);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->tick = hd.tick;
    return TVOLAP_OK;
}

int tvolap_set_option(tvolap_t h, int option, int value)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (option == TVOLAP_OPT_MAC_STAGING) {
        if (value < 0 || value > 5) return TVOLAP_ERR_ARG;
        h->mac_variant = value;
        return TVOLAP_OK;
    }
    if (option == TVOLAP_OPT_XFORM_THREADS) {
        if (value != 0 && value != 64 && value != 128 && value != 256) return TVOLAP_ERR_ARG;
        h->xform_threads = value;
        return TVOLAP_OK;
    }
    if (option == TVOLAP_OPT_STAGE_TIMING) {
        if (value != 0 && value != 1) return TVOLAP_ERR_ARG;
        cudaError_t e = timing_collect(h);
        for (int i = 0; i < 4 && e == cudaSuccess && value; ++i)
            if (!h->tev[i]) e = cudaEventCreate(&h->tev[i]);
        if (e != cudaSuccess) return cuda_status(e);
        h->timing = value;
        h->stage_ms[0] = h->stage_ms[1] = h->stage_ms[2] = 0.0;
        h->timed_ticks = 0;
        return TVOLAP_OK;
    }
    return TVOLAP_ERR_ARG;
}

int tvolap_stage_times(tvolap_t h, double *stage_ms, int64_t *ticks)
{
    if (!h) return TVOLAP_ERR_STATE;
    if (!stage_ms) return TVOLAP_ERR_ARG;
    const cudaError_t e = timing_collect(h);
    if (e != cudaSuccess) return cuda_status(e);
    for (int i = 0; i < 3; ++i) stage_ms[i] = h->stage_ms[i];
    if (ticks) *ticks = h->timed_ticks;
    return TVOLAP_OK;
}

}  // extern "C"

// C ABI of batched sources (tvolap_batch_*): sources grouped by hop, one plan
// and one ragged call per group (tvolap_process_ragged). Each group runs on a
// stream of its own, forked from the batch's stream at the start of a run and
// joined back at its end, so the groups' kernels overlap on the GPU; the run
// is captured as one CUDA graph of parallel branches. Per-group choice of the
// multiply-accumulate staging and of the transforms' CTA size by timing the
// variants on the batch itself.
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tvolap.h"
#include "trace.h"

namespace {

struct BatchGroup {
    int L = 0, M = 0, staging = 0, xform_threads = 0;
    tvolap_t plan = nullptr;
    std::vector<int> src;                 // source indices, in row order
    std::vector<int> slot_base;           // first filter slot of each row
    int64_t max_n = 0, max_out = 0, nb = 0;
    float *x = nullptr, *y = nullptr;     // [rows][max_n], [rows][max_out]
    int32_t *sched = nullptr;             // [rows][nb]
    int64_t *n_dev = nullptr, *ol_dev = nullptr;
    int32_t *parts_dev = nullptr;
    cudaStream_t st = nullptr;            // the group's stream (its plan's)
    cudaEvent_t done = nullptr;           // the group's work of a run has finished
};

int64_t blocks_of(int64_t out_len, int L) { return out_len <= 0 ? 0 : (out_len - 1) / L + 2; }

// Schedule of one source into its group's slots: local index i of the source's
// n_filters becomes base + i; anything else becomes -1, which the
// multiply-accumulate replaces by the all-zero filter and records.
__global__ void k_batch_sched(const int32_t *__restrict__ local, int64_t n, int n_filters, int base,
                              int32_t *__restrict__ global)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = local[i];
        global[i] = (v >= 0 && v < n_filters) ? base + v : -1;
    }
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return TVOLAP_OK;
    if (e == cudaErrorMemoryAllocation) return TVOLAP_ERR_OOM;
    return TVOLAP_ERR_CUDA;
}

}  // namespace

struct tvolap_batch {
    std::vector<tvolap_batch_source> src;
    std::vector<int> group_of, row_of;
    std::vector<BatchGroup> groups;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t fork = nullptr;           // the batch stream's work before a run
};

namespace {

void release(tvolap_batch *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (BatchGroup &g : b->groups) {
        tvolap_destroy(g.plan);
        if (g.done) cudaEventDestroy(g.done);
        if (g.st) cudaStreamDestroy(g.st);
        cudaFree(g.x);
        cudaFree(g.y);
        cudaFree(g.sched);
        cudaFree(g.n_dev);
        cudaFree(g.ol_dev);
        cudaFree(g.parts_dev);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// The groups' streams (all, or group `only`) wait for the work enqueued on
// the batch's stream so far.
cudaError_t fork_groups(tvolap_batch *b, BatchGroup *only = nullptr)
{
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (BatchGroup &g : b->groups)
        if (e == cudaSuccess && (!only || only == &g)) e = cudaStreamWaitEvent(g.st, b->fork, 0);
    return e;
}

// The batch's stream waits for the work enqueued on the groups' streams.
cudaError_t join_groups(tvolap_batch *b, BatchGroup *only = nullptr)
{
    cudaError_t e = cudaSuccess;
    for (BatchGroup &g : b->groups) {
        if (only && only != &g) continue;
        const cudaError_t r = cudaEventRecord(g.done, g.st);
        const cudaError_t w = r == cudaSuccess ? cudaStreamWaitEvent(b->stream, g.done, 0) : r;
        if (e == cudaSuccess) e = w;
    }
    return e;
}

int ragged(BatchGroup &g)
{
    return tvolap_process_ragged(g.plan, g.x, g.max_n, g.n_dev, g.ol_dev, g.parts_dev, g.max_out,
                                 g.sched, nullptr, nullptr, g.nb, g.y, g.max_out);
}

// One run: every group on its own stream, between a fork and a join.
int run_direct(tvolap_batch *b)
{
    cudaError_t ce = fork_groups(b);
    int e = ce == cudaSuccess ? TVOLAP_OK : cuda_status(ce);
    for (BatchGroup &g : b->groups)
        if (e == TVOLAP_OK && g.max_out > 0) e = ragged(g);
    ce = join_groups(b);                   // also after an error: a capture needs every branch joined
    return e != TVOLAP_OK ? e : cuda_status(ce);
}

}  // namespace

extern "C" {

int tvolap_batch_create(tvolap_batch_t *out, const tvolap_batch_source *src, int n_src,
                        void *stream)
{
    if (!out) return TVOLAP_ERR_ARG;
    *out = nullptr;
    if (n_src < 1 || !src) return TVOLAP_ERR_ARG;
    for (int i = 0; i < n_src; ++i) {
        const tvolap_batch_source &s = src[i];
        if (!pow2(s.L) || s.L < 16 || s.L > 1024 || s.M < 1 || s.n_filters < 1 || s.N < 0 ||
            s.out_len < 0 || blocks_of(s.out_len, s.L) > 0x3fffffff)
            return TVOLAP_ERR_ARG;
    }
    tvolap_batch *b = new (std::nothrow) tvolap_batch;
    if (!b) return TVOLAP_ERR_OOM;
    auto fail = [&](int code) {
        release(b);
        return code;
    };
    b->src.assign(src, src + n_src);
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(TVOLAP_ERR_CUDA);
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        b->own_stream = true;
    }
    std::map<int, std::vector<int>> by_hop;
    for (int i = 0; i < n_src; ++i) by_hop[src[i].L].push_back(i);
    b->group_of.assign(n_src, 0);
    b->row_of.assign(n_src, 0);
    b->groups.resize(by_hop.size());
    int gi = 0;
    for (auto &kv : by_hop) {
        BatchGroup &g = b->groups[gi];
        g.L = kv.first;
        g.src = kv.second;
        const int n = (int)g.src.size();
        int n_slots = 0;
        std::vector<int64_t> nh(n), olh(n);
        std::vector<int32_t> ph(n);
        for (int r = 0; r < n; ++r) {
            const tvolap_batch_source &s = src[g.src[r]];
            b->group_of[g.src[r]] = gi;
            b->row_of[g.src[r]] = r;
            g.slot_base.push_back(n_slots);
            n_slots += s.n_filters;
            g.M = std::max(g.M, s.M);
            g.max_n = std::max(g.max_n, s.N);
            g.max_out = std::max(g.max_out, s.out_len);
            nh[r] = s.N;
            olh[r] = s.out_len;
            ph[r] = s.M;
        }
        g.nb = blocks_of(g.max_out, g.L);
        if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        int e = tvolap_create(&g.plan, g.L, g.M, 0, n, n, nullptr, n_slots, g.st);
        if (e != TVOLAP_OK) return fail(e);
        const size_t xs = (size_t)n * std::max<int64_t>(g.max_n, 1) * sizeof(float);
        const size_t ys = (size_t)n * std::max<int64_t>(g.max_out, 1) * sizeof(float);
        const size_t ss = (size_t)n * std::max<int64_t>(g.nb, 1) * sizeof(int32_t);
        if (cudaMalloc(&g.x, xs) != cudaSuccess || cudaMalloc(&g.y, ys) != cudaSuccess ||
            cudaMalloc(&g.sched, ss) != cudaSuccess ||
            cudaMalloc(&g.n_dev, n * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&g.ol_dev, n * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&g.parts_dev, n * sizeof(int32_t)) != cudaSuccess)
            return fail(TVOLAP_ERR_OOM);
        if (cudaMemsetAsync(g.x, 0, xs, b->stream) != cudaSuccess ||
            cudaMemsetAsync(g.y, 0, ys, b->stream) != cudaSuccess ||
            cudaMemsetAsync(g.sched, 0, ss, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(g.n_dev, nh.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess ||
            cudaMemcpyAsync(g.ol_dev, olh.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess ||
            cudaMemcpyAsync(g.parts_dev, ph.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        // the host arrays above are copied before they go out of scope; the
        // plan's tables are made on the group's stream
        if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
            cudaStreamSynchronize(g.st) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        ++gi;
    }
    *out = b;
    return TVOLAP_OK;
}

int tvolap_batch_destroy(tvolap_batch_t b)
{
    if (!b) return TVOLAP_OK;
    cudaStreamSynchronize(b->stream);
    for (BatchGroup &g : b->groups) cudaStreamSynchronize(g.st);
    release(b);
    return TVOLAP_OK;
}

int tvolap_batch_source_view(tvolap_batch_t b, int i, float **x, int32_t **sched, float **y,
                             int *slot_base, int64_t *n_blocks)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (i < 0 || i >= (int)b->src.size()) return TVOLAP_ERR_ARG;
    const BatchGroup &g = b->groups[b->group_of[i]];
    const int r = b->row_of[i];
    if (x) *x = g.x + (int64_t)r * std::max<int64_t>(g.max_n, 1);
    if (sched) *sched = g.sched + (int64_t)r * std::max<int64_t>(g.nb, 1);
    if (y) *y = g.y + (int64_t)r * std::max<int64_t>(g.max_out, 1);
    if (slot_base) *slot_base = g.slot_base[r];
    if (n_blocks) *n_blocks = blocks_of(b->src[i].out_len, b->src[i].L);
    return TVOLAP_OK;
}

int tvolap_batch_set_source(tvolap_batch_t b, int i, const float *x_dev, const int32_t *sched_dev)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (i < 0 || i >= (int)b->src.size()) return TVOLAP_ERR_ARG;
    const tvolap_batch_source &s = b->src[i];
    const int64_t nb = blocks_of(s.out_len, s.L);
    if ((s.N > 0 && !x_dev) || (nb > 0 && !sched_dev)) return TVOLAP_ERR_ARG;
    const BatchGroup &g = b->groups[b->group_of[i]];
    const int r = b->row_of[i];
    if (s.N > 0) {
        cudaError_t e = cudaMemcpyAsync(g.x + (int64_t)r * std::max<int64_t>(g.max_n, 1), x_dev,
                                        s.N * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (nb > 0) {
        const int grid = (int)std::min<int64_t>((nb + 255) / 256, 1024);
        k_batch_sched<<<grid, 256, 0, b->stream>>>(sched_dev, nb, s.n_filters, g.slot_base[r],
                                                  g.sched + (int64_t)r * std::max<int64_t>(g.nb, 1));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    return TVOLAP_OK;
}

int tvolap_batch_get_output(tvolap_batch_t b, int i, float *y_dev)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (i < 0 || i >= (int)b->src.size()) return TVOLAP_ERR_ARG;
    const tvolap_batch_source &s = b->src[i];
    if (s.out_len == 0) return TVOLAP_OK;
    if (!y_dev) return TVOLAP_ERR_ARG;
    const BatchGroup &g = b->groups[b->group_of[i]];
    const int r = b->row_of[i];
    return cuda_status(cudaMemcpyAsync(y_dev, g.y + (int64_t)r * std::max<int64_t>(g.max_out, 1),
                                       s.out_len * sizeof(float), cudaMemcpyDeviceToDevice,
                                       b->stream));
}

int tvolap_batch_load_filters(tvolap_batch_t b, int i, const float *ir_dev, int ir_len,
                              int64_t ir_stride)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (i < 0 || i >= (int)b->src.size()) return TVOLAP_ERR_ARG;
    const tvolap_batch_source &s = b->src[i];
    if (ir_len > 2 * (int64_t)s.L * s.M) return TVOLAP_ERR_ARG;
    BatchGroup &g = b->groups[b->group_of[i]];
    // on the group's stream, ordered after and before the batch stream's work
    cudaError_t ce = fork_groups(b, &g);
    if (ce != cudaSuccess) return cuda_status(ce);
    const int e = tvolap_load_bank(g.plan, g.slot_base[b->row_of[i]], s.n_filters, ir_dev, ir_len,
                                   ir_stride);
    ce = join_groups(b, &g);
    return e != TVOLAP_OK ? e : cuda_status(ce);
}

int tvolap_batch_run(tvolap_batch_t b)
{
    TVOLAP_TRACE();
    if (!b) return TVOLAP_ERR_STATE;
    if (b->graph) return cuda_status(cudaGraphLaunch(b->graph, b->stream));
    return run_direct(b);
}

int tvolap_batch_capture(tvolap_batch_t b)
{
    TVOLAP_TRACE();
    if (!b) return TVOLAP_ERR_STATE;
    int e = run_direct(b);                 // sizes every workspace before the capture
    if (e != TVOLAP_OK) return e;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TVOLAP_ERR_CUDA;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_status(ce);
    e = run_direct(b);
    ce = cudaStreamEndCapture(b->stream, &graph);
    if (e != TVOLAP_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e != TVOLAP_OK ? e : cuda_status(ce);
    }
    ce = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    return cuda_status(ce);
}

int tvolap_batch_autotune(tvolap_batch_t b, int reps, int *chosen)
{
    TVOLAP_TRACE();
    if (!b) return TVOLAP_ERR_STATE;
    if (reps < 1) return TVOLAP_ERR_ARG;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return TVOLAP_ERR_CUDA;
    }
    int status = TVOLAP_OK;
    for (size_t gi = 0; gi < b->groups.size() && status == TVOLAP_OK; ++gi) {
        BatchGroup &g = b->groups[gi];
        float best = -1.f;
        int best_opt = 0;
        if (fork_groups(b, &g) != cudaSuccess) status = TVOLAP_ERR_CUDA;
        for (int opt = 0; opt <= 5 && status == TVOLAP_OK; ++opt) {
            status = tvolap_set_option(g.plan, TVOLAP_OPT_MAC_STAGING, opt);
            if (status != TVOLAP_OK || g.max_out == 0) break;
            status = ragged(g);                                    // warm: workspaces, caches
            if (status != TVOLAP_OK) break;
            cudaEventRecord(e0, g.st);
            for (int r = 0; r < reps && status == TVOLAP_OK; ++r) status = ragged(g);
            cudaEventRecord(e1, g.st);
            if (cudaEventSynchronize(e1) != cudaSuccess) status = TVOLAP_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0.f || ms < best) {
                best = ms;
                best_opt = opt;
            }
        }
        if (status == TVOLAP_OK) {
            status = tvolap_set_option(g.plan, TVOLAP_OPT_MAC_STAGING, best_opt);
            g.staging = best_opt;
            if (chosen) chosen[gi] = best_opt;
        }
        // then the transforms' CTA size (transforms per CTA), with that staging
        float best_t = -1.f;
        int best_th = 0;
        const int ths[3] = {256, 128, 64};
        for (int k = 0; k < 3 && status == TVOLAP_OK && g.max_out > 0; ++k) {
            status = tvolap_set_option(g.plan, TVOLAP_OPT_XFORM_THREADS, ths[k]);
            if (status == TVOLAP_OK) status = ragged(g);
            if (status != TVOLAP_OK) break;
            cudaEventRecord(e0, g.st);
            for (int r = 0; r < reps && status == TVOLAP_OK; ++r) status = ragged(g);
            cudaEventRecord(e1, g.st);
            if (cudaEventSynchronize(e1) != cudaSuccess) status = TVOLAP_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_t < 0.f || ms < best_t) {
                best_t = ms;
                best_th = ths[k];
            }
        }
        if (status == TVOLAP_OK && best_th > 0) {
            status = tvolap_set_option(g.plan, TVOLAP_OPT_XFORM_THREADS, best_th);
            g.xform_threads = best_th;
        }
        if (join_groups(b, &g) != cudaSuccess && status == TVOLAP_OK) status = TVOLAP_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}

int tvolap_batch_set_staging(tvolap_batch_t b, int g, int staging)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (g < -1 || g >= (int)b->groups.size() || staging < 0 || staging > 5) return TVOLAP_ERR_ARG;
    for (int k = 0; k < (int)b->groups.size(); ++k) {
        if (g != -1 && k != g) continue;
        const int e = tvolap_set_option(b->groups[k].plan, TVOLAP_OPT_MAC_STAGING, staging);
        if (e != TVOLAP_OK) return e;
        b->groups[k].staging = staging;
    }
    if (b->graph) {                        // the graph holds the old kernels
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return TVOLAP_OK;
}

int tvolap_batch_groups(tvolap_batch_t b, int *n_groups)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (!n_groups) return TVOLAP_ERR_ARG;
    *n_groups = (int)b->groups.size();
    return TVOLAP_OK;
}

int tvolap_batch_group_info(tvolap_batch_t b, int g, int *L, int *n_sources, int *staging)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (g < 0 || g >= (int)b->groups.size()) return TVOLAP_ERR_ARG;
    if (L) *L = b->groups[g].L;
    if (n_sources) *n_sources = (int)b->groups[g].src.size();
    if (staging) *staging = b->groups[g].staging;
    return TVOLAP_OK;
}

int tvolap_batch_group_tiling(tvolap_batch_t b, int g, int *mac_staging, int *xform_threads)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (g < 0 || g >= (int)b->groups.size()) return TVOLAP_ERR_ARG;
    if (mac_staging) *mac_staging = b->groups[g].staging;
    if (xform_threads) *xform_threads = b->groups[g].xform_threads;
    return TVOLAP_OK;
}

int tvolap_batch_check(tvolap_batch_t b)
{
    if (!b) return TVOLAP_ERR_STATE;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TVOLAP_ERR_CUDA;
    int worst = TVOLAP_OK;
    for (BatchGroup &g : b->groups) {
        const int e = tvolap_check(g.plan);
        if (e != TVOLAP_OK && worst == TVOLAP_OK) worst = e;
    }
    return worst;
}

}  // extern "C"

// C ABI of the streaming server (tvolap_server_*): the host object that owns
// the arena, the staging, the per-class tables and the tick graphs, and turns
// the scheduler's due list into one tick of work.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tvolap.h"
#include "internal.h"
#include "server_dev.h"
#include "server_sched.h"
#include "trace.h"

using namespace tvolap;

struct tvolap_server {
    Scheduler sch;
    int dev = 0, n_sm = 0;
    cudaStream_t stream = nullptr, adm = nullptr;
    bool own_stream = false;
    char *arena = nullptr;
    int n_cls = 0;
    SrvClassTables cls[SRV_MAX_CLASSES] = {};
    float *tables = nullptr;                 // all classes' tables, one allocation
    SrvDesc *desc_d = nullptr, *desc_h = nullptr;
    float2 *part = nullptr;                  // partial sums [part_slots][max_out][64]
    int64_t part_slots = 0;
    int Pmax = 0, gmax = 1, max_chunks = SRV_MAX_CHUNKS;
    char *ctl_h[2] = {nullptr, nullptr};     // mapped pinned: head, due[capacity], items
    size_t ctl_bytes = 0;
    unsigned *counter = nullptr;             // device
    int *skip = nullptr;                     // device
    SrvStatus *status = nullptr;             // mapped pinned
    float *in_h = nullptr, *out_h = nullptr;
    int32_t *sel_h = nullptr;
    SrvLaunch launch[2] = {};
    SrvStatus *status_d = nullptr;
    const SrvHead *head_d[2] = {nullptr, nullptr};
    cudaEvent_t tick_ev[2] = {nullptr, nullptr};
    cudaEvent_t tev[2][4] = {};
    bool inflight[2] = {false, false}, timed[2] = {false, false};
    std::vector<int> due_of[2];
    uint64_t seq_of[2] = {0, 0};
    int64_t inc_of[2][3] = {};               // stream blocks, samples, MAC bytes of the tick
    std::vector<cudaEvent_t> adm_ev;
    std::vector<int> pending;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int use_graph = 1, timing = 0;
    int64_t wait_us = 0;
    uint64_t seq = 0;                        // ticks enqueued
    tvolap_server_stats stats = {};
    std::vector<int> ids;                    // scratch
};

namespace {

int lg2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return TVOLAP_OK;
    if (e == cudaErrorMemoryAllocation) return TVOLAP_ERR_OOM;
    return TVOLAP_ERR_CUDA;
}

void release(tvolap_server *s)
{
    if (!s) return;
    for (int b = 0; b < 2; ++b) {
        if (s->gexec[b]) cudaGraphExecDestroy(s->gexec[b]);
        if (s->tick_ev[b]) cudaEventDestroy(s->tick_ev[b]);
        for (int i = 0; i < 4; ++i)
            if (s->tev[b][i]) cudaEventDestroy(s->tev[b][i]);
        if (s->ctl_h[b]) cudaFreeHost(s->ctl_h[b]);
    }
    for (cudaEvent_t e : s->adm_ev)
        if (e) cudaEventDestroy(e);
    if (s->adm) cudaStreamDestroy(s->adm);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    cudaFree(s->arena);
    cudaFree(s->tables);
    cudaFree(s->desc_d);
    cudaFree(s->part);
    cudaFree(s->counter);
    cudaFree(s->skip);
    cudaFreeHost(s->desc_h);
    cudaFreeHost(s->status);
    cudaFreeHost(s->in_h);
    cudaFreeHost(s->out_h);
    cudaFreeHost(s->sel_h);
    delete s;
}

template <class T>
T *dev_view(T *host)
{
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, (void *)host, 0) != cudaSuccess) return nullptr;
    return static_cast<T *>(d);
}

// Layout of one control buffer: head, due[capacity], items[capacity * gmax].
size_t due_offset() { return sizeof(SrvHead); }
size_t item_offset(const tvolap_server *s)
{
    return align_up(sizeof(SrvHead) + (size_t)s->sch.capacity * sizeof(SrvDue), 64);
}

// Finish the tick held in control buffer b (its event has completed).
void complete(tvolap_server *s, int b)
{
    if (!s->inflight[b]) return;
    if (s->timed[b]) {
        for (int i = 0; i < 3; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s->tev[b][i], s->tev[b][i + 1]) == cudaSuccess)
                s->stats.stage_ms[i] += ms;
        }
        s->stats.timed_ticks += 1;
        s->timed[b] = false;
    }
    s->inflight[b] = false;
}

// Wait for every enqueued tick and the admission stream; roll back a tick
// whose input wait ran out.
int finish(tvolap_server *s)
{
    cudaError_t e1 = cudaStreamSynchronize(s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->adm);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return TVOLAP_ERR_CUDA;
    // complete in tick order
    int first = (s->inflight[0] && s->inflight[1]) ? (s->seq_of[0] < s->seq_of[1] ? 0 : 1) : -1;
    if (first >= 0) {
        complete(s, first);
        complete(s, 1 - first);
    } else {
        complete(s, 0);
        complete(s, 1);
    }
    volatile SrvStatus *st = s->status;
    if (st->err & SRV_ERR_TIMEOUT) {
        const uint64_t failed = st->failed_seq;
        // with the wait option one tick is in flight: it is the last one
        for (int b = 0; b < 2; ++b) {
            if (s->seq_of[b] == failed && failed == s->seq) {
                s->sch.rollback(s->due_of[b]);
                s->seq -= 1;
                s->stats.ticks -= 1;
                s->stats.stream_blocks -= s->inc_of[b][0];
                s->stats.channel_samples -= s->inc_of[b][1];
                s->stats.mac_bytes -= s->inc_of[b][2];
                s->seq_of[b] = 0;
            }
        }
        st->err = st->err & ~SRV_ERR_TIMEOUT;
        return TVOLAP_ERR_TIMEOUT;
    }
    return TVOLAP_OK;
}

void invalidate_graphs(tvolap_server *s)
{
    for (int b = 0; b < 2; ++b) {
        if (s->gexec[b]) cudaGraphExecDestroy(s->gexec[b]);
        s->gexec[b] = nullptr;
    }
}

// Enqueue the work of one tick reading control buffer b.
cudaError_t enqueue(tvolap_server *s, int b, bool with_events)
{
    const SrvLaunch &a = s->launch[b];
    cudaError_t e;
    if (s->wait_us > 0) {
        const long long ns = s->wait_us * 1000LL;
        e = srv_launch_gate(s->head_d[b], s->status_d, s->skip, ns, 4 * (s->wait_us + 1000),
                            s->stream);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(s->counter, 0, sizeof(unsigned), s->stream);
    if (e != cudaSuccess) return e;
    if (with_events) cudaEventRecord(s->tev[b][0], s->stream);
    e = srv_launch_forward(a, s->stream);
    if (e != cudaSuccess) return e;
    if (with_events) cudaEventRecord(s->tev[b][1], s->stream);
    e = srv_launch_mac(a, s->stream);
    if (e != cudaSuccess) return e;
    if (with_events) cudaEventRecord(s->tev[b][2], s->stream);
    e = srv_launch_inverse(a, s->stream);
    if (e != cudaSuccess) return e;
    if (with_events) cudaEventRecord(s->tev[b][3], s->stream);
    return cudaSuccess;
}

cudaError_t capture(tvolap_server *s, int b)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e_enq = enqueue(s, b, false);
    e = cudaStreamEndCapture(s->stream, &g);
    if (e_enq != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e_enq;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&s->gexec[b], g, 0);
    cudaGraphDestroy(g);
    return e;
}

void activate_ready(tvolap_server *s)
{
    for (size_t i = 0; i < s->pending.size();) {
        const int id = s->pending[i];
        if (cudaEventQuery(s->adm_ev[id]) == cudaSuccess) {
            s->sch.activate(id);
            cudaMemcpyAsync(s->desc_d + id, s->desc_h + id, sizeof(SrvDesc), cudaMemcpyHostToDevice,
                            s->stream);
            s->pending[i] = s->pending.back();
            s->pending.pop_back();
        } else {
            ++i;
        }
    }
}

int class_of(const tvolap_server *s, int L)
{
    for (int c = 0; c < s->n_cls; ++c)
        if (s->cls[c].L == L) return c;
    return -1;
}

}  // namespace

extern "C" {

int tvolap_server_create(tvolap_server_t *out, int base_hop, int max_hop, int capacity,
                         int max_out, int64_t arena_bytes, void *stream)
{
    if (!out) return TVOLAP_ERR_ARG;
    *out = nullptr;
    tvolap_server *s = new (std::nothrow) tvolap_server;
    if (!s) return TVOLAP_ERR_OOM;
    int e = s->sch.init(base_hop, max_hop, capacity, max_out, arena_bytes);
    if (e != TVOLAP_OK) {
        delete s;
        return e;
    }
    auto fail = [&](int code) {
        release(s);
        return code;
    };
    cudaError_t ce = cudaGetDevice(&s->dev);
    if (ce != cudaSuccess) return fail(TVOLAP_ERR_CUDA);
    ce = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->dev);
    if (ce != cudaSuccess) return fail(TVOLAP_ERR_CUDA);
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        s->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&s->adm, cudaStreamNonBlocking) != cudaSuccess)
        return fail(TVOLAP_ERR_CUDA);
    // hop classes and their tables
    s->n_cls = 0;
    for (int L = base_hop; L <= max_hop; L *= 2) {
        SrvClassTables &t = s->cls[s->n_cls++];
        t.L = L;
        t.lgP = lg2(2 * L);
    }
    size_t tab_floats = 0;
    for (int c = 0; c < s->n_cls; ++c) tab_floats += (size_t)2 * s->cls[c].L * 8;   // 8P floats
    if (cudaMalloc(&s->tables, tab_floats * sizeof(float)) != cudaSuccess) return fail(TVOLAP_ERR_OOM);
    float *p = s->tables;
    for (int c = 0; c < s->n_cls; ++c) {
        SrvClassTables &t = s->cls[c];
        const int P = 2 * t.L;
        float2 *tw = reinterpret_cast<float2 *>(p);          // 2P twiddles (stage-major)
        float2 *rot = tw + 2 * P;
        float2 *post = rot + P;
        float *win = reinterpret_cast<float *>(post + P / 2);
        p = win + P;
        t.tw = tw;
        t.rot = rot;
        t.post = post;
        t.win = win;
        if (launch_tables_raw(tw, rot, post, win, t.L, s->stream) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        t.fwd_grid = srv_grid_transforms(t.lgP, capacity, s->n_sm);
        t.inv_grid = srv_grid_transforms(t.lgP, (int64_t)capacity * max_out, s->n_sm);
    }
    s->Pmax = 2 * max_hop;
    s->gmax = std::max(1, s->Pmax / SRV_GROUP_BINS);
    // partial-sum slots: every due stream at most gmax groups x max_chunks chunks
    // (fewer chunks when that would take more than 1 GiB)
    const int64_t slot_bytes = (int64_t)max_out * SRV_GROUP_BINS * sizeof(float2);
    while (s->max_chunks > 1 &&
           (int64_t)capacity * s->gmax * s->max_chunks * slot_bytes > ((int64_t)1 << 30))
        s->max_chunks /= 2;
    s->part_slots = (int64_t)capacity * s->gmax * s->max_chunks;
    const int64_t arena = s->sch.arena_bytes;
    if (arena > 0 && cudaMalloc(&s->arena, arena) != cudaSuccess) return fail(TVOLAP_ERR_OOM);
    if (cudaMalloc(&s->desc_d, (size_t)capacity * sizeof(SrvDesc)) != cudaSuccess ||
        cudaMalloc(&s->part, (size_t)(s->part_slots * slot_bytes)) != cudaSuccess ||
        cudaMalloc(&s->counter, 64) != cudaSuccess || cudaMalloc(&s->skip, 64) != cudaSuccess)
        return fail(TVOLAP_ERR_OOM);
    if (cudaMemsetAsync(s->desc_d, 0, (size_t)capacity * sizeof(SrvDesc), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->skip, 0, 64, s->stream) != cudaSuccess)
        return fail(TVOLAP_ERR_CUDA);
    const unsigned mapped = cudaHostAllocMapped | cudaHostAllocPortable;
    s->ctl_bytes = item_offset(s) + (size_t)s->part_slots * sizeof(SrvItem);
    const size_t io = (size_t)2 * capacity * max_hop * sizeof(float);    // two staging sets
    if (cudaHostAlloc((void **)&s->desc_h, (size_t)capacity * sizeof(SrvDesc), cudaHostAllocPortable) != cudaSuccess ||
        cudaHostAlloc((void **)&s->status, sizeof(SrvStatus), mapped) != cudaSuccess ||
        cudaHostAlloc((void **)&s->in_h, io, mapped) != cudaSuccess ||
        cudaHostAlloc((void **)&s->out_h, io * max_out, mapped) != cudaSuccess ||
        cudaHostAlloc((void **)&s->sel_h, (size_t)capacity * sizeof(int32_t), cudaHostAllocPortable) != cudaSuccess ||
        cudaHostAlloc((void **)&s->ctl_h[0], s->ctl_bytes, mapped) != cudaSuccess ||
        cudaHostAlloc((void **)&s->ctl_h[1], s->ctl_bytes, mapped) != cudaSuccess)
        return fail(TVOLAP_ERR_OOM);
    std::memset(s->desc_h, 0, (size_t)capacity * sizeof(SrvDesc));
    std::memset(s->status, 0, sizeof(SrvStatus));
    std::memset(s->in_h, 0, io);
    std::memset(s->out_h, 0, io * max_out);
    std::memset(s->sel_h, 0, (size_t)capacity * sizeof(int32_t));
    std::memset(s->ctl_h[0], 0, s->ctl_bytes);
    std::memset(s->ctl_h[1], 0, s->ctl_bytes);
    s->status_d = dev_view(s->status);
    const float *in_d = dev_view(s->in_h);
    float *out_d = dev_view(s->out_h);
    if (!s->status_d || !in_d || !out_d) return fail(TVOLAP_ERR_CUDA);
    int occ = 0;
    if (srv_mac_occupancy(&occ) != cudaSuccess || occ < 1) return fail(TVOLAP_ERR_CUDA);
    for (int b = 0; b < 2; ++b) {
        char *cd = dev_view(s->ctl_h[b]);
        if (!cd) return fail(TVOLAP_ERR_CUDA);
        SrvLaunch &a = s->launch[b];
        a.head = reinterpret_cast<const SrvHead *>(cd);
        a.due = reinterpret_cast<const SrvDue *>(cd + due_offset());
        a.items = reinterpret_cast<const SrvItem *>(cd + item_offset(s));
        a.desc = s->desc_d;
        a.part = s->part;
        a.max_out = max_out;
        a.capacity = capacity;
        a.in = in_d + (size_t)b * capacity * max_hop;
        a.out = out_d + (size_t)b * capacity * max_out * max_hop;
        a.io_stride = max_hop;
        a.counter = s->counter;
        a.skip = s->skip;
        a.mac_grid = s->n_sm * occ;
        a.n_cls = s->n_cls;
        a.fwd_start[0] = a.inv_start[0] = 0;
        for (int c = 0; c < s->n_cls; ++c) {
            a.cls[c] = s->cls[c];
            a.fwd_start[c + 1] = a.fwd_start[c] + s->cls[c].fwd_grid;
            a.inv_start[c + 1] = a.inv_start[c] + s->cls[c].inv_grid;
        }
        s->head_d[b] = a.head;
        if (cudaEventCreateWithFlags(&s->tick_ev[b], cudaEventDisableTiming) != cudaSuccess)
            return fail(TVOLAP_ERR_CUDA);
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&s->tev[b][i]) != cudaSuccess) return fail(TVOLAP_ERR_CUDA);
    }
    s->adm_ev.assign(capacity, nullptr);
    s->stats.arena_bytes = arena;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(TVOLAP_ERR_CUDA);
    *out = s;
    return TVOLAP_OK;
}

int tvolap_server_destroy(tvolap_server_t s)
{
    if (!s) return TVOLAP_OK;
    cudaStreamSynchronize(s->stream);
    cudaStreamSynchronize(s->adm);
    release(s);
    return TVOLAP_OK;
}

int tvolap_server_footprint(tvolap_server_t s, int L, int M, int n_out, int n_filters,
                            int64_t *bytes)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!bytes) return TVOLAP_ERR_ARG;
    const int e = s->sch.check_stream_args(L, M, n_out, n_filters);
    if (e != TVOLAP_OK) return e;
    *bytes = stream_layout(L, M, n_out, n_filters).total;
    return TVOLAP_OK;
}

}  // extern "C"

namespace {

// A slot and an arena piece for a new stream (admission or restore): its
// descriptor, its admission event, and the admission stream ordered after
// the last enqueued tick (the piece may have belonged to a retired stream
// those ticks still read).
int take_slot(tvolap_server *s, int L, int M, int n_out, int n_filters, int c, int *id)
{
    int i = -1;
    int e = s->sch.admit(L, M, n_out, n_filters, &i);
    if (e != TVOLAP_OK) return e;
    const SchedStream &ss = s->sch.st[i];
    char *base = s->arena + ss.offset;
    SrvDesc d{};
    d.bank = reinterpret_cast<float2 *>(base + ss.lay.bank);
    d.ring = reinterpret_cast<float2 *>(base + ss.lay.ring);
    d.ola = reinterpret_cast<float *>(base + ss.lay.ola);
    d.hist = reinterpret_cast<float *>(base + ss.lay.hist);
    d.L = L;
    d.M = M;
    d.n_out = n_out;
    d.n_filters = n_filters;
    d.lgP = s->cls[c].lgP;
    s->desc_h[i] = d;
    if ((!s->adm_ev[i] && cudaEventCreateWithFlags(&s->adm_ev[i], cudaEventDisableTiming) != cudaSuccess) ||
        (s->seq > 0 && cudaStreamWaitEvent(s->adm, s->tick_ev[(s->seq - 1) & 1], 0) != cudaSuccess)) {
        s->sch.retire(i);
        return TVOLAP_ERR_CUDA;
    }
    *id = i;
    return TVOLAP_OK;
}

// Arguments of an admission (or a submitted request): responses, hop class.
int check_admit_args(tvolap_server *s, int L, int M, int n_out, int n_filters, const float *ir_dev,
                     int ir_len, int64_t ir_stride, int *cls)
{
    if (ir_len < 0 || (int64_t)ir_len > 2 * (int64_t)L * M || (ir_len > 0 && !ir_dev) ||
        ir_stride < ir_len)
        return TVOLAP_ERR_ARG;
    if (ir_dev && (reinterpret_cast<uintptr_t>(ir_dev) & 3u)) return TVOLAP_ERR_ARG;
    const int e = s->sch.check_stream_args(L, M, n_out, n_filters);
    if (e != TVOLAP_OK) return e;
    *cls = class_of(s, L);
    return *cls < 0 ? TVOLAP_ERR_ARG : TVOLAP_OK;
}

// Admission proper: a slot and piece, the state zeroed and the bank
// transformed (Eqs. 2, 4, 6) on the admission stream; live once that is done.
int admit_now(tvolap_server *s, int L, int M, int n_out, int n_filters, const float *ir_dev,
              int ir_len, int64_t ir_stride, int c, int *id)
{
    int i = -1;
    int e = take_slot(s, L, M, n_out, n_filters, c, &i);
    if (e != TVOLAP_OK) return e;
    const SchedStream &ss = s->sch.st[i];
    char *base = s->arena + ss.offset;
    const SrvDesc &d = s->desc_h[i];
    auto undo = [&](int code) {
        s->sch.retire(i);
        return code;
    };
    if (cudaMemsetAsync(base + ss.lay.ring, 0, ss.lay.total - ss.lay.ring, s->adm) != cudaSuccess)
        return undo(TVOLAP_ERR_CUDA);
    const int64_t count = (int64_t)n_filters * n_out;
    cudaError_t ce;
    if (ir_len > 0)
        ce = launch_bank_raw(s->cls[c].lgP, L, M, count, ir_dev, ir_len, ir_stride, s->cls[c].rot,
                             s->cls[c].post, s->cls[c].tw, d.bank, s->adm);
    else
        ce = cudaMemsetAsync(d.bank, 0, ss.lay.ring, s->adm);
    if (ce != cudaSuccess) return undo(TVOLAP_ERR_CUDA);
    if (cudaEventRecord(s->adm_ev[i], s->adm) != cudaSuccess) return undo(TVOLAP_ERR_CUDA);
    s->pending.push_back(i);
    *id = i;
    return TVOLAP_OK;
}

// Admit queued requests, oldest first, while slots and arena pieces allow.
int pump_queue(tvolap_server *s)
{
    return s->sch.pump([&](const AdmitRequest &r, int *id) {
        return admit_now(s, r.L, r.M, r.n_out, r.n_filters, static_cast<const float *>(r.payload),
                         (int)r.arg0, r.arg1, class_of(s, r.L), id);
    }, nullptr);
}

// Stream snapshot: this header, then the stream's arena piece (transformed
// filters, delay line, pending sums, input history) at byte 256.
struct StreamSnapHeader {
    uint32_t magic, version;
    int32_t L, M, n_out, n_filters, sel, pad;
    int64_t blocks, piece;
};
constexpr uint32_t SNAP_MAGIC = 0x53535654u;   // "TVSS"
constexpr int64_t SNAP_DATA = 256;
static_assert(sizeof(StreamSnapHeader) <= SNAP_DATA, "snapshot header");

}  // namespace

extern "C" {

int tvolap_server_admit(tvolap_server_t s, int L, int M, int n_out, int n_filters,
                        const float *ir_dev, int ir_len, int64_t ir_stride, int *id)
{
    TVOLAP_TRACE();
    if (!s) return TVOLAP_ERR_STATE;
    if (!id) return TVOLAP_ERR_ARG;
    int c = -1;
    const int e = check_admit_args(s, L, M, n_out, n_filters, ir_dev, ir_len, ir_stride, &c);
    if (e != TVOLAP_OK) return e;
    return admit_now(s, L, M, n_out, n_filters, ir_dev, ir_len, ir_stride, c, id);
}

int tvolap_server_submit(tvolap_server_t s, int L, int M, int n_out, int n_filters,
                         const float *ir_dev, int ir_len, int64_t ir_stride, int64_t *ticket)
{
    TVOLAP_TRACE();
    if (!s) return TVOLAP_ERR_STATE;
    if (!ticket) return TVOLAP_ERR_ARG;
    int c = -1;
    int e = check_admit_args(s, L, M, n_out, n_filters, ir_dev, ir_len, ir_stride, &c);
    if (e != TVOLAP_OK) return e;
    e = s->sch.submit(L, M, n_out, n_filters, ir_dev, ir_len, ir_stride, ticket);
    if (e != TVOLAP_OK) return e;
    return pump_queue(s);
}

int tvolap_server_admitted(tvolap_server_t s, int64_t *tickets, int32_t *ids, int64_t *wait_ticks,
                           int cap, int *count)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!count || cap < 0 || (cap > 0 && (!tickets || !ids))) return TVOLAP_ERR_ARG;
    *count = s->sch.take_admitted(tickets, ids, wait_ticks, cap);
    return TVOLAP_OK;
}

int tvolap_server_cancel(tvolap_server_t s, int64_t ticket)
{
    if (!s) return TVOLAP_ERR_STATE;
    return s->sch.cancel(ticket);
}

int tvolap_server_queue(tvolap_server_t s, int *waiting, int64_t *oldest_wait_ticks,
                        int64_t *admitted_total, int64_t *max_wait_ticks)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (waiting) *waiting = s->sch.queue_len();
    if (oldest_wait_ticks) *oldest_wait_ticks = s->sch.oldest_wait();
    if (admitted_total) *admitted_total = s->sch.admitted_from_queue;
    if (max_wait_ticks) *max_wait_ticks = s->sch.max_wait;
    return TVOLAP_OK;
}

int tvolap_server_stream_bytes(tvolap_server_t s, int id, int64_t *bytes)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!bytes || !s->sch.valid_id(id)) return TVOLAP_ERR_ARG;
    *bytes = SNAP_DATA + s->sch.st[id].lay.total;
    return TVOLAP_OK;
}

int tvolap_server_snapshot(tvolap_server_t s, int id, void *buf, int64_t cap)
{
    TVOLAP_TRACE();
    if (!s) return TVOLAP_ERR_STATE;
    if (!buf || !s->sch.valid_id(id)) return TVOLAP_ERR_ARG;
    const SchedStream &ss = s->sch.st[id];
    if (cap < SNAP_DATA + ss.lay.total) return TVOLAP_ERR_ARG;
    const int e = finish(s);                // ticks in flight and admissions complete
    if (e != TVOLAP_OK) return e;
    const StreamSnapHeader hd{SNAP_MAGIC, 1, ss.L, ss.M, ss.n_out, ss.n_filters, s->sel_h[id], 0,
                              ss.blocks, ss.lay.total};
    char *dst = static_cast<char *>(buf);
    if (cudaMemcpy(dst, &hd, sizeof(hd), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(dst + SNAP_DATA, s->arena + ss.offset, (size_t)ss.lay.total, cudaMemcpyDefault) !=
            cudaSuccess)
        return TVOLAP_ERR_CUDA;
    return TVOLAP_OK;
}

int tvolap_server_restore(tvolap_server_t s, const void *buf, int64_t bytes, int *id)
{
    TVOLAP_TRACE();
    if (!s) return TVOLAP_ERR_STATE;
    if (!buf || !id || bytes < SNAP_DATA) return TVOLAP_ERR_ARG;
    StreamSnapHeader hd;
    if (cudaMemcpy(&hd, buf, sizeof(hd), cudaMemcpyDefault) != cudaSuccess) return TVOLAP_ERR_CUDA;
    if (hd.magic != SNAP_MAGIC || hd.version != 1 || hd.blocks < 0) return TVOLAP_ERR_ARG;
    int e = s->sch.check_stream_args(hd.L, hd.M, hd.n_out, hd.n_filters);
    if (e != TVOLAP_OK) return e;
    const int c = class_of(s, hd.L);
    if (c < 0 || hd.sel < 0 || hd.sel >= hd.n_filters) return TVOLAP_ERR_ARG;
    if (stream_layout(hd.L, hd.M, hd.n_out, hd.n_filters).total != hd.piece ||
        bytes < SNAP_DATA + hd.piece)
        return TVOLAP_ERR_ARG;
    int i = -1;
    e = take_slot(s, hd.L, hd.M, hd.n_out, hd.n_filters, c, &i);
    if (e != TVOLAP_OK) return e;
    const SchedStream &ss = s->sch.st[i];
    if (cudaMemcpyAsync(s->arena + ss.offset, static_cast<const char *>(buf) + SNAP_DATA,
                        (size_t)hd.piece, cudaMemcpyDefault, s->adm) != cudaSuccess ||
        cudaEventRecord(s->adm_ev[i], s->adm) != cudaSuccess) {
        s->sch.retire(i);
        return TVOLAP_ERR_CUDA;
    }
    s->sch.st[i].blocks = hd.blocks;
    s->sel_h[i] = hd.sel;
    s->pending.push_back(i);
    *id = i;
    return TVOLAP_OK;
}

int tvolap_server_retire(tvolap_server_t s, int id)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!s->sch.valid_id(id)) return TVOLAP_ERR_ARG;
    s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), id), s->pending.end());
    return s->sch.retire(id);
}

int tvolap_server_state(tvolap_server_t s, int id, int *state, int64_t *blocks, int *phase)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (id < 0 || id >= s->sch.capacity || !state) return TVOLAP_ERR_ARG;
    const SchedStream &ss = s->sch.st[id];
    *state = ss.state;
    if (blocks) *blocks = ss.blocks;
    if (phase) *phase = ss.phase;
    return TVOLAP_OK;
}

int tvolap_server_staging(tvolap_server_t s, int buffer, float **in, int64_t *in_stride,
                          int32_t **sel, float **out, int64_t *out_stride)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (buffer != 0 && buffer != 1) return TVOLAP_ERR_ARG;
    const size_t cap = s->sch.capacity, hop = s->sch.max_hop;
    if (in) *in = s->in_h + buffer * cap * hop;
    if (in_stride) *in_stride = (int64_t)hop;
    if (sel) *sel = s->sel_h;
    if (out) *out = s->out_h + buffer * cap * s->sch.max_out * hop;
    if (out_stride) *out_stride = (int64_t)hop;
    return TVOLAP_OK;
}

int tvolap_server_due(tvolap_server_t s, int32_t *ids_host, int cap, int *count, int *buffer)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!count || cap < 0 || (cap > 0 && !ids_host)) return TVOLAP_ERR_ARG;
    const int b = (int)(s->seq & 1);
    if (s->inflight[b]) {                      // the tick that last used this staging set
        if (cudaEventSynchronize(s->tick_ev[b]) != cudaSuccess) return TVOLAP_ERR_CUDA;
        complete(s, b);
    }
    activate_ready(s);
    const int pe = pump_queue(s);            // requests waiting for a slot and memory
    if (pe != TVOLAP_OK) return pe;
    s->sch.due(s->ids);
    for (int i = 0; i < (int)s->ids.size() && i < cap; ++i) ids_host[i] = s->ids[i];
    *count = (int)s->ids.size();
    if (buffer) *buffer = b;
    return TVOLAP_OK;
}

int tvolap_server_tick(tvolap_server_t s)
{
    TVOLAP_TRACE();
    if (!s) return TVOLAP_ERR_STATE;
    if (s->wait_us > 0) {                      // one tick in flight
        const int e = finish(s);
        if (e != TVOLAP_OK) return e;
    }
    const int b = (int)(s->seq & 1);
    if (s->inflight[b]) {                      // the tick two back used this buffer
        if (cudaEventSynchronize(s->tick_ev[b]) != cudaSuccess) return TVOLAP_ERR_CUDA;
        complete(s, b);
    }
    std::vector<int> &ids = s->ids;
    s->sch.due(ids);
    for (int id : ids) {
        const int f = s->sel_h[id];
        if (f < 0 || f >= s->sch.st[id].n_filters) return TVOLAP_ERR_ARG;
    }
    // due entries grouped by hop class; each stream's partitions cut into at
    // most max_chunks chunks of >= SRV_MIN_CHUNK partitions
    char *ctl = s->ctl_h[b];
    SrvHead *head = reinterpret_cast<SrvHead *>(ctl);
    SrvDue *due = reinterpret_cast<SrvDue *>(ctl + due_offset());
    SrvItem *items = reinterpret_cast<SrvItem *>(ctl + item_offset(s));
    std::memset(head, 0, sizeof(SrvHead));
    int n = 0;
    int64_t mac_bytes = 0, samples = 0, slots = 0;
    for (int c = 0; c < s->n_cls; ++c) {
        head->cls_off[c] = n;
        for (int id : ids) {
            const SchedStream &ss = s->sch.st[id];
            if (ss.L != s->cls[c].L) continue;
            const int64_t t = ss.blocks;
            const int R = 2 * ss.M;
            SrvDue d;
            d.slot = id;
            d.pos = (int)(t % R);
            d.sel = s->sel_h[id];
            d.m_end = (int)std::min<int64_t>(ss.M, t / 2 + 1);
            d.chunk_len = std::max(SRV_MIN_CHUNK, (d.m_end + s->max_chunks - 1) / s->max_chunks);
            d.n_chunks = (d.m_end + d.chunk_len - 1) / d.chunk_len;
            d.part_base = (int)slots;
            d.pad = 0;
            slots += (int64_t)std::max(1, 2 * ss.L / SRV_GROUP_BINS) * d.n_chunks;
            due[n++] = d;
            const int64_t spec = 2 * (int64_t)ss.L * 8;
            mac_bytes += (int64_t)(1 + ss.n_out) * d.m_end * spec + (int64_t)ss.n_out * spec;
            samples += (int64_t)ss.n_out * ss.L;
        }
        head->cls_n[c] = n - head->cls_off[c];
    }
    // chunks are at most max_chunks per group and at least SRV_MIN_CHUNK long,
    // so items are of similar size: they go in due order, chunk by chunk
    int n_items = 0;
    for (int i = 0; i < n; ++i) {
        const int groups = std::max(1, 2 * s->sch.st[due[i].slot].L / SRV_GROUP_BINS);
        for (int g = 0; g < groups; ++g)
            for (int ch = 0; ch < due[i].n_chunks; ++ch) items[n_items++] = SrvItem{i, g, ch, 0};
    }
    head->seq = s->seq + 1;
    head->n_items = (uint32_t)n_items;
    head->n_due = (uint32_t)n;
    std::atomic_thread_fence(std::memory_order_release);
    cudaError_t ce;
    const bool timed = s->timing != 0;
    if (s->use_graph && !timed) {
        if (!s->gexec[b]) {
            ce = capture(s, b);
            if (ce != cudaSuccess) return cuda_status(ce);
        }
        ce = cudaGraphLaunch(s->gexec[b], s->stream);
    } else {
        ce = enqueue(s, b, timed);
    }
    if (ce != cudaSuccess) return cuda_status(ce);
    if (cudaEventRecord(s->tick_ev[b], s->stream) != cudaSuccess) return TVOLAP_ERR_CUDA;
    s->inflight[b] = true;
    s->timed[b] = timed;
    s->due_of[b] = ids;
    s->seq_of[b] = s->seq + 1;
    s->inc_of[b][0] = n;
    s->inc_of[b][1] = samples;
    s->inc_of[b][2] = mac_bytes;
    s->sch.advance(ids);
    s->seq += 1;
    s->stats.ticks += 1;
    s->stats.stream_blocks += n;
    s->stats.channel_samples += samples;
    s->stats.mac_bytes += mac_bytes;
    s->stats.last_due = n;
    s->stats.last_items = n_items;
    return TVOLAP_OK;
}

int tvolap_server_wait(tvolap_server_t s)
{
    TVOLAP_TRACE();
    if (!s) return TVOLAP_ERR_STATE;
    return finish(s);
}

int tvolap_server_post(tvolap_server_t s, uint64_t seq)
{
    if (!s) return TVOLAP_ERR_STATE;
    std::atomic_thread_fence(std::memory_order_release);
    volatile uint64_t *p = &s->status->posted;
    if (seq > *p) *p = seq;
    return TVOLAP_OK;
}

int tvolap_server_set_option(tvolap_server_t s, int option, int64_t value)
{
    if (!s) return TVOLAP_ERR_STATE;
    switch (option) {
    case TVOLAP_SERVER_OPT_GRAPH:
        if (value != 0 && value != 1) return TVOLAP_ERR_ARG;
        s->use_graph = (int)value;
        return TVOLAP_OK;
    case TVOLAP_SERVER_OPT_WAIT_US: {
        if (value < 0 || value > 2000000) return TVOLAP_ERR_ARG;
        const int e = finish(s);
        if (e != TVOLAP_OK && e != TVOLAP_ERR_TIMEOUT) return e;
        s->wait_us = value;
        invalidate_graphs(s);
        if (cudaMemsetAsync(s->skip, 0, sizeof(int), s->stream) != cudaSuccess) return TVOLAP_ERR_CUDA;
        return TVOLAP_OK;
    }
    case TVOLAP_SERVER_OPT_TIMING:
        if (value != 0 && value != 1) return TVOLAP_ERR_ARG;
        s->timing = (int)value;
        return TVOLAP_OK;
    case TVOLAP_SERVER_OPT_FAIL_ADMITS:
        if (value < 0) return TVOLAP_ERR_ARG;
        s->sch.fail_admits = value;
        return TVOLAP_OK;
    default:
        return TVOLAP_ERR_ARG;
    }
}

int tvolap_server_stats_get(tvolap_server_t s, tvolap_server_stats *st)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!st) return TVOLAP_ERR_ARG;
    int live = 0, pend = 0;
    for (const SchedStream &x : s->sch.st) {
        if (x.state == 2) ++live;
        if (x.state == 1) ++pend;
    }
    s->stats.live = live;
    s->stats.pending = pend;
    s->stats.arena_used = s->sch.used;
    *st = s->stats;
    return TVOLAP_OK;
}

}  // extern "C"

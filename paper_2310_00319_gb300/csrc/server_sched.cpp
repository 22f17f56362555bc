// Host-side scheduler of the streaming server and its stand-alone C ABI
// (tvolap_sched_*), which runs without a GPU.
#include "server_sched.h"

#include <iterator>
#include <new>

#include "../../include/tvolap.h"

namespace tvolap {

namespace {
bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
}  // namespace

StreamLayout stream_layout(int L, int M, int n_out, int n_filters)
{
    const int64_t P = 2 * (int64_t)L, spec = P * 8;
    StreamLayout s{};
    s.bank = 0;
    s.ring = align_up((int64_t)n_filters * n_out * M * spec, SRV_ALIGN);
    s.ola = s.ring + align_up(2 * (int64_t)M * spec, SRV_ALIGN);
    s.hist = s.ola + align_up((int64_t)n_out * 3 * L * 4, SRV_ALIGN);
    s.total = s.hist + align_up((int64_t)L * 4, SRV_ALIGN);
    return s;
}

int64_t stream_block_bytes(int L, int M, int n_out)
{
    const int64_t spec = 2 * (int64_t)L * 8;
    return (int64_t)(1 + n_out) * M * spec + (int64_t)n_out * spec;
}

int Scheduler::init(int base, int mx, int cap, int mo, int64_t arena)
{
    if (!pow2(base) || base < 16 || base > 1024 || !pow2(mx) || mx < base || mx > 1024 ||
        mx > 8 * base || cap < 1 || cap > 65536 || mo < 1 || mo > 2 || arena < 0)
        return TVOLAP_ERR_ARG;
    base_hop = base;
    max_hop = mx;
    capacity = cap;
    max_out = mo;
    n_phase = mx / base;
    arena_bytes = arena / SRV_ALIGN * SRV_ALIGN;
    used = 0;
    tick = 0;
    st.assign(cap, SchedStream{});
    phase_load.assign(n_phase, 0);
    free_ids_.clear();
    for (int i = 0; i < cap; ++i) free_ids_.insert(i);
    free_.clear();
    if (arena_bytes > 0) free_[0] = arena_bytes;
    queue_.clear();
    admitted_.clear();
    next_ticket_ = 1;
    submitted = admitted_from_queue = cancelled = max_wait = sum_wait = 0;
    return TVOLAP_OK;
}

int Scheduler::check_stream_args(int L, int M, int n_out, int n_filters) const
{
    if (!pow2(L) || L < base_hop || L > max_hop || M < 1 || n_out < 1 || n_out > max_out ||
        n_filters < 1)
        return TVOLAP_ERR_ARG;
    // keep every index of the device kernels inside 32 bits where they use int
    if ((int64_t)n_filters * n_out * M > (int64_t)1 << 30 || M > (1 << 24)) return TVOLAP_ERR_ARG;
    return TVOLAP_OK;
}

int64_t Scheduler::take(int64_t bytes)
{
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second >= bytes) {
            const int64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest > 0) free_[off + bytes] = rest;
            return off;
        }
    }
    return -1;
}

void Scheduler::give(int64_t off, int64_t bytes)
{
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + bytes == nx->first) {      // merge with the next piece
        bytes += nx->second;
        nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {                                // merge with the previous piece
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            pv->second += bytes;
            return;
        }
    }
    free_[off] = bytes;
}

int64_t Scheduler::largest_free() const
{
    int64_t m = 0;
    for (const auto &kv : free_)
        if (kv.second > m) m = kv.second;
    return m;
}

int Scheduler::admit(int L, int M, int n_out, int n_filters, int *id)
{
    int e = check_stream_args(L, M, n_out, n_filters);
    if (e != TVOLAP_OK) return e;
    if (fail_admits > 0) {
        --fail_admits;
        return TVOLAP_ERR_CAPACITY;
    }
    if (free_ids_.empty()) return TVOLAP_ERR_CAPACITY;
    const StreamLayout lay = stream_layout(L, M, n_out, n_filters);
    const int64_t off = take(lay.total);
    if (off < 0) return TVOLAP_ERR_CAPACITY;
    const int i = *free_ids_.begin();
    free_ids_.erase(free_ids_.begin());
    SchedStream &s = st[i];
    s = SchedStream{};
    s.state = 1;
    s.L = L;
    s.ratio = L / base_hop;
    s.M = M;
    s.n_out = n_out;
    s.n_filters = n_filters;
    s.offset = off;
    s.lay = lay;
    s.load = stream_block_bytes(L, M, n_out);
    // phase: the base ticks the stream would be due in are the least loaded
    // ones: smallest heaviest tick among them, then smallest sum, then lowest
    int best = 0;
    int64_t best_max = -1, best_sum = -1;
    for (int ph = 0; ph < s.ratio; ++ph) {
        int64_t mx = 0, sum = 0;
        for (int q = ph; q < n_phase; q += s.ratio) {
            mx = phase_load[q] > mx ? phase_load[q] : mx;
            sum += phase_load[q];
        }
        if (best_max < 0 || mx < best_max || (mx == best_max && sum < best_sum)) {
            best_max = mx;
            best_sum = sum;
            best = ph;
        }
    }
    s.phase = best;
    for (int q = 0; q < n_phase; ++q)
        if (q % s.ratio == best) phase_load[q] += s.load;
    used += lay.total;
    *id = i;
    return TVOLAP_OK;
}

int Scheduler::submit(int L, int M, int n_out, int n_filters, const void *payload, int64_t arg0,
                      int64_t arg1, int64_t *ticket)
{
    const int e = check_stream_args(L, M, n_out, n_filters);
    if (e != TVOLAP_OK) return e;
    if (stream_layout(L, M, n_out, n_filters).total > arena_bytes) return TVOLAP_ERR_CAPACITY;
    AdmitRequest r;
    r.ticket = next_ticket_++;
    r.submit_tick = tick;
    r.L = L;
    r.M = M;
    r.n_out = n_out;
    r.n_filters = n_filters;
    r.payload = payload;
    r.arg0 = arg0;
    r.arg1 = arg1;
    queue_.push_back(r);
    ++submitted;
    *ticket = r.ticket;
    return TVOLAP_OK;
}

int Scheduler::cancel(int64_t ticket)
{
    for (auto it = queue_.begin(); it != queue_.end(); ++it) {
        if (it->ticket == ticket) {
            queue_.erase(it);
            ++cancelled;
            return TVOLAP_OK;
        }
    }
    return TVOLAP_ERR_ARG;
}

int Scheduler::take_admitted(int64_t *tickets, int32_t *ids, int64_t *waits, int cap)
{
    int n = 0;
    while (n < cap && !admitted_.empty()) {
        const AdmitRecord &r = admitted_.front();
        if (tickets) tickets[n] = r.ticket;
        if (ids) ids[n] = r.id;
        if (waits) waits[n] = r.wait_ticks;
        admitted_.pop_front();
        ++n;
    }
    return n;
}

int Scheduler::activate(int id)
{
    if (!valid_id(id) || st[id].state != 1) return TVOLAP_ERR_ARG;
    st[id].state = 2;
    return TVOLAP_OK;
}

int Scheduler::retire(int id)
{
    if (!valid_id(id)) return TVOLAP_ERR_ARG;
    SchedStream &s = st[id];
    for (int q = 0; q < n_phase; ++q)
        if (q % s.ratio == s.phase) phase_load[q] -= s.load;
    give(s.offset, s.lay.total);
    used -= s.lay.total;
    s = SchedStream{};
    free_ids_.insert(id);
    return TVOLAP_OK;
}

void Scheduler::due(std::vector<int> &ids) const
{
    ids.clear();
    for (int i = 0; i < capacity; ++i) {
        const SchedStream &s = st[i];
        if (s.state == 2 && (tick % s.ratio) == s.phase) ids.push_back(i);
    }
}

void Scheduler::advance(const std::vector<int> &ids)
{
    for (int i : ids) st[i].blocks += 1;
    tick += 1;
}

void Scheduler::rollback(const std::vector<int> &ids)
{
    for (int i : ids)
        if (st[i].blocks > 0) st[i].blocks -= 1;
    if (tick > 0) tick -= 1;
}

}  // namespace tvolap

// ----------------------------------------------------------------------------- C ABI
struct tvolap_sched {
    tvolap::Scheduler s;
};

extern "C" {

int tvolap_sched_create(tvolap_sched_t *out, int base_hop, int max_hop, int capacity, int max_out,
                        int64_t arena_bytes)
{
    if (!out) return TVOLAP_ERR_ARG;
    *out = nullptr;
    tvolap_sched *h = new (std::nothrow) tvolap_sched;
    if (!h) return TVOLAP_ERR_OOM;
    const int e = h->s.init(base_hop, max_hop, capacity, max_out, arena_bytes);
    if (e != TVOLAP_OK) {
        delete h;
        return e;
    }
    *out = h;
    return TVOLAP_OK;
}

int tvolap_sched_destroy(tvolap_sched_t s)
{
    delete s;
    return TVOLAP_OK;
}

int tvolap_sched_footprint(int L, int M, int n_out, int n_filters, int64_t *bytes)
{
    if (!bytes || !tvolap::pow2(L) || L < 16 || L > 1024 || M < 1 || n_out < 1 || n_out > 2 ||
        n_filters < 1)
        return TVOLAP_ERR_ARG;
    *bytes = tvolap::stream_layout(L, M, n_out, n_filters).total;
    return TVOLAP_OK;
}

int tvolap_sched_admit(tvolap_sched_t s, int L, int M, int n_out, int n_filters, int *id,
                       int64_t *offset, int *phase)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!id) return TVOLAP_ERR_ARG;
    const int e = s->s.admit(L, M, n_out, n_filters, id);
    if (e != TVOLAP_OK) return e;
    if (offset) *offset = s->s.st[*id].offset;
    if (phase) *phase = s->s.st[*id].phase;
    return TVOLAP_OK;
}

int tvolap_sched_fail_admits(tvolap_sched_t s, int64_t n)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (n < 0) return TVOLAP_ERR_ARG;
    s->s.fail_admits = n;
    return TVOLAP_OK;
}

int tvolap_sched_submit(tvolap_sched_t s, int L, int M, int n_out, int n_filters, int64_t *ticket)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!ticket) return TVOLAP_ERR_ARG;
    int e = s->s.submit(L, M, n_out, n_filters, nullptr, 0, 0, ticket);
    if (e != TVOLAP_OK) return e;
    return s->s.pump([&](const tvolap::AdmitRequest &r, int *id) {
        return s->s.admit(r.L, r.M, r.n_out, r.n_filters, id);
    }, nullptr);
}

int tvolap_sched_pump(tvolap_sched_t s, int *admitted)
{
    if (!s) return TVOLAP_ERR_STATE;
    return s->s.pump([&](const tvolap::AdmitRequest &r, int *id) {
        return s->s.admit(r.L, r.M, r.n_out, r.n_filters, id);
    }, admitted);
}

int tvolap_sched_cancel(tvolap_sched_t s, int64_t ticket)
{
    if (!s) return TVOLAP_ERR_STATE;
    return s->s.cancel(ticket);
}

int tvolap_sched_admitted(tvolap_sched_t s, int64_t *tickets, int32_t *ids, int64_t *wait_ticks,
                          int cap, int *count)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!count || cap < 0) return TVOLAP_ERR_ARG;
    *count = s->s.take_admitted(tickets, ids, wait_ticks, cap);
    return TVOLAP_OK;
}

int tvolap_sched_queue(tvolap_sched_t s, int *waiting, int64_t *oldest_wait_ticks)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (waiting) *waiting = s->s.queue_len();
    if (oldest_wait_ticks) *oldest_wait_ticks = s->s.oldest_wait();
    return TVOLAP_OK;
}

int tvolap_sched_activate(tvolap_sched_t s, int id)
{
    if (!s) return TVOLAP_ERR_STATE;
    return s->s.activate(id);
}

int tvolap_sched_retire(tvolap_sched_t s, int id)
{
    if (!s) return TVOLAP_ERR_STATE;
    return s->s.retire(id);
}

int tvolap_sched_due(tvolap_sched_t s, int32_t *ids_host, int cap, int *count)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!count || cap < 0 || (cap > 0 && !ids_host)) return TVOLAP_ERR_ARG;
    std::vector<int> ids;
    s->s.due(ids);
    for (int i = 0; i < (int)ids.size() && i < cap; ++i) ids_host[i] = ids[i];
    *count = (int)ids.size();
    return TVOLAP_OK;
}

int tvolap_sched_advance(tvolap_sched_t s)
{
    if (!s) return TVOLAP_ERR_STATE;
    std::vector<int> ids;
    s->s.due(ids);
    s->s.advance(ids);
    return TVOLAP_OK;
}

int tvolap_sched_phase_loads(tvolap_sched_t s, int64_t *loads, int cap, int *n)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (!n || cap < 0 || (cap > 0 && !loads)) return TVOLAP_ERR_ARG;
    for (int q = 0; q < s->s.n_phase && q < cap; ++q) loads[q] = s->s.phase_load[q];
    *n = s->s.n_phase;
    return TVOLAP_OK;
}

int tvolap_sched_arena(tvolap_sched_t s, int64_t *used, int64_t *largest_free)
{
    if (!s) return TVOLAP_ERR_STATE;
    if (used) *used = s->s.used;
    if (largest_free) *largest_free = s->s.largest_free();
    return TVOLAP_OK;
}

}  // extern "C"

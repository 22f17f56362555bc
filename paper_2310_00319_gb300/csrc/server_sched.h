// Host-side scheduler of the streaming server: stream slots, placement in the
// device arena (first fit, 256-byte aligned, freed pieces merged with their
// neighbours), the phase of each stream and the due lists per base tick.
// Plain C++; it touches no device memory.
#pragma once

#include <cstdint>
#include <deque>
#include <map>
#include <set>
#include <vector>

#include "../../include/tvolap.h"

namespace tvolap {

constexpr int64_t SRV_ALIGN = 256;

inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Offsets of the four parts of a stream's arena piece, and its total size.
struct StreamLayout {
    int64_t bank, ring, ola, hist, total;
};

// bank: n_filters * n_out * M spectra; delay line: 2M spectra; overlap state:
// 3L floats per output; input history: L floats (spectra of P = 2L float2).
StreamLayout stream_layout(int L, int M, int n_out, int n_filters);

// Bytes of Eq. 7 per block of a stream at full depth: M delay-line spectra and
// n_out * M filter spectra read, n_out spectra written.
int64_t stream_block_bytes(int L, int M, int n_out);

struct SchedStream {
    int state = 0;          // 0 free, 1 admitted (pending), 2 live
    int L = 0, ratio = 1, phase = 0, M = 0, n_out = 0, n_filters = 0;
    int64_t offset = 0;     // arena piece
    StreamLayout lay{};
    int64_t blocks = 0;     // blocks given so far
    int64_t load = 0;       // stream_block_bytes
};

// A request waiting for admission: a stream's shape, the base tick at which
// it was submitted and an opaque payload that the server keeps for it (its
// response buffer); the scheduler never dereferences the payload.
struct AdmitRequest {
    int64_t ticket = 0, submit_tick = 0;
    int L = 0, M = 0, n_out = 0, n_filters = 0;
    const void *payload = nullptr;
    int64_t arg0 = 0, arg1 = 0;
};

// A request that left the queue: its ticket, the stream id it received and
// the base ticks it waited.
struct AdmitRecord {
    int64_t ticket = 0;
    int id = -1;
    int64_t wait_ticks = 0;
};

class Scheduler {
public:
    // Returns 0 or a negative tvolap_status.
    int init(int base_hop, int max_hop, int capacity, int max_out, int64_t arena_bytes);
    int check_stream_args(int L, int M, int n_out, int n_filters) const;
    int admit(int L, int M, int n_out, int n_filters, int *id);
    int activate(int id);
    int retire(int id);
    // Live streams due at the current tick, increasing id.
    void due(std::vector<int> &ids) const;
    // The given streams took one block each; the tick advances.
    void advance(const std::vector<int> &ids);
    // Undo advance(ids) of the last tick.
    void rollback(const std::vector<int> &ids);

    // Admission queue (continuous batching): requests wait in arrival order
    // and are admitted, oldest first, as slots and arena pieces free up.
    // submit() refuses only a request that could never fit (its footprint is
    // larger than the whole arena) with TVOLAP_ERR_CAPACITY.
    int submit(int L, int M, int n_out, int n_filters, const void *payload, int64_t arg0,
               int64_t arg1, int64_t *ticket);
    // Admit from the head of the queue while admission succeeds; try_admit(req, &id)
    // returns a tvolap_status and, on success, the new stream's id. Stops at the
    // first TVOLAP_ERR_CAPACITY (strict arrival order: nothing overtakes the
    // head); any other error is returned with the head still queued.
    template <class F>
    int pump(F try_admit, int *n_admitted)
    {
        int n = 0;
        while (!queue_.empty()) {
            const AdmitRequest &r = queue_.front();
            int id = -1;
            const int e = try_admit(r, &id);
            if (e != TVOLAP_OK) {
                if (n_admitted) *n_admitted = n;
                return e == TVOLAP_ERR_CAPACITY ? TVOLAP_OK : e;   // no room yet: wait
            }
            admitted_.push_back(AdmitRecord{r.ticket, id, tick - r.submit_tick});
            wait_hist_add(tick - r.submit_tick);
            queue_.pop_front();
            ++n;
        }
        if (n_admitted) *n_admitted = n;
        return TVOLAP_OK;
    }
    int cancel(int64_t ticket);
    // Moves up to cap records of admissions from the queue (oldest first) out.
    int take_admitted(int64_t *tickets, int32_t *ids, int64_t *waits, int cap);
    int queue_len() const { return (int)queue_.size(); }
    int64_t oldest_wait() const { return queue_.empty() ? 0 : tick - queue_.front().submit_tick; }
    int64_t submitted = 0, admitted_from_queue = 0, cancelled = 0, max_wait = 0, sum_wait = 0;

    int64_t largest_free() const;
    bool valid_id(int id) const { return id >= 0 && id < capacity && st[id].state != 0; }

    int base_hop = 0, max_hop = 0, capacity = 0, max_out = 0, n_phase = 1;
    int64_t arena_bytes = 0, used = 0, tick = 0;
    // Fault injection on the host: the next fail_admits admissions with valid
    // arguments are refused with TVOLAP_ERR_CAPACITY as if no arena piece were
    // free, changing nothing else.
    int64_t fail_admits = 0;
    std::vector<SchedStream> st;
    std::vector<int64_t> phase_load;     // per base tick mod n_phase

private:
    void wait_hist_add(int64_t w)
    {
        ++admitted_from_queue;
        sum_wait += w;
        if (w > max_wait) max_wait = w;
    }
    int64_t take(int64_t bytes);         // arena offset or -1
    std::deque<AdmitRequest> queue_;
    std::deque<AdmitRecord> admitted_;
    int64_t next_ticket_ = 1;
    void give(int64_t off, int64_t bytes);
    std::set<int> free_ids_;
    std::map<int64_t, int64_t> free_;    // offset -> size
};

}  // namespace tvolap

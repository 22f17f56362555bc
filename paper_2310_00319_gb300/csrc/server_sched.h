// Host-side scheduler of the streaming server: stream slots, placement in the
// device arena (first fit, 256-byte aligned, freed pieces merged with their
// neighbours), the phase of each stream and the due lists per base tick.
// Plain C++; it touches no device memory.
#pragma once

#include <cstdint>
#include <map>
#include <set>
#include <vector>

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
    int64_t take(int64_t bytes);         // arena offset or -1
    void give(int64_t off, int64_t bytes);
    std::set<int> free_ids_;
    std::map<int64_t, int64_t> free_;    // offset -> size
};

}  // namespace tvolap

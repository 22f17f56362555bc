// Device-visible records of the streaming server, shared by its kernels and
// its host code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tvolap {

// Per stream slot, in device memory (written when the stream turns live).
struct SrvDesc {
    float2 *bank;       // [n_filters][n_out][M][P]
    float2 *ring;       // [2M][P] delay line, block t in row t mod 2M
    float *ola;         // [n_out][3L] pending overlap-add sums
    float *hist;        // [L] last L input samples
    int L, M, n_out, n_filters;
    int lgP, pad0, pad1, pad2;
};
static_assert(sizeof(SrvDesc) == 64, "SrvDesc layout");

constexpr int SRV_MAX_CLASSES = 4;      // hops base, 2 base, 4 base, 8 base

// Per tick, in mapped pinned host memory (read by the kernels in place).
struct SrvHead {
    uint64_t seq;                       // tick number, from 1
    uint32_t n_items, n_due;
    int32_t cls_off[SRV_MAX_CLASSES];   // due entries of hop class c: [off, off + n)
    int32_t cls_n[SRV_MAX_CLASSES];
    uint64_t pad[2];
};
static_assert(sizeof(SrvHead) == 64, "SrvHead layout");

struct SrvDue {
    int32_t slot;       // stream id
    int32_t pos;        // delay-line row of this block: t mod 2M
    int32_t sel;        // filter index of this block
    int32_t m_end;      // partitions with data: min(M, t/2 + 1)
    int32_t part_base;  // first partial-sum slot of this stream (see SrvItem)
    int32_t n_chunks;   // partition chunks per 64-bin group
    int32_t chunk_len;  // partitions per chunk (the last may be shorter)
    int32_t pad;
};

// One unit of multiply-accumulate work: 64 bins (group) of one due stream,
// partitions [chunk * chunk_len, min((chunk + 1) * chunk_len, m_end)). Its sums
// go to partial slot part_base + group * n_chunks + chunk; the inverse adds a
// group's chunks in chunk order.
struct SrvItem {
    int32_t due, group, chunk, pad;
};

constexpr int SRV_MAX_CHUNKS = 16;      // partition chunks per group at most
constexpr int SRV_MIN_CHUNK = 128;      // partitions per chunk at least

// Mapped pinned host words shared with the gate kernel.
struct SrvStatus {
    uint32_t err;              // bit 2: an input wait ran out
    uint32_t pad;
    uint64_t failed_seq;       // tick whose wait ran out
    uint64_t posted;           // highest tick whose staging is declared written
};

constexpr unsigned SRV_ERR_TIMEOUT = 2;
constexpr int SRV_GROUP_BINS = 64;      // bins per multiply-accumulate item

struct SrvClassTables {
    int L, lgP, fwd_grid, inv_grid;
    const float2 *tw, *rot, *post;
    const float *win;
};

// Launchers (kernels_server.cu). Pointers to SrvHead / SrvDue / SrvItem /
// SrvStatus / in / out are device views of mapped host memory.
struct SrvLaunch {
    const SrvHead *head;
    const SrvDue *due;
    const SrvItem *items;
    const SrvDesc *desc;
    float2 *part;               // partial sums [slots][max_out][64]
    int max_out, capacity;
    const float *in;            // [capacity][io_stride]
    float *out;                 // [capacity][max_out][io_stride]
    int64_t io_stride;
    unsigned *counter;          // device work counter of the multiply-accumulate
    int *skip;                  // device flag: 1 = this tick's input wait ran out
    int mac_grid;
    int n_cls;
    int fwd_start[SRV_MAX_CLASSES + 1];   // first CTA of each class in the fused launches
    int inv_start[SRV_MAX_CLASSES + 1];
    SrvClassTables cls[SRV_MAX_CLASSES];
};

cudaError_t srv_mac_occupancy(int *blocks_per_sm);
cudaError_t srv_launch_gate(const SrvHead *head, SrvStatus *status, int *skip, long long wait_ns,
                            long long max_iter, cudaStream_t st);
// one launch each for all hop classes (256 threads, SRV_FFT_SMEM bytes per CTA)
cudaError_t srv_launch_forward(const SrvLaunch &a, cudaStream_t st);
cudaError_t srv_launch_mac(const SrvLaunch &a, cudaStream_t st);
cudaError_t srv_launch_inverse(const SrvLaunch &a, cudaStream_t st);
int srv_grid_transforms(int lgP, int64_t transforms, int n_sm);

}  // namespace tvolap

// Kernels of the streaming server (sm_103a). One tick runs, on the server's
// stream:
//   k_srv_gate       (optional) bounded wait until the producer has declared
//                    this tick's staging written
//   k_srv_forward    Eqs. 1, 3, 5 for each due stream's new block, into its
//                    delay line (row t mod 2M); one launch for all hop classes
//   k_srv_mac        Eq. 7 for every due stream and output, with the filter
//                    selected for the block; persistent CTAs take items (64
//                    bins x a chunk of partitions) from a work counter and
//                    store partial sums
//   k_srv_inverse    Eq. 8 and the overlap-add of Eqs. 9-12 on the summed
//                    partials, output block written straight to the host
//                    staging; one launch for all hop classes
// The due list, the items and the tick header live in mapped pinned host
// memory and are read in place; per-stream descriptors, delay lines, banks and
// overlap state live in the device arena.
#include "fft_block.cuh"
#include "server_dev.h"

namespace tvolap {

namespace {

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Single thread: wait until status->posted >= head->seq, for at most wait_ns
// nanoseconds and max_iter polls. On time-out the tick is marked skipped and
// the failure recorded for the host.
__global__ void k_srv_gate(const SrvHead *head, SrvStatus *status, int *skip, long long wait_ns,
                           long long max_iter)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t seq = *reinterpret_cast<const volatile uint64_t *>(&head->seq);
    const volatile uint64_t *posted = &status->posted;
    const uint64_t t0 = global_ns();
    bool ok = false;
    for (long long it = 0; it < max_iter; ++it) {
        if (*posted >= seq) {
            ok = true;
            break;
        }
        if ((long long)(global_ns() - t0) > wait_ns) break;
        __nanosleep(1000);
    }
    if (!ok && *posted >= seq) ok = true;      // last look after the final sleep
    *skip = ok ? 0 : 1;
    if (!ok) {
        volatile SrvStatus *vs = status;
        vs->failed_seq = seq;
        __threadfence_system();
        vs->err = vs->err | SRV_ERR_TIMEOUT;
        __threadfence_system();
    }
}

// Forward transforms of the due streams of class c (this CTA is block b of nb
// of that class): each takes the L samples of history and the L new ones,
// writes its spectrum into delay-line row pos and keeps the new samples.
template <int LG>
__device__ __forceinline__ void srv_forward_body(const SrvLaunch &a, int c, int b, int nb,
                                                 float2 *sm)
{
    constexpr int P = 1 << LG, L = P / 2, T = Geo<P>::T, F = Geo<P>::F;
    const SrvClassTables &t = a.cls[c];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *A = sm + f * P, *B = sm + (F + f) * P;
    const int n = a.head->cls_n[c], off = a.head->cls_off[c];
    for (int base = b * F; base < n; base += nb * F) {             // uniform per CTA
        const int g = base + f;
        const bool active = g < n;
        const SrvDue d = a.due[off + (active ? g : 0)];
        const SrvDesc ds = a.desc[d.slot];
        const float *hc = ds.hist;
        const float *ic = a.in + (int64_t)d.slot * a.io_stride;
        auto src = [&](int s) {      // s even: s and s + 1 lie on the same side of L
            const float2 v = *reinterpret_cast<const float2 *>((s < L) ? (hc + s) : (ic + s - L));
            const float2 w = __ldg(reinterpret_cast<const float2 *>(t.win) + (s >> 1));
            return make_float2(v.x * w.x, v.y * w.y);
        };
        float2 *Xo = ds.ring + (int64_t)d.pos * P;
        forward_block<P>(A, B, j, active, src, t.rot, t.post, t.tw, [&](int k, float2 v) {
            if (active) Xo[k] = v;
        });
        // the history was read before the first barrier inside forward_block
        if (active)
            for (int i = j; i < L; i += T) ds.hist[i] = ic[i];
        __syncthreads();     // shared buffers are reused by the next round
    }
}

// The class of CTA blockIdx.x in a fused launch whose classes start at start[].
__device__ __forceinline__ int srv_class_of(const int *start, int n_cls, int &b, int &nb)
{
    int c = 0;
    while (c + 1 < n_cls && (int)blockIdx.x >= start[c + 1]) ++c;
    b = blockIdx.x - start[c];
    nb = start[c + 1] - start[c];
    return c;
}

// Every transform size runs 256 threads and 2 x 2048 float2 of shared memory
// (F transforms of P points), so one launch serves all classes.
__global__ void __launch_bounds__(256)
k_srv_forward(SrvLaunch a)
{
    if (*a.skip) return;
    extern __shared__ float2 sm[];
    int b, nb;
    const int c = srv_class_of(a.fwd_start, a.n_cls, b, nb);
    switch (a.cls[c].lgP) {                                       // uniform per CTA
    case 5: srv_forward_body<5>(a, c, b, nb, sm); break;
    case 6: srv_forward_body<6>(a, c, b, nb, sm); break;
    case 7: srv_forward_body<7>(a, c, b, nb, sm); break;
    case 8: srv_forward_body<8>(a, c, b, nb, sm); break;
    case 9: srv_forward_body<9>(a, c, b, nb, sm); break;
    case 10: srv_forward_body<10>(a, c, b, nb, sm); break;
    default: srv_forward_body<11>(a, c, b, nb, sm); break;
    }
}

constexpr int MAC_THREADS = 256, MAC_WARPS = MAC_THREADS / 32;

__device__ __forceinline__ void cfma4(float4 &acc, float4 h, float4 x)   // acc += h * x
{
    acc.x = fmaf(h.x, x.x, acc.x);
    acc.x = fmaf(-h.y, x.y, acc.x);
    acc.y = fmaf(h.x, x.y, acc.y);
    acc.y = fmaf(h.y, x.x, acc.y);
    acc.z = fmaf(h.z, x.z, acc.z);
    acc.z = fmaf(-h.w, x.w, acc.z);
    acc.w = fmaf(h.z, x.w, acc.w);
    acc.w = fmaf(h.w, x.z, acc.w);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b)
{
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Item = (due stream, group of 64 bins, chunk of partitions). Lane l holds
// bins k, k + 1 with k = 64 group + 2 l; warp w takes the chunk's partitions
// m = m0 + w, m0 + w + 8, ...; the eight partial sums are added in warp order
// and stored in the item's partial slot, so each output depends only on its own
// stream's data.
__global__ void __launch_bounds__(MAC_THREADS)
k_srv_mac(SrvLaunch a)
{
    __shared__ float4 red[2][MAC_WARPS][32];
    __shared__ int s_item;
    if (*a.skip) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned n_items = a.head->n_items;
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int it = s_item;
        if ((unsigned)it >= n_items) break;             // uniform
        const SrvItem item = a.items[it];
        const SrvDue d = a.due[item.due];
        const SrvDesc ds = a.desc[d.slot];
        const int P = 2 * ds.L, P4 = ds.L;              // float4 per spectrum
        const int k = item.group * SRV_GROUP_BINS + 2 * lane;
        const bool on = k < P;
        const int R = 2 * ds.M;
        const int m0 = item.chunk * d.chunk_len;
        const int m1 = m0 + d.chunk_len < d.m_end ? m0 + d.chunk_len : d.m_end;
        const float4 *X = reinterpret_cast<const float4 *>(ds.ring + (on ? k : 0));
        const int64_t MP4 = (int64_t)ds.M * P4;
        const float4 *H0 = reinterpret_cast<const float4 *>(
            ds.bank + ((int64_t)d.sel * ds.n_out) * ds.M * P + (on ? k : 0));
        const bool two = ds.n_out > 1;
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        if (on) {
            if (two) {
#pragma unroll 4
                for (int m = m0 + w; m < m1; m += MAC_WARPS) {
                    int row = d.pos - 2 * m;
                    if (row < 0) row += R;
                    const float4 x = __ldg(X + (int64_t)row * P4);
                    const float4 h0 = __ldg(H0 + (int64_t)m * P4);
                    const float4 h1 = __ldg(H0 + MP4 + (int64_t)m * P4);
                    cfma4(acc0, h0, x);
                    cfma4(acc1, h1, x);
                }
            } else {
#pragma unroll 4
                for (int m = m0 + w; m < m1; m += MAC_WARPS) {
                    int row = d.pos - 2 * m;
                    if (row < 0) row += R;
                    cfma4(acc0, __ldg(H0 + (int64_t)m * P4), __ldg(X + (int64_t)row * P4));
                }
            }
        }
        red[0][w][lane] = acc0;
        red[1][w][lane] = acc1;
        __syncthreads();
        if (w < 2 && on && w < ds.n_out) {
            float4 s = red[w][0][lane];
#pragma unroll
            for (int q = 1; q < MAC_WARPS; ++q) s = add4(s, red[w][q][lane]);
            const int64_t slot = d.part_base + item.group * d.n_chunks + item.chunk;
            reinterpret_cast<float4 *>(a.part + (slot * a.max_out + w) * SRV_GROUP_BINS)[lane] = s;
        }
        __syncthreads();     // red and s_item are reused by the next item
    }
}

// Inverse transforms and overlap-add of the due streams of class c (one per
// output): Y(k) is the sum of the bin's chunk partials, in chunk order.
template <int LG>
__device__ __forceinline__ void srv_inverse_body(const SrvLaunch &a, int c, int b, int nb,
                                                 float2 *sm)
{
    constexpr int P = 1 << LG, L = P / 2, T = Geo<P>::T, F = Geo<P>::F;
    const SrvClassTables &t = a.cls[c];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *A = sm + f * P, *B = sm + (F + f) * P;
    const int n = a.head->cls_n[c] * a.max_out, off = a.head->cls_off[c];
    for (int base = b * F; base < n; base += nb * F) {             // uniform per CTA
        const int g = base + f;
        const int gi = g < n ? g : 0;
        const SrvDue d = a.due[off + gi / a.max_out];
        const int o = gi % a.max_out;
        const SrvDesc ds = a.desc[d.slot];
        const bool active = g < n && o < ds.n_out;
        const float2 *po = a.part + ((int64_t)d.part_base * a.max_out + o) * SRV_GROUP_BINS;
        const int nc = d.n_chunks;
        const int64_t cstride = (int64_t)a.max_out * SRV_GROUP_BINS;   // next partial slot
        auto ld = [&](int k) {
            const float2 *q = po + ((int64_t)(k / SRV_GROUP_BINS) * nc) * cstride + k % SRV_GROUP_BINS;
            float2 v = q[0];
            for (int ch = 1; ch < nc; ++ch) v = cadd(v, q[ch * cstride]);
            return v;
        };
        float *st = ds.ola + (int64_t)o * 3 * L;
        float *ou = a.out + ((int64_t)d.slot * a.max_out + o) * a.io_stride;
        inverse_stream_block<P>(A, B, j, active, ld, st, ou, t.rot, t.post, t.tw);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_srv_inverse(SrvLaunch a)
{
    if (*a.skip) return;
    extern __shared__ float2 sm[];
    int b, nb;
    const int c = srv_class_of(a.inv_start, a.n_cls, b, nb);
    switch (a.cls[c].lgP) {                                       // uniform per CTA
    case 5: srv_inverse_body<5>(a, c, b, nb, sm); break;
    case 6: srv_inverse_body<6>(a, c, b, nb, sm); break;
    case 7: srv_inverse_body<7>(a, c, b, nb, sm); break;
    case 8: srv_inverse_body<8>(a, c, b, nb, sm); break;
    case 9: srv_inverse_body<9>(a, c, b, nb, sm); break;
    case 10: srv_inverse_body<10>(a, c, b, nb, sm); break;
    default: srv_inverse_body<11>(a, c, b, nb, sm); break;
    }
}

}  // namespace

cudaError_t srv_mac_occupancy(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_srv_mac, MAC_THREADS, 0);
}

int srv_grid_transforms(int lgP, int64_t transforms, int n_sm)
{
    const int P = 1 << lgP, T = P / 8, F = (256 / T) > 0 ? 256 / T : 1;
    int64_t g = (transforms + F - 1) / F;
    const int64_t cap = 4 * (int64_t)n_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

cudaError_t srv_launch_gate(const SrvHead *head, SrvStatus *status, int *skip, long long wait_ns,
                            long long max_iter, cudaStream_t st)
{
    k_srv_gate<<<1, 32, 0, st>>>(head, status, skip, wait_ns, max_iter);
    return cudaGetLastError();
}

// shared memory of the fused transform launches: 2 F P float2 is 4096 float2
// for every P (F = 2048 / P transforms of P points)
constexpr size_t SRV_FFT_SMEM = 2 * 2048 * sizeof(float2);

cudaError_t srv_launch_forward(const SrvLaunch &a, cudaStream_t st)
{
    k_srv_forward<<<a.fwd_start[a.n_cls], 256, SRV_FFT_SMEM, st>>>(a);
    return cudaGetLastError();
}

cudaError_t srv_launch_mac(const SrvLaunch &a, cudaStream_t st)
{
    k_srv_mac<<<a.mac_grid, MAC_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t srv_launch_inverse(const SrvLaunch &a, cudaStream_t st)
{
    k_srv_inverse<<<a.inv_start[a.n_cls], 256, SRV_FFT_SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tvolap

// Partition multiply-accumulate of TVOLAP (Eq. 7) on sm_103a: the cp.async
// variant of the offline kernel, the streaming tick and the selection kernel.
// (The TMA-staged offline kernel is in kernels_mac_tma.cu.)
//
//   Y(k, t) = sum_{m < M, t - 2m >= 0} H_t(k, m) X(k, t - 2m),
//   H_t = H[a_t] + alpha_t (H[b_t] - H[a_t])
//
// The product is elementwise per bin, so it runs on the FP32 pipes (no tensor
// cores: it is not a dense contraction).
//
// Offline mapping: a lane owns one bin, a warp owns a run of R output blocks
// of equal parity t0, t0+2, .., t0+2(R-1). Along m the X values a run needs
// slide by one block per step (X(t0 + 2(r - m))), so each step brings one new
// X value and the run's filter values of partition m, and does R complex
// multiply-accumulates from registers (mac_common.cuh gives the slot form of
// the filter mix). Here each lane prefetches its operands D steps ahead with
// 8-byte cp.async into a per-thread ring in shared memory.
//
// Streaming tick: a CTA owns 64 bins of one output; its 8 warps split the
// partitions, each lane streams float4 (two bins) of delay line and filter,
// and the 8 partial sums are added in fixed order through shared memory.
#include "internal.h"
#include "mac_common.cuh"

namespace tvolap {

using namespace mac;

namespace {

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 8 : 0;          // 0: fill the destination with zeros
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int LSU_R = 8;        // output blocks per warp
constexpr int LSU_D = 4;        // cp.async steps in flight
constexpr int LSU_WARPS = 4;

struct LsuArgs {
    const float2 *Xc;          // X of this output's input channel, offset to the lane's bin
    const float2 *bk;          // bank offset to the lane's bin
    float2 *Yo;                // Y of this output, offset to the lane's bin
    const int32_t *ao, *bo;    // schedule rows of this output (bo may be null)
    const float *alo;          // may be null
    int M, P, n_blocks, n_slots_total, null_slot;   // M: slot stride; n_blocks: this output's
    int Mo;                    // partitions this output uses (loop bound, <= M)
    unsigned *err;
    float2 *ring;              // this thread's ring base
    int ring_stride;
    int lane;
};

template <int R, int D, int NS>
__device__ __forceinline__ void lsu_run(const LsuArgs &g, int tf, int m_end, const RunSlots<R> &rs,
                                        CAcc (&acc)[R])
{
    const float2 zero = make_float2(0.f, 0.f);
    const int64_t MP = (int64_t)g.M * g.P;
    const int P = g.P;
    const float2 *H[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) H[j] = g.bk + (int64_t)rs.sl[j] * MP;
    // ring row j of stage q: ring[(q * (NS + 1) + j) * ring_stride]; row NS holds X
    auto issue = [&](int m) {
        float2 *st = g.ring + (int64_t)((m % D) * (NS + 1)) * g.ring_stride;
        const bool live = m < m_end;
        const int tq = tf - 2 * m;
        cp_async8(st + NS * g.ring_stride, g.Xc + (int64_t)(tq > 0 ? tq : 0) * P,
                  live && m > 0 && tq >= 0);
#pragma unroll
        for (int j = 0; j < NS; ++j)
            cp_async8(st + j * g.ring_stride, H[j] + (int64_t)(live ? m : 0) * P, live);
        cp_async_commit();
    };
    float2 xw[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        xw[r] = (t < g.n_blocks) ? __ldg(g.Xc + (int64_t)t * P) : zero;
        acc[r] = cacc_zero();
    }
#pragma unroll
    for (int q = 0; q < D; ++q) issue(q);
    for (int m0 = 0; m0 < m_end; m0 += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int m = m0 + u;
            if (m < m_end) {
                cp_async_wait<D - 1>();
                const float2 *st = g.ring + (int64_t)((m % D) * (NS + 1)) * g.ring_stride;
                if (m > 0) xw[(R - u) % R] = st[NS * g.ring_stride];   // X(tf - 2m) enters
                float2 hs[NS > 1 ? NS - 1 : 1];
#pragma unroll
                for (int j = 1; j < NS; ++j) hs[j - 1] = st[j * g.ring_stride];
                run_step<R, NS>(acc, xw, st[0], hs, rs.w, u);
                issue(m + D);
            }
        }
    }
    cp_async_wait<0>();
}

// Blocks tf, tf+2, .., tf+2(R-1) of one output: up to MAX_NS distinct slots
// run the slot form, otherwise the run is split in halves (one block never
// mixes more than two slots, so the split ends).
template <int R, int D>
__device__ __forceinline__ void lsu_process_run(const LsuArgs &g, int tf)
{
    RunSlots<R> rs;
    run_slots<R>(g.ao, g.bo, g.alo, tf, g.n_blocks, g.n_slots_total, g.null_slot, g.err, g.lane, rs);
    if constexpr (R > 1) {
        if (rs.overflow) {
            lsu_process_run<R / 2, D>(g, tf);
            if (tf + R < g.n_blocks) lsu_process_run<R / 2, D>(g, tf + R);
            return;
        }
    }
    int m_end = (tf + 2 * (R - 1)) / 2 + 1;     // partitions with t - 2m >= 0 for some block
    if (m_end > g.Mo) m_end = g.Mo;
    CAcc acc[R];
    if (rs.ns == 1) {
        lsu_run<R, D, 1>(g, tf, m_end, rs, acc);
    } else if (rs.ns == 2) {
        lsu_run<R, D, 2>(g, tf, m_end, rs, acc);
    } else {
        lsu_run<R, D, 3>(g, tf, m_end, rs, acc);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        if (t < g.n_blocks) g.Yo[(int64_t)t * g.P] = cacc_value(acc[r]);
    }
}

// grid: x = run groups (4 runs of R blocks = 4R consecutive blocks), y = 32-bin
// tiles, z = output channels. Warp w runs parity w & 1, run w >> 1.
template <int R, int D>
__global__ void __launch_bounds__(32 * LSU_WARPS)
k_mac_signal_lsu(const float2 *__restrict__ X, int n_blocks, int M, int P,
                 const float2 *__restrict__ bank, int n_slots_total, int null_slot,
                 const int32_t *__restrict__ out_to_in, const int32_t *__restrict__ sa,
                 const int32_t *__restrict__ sb, const float *__restrict__ sal,
                 int64_t sched_stride, float2 *__restrict__ Y, unsigned *err, Ragged rg)
{
    __shared__ float2 ring_all[D * (MAX_NS + 1) * 32 * LSU_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = blockIdx.y * 32 + lane;
    const int o = blockIdx.z;
    const int tf = blockIdx.x * (4 * R) + (w >> 1) * (2 * R) + (w & 1);
    int nb_o = n_blocks, Mo = M;
    if (rg.out_len) {                                 // ragged: this output's blocks, partitions
        const int64_t b = blocks_of(rg.out_len[o], P / 2);
        nb_o = b < n_blocks ? (int)b : n_blocks;
        const int po = rg.parts[o];
        Mo = po < 1 ? 1 : (po < M ? po : M);
    }
    if (tf >= nb_o) return;                           // whole warp; no barriers below
    LsuArgs g;
    g.Xc = X + (int64_t)out_to_in[o] * n_blocks * P + k;
    g.bk = bank + k;
    g.Yo = Y + (int64_t)o * n_blocks * P + k;
    g.ao = sa + (int64_t)o * sched_stride;
    g.bo = sb ? sb + (int64_t)o * sched_stride : nullptr;
    g.alo = sal ? sal + (int64_t)o * sched_stride : nullptr;
    g.M = M;
    g.Mo = Mo;
    g.P = P;
    g.n_blocks = nb_o;
    g.n_slots_total = n_slots_total;
    g.null_slot = null_slot;
    g.err = err;
    g.ring = ring_all + threadIdx.x;
    g.ring_stride = 32 * LSU_WARPS;
    g.lane = lane;
    lsu_process_run<R, D>(g, tf);
}

// One streaming tick. grid: x = 64-bin tiles, y = outputs; 256 threads.
__global__ void __launch_bounds__(256)
k_mac_stream(const float2 *__restrict__ ring, int M, int P, int64_t tick,
             const float2 *__restrict__ bank, int n_slots_total, int null_slot,
             const int32_t *__restrict__ out_to_in, const int32_t *sa, const int32_t *sb,
             const float *sal, int32_t *cur_a, int32_t *cur_b, float *cur_al, int keep,
             float2 *__restrict__ Ys, unsigned *err)
{
    __shared__ float4 red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int o = blockIdx.y;
    const int k = blockIdx.x * 64 + 2 * lane;          // bins k, k+1
    const bool lane_on = k < P;
    int a = sa[o];
    int b = sb ? sb[o] : a;
    float al = sal ? sal[o] : 0.f;
    if (keep && blockIdx.x == 0 && threadIdx.x == 0) {  // persist this tick's selection
        cur_a[o] = a;
        cur_b[o] = b;
        cur_al[o] = al;
    }
    a = checked_slot(a, n_slots_total, null_slot, err);
    b = checked_slot(b, n_slots_total, null_slot, err);
    const bool single = (a == b) || (al == 0.f);
    const int R = 2 * M;
    const int c = out_to_in[o];
    const float4 *ringc = reinterpret_cast<const float4 *>(ring + (int64_t)c * R * P + (lane_on ? k : 0));
    const float4 *Ha = reinterpret_cast<const float4 *>(bank + (int64_t)a * M * P + (lane_on ? k : 0));
    const float4 *Hb = reinterpret_cast<const float4 *>(bank + (int64_t)b * M * P + (lane_on ? k : 0));
    const int P4 = P / 2;                               // float4 per spectrum
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane_on) {
        const int tslot = (int)(tick % R);
#pragma unroll 4
        for (int m = w; m < M; m += 8) {
            int slot = tslot - 2 * m;
            if (slot < 0) slot += R;
            const float4 x = __ldg(ringc + (int64_t)slot * P4);
            float4 h = __ldg(Ha + (int64_t)m * P4);
            if (!single) {
                const float4 g = __ldg(Hb + (int64_t)m * P4);
                h.x = fmaf(al, g.x - h.x, h.x);
                h.y = fmaf(al, g.y - h.y, h.y);
                h.z = fmaf(al, g.z - h.z, h.z);
                h.w = fmaf(al, g.w - h.w, h.w);
            }
            acc.x = fmaf(h.x, x.x, acc.x);
            acc.x = fmaf(-h.y, x.y, acc.x);
            acc.y = fmaf(h.x, x.y, acc.y);
            acc.y = fmaf(h.y, x.x, acc.y);
            acc.z = fmaf(h.z, x.z, acc.z);
            acc.z = fmaf(-h.w, x.w, acc.z);
            acc.w = fmaf(h.z, x.w, acc.w);
            acc.w = fmaf(h.w, x.z, acc.w);
        }
    }
    red[w][lane] = acc;
    __syncthreads();
    if (w == 0 && lane_on) {
        float4 s = red[0][lane];
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            const float4 v = red[q][lane];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        reinterpret_cast<float4 *>(Ys + (int64_t)o * P + k)[0] = s;
    }
}

__global__ void k_select(int32_t *cur_a, int32_t *cur_b, float *cur_al, int o, int a, int b,
                         float al)
{
    cur_a[o] = a;
    cur_b[o] = b;
    cur_al[o] = al;
}

}  // namespace

cudaError_t launch_mac_signal_lsu(tvolap_plan *h, const float2 *X, int n_blocks,
                                  const int32_t *sa, const int32_t *sb, const float *sal,
                                  int64_t sched_stride, float2 *Y, Ragged rg)
{
    if (n_blocks <= 0) return cudaSuccess;
    constexpr int R = LSU_R;
    dim3 grid((unsigned)((n_blocks + 4 * R - 1) / (4 * R)), (unsigned)(h->P / 32),
              (unsigned)h->n_out);
    k_mac_signal_lsu<R, LSU_D><<<grid, 32 * LSU_WARPS, 0, h->stream>>>(
        X, n_blocks, h->M, h->P, h->bank, h->n_slots_total, h->null_slot, h->out_to_in, sa, sb,
        sal, sched_stride, Y, h->err, rg);
    return cudaGetLastError();
}

cudaError_t launch_mac_stream(tvolap_plan *h, const int32_t *sa, const int32_t *sb,
                              const float *sal)
{
    int keep = 1;
    if (!sa) {                       // current selection
        sa = h->sel_a;
        sb = h->sel_b;
        sal = h->sel_alpha;
        keep = 0;
    }
    dim3 grid((unsigned)((h->P + 63) / 64), (unsigned)h->n_out);
    k_mac_stream<<<grid, 256, 0, h->stream>>>(h->ring, h->M, h->P, h->tick, h->bank,
                                              h->n_slots_total, h->null_slot, h->out_to_in, sa,
                                              sb, sal, h->sel_a, h->sel_b, h->sel_alpha, keep,
                                              h->Ystream, h->err);
    return cudaGetLastError();
}

cudaError_t launch_select(tvolap_plan *h, int out_ch, int a, int b, float alpha)
{
    k_select<<<1, 1, 0, h->stream>>>(h->sel_a, h->sel_b, h->sel_alpha, out_ch, a, b, alpha);
    return cudaGetLastError();
}

}  // namespace tvolap

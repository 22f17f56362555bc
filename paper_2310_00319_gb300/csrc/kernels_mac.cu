// Partition multiply-accumulate of TVOLAP (Eq. 7) on sm_103a.
//
//   Y(k, t) = sum_{m < M, t - 2m >= 0} H_t(k, m) X(k, t - 2m),
//   H_t = H[a_t] + alpha_t (H[b_t] - H[a_t])
//
// The product is elementwise per bin, so it runs on the FP32 pipes (no tensor
// cores: it is not a dense contraction).
//
// k_mac_signal (offline): a lane owns one bin, a warp owns a run of R output
// blocks of equal parity t0, t0+2, .., t0+2(R-1). Along m the X values the run
// needs slide by one block per step (X(t0 + 2(r - m))), so each step loads one
// new X value, the two filter values of partition m, and does R complex
// multiply-accumulates from registers. The filter pair of a run is normally
// the same for all R blocks (only the mix weight changes); runs whose pair
// changes inside take a path that loads the filter per block.
//
// k_mac_stream (one tick): a CTA owns 64 bins of one output; its 8 warps split
// the partitions, each lane streams float4 (two bins) of delay line and
// filter, and the 8 partial sums are added in fixed order through shared
// memory.
#include "fft_core.cuh"
#include "internal.h"

namespace tvolap {

namespace {

constexpr unsigned ERR_BAD_SLOT = 1u;

__device__ __forceinline__ int checked_slot(int s, int n_slots_total, int null_slot, unsigned *err)
{
    if (s < 0 || s >= n_slots_total) {
        atomicOr(err, ERR_BAD_SLOT);
        return null_slot;
    }
    return s;
}

// acc += h * x
__device__ __forceinline__ void cmac(float2 &acc, float2 h, float2 x)
{
    acc.x = fmaf(h.x, x.x, acc.x);
    acc.x = fmaf(-h.y, x.y, acc.x);
    acc.y = fmaf(h.x, x.y, acc.y);
    acc.y = fmaf(h.y, x.x, acc.y);
}

enum { MODE_SINGLE = 0, MODE_LERP = 1, MODE_GENERAL = 2 };

template <int R, int MODE>
__device__ __forceinline__ void mac_run(const float2 *__restrict__ Xc, const float2 *__restrict__ bank,
                                        int M, int P, int tf, int n_blocks, int m_end,
                                        const int (&a)[R], const int (&b)[R], const float (&al)[R],
                                        float2 (&acc)[R])
{
    const float2 zero = make_float2(0.f, 0.f);
    float2 xw[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        xw[r] = (t < n_blocks) ? __ldg(Xc + (int64_t)t * P) : zero;
        acc[r] = zero;
    }
    const int64_t MP = (int64_t)M * P;
    const float2 *Ha = bank + (int64_t)a[0] * MP;
    const float2 *Hb = bank + (int64_t)b[0] * MP;
    // prefetched operands of the current step
    float2 ha = __ldg(Ha), hb = (MODE == MODE_LERP) ? __ldg(Hb) : zero;
    float2 xn = (m_end > 1 && tf - 2 >= 0) ? __ldg(Xc + (int64_t)(tf - 2) * P) : zero;
    for (int m0 = 0; m0 < m_end; m0 += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int m = m0 + u;
            if (m < m_end) {
                if (m > 0) xw[(R - u) % R] = xn;          // X(tf - 2m) enters the window
                // prefetch the next step
                const int mn = m + 1;
                const int tq = tf - 2 * mn;                // X entering at step m + 1
                const float2 xnn = (mn < m_end && tq >= 0) ? __ldg(Xc + (int64_t)tq * P) : zero;
                float2 han = zero, hbn = zero;
                if (MODE != MODE_GENERAL && mn < m_end) {
                    han = __ldg(Ha + (int64_t)mn * P);
                    if (MODE == MODE_LERP) hbn = __ldg(Hb + (int64_t)mn * P);
                }
                if (MODE == MODE_SINGLE) {
#pragma unroll
                    for (int r = 0; r < R; ++r) cmac(acc[r], ha, xw[(r - u + R) % R]);
                } else if (MODE == MODE_LERP) {
                    const float2 d = csub(hb, ha);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float2 h = make_float2(fmaf(al[r], d.x, ha.x), fmaf(al[r], d.y, ha.y));
                        cmac(acc[r], h, xw[(r - u + R) % R]);
                    }
                } else {
                    const int64_t off = (int64_t)m * P;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float2 pa = __ldg(bank + (int64_t)a[r] * MP + off);
                        const float2 pb = __ldg(bank + (int64_t)b[r] * MP + off);
                        const float2 h = make_float2(fmaf(al[r], pb.x - pa.x, pa.x),
                                                     fmaf(al[r], pb.y - pa.y, pa.y));
                        cmac(acc[r], h, xw[(r - u + R) % R]);
                    }
                }
                xn = xnn;
                ha = han;
                hb = hbn;
            }
        }
    }
}

// grid: x = run groups (4 runs of R blocks = 4R consecutive blocks), y = 32-bin
// tiles, z = output channels. 4 warps: warp w runs parity w & 1, run w >> 1.
template <int R>
__global__ void __launch_bounds__(128)
k_mac_signal(const float2 *__restrict__ X, int n_blocks, int M, int P,
             const float2 *__restrict__ bank, int n_slots_total, int null_slot,
             const int32_t *__restrict__ out_to_in, const int32_t *__restrict__ sa,
             const int32_t *__restrict__ sb, const float *__restrict__ sal, int64_t sched_stride,
             float2 *__restrict__ Y, unsigned *err)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = blockIdx.y * 32 + lane;
    const int o = blockIdx.z;
    const int tf = blockIdx.x * (4 * R) + (w >> 1) * (2 * R) + (w & 1);
    if (tf >= n_blocks) return;                       // whole warp; no barriers below
    const int c = out_to_in[o];
    const int32_t *ao = sa + (int64_t)o * sched_stride;
    const int32_t *bo = sb ? sb + (int64_t)o * sched_stride : nullptr;
    const float *alo = sal ? sal + (int64_t)o * sched_stride : nullptr;
    int a[R], b[R];
    float al[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        if (t < n_blocks) {
            a[r] = checked_slot(ao[t], n_slots_total, null_slot, err);
            b[r] = bo ? checked_slot(bo[t], n_slots_total, null_slot, err) : a[r];
            al[r] = alo ? alo[t] : 0.f;
        } else {                                      // past the end: repeat (results dropped)
            a[r] = r ? a[r - 1] : 0;
            b[r] = r ? b[r - 1] : 0;
            al[r] = r ? al[r - 1] : 0.f;
        }
    }
    bool same_pair = true, all0 = true, all1 = true;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        same_pair &= (a[r] == a[0]) && (b[r] == b[0]);
        all0 &= (al[r] == 0.f);
        all1 &= (al[r] == 1.f);
    }
    // m with t - 2m >= 0 for some block of the run
    int m_end = (tf + 2 * (R - 1)) / 2 + 1;
    if (m_end > M) m_end = M;
    const float2 *Xc = X + (int64_t)c * n_blocks * P + k;
    const float2 *bk = bank + k;
    float2 acc[R];
    if (same_pair && (a[0] == b[0] || all0 || all1)) {
        if (all1 && a[0] != b[0]) {
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = b[r];
        }
        mac_run<R, MODE_SINGLE>(Xc, bk, M, P, tf, n_blocks, m_end, a, b, al, acc);
    } else if (same_pair) {
        mac_run<R, MODE_LERP>(Xc, bk, M, P, tf, n_blocks, m_end, a, b, al, acc);
    } else {
        mac_run<R, MODE_GENERAL>(Xc, bk, M, P, tf, n_blocks, m_end, a, b, al, acc);
    }
    float2 *Yo = Y + (int64_t)o * n_blocks * P + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        if (t < n_blocks) Yo[(int64_t)t * P] = acc[r];
    }
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

cudaError_t launch_mac_signal(tvolap_plan *h, const float2 *X, int n_blocks, const int32_t *sa,
                              const int32_t *sb, const float *sal, int64_t sched_stride,
                              float2 *Y)
{
    if (n_blocks <= 0) return cudaSuccess;
    constexpr int R = 8;
    dim3 grid((unsigned)((n_blocks + 4 * R - 1) / (4 * R)), (unsigned)(h->P / 32),
              (unsigned)h->n_out);
    k_mac_signal<R><<<grid, 128, 0, h->stream>>>(X, n_blocks, h->M, h->P, h->bank,
                                                 h->n_slots_total, h->null_slot, h->out_to_in,
                                                 sa, sb, sal, sched_stride, Y, h->err);
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

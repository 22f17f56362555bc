// Device helpers shared by the multiply-accumulate kernels of Eq. 7.
#pragma once

#include "fft_core.cuh"

namespace tvolap {
namespace mac {

constexpr unsigned ERR_BAD_SLOT = 1u;   // a schedule named a slot outside the bank
constexpr unsigned ERR_TIMEOUT = 2u;    // a bounded wait on a copy gave up

__device__ __forceinline__ int checked_slot(int s, int n_slots_total, int null_slot, unsigned *err)
{
    if (s < 0 || s >= n_slots_total) {
        atomicOr(err, ERR_BAD_SLOT);
        return null_slot;
    }
    return s;
}

// Sum over partitions of one block's complex products h * x, kept as four
// partial sums: p = (sum h.re x.re, sum h.im x.im), q = (sum h.re x.im,
// sum h.im x.re). Each of a product's four FMAs adds into its own register,
// so no accumulator meets both the real and the imaginary part of x (the
// interleaved two-sum form held the FMA pipe about 10 % lower). The value is
// (p.x - p.y, q.x + q.y).
struct CAcc {
    float2 p, q;
};

__device__ __forceinline__ CAcc cacc_zero()
{
    CAcc a;
    a.p = make_float2(0.f, 0.f);
    a.q = make_float2(0.f, 0.f);
    return a;
}

// a += h * x
__device__ __forceinline__ void cmac(CAcc &a, float2 h, float2 x)
{
    a.p.x = fmaf(h.x, x.x, a.p.x);
    a.p.y = fmaf(h.y, x.y, a.p.y);
    a.q.x = fmaf(h.x, x.y, a.q.x);
    a.q.y = fmaf(h.y, x.x, a.q.y);
}

__device__ __forceinline__ float2 cacc_value(const CAcc &a)
{
    return make_float2(a.p.x - a.p.y, a.q.x + a.q.y);
}

// Within a run of R blocks the filter of block r is a mix of the run's
// distinct slots s_0 .. s_{ns-1}: H_r = sum_j w_rj H_{s_j} with sum_j w_rj = 1,
// so H_r = H_{s_0} + sum_{j>=1} w_rj (H_{s_j} - H_{s_0}). NSM is the most
// distinct slots a run may hold (MAX_NS unless a kernel is built for more).
constexpr int MAX_NS = 3;

template <int R, int NSM = MAX_NS>
struct RunSlots {
    int sl[NSM];
    int ns;
    bool overflow;               // more than NSM distinct slots
    float2 w[R][NSM - 1];        // weights of s_1 .. s_{NSM-1} per block, as (w, w) pairs
};

// Distinct slots and mix weights of a run, for a warp whose lanes all take
// that run: lane r < R holds block r's schedule entries a, b, al (already
// checked; other lanes' values are ignored). Slots come in order of first use
// (block order, a before b), a slot counted only where its weight is nonzero,
// found with ballots over the R lanes; every lane ends with the same RunSlots
// (the weights of all R blocks for slots 1 .. NW; a kernel whose runs mix at
// most NW + 1 slots needs no more). The warp must be converged.
template <int R, int NSM, int NW = NSM - 1>
__device__ __forceinline__ void run_slots_lanes(int a, int b, float al, int lane, RunSlots<R, NSM> &rs)
{
    bool va = false, vb = false;
    if (lane < R) {
        va = (al != 1.f) || (a == b);                // a's weight 1 - al, or a single slot
        vb = (al != 0.f) && (b != a);
    }
    int ns = 0;
#pragma unroll
    for (int j = 0; j < NSM; ++j) rs.sl[j] = 0;
#pragma unroll
    for (int j = 0; j < NSM; ++j) {
        const unsigned m = __ballot_sync(0xffffffffu, va || vb);
        if (!m) break;                               // every slot found (uniform)
        const int v = __shfl_sync(0xffffffffu, va ? a : b, __ffs(m) - 1);
        rs.sl[j] = v;
        ns = j + 1;
        va = va && (a != v);
        vb = vb && (b != v);
    }
    rs.overflow = __any_sync(0xffffffffu, va || vb);   // more than NSM distinct slots
    const int a0 = __shfl_sync(0xffffffffu, a, 0);
    if (ns == 0) {
        rs.sl[0] = a0;
        ns = 1;
    }
    rs.ns = ns;
#pragma unroll
    for (int j = 1; j <= NW; ++j) {
        const float wj = (a == rs.sl[j] ? 1.f - al : 0.f) + (b == rs.sl[j] ? al : 0.f);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float wr = __shfl_sync(0xffffffffu, wj, r);
            rs.w[r][j - 1] = make_float2(wr, wr);
        }
    }
}

// run_slots_lanes for blocks tf, tf+2, .., tf+2(R-1) read from the schedule:
// lane r < R loads and checks block r's entries; rows past n_blocks repeat
// the last valid row (their results are dropped).
template <int R, int NSM = MAX_NS>
__device__ __forceinline__ void run_slots(const int32_t *__restrict__ ao, const int32_t *__restrict__ bo,
                                          const float *__restrict__ alo, int tf, int n_blocks,
                                          int n_slots_total, int null_slot, unsigned *err, int lane,
                                          RunSlots<R, NSM> &rs)
{
    int a = 0, b = 0;
    float al = 0.f;
    const int t = tf + 2 * lane;
    if (lane < R && t < n_blocks) {
        a = checked_slot(__ldg(ao + t), n_slots_total, null_slot, err);
        b = bo ? checked_slot(__ldg(bo + t), n_slots_total, null_slot, err) : a;
        al = alo ? __ldg(alo + t) : 0.f;
    }
    // the last valid row of the run (none: every row reads as zeros)
    int last = tf < n_blocks ? (n_blocks - 1 - tf) / 2 : 0;
    if (last > R - 1) last = R - 1;
    const int src = lane < last ? lane : last;
    a = __shfl_sync(0xffffffffu, a, src);
    b = __shfl_sync(0xffffffffu, b, src);
    al = __shfl_sync(0xffffffffu, al, src);
    run_slots_lanes<R, NSM>(a, b, al, lane, rs);
}

// One step of Eq. 7 for the R blocks of a run: partition values h0 = H_{s_0}(m),
// hs[j-1] = H_{s_j}(m); xw holds X(tf + 2(r - m)) at index (r - u) mod R, with
// u = m mod R. Callers unroll over u so every register index is a constant.
template <int R, int NS, int NSM = MAX_NS>
__device__ __forceinline__ void run_step(CAcc (&acc)[R], const float2 (&xw)[R], float2 h0,
                                         const float2 *hs, const float2 (&w)[R][NSM - 1], int u)
{
    // the mix h = h0 + w (h_j - h0) runs as packed pairs (one fma.rn.f32x2 per
    // slot: the same roundings as two fmaf, half the issue slots)
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 dj[NS > 1 ? NS - 1 : 1];
#pragma unroll
    for (int j = 1; j < NS; ++j) dj[j - 1] = __ffma2_rn(h0, m1, hs[j - 1]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float2 h = h0;
#pragma unroll
        for (int j = 1; j < NS; ++j) h = __ffma2_rn(w[r][j - 1], dj[j - 1], h);
        cmac(acc[r], h, xw[(r - u % R + R) % R]);
    }
}

// run_step for a lane that owns BPL adjacent bins: the run's weights are
// shared by the bins, every bin takes exactly the operations of run_step.
template <int R, int NS, int NSM, int BPL>
__device__ __forceinline__ void run_step_bins(CAcc (&acc)[R][BPL], const float2 (&xw)[R][BPL],
                                              const float2 (&h0)[BPL],
                                              const float2 (&hs)[NS > 1 ? NS - 1 : 1][BPL],
                                              const float2 (&w)[R][NSM - 1], int u)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 dj[NS > 1 ? NS - 1 : 1][BPL];
#pragma unroll
    for (int j = 1; j < NS; ++j)
#pragma unroll
        for (int b = 0; b < BPL; ++b) dj[j - 1][b] = __ffma2_rn(h0[b], m1, hs[j - 1][b]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int b = 0; b < BPL; ++b) {
            float2 h = h0[b];
#pragma unroll
            for (int j = 1; j < NS; ++j) h = __ffma2_rn(w[r][j - 1], dj[j - 1][b], h);
            cmac(acc[r][b], h, xw[(r - u % R + R) % R][b]);
        }
    }
}

}  // namespace mac
}  // namespace tvolap

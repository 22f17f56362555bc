// Offline multiply-accumulate of Eq. 7 with TMA staging (sm_103a).
//
// Same work split as the cp.async variant (kernels_mac.cu): a lane owns one
// bin, a warp owns a run of R output blocks of one parity, and each step of m
// brings one new X value and the run's filter values of partition m. Here the
// operands of D consecutive steps arrive as tiles: one lane of the warp issues
// a tiled bulk tensor copy per slot (D partitions x 32 bins of the bank) and
// one for X (D same-parity block rows x 32 bins, read with an element stride of
// two rows), completing on the warp's mbarrier; a double-buffered pair of such
// stages keeps the copies a full chunk ahead of the multiply-accumulates, and
// a step costs the warp only its shared-memory reads and FMAs. Copies that
// start before block 0 or run past partition M - 1 are zero-filled by the copy
// engine. Waits on the mbarriers are bounded: on expiry the warp records
// ERR_TIMEOUT, waits (bounded) for its outstanding copies and leaves.
#include <cuda.h>

#include <mutex>

#include "internal.h"
#include "mac_common.cuh"

namespace tvolap {

using namespace mac;

namespace {

constexpr int TMA_R = 8;          // output blocks per warp
constexpr int TMA_D = TMA_R;      // partitions per staged chunk (one register rotation)
constexpr int TMA_WARPS = 4;
constexpr int ROW_BYTES = 32 * 8; // 32 bins of float2
constexpr int STAGE_ROWS = (1 + MAX_NS) * TMA_D;
constexpr int WARP_BYTES = 128 + TMA_R * ROW_BYTES + 2 * STAGE_ROWS * ROW_BYTES;
static_assert(TMA_R % TMA_D == 0 || TMA_D % TMA_R == 0, "chunk and rotation must nest");
constexpr long long WAIT_CYCLES = 1LL << 32;   // about two seconds at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// The thread sleeps until the phase completes or the hint (ns) expires, so a
// wait costs no issue slots while the copy is in flight.
constexpr uint32_t WAIT_HINT_NS = 1000000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(WAIT_HINT_NS)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete; the outcome
// is made uniform across the warp so every lane takes the same path.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    bool ok = false;
    while (!(ok = mbar_try_wait(bar, parity)) && clock64() - t0 < WAIT_CYCLES) {
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

struct TmaArgs {
    const CUtensorMap *xmap;   // X as [n_in][n_blocks][P] int64, box 32 x D rows (stride 2)
    const CUtensorMap *hmap;   // bank as [slots][M][P] int64, box 32 x D rows
    float2 *Yo;                // Y of this output, offset to the lane's bin
    const int32_t *ao, *bo;
    const float *alo;
    int M, P, n_blocks, n_slots_total, null_slot, cin, k0, lane;
    unsigned *err;
    uint64_t *bar;             // [0] window, [1], [2] stages
    float2 *win;               // [R][32]
    float2 *stage;             // [2][STAGE_ROWS][32]
};

// Per-warp pipeline state carried across the runs of one warp (identical in
// every lane: all decisions that change it are warp-uniform).
struct Pipe {
    uint32_t phase;            // bit q: parity of the next completion of barrier q
    uint32_t inflight;         // bit q: barrier q has copies outstanding
    bool ok;
};

// lane 0: stage q <- X rows and the NS slots' rows of chunk c (partitions
// c*D .. c*D + D - 1) of the run starting at tf.
template <int NS>
__device__ __forceinline__ void issue_chunk(const TmaArgs &g, const int (&sl)[MAX_NS], int tf, int c,
                                            int q)
{
    uint64_t *bar = g.bar + 1 + q;
    float2 *st = g.stage + q * STAGE_ROWS * 32;
    const int m0 = c * TMA_D;
    mbar_expect_tx(bar, (uint32_t)((1 + NS) * TMA_D * ROW_BYTES));
    // X rows t = tf - 2(m0 + D - 1) .. tf - 2 m0 (ascending, stride 2)
    tma_load_3d(st, g.xmap, g.k0, tf - 2 * (m0 + TMA_D - 1), g.cin, bar);
#pragma unroll
    for (int j = 0; j < NS; ++j)
        tma_load_3d(st + (1 + j) * TMA_D * 32, g.hmap, g.k0, m0, sl[j], bar);
}

// One chunk of D steps from stage buffer st; GUARD: the chunk may pass m_end.
template <int R, int NS, bool GUARD>
__device__ __forceinline__ void tma_chunk(const float2 *st, int c, int cu, int m_end,
                                          const RunSlots<R> &rs, float2 (&xw)[R], CAcc (&acc)[R])
{
    constexpr int D = TMA_D;
#pragma unroll
    for (int u = 0; u < D; ++u) {
        const int m = c * D + u;
        const int rot = (cu * D + u) % R;
        if (!GUARD || m < m_end) {
            if (m > 0) xw[(R - rot) % R] = st[(D - 1 - u) * 32];   // X(tf - 2m) enters
            float2 hs[NS > 1 ? NS - 1 : 1];
#pragma unroll
            for (int j = 1; j < NS; ++j) hs[j - 1] = st[((1 + j) * D + u) * 32];
            run_step<R, NS>(acc, xw, st[(D + u) * 32], hs, rs.w, rot);
        }
    }
}

template <int R, int NS>
__device__ __forceinline__ void tma_run(const TmaArgs &g, Pipe &pp, int tf, int m_end,
                                        const RunSlots<R> &rs, CAcc (&acc)[R])
{
    constexpr int D = TMA_D;
    const int lane = g.lane;
    const int nchunks = (m_end + D - 1) / D;
    pp.inflight |= (nchunks > 1) ? 7u : 3u;
    if (lane == 0) {
        // window rows t = tf + 2r, r < R (rows past the end arrive as zeros)
        mbar_expect_tx(g.bar, (uint32_t)(((R + D - 1) / D) * D * ROW_BYTES));
        for (int r0 = 0; r0 < R; r0 += D) tma_load_3d(g.win + r0 * 32, g.xmap, g.k0, tf + 2 * r0, g.cin, g.bar);
        issue_chunk<NS>(g, rs.sl, tf, 0, 0);
        if (nchunks > 1) issue_chunk<NS>(g, rs.sl, tf, 1, 1);
    }
    float2 xw[R];
    if (!mbar_wait(g.bar, pp.phase & 1u)) {
        pp.ok = false;
        return;
    }
    pp.phase ^= 1u;
    pp.inflight &= ~1u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        xw[r] = g.win[r * 32 + lane];
        acc[r] = cacc_zero();
    }
    constexpr int CU = (R >= D) ? R / D : 1;        // chunks per register rotation
    for (int c0 = 0; c0 < nchunks; c0 += CU) {
#pragma unroll
        for (int cu = 0; cu < CU; ++cu) {
            const int c = c0 + cu;
            if (c < nchunks) {
                const int q = c & 1;
                if (!mbar_wait(g.bar + 1 + q, (pp.phase >> (1 + q)) & 1u)) {
                    pp.ok = false;
                    return;
                }
                pp.phase ^= (2u << q);
                pp.inflight &= ~(2u << q);
                const float2 *st = g.stage + q * STAGE_ROWS * 32 + lane;
                if ((c + 1) * D <= m_end)
                    tma_chunk<R, NS, false>(st, c, cu, m_end, rs, xw, acc);
                else
                    tma_chunk<R, NS, true>(st, c, cu, m_end, rs, xw, acc);
                __syncwarp();
                if (c + 2 < nchunks) {
                    pp.inflight |= (2u << q);
                    if (lane == 0) issue_chunk<NS>(g, rs.sl, tf, c + 2, q);
                }
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void tma_process_run(const TmaArgs &g, Pipe &pp, int tf)
{
    RunSlots<R> rs;
    run_slots<R>(g.ao, g.bo, g.alo, tf, g.n_blocks, g.n_slots_total, g.null_slot, g.err, g.lane, rs);
    if constexpr (R > 1) {
        if (rs.overflow) {
            tma_process_run<R / 2>(g, pp, tf);
            if (pp.ok && tf + R < g.n_blocks) tma_process_run<R / 2>(g, pp, tf + R);
            return;
        }
    }
    int m_end = (tf + 2 * (R - 1)) / 2 + 1;     // partitions with t - 2m >= 0 for some block
    if (m_end > g.M) m_end = g.M;
    CAcc acc[R];
    if (rs.ns == 1) {
        tma_run<R, 1>(g, pp, tf, m_end, rs, acc);
    } else if (rs.ns == 2) {
        tma_run<R, 2>(g, pp, tf, m_end, rs, acc);
    } else {
        tma_run<R, 3>(g, pp, tf, m_end, rs, acc);
    }
    if (!pp.ok) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        if (t < g.n_blocks) g.Yo[(int64_t)t * g.P] = cacc_value(acc[r]);
    }
}

// A group: 4 consecutive runs of one parity, blocks t = T0 + 2i, i < 32, with
// T0 = parity + 64 * group; run w of the group starts at tf = T0 + 16 w.
constexpr int GW = 4;                           // runs (warps) per group
constexpr int GROUP_ROWS = GW * TMA_R;          // same-parity blocks per group

__device__ __forceinline__ void group_origin(int p, int grp, int &T0) { T0 = p + 2 * GROUP_ROWS * grp; }

// Per-warp kernel for groups whose runs together mix more than MAX_NS slots
// (listed by the group kernel): each warp stages its own run's slots.
// Persistent: CTA b takes list entries b, b + gridDim.x, ...
__global__ void __launch_bounds__(32 * TMA_WARPS)
k_mac_overflow_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap hmap,
                   int n_blocks, int M, int P, int n_slots_total, int null_slot,
                   const int32_t *__restrict__ out_to_in, const int32_t *__restrict__ sa,
                   const int32_t *__restrict__ sb, const float *__restrict__ sal,
                   int64_t sched_stride, float2 *__restrict__ Y, unsigned *err,
                   const int4 *__restrict__ list, const int *__restrict__ count, Ragged rg)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int R = TMA_R;
    const int n = *count;
    if ((int)blockIdx.x >= n) return;
    if (*(volatile unsigned *)err & ERR_TIMEOUT) return;
    unsigned char *base = smem_raw + w * WARP_BYTES;
    TmaArgs g;
    g.xmap = &xmap;
    g.hmap = &hmap;
    g.lane = lane;
    g.P = P;
    g.n_slots_total = n_slots_total;
    g.null_slot = null_slot;
    g.err = err;
    g.bar = reinterpret_cast<uint64_t *>(base);
    g.win = reinterpret_cast<float2 *>(base + 128);
    g.stage = reinterpret_cast<float2 *>(base + 128 + R * ROW_BYTES);
    if (lane == 0) {
        for (int q = 0; q < 3; ++q) mbar_init(g.bar + q, 1);
        mbar_init_fence();
    }
    __syncwarp();
    Pipe pp{0u, 0u, true};
    for (int e = blockIdx.x; e < n && pp.ok; e += gridDim.x) {
        const int4 ent = list[e];                      // (output, bin tile, parity, group)
        int T0;
        group_origin(ent.z, ent.w, T0);
        const int o = ent.x;
        int nb_o = n_blocks, Mo = M;
        if (rg.out_len) {
            const int64_t b = blocks_of(rg.out_len[o], P / 2);
            nb_o = b < n_blocks ? (int)b : n_blocks;
            const int po = rg.parts[o];
            Mo = po < 1 ? 1 : (po < M ? po : M);
        }
        const int tf = T0 + 2 * R * w;
        if (tf >= nb_o) continue;
        g.n_blocks = nb_o;                             // bounds; rows keep the launch stride
        g.M = Mo;                                      // loop bound (bank rows are addressed by the map)
        g.k0 = ent.y * 32;
        g.cin = out_to_in[o];
        g.Yo = Y + (int64_t)o * n_blocks * P + g.k0 + lane;
        g.ao = sa + (int64_t)o * sched_stride;
        g.bo = sb ? sb + (int64_t)o * sched_stride : nullptr;
        g.alo = sal ? sal + (int64_t)o * sched_stride : nullptr;
        tma_process_run<R>(g, pp, tf);
    }
    if (!pp.ok) {
        // a copy did not land in time: report it, then give each barrier with
        // copies outstanding another bounded wait before the CTA's shared
        // memory is released
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        for (int q = 0; q < 3; ++q)
            if (pp.inflight & (1u << q)) mbar_wait(g.bar + q, (pp.phase >> q) & 1u);
    }
}

// ---------------------------------------------------------------------------
// Group kernel. The 4 consumer warps of a CTA take the 4 runs of a group; a
// fifth warp only loads. Two facts make the loads cheap:
//  * all four runs of a group share the group's slots, so one copy of each
//    slot's rows serves four runs (groups mixing more than NSM slots go to
//    the overflow list and the per-warp kernel);
//  * the runs are consecutive, so the X rows warp w needs at chunk c + 1 are
//    the rows warp w - 1 used at chunk c: every chunk brings only 8 new X rows.
// Rows of the group's parity are numbered i (block t = T0 + 2i) and kept in a
// ring of XRING rows at slot (i + 7) mod XRING; the filter rows of chunk c sit
// in stage c mod NSTAGE. The loader runs up to NSTAGE chunks ahead; consumers
// release a stage on its 'empty' barrier. Rows before block 0 and partitions
// at or past M arrive as zeros, so a chunk always runs all D steps: the extra
// products are exact zeros.
// BPL: adjacent bins per lane (1 or 2); a CTA covers 32 * BPL bins. Two bins
// per lane give each warp two independent bins per step under one set of
// weights and halve the per-CTA costs (census, barriers, window, run set-up)
// per unit of work; each bin's arithmetic is the same either way.
constexpr int NSTAGE = 3;
constexpr int XRING = 64;                             // rows; chunk c writes slots [-8c, -8c+8) mod 64
// NSM: most distinct slots a group may stage (3, or 4 for schedules cycling
// four filters); groups with more go to the overflow list.
template <int NSM, int BPL>
struct GroupGeo {
    static constexpr int HSTAGE_ROWS = NSM * TMA_D;
    static constexpr int BYTES = 256 + (XRING + NSTAGE * HSTAGE_ROWS) * ROW_BYTES * BPL;
    // CTAs per SM the registers must allow
    static constexpr int MIN_CTAS = BPL == 2 ? 2 : 3;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int NSM>
struct GroupSmem {
    uint64_t bar[1 + 2 * NSTAGE];     // 0 window, 1.. full, 1+NSTAGE.. empty
    int U, overflow, n_active;
    int slot[NSM];
};
static_assert(sizeof(GroupSmem<4>) <= 256, "group header must fit its 256 bytes");

__device__ __forceinline__ int ring_slot(int j) { return j & (XRING - 1); }

__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// the lane's BPL adjacent bins of one staged row
template <int BPL>
__device__ __forceinline__ void ld_bins(const float2 *p, float2 (&v)[BPL])
{
    if constexpr (BPL == 2) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    } else {
        v[0] = *p;
    }
}

template <int NS, int NSM, int BPL>
__device__ __forceinline__ void group_chunk(const float2 *xs, const float2 *const (&hb)[NSM],
                                            int c, const RunSlots<TMA_R, NSM> &rs,
                                            float2 (&xw)[TMA_R][BPL], CAcc (&acc)[TMA_R][BPL])
{
    constexpr int D = TMA_D, R = TMA_R, ROWB = 32 * BPL;
#pragma unroll
    for (int u = 0; u < D; ++u) {
        if (c > 0 || u > 0) ld_bins<BPL>(xs + (D - 1 - u) * ROWB, xw[(R - u) % R]);   // X(tf - 2m) enters
        float2 h0[BPL];
        float2 hs[NS > 1 ? NS - 1 : 1][BPL];
        ld_bins<BPL>(hb[0] + u * ROWB, h0);
#pragma unroll
        for (int j = 1; j < NS; ++j) ld_bins<BPL>(hb[j] + u * ROWB, hs[j - 1]);
        run_step_bins<R, NS, NSM, BPL>(acc, xw, h0, hs, rs.w, u);
    }
}

template <int NS, int NSM, int BPL>
__device__ __forceinline__ bool group_consume(GroupSmem<NSM> *gs, const float2 *xring,
                                              const float2 *hst, int w, int lane, int nchunks,
                                              int m_end, const RunSlots<TMA_R, NSM> &rs,
                                              const int (&idx)[NSM], CAcc (&acc)[TMA_R][BPL])
{
    constexpr int D = TMA_D, R = TMA_R, ROWB = 32 * BPL;
    float2 xw[R][BPL];
    // window rows i = 8w + r, r < R, at ring slots 8w + 7 + r (row 0 comes with chunk 0)
    if (!mbar_wait(gs->bar, 0u) || !mbar_wait(gs->bar + 1, 0u)) return false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ld_bins<BPL>(xring + ring_slot(R * w + 7 + r) * ROWB + lane * BPL, xw[r]);
#pragma unroll
        for (int b = 0; b < BPL; ++b) acc[r][b] = cacc_zero();
    }
    for (int c = 0; c < nchunks; ++c) {
        const int q = c % NSTAGE;
        if (c > 0 && !mbar_wait(gs->bar + 1 + q, (uint32_t)(c / NSTAGE) & 1u)) return false;
        if (c * D < m_end) {
            // rows i = 8w - 8c - u, u < 8: ring slots 8(w - c) .. 8(w - c) + 7, row 7 - u
            const float2 *xs = xring + ring_slot(D * (w - c)) * ROWB + lane * BPL;
            const float2 *st = hst + q * GroupGeo<NSM, BPL>::HSTAGE_ROWS * ROWB + lane * BPL;
            const float2 *hb[NSM];
#pragma unroll
            for (int j = 0; j < NSM; ++j) hb[j] = st + idx[j] * D * ROWB;
            group_chunk<NS, NSM, BPL>(xs, hb, c, rs, xw, acc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(gs->bar + 1 + NSTAGE + q);
    }
    return true;
}

// grid: x = (group, parity) pairs, y = (32 * BPL)-bin tiles, z = output
// channels; 4 consumer warps + 1 loader warp. The tensor maps' boxes are
// 32 * BPL bins wide.
template <int NSM, int BPL>
__global__ void __launch_bounds__(32 * (GW + 1), GroupGeo<NSM, BPL>::MIN_CTAS)
k_mac_signal_group(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap hmap,
                   int n_blocks, int M, int P, int n_slots_total, int null_slot,
                   const int32_t *__restrict__ out_to_in, const int32_t *__restrict__ sa,
                   const int32_t *__restrict__ sb, const float *__restrict__ sal,
                   int64_t sched_stride, float2 *__restrict__ Y, unsigned *err,
                   int4 *__restrict__ list, int *__restrict__ count, Ragged rg)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int R = TMA_R, D = TMA_D, ROWB = 32 * BPL;
    constexpr int RB = ROW_BYTES * BPL;                // bytes per staged row
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x & 1, grp = blockIdx.x >> 1;
    const int64_t y_rows = n_blocks;                   // row stride of Y for every output
    if (rg.out_len) {                                  // ragged: this output's blocks, partitions
        const int64_t b = blocks_of(rg.out_len[blockIdx.z], P / 2);
        if (b < n_blocks) n_blocks = (int)b;
        const int po = rg.parts[blockIdx.z];
        M = po < 1 ? 1 : (po < M ? po : M);
    }
    int T0;
    group_origin(p, grp, T0);
    if (T0 >= n_blocks) return;                        // whole CTA
    // a copy wait of another CTA gave up: the whole CTA leaves (one decision for all threads)
    if (__syncthreads_or(threadIdx.x == 0 && (*(volatile unsigned *)err & ERR_TIMEOUT))) return;
    GroupSmem<NSM> *gs = reinterpret_cast<GroupSmem<NSM> *>(smem_raw);
    float2 *xring = reinterpret_cast<float2 *>(smem_raw + 256);
    float2 *hst = reinterpret_cast<float2 *>(smem_raw + 256 + XRING * RB);
    const int o = blockIdx.z, k0 = blockIdx.y * ROWB;
    const int32_t *ao = sa + (int64_t)o * sched_stride;
    const int32_t *bo = sb ? sb + (int64_t)o * sched_stride : nullptr;
    const float *alo = sal ? sal + (int64_t)o * sched_stride : nullptr;
    if (w == GW) {
        // loader warp: distinct slots with nonzero weight over the group's
        // 32 blocks (lane i: block T0 + 2i), then the barriers
        const int t = T0 + 2 * lane;
        int a = 0, b = 0;
        bool va = false, vb = false;
        if (t < n_blocks) {
            a = checked_slot(__ldg(ao + t), n_slots_total, null_slot, err);
            b = bo ? checked_slot(__ldg(bo + t), n_slots_total, null_slot, err) : a;
            const float al = alo ? __ldg(alo + t) : 0.f;
            va = (al != 1.f) || (a == b);
            vb = (al != 0.f) && (b != a);
        }
        int U = 0, ovf = 0;
        for (int it = 0; it <= NSM; ++it) {
            const unsigned ma = __ballot_sync(0xffffffffu, va), mb = __ballot_sync(0xffffffffu, vb);
            if (!ma && !mb) break;
            const int v = ma ? __shfl_sync(0xffffffffu, a, __ffs(ma) - 1)
                             : __shfl_sync(0xffffffffu, b, __ffs(mb) - 1);
            if (U == NSM) {
                ovf = 1;
                break;
            }
            if (lane == 0) gs->slot[U] = v;
            ++U;
            va = va && (a != v);
            vb = vb && (b != v);
        }
        int n_active = (n_blocks - T0 + 2 * R - 1) / (2 * R);
        if (n_active > GW) n_active = GW;
        if (lane == 0) {
            gs->U = U;
            gs->overflow = ovf;
            gs->n_active = n_active;
            mbar_init(gs->bar, 1);
            for (int q = 0; q < NSTAGE; ++q) {
                mbar_init(gs->bar + 1 + q, 1);
                mbar_init(gs->bar + 1 + NSTAGE + q, n_active);
            }
            mbar_init_fence();
        }
    }
    __syncthreads();
    if (gs->overflow) {
        // the per-warp kernel takes 32-bin tiles
        if (threadIdx.x == 0) {
            const int e = atomicAdd(count, BPL);
#pragma unroll
            for (int b = 0; b < BPL; ++b) list[e + b] = make_int4(o, blockIdx.y * BPL + b, p, grp);
        }
        return;
    }
    const int n_active = gs->n_active;
    const int U = gs->U;
    const int cin = out_to_in[o];
    // the chunks cover the partitions of the group's last run (the longest)
    const int t_last = T0 + 2 * R * (n_active - 1);
    int m_all = (t_last + 2 * (R - 1)) / 2 + 1;
    if (m_all > M) m_all = M;
    const int nchunks = (m_all + D - 1) / D;

    if (w == GW) {                                     // ---- loader
        uint32_t filled = 0, ppar = 0;                 // bit q: stage q was filled; its last parity
        bool ok = true;
        if (lane == 0) {
            // window rows i = 1 .. 32 (ring slots 8 .. 39); row i = 0 comes with chunk 0
            mbar_expect_tx(gs->bar, (uint32_t)(4 * D * RB));
            for (int k = 0; k < 4; ++k)
                tma_load_3d(xring + (8 + k * D) * ROWB, &xmap, k0, T0 + 2 + 2 * k * D, cin, gs->bar);
        }
        for (int c = 0; c < nchunks && ok; ++c) {
            const int q = c % NSTAGE;
            if (c >= NSTAGE) {
                // stage q last held chunk c - NSTAGE; the X slots this chunk
                // overwrites were last read by chunk c - 5 < c - NSTAGE
                ok = mbar_wait(gs->bar + 1 + NSTAGE + q, (uint32_t)((c - NSTAGE) / NSTAGE) & 1u);
                if (!ok) break;
            }
            filled |= 1u << q;
            ppar = (ppar & ~(1u << q)) | ((uint32_t)(c / NSTAGE & 1) << q);
            {
                uint64_t *bar = gs->bar + 1 + q;
                if (lane == 0) mbar_expect_tx(bar, (uint32_t)((1 + U) * D * RB));
                __syncwarp();
                // the chunk's copies from U + 1 lanes at once: lane 0 the new X rows
                // i = -8c - 7 .. -8c (blocks T0 - 16c - 14 .. T0 - 16c), lane 1 + j
                // the rows of slot j
                if (lane == 0)
                    tma_load_3d(xring + ring_slot(-D * c) * ROWB, &xmap, k0, T0 - 2 * D * c - 2 * (D - 1),
                                cin, bar);
                else if (lane <= U)
                    tma_load_3d(hst + (q * GroupGeo<NSM, BPL>::HSTAGE_ROWS + (lane - 1) * D) * ROWB, &hmap,
                                k0, c * D, gs->slot[lane - 1], bar);
            }
        }
        if (!ok) {
            // give every copy this warp issued a bounded chance to land before
            // the CTA's shared memory is released (a completed fill returns at once)
            if (lane == 0) atomicOr(err, ERR_TIMEOUT);
            mbar_wait(gs->bar, 0u);
            for (int q = 0; q < NSTAGE; ++q)
                if (filled & (1u << q)) mbar_wait(gs->bar + 1 + q, (ppar >> q) & 1u);
        }
        return;
    }
    if (w >= n_active) return;                        // ---- consumers (no CTA barriers below)
    const int tf = T0 + 2 * R * w;
    RunSlots<R, NSM> rs;
    run_slots<R, NSM>(ao, bo, alo, tf, n_blocks, n_slots_total, null_slot, err, lane, rs);
    int idx[NSM];
#pragma unroll
    for (int j = 0; j < NSM; ++j) {
        idx[j] = 0;
        for (int q = 0; q < U; ++q)
            if (j < rs.ns && gs->slot[q] == rs.sl[j]) idx[j] = q;
    }
    int m_end = (tf + 2 * (R - 1)) / 2 + 1;
    if (m_end > M) m_end = M;
    CAcc acc[R][BPL];
    bool ok;
    if (rs.ns == 1)
        ok = group_consume<1, NSM, BPL>(gs, xring, hst, w, lane, nchunks, m_end, rs, idx, acc);
    else if (rs.ns == 2)
        ok = group_consume<2, NSM, BPL>(gs, xring, hst, w, lane, nchunks, m_end, rs, idx, acc);
    else if (NSM == 3 || rs.ns == 3)
        ok = group_consume<3, NSM, BPL>(gs, xring, hst, w, lane, nchunks, m_end, rs, idx, acc);
    else
        ok = group_consume<NSM, NSM, BPL>(gs, xring, hst, w, lane, nchunks, m_end, rs, idx, acc);
    if (!ok) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        return;
    }
    float2 *Yo = Y + (int64_t)o * y_rows * P + k0 + lane * BPL;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tf + 2 * r;
        if (t < n_blocks) {
            if constexpr (BPL == 2)
                *reinterpret_cast<float4 *>(Yo + (int64_t)t * P) =
                    pack2(cacc_value(acc[r][0]), cacc_value(acc[r][1]));
            else
                Yo[(int64_t)t * P] = cacc_value(acc[r][0]);
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent group kernel: the same groups, runs and chunks as
// k_mac_signal_group, but each CTA takes group after group from a work
// counter, so a group's first copies are issued while the CTA still computes
// the previous group. Two group contexts alternate: each has its half of a
// two-part X ring, its window barrier and the group's description (output,
// tile, the staged slots and the 32 blocks' schedule entries; each consumer
// warp derives its run's slot order and weights from them with ballots over
// eight lanes). The filter stages and
// their full/empty barriers are shared and run on through the groups; with
// PSTAGE stages the loader keeps up to PSTAGE chunks in flight. The loader
// fills context k for group i as soon as the consumers have released it
// (group i - 2 done: barrier 'freed'), publishes it ('ready'), issues its
// window, then its chunks as stages come free (a chunk's copies from several
// lanes at once); the next group's schedule entries load while the current
// group's chunks are issued, and one work-counter request is always in
// flight. Taking groups in counter order keeps the CTAs on neighbouring
// groups, whose X rows and filter rows overlap in L2. Consumer warps without
// a run in a group (past the output's last block) still take part in every
// chunk's barriers, so the empty barriers always count four arrivals.
//
// X ring halves: row i of a group (block T0 + 2i) sits at slot (i + 7) mod
// PRING. Chunks 0 .. PSTAGE-1 of a group may land before the group's window
// has been read into registers, so they must miss the window's slots 8..39:
// chunk c writes slots -8c .. -8c + 7 (mod PRING), hence PRING >= 8 (PSTAGE + 4);
// later chunks wait for chunk c - PSTAGE to be released, after which the
// rows still to be read span 24 + 8 PSTAGE slots, which that bound also covers.

struct PersistCtx {
    int T0, o, k0, cin, n_blocks, M, nchunks, n_active, U, end;
    int slot[4];                               // the group's staged slots
    int a[GROUP_ROWS], b[GROUP_ROWS];          // checked schedule entries of blocks T0 + 2i
    float al[GROUP_ROWS];
};

struct PersistSmem {
    uint64_t win[2], ready[2], freed[2], full[5], empty[5];
    PersistCtx ctx[2];
};
constexpr int PERSIST_HEAD = 2048;
static_assert(sizeof(PersistSmem) <= PERSIST_HEAD, "persistent header must fit its bytes");

// PST filter stages (at most 5: the barrier arrays), ring halves of PRING rows.
template <int NSM, int BPL, int PST>
struct PersistGeo {
    static_assert(PST >= 2 && PST <= 5, "stages");
    static constexpr int PSTAGE = PST;
    static constexpr int PRING = PST <= 4 ? 64 : 8 * (PST + 4);   // >= 8 (PST + 4)
    static constexpr int HSTAGE_ROWS = NSM * TMA_D;
    static constexpr int BYTES = PERSIST_HEAD + (2 * PRING + PSTAGE * HSTAGE_ROWS) * ROW_BYTES * BPL;
};

template <int N>
__device__ __forceinline__ int pring_slot(int j)
{
    const int s = j % N;
    return s < 0 ? s + N : s;
}

// One group for a consumer warp: chunk loop over the shared stages (seq: the
// CTA's running chunk count). m_end = 0 for a warp without a run: it only
// keeps the barriers' count.
template <int NS, int NSM, int BPL, int PST>
__device__ __forceinline__ bool persist_consume(PersistSmem *ps, const float2 *xring, const float2 *hst,
                                                int w, int lane, int nchunks, int m_end, uint32_t &seq,
                                                const RunSlots<TMA_R, NSM> &rs, const int (&idx)[NSM],
                                                CAcc (&acc)[TMA_R][BPL])
{
    using G = PersistGeo<NSM, BPL, PST>;
    constexpr int D = TMA_D, R = TMA_R, ROWB = 32 * BPL, NST = PST;
    float2 xw[R][BPL];
    {
        const int q = seq % NST;
        if (!mbar_wait(&ps->full[q], (seq / NST) & 1u)) return false;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ld_bins<BPL>(xring + pring_slot<G::PRING>(R * w + 7 + r) * ROWB + lane * BPL, xw[r]);
#pragma unroll
        for (int b = 0; b < BPL; ++b) acc[r][b] = cacc_zero();
    }
    for (int c = 0; c < nchunks; ++c, ++seq) {
        const int q = seq % NST;
        if (c > 0 && !mbar_wait(&ps->full[q], (seq / NST) & 1u)) return false;
        if (c * D < m_end) {
            const float2 *xs = xring + pring_slot<G::PRING>(D * (w - c)) * ROWB + lane * BPL;
            const float2 *st = hst + q * G::HSTAGE_ROWS * ROWB + lane * BPL;
            const float2 *hb[NSM];
#pragma unroll
            for (int j = 0; j < NSM; ++j) hb[j] = st + idx[j] * D * ROWB;
            group_chunk<NS, NSM, BPL>(xs, hb, c, rs, xw, acc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ps->empty[q]);
    }
    return true;
}

// A work item (output o, bin tile, parity, group) and the raw schedule entries
// of its 32 blocks (lane i: block T0 + 2i), loaded ahead of use.
struct PersistItem {
    int id, o, tile, p, grp, T0, nb, M;
    int a, b;
    float al;
};

// RNS: most filters one run (its 8 blocks of one parity) may mix in this
// kernel (NSM or 3); with 3, every run takes the arithmetic of the
// three-filter kernels.
template <int NSM, int RNS, int BPL, int PST, int MINB>
__global__ void __launch_bounds__(32 * (GW + 1), MINB)
k_mac_signal_persist(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap hmap,
                     int n_blocks, int M, int P, int n_slots_total, int null_slot,
                     const int32_t *__restrict__ out_to_in, const int32_t *__restrict__ sa,
                     const int32_t *__restrict__ sb, const float *__restrict__ sal,
                     int64_t sched_stride, float2 *__restrict__ Y, unsigned *err,
                     int4 *__restrict__ list, int *__restrict__ count, int n_items, Ragged rg)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using G = PersistGeo<NSM, BPL, PST>;
    constexpr int R = TMA_R, D = TMA_D, ROWB = 32 * BPL, NST = PST;
    constexpr int RB = ROW_BYTES * BPL;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    PersistSmem *ps = reinterpret_cast<PersistSmem *>(smem_raw);
    float2 *xring = reinterpret_cast<float2 *>(smem_raw + PERSIST_HEAD);
    float2 *hst = xring + 2 * G::PRING * ROWB;
    const int groups2 = 2 * (((n_blocks + 1) / 2 + GROUP_ROWS - 1) / GROUP_ROWS);
    const int tiles = P / ROWB;
    const int64_t y_rows = n_blocks;
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(&ps->win[k], 1);
            mbar_init(&ps->ready[k], 1);
            mbar_init(&ps->freed[k], GW);
        }
        for (int q = 0; q < NST; ++q) {
            mbar_init(&ps->full[q], 1);
            mbar_init(&ps->empty[q], GW);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (w == GW) {                                     // ---- loader
        // work indices (uniform) come from a counter, one request kept in flight (lane 0)
        // so that its latency hides behind a group; none once a wait anywhere
        // gave up
        int pend = lane == 0 ? atomicAdd(count + 1, 1) : 0;
        auto fetch = [&]() {
            int v = __shfl_sync(0xffffffffu, pend, 0);
            if (lane == 0) pend = atomicAdd(count + 1, 1);
            if (*(volatile unsigned *)err & ERR_TIMEOUT) v = n_items;
            return v;
        };
        // decode item id and start loading its blocks' schedule entries
        auto prefetch = [&](int id, PersistItem &I) {
            I.id = id;
            if (id >= n_items) return;
            const int x = id % groups2, rest = id / groups2;
            I.tile = rest % tiles;
            I.o = rest / tiles;
            I.p = x & 1;
            I.grp = x >> 1;
            group_origin(I.p, I.grp, I.T0);
            I.nb = n_blocks;
            I.M = M;
            if (rg.out_len) {
                const int64_t bo_ = blocks_of(rg.out_len[I.o], P / 2);
                if (bo_ < n_blocks) I.nb = (int)bo_;
                const int po = rg.parts[I.o];
                I.M = po < 1 ? 1 : (po < M ? po : M);
            }
            const int t = I.T0 + 2 * lane;
            const int64_t off = (int64_t)I.o * sched_stride + t;
            I.a = 0;
            I.b = 0;
            I.al = 0.f;
            if (t < I.nb) {
                I.a = __ldg(sa + off);
                I.b = sb ? __ldg(sb + off) : I.a;
                I.al = sal ? __ldg(sal + off) : 0.f;
            }
        };
        uint32_t seq = 0, filled = 0, ppar = 0, wdone = 0, wpar = 0;
        bool ok = true;
        PersistItem I;
        prefetch(fetch(), I);
        for (int it = 0;; ++it) {
            const int k = it & 1;
            if (it >= 2 && !(ok = mbar_wait(&ps->freed[k], (uint32_t)((it >> 1) - 1) & 1u))) break;
            PersistCtx &cx = ps->ctx[k];
            // the next item with work that fits the staging (others: skipped or listed)
            bool found = false;
            int U = 0, a = 0, b = 0, rns = 0;
            float al = 0.f;
            while (I.id < n_items) {
                if (I.T0 >= I.nb) {
                    prefetch(fetch(), I);
                    continue;
                }
                const int t = I.T0 + 2 * lane;
                bool va = false, vb = false;
                a = b = 0;
                al = 0.f;
                if (t < I.nb) {
                    a = checked_slot(I.a, n_slots_total, null_slot, err);
                    b = sb ? checked_slot(I.b, n_slots_total, null_slot, err) : a;
                    al = I.al;
                    va = (al != 1.f) || (a == b);
                    vb = (al != 0.f) && (b != a);
                }
                // census: the group's distinct slots with a nonzero weight (in block
                // order, a before b; rows past the output's last block take no part)
                U = 0;
                int ovf = 0;
                const bool va0 = va, vb0 = vb;
                for (int i = 0; i <= NSM; ++i) {
                    const unsigned m = __ballot_sync(0xffffffffu, va || vb);
                    if (!m) break;
                    const int v = __shfl_sync(0xffffffffu, va ? a : b, __ffs(m) - 1);
                    if (U == NSM) {
                        ovf = 1;
                        break;
                    }
                    if (lane == 0) cx.slot[U] = v;
                    ++U;
                    va = va && (a != v);
                    vb = vb && (b != v);
                }
                if (!ovf && U > RNS) {
                    // only a group staging more than RNS filters can hold a run that
                    // mixes more: run w = lanes 8w .. 8w + 7, its distinct slots as
                    // run_slots_lanes counts them
                    const int sh = lane & ~(R - 1);
                    bool ra = va0, rb = vb0;
                    rns = 0;
#pragma unroll
                    for (int j = 0; j < NSM; ++j) {
                        const unsigned m = (__ballot_sync(0xffffffffu, ra || rb) >> sh) & 0xffu;
                        const int v = __shfl_sync(0xffffffffu, ra ? a : b, sh + (m ? __ffs(m) - 1 : 0));
                        if (m) {
                            rns = j + 1;
                            ra = ra && (a != v);
                            rb = rb && (b != v);
                        }
                    }
                    // a run mixing more than RNS filters goes to the per-warp
                    // kernel with its whole group (that kernel splits it)
                    if (__any_sync(0xffffffffu, rns > RNS)) ovf = 1;
                }
                if (ovf) {
                    // the per-warp kernel takes 32-bin tiles
                    if (lane == 0) {
                        const int e = atomicAdd(count, BPL);
#pragma unroll
                        for (int bb = 0; bb < BPL; ++bb) list[e + bb] = make_int4(I.o, I.tile * BPL + bb, I.p, I.grp);
                    }
                    prefetch(fetch(), I);
                    continue;
                }
                found = true;
                break;
            }
            if (!found) {
                if (lane == 0) {
                    cx.end = 1;
                    mbar_arrive(&ps->ready[k]);
                }
                break;
            }
            const PersistItem cur = I;
            int n_active = (cur.nb - cur.T0 + 2 * R - 1) / (2 * R);
            if (n_active > GW) n_active = GW;
            const int t_last = cur.T0 + 2 * R * (n_active - 1);
            int m_all = (t_last + 2 * (R - 1)) / 2 + 1;
            if (m_all > cur.M) m_all = cur.M;
            const int nchunks = (m_all + D - 1) / D;
            const int k0 = cur.tile * ROWB, cin = out_to_in[cur.o];
            if (lane == 0) {
                cx.T0 = cur.T0;
                cx.o = cur.o;
                cx.k0 = k0;
                cx.cin = cin;
                cx.n_blocks = cur.nb;
                cx.M = cur.M;
                cx.nchunks = nchunks;
                cx.n_active = n_active;
                cx.U = U;
                cx.end = 0;
            }
            __syncwarp();
            cx.a[lane] = a;
            cx.b[lane] = b;
            cx.al[lane] = al;
            __syncwarp();
            float2 *half = xring + k * G::PRING * ROWB;
            if (lane == 0) {
                mbar_arrive(&ps->ready[k]);
                // window rows i = 1 .. 32 (ring slots 8 .. 39); row i = 0 comes with chunk 0
                mbar_expect_tx(&ps->win[k], (uint32_t)(4 * D * RB));
                for (int kk = 0; kk < 4; ++kk)
                    tma_load_3d(half + (8 + kk * D) * ROWB, &xmap, k0, cur.T0 + 2 + 2 * kk * D, cin, &ps->win[k]);
            }
            wdone |= 1u << k;
            wpar = (wpar & ~(1u << k)) | (((uint32_t)(it >> 1) & 1u) << k);
            prefetch(fetch(), I);                      // the next item's schedule entries load meanwhile
            for (int c = 0; c < nchunks; ++c, ++seq) {
                const int q = seq % NST;
                // stage q last held chunk seq - NST
                if (seq >= NST && !(ok = mbar_wait(&ps->empty[q], ((seq - NST) / NST) & 1u))) break;
                filled |= 1u << q;
                ppar = (ppar & ~(1u << q)) | (((seq / NST) & 1u) << q);
                {
                    uint64_t *bar = &ps->full[q];
                    if (lane == 0) mbar_expect_tx(bar, (uint32_t)((1 + U) * D * RB));
                    __syncwarp();
                    // the chunk's copies from U + 1 lanes at once (about a fifth less
                    // issue time than one lane issuing them in turn): lane 0 the new
                    // X rows i = -8c - 7 .. -8c, lane 1 + j the rows of slot j
                    if (lane == 0)
                        tma_load_3d(half + pring_slot<G::PRING>(-D * c) * ROWB, &xmap, k0,
                                    cur.T0 - 2 * D * c - 2 * (D - 1), cin, bar);
                    else if (lane <= U)
                        tma_load_3d(hst + (q * G::HSTAGE_ROWS + (lane - 1) * D) * ROWB, &hmap, k0, c * D,
                                    cx.slot[lane - 1], bar);
                }
            }
            if (!ok) break;
        }
        if (!ok) {
            // a wait gave up: report it and give the copies this warp issued a
            // bounded chance to land before the CTA's shared memory is released
            // (the consumers' own waits end by their bounds)
            if (lane == 0) atomicOr(err, ERR_TIMEOUT);
            for (int kk = 0; kk < 2; ++kk)
                if (wdone & (1u << kk)) mbar_wait(&ps->win[kk], (wpar >> kk) & 1u);
            for (int q = 0; q < NST; ++q)
                if (filled & (1u << q)) mbar_wait(&ps->full[q], (ppar >> q) & 1u);
        }
        return;
    }

    // ---- consumers
    uint32_t seq = 0;
    for (int it = 0;; ++it) {
        const int k = it & 1;
        const uint32_t use = (uint32_t)(it >> 1) & 1u;
        if (!mbar_wait(&ps->ready[k], use)) break;
        const PersistCtx &cx = ps->ctx[k];
        if (cx.end) return;
        const int T0 = cx.T0, nb_o = cx.n_blocks, nchunks = cx.nchunks, U = cx.U;
        const int tf = T0 + 2 * R * w;
        const bool active = w < cx.n_active;
        // the run's slots and weights from the blocks' entries (lane r < 8: block r)
        RunSlots<R, NSM> rs;
        int idx[NSM];
        {
            // rows past the output's last block repeat the run's last valid row
            int lastr = tf < nb_o ? (nb_o - 1 - tf) / 2 : 0;
            if (lastr > R - 1) lastr = R - 1;
            const int rr = lane < lastr ? lane : lastr;
            run_slots_lanes<R, NSM, RNS - 1>(cx.a[R * w + rr], cx.b[R * w + rr], cx.al[R * w + rr], lane, rs);
#pragma unroll
            for (int j = 0; j < NSM; ++j) {
                int q0 = 0;
#pragma unroll
                for (int q = 0; q < NSM; ++q)
                    if (q < U && j < rs.ns && cx.slot[q] == rs.sl[j]) q0 = q;
                idx[j] = q0;
            }
        }
        int m_end = 0;
        if (active) {
            m_end = (tf + 2 * (R - 1)) / 2 + 1;
            if (m_end > cx.M) m_end = cx.M;
        }
        if (!mbar_wait(&ps->win[k], use)) break;
        const float2 *half = xring + k * G::PRING * ROWB;
        CAcc acc[R][BPL];
        bool ok;
        if (!active || rs.ns == 1)
            ok = persist_consume<1, NSM, BPL, PST>(ps, half, hst, w, lane, nchunks, m_end, seq, rs, idx, acc);
        else if (rs.ns == 2)
            ok = persist_consume<2, NSM, BPL, PST>(ps, half, hst, w, lane, nchunks, m_end, seq, rs, idx, acc);
        else if (RNS == 3 || rs.ns == 3)
            ok = persist_consume<3, NSM, BPL, PST>(ps, half, hst, w, lane, nchunks, m_end, seq, rs, idx, acc);
        else
            ok = persist_consume<NSM, NSM, BPL, PST>(ps, half, hst, w, lane, nchunks, m_end, seq, rs, idx, acc);
        if (!ok) break;
        if (active) {
            float2 *Yo = Y + (int64_t)cx.o * y_rows * P + cx.k0 + lane * BPL;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int t = tf + 2 * r;
                if (t < nb_o) {
                    if constexpr (BPL == 2)
                        *reinterpret_cast<float4 *>(Yo + (int64_t)t * P) =
                            pack2(cacc_value(acc[r][0]), cacc_value(acc[r][1]));
                    else
                        Yo[(int64_t)t * P] = cacc_value(acc[r][0]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ps->freed[k]);
    }
    if (lane == 0) atomicOr(err, ERR_TIMEOUT);         // only a wait that gave up gets here
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// 3-D map over [dim2][dim1][P] spectra (8-byte elements), box box_bins bins x rows.
bool encode_spectra(CUtensorMap *map, const void *base, int P, int64_t dim1, int64_t dim2,
                    int box_rows, int row_stride, int box_bins = 32)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)dim1, (cuuint64_t)dim2};
    cuuint64_t strides[2] = {(cuuint64_t)P * 8, (cuuint64_t)P * 8 * (cuuint64_t)dim1};
    cuuint32_t box[3] = {(cuuint32_t)box_bins, (cuuint32_t)(box_rows * row_stride), 1};
    cuuint32_t estr[3] = {1, (cuuint32_t)row_stride, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int NSM, int BPL>
cudaError_t launch_group(const float2 *X, int n_blocks, tvolap_plan *h, int groups,
                         const int32_t *sa, const int32_t *sb, const float *sal,
                         int64_t sched_stride, float2 *Y, Ragged rg)
{
    CUtensorMap xmap, hmap;
    if (!encode_spectra(&xmap, X, h->P, n_blocks, h->n_in, TMA_D, 2, 32 * BPL) ||
        !encode_spectra(&hmap, h->bank, h->P, h->M, h->n_slots_total + 1, TMA_D, 1, 32 * BPL))
        return cudaErrorInvalidValue;
    const size_t gsmem = GroupGeo<NSM, BPL>::BYTES;
    if (gsmem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_mac_signal_group<NSM, BPL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(2 * groups), (unsigned)(h->P / (32 * BPL)), (unsigned)h->n_out);
    k_mac_signal_group<NSM, BPL><<<grid, 32 * (GW + 1), gsmem, h->stream>>>(
        xmap, hmap, n_blocks, h->M, h->P, h->n_slots_total, h->null_slot, h->out_to_in, sa, sb,
        sal, sched_stride, Y, h->err, h->ovf_list, h->ovf_count, rg);
    return cudaGetLastError();
}

template <int NSM, int RNS, int BPL, int PST, int MINB>
cudaError_t launch_persist(const float2 *X, int n_blocks, tvolap_plan *h, int groups,
                           const int32_t *sa, const int32_t *sb, const float *sal,
                           int64_t sched_stride, float2 *Y, Ragged rg)
{
    CUtensorMap xmap, hmap;
    if (!encode_spectra(&xmap, X, h->P, n_blocks, h->n_in, TMA_D, 2, 32 * BPL) ||
        !encode_spectra(&hmap, h->bank, h->P, h->M, h->n_slots_total + 1, TMA_D, 1, 32 * BPL))
        return cudaErrorInvalidValue;
    const int smem = PersistGeo<NSM, BPL, PST>::BYTES;
    static int per_sm = 0;                       // resident CTAs per SM (same for every device here)
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_mac_signal_persist<NSM, RNS, BPL, PST, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mac_signal_persist<NSM, RNS, BPL, PST, MINB>,
                                                          32 * (GW + 1), smem);
        if (e != cudaSuccess) return e;
        per_sm = n > 0 ? n : 1;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int64_t n_items = (int64_t)2 * groups * (h->P / (32 * BPL)) * h->n_out;
    const int64_t grid = n_items < (int64_t)per_sm * sms ? n_items : (int64_t)per_sm * sms;
    k_mac_signal_persist<NSM, RNS, BPL, PST, MINB><<<(unsigned)grid, 32 * (GW + 1), smem, h->stream>>>(
        xmap, hmap, n_blocks, h->M, h->P, h->n_slots_total, h->null_slot, h->out_to_in, sa, sb,
        sal, sched_stride, Y, h->err, h->ovf_list, h->ovf_count, (int)n_items, rg);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mac_signal(tvolap_plan *h, const float2 *X, int n_blocks, const int32_t *sa,
                              const int32_t *sb, const float *sal, int64_t sched_stride,
                              float2 *Y, Ragged rg)
{
    if (n_blocks <= 0) return cudaSuccess;
    CUtensorMap xrun, hmap;
    const bool tma = h->mac_variant != 1 &&
                     encode_spectra(&xrun, X, h->P, n_blocks, h->n_in, TMA_D, 2) &&
                     encode_spectra(&hmap, h->bank, h->P, h->M, h->n_slots_total + 1, TMA_D, 1);
    if (!tma) return launch_mac_signal_lsu(h, X, n_blocks, sa, sb, sal, sched_stride, Y, rg);
    const int tiles = h->P / 32;
    const int groups = ((n_blocks + 1) / 2 + GROUP_ROWS - 1) / GROUP_ROWS;
    const int64_t max_entries = (int64_t)2 * groups * tiles * h->n_out;
    cudaError_t e = ensure_overflow(h, max_entries);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->ovf_count, 0, 2 * sizeof(int), h->stream);   // overflow count, work counter
    if (e != cudaSuccess) return e;
    // 0: persistent groups of up to four filters, runs of up to three; 2: groups
    // (and runs) of up to four filters; 3: one group per CTA; 4: as 3 with two
    // bins per thread where the bins split into 64-bin tiles; 5: as 0 with runs
    // of up to four filters
    if (h->mac_variant == 0)
        e = launch_persist<4, 3, 1, 4, 3>(X, n_blocks, h, groups, sa, sb, sal, sched_stride, Y, rg);
    else if (h->mac_variant == 5)
        e = launch_persist<4, 4, 1, 4, 3>(X, n_blocks, h, groups, sa, sb, sal, sched_stride, Y, rg);
    else if (h->mac_variant == 2)
        e = launch_group<4, 1>(X, n_blocks, h, groups, sa, sb, sal, sched_stride, Y, rg);
    else if (h->mac_variant == 4 && h->P % 64 == 0)
        e = launch_group<3, 2>(X, n_blocks, h, groups, sa, sb, sal, sched_stride, Y, rg);
    else
        e = launch_group<3, 1>(X, n_blocks, h, groups, sa, sb, sal, sched_stride, Y, rg);
    if (e != cudaSuccess) return e;
    const size_t wsmem = (size_t)TMA_WARPS * WARP_BYTES;
    if (wsmem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_mac_overflow_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wsmem);
        if (e != cudaSuccess) return e;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int64_t ogrid = max_entries < 2LL * sms ? max_entries : 2LL * sms;
    k_mac_overflow_tma<<<(unsigned)ogrid, 32 * TMA_WARPS, wsmem, h->stream>>>(
        xrun, hmap, n_blocks, h->M, h->P, h->n_slots_total, h->null_slot, h->out_to_in, sa, sb, sal,
        sched_stride, Y, h->err, h->ovf_list, h->ovf_count, rg);
    return cudaGetLastError();
}

}  // namespace tvolap

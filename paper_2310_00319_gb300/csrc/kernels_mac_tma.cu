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
constexpr int TMA_D = 4;          // partitions per staged chunk
constexpr int TMA_WARPS = 4;
constexpr int ROW_BYTES = 32 * 8; // 32 bins of float2
constexpr int STAGE_ROWS = (1 + MAX_NS) * TMA_D;
constexpr int WARP_BYTES = 128 + TMA_R * ROW_BYTES + 2 * STAGE_ROWS * ROW_BYTES;
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

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
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

template <int R, int NS>
__device__ __forceinline__ void tma_run(const TmaArgs &g, Pipe &pp, int tf, int m_end,
                                        const RunSlots<R> &rs, float2 (&acc)[R])
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
    const float2 zero = make_float2(0.f, 0.f);
    if (!mbar_wait(g.bar, pp.phase & 1u)) {
        pp.ok = false;
        return;
    }
    pp.phase ^= 1u;
    pp.inflight &= ~1u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        xw[r] = g.win[r * 32 + lane];
        acc[r] = zero;
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
#pragma unroll
                for (int u = 0; u < D; ++u) {
                    const int m = c * D + u;
                    const int rot = (cu * D + u) % R;
                    if (m < m_end) {
                        if (m > 0) xw[(R - rot) % R] = st[(D - 1 - u) * 32];   // X(tf - 2m)
                        float2 hs[NS > 1 ? NS - 1 : 1];
#pragma unroll
                        for (int j = 1; j < NS; ++j) hs[j - 1] = st[((1 + j) * D + u) * 32];
                        run_step<R, NS>(acc, xw, st[(D + u) * 32], hs, rs.w, rot);
                    }
                }
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
    run_slots<R>(g.ao, g.bo, g.alo, tf, g.n_blocks, g.n_slots_total, g.null_slot, g.err, rs);
    if constexpr (R > 1) {
        if (rs.overflow) {
            tma_process_run<R / 2>(g, pp, tf);
            if (pp.ok && tf + R < g.n_blocks) tma_process_run<R / 2>(g, pp, tf + R);
            return;
        }
    }
    int m_end = (tf + 2 * (R - 1)) / 2 + 1;     // partitions with t - 2m >= 0 for some block
    if (m_end > g.M) m_end = g.M;
    float2 acc[R];
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
        if (t < g.n_blocks) g.Yo[(int64_t)t * g.P] = acc[r];
    }
}

// grid: x = run groups (4 runs of R blocks = 4R consecutive blocks), y = 32-bin
// tiles, z = output channels. Warp w runs parity w & 1, run w >> 1.
__global__ void __launch_bounds__(32 * TMA_WARPS)
k_mac_signal_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap hmap,
                 int n_blocks, int M, int P, int n_slots_total, int null_slot,
                 const int32_t *__restrict__ out_to_in, const int32_t *__restrict__ sa,
                 const int32_t *__restrict__ sb, const float *__restrict__ sal,
                 int64_t sched_stride, float2 *__restrict__ Y, unsigned *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int R = TMA_R;
    const int tf = blockIdx.x * (4 * R) + (w >> 1) * (2 * R) + (w & 1);
    if (tf >= n_blocks) return;                       // whole warp; no CTA barriers used
    // once any wait has expired, the remaining warps leave at once
    if (*(volatile unsigned *)err & ERR_TIMEOUT) return;
    unsigned char *base = smem_raw + w * WARP_BYTES;
    TmaArgs g;
    g.xmap = &xmap;
    g.hmap = &hmap;
    g.k0 = blockIdx.y * 32;
    g.lane = lane;
    const int o = blockIdx.z;
    g.cin = out_to_in[o];
    g.Yo = Y + (int64_t)o * n_blocks * P + g.k0 + lane;
    g.ao = sa + (int64_t)o * sched_stride;
    g.bo = sb ? sb + (int64_t)o * sched_stride : nullptr;
    g.alo = sal ? sal + (int64_t)o * sched_stride : nullptr;
    g.M = M;
    g.P = P;
    g.n_blocks = n_blocks;
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
    tma_process_run<R>(g, pp, tf);
    if (!pp.ok) {
        // a copy did not land in time: report it, then give each barrier with
        // copies outstanding another bounded wait before the CTA's shared
        // memory is released
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        for (int q = 0; q < 3; ++q)
            if (pp.inflight & (1u << q)) mbar_wait(g.bar + q, (pp.phase >> q) & 1u);
    }
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

// 3-D map over [dim2][dim1][P] spectra (8-byte elements), box 32 bins x rows.
bool encode_spectra(CUtensorMap *map, const void *base, int P, int64_t dim1, int64_t dim2,
                    int box_rows, int row_stride)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)dim1, (cuuint64_t)dim2};
    cuuint64_t strides[2] = {(cuuint64_t)P * 8, (cuuint64_t)P * 8 * (cuuint64_t)dim1};
    cuuint32_t box[3] = {32, (cuuint32_t)(box_rows * row_stride), 1};
    cuuint32_t estr[3] = {1, (cuuint32_t)row_stride, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_mac_signal(tvolap_plan *h, const float2 *X, int n_blocks, const int32_t *sa,
                              const int32_t *sb, const float *sal, int64_t sched_stride,
                              float2 *Y)
{
    if (n_blocks <= 0) return cudaSuccess;
    CUtensorMap xmap, hmap;
    const bool tma = h->mac_variant != 1 &&
                     encode_spectra(&xmap, X, h->P, n_blocks, h->n_in, TMA_D, 2) &&
                     encode_spectra(&hmap, h->bank, h->P, h->M, h->n_slots_total + 1, TMA_D, 1);
    if (!tma) return launch_mac_signal_lsu(h, X, n_blocks, sa, sb, sal, sched_stride, Y);
    constexpr int R = TMA_R;
    dim3 grid((unsigned)((n_blocks + 4 * R - 1) / (4 * R)), (unsigned)(h->P / 32),
              (unsigned)h->n_out);
    const size_t smem = (size_t)TMA_WARPS * WARP_BYTES;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_mac_signal_tma,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_mac_signal_tma<<<grid, 32 * TMA_WARPS, smem, h->stream>>>(
        xmap, hmap, n_blocks, h->M, h->P, h->n_slots_total, h->null_slot, h->out_to_in, sa, sb, sal,
        sched_stride, Y, h->err);
    return cudaGetLastError();
}

}  // namespace tvolap

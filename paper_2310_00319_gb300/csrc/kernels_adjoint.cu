// Differentiable TVOLAP: Eq. 7 with free per-block partition spectra, and its
// adjoint (sm_103a).
//
// Parameters P[o][t][m][k] (t < p_blocks, m < M, k < P) replace the filter
// spectra of Eq. 7: Y(t) = sum_{m, t-2m >= 0} P(t, m) X(t - 2m). Nothing in P is
// reused across blocks, so both kernels stream P once from HBM and are
// bandwidth-bound; X and the gradient spectra G are small and come from L2.
//
//   k_mac_params   Y(t) for t in a range.
//   k_adjoint_mac  for q in a range: dX(q) = sum_m G(q + 2m) conj P(q + 2m, m)
//                  (the delay line run backwards) and, in the same pass, every
//                  dP(t, m) with t - 2m = q: dP(t, m) = G(t) conj X(q). When the
//                  range starts at 0, extra threads for q = -(2M-2) .. -1 write
//                  the zero gradients of the P entries that only ever multiply
//                  blocks before the signal.
// A thread owns two bins (16-byte loads and stores) of one block; the partition
// loop is unrolled 8 deep to keep enough loads in flight.
#include "fft_block.cuh"
#include "fft_lane.cuh"
#include "internal.h"

namespace tvolap {

namespace {

__device__ __forceinline__ void cmac4(float4 &acc, float4 a, float4 b)    // acc += a * b
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.z = fmaf(a.z, b.z, acc.z);
    acc.z = fmaf(-a.w, b.w, acc.z);
    acc.w = fmaf(a.z, b.w, acc.w);
    acc.w = fmaf(a.w, b.z, acc.w);
}

__device__ __forceinline__ void cmacc4(float4 &acc, float4 a, float4 b)   // acc += a * conj(b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.y = fmaf(-a.x, b.y, acc.y);
    acc.z = fmaf(a.z, b.z, acc.z);
    acc.z = fmaf(a.w, b.w, acc.z);
    acc.w = fmaf(a.w, b.z, acc.w);
    acc.w = fmaf(-a.z, b.w, acc.w);
}

__device__ __forceinline__ float4 mulc4(float4 a, float4 b)               // a * conj(b)
{
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    cmacc4(r, a, b);
    return r;
}

constexpr int AT = 128;   // threads per CTA (one bin pair each)

// grid: x = t_count, y = outputs, z = groups of AT bin pairs
__global__ void __launch_bounds__(AT)
k_mac_params(const float4 *__restrict__ X, int64_t x_first, int x_count, const float4 *__restrict__ Pm,
             int64_t p_blocks, int M, int P4, int64_t t_first, int t_count,
             const int32_t *__restrict__ out_to_in, float4 *__restrict__ Y, int64_t y_rows)
{
    const int k = blockIdx.z * AT + threadIdx.x;
    if (k >= P4) return;
    const int o = blockIdx.y;
    const int64_t i = blockIdx.x;
    const int64_t t = t_first + i;
    const int c = out_to_in[o];
    const float4 *Pt = Pm + ((int64_t)o * p_blocks + t) * M * P4 + k;
    const float4 *Xt = X + ((int64_t)c * x_count + (t - x_first)) * P4 + k;   // row of X(t)
    int m_end = (int)(t / 2) + 1;                       // t - 2m >= 0
    if (m_end > M) m_end = M;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int m = 0; m < m_end; ++m)   // P is read once: evict-first; X comes from L2
        cmac4(acc, __ldcs(Pt + (int64_t)m * P4), __ldg(Xt - (int64_t)(2 * m) * P4));
    Y[((int64_t)o * y_rows + i) * P4 + k] = acc;
}

// grid: x = q_count + extra (the virtual blocks q < 0 when q_first == 0),
// y = outputs, z = groups of AT bin pairs
__global__ void __launch_bounds__(AT)
k_adjoint_mac(const float4 *__restrict__ G, int64_t g_first, int g_count,
              const float4 *__restrict__ X, int64_t x_first, int x_count,
              const float4 *__restrict__ Pm, int64_t p_blocks, int M, int P4, int64_t q_first,
              int q_count, const int32_t *__restrict__ out_to_in, float4 *__restrict__ dP,
              float4 *__restrict__ dX, int64_t dx_rows)
{
    const int k = blockIdx.z * AT + threadIdx.x;
    if (k >= P4) return;
    const int o = blockIdx.y;
    const int64_t q = (int64_t)blockIdx.x < q_count ? q_first + blockIdx.x
                                                    : -(int64_t)(blockIdx.x - q_count) - 1;
    const int64_t MP4 = (int64_t)M * P4;
    float4 *dPo = dP + (int64_t)o * p_blocks * MP4 + k;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < 0) {
        // P(t, m) with t = q + 2m < 2m multiplies only blocks before the signal
        for (int m = 0; m < M; ++m) {
            const int64_t t = q + 2 * m;
            if (t >= 0 && t < p_blocks) dPo[t * MP4 + (int64_t)m * P4] = zero;
        }
        return;
    }
    const int c = out_to_in[o];
    const float4 xq = __ldg(X + ((int64_t)c * x_count + (q - x_first)) * P4 + k);
    const float4 *Gq = G + ((int64_t)o * g_count + (q - g_first)) * P4 + k;   // row of G(q)
    const float4 *Pq = Pm + (int64_t)o * p_blocks * MP4 + q * MP4 + k;        // P(q, 0)
    float4 *dPq = dPo + q * MP4;
    int m_end = M;
    if (q + 2 * (int64_t)(M - 1) >= p_blocks) m_end = (int)((p_blocks - 1 - q) / 2) + 1;
    float4 acc = zero;
    // row t = q + 2m of P(t, m) sits at (2m) * M * P4 + m * P4 from P(q, 0)
#pragma unroll 8
    for (int m = 0; m < m_end; ++m) {
        const int64_t off = (int64_t)(2 * m) * MP4 + (int64_t)m * P4;
        const float4 g = __ldg(Gq + (int64_t)(2 * m) * P4);
        cmacc4(acc, g, __ldg(Pq + off));
        dPq[off] = mulc4(g, xq);
    }
    dX[((int64_t)o * dx_rows + (q - q_first)) * P4 + k] = acc;
}

// The adjoint of k_adjoint_mac with the input spectra recomputed in place: a
// CTA transforms F consecutive blocks q of its output's input channel (Eqs. 1,
// 3, 5, the same arithmetic as the forward transform kernel), keeps their
// spectra in shared memory, then runs the adjoint of Eq. 7 for those blocks
// exactly as k_adjoint_mac does. No input spectra are stored anywhere.
// grid: x = ceil(q_count / F), y = outputs.
template <int LG>
__global__ void __launch_bounds__(Lane<(1 << LG)>::THREADS)
k_adjoint_mac_x(const float4 *__restrict__ G, int64_t g_first, int g_count,
                const float *__restrict__ x, int64_t N, int64_t x_stride, int L,
                const float *__restrict__ win, const float2 *__restrict__ rot,
                const float2 *__restrict__ post, const float2 *__restrict__ tw,
                const float4 *__restrict__ Pm, int64_t p_blocks, int M, int64_t q_first,
                int q_count, const int32_t *__restrict__ out_to_in, float4 *__restrict__ dP,
                float4 *__restrict__ dX, int64_t dx_rows)
{
    constexpr int P = 1 << LG, T = Lane<P>::T, F = Lane<P>::F, P4 = P / 2;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *buf = sm + f * lane_buf(P);                // the transform's buffer, then its spectrum
    const int o = blockIdx.y;
    const int c = out_to_in[o];
    const int64_t q0 = q_first + (int64_t)blockIdx.x * F;
    const int64_t q_end = q_first + q_count;
    // forward transform of block q = q0 + f, as the forward transform kernel
    // computes it; its spectrum replaces the transform's data in its buffer
    {
        const int64_t q = q0 + f;
        const bool active = q < q_end;
        SignalPairs src;
        src.xc = x + (int64_t)c * x_stride;
        src.win = win;
        src.start = (q - 1) * (int64_t)L;               // block l = q - 1 starts at l*L
        src.N = N;
        src.pairs = (reinterpret_cast<uintptr_t>(src.xc) & 7) == 0;
        src.set_range(L);
        forward_lane<P, true>(buf, j, f, active, src, rot, post, tw,
                              [&](int k, float2 v) { buf[k] = v; });
    }
    __syncthreads();
    const int64_t MP4 = (int64_t)M * P4;
    float4 *dPo = dP + (int64_t)o * p_blocks * MP4;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = threadIdx.x; it < F * P4; it += blockDim.x) {
        const int ff = it / P4, k = it % P4;
        const int64_t q = q0 + ff;
        if (q >= q_end) continue;
        const float4 xq = reinterpret_cast<const float4 *>(sm + ff * lane_buf(P))[k];
        const float4 *Gq = G + ((int64_t)o * g_count + (q - g_first)) * P4 + k;
        const float4 *Pq = Pm + (int64_t)o * p_blocks * MP4 + q * MP4 + k;
        float4 *dPq = dPo + q * MP4 + k;
        int m_end = M;
        if (q + 2 * (int64_t)(M - 1) >= p_blocks) m_end = (int)((p_blocks - 1 - q) / 2) + 1;
        float4 acc = zero;
#pragma unroll 8
        for (int m = 0; m < m_end; ++m) {
            const int64_t off = (int64_t)(2 * m) * MP4 + (int64_t)m * P4;
            const float4 g = __ldg(Gq + (int64_t)(2 * m) * P4);
            cmacc4(acc, g, __ldg(Pq + off));
            dPq[off] = mulc4(g, xq);
        }
        dX[((int64_t)o * dx_rows + (q - q_first)) * P4 + k] = acc;
    }
}

}  // namespace

cudaError_t launch_mac_params(tvolap_plan *h, const float2 *X, int64_t x_first, int x_count,
                              const float2 *Pm, int64_t p_blocks, int64_t t_first, int t_count,
                              float2 *Y, int64_t y_rows)
{
    if (t_count <= 0) return cudaSuccess;
    const int P4 = h->P / 2;
    dim3 grid((unsigned)t_count, (unsigned)h->n_out, (unsigned)((P4 + AT - 1) / AT));
    k_mac_params<<<grid, AT, 0, h->stream>>>(reinterpret_cast<const float4 *>(X), x_first, x_count,
                                             reinterpret_cast<const float4 *>(Pm), p_blocks, h->M,
                                             P4, t_first, t_count, h->out_to_in,
                                             reinterpret_cast<float4 *>(Y), y_rows);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mac(tvolap_plan *h, const float2 *G, int64_t g_first, int g_count,
                               const float2 *X, int64_t x_first, int x_count, const float2 *Pm,
                               int64_t p_blocks, int64_t q_first, int q_count, float2 *dP,
                               float2 *dX, int64_t dx_rows)
{
    if (q_count <= 0) return cudaSuccess;
    const int extra = (q_first == 0) ? 2 * (h->M - 1) : 0;
    const int P4 = h->P / 2;
    dim3 grid((unsigned)(q_count + extra), (unsigned)h->n_out, (unsigned)((P4 + AT - 1) / AT));
    k_adjoint_mac<<<grid, AT, 0, h->stream>>>(
        reinterpret_cast<const float4 *>(G), g_first, g_count, reinterpret_cast<const float4 *>(X),
        x_first, x_count, reinterpret_cast<const float4 *>(Pm), p_blocks, h->M, P4, q_first, q_count,
        h->out_to_in, reinterpret_cast<float4 *>(dP), reinterpret_cast<float4 *>(dX), dx_rows);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mac_x(tvolap_plan *h, const float2 *G, int64_t g_first, int g_count,
                                 const float *x, int64_t N, int64_t x_stride, const float2 *Pm,
                                 int64_t p_blocks, int64_t q_first, int q_count, float2 *dP,
                                 float2 *dX, int64_t dx_rows)
{
    if (q_count <= 0) return cudaSuccess;
    const int P4 = h->P / 2;
    if (q_first == 0 && h->M > 1) {
        // dP(t, m) with t < 2m: the virtual blocks before the signal (no X, no G read)
        dim3 grid((unsigned)(2 * (h->M - 1)), (unsigned)h->n_out, (unsigned)((P4 + AT - 1) / AT));
        k_adjoint_mac<<<grid, AT, 0, h->stream>>>(
            reinterpret_cast<const float4 *>(G), g_first, g_count, nullptr, 0, 0,
            reinterpret_cast<const float4 *>(Pm), p_blocks, h->M, P4, 0, 0, h->out_to_in,
            reinterpret_cast<float4 *>(dP), reinterpret_cast<float4 *>(dX), dx_rows);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const size_t sm = smem_lane<LG>(Lane<P>::THREADS);
        cudaError_t e = set_smem(k_adjoint_mac_x<LG>, sm);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((q_count + Lane<P>::F - 1) / Lane<P>::F), (unsigned)h->n_out);
        k_adjoint_mac_x<LG><<<grid, Lane<P>::THREADS, sm, h->stream>>>(
            reinterpret_cast<const float4 *>(G), g_first, g_count, x, N, x_stride, h->L, h->win,
            h->rot, h->post, h->tw, reinterpret_cast<const float4 *>(Pm), p_blocks, h->M, q_first,
            q_count, h->out_to_in, reinterpret_cast<float4 *>(dP), reinterpret_cast<float4 *>(dX),
            dx_rows);
    });
    return cudaGetLastError();
}

}  // namespace tvolap

// Transform kernels of the TVOLAP path (sm_103a):
//   k_tables            FP64-generated FP32 twiddle, rotation and window tables
//   k_forward_signal    Eqs. 1, 3, 5 for every block of every input channel
//   k_bank              Eqs. 2, 4, 6 for every partition of a set of responses
//   k_inverse_ola       Eq. 8 and the overlap-add of Eqs. 9-12, offline
//   k_forward_stream    one new block per input into the delay line
//   k_inverse_stream    one block per output, overlap-add against the state
// Every transform is P = 2L complex points (see fft_core.cuh). The offline
// forward, bank and inverse kernels and the streaming inverse run T = P/16
// threads per transform with sixteen values each (fft_lane.cuh); the
// streaming forward (where one transform's latency counts) and the adjoint
// transforms run T = P/8 threads per transform (fft_block.cuh). F transforms
// share a CTA.
#include "fft_block.cuh"
#include "fft_lane.cuh"
#include "internal.h"

namespace tvolap {

namespace {

__global__ void k_tables(float2 *tw, float2 *rot, float2 *post, float *win, int L)
{
    const int P = 2 * L;
    const int n_tw = tw_size(P);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tw; i += gridDim.x * blockDim.x) {
        // stage-major twiddle rows (see tw_offset): find the stage of entry i
        int q = i, Ns = stage_radix(P, 1);
        while (q >= (stage_radix(P, Ns) - 1) * Ns) {
            q -= (stage_radix(P, Ns) - 1) * Ns;
            Ns *= stage_radix(P, Ns);
        }
        const int r = q / Ns + 1, k = q % Ns, R = stage_radix(P, Ns);
        double s, c;
        sincospi(2.0 * (double)(r * k) / (double)(Ns * R), &s, &c);   // e^{-2 pi i r k / (Ns R)}
        tw[i] = make_float2((float)c, (float)-s);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        double s, c;
        sincospi((double)i / (double)P, &s, &c);            // e^{-i pi r / P}
        rot[i] = make_float2((float)c, (float)-s);
        if (i < P / 2) {
            sincospi((2.0 * i + 1.0) / (2.0 * P), &s, &c);  // W_{4L}^{k + 1/2}
            post[i] = make_float2((float)c, (float)-s);
        }
        // periodic Hann of length 2L with amplitude 1/2 (hop-L windows sum to 1)
        win[i] = (float)(0.5 * (1.0 - cospi((double)i / (double)L)));
    }
}

// Forward transforms of every block of every input channel (Eqs. 1, 3, 5):
// transform g = (channel, block) per group of T threads.
template <int LG>
__global__ void __launch_bounds__(Lane<(1 << LG)>::THREADS)
k_forward_signal(const float *__restrict__ x, int64_t N, int64_t x_stride, int L, int n_blocks,
                 int64_t total, const float *__restrict__ win, const float2 *__restrict__ rot,
                 const float2 *__restrict__ post, const float2 *__restrict__ tw,
                 float2 *__restrict__ X, int64_t t_first, Ragged rg)
{
    constexpr int P = 1 << LG, T = Lane<P>::T;
    const int F = blockDim.x / T;                      // transforms per CTA (launch's choice)
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *buf = sm + f * lane_buf(P);
    const int64_t g = (int64_t)blockIdx.x * F + f;
    bool active = g < total;
    const int64_t c = active ? g / n_blocks : 0;
    const int64_t t = active ? g % n_blocks : 0;
    if (rg.n) {                                        // ragged: this channel's length and blocks
        int64_t nc = rg.n[c];
        N = nc < 0 ? 0 : (nc < N ? nc : N);
        int64_t oc = rg.out_len[c];
        active = active && (t_first + t < blocks_of(oc, L));
        // past every channel's last block: the whole CTA leaves (uniform vote,
        // before the transform's barriers)
        if (!__syncthreads_or(active)) return;
    }
    SignalPairs src;
    src.xc = x + c * x_stride;
    src.win = win;
    src.start = (t_first + t - 1) * (int64_t)L;        // block l = t - 1 starts at l*L
    src.N = N;
    // start is even: a pair is one 8-byte load when the row is 8-byte aligned
    src.pairs = (reinterpret_cast<uintptr_t>(src.xc) & 7) == 0;
    src.set_range(L);
    float2 *Xo = X + g * P;
    forward_lane<P>(buf, j, f, active, src, rot, post, tw, [&](int k, float2 v) {
        if (active) Xo[k] = v;
    });
}

template <int LG>
__global__ void __launch_bounds__(Lane<(1 << LG)>::THREADS)
k_bank(const float *__restrict__ ir, int ir_len, int64_t ir_stride, int M, int L, int64_t total,
       const float2 *__restrict__ rot, const float2 *__restrict__ post,
       const float2 *__restrict__ tw, float2 *__restrict__ bank_out)
{
    constexpr int P = 1 << LG, T = Lane<P>::T;
    const int F = blockDim.x / T;                      // transforms per CTA (launch's choice)
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *buf = sm + f * lane_buf(P);
    const int64_t g = (int64_t)blockIdx.x * F + f;     // transform = (response, partition)
    const bool active = g < total;
    const int64_t s = active ? g / M : 0;
    const int64_t m = active ? g % M : 0;
    const float *h = ir + s * ir_stride;
    const int64_t base = 2 * m * (int64_t)L;            // partition m: taps [2mL, 2mL + 2L)
    auto src = [&](int n) {                            // taps 2n, 2n+1 of the partition
        const int64_t i0 = base + 2 * n;
        const float a = (i0 < ir_len) ? __ldg(h + i0) : 0.f;
        const float b = (i0 + 1 < ir_len) ? __ldg(h + i0 + 1) : 0.f;
        return make_float2(a, b);
    };
    float2 *Ho = bank_out + g * P;                     // slots are consecutive [s][m][P]
    forward_lane<P>(buf, j, f, active, src, rot, post, tw, [&](int k, float2 v) {
        if (active) Ho[k] = v;
    });
}

// Adjoint of Eq. 8 for the gradient g = dL/dy of every output: for block
// t = t_first + i, G[o][i] = (1/2L) * half-bin DFT of the 4L samples
// g[o][(t-1)L .. (t+3)L) (zeros outside [0, g_len)): all 4L inputs, no window.
template <int LG>
__global__ void __launch_bounds__(Geo<(1 << LG)>::THREADS)
k_adjoint_output(const float *__restrict__ g, int64_t g_len, int64_t g_stride, int L,
                 int n_blocks, int64_t total, int64_t t_first, const float2 *__restrict__ rot,
                 const float2 *__restrict__ post, const float2 *__restrict__ tw,
                 float2 *__restrict__ G)
{
    constexpr int P = 1 << LG, T = Geo<P>::T, F = Geo<P>::F;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *A = sm + f * P, *B = sm + (F + f) * P;
    const int64_t gi = (int64_t)blockIdx.x * F + f;    // transform = (output, block)
    const bool active = gi < total;
    const int64_t o = active ? gi / n_blocks : 0;
    const int64_t t = active ? gi % n_blocks : 0;
    const int64_t start = (t_first + t - 1) * (int64_t)L;
    const float *go = g + o * g_stride;
    const float scale = 1.0f / (float)P;               // 1 / 2L
    auto src = [&](int n) {
        const int64_t i0 = start + n;
        const float a = (i0 >= 0 && i0 < g_len) ? __ldg(go + i0) : 0.f;
        const float b = (i0 + 1 >= 0 && i0 + 1 < g_len) ? __ldg(go + i0 + 1) : 0.f;
        return make_float2(a * scale, b * scale);
    };
    float2 *Go = G + gi * P;
    forward_block<P, true>(A, B, j, active, src, rot, post, tw, [&](int k, float2 v) {
        if (active) Go[k] = v;
    });
}

// Offline inverse (Eq. 8) and overlap-add (Eqs. 9-12). A transform's T
// threads own one segment of seg output hops of one output and run its blocks
// in order, from the three blocks before the segment (whose 4L outputs reach
// into it) to its last one; thread j keeps the pending sums of the sample
// pairs r = j + T q (q < 12) of the next three hops in registers (the pairs a
// block gives it: a hop moves a pair by P/4 = 4T, q by 4). A hop's samples are
// final, and written, after the block that starts there: pending (the earlier
// blocks, added in increasing block order) plus that block's first L samples,
// the same summation order as adding the blocks one after another.
template <int LG>
__global__ void __launch_bounds__(Lane<(1 << LG)>::THREADS, 2)
k_inverse_ola(const float2 *__restrict__ Y, int n_blocks, int L, int seg, int n_seg,
              float *__restrict__ y, int64_t out_len, int64_t y_stride,
              const float2 *__restrict__ rot, const float2 *__restrict__ post,
              const float2 *__restrict__ tw, Ragged rg, int n_outputs)
{
    constexpr int P = 1 << LG, T = Lane<P>::T;
    const int F = blockDim.x / T;                      // transforms per CTA (launch's choice)
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *buf = sm + f * lane_buf(P);
    const int64_t unit = (int64_t)blockIdx.x * F + f;  // (output, segment)
    bool on = unit < (int64_t)n_seg * n_outputs;
    const int o = on ? (int)(unit / n_seg) : 0;
    const int64_t tile0 = on ? (unit % n_seg) * seg : 0;   // first output hop of the segment
    const int64_t s0 = tile0 * L;
    int64_t olen = out_len;
    int64_t nb_o = n_blocks;
    if (on && rg.out_len) {                            // ragged: this output's length
        const int64_t oc = rg.out_len[o];
        if (oc < olen) olen = oc < 0 ? 0 : oc;
        nb_o = blocks_of(olen, L);
    }
    on = on && s0 < olen;
    // a transform without a segment still takes part in its warp's barriers
    if constexpr (T > 32) {
        if (!on) return;                               // its barrier holds its threads only
    } else {
        if (!__any_sync(0xffffffffu, on)) return;      // the whole warp has nothing to do
    }
    const int64_t s_end = s0 + (int64_t)seg * L;
    const int64_t w_end = s_end < olen ? s_end : olen; // samples this segment writes
    const float2 *Yo = Y + (int64_t)o * n_blocks * P;
    float *yo = y + (int64_t)o * y_stride;
    const bool pairs = (reinterpret_cast<uintptr_t>(yo) & 7) == 0;
    const bool pf = (reinterpret_cast<uintptr_t>(Yo) & 15) == 0;
    const int64_t t_lo = tile0 - 2 > 0 ? tile0 - 2 : 0;
    int64_t t_hi = tile0 + seg;
    if (t_hi > nb_o - 1) t_hi = nb_o - 1;
    if (!on) t_hi = t_lo - 1;                          // no blocks, barriers only below
    float2 pend[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) pend[c][i] = make_float2(0.f, 0.f);
    // every transform of a warp runs the same number of blocks (barriers)
    int64_t n_run = t_hi - t_lo + 1;
    if constexpr (T < 32) {
        int64_t mx = n_run;
#pragma unroll
        for (int d = T; d < 32; d *= 2) {
            const int64_t other = __shfl_xor_sync(0xffffffffu, mx, d);
            mx = other > mx ? other : mx;
        }
        n_run = mx;
    }
    for (int64_t it = 0; it < n_run; ++it) {
        const int64_t t = t_lo + it;
        const bool act = on && t <= t_hi;
        const float2 *Yt = Yo + (act ? t : 0) * P;
        // the next block's spectrum moves to L2 while this one is transformed
        // (a bulk prefetch wants a 16-byte aligned source: Y's rows are 8P bytes)
        if (j == 0 && act && t < t_hi && pf)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Yt + P), "r"(P * 8) : "memory");
        // hop t - 1 (block l = t - 1 starts at sample l*L) is final after this
        // block: pending + the block's first hop; the other hops add to pending
        const int64_t n0 = (t - 1) * (int64_t)L;
        inverse_lane<P>(buf, j, f, [&](int k) { return act ? __ldg(Yt + k) : make_float2(0.f, 0.f); },
                        rot, post, tw, [&](int q, float2 v) {
            const int c = q >> 2, i = q & 3;
            if (c == 0) {
                const float2 fin = cadd(pend[0][i], v);
                const int64_t n = n0 + 2 * (j + T * i);
                if (!act) return;
                if (n >= s0 && n + 1 < w_end && pairs) {
                    *reinterpret_cast<float2 *>(yo + n) = fin;
                } else {
                    if (n >= s0 && n < w_end) yo[n] = fin.x;
                    if (n + 1 >= s0 && n + 1 < w_end) yo[n + 1] = fin.y;
                }
            } else if (c == 1) {
                pend[0][i] = cadd(pend[1][i], v);
            } else if (c == 2) {
                pend[1][i] = cadd(pend[2][i], v);
            } else {
                pend[2][i] = v;
            }
        });
    }
}

// Adjoint of Eqs. 1, 3, 5 for the input: dx[c][s] += sum over blocks q of the
// range with 0 <= n = s - (q-1)L < 2L of w(n) * Re sum_{k<2L} dX_q(k) e^{+i pi n (2k+1)/4L}.
// The inverse transform below gives (1/2L) Re sum_k ..., so the 2L and the 1/P
// of the inverse cancel. CTA (segment, channel) owns samples [s0, s0 + seg*L),
// reached by blocks q = s0/L .. s0/L + seg; contributions are added in
// increasing q to the value dx already holds.
template <int LG>
__global__ void __launch_bounds__(Geo<(1 << LG)>::THREADS)
k_adjoint_input(const float2 *__restrict__ dX, int q_count, int64_t q_first, int L, int seg,
                float *__restrict__ dx, int64_t N, int64_t x_stride, const float *__restrict__ win,
                const float2 *__restrict__ rot, const float2 *__restrict__ post,
                const float2 *__restrict__ tw)
{
    constexpr int P = 1 << LG, T = Geo<P>::T, F = Geo<P>::F;
    extern __shared__ float2 sm[];
    float *acc = reinterpret_cast<float *>(sm + 2 * F * P);
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *A = sm + f * P, *B = sm + (F + f) * P;
    const int c = blockIdx.y;
    // blocks q of the range reach samples [(q_first - 1)L, (q_first + q_count)L)
    const int64_t tile_base = q_first > 0 ? (q_first - 1) / seg : 0;
    const int64_t tile0 = (tile_base + blockIdx.x) * seg;
    const int64_t s0 = tile0 * L;
    const int nseg = seg * L;
    float *xo = dx + (int64_t)c * x_stride;
    for (int i = threadIdx.x; i < nseg; i += blockDim.x) acc[i] = (s0 + i < N) ? xo[s0 + i] : 0.f;
    const float2 *dXc = dX + (int64_t)c * q_count * P;
    int64_t q_lo = tile0, q_hi = tile0 + seg;             // blocks reaching the segment
    if (q_lo < q_first) q_lo = q_first;
    if (q_hi > q_first + q_count - 1) q_hi = q_first + q_count - 1;
    for (int64_t qb = q_lo; qb <= q_hi; qb += F) {
        const int64_t q = qb + f;
        const bool active = q <= q_hi;
        const float2 *Xq = dXc + (active ? q - q_first : 0) * P;
        merge_inverse<P>(A, j, post, [&](int k) {
            return active ? Xq[k] : make_float2(0.f, 0.f);
        });
        __syncthreads();
        float2 *Z = fft_complex<P, true>(A, B, j, tw, [&](int r, float2 v) {
            return cmulc(v, __ldg(rot + r));
        });
        const float2 *Zbase = Z - f * P;
        const int64_t w0 = (qb - 1) * L;                 // first sample of block qb
        const int span = (F + 1) * L;
        for (int p = threadIdx.x; p < span; p += blockDim.x) {
            const int64_t a = w0 + p - s0;
            if (a < 0 || a >= nseg) continue;
            float v = acc[a];
            for (int ff = 0; ff < F; ++ff) {
                if (qb + ff > q_hi) break;
                const int n = p - ff * L;                // position within block qb+ff
                if (n >= 0 && n < 2 * L)
                    v = fmaf(__ldg(win + n), reinterpret_cast<const float *>(Zbase + ff * P)[n], v);
            }
            acc[a] = v;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < nseg; i += blockDim.x)
        if (s0 + i < N) xo[s0 + i] = acc[i];
}

// Streaming forward: one block per input channel from the L samples of
// history and the L new samples; spectrum into delay-line slot tick mod 2M.
template <int LG>
__global__ void __launch_bounds__(Geo<(1 << LG)>::THREADS)
k_forward_stream(const float *__restrict__ in, float *__restrict__ hist, int L, int n_in, int R,
                 int slot, const float *__restrict__ win, const float2 *__restrict__ rot,
                 const float2 *__restrict__ post, const float2 *__restrict__ tw,
                 float2 *__restrict__ ring)
{
    constexpr int P = 1 << LG, T = Geo<P>::T, F = Geo<P>::F;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *A = sm + f * P, *B = sm + (F + f) * P;
    const int c = blockIdx.x * F + f;
    const bool active = c < n_in;
    const float *hc = hist + (int64_t)(active ? c : 0) * L;
    const float *ic = in + (int64_t)(active ? c : 0) * L;
    // the history rows are 8-byte aligned; the caller's input may not be
    const bool pairs = (reinterpret_cast<uintptr_t>(ic) & 7) == 0;
    auto src = [&](int n) {       // n even, so n and n + 1 lie on the same side of L
        const float *p = (n < L) ? (hc + n) : (ic + n - L);
        const float2 v = (n < L || pairs) ? *reinterpret_cast<const float2 *>(p)
                                          : make_float2(p[0], p[1]);
        const float2 w = __ldg(reinterpret_cast<const float2 *>(win) + (n >> 1));
        return make_float2(v.x * w.x, v.y * w.y);
    };
    float2 *Xo = ring + ((int64_t)(active ? c : 0) * R + slot) * P;
    forward_block<P>(A, B, j, active, src, rot, post, tw, [&](int k, float2 v) {
        if (active) Xo[k] = v;
    });
    // history reads happened before the first barrier inside forward_block
    if (active) {
        float *hw = hist + (int64_t)c * L;
        for (int i = j; i < L; i += T) hw[i] = ic[i];
    }
}

// Streaming inverse: output block -> L samples, with the 3L pending sums st of
// the output. Thread j owns the sample pairs 2 (j + T i) + {0, 1}, i < 4, of
// each hop of the frame, and so the same positions of the pending sums: it
// reads its 12 pending pairs, adds this block's contributions in hop order and
// writes its output pairs and new pending pairs (the offline kernel's order).
template <int LG>
__global__ void __launch_bounds__(Lane<(1 << LG)>::THREADS)
k_inverse_stream(const float2 *__restrict__ Ys, float *__restrict__ ola, float *__restrict__ out,
                 int L, int n_out, const float2 *__restrict__ rot, const float2 *__restrict__ post,
                 const float2 *__restrict__ tw)
{
    constexpr int P = 1 << LG, T = Lane<P>::T;
    const int F = blockDim.x / T;
    extern __shared__ float2 sm[];
    const int f = threadIdx.x / T, j = threadIdx.x % T;
    float2 *buf = sm + f * lane_buf(P);
    const int o = blockIdx.x * F + f;
    const bool active = o < n_out;
    const float2 *Yo = Ys + (int64_t)(active ? o : 0) * P;
    float *st = ola + (int64_t)(active ? o : 0) * 3 * L;
    float *ou = out + (int64_t)(active ? o : 0) * L;
    const bool pairs = (reinterpret_cast<uintptr_t>(ou) & 7) == 0;
    float2 pend[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            pend[c][i] = active ? *reinterpret_cast<const float2 *>(st + c * L + 2 * (j + T * i))
                                : make_float2(0.f, 0.f);
    inverse_lane<P>(buf, j, f, [&](int k) { return active ? Yo[k] : make_float2(0.f, 0.f); }, rot,
                    post, tw, [&](int q, float2 v) {
        const int c = q >> 2, i = q & 3;
        if (c == 0) {
            const float2 fin = cadd(pend[0][i], v);
            const int n = 2 * (j + T * i);
            if (active) {
                if (pairs) {
                    *reinterpret_cast<float2 *>(ou + n) = fin;
                } else {
                    ou[n] = fin.x;
                    ou[n + 1] = fin.y;
                }
            }
        } else if (c == 1) {
            pend[0][i] = cadd(pend[1][i], v);
        } else if (c == 2) {
            pend[1][i] = cadd(pend[2][i], v);
        } else {
            pend[2][i] = v;
        }
    });
    if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<float2 *>(st + c * L + 2 * (j + T * i)) = pend[c][i];
    }
}

// Output hops per segment of the offline inverse. Each segment also
// transforms the three blocks before it, so long segments waste less; the
// segments of all outputs should fill one wave of the resident transform
// groups (groups = SMs x resident CTAs x transforms per CTA) and no more,
// since a second, partial wave would run nearly alone.
int64_t ola_seg(int64_t hops_per_output, int n_outputs, int64_t groups)
{
    int64_t per_out = groups / (n_outputs > 0 ? n_outputs : 1);
    if (per_out < 1) per_out = 1;
    int64_t seg = (hops_per_output + per_out - 1) / per_out;
    if (seg < 5) seg = 5;                              // at most 3 extra blocks per 5
    return seg;
}

// Segment length (output hops per CTA) of the input adjoint.
int inverse_seg(int L)
{
    int seg = 12288 / L - 3;            // about 48 KB of accumulator
    if (seg > 29) seg = 29;
    if (seg < 4) seg = 4;
    return seg;
}

// Frequency-domain mixdown: by linearity of Eq. 8 and of the overlap-add of
// Eqs. 9-12, one inverse transform of the sum of several outputs' spectra
// equals the sum of their outputs. Thread i of the grid-stride loop takes bin
// pair i of mix output e and adds the members' values in increasing output
// order (two bins per 16-byte load).
__global__ void __launch_bounds__(256)
k_mix_spectra(const float4 *__restrict__ Y, float4 *__restrict__ Ymix, int64_t per_out, int n_mix,
              const int32_t *__restrict__ off, const int32_t *__restrict__ members)
{
    const int64_t total = per_out * n_mix;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i / per_out);
        const int64_t r = i - (int64_t)e * per_out;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int m = __ldg(off + e), m_end = __ldg(off + e + 1); m < m_end; ++m) {
            const float4 v = __ldg(Y + (int64_t)__ldg(members + m) * per_out + r);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        Ymix[i] = acc;
    }
}

}  // namespace

cudaError_t launch_tables(tvolap_plan *h)
{
    k_tables<<<(h->P + 255) / 256, 256, 0, h->stream>>>(h->tw, h->rot, h->post, h->win, h->L);
    return cudaGetLastError();
}


cudaError_t launch_forward_signal(tvolap_plan *h, const float *x, int64_t N, int64_t x_stride,
                                  int n_blocks, float2 *X)
{
    return launch_block_spectra(h, x, N, x_stride, 0, n_blocks, X);
}

cudaError_t launch_block_spectra(tvolap_plan *h, const float *x, int64_t N, int64_t x_stride,
                                 int64_t t_first, int n_blocks, float2 *X, Ragged rg)
{
    const int64_t total = (int64_t)h->n_in * n_blocks;
    if (total == 0) return cudaSuccess;
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const int th = lane_threads<P>(h->xform_threads), F = th / Lane<P>::T;
        const int64_t grid = (total + F - 1) / F;
        const size_t sm = smem_lane<LG>(th);
        cudaError_t e = set_smem(k_forward_signal<LG>, smem_lane<LG>(Lane<P>::THREADS));
        if (e != cudaSuccess) return e;
        k_forward_signal<LG><<<(unsigned)grid, th, sm, h->stream>>>(
            x, N, x_stride, h->L, n_blocks, total, h->win, h->rot, h->post, h->tw, X, t_first, rg);
    });
    return cudaGetLastError();
}

cudaError_t launch_bank(tvolap_plan *h, int first_slot, int count, const float *ir, int ir_len,
                        int64_t ir_stride)
{
    const int64_t total = (int64_t)count * h->M;
    if (total == 0) return cudaSuccess;
    float2 *dst = h->bank + (int64_t)first_slot * h->M * h->P;
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const int th = lane_threads<P>(h->xform_threads), F = th / Lane<P>::T;
        const int64_t grid = (total + F - 1) / F;
        const size_t sm = smem_lane<LG>(th);
        cudaError_t e = set_smem(k_bank<LG>, smem_lane<LG>(Lane<P>::THREADS));
        if (e != cudaSuccess) return e;
        k_bank<LG><<<(unsigned)grid, th, sm, h->stream>>>(
            ir, ir_len, ir_stride, h->M, h->L, total, h->rot, h->post, h->tw, dst);
    });
    return cudaGetLastError();
}

cudaError_t launch_tables_raw(float2 *tw, float2 *rot, float2 *post, float *win, int L,
                              cudaStream_t st)
{
    k_tables<<<(2 * L + 255) / 256, 256, 0, st>>>(tw, rot, post, win, L);
    return cudaGetLastError();
}

cudaError_t launch_bank_raw(int lgP, int L, int M, int64_t count, const float *ir, int ir_len,
                            int64_t ir_stride, const float2 *rot, const float2 *post,
                            const float2 *tw, float2 *dst, cudaStream_t st)
{
    const int64_t total = count * M;
    if (total == 0) return cudaSuccess;
    TVOLAP_DISPATCH(lgP, {
        constexpr int P = 1 << LG;
        const int64_t grid = (total + Lane<P>::F - 1) / Lane<P>::F;
        const size_t sm = smem_lane<LG>(Lane<P>::THREADS);
        cudaError_t e = set_smem(k_bank<LG>, sm);
        if (e != cudaSuccess) return e;
        k_bank<LG><<<(unsigned)grid, Lane<P>::THREADS, sm, st>>>(ir, ir_len, ir_stride, M, L, total,
                                                              rot, post, tw, dst);
    });
    return cudaGetLastError();
}

cudaError_t launch_inverse_ola(tvolap_plan *h, const float2 *Y, int n_blocks, float *y,
                               int64_t out_len, int64_t y_stride, Ragged rg, int n_outputs)
{
    if (out_len <= 0) return cudaSuccess;
    if (n_outputs < 0) n_outputs = h->n_out;
    if (n_outputs == 0) return cudaSuccess;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const int th = lane_threads<P>(h->xform_threads), F = th / Lane<P>::T;
        const size_t sm = smem_lane<LG>(th);
        cudaError_t e = set_smem(k_inverse_ola<LG>, smem_lane<LG>(Lane<P>::THREADS));
        if (e != cudaSuccess) return e;
        static int per_sm[3] = {0, 0, 0};              // resident CTAs per launch size
        const int slot = th == 64 ? 0 : th == 128 ? 1 : 2;
        if (per_sm[slot] == 0) {
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_inverse_ola<LG>, th, sm);
            if (e != cudaSuccess) return e;
            per_sm[slot] = n > 0 ? n : 1;
        }
        const int64_t seg = ola_seg((out_len + h->L - 1) / h->L, n_outputs,
                                    (int64_t)sms * per_sm[slot] * F);
        if (seg > 0x7fffffffLL / h->L) return cudaErrorInvalidValue;
        const int64_t n_seg = (out_len + seg * h->L - 1) / (seg * h->L);
        if (n_seg * n_outputs > 0x7fffffffLL) return cudaErrorInvalidValue;
        const int64_t units = n_seg * n_outputs;
        const int64_t grid = (units + F - 1) / F;
        k_inverse_ola<LG><<<(unsigned)grid, th, sm, h->stream>>>(
            Y, n_blocks, h->L, (int)seg, (int)n_seg, y, out_len, y_stride, h->rot, h->post, h->tw,
            rg, n_outputs);
    });
    return cudaGetLastError();
}

cudaError_t launch_adjoint_output(tvolap_plan *h, const float *g, int64_t g_len, int64_t g_stride,
                                  int64_t t_first, int n_blocks, float2 *G)
{
    const int64_t total = (int64_t)h->n_out * n_blocks;
    if (total == 0) return cudaSuccess;
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const int64_t grid = (total + Geo<P>::F - 1) / Geo<P>::F;
        const size_t sm = smem_fft<LG>();
        cudaError_t e = set_smem(k_adjoint_output<LG>, sm);
        if (e != cudaSuccess) return e;
        k_adjoint_output<LG><<<(unsigned)grid, Geo<P>::THREADS, sm, h->stream>>>(
            g, g_len, g_stride, h->L, n_blocks, total, t_first, h->rot, h->post, h->tw, G);
    });
    return cudaGetLastError();
}

cudaError_t launch_adjoint_input(tvolap_plan *h, const float2 *dX, int64_t q_first, int q_count,
                                 float *dx, int64_t N, int64_t x_stride)
{
    if (N <= 0 || q_count <= 0) return cudaSuccess;
    const int seg = inverse_seg(h->L);
    // output hops (of L samples) the blocks of the range reach, in units of seg
    const int64_t hop_lo = q_first > 0 ? q_first - 1 : 0;
    int64_t hop_hi = q_first + q_count;                   // exclusive
    const int64_t n_hops = (N + h->L - 1) / h->L;
    if (hop_hi > n_hops) hop_hi = n_hops;
    if (hop_hi <= hop_lo) return cudaSuccess;
    const int64_t n_seg = (hop_hi - 1) / seg - hop_lo / seg + 1;
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const size_t sm = smem_fft<LG>() + (size_t)seg * h->L * sizeof(float);
        cudaError_t e = set_smem(k_adjoint_input<LG>, sm);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)n_seg, (unsigned)h->n_in);
        k_adjoint_input<LG><<<grid, Geo<P>::THREADS, sm, h->stream>>>(
            dX, q_count, q_first, h->L, seg, dx, N, x_stride, h->win, h->rot, h->post, h->tw);
    });
    return cudaGetLastError();
}

cudaError_t launch_forward_stream(tvolap_plan *h, const float *in)
{
    const int R = 2 * h->M;
    const int slot = (int)(h->tick % R);
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        const int grid = (h->n_in + Geo<P>::F - 1) / Geo<P>::F;
        const size_t sm = smem_fft<LG>();
        cudaError_t e = set_smem(k_forward_stream<LG>, sm);
        if (e != cudaSuccess) return e;
        k_forward_stream<LG><<<grid, Geo<P>::THREADS, sm, h->stream>>>(
            in, h->hist, h->L, h->n_in, R, slot, h->win, h->rot, h->post, h->tw, h->ring);
    });
    return cudaGetLastError();
}

cudaError_t launch_inverse_stream(tvolap_plan *h, float *out, const float2 *Ys, float *ola,
                                  int n_outputs)
{
    if (!Ys) Ys = h->Ystream;
    if (!ola) ola = h->ola;
    if (n_outputs < 0) n_outputs = h->n_out;
    if (n_outputs == 0) return cudaSuccess;
    TVOLAP_DISPATCH(h->lgP, {
        constexpr int P = 1 << LG;
        constexpr int TH = Lane<P>::T < 32 ? 32 : Lane<P>::T, F = TH / Lane<P>::T;
        const int grid = (n_outputs + F - 1) / F;
        const size_t sm = smem_lane<LG>(TH);
        cudaError_t e = set_smem(k_inverse_stream<LG>, sm);
        if (e != cudaSuccess) return e;
        k_inverse_stream<LG><<<grid, TH, sm, h->stream>>>(
            Ys, ola, out, h->L, n_outputs, h->rot, h->post, h->tw);
    });
    return cudaGetLastError();
}

cudaError_t launch_mix_spectra(tvolap_plan *h, const float2 *Y, int n_blocks, float2 *Ymix)
{
    const int64_t per_out = (int64_t)n_blocks * h->P / 2;      // bin pairs of one output
    const int64_t total = per_out * h->n_mix;
    if (total == 0) return cudaSuccess;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    int64_t grid = (total + 255) / 256;
    if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
    k_mix_spectra<<<(unsigned)grid, 256, 0, h->stream>>>(reinterpret_cast<const float4 *>(Y),
                                                         reinterpret_cast<float4 *>(Ymix), per_out,
                                                         h->n_mix, h->mix_off, h->mix_members);
    return cudaGetLastError();
}

}  // namespace tvolap

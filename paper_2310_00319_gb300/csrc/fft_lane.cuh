// Transforms with sixteen values per thread (sm_103a), for the offline
// forward transform, the partition bank and the offline inverse with its
// overlap-add.
//
// The arithmetic is that of fft_core.cuh: a real block of 4L samples whose
// upper half is zero (Eqs. 3-4) goes through a P = 2L point complex Stockham
// FFT of z(r) = x(2r) + i x(2r+1) pre-rotated by e^{-i pi r/P}, radix 8 while
// three or more bits remain, then one radix-4 or radix-2 stage, and a split
// step gives the P half-bin spectrum values; the inverse runs it backwards.
// What differs is the work split: T = P/16 threads run one transform (one
// warp at P = 512), each thread holding sixteen values, and the butterflies a
// thread runs are chosen so that
//   * the first stage runs on the registers the inputs were loaded into;
//   * in the forward transform the last stage leaves Z(k) and Z(P-1-k) in the
//     same thread, so the split step needs no shared-memory pass and each
//     thread stores its spectrum values straight to memory;
//   * in the inverse the merge step (the split's inverse) runs on the values
//     a thread loads, and the last stage leaves each thread the output pairs
//     r = j + T q (q < 16), a set that a hop of L samples (P/4 pairs) maps
//     onto itself, so the overlap-add of consecutive blocks runs on registers.
// Twiddles come from one table load per butterfly (the stage's first row)
// raised to the needed powers; rotations and split factors from one table
// load times the constants e^{-i pi k/16}. Threads of a transform wait for
// each other with __syncwarp when the transform fits in a warp, else on a
// named barrier of its T threads.
#pragma once

#include "fft_core.cuh"

namespace tvolap {

template <int P>
struct Lane {
    static_assert(P >= 32 && P <= 2048, "transform size");
    static constexpr int T = P / 16;                 // threads per transform
    static constexpr int THREADS = 256;
    static constexpr int F = THREADS / T;            // transforms per CTA
    static constexpr int S = 2 * T;                  // first-stage butterflies (P / 8)
};

// e^{-i pi k / 16}, k < 16
__device__ __forceinline__ float2 c16(int k)
{
    constexpr float re[16] = {1.0f, 0.98078525066375732f, 0.92387950420379639f, 0.83146959543228149f,
                              0.70710676908493042f, 0.55557024478912354f, 0.38268342614173889f,
                              0.19509032368659973f, 0.0f, -0.19509032368659973f,
                              -0.38268342614173889f, -0.55557024478912354f, -0.70710676908493042f,
                              -0.83146959543228149f, -0.92387950420379639f, -0.98078525066375732f};
    constexpr float im[16] = {-0.0f, -0.19509032368659973f, -0.38268342614173889f,
                              -0.55557024478912354f, -0.70710676908493042f, -0.83146959543228149f,
                              -0.92387950420379639f, -0.98078525066375732f, -1.0f,
                              -0.98078525066375732f, -0.92387950420379639f, -0.83146959543228149f,
                              -0.70710676908493042f, -0.55557024478912354f, -0.38268342614173889f,
                              -0.19509032368659973f};
    return make_float2(re[k], im[k]);
}

// Buffer layouts (a transform's P values in lane_buf(P) slots). Every array
// between two stages is written once and read once, each in its own layout,
// chosen so that a half warp's 64-bit accesses fall on 16 different positions
// for both its writer and its reader:
//   * layout A, the first stage's output (written as rows of eight consecutive
//     values 8b + s, read as 16 consecutive values per half warp): one unused
//     slot after every 16 values, pa(n) = n + n/16;
//   * layout B, a middle stage's output (written as two groups of eight values
//     64 apart, read as 16 consecutive values): bit 3 flipped where bit 6 is
//     set, pb(n) = n ^ ((n >> 3) & 8), a permutation within each 16 values.
// For the common strides, every offset a thread uses within a stage is one or
// two runtime bases plus compile-time constants.
__host__ __device__ constexpr int lane_buf(int P) { return P + P / 16; }
__device__ __forceinline__ int pa(int n) { return n + (n >> 4); }
__device__ __forceinline__ int pb(int n) { return n ^ ((n >> 3) & 8); }

// Dynamic shared memory of a lane kernel of `threads` threads: one buffer per
// transform.
template <int LG>
inline size_t smem_lane(int threads)
{
    return (size_t)(threads / Lane<(1 << LG)>::T) * lane_buf(1 << LG) * sizeof(float2);
}

// Threads of a lane kernel's CTA for the plan option (0: the default 256), at
// least one transform's T threads: 64, 128 or 256.
template <int P>
inline int lane_threads(int option)
{
    int th = option == 64 || option == 128 ? option : Lane<P>::THREADS;
    return th < Lane<P>::T ? Lane<P>::T : th;
}

// dft8 (forward) of v[0..3] with v[4..7] zero: the first radix-2 layer of the
// even/odd split reduces to copies. Same values as dft8 on zero-padded inputs
// up to the sign of zero.
__device__ __forceinline__ void dft8_half(float2 *v)
{
    const float h = 0.70710678118654752440f;
    // even half e = DFT4(v0, v2, 0, 0), odd half o = DFT4(v1, v3, 0, 0)
    const float2 e0 = cadd(v[0], v[2]), e2 = csub(v[0], v[2]);
    const float2 e1 = make_float2(v[0].x + v[2].y, v[0].y - v[2].x);   // v0 - i v2
    const float2 e3 = make_float2(v[0].x - v[2].y, v[0].y + v[2].x);   // v0 + i v2
    float2 o0 = cadd(v[1], v[3]), o2 = csub(v[1], v[3]);
    float2 o1 = make_float2(v[1].x + v[3].y, v[1].y - v[3].x);
    float2 o3 = make_float2(v[1].x - v[3].y, v[1].y + v[3].x);
    o1 = cmul(o1, make_float2(h, -h));
    o2 = make_float2(o2.y, -o2.x);                                      // -i o2
    o3 = cmul(o3, make_float2(-h, -h));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// Wait for the T threads of transform f.
template <int T>
__device__ __forceinline__ void lane_sync(int f)
{
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(f + 1), "r"(T) : "memory");
    }
}

// Radix of the stage at Ns (as fft_core.cuh: 8 while P/Ns >= 8).
template <int P, int Ns>
struct LStage {
    static constexpr int R = stage_radix(P, Ns);
    static constexpr bool LAST = Ns * R == P;
    static constexpr int NB = 16 / R;                // butterflies per thread
};

// w[r] = w1^r, r < R (w[0] = 1)
template <int R>
__device__ __forceinline__ void powers(float2 w1, float2 (&w)[R])
{
    w[0] = make_float2(1.f, 0.f);
    if constexpr (R > 1) w[1] = w1;
    if constexpr (R > 2) w[2] = cmul(w1, w1);
    if constexpr (R > 3) w[3] = cmul(w[2], w1);
    if constexpr (R > 4) {
        w[4] = cmul(w[2], w[2]);
        w[5] = cmul(w[4], w1);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
    }
}

// The R inputs of butterfly b of stage (Ns, R) from the buffer (layout A
// after the first stage, B after a middle one).
template <int P, int Ns>
__device__ __forceinline__ void lane_load(const float2 *buf, int b, float2 (&v)[LStage<P, Ns>::R])
{
    constexpr int R = LStage<P, Ns>::R, stride = P / R;
    if constexpr (Ns == 8) {                           // input in layout A
        if constexpr (stride % 16 == 0) {
            const float2 *bp = buf + pa(b);            // pa(b + 16k) = pa(b) + 17k
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = bp[r * stride / 16 * 17];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = buf[pa(b + r * stride)];
        }
    } else {                                           // input in layout B
        if constexpr (stride % 64 == 0) {
            // pb(b + 64k) = pb(b) ^ (8 (k mod 2)) + 64k
            const int b0 = pb(b), b1 = b0 ^ 8;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = buf[((r * stride / 64) & 1 ? b1 : b0) + r * stride];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = buf[pb(b + r * stride)];
        }
    }
}

// The stage's twiddles w[r] = e^{-2 pi i r k / (Ns R)} of butterfly index k = b mod Ns.
template <int P, int Ns>
__device__ __forceinline__ void lane_twiddles(int b, const float2 *__restrict__ tw,
                                              float2 (&w)[LStage<P, Ns>::R])
{
    powers<LStage<P, Ns>::R>(__ldg(tw + tw_offset(P, Ns) + (b & (Ns - 1))), w);
}

// Butterfly v (inputs loaded) rotated by the twiddles w, transformed.
template <int P, int Ns, bool INV>
__device__ __forceinline__ void lane_apply(float2 (&v)[LStage<P, Ns>::R],
                                           const float2 (&w)[LStage<P, Ns>::R])
{
    constexpr int R = LStage<P, Ns>::R;
    if constexpr (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = INV ? cmulc(v[r], w[r]) : cmul(v[r], w[r]);
    }
    dftR<R, INV>(v);
}

// Butterfly b of stage (Ns, R): loaded, rotated by its twiddles, transformed.
template <int P, int Ns, bool INV>
__device__ __forceinline__ void lane_bfly(const float2 *buf, int b, const float2 *__restrict__ tw,
                                          float2 (&v)[LStage<P, Ns>::R])
{
    constexpr int R = LStage<P, Ns>::R;
    lane_load<P, Ns>(buf, b, v);
    float2 w[R];
    if constexpr (Ns > 1) lane_twiddles<P, Ns>(b, tw, w);
    lane_apply<P, Ns, INV>(v, w);
}

// Outputs of butterfly b of a non-last stage: the first stage's in layout A,
// a middle stage's in layout B.
template <int P, int Ns>
__device__ __forceinline__ void lane_store(float2 *buf, int b, const float2 (&v)[LStage<P, Ns>::R])
{
    constexpr int R = LStage<P, Ns>::R;
    const int base = (b / Ns) * Ns * R + (b & (Ns - 1));
    if constexpr (Ns == 1) {
        float2 *bp = buf + 8 * b + (b >> 1);           // pa(8 b + s) = 8 b + b/2 + s, s < 8 = R
#pragma unroll
        for (int s = 0; s < R; ++s) bp[s] = v[s];
    } else if constexpr (Ns == 8) {
        // base + 8 s keeps base's bit 6: pb flips bit 3 of 8 s, i.e. +-8
        const int m = (base >> 3) & 8;
#pragma unroll
        for (int s = 0; s < R; ++s) buf[(s & 1 ? base - m : base + m) + s * Ns] = v[s];
    } else if constexpr (Ns % 64 == 0) {
        // bit 6 of base + s Ns is bit 6 of base xor bit 0 of s Ns / 64
        const int b0 = pb(base), b1 = b0 ^ 8;
#pragma unroll
        for (int s = 0; s < R; ++s) buf[((s * Ns / 64) & 1 ? b1 : b0) + s * Ns] = v[s];
    } else {
#pragma unroll
        for (int s = 0; s < R; ++s) buf[pb(base + s * Ns)] = v[s];
    }
}

// Middle stages (neither the first nor the last): butterflies b = j + T u.
// Enters with the stage's input in buf (synchronised) and leaves with its
// output there (synchronised).
template <int P, int Ns, bool INV>
__device__ __forceinline__ void lane_middle(float2 *buf, int j, int f, const float2 *__restrict__ tw)
{
    if constexpr (!LStage<P, Ns>::LAST) {
        constexpr int R = LStage<P, Ns>::R, NB = LStage<P, Ns>::NB, T = Lane<P>::T;
        float2 v[NB][R];
        if constexpr (T % Ns == 0) {
            // every butterfly j + T u has the twiddle index j mod Ns: one set for all
            float2 w[R];
            lane_twiddles<P, Ns>(j, tw, w);
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                lane_load<P, Ns>(buf, j + T * u, v[u]);
                lane_apply<P, Ns, INV>(v[u], w);
            }
        } else {
#pragma unroll
            for (int u = 0; u < NB; ++u) lane_bfly<P, Ns, INV>(buf, j + T * u, tw, v[u]);
        }
        lane_sync<T>(f);
#pragma unroll
        for (int u = 0; u < NB; ++u) lane_store<P, Ns>(buf, j + T * u, v[u]);
        lane_sync<T>(f);
        lane_middle<P, Ns * R, INV>(buf, j, f, tw);
    }
}

// Ns of the last stage.
template <int P, int Ns = 1>
__host__ __device__ constexpr int last_ns()
{
    if constexpr (LStage<P, Ns>::LAST) {
        return Ns;
    } else {
        return last_ns<P, Ns * LStage<P, Ns>::R>();
    }
}

// The windowed input pair n (samples 2n, 2n+1 of the block starting at
// sample `start`, Eq. 1 with the half-amplitude Hann window): 8-byte loads
// where the row allows, zero outside [0, N).
struct SignalPairs {
    const float *xc;
    const float *win;
    int64_t start, N;
    bool pairs, inside;   // 8-byte aligned row; and every pair of the block in [0, N)
    __device__ __forceinline__ void set_range(int L)
    {
        inside = pairs && start >= 0 && start + 2 * (int64_t)L <= N;
    }
    __device__ __forceinline__ float2 operator()(int n) const
    {
        const int64_t i0 = start + 2 * n;
        const float2 w = __ldg(reinterpret_cast<const float2 *>(win) + n);
        float2 v;
        if (inside) {                                  // the whole block lies in [0, N)
            v = __ldg(reinterpret_cast<const float2 *>(xc + i0));
        } else if (pairs && i0 >= 0 && i0 + 1 < N) {
            v = __ldg(reinterpret_cast<const float2 *>(xc + i0));
        } else {
            v.x = (i0 >= 0 && i0 < N) ? __ldg(xc + i0) : 0.f;
            v.y = (i0 + 1 >= 0 && i0 + 1 < N) ? __ldg(xc + i0 + 1) : 0.f;
        }
        return __fmul2_rn(v, w);
    }
};

// The inputs a thread's first-stage butterflies (j and S - 1 - j) take from a
// block: z[u][r] = src(bb[u] + S r), r < 4 (the upper half is zero padding);
// src(n) gives the windowed pair (x(2n), x(2n+1)) for n < P/2.
template <int P, class Src>
__device__ __forceinline__ void forward_inputs(int j, bool active, Src src, float2 (&z)[2][4])
{
    constexpr int S = Lane<P>::S;
    const int bb[2] = {j, S - 1 - j};
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) z[u][r] = active ? src(bb[u] + S * r) : make_float2(0.f, 0.f);
}

// The forward transform of one block from its inputs (forward_inputs);
// st(k, v) receives X(k), each k < P exactly once per thread set. The buffer
// holds lane_buf(P) values; on entry it may still be read by
// this transform's threads for an earlier transform (the first barrier covers
// that).
template <int P, bool SYNC_OUT = false, class Store>
__device__ __forceinline__ void forward_lane_z(float2 *buf, int j, int f, bool active,
                                               const float2 (&z)[2][4],
                                               const float2 *__restrict__ rot,
                                               const float2 *__restrict__ post,
                                               const float2 *__restrict__ tw, Store st)
{
    constexpr int T = Lane<P>::T, S = Lane<P>::S;
    // first stage (Ns = 1, radix 8, stride S): butterflies j and S - 1 - j run
    // on this thread's inputs, pre-rotated by rot(n) = rot(b) e^{-i pi r/8}
    const int bb[2] = {j, S - 1 - j};
    float2 v[2][8];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const float2 r0 = active ? __ldg(rot + bb[u]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 4; ++r) v[u][r] = cmul(z[u][r], cmul(r0, c16(2 * r)));
        dft8_half(v[u]);
    }
    lane_sync<T>(f);
#pragma unroll
    for (int u = 0; u < 2; ++u) lane_store<P, 1>(buf, bb[u], v[u]);
    lane_sync<T>(f);
    lane_middle<P, 8, false>(buf, j, f, tw);
    // last stage: butterflies b and Ns - 1 - b hold Z(k) and Z(P - 1 - k)
    constexpr int NS = last_ns<P>(), R = LStage<P, NS>::R, H = LStage<P, NS>::NB / 2;
    float2 lo[H][R], hi[H][R];
#pragma unroll
    for (int u = 0; u < H; ++u) {
        lane_bfly<P, NS, false>(buf, j + T * u, tw, lo[u]);
        lane_bfly<P, NS, false>(buf, NS - 1 - j - T * u, tw, hi[u]);
    }
    // SYNC_OUT: every thread of the transform has read the buffer, so st may
    // write into it
    if constexpr (SYNC_OUT) lane_sync<T>(f);
    // split: for k < P/2 in butterfly b (s < R/2), the partner P - 1 - k is
    // output R - 1 - s of butterfly NS - 1 - b
    const float2 half = make_float2(0.5f, 0.5f);
    auto split = [&](float2 zk, float2 zkk, float2 w, int k) {
        // E = (zk + conj zkk) / 2, d = (zk - conj zkk) / 2 (each lane rounded as
        // the scalar sum, then halved exactly)
        const float2 E = __fmul2_rn(__ffma2_rn(zkk, make_float2(1.f, -1.f), zk), half);
        const float2 d = __fmul2_rn(__ffma2_rn(zkk, make_float2(-1.f, 1.f), zk), half);
        const float2 O = make_float2(d.y, -d.x);           // (zk - conj zkk) / 2i
        const float2 t = cmul(w, O);
        st(k, cadd(E, t));
        st(P - 1 - k, cconj(csub(E, t)));
    };
#pragma unroll
    for (int u = 0; u < H; ++u) {
        const int b = j + T * u, bh = NS - 1 - b;
        const float2 pb = __ldg(post + b), ph = __ldg(post + bh);
#pragma unroll
        for (int s = 0; s < R / 2; ++s) {
            // W^{k + 1/2} for k = b + s NS: post(b) e^{-i pi s / R}
            split(lo[u][s], hi[u][R - 1 - s], cmul(pb, c16(16 / R * s)), b + s * NS);
            split(hi[u][s], lo[u][R - 1 - s], cmul(ph, c16(16 / R * s)), bh + s * NS);
        }
    }
}

// The forward transform of one block whose inputs src(n) gives (as
// forward_inputs), loaded and transformed in one go.
template <int P, bool SYNC_OUT = false, class Src, class Store>
__device__ __forceinline__ void forward_lane(float2 *buf, int j, int f, bool active, Src src,
                                             const float2 *__restrict__ rot,
                                             const float2 *__restrict__ post,
                                             const float2 *__restrict__ tw, Store st)
{
    float2 z[2][4];
    forward_inputs<P>(j, active, src, z);
    forward_lane_z<P, SYNC_OUT>(buf, j, f, active, z, rot, post, tw, st);
}

// The inverse transform of one block, its rotation undone and scaled by 1/P:
// ld(k) gives Y(k); emit(q, v) receives v = (y(2r), y(2r+1)) for the pairs
// r = j + T q, q < 16, with q / 4 increasing for each q mod 4 (the order the
// overlap-add needs). Buffer as forward_lane.
template <int P, class Load, class Emit>
__device__ __forceinline__ void inverse_lane(float2 *buf, int j, int f, Load ld,
                                             const float2 *__restrict__ rot,
                                             const float2 *__restrict__ post,
                                             const float2 *__restrict__ tw, Emit emit)
{
    constexpr int T = Lane<P>::T, S = Lane<P>::S;
    // merge: butterflies j and S - 1 - j of the first stage hold both members
    // of every pair (n, P - 1 - n) of their inputs
    const int bb[2] = {j, S - 1 - j};
    float2 v[2][8];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int r = 0; r < 8; ++r) v[u][r] = ld(bb[u] + S * r);
    const float2 pb[2] = {__ldg(post + bb[0]), __ldg(post + bb[1])};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            // n = bb[u] + S r < P/2, partner P - 1 - n = input 7 - r of the other butterfly
            const float2 yk = v[u][r], ykk = v[1 - u][7 - r];
            const float2 half = make_float2(0.5f, 0.5f);
            const float2 E = __fmul2_rn(__ffma2_rn(ykk, make_float2(1.f, -1.f), yk), half);
            const float2 d = __fmul2_rn(__ffma2_rn(ykk, make_float2(-1.f, 1.f), yk), half);
            const float2 O = cmulc(d, cmul(pb[u], c16(2 * r)));   // post(n) = post(b) e^{-i pi r/8}
            v[u][r] = cadd(E, make_float2(-O.y, O.x));               // E + i O
            v[1 - u][7 - r] = cadd(cconj(E), make_float2(O.y, O.x)); // conj E + i conj O
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) dft8<true>(v[u]);
    lane_sync<T>(f);
#pragma unroll
    for (int u = 0; u < 2; ++u) lane_store<P, 1>(buf, bb[u], v[u]);
    lane_sync<T>(f);
    lane_middle<P, 8, true>(buf, j, f, tw);
    // last stage: butterflies b = j + T u give the pairs r = b + s NS = j + T q,
    // q = u + NB s
    constexpr int NS = last_ns<P>(), R = LStage<P, NS>::R, NB = LStage<P, NS>::NB;
    const float inv_p = 1.0f / (float)P;
    const float2 r0 = __ldg(rot + j);
    // y(2r) + i y(2r+1) = Z(r) e^{+i pi r/P} / P, rot(r) = rot(j) e^{-i pi q/16}
    auto out = [&](int q, float2 z) { return cscale(cmulc(z, cmul(r0, c16(q))), inv_p); };
    if constexpr (R >= 4) {
        // q = u + NB s: for a given q mod 4 (fixed u, NB | 4 or NB = 2), q / 4 grows with s
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            float2 w[R];
            lane_bfly<P, NS, true>(buf, j + T * u, tw, w);
#pragma unroll
            for (int s = 0; s < R; ++s) emit(u + NB * s, out(u + NB * s, w[s]));
        }
    } else {
        // radix 2: a butterfly gives hops q / 4 and q / 4 + 2; emit in q order
        float2 o[16];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            float2 w[R];
            lane_bfly<P, NS, true>(buf, j + T * u, tw, w);
#pragma unroll
            for (int s = 0; s < R; ++s) o[u + NB * s] = out(u + NB * s, w[s]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) emit(q, o[q]);
    }
}

}  // namespace tvolap

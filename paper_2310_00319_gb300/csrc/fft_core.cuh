// Shared-memory FFT building blocks for the TVOLAP kernels (sm_103a).
//
// A real block of 4L samples whose upper half is zero (Eqs. 3-4) is
// transformed through a P = 2L point complex FFT: pairs of samples form one
// complex value z(r) = x(2r) + i x(2r+1), pre-rotated by e^{-i pi r / P}; the
// complex FFT is a Stockham autosort FFT (radix-8 stages, then one radix-4
// or radix-2 stage) with T = P/8 threads per transform exchanging data through
// shared memory; a split step turns the P complex outputs into the P
// half-bin spectrum values X(k), k < P, of the real block:
//     E(k) = (Z(k) + conj Z(P-1-k)) / 2,  O(k) = (Z(k) - conj Z(P-1-k)) / 2i,
//     X(k) = E(k) + W^{k+1/2} O(k),       X(P-1-k) = conj(E(k) - W^{k+1/2} O(k)),
// W = e^{-2 pi i / 4L}. The inverse runs the same steps backwards and
// scales by 1/P, which together with the halves above is the 1/4L of Eq. 8.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tvolap {

// Packed two-lane arithmetic (one instruction for both components, each
// rounded to nearest as the scalar operation would be; a - b as fma(b, -1, a)
// is exactly the rounded difference).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFTs of size 2, 4, 8 (natural order in and out). Forward uses
// e^{-2 pi i rs/R}; INV uses the conjugate kernel (no scaling).
template <bool INV>
__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 *v)
{
    const float h = 0.70710678118654752440f;
    // even / odd halves
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    // twiddles W8^s, s = 0..3 (forward W8 = e^{-i pi/4})
    float2 w1 = INV ? make_float2(h, h) : make_float2(h, -h);
    float2 w3 = INV ? make_float2(-h, h) : make_float2(-h, -h);
    o1 = cmul(o1, w1);
    o2 = mul_mi<INV>(o2);
    o3 = cmul(o3, w3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2 *v)
{
    if constexpr (R == 8) {
        dft8<INV>(v);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else {
        dft2<INV>(v[0], v[1]);
    }
}

// Stages of a P-point transform: Ns = 1, 8, 64, ... with radix 8 while three
// or more bits remain, then one radix-4 or radix-2 stage.
__host__ __device__ constexpr int stage_radix(int P, int Ns) { return P / Ns >= 8 ? 8 : P / Ns; }

// Twiddles are stored stage after stage (stages with Ns > 1), each as rows
// r = 1 .. R-1 of its Ns values: entry tw_offset(P, Ns) + (r - 1) Ns + k holds
// e^{-2 pi i r k / (Ns R)}, so the lanes of a warp (consecutive k) read
// consecutive entries.
__host__ __device__ constexpr int tw_offset(int P, int Ns)
{
    int off = 0;
    for (int n = stage_radix(P, 1); n < Ns; n *= stage_radix(P, n)) off += (stage_radix(P, n) - 1) * n;
    return off;
}
__host__ __device__ constexpr int tw_size(int P) { return tw_offset(P, P); }

// Between stages the transform lives in shared memory in a swizzled order:
// value n sits at swz(n), which permutes the 16 values of each 128-byte row r
// by XOR with g(r) = (r mod 8) + 8 * (bit 2 of r). A 64-bit shared access is
// served half a warp at a time, so the scattered stores of the first stage
// (index 8j + s: rows j/2, positions 8 (j mod 2) + s) and of the second
// ((j/8) 64 + j mod 8 + 8s: rows 4 (j/8) + s/2) must put each half warp's 16
// values on 16 different positions: the first needs g mod 8 distinct over 8
// consecutive rows, the second different bit 3 in rows r and r + 4. The
// strided loads stay one row per half warp. A transform's input (filled by
// the caller) and output are in natural order.
__device__ __forceinline__ int swz(int n)
{
    const int r = n >> 4;
    return n ^ ((r & 7) | ((r & 4) << 1));
}

// One Stockham stage of radix R on a P-point transform: butterfly j reads
// src[j + r P/R], rotates input r by the twiddle r * (j mod Ns) / (Ns R) of a
// turn, transforms, and writes dst[(j / Ns) Ns R + (j mod Ns) + s Ns] (SW_IN,
// SW_OUT: src, dst in swizzled order). Output transform of the last stage:
// epi(n, v) is stored at natural index n.
struct NoEpi {
    __device__ __forceinline__ float2 operator()(int, float2 v) const { return v; }
};

template <int P, int Ns, int R, bool INV, bool SW_IN, bool SW_OUT, class Epi = NoEpi>
__device__ __forceinline__ void stockham_stage(const float2 *__restrict__ src, float2 *__restrict__ dst,
                                               int j, const float2 *__restrict__ tw, Epi epi = Epi())
{
    constexpr int stride = P / R;
    const int k = j & (Ns - 1);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int n = j + r * stride;
        v[r] = src[SW_IN ? swz(n) : n];
    }
    if constexpr (Ns > 1) {
        const float2 *tws = tw + tw_offset(P, Ns) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = __ldg(tws + (r - 1) * Ns);
            v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
        }
    }
    dftR<R, INV>(v);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const int n = base + s * Ns;
        dst[SW_OUT ? swz(n) : n] = epi(n, v[s]);
    }
}

// Stages for P = 2^LG: radix 8 while three or more bits remain, then one
// radix-4 or radix-2 stage. Thread j of T = P/8 runs one butterfly per
// radix-8 stage, two per radix-4 stage, four per radix-2 stage. epi is applied
// to the values of the last stage as they are stored. The stage at Ns = 1
// reads natural order, later stages swizzled; the last stage writes natural.
template <int P, int Ns, bool INV, class Epi = NoEpi>
__device__ __forceinline__ float2 *fft_stages(float2 *a, float2 *b, int j, const float2 *__restrict__ tw,
                                              Epi epi = Epi())
{
    constexpr int T = P / 8;
    constexpr bool SW_IN = Ns > 1;
    if constexpr (Ns == P) {
        return a;
    } else if constexpr (P / Ns >= 8) {
        if constexpr (P / Ns == 8)
            stockham_stage<P, Ns, 8, INV, SW_IN, false>(a, b, j, tw, epi);
        else
            stockham_stage<P, Ns, 8, INV, SW_IN, true>(a, b, j, tw);
        __syncthreads();
        return fft_stages<P, Ns * 8, INV>(b, a, j, tw, epi);
    } else if constexpr (P / Ns == 4) {
        stockham_stage<P, Ns, 4, INV, SW_IN, false>(a, b, j, tw, epi);
        stockham_stage<P, Ns, 4, INV, SW_IN, false>(a, b, j + T, tw, epi);
        __syncthreads();
        return b;
    } else {
        static_assert(P / Ns == 2, "radix plan");
#pragma unroll
        for (int u = 0; u < 4; ++u) stockham_stage<P, Ns, 2, INV, SW_IN, false>(a, b, j + u * T, tw, epi);
        __syncthreads();
        return b;
    }
}

// Complex P-point FFT of a[0..P) (natural order), result returned (a or b).
// Caller must __syncthreads() after filling a.
template <int P, bool INV, class Epi = NoEpi>
__device__ __forceinline__ float2 *fft_complex(float2 *a, float2 *b, int j, const float2 *__restrict__ tw,
                                               Epi epi = Epi())
{
    return fft_stages<P, 1, INV>(a, b, j, tw, epi);
}

// The same FFT when thread j already holds inputs j + s T (s < 8) in z: the
// first radix-8 stage (no twiddles) runs on the registers and stores into b.
template <int P, bool INV, class Epi = NoEpi>
__device__ __forceinline__ float2 *fft_complex_regs(float2 (&z)[8], float2 *a, float2 *b, int j,
                                                    const float2 *__restrict__ tw, Epi epi = Epi())
{
    static_assert(P >= 16, "a radix-8 first stage and at least one stage after it");
    dftR<8, INV>(z);
#pragma unroll
    for (int s = 0; s < 8; ++s) b[swz(j * 8 + s)] = z[s];   // stage Ns = 1: dst (j * 8 + s), swizzled
    __syncthreads();
    return fft_stages<P, 8, INV>(b, a, j, tw, epi);
}

// Split step after the forward FFT: thread j handles pairs k = j + s T.
// Writes X(k) and X(P-1-k) through the functor st(k, value).
template <int P, class Store>
__device__ __forceinline__ void split_forward(const float2 *Z, int j, const float2 *__restrict__ post,
                                              Store st)
{
    constexpr int T = P / 8;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int k = j + s * T;
        const int kk = P - 1 - k;
        const float2 zk = Z[k], zkk = Z[kk];
        const float2 E = make_float2(0.5f * (zk.x + zkk.x), 0.5f * (zk.y - zkk.y));
        // O = (zk - conj zkk) / 2i
        const float2 d = make_float2(0.5f * (zk.x - zkk.x), 0.5f * (zk.y + zkk.y));
        const float2 O = make_float2(d.y, -d.x);
        const float2 t = cmul(__ldg(post + k), O);
        st(k, cadd(E, t));
        st(kk, cconj(csub(E, t)));
    }
}

// Merge step before the inverse FFT: from Y(k), Y(P-1-k) build
// Z(k) = E + i O and Z(P-1-k) = conj E + i conj O, where
// E = (Y(k) + conj Y(P-1-k)) / 2 and O = (Y(k) - conj Y(P-1-k)) conj(W^{k+1/2}) / 2.
template <int P, class Load>
__device__ __forceinline__ void merge_inverse(float2 *Z, int j, const float2 *__restrict__ post, Load ld)
{
    constexpr int T = P / 8;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int k = j + s * T;
        const int kk = P - 1 - k;
        const float2 yk = ld(k), ykk = ld(kk);
        const float2 E = make_float2(0.5f * (yk.x + ykk.x), 0.5f * (yk.y - ykk.y));
        const float2 d = make_float2(0.5f * (yk.x - ykk.x), 0.5f * (yk.y + ykk.y));
        const float2 O = cmulc(d, __ldg(post + k));
        // i O
        const float2 iO = make_float2(-O.y, O.x);
        const float2 iOc = make_float2(O.y, O.x);  // i conj(O)
        Z[k] = cadd(E, iO);
        Z[kk] = cadd(cconj(E), iOc);
    }
}

}  // namespace tvolap

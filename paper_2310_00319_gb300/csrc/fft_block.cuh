// One-block transforms shared by the plan kernels and the streaming server.
// A transform is P = 2L complex points run by T = P/8 threads; F = 256/T
// transforms share a 256-thread CTA (see fft_core.cuh for the FFT itself).
#pragma once

#include "fft_core.cuh"

namespace tvolap {

template <int P>
struct Geo {
    static constexpr int T = P / 8;                         // threads per transform
    static constexpr int F = (256 / T) > 0 ? 256 / T : 1;   // transforms per CTA
    static constexpr int THREADS = T * F;
};

template <int LG>
inline size_t smem_fft()
{
    constexpr int P = 1 << LG;
    return (size_t)2 * Geo<P>::F * P * sizeof(float2);
}

// Forward real transform of one zero-padded block whose first 2L samples are
// given by src(n) (n < 2L, n even: src returns samples n and n+1): fills A,
// runs the FFT, splits into the P half-bin spectrum values through st(k, v).
template <int P, bool FULL = false, class Src, class Store>
__device__ __forceinline__ void forward_block(float2 *A, float2 *B, int j, bool active, Src src,
                                              const float2 *__restrict__ rot,
                                              const float2 *__restrict__ post,
                                              const float2 *__restrict__ tw, Store st)
{
    constexpr int T = P / 8;
    float2 z[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int r = j + s * T;
        z[s] = make_float2(0.f, 0.f);
        // r < P/2 = L unless FULL: the upper half is the zero padding of Eqs. 3-4
        if ((FULL || s < 4) && active) {
            z[s] = cmul(src(2 * r), __ldg(rot + r));
        }
    }
    // the first stage reads exactly inputs j + s T: it runs on the registers
    float2 *Z = fft_complex_regs<P, false>(z, A, B, j, tw);
    split_forward<P>(Z, j, post, st);
}

// Streaming inverse of one output block (Eq. 8) and the overlap-add of
// Eqs. 9-12 against the 3L pending sums st of this output: out[0..L) receives
// the finished samples and st the new pending sums. ld(k) gives Y(k).
template <int P, class Load>
__device__ __forceinline__ void inverse_stream_block(float2 *A, float2 *B, int j, bool active,
                                                     Load ld, float *st, float *out,
                                                     const float2 *__restrict__ rot,
                                                     const float2 *__restrict__ post,
                                                     const float2 *__restrict__ tw)
{
    constexpr int T = P / 8, L = P / 2;
    merge_inverse<P>(A, j, post, [&](int k) { return active ? ld(k) : make_float2(0.f, 0.f); });
    __syncthreads();
    // undo the pre-rotation and scale as the last stage stores:
    // y(2r) + i y(2r+1) = Z(r) e^{+i pi r/P} / P
    const float inv_p = 1.0f / (float)P;
    float2 *Z = fft_complex<P, true>(A, B, j, tw, [&](int r, float2 v) {
        return cscale(cmulc(v, __ldg(rot + r)), inv_p);
    });
    const float *yb = reinterpret_cast<const float *>(Z);
    // read every pending sum this thread rewrites before any thread writes;
    // T = L/4 threads cover the 3L pending sums in exactly 12 steps
    float keep[12];
#pragma unroll
    for (int u = 0; u < 12; ++u) {
        const int i = j + u * T;
        float v = yb[i + L];
        if (active && i < 2 * L) v += st[i + L];
        keep[u] = v;
    }
    if (active)
        for (int i = j; i < L; i += T) out[i] = st[i] + yb[i];
    __syncthreads();
    if (active) {
#pragma unroll
        for (int u = 0; u < 12; ++u) st[j + u * T] = keep[u];
    }
}

// Host-side dispatch of a launcher body over the transform size P = 1 << LGV.
#define TVOLAP_DISPATCH(LGV, ...)             \
    switch (LGV) {                            \
    case 5: { constexpr int LG = 5; __VA_ARGS__; } break;   \
    case 6: { constexpr int LG = 6; __VA_ARGS__; } break;   \
    case 7: { constexpr int LG = 7; __VA_ARGS__; } break;   \
    case 8: { constexpr int LG = 8; __VA_ARGS__; } break;   \
    case 9: { constexpr int LG = 9; __VA_ARGS__; } break;   \
    case 10: { constexpr int LG = 10; __VA_ARGS__; } break; \
    case 11: { constexpr int LG = 11; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;    \
    }


template <class Kern>
inline cudaError_t set_smem(Kern k, size_t bytes)
{
    if (bytes > 48 * 1024)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

}  // namespace tvolap

// Batched shared-memory Stockham FFT used by the NUFFT kernels.
//
// One transform of power-of-two length N lives in shared memory at
// s[i * stride], i < N, and is processed by N/8 threads.  Each pass of radix R
// (8 while the remaining factor allows, then 4 or 2) reads R strided inputs
// per butterfly, applies the twiddles, runs an R-point DFT in registers and
// writes to the self-sorting (Stockham) positions, so the result comes out in
// natural order with no bit reversal.  Every thread of the block calls each
// pass (idle ones with active = false) because passes end in __syncthreads().
//
// Forward: X[m] = sum_n x[n] exp(-2 pi i m n / N); inverse (INV): the same
// sum with exp(+2 pi i m n / N), unnormalised.
#pragma once
#include "common.h"

namespace mrf {

// tw[k] = exp(-2 pi i k / N), k < N, built once per block.
template <int N>
__device__ __forceinline__ void fft_twiddles(float2* tw) {
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float s, c;
        sincospif(-2.0f * (float)k / (float)N, &s, &c);
        tw[k] = make_float2(c, s);
    }
}

template <bool INV>
__device__ __forceinline__ float2 twiddle(float2 v, float2 w) {
    return INV ? cmulc(v, w) : cmul(v, w);
}

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 v) {
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
    float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    float2 a2 = cadd(v[1], v[3]), a3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    const float h = 0.70710678118654752f;
    // even part: 4-point DFT of v0, v2, v4, v6
    float2 a0 = cadd(v[0], v[4]), a1 = csub(v[0], v[4]);
    float2 a2 = cadd(v[2], v[6]), a3 = rot90<INV>(csub(v[2], v[6]));
    float2 e0 = cadd(a0, a2), e2 = csub(a0, a2), e1 = cadd(a1, a3), e3 = csub(a1, a3);
    // odd part: 4-point DFT of v1, v3, v5, v7
    float2 b0 = cadd(v[1], v[5]), b1 = csub(v[1], v[5]);
    float2 b2 = cadd(v[3], v[7]), b3 = rot90<INV>(csub(v[3], v[7]));
    float2 o0 = cadd(b0, b2), o2 = rot90<INV>(csub(b0, b2)), o1 = cadd(b1, b3), o3 = csub(b1, b3);
    // twiddles W8^1 and W8^3 (conjugated for the inverse)
    float2 w1 = INV ? make_float2(h, h) : make_float2(h, -h);
    float2 w3 = INV ? make_float2(-h, h) : make_float2(-h, -h);
    o1 = cmul(o1, w1);
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
__device__ __forceinline__ void dft_r(float2* v) {
    if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else dft2<INV>(v);
}

// One Stockham pass of radix R over a length-N transform.  Ns = product of the
// radices of the passes already done.
template <int N, int R, bool INV>
__device__ __forceinline__ void stockham_pass(float2* s, int stride, int Ns, int tid, bool active,
                                              const float2* tw) {
    constexpr int NB = N / R;       // butterflies
    constexpr int TPF = N / 8;      // threads per transform
    constexpr int PER = NB / TPF;   // butterflies per thread (8 / R)
    float2 v[PER][R];
    if (active) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * TPF;
            const int jm = j & (Ns - 1);
            const int step = N / (Ns * R);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 x = s[(j + r * NB) * stride];
                if (r > 0) x = twiddle<INV>(x, tw[r * jm * step]);
                v[q][r] = x;
            }
            dft_r<R, INV>(v[q]);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * TPF;
            const int jm = j & (Ns - 1);
            const int d = (j - jm) * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) s[(d + r * Ns) * stride] = v[q][r];
        }
    }
    __syncthreads();
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Full in-place transform; ends with the data in natural order and synced.
template <int N, bool INV>
__device__ __forceinline__ void fft_smem(float2* s, int stride, int tid, bool active, const float2* tw) {
    constexpr int L = ilog2(N);
    constexpr int N8 = L / 3;
    constexpr int REM = L % 3;
    int Ns = 1;
#pragma unroll
    for (int p = 0; p < N8; ++p) {
        stockham_pass<N, 8, INV>(s, stride, Ns, tid, active, tw);
        Ns *= 8;
    }
    if constexpr (REM == 2) stockham_pass<N, 4, INV>(s, stride, Ns, tid, active, tw);
    if constexpr (REM == 1) stockham_pass<N, 2, INV>(s, stride, Ns, tid, active, tw);
}

}  // namespace mrf

namespace mrf {

// ---------------------------------------------------------------------------
// Batched form: B independent length-N transforms processed by the whole
// block of NT threads.  Thread t works on transform t % B and on butterflies
// t / B, t / B + NT / B, ... of every pass, so consecutive lanes touch the
// same element of consecutive transforms.  Element i of transform b lives at
// s[b * bstride + i * estride]; with columns of a [rows][B] tile (estride = B,
// bstride = 1) or rows padded to an odd stride (estride = 1, bstride = N + 1)
// every shared-memory access of a warp is bank-conflict free.
// ---------------------------------------------------------------------------
template <int N, int R, int NWK, bool INV>
__device__ __forceinline__ void batch_pass(float2* t, int es, int Ns, int wk, const float2* tw) {
    constexpr int NB = N / R;
    constexpr int PER = (NB + NWK - 1) / NWK;
    float2 v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int j = wk + q * NWK;
        if (j < NB) {
            const int jm = j & (Ns - 1);
            const int step = N / (Ns * R);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 x = t[(j + r * NB) * es];
                if (r > 0) x = twiddle<INV>(x, tw[r * jm * step]);
                v[q][r] = x;
            }
            dft_r<R, INV>(v[q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int j = wk + q * NWK;
        if (j < NB) {
            const int jm = j & (Ns - 1);
            const int d = (j - jm) * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) t[(d + r * Ns) * es] = v[q][r];
        }
    }
    __syncthreads();
}

template <int N, int B, int NT, bool INV>
__device__ __forceinline__ void fft_batch(float2* s, int estride, int bstride, const float2* tw) {
    static_assert(NT % B == 0, "block size must be a multiple of the batch");
    constexpr int NWK = NT / B;
    constexpr int L = ilog2(N);
    constexpr int N8 = L / 3;
    constexpr int REM = L % 3;
    float2* t = s + (threadIdx.x % B) * bstride;
    const int wk = threadIdx.x / B;
    int Ns = 1;
#pragma unroll
    for (int p = 0; p < N8; ++p) {
        batch_pass<N, 8, NWK, INV>(t, estride, Ns, wk, tw);
        Ns *= 8;
    }
    if constexpr (REM == 2) batch_pass<N, 4, NWK, INV>(t, estride, Ns, wk, tw);
    if constexpr (REM == 1) batch_pass<N, 2, NWK, INV>(t, estride, Ns, wk, tw);
}

}  // namespace mrf

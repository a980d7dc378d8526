// Batched shared-memory Stockham FFT used by the NUFFT kernels.
//
// One transform of length N (a power of two, or 3 times one) lives in shared
// memory at a fixed stride.  Each pass of radix R (3 for the factor 3, 8 while
// the remaining factor allows, then 4 or 2) reads R strided inputs per
// butterfly, applies the twiddles, runs an R-point DFT in registers and
// writes to the self-sorting (Stockham) positions, so the result comes out in
// natural order with no bit reversal.  Every thread of the block calls each
// pass because passes end in __syncthreads().
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

// X0 = a + b + c, X1,2 = a - (b + c)/2 -/+ i (sqrt(3)/2)(b - c) (forward;
// the sign of the i term flips for the inverse)
template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
    const float h = 0.86602540378443865f;       // sqrt(3) / 2
    const float2 a = v[0], t1 = cadd(v[1], v[2]);
    const float2 t2 = csub(a, cscale(t1, 0.5f));
    const float2 t3 = rot90<INV>(cscale(csub(v[1], v[2]), h));
    v[0] = cadd(a, t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v) {
    if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else dft2<INV>(v);
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
// One pass of radix R after sub-transforms of length Ns (POW2: Ns a power of
// two, so j mod Ns is a mask).
template <int N, int R, int NWK, bool INV, bool POW2>
__device__ __forceinline__ void batch_pass(float2* t, int es, int Ns, int wk, const float2* tw) {
    constexpr int NB = N / R;
    constexpr int PER = (NB + NWK - 1) / NWK;
    float2 v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int j = wk + q * NWK;
        if (j < NB) {
            const int jm = POW2 ? (j & (Ns - 1)) : (j % Ns);
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
            const int jm = POW2 ? (j & (Ns - 1)) : (j % Ns);
            const int d = (j - jm) * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) t[(d + r * Ns) * es] = v[q][r];
        }
    }
    __syncthreads();
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Lengths N = 2^a, or 3 x 2^a (a radix-3 pass first, then the power of two).
template <int N, int B, int NT, bool INV>
__device__ __forceinline__ void fft_batch(float2* s, int estride, int bstride, const float2* tw) {
    static_assert(NT % B == 0, "block size must be a multiple of the batch");
    constexpr bool POW2 = (N & (N - 1)) == 0;
    static_assert(POW2 || (N % 3 == 0 && ((N / 3) & (N / 3 - 1)) == 0), "N = 2^a or 3 x 2^a");
    constexpr int NWK = NT / B;
    constexpr int M = POW2 ? N : N / 3;       // the power-of-two part
    constexpr int L = ilog2(M);
    constexpr int N8 = L / 3;
    constexpr int REM = L % 3;
    float2* t = s + (threadIdx.x % B) * bstride;
    const int wk = threadIdx.x / B;
    int Ns = 1;
    if constexpr (!POW2) {
        batch_pass<N, 3, NWK, INV, false>(t, estride, Ns, wk, tw);
        Ns = 3;
    }
#pragma unroll
    for (int p = 0; p < N8; ++p) {
        batch_pass<N, 8, NWK, INV, POW2>(t, estride, Ns, wk, tw);
        Ns *= 8;
    }
    if constexpr (REM == 2) batch_pass<N, 4, NWK, INV, POW2>(t, estride, Ns, wk, tw);
    if constexpr (REM == 1) batch_pass<N, 2, NWK, INV, POW2>(t, estride, Ns, wk, tw);
}

// ---------------------------------------------------------------------------
// Register-resident four-step transform of 512-point columns (the strip
// kernels at grid 512).  N = 512 = 16 x 32 with n = t + 16 m, k = k1 + 32 k2:
//   X[k1 + 32 k2] = sum_t W16^(t k2) W512^(t k1) sum_m W32^(m k1) x[t + 16 m].
// A 16-column strip takes 256 threads, thread (c = tid % 16, t = tid / 16):
// the 32-point DFT over m of its column's elements t + 16 m in registers,
// the W512^(t k1) twiddles, one exchange through shared memory, then the two
// 16-point DFTs over t for k1 = 2 t, 2 t + 1 in registers.  Each element
// crosses shared memory once (a write and a read) instead of once per
// radix-8 pass (three, plus the twiddle reads).
// ---------------------------------------------------------------------------
// exp(-2 pi i j / 32)
static __constant__ float2 c_w32[32] = {
    {1.0f, 0.0f}, {0.98078528f, -0.195090322f}, {0.923879533f, -0.382683432f}, {0.831469612f, -0.555570233f},
    {0.707106781f, -0.707106781f}, {0.555570233f, -0.831469612f}, {0.382683432f, -0.923879533f}, {0.195090322f, -0.98078528f},
    {0.0f, -1.0f}, {-0.195090322f, -0.98078528f}, {-0.382683432f, -0.923879533f}, {-0.555570233f, -0.831469612f},
    {-0.707106781f, -0.707106781f}, {-0.831469612f, -0.555570233f}, {-0.923879533f, -0.382683432f}, {-0.98078528f, -0.195090322f},
    {-1.0f, 0.0f}, {-0.98078528f, 0.195090322f}, {-0.923879533f, 0.382683432f}, {-0.831469612f, 0.555570233f},
    {-0.707106781f, 0.707106781f}, {-0.555570233f, 0.831469612f}, {-0.382683432f, 0.923879533f}, {-0.195090322f, 0.98078528f},
    {0.0f, 1.0f}, {0.195090322f, 0.98078528f}, {0.382683432f, 0.923879533f}, {0.555570233f, 0.831469612f},
    {0.707106781f, 0.707106781f}, {0.831469612f, 0.555570233f}, {0.923879533f, 0.382683432f}, {0.98078528f, 0.195090322f}};

// natural-order DFT of length 32 (m = a + 4 b: DFT8 over b, twiddles
// W32^(a kb), DFT4 over a; X[kb + 8 ka])
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
    float2 u[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) u[a][b] = v[a + 4 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a) dft8<INV>(u[a]);
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
        for (int kb = 1; kb < 8; ++kb) u[a][kb] = twiddle<INV>(u[a][kb], c_w32[a * kb]);
#pragma unroll
    for (int kb = 0; kb < 8; ++kb) {
        float2 w[4] = {u[0][kb], u[1][kb], u[2][kb], u[3][kb]};
        dft4<INV>(w);
#pragma unroll
        for (int ka = 0; ka < 4; ++ka) v[kb + 8 * ka] = w[ka];
    }
}

// natural-order DFT of length 16 (m = a + 4 b: DFT4 over b, twiddles
// W16^(a kb) = W32^(2 a kb), DFT4 over a; X[kb + 4 ka])
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
    float2 u[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) u[a][b] = v[a + 4 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a) dft4<INV>(u[a]);
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
        for (int kb = 1; kb < 4; ++kb) u[a][kb] = twiddle<INV>(u[a][kb], c_w32[2 * a * kb]);
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        float2 w[4] = {u[0][kb], u[1][kb], u[2][kb], u[3][kb]};
        dft4<INV>(w);
#pragma unroll
        for (int ka = 0; ka < 4; ++ka) v[kb + 4 * ka] = w[ka];
    }
}

// The four-step transform of a 16-column strip (blockDim 256).  x: the
// thread's inputs x[t + 16 m], m = 0..31, of column c; buf: [512][16] shared
// scratch (free on entry; free again on return); tw: tw[k] = exp(-2 pi i k /
// 512).  out[j][k2] = X[(2 t + j) + 32 k2] of column c.
template <bool INV>
__device__ __forceinline__ void col512(float2 (&x)[32], float2* buf, const float2* tw, float2 (&out)[2][16]) {
    const int c = threadIdx.x & 15, t = threadIdx.x >> 4;
    dft32<INV>(x);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) x[k1] = twiddle<INV>(x[k1], tw[(t * k1) & 511]);
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) buf[(k1 * 16 + t) * 16 + c] = x[k1];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int k1 = 2 * t + j;
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) out[j][tt] = buf[(k1 * 16 + tt) * 16 + c];
        dft16<INV>(out[j]);
    }
    __syncthreads();
}

// The same four-step transform for 16 rows of 512 points held one row per
// 16 threads (blockDim 256, thread (t = tid % 16, r = tid / 16)): x holds
// x[t + 16 m] of row r.  buf: 32 x 257 shared scratch (free on entry and on
// return; the odd stride keeps both exchange directions conflict-free); tw2:
// tw2[k1 * 16 + t] = exp(-2 pi i t k1 / 512) (row512_twiddles).
// out[j][k2] = X[(t + 16 j) + 32 k2] of row r.
constexpr int kRow512Buf = 32 * 257;

__device__ __forceinline__ void row512_twiddles(float2* tw2) {
    for (int i = threadIdx.x; i < 512; i += blockDim.x) {
        const int k1 = i >> 4, t = i & 15;
        float s, c;
        sincospif(-2.0f * (float)((t * k1) & 511) / 512.0f, &s, &c);
        tw2[i] = make_float2(c, s);
    }
}

template <bool INV>
__device__ __forceinline__ void row512(float2 (&x)[32], float2* buf, const float2* tw2, float2 (&out)[2][16]) {
    const int t = threadIdx.x & 15, r = threadIdx.x >> 4;
    dft32<INV>(x);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) x[k1] = twiddle<INV>(x[k1], tw2[k1 * 16 + t]);
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) buf[k1 * 257 + r * 16 + t] = x[k1];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int k1 = t + 16 * j;
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) out[j][tt] = buf[k1 * 257 + r * 16 + tt];
        dft16<INV>(out[j]);
    }
    __syncthreads();
}

}  // namespace mrf

// Device helpers shared by the tensor-core matchers (match_tc.cu: subspace
// lengths with the whole fingerprint tile resident in shared memory;
// match_tc_long.cu: full-length fingerprints streamed along the reduction
// axis).
#pragma once
#include <cuda_bf16.h>

#include "common.h"

namespace mrf {

// Operand value of the split form: with SPLIT = 3 the reduction axis holds
// three copies of the 2 len real coefficients, (hi, hi, lo) for A and
// (hi, lo, hi) for B, hi = bf16(v), lo = bf16(v - hi), so that the product sums
// A_hi B_hi + A_hi B_lo + A_lo B_hi (relative error ~2^-16) in one GEMM.
__device__ __forceinline__ __nv_bfloat16 split_part(float v, int part, bool is_a, int split) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    if (split == 1) return hi;
    const bool want_lo = is_a ? (part == 2) : (part == 1);
    return want_lo ? __float2bfloat16_rn(v - __bfloat162float(hi)) : hi;
}

// Row order of an atom tile (and so TMEM column order): each group of 16 rows
// holds the Re rows of 8 consecutive atoms, then their Im rows, so that a
// 16-column TMEM read gives 8 real parts and 8 imaginary parts in order (two
// atoms' parts side by side for the packed FP32 score).
__host__ __device__ __forceinline__ void tile_row(int row, int* atom, int* imag) {
    *atom = ((row >> 4) << 3) + (row & 7);
    *imag = (row >> 3) & 1;
}

// (a.x^2 + b.x^2, a.y^2 + b.y^2) with packed FP32 arithmetic (two lanes of
// one instruction each): a = the real parts, b = the imaginary parts of two atoms
__device__ __forceinline__ float2 abs2_pair(float2 re, float2 im) {
    float2 d;
    asm("{\n\t.reg .b64 r, i, t;\n\t"
        "mov.b64 r, {%2, %3};\n\tmov.b64 i, {%4, %5};\n\t"
        "mul.rn.f32x2 t, i, i;\n\tfma.rn.f32x2 t, r, r, t;\n\t"
        "mov.b64 {%0, %1}, t;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(re.x), "f"(re.y), "f"(im.x), "f"(im.y));
    return d;
}

__device__ __forceinline__ bool better_cand(float s, int i, float bs, int bi) {
    return s > bs || (s == bs && i < bi);
}

// FP32 inner products s_q = <d_{a_q}, x> = sum_k conj(d_{a_q,k}) x_k of C atoms
// with one fingerprint row, summed in k order (atoms with a_q outside [0, m)
// give 0).  The row and the atoms are read U coefficients at a time with all
// of a chunk's loads issued before its arithmetic, so a row costs ~len / U
// memory round trips instead of C len.
template <int C>
__device__ __forceinline__ void atom_products(const float2* __restrict__ xr, int len, const int (&a)[C],
                                              const float2* __restrict__ dict, int m, float2 (&s)[C]) {
    constexpr int U = C <= 4 ? 4 : 2;
#pragma unroll
    for (int q = 0; q < C; ++q) s[q] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < len; k0 += U) {
        float2 xv[U], dv[C][U];
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = k0 + u < len ? xr[k0 + u] : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < C; ++q)
#pragma unroll
            for (int u = 0; u < U; ++u)
                dv[q][u] = (a[q] >= 0 && a[q] < m && k0 + u < len) ? dict[(size_t)a[q] * len + k0 + u]
                                                                    : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < C; ++q)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k0 + u < len) s[q] = cadd(s[q], cconjmul(dv[q][u], xv[u]));
    }
}

}  // namespace mrf

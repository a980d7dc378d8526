// Singular value thresholding of every patch (Eq. 18): with
// Q_i(X) = A = sum_j sigma_j u_j v_j^H (A: the patch's p^2 x K coefficient
// block; its singular values are those of the p^2 x T patch because the
// temporal basis is orthonormal),
//   P_i = sum_j max(sigma_j - tau, 0) u_j v_j^H = B diag(f) V^H,
//   B = A V,  sigma_j = ||b_j||,  f_j = max(sigma_j - tau, 0) / sigma_j,
// and the patch's nuclear norm sum_j sigma_j (for the cost of Algorithm 1).
//
// V (the right singular vectors) diagonalises the K x K Gram matrix
// G = A^H A; it is found by cyclic two-sided Jacobi on G, started from the
// previous iteration's V (G' = V_prev^H G V_prev is then nearly diagonal and
// a few sweeps finish it).  The p^2-row matrix is touched only four times
// (G, and B = A V, and P, plus the load), so the iteration works on K x K
// data instead of p^2 x K columns.  The singular values are taken as the
// column norms of B, computed from A directly, which keeps the small ones
// (and so the nuclear norm) accurate even though G squares the condition
// number.  Jacobi rotates a pair while |G_pq| exceeds both kSvtTol (relative,
// |G_pq| / sqrt(G_pp G_qq): the cosine between the two columns of A V) and a
// floor of a few FP32 roundings of trace(G), below which G_pq is rounding
// noise of the Gram products; a sweep without rotations ends the loop, and so
// does a sweep whose rotations were all below kSvtQuad (Jacobi converges
// quadratically: what such a sweep leaves is of order kSvtQuad^2).
//
// Layout: LANES lanes per patch (16: two patches per warp; 32: one), R rows of
// the patch per lane (row = sl + LANES r).  The K x K work lives in shared
// memory: a round of the parallel cyclic order pairs every index once
// (NPAIR disjoint pairs, circle schedule); lane sl < NPAIR computes pair sl's
// rotation and updates that pair's 2 x 2 diagonal block in closed form, the
// off-diagonal 2 x 2 blocks (pair P rows, pair Q columns, P < Q, and their
// mirror) are each updated by one lane, and the rotation matrix W
// accumulates J column-pair by column-pair.  Every 2 x 2 block is read and
// written by one lane only within a round, so a round needs one exchange of
// the rotation parameters and one sync at its end.
#pragma once
#include "common.h"

namespace mrf {

// sum over the LANES lanes of one patch (a whole warp, or one half of it)
template <int LANES>
__device__ __forceinline__ float lane_sum(float v) {
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr float kSvtTol = 2e-6f;
constexpr float kSvtQuad = 3e-4f;
constexpr int kSvtMaxSweeps = 20;

__host__ __device__ constexpr int svt_npair(int KP) { return KP / 2; }
__host__ __device__ constexpr int svt_ng(int KP) { return KP * (KP + 1) / 2; }
// shared memory of one patch, in float2 units: G, then a region holding either
// the Gram reduction partials (8 per entry of the upper triangle) or W and
// V_prev, then the NPAIR rotations (2 float2 each)
__host__ __device__ constexpr int svt_region(int KP) {
    return 8 * svt_ng(KP) > 2 * KP * KP ? 8 * svt_ng(KP) : 2 * KP * KP;
}
__host__ __device__ constexpr int svt_patch_f2(int KP) { return KP * KP + svt_region(KP) + 2 * svt_npair(KP); }

// index pair (p, q) of pair i in round rd of the circle schedule on KP
// indices: index KP - 1 meets rd, and (rd + i) meets (rd - i) (mod KP - 1)
__device__ __forceinline__ void svt_pair(int KP, int rd, int i, int& p, int& q) {
    const int m = KP - 1;
    if (i == 0) {
        p = rd;
        q = m;
    } else {
        p = rd + i;
        if (p >= m) p -= m;
        q = rd - i;
        if (q < 0) q += m;
    }
}

// J = [[cs, sn], [-sn ph, cs ph]] acting on a column pair; rows mix with J^H
struct SvtRot {
    float cs, sn;
    float2 ph;
};

__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// [x, y] J: (cs x - sn ph y, sn x + cs ph y)
__device__ __forceinline__ void rot_cols(const SvtRot& r, float2& x, float2& y) {
    const float2 py = cmul(r.ph, y);
    const float2 nx = csub(cscale(x, r.cs), cscale(py, r.sn));
    y = cadd(cscale(x, r.sn), cscale(py, r.cs));
    x = nx;
}

// J^H [x; y]: (cs x - sn conj(ph) y, sn x + cs conj(ph) y)
__device__ __forceinline__ void rot_rows(const SvtRot& r, float2& x, float2& y) {
    const float2 py = cmul(cconj(r.ph), y);
    const float2 nx = csub(cscale(x, r.cs), cscale(py, r.sn));
    y = cadd(cscale(x, r.sn), cscale(py, r.cs));
    x = nx;
}

}  // namespace mrf

namespace mrf {

__device__ __forceinline__ bool rot_is_identity(const SvtRot& r) {
    return r.sn == 0.f && r.ph.x == 1.f && r.ph.y == 0.f;
}

// Vio (nullable) holds each patch's right singular vectors [np][KP][KP]
// (row = coordinate, column = singular vector): with warm != 0 the Jacobi
// iteration starts from them; the new ones are stored back.  The SVD computed
// is the same either way.  A slot past the last patch works on zeros.
template <int R, int KP, int LANES>
__global__ void __launch_bounds__(128, 4)
    k_svt(const float2* __restrict__ alpha, PatchGeom g, int K, float tau, float2* __restrict__ P,
          double* __restrict__ nuc, float2* __restrict__ Vio, int warm, unsigned long long* __restrict__ stats) {
    constexpr int NPAIR = svt_npair(KP), NG = svt_ng(KP), NOFF = NPAIR * (NPAIR - 1) / 2;
    constexpr int NU = (NOFF + LANES - 1) / LANES;               // off-diagonal blocks per lane
    constexpr int NWU = (KP * NPAIR + LANES - 1) / LANES;        // W column-pair tasks per lane
    constexpr int KK = KP * KP;
    extern __shared__ float2 svt_sm[];
    const int lane = threadIdx.x & 31;
    const int sl = lane & (LANES - 1);
    const int slot = (int)(threadIdx.x >> 5) * (32 / LANES) + lane / LANES;
    const int j = (int)blockIdx.x * ((int)blockDim.x / LANES) + slot;
    const bool active = j < g.count();
    float2* Gs = svt_sm + (size_t)slot * svt_patch_f2(KP);
    float2* reg = Gs + KK;                 // Gram partials, then W and V_prev
    float2* Ws = reg;
    float2* Vs = reg + KK;
    SvtRot* rot = reinterpret_cast<SvtRot*>(reg + svt_region(KP));

    const int pp = g.p * g.p;
    const int jy = active ? g.origin(j / g.cnt) : 0, jx = active ? g.origin(j % g.cnt) : 0;
    float2 a[R][KP];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = sl + LANES * r;
        const bool ok = active && row < pp;
        const int py = ok ? row / g.p : 0, px = ok ? row - py * g.p : 0;
        const float2* src = alpha + ((size_t)(jy + py) * g.n + jx + px) * K;
#pragma unroll
        for (int k = 0; k < KP; ++k) a[r][k] = (ok && k < K) ? src[k] : make_float2(0.f, 0.f);
    }

    // G = A^H A, upper triangle row by row: lane partials, summed by shuffles
    // down to 8 partials per entry, then through shared memory
#pragma unroll
    for (int i = 0; i < KP; ++i) {
#pragma unroll
        for (int c = i; c < KP; ++c) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < R; ++r) s = cadd(s, cconjmul(a[r][i], a[r][c]));
#pragma unroll
            for (int o = LANES / 2; o >= 8; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            if (sl < 8) reg[(i * KP - i * (i - 1) / 2 + (c - i)) * 8 + sl] = s;
        }
    }
    __syncwarp();
    for (int e = sl; e < NG; e += LANES) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 8; ++q) s = cadd(s, reg[e * 8 + q]);
        int i = 0, rem = e;
        while (rem >= KP - i) { rem -= KP - i; ++i; }
        const int c = i + rem;
        Gs[i * KP + c] = c == i ? make_float2(s.x, 0.f) : s;
        if (c != i) Gs[c * KP + i] = cconj(s);
    }
    __syncwarp();

    // warm start: G <- V_prev^H G V_prev (T = G V_prev in Ws first)
    const bool use_warm = Vio != nullptr && warm != 0;
    if (use_warm) {
        for (int e = sl; e < KK; e += LANES)
            Vs[e] = active ? Vio[(size_t)j * KK + e] : make_float2(e / KP == e % KP ? 1.f : 0.f, 0.f);
        __syncwarp();
        for (int e = sl; e < KK; e += LANES) {
            const int i = e / KP, k = e - i * KP;
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < KP; ++l) s = cadd(s, cmul(Gs[i * KP + l], Vs[l * KP + k]));
            Ws[e] = s;
        }
        __syncwarp();
        for (int e = sl; e < KK; e += LANES) {
            const int i = e / KP, k = e - i * KP;
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < KP; ++l) s = cadd(s, cconjmul(Vs[l * KP + i], Ws[l * KP + k]));
            Gs[e] = i == k ? make_float2(s.x, 0.f) : s;
        }
        __syncwarp();
    }
    for (int e = sl; e < KK; e += LANES) Ws[e] = make_float2(e / KP == e % KP ? 1.f : 0.f, 0.f);
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < KP; ++i) tr += Gs[i * KP + i].x;
    // below this, an off-diagonal entry of G is rounding noise of the Gram products
    const float floor2 = (0x1p-22f * tr) * (0x1p-22f * tr);

    // this lane's off-diagonal blocks (P < Q, enumerated row by row) and W tasks
    int bP[NU > 0 ? NU : 1], bQ[NU > 0 ? NU : 1];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        int t = sl + LANES * u, Pi = -1, Qi = -1;
        if (t < NOFF) {
            Pi = 0;
            while (t >= NPAIR - 1 - Pi) { t -= NPAIR - 1 - Pi; ++Pi; }
            Qi = Pi + 1 + t;
        }
        bP[u] = Pi;
        bQ[u] = Qi;
    }
    __syncwarp();

    int nsweep = 0, nrot = 0;     // executed sweeps and rotations of this patch (for stats)
    for (int sweep = 0; sweep < kSvtMaxSweeps; ++sweep) {
        ++nsweep;
        bool rotated = false, large = false;
#pragma unroll 1
        for (int rd = 0; rd < KP - 1; ++rd) {
            if (sl < NPAIR) {
                int p, q;
                svt_pair(KP, rd, sl, p, q);
                const float al = Gs[p * KP + p].x, be = Gs[q * KP + q].x;
                const float2 c = Gs[p * KP + q];
                const float g2 = c.x * c.x + c.y * c.y;
                SvtRot r{1.f, 0.f, make_float2(1.f, 0.f)};
                if (g2 > floor2 && g2 > kSvtTol * kSvtTol * al * be) {
                    rotated = true;
                    ++nrot;
                    large |= g2 > kSvtQuad * kSvtQuad * al * be;
                    const float ig = rsqrtf(g2), gabs = g2 * ig;
                    // t: the root of t^2 + 2 zeta t - 1 = 0 of smaller magnitude,
                    // zeta = (G_qq - G_pp) / (2 |G_pq|)
                    const float d = be - al;
                    const float t = __fdividef(2.f * gabs, d + copysignf(sqrtf(d * d + 4.f * g2), d));
                    const float cs = rsqrtf(1.f + t * t);
                    r.cs = cs;
                    r.sn = cs * t;
                    r.ph = make_float2(c.x * ig, -c.y * ig);        // conj(G_pq) / |G_pq|
                    // the pair's diagonal block in closed form
                    Gs[p * KP + p] = make_float2(al - t * gabs, 0.f);
                    Gs[q * KP + q] = make_float2(be + t * gabs, 0.f);
                    Gs[p * KP + q] = make_float2(0.f, 0.f);
                    Gs[q * KP + p] = make_float2(0.f, 0.f);
                }
                rot[sl] = r;
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                if (bP[u] < 0) continue;
                const SvtRot rp = rot[bP[u]], rq = rot[bQ[u]];
                if (rot_is_identity(rp) && rot_is_identity(rq)) continue;
                int pP, qP, pQ, qQ;
                svt_pair(KP, rd, bP[u], pP, qP);
                svt_pair(KP, rd, bQ[u], pQ, qQ);
                float2 b00 = Gs[pP * KP + pQ], b01 = Gs[pP * KP + qQ];
                float2 b10 = Gs[qP * KP + pQ], b11 = Gs[qP * KP + qQ];
                rot_rows(rp, b00, b10);
                rot_rows(rp, b01, b11);
                rot_cols(rq, b00, b01);
                rot_cols(rq, b10, b11);
                Gs[pP * KP + pQ] = b00;
                Gs[pP * KP + qQ] = b01;
                Gs[qP * KP + pQ] = b10;
                Gs[qP * KP + qQ] = b11;
                Gs[pQ * KP + pP] = cconj(b00);
                Gs[qQ * KP + pP] = cconj(b01);
                Gs[pQ * KP + qP] = cconj(b10);
                Gs[qQ * KP + qP] = cconj(b11);
            }
#pragma unroll
            for (int v = 0; v < NWU; ++v) {
                const int w = sl + LANES * v;
                if (w >= KP * NPAIR) break;
                const int jr = w / NPAIR, Q = w - jr * NPAIR;
                const SvtRot rq = rot[Q];
                if (rot_is_identity(rq)) continue;
                int pQ, qQ;
                svt_pair(KP, rd, Q, pQ, qQ);
                float2 x = Ws[jr * KP + pQ], y = Ws[jr * KP + qQ];
                rot_cols(rq, x, y);
                Ws[jr * KP + pQ] = x;
                Ws[jr * KP + qQ] = y;
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, rotated && large)) break;
    }

    // V = V_prev W (into Gs, which is free now), or W
    const float2* Vn = Ws;
    if (use_warm) {
        for (int e = sl; e < KK; e += LANES) {
            const int i = e / KP, k = e - i * KP;
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < KP; ++l) s = cadd(s, cmul(Vs[i * KP + l], Ws[l * KP + k]));
            Gs[e] = s;
        }
        Vn = Gs;
        __syncwarp();
    }
    // sigma_k = ||A v_k||, column by column of B = A V (B is not kept)
    float f[KP];
    float nsum = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        float2 bk[R];
#pragma unroll
        for (int r = 0; r < R; ++r) bk[r] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < KP; ++l) {
            const float2 v = Vn[l * KP + k];
#pragma unroll
            for (int r = 0; r < R; ++r) bk[r] = cadd(bk[r], cmul(a[r][l], v));
        }
        float s2 = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) s2 += cabs2(bk[r]);
        const float sg = sqrtf(lane_sum<LANES>(s2));
        nsum += sg;
        f[k] = sg > tau ? (sg - tau) / sg : 0.f;
    }
    if (nuc && active && sl == 0) nuc[j] = (double)nsum;     // the patch's share, summed in order later
    if (stats) {
        // block totals first: one atomic pair per block instead of per patch
        __shared__ unsigned s_sweeps, s_rots;
        if (threadIdx.x == 0) { s_sweeps = 0u; s_rots = 0u; }
        __syncthreads();
        if (active && sl == 0) atomicAdd(&s_sweeps, (unsigned)nsweep);
        if (active && nrot) atomicAdd(&s_rots, (unsigned)nrot);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&stats[0], (unsigned long long)s_sweeps);
            atomicAdd(&stats[1], (unsigned long long)s_rots);
        }
    }
    if (Vio && active)
        for (int e = sl; e < KK; e += LANES) Vio[(size_t)j * KK + e] = Vn[e];
    if (!P) return;
    // P = B diag(f) V^H = A M with M = V diag(f) V^H (its first K columns),
    // built in Vs (free once V is known); only columns with f_k > 0 enter
    float2* Ms = Vs;
    for (int e = sl; e < KP * K; e += LANES) {
        const int l = e / K, kq = e - l * K;
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KP; ++k)
            if (f[k] > 0.f) s = cadd(s, cscale(cmulc(Vn[l * KP + k], Vn[kq * KP + k]), f[k]));
        Ms[l * K + kq] = s;
    }
    __syncwarp();
    for (int kq = 0; kq < K; ++kq) {
        float2 acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < KP; ++l) {
            const float2 m = Ms[l * K + kq];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = cadd(acc[r], cmul(a[r][l], m));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = sl + LANES * r;
            if (active && row < pp) P[((size_t)j * pp + row) * K + kq] = acc[r];
        }
    }
}

}  // namespace mrf

// Multi-frame Kaiser-Bessel NUFFT: the acquisition operator A = F_u of Eq. 1
// (one coil) and its adjoint, for all T frames of an MRF series.
//
// Forward, per frame:  deapodise + zero-pad + FFT along x   (k_rows_fwd)
//                      FFT along y + KB interpolation       (k_cols_interp)
// Adjoint, per frame:  KB spread + inverse FFT along y      (k_spread_cols)
//                      inverse FFT along x + crop + deapod  (k_rows_adj)
//
// The oversampled grid G x G of a frame is never written to HBM: the column
// kernels own a 16-column strip of the frame in shared memory ([G][16], 64 KB
// at G = 512, so three blocks share an SM and one block's loads overlap
// another's transforms), transform it there and interpolate (or spread) the
// samples binned to that strip.  A forward strip owns 16 - (W - 1) columns
// and carries W - 1 halo columns so each sample's W x W nodes are in the
// tile; an adjoint strip owns all 16 columns and a sample that straddles two
// strips is spread by both.  Only the half-oversampled intermediate
// H1 [T][ny][G] (rows transformed along x) goes through memory.  Row kernels
// transform 16 rows per block in a [16][G + 1] tile (odd row stride, one row
// per lane).  Samples are binned on the host when the plan is built; frames
// with identical sample positions share one binned copy.
//
// Kernel: psi(u) = I0(beta sqrt(1 - (2u/W)^2)), |u| <= W/2, with Beatty's
// beta = pi sqrt((W/os)^2 (os - 1/2)^2 - 0.8); deapodisation divides by its
// continuous Fourier transform W sinh(z)/z, z = sqrt(beta^2 - (pi W f)^2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "common.h"
#include "fft.cuh"
#include "nufft_plan.h"

namespace mrf {

constexpr int kTile = 16;        // columns per strip tile (64 KB at G = 512: three blocks per SM)
constexpr int kColThreads = 256; // threads of the strip kernels
constexpr int kRowB = 16;        // rows (or frames) per row-kernel block
constexpr int kRowThreads = 256; // threads of the row kernels
// elements of the row kernels' [kRowB][G + 1] row tile, enlarged at grid 512
// to hold the four-step transform's exchange buffer
__host__ __device__ constexpr int row_region(int G) {
    return G == 512 && kRow512Buf > kRowB * (G + 1) ? kRow512Buf : kRowB * (G + 1);
}

template <int W>
__device__ __forceinline__ void kb_weights(float f, float beta, float* w) {
#pragma unroll
    for (int a = 0; a < W; ++a) {
        const float z = 2.0f * (f - (float)a) / (float)W;
        w[a] = cyl_bessel_i0f(beta * sqrtf(fmaxf(0.0f, 1.0f - z * z)));
    }
}

__device__ __forceinline__ void unpack(const int4 r, int& j, int& mx0, int& my0, float& fx, float& fy) {
    j = r.x;
    mx0 = r.y & 0xffff;
    my0 = (r.y >> 16) & 0xffff;
    fx = __int_as_float(r.z);
    fy = __int_as_float(r.w);
}

// KB weights of every strip record, computed once per plan (they depend on
// the trajectory only): w[i][0..W) along x, w[i][W..2W) along y
template <int W>
__global__ void k_rec_weights(const int4* __restrict__ rec, int n, float beta, float* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j, mx0, my0;
    float fx, fy;
    unpack(rec[i], j, mx0, my0, fx, fy);
    float wx[W], wy[W];
    kb_weights<W>(fx, beta, wx);
    kb_weights<W>(fy, beta, wy);
#pragma unroll
    for (int a = 0; a < W; ++a) {
        w[(size_t)i * 2 * W + a] = wx[a];
        w[(size_t)i * 2 * W + W + a] = wy[a];
    }
}

// the stored weights of record i (2 W floats, 16-byte aligned: W = 4 or 6)
template <int W>
__device__ __forceinline__ void load_weights(const float* __restrict__ w, int i, float (&wx)[W], float (&wy)[W]) {
    const float4* q = reinterpret_cast<const float4*>(w) + (size_t)i * (W / 2);
    float v[2 * W];
#pragma unroll
    for (int c = 0; c < W / 2; ++c) {
        const float4 f = q[c];
        v[4 * c] = f.x;
        v[4 * c + 1] = f.y;
        v[4 * c + 2] = f.z;
        v[4 * c + 3] = f.w;
    }
#pragma unroll
    for (int a = 0; a < W; ++a) {
        wx[a] = v[a];
        wy[a] = v[W + a];
    }
}

// centred coordinate held at grid index g
template <int G>
__device__ __forceinline__ int centred(int g) { return g < G / 2 ? g : g - G; }

// Block-wide global -> shared staging: element i in [0, n) is produced by
// ld(i) (a global load, or zero) and stored by st(i, v); each thread issues
// U loads before its U stores, so U loads per thread are in flight at once
// instead of one load-to-store round trip per element.
template <int U, typename Ld, typename St>
__device__ __forceinline__ void stage_block(int n, Ld ld, St st) {
    for (int b = threadIdx.x; b < n; b += U * (int)blockDim.x) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = b + u * (int)blockDim.x;
            v[u] = i < n ? ld(i) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = b + u * (int)blockDim.x;
            if (i < n) st(i, v[u]);
        }
    }
}

// v mod G in [0, G) (grids of 2^a or 3 x 2^a points)
template <int G>
__device__ __forceinline__ int wrapg(int v) {
    if constexpr ((G & (G - 1)) == 0) {
        return v & (G - 1);
    } else {
        const int r = v % G;
        return r < 0 ? r + G : r;
    }
}

// ---------------------------------------------------------------------------
// Forward stage 1: rows.  SRC 0: frames x[t][iy][ix]; SRC 1: coefficient image
// k of alpha[iy][ix][K] (blockIdx.y = k).  Block: 16 rows of one frame.
// ---------------------------------------------------------------------------
template <int G, int SRC>
__global__ void __launch_bounds__(kRowThreads) k_rows_fwd(const float2* __restrict__ x, int K,
                                                          float2* __restrict__ h1,
                                                          const float* __restrict__ inv_dx,
                                                          const float* __restrict__ inv_dy, int nx, int ny) {
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* rows = sm + G;                        // [kRowB][G + 1]
    constexpr int LD = G + 1;
    const int t = blockIdx.y;
    const int iy0 = blockIdx.x * kRowB;
    auto value = [&](int iy, int g) {
        const int ix = centred<G>(g) + nx / 2;
        float2 v = make_float2(0.f, 0.f);
        if (iy < ny && ix >= 0 && ix < nx) {
            v = SRC == 0 ? x[((size_t)t * ny + iy) * nx + ix] : x[((size_t)iy * nx + ix) * K + t];
            v = cscale(v, inv_dx[ix] * inv_dy[iy]);
        }
        return v;
    };
    if constexpr (G == 512) {
        // row r's elements tq + 16 m straight into registers, the four-step
        // transform, the spectrum straight out of them
        const int tq = threadIdx.x & 15, r = threadIdx.x >> 4, iy = iy0 + r;
        row512_twiddles(tw);
        float2 xr[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) xr[m] = value(iy, tq + 16 * m);
        __syncthreads();                                // the twiddle table
        float2 out[2][16];
        row512<false>(xr, rows, tw, out);
        if (iy < ny) {
            float2* dst = h1 + ((size_t)t * ny + iy) * G;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) dst[(tq + 16 * j) + 32 * k2] = out[j][k2];
        }
    } else {
        fft_twiddles<G>(tw);
        stage_block<8>(
            kRowB * G, [&](int idx) { return value(iy0 + idx / G, idx % G); },
            [&](int idx, float2 v) { rows[(idx / G) * LD + idx % G] = v; });
        __syncthreads();
        fft_batch<G, kRowB, kRowThreads, false>(rows, 1, LD, tw);
        for (int idx = threadIdx.x; idx < kRowB * G; idx += kRowThreads) {
            const int r = idx / G, g = idx - r * G;
            const int iy = iy0 + r;
            if (iy < ny) h1[((size_t)t * ny + iy) * G + g] = rows[r * LD + g];
        }
    }
}

// Forward stage 1 in subspace form: frame t row iy is sum_k alpha[iy][ix][k]
// conj(phi[t][k]).  Block = one image row x 16 frames.
template <int G>
__global__ void __launch_bounds__(kRowThreads, 3) k_rows_fwd_expand(const float2* __restrict__ alpha,
                                                                 const float2* __restrict__ phi, int K, int T,
                                                                 float2* __restrict__ h1,
                                                                 const float* __restrict__ inv_dx,
                                                                 const float* __restrict__ inv_dy, int nx,
                                                                 int ny) {
    extern __shared__ float2 sm[];
    constexpr int LD = G + 1;
    float2* tw = sm;                       // (grid 512: the four-step table, row512_twiddles)
    float2* rows = sm + G;                 // [kRowB][G + 1]
    float2* ph = rows + row_region(G);     // [kRowB][K]
    const int iy = blockIdx.x;
    const int t0 = blockIdx.y * kRowB;
    if constexpr (G == 512) row512_twiddles(tw);
    else fft_twiddles<G>(tw);
    for (int i = threadIdx.x; i < kRowB * K; i += kRowThreads) {
        const int tt = t0 + i / K;
        ph[i] = tt < T ? phi[(size_t)tt * K + (i % K)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float sy = inv_dy[iy];
    // a thread per grid column: the pixel's K coefficients in registers, the
    // 16 frames' basis rows read as shared-memory broadcasts
    for (int g = threadIdx.x; g < G; g += kRowThreads) {
        const int ix = centred<G>(g) + nx / 2;
        if (ix < 0 || ix >= nx) {
#pragma unroll
            for (int r = 0; r < kRowB; ++r) rows[r * LD + g] = make_float2(0.f, 0.f);
            continue;
        }
        // (read once from the coefficient image: the row's 20 KB stay in L1)
        const float2* arow = alpha + ((size_t)iy * nx + ix) * K;
        float2 a[16];                                   // K <= 16 (unrolled: stays in registers)
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = k < K ? arow[k] : make_float2(0.f, 0.f);
        const float sc = inv_dx[ix] * sy;
#pragma unroll 4
        for (int r = 0; r < kRowB; ++r) {
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < K) v = cadd(v, cmulc(a[k], ph[r * K + k]));
            rows[r * LD + g] = t0 + r < T ? cscale(v, sc) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    if constexpr (G == 512) {
        // frame row r's elements t + 16 m into registers, the four-step
        // transform, the spectrum straight from registers to H1
        static_assert(kRowB == 16 && kRowThreads == 256, "the four-step form maps 256 threads to 16 rows");
        const int t = threadIdx.x & 15, r = threadIdx.x >> 4;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) x[m] = rows[r * LD + t + 16 * m];
        __syncthreads();                                // every row read before the exchange reuses them
        float2 out[2][16];
        row512<false>(x, rows, tw, out);
        if (t0 + r < T) {
            float2* dst = h1 + ((size_t)(t0 + r) * ny + iy) * G;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) dst[(t + 16 * j) + 32 * k2] = out[j][k2];
        }
    } else {
        fft_batch<G, kRowB, kRowThreads, false>(rows, 1, LD, tw);
        for (int idx = threadIdx.x; idx < kRowB * G; idx += kRowThreads) {
            const int r = idx / G, g = idx - r * G;
            if (t0 + r < T) h1[((size_t)(t0 + r) * ny + iy) * G + g] = rows[r * LD + g];
        }
    }
}

// Load a strip (TILE columns starting at c0, wrapping) of one image's H1 into
// the shared tile [G][TILE]; rows outside the image's support are zero.
template <int G, int TILE = kTile>
__device__ __forceinline__ void load_strip(float2* tile, const float2* __restrict__ h1f, int c0, int ny) {
    stage_block<4>(
        G * TILE,
        [&](int idx) {
            const int gy = idx / TILE, c = idx & (TILE - 1);
            const int iy = centred<G>(gy) + ny / 2;
            return (iy >= 0 && iy < ny) ? h1f[(size_t)iy * G + wrapg<G>(c0 + c)] : make_float2(0.f, 0.f);
        },
        [&](int idx, float2 v) { tile[idx] = v; });
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Forward stage 2: FFT of a strip's columns in shared memory, then KB
// interpolation of the samples whose first x-node falls in the strip's owned
// columns.  y = scale * interp - b  (b nullable).
// ---------------------------------------------------------------------------
template <int G, int W>
__global__ void __launch_bounds__(kColThreads, G == 512 ? 2 : 3) k_cols_interp(const float2* __restrict__ h1,
                                                             float2* __restrict__ y,
                                                             const float2* __restrict__ bsub, float scale,
                                                             const int4* __restrict__ rec,
                                                             const float* __restrict__ wts,
                                                             const int* __restrict__ off,
                                                             const int* __restrict__ group_of, int ny, int ns,
                                                             int nstrips) {
    constexpr int SF = kTile - (W - 1);
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tile = sm + G;
    const int strip = blockIdx.x, t = blockIdx.y;
    const int c0 = strip * SF;
    fft_twiddles<G>(tw);
    if constexpr (G == 512) {
        // the strip's columns straight into registers (rows t' + 16 m of
        // column c), the four-step transform, the spectrum into the tile
        static_assert(kTile == 16 && kColThreads == 256, "the four-step form maps 256 threads to 16 columns");
        const int c = threadIdx.x & 15, tq = threadIdx.x >> 4;
        const float2* h1f = h1 + (size_t)t * ny * G;
        const int col = wrapg<G>(c0 + c);
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int iy = centred<G>(tq + 16 * m) + ny / 2;
            x[m] = (iy >= 0 && iy < ny) ? h1f[(size_t)iy * G + col] : make_float2(0.f, 0.f);
        }
        __syncthreads();                                // the twiddle table
        float2 out[2][16];
        col512<false>(x, tile, tw, out);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) tile[((2 * tq + j) + 32 * k2) * kTile + c] = out[j][k2];
        __syncthreads();
    } else {
        load_strip<G>(tile, h1 + (size_t)t * ny * G, c0, ny);
        fft_batch<G, kTile, kColThreads, false>(tile, kTile, 1, tw);
    }
    const int g = group_of[t];
    const int beg = off[g * nstrips + strip], end = off[g * nstrips + strip + 1];
    for (int i = beg + threadIdx.x; i < end; i += kColThreads) {
        int j, mx0, my0;
        float fx, fy;
        unpack(rec[i], j, mx0, my0, fx, fy);
        float wx[W], wy[W];
        load_weights<W>(wts, i, wx, wy);
        const int lc = mx0 - c0;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2* tr = tile + (wrapg<G>(my0 + b)) * kTile + lc;
            float2 rs = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < W; ++a) rs = cadd(rs, cscale(tr[a], wx[a]));
            acc = cadd(acc, cscale(rs, wy[b]));
        }
        acc = cscale(acc, scale);
        const size_t o = (size_t)t * ns + j;
        if (bsub) acc = csub(acc, bsub[o]);
        y[o] = acc;
    }
}

// Column FFTs of whole images, spectrum written out (grouped subspace form).
// Strips of TILE columns (16 workers per column: TILE * 16 threads); the
// width is chosen per plan by tune_cols.
template <int G, int TILE>
__global__ void __launch_bounds__(TILE * 16) k_cols_store(const float2* __restrict__ h1,
                                                         float2* __restrict__ spec, int ny) {
    constexpr int NT = TILE * 16;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tile = sm + G;
    const int strip = blockIdx.x, f = blockIdx.y;
    const int c0 = strip * TILE;
    fft_twiddles<G>(tw);
    float2* dst = spec + (size_t)f * G * G;
    if constexpr (G == 512 && TILE == 16) {
        // register-resident four-step transform: the image's columns straight
        // into registers, the spectrum straight out of them
        const int c = threadIdx.x & 15, tq = threadIdx.x >> 4;
        const float2* h1f = h1 + (size_t)f * ny * G;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int iy = centred<G>(tq + 16 * m) + ny / 2;
            x[m] = (iy >= 0 && iy < ny) ? h1f[(size_t)iy * G + c0 + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();                                // the twiddle table
        float2 out[2][16];
        col512<false>(x, tile, tw, out);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) dst[(size_t)((2 * tq + j) + 32 * k2) * G + c0 + c] = out[j][k2];
    } else {
        load_strip<G, TILE>(tile, h1 + (size_t)f * ny * G, c0, ny);
        fft_batch<G, TILE, NT, false>(tile, TILE, 1, tw);
        for (int idx = threadIdx.x; idx < G * TILE; idx += NT) {
            const int gy = idx / TILE, c = idx & (TILE - 1);
            dst[(size_t)gy * G + c0 + c] = tile[idx];
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint stage 1: spread the samples touching a strip into a shared tile
// (shared-memory atomics), inverse FFT of the strip's columns, keep the image
// rows.  SRC 0: y[t][j] per frame (blockIdx.y = t);  SRC 1: grouped values
// R[g][j][k] of every group (blockIdx.y = k).
// ---------------------------------------------------------------------------
template <int G, int W, int SRC>
__global__ void __launch_bounds__(kColThreads, 3) k_spread_cols(const float2* __restrict__ y, int K,
                                                             float2* __restrict__ h1,
                                                             const int4* __restrict__ rec,
                                                             const float* __restrict__ wts,
                                                             const int* __restrict__ off,
                                                             const int* __restrict__ group_of, int ngroups,
                                                             int ny, int ns, int nstrips) {
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tile = sm + G;                 // [G][kTile]
    const int strip = blockIdx.x, f = blockIdx.y;
    const int c0 = strip * kTile;
    fft_twiddles<G>(tw);
    for (int i = threadIdx.x; i < G * kTile; i += kColThreads) tile[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int g_lo = SRC == 0 ? group_of[f] : 0;
    const int g_hi = SRC == 0 ? g_lo + 1 : ngroups;
    for (int g = g_lo; g < g_hi; ++g) {
        const int beg = off[g * nstrips + strip], end = off[g * nstrips + strip + 1];
        for (int i = beg + threadIdx.x; i < end; i += kColThreads) {
            int j, mx0, my0;
            float fx, fy;
            unpack(rec[i], j, mx0, my0, fx, fy);
            const float2 v = SRC == 0 ? y[(size_t)f * ns + j] : y[((size_t)g * ns + j) * K + f];
            float wx[W], wy[W];
            load_weights<W>(wts, i, wx, wy);
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const int lc = (wrapg<G>(mx0 + a)) - c0;
                if (lc < 0 || lc >= kTile) continue;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    float2* p = tile + (wrapg<G>(my0 + b)) * kTile + lc;
                    const float w = wx[a] * wy[b];
                    atomicAdd(&p->x, w * v.x);
                    atomicAdd(&p->y, w * v.y);
                }
            }
        }
    }
    __syncthreads();
    // (the register-resident four-step transform of the strip kernels at grid
    // 512 needs 128 registers here, which halves the blocks per SM; the
    // spread phase's shared-memory atomics need them more than the transform
    // gains: measured 1.11 against 1.04 ms per 1000 frames)
    fft_batch<G, kTile, kColThreads, true>(tile, kTile, 1, tw);
    float2* dst = h1 + (size_t)f * ny * G;
    for (int idx = threadIdx.x; idx < ny * kTile; idx += kColThreads) {
        const int iy = idx / kTile, c = idx & (kTile - 1);
        const int gy = wrapg<G>(iy - ny / 2);
        dst[(size_t)iy * G + c0 + c] = tile[gy * kTile + c];
    }
}

// Frame-form adjoint stage 1 as a sorted gather: the strip's (point, sample,
// weight) entries of its frame's interleaf group, ordered by point.  Each
// thread reduces a run of kSpRun consecutive entries and adds a partial sum
// to the tile only where the point changes, so the crowded k-space centre
// costs a few shared-memory adds instead of contended atomics per tap.  Then
// the inverse FFT of the strip's columns and the image rows, as k_spread_cols.
constexpr int kSpRun = 8;

template <int G>
__global__ void __launch_bounds__(kColThreads, G == 512 ? 2 : 3) k_spread_gather(const float2* __restrict__ y,
                                                               float2* __restrict__ h1,
                                                               const int* __restrict__ loc,
                                                               const int* __restrict__ smp,
                                                               const float* __restrict__ w,
                                                               const int* __restrict__ off,
                                                               const int* __restrict__ group_of, int ny, int ns,
                                                               int nstrips) {
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tile = sm + G;                 // [G][kTile]
    float* tf = reinterpret_cast<float*>(tile);
    const int strip = blockIdx.x, f = blockIdx.y;
    const int c0 = strip * kTile;
    fft_twiddles<G>(tw);
    for (int i = threadIdx.x; i < G * kTile; i += kColThreads) tile[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int g = group_of[f];
    const int beg = off[g * nstrips + strip], end = off[g * nstrips + strip + 1];
    const float2* yf = y + (size_t)f * ns;
    for (int b = beg + threadIdx.x * kSpRun; b < end; b += kColThreads * kSpRun) {
        const int e = min(b + kSpRun, end);
        int cur = loc[b];
        float2 acc = make_float2(0.f, 0.f);
        for (int i = b; i < e; ++i) {
            const int p = loc[i];
            if (p != cur) {
                atomicAdd(&tf[2 * cur], acc.x);
                atomicAdd(&tf[2 * cur + 1], acc.y);
                acc = make_float2(0.f, 0.f);
                cur = p;
            }
            const float2 v = yf[smp[i]];
            const float wi = w[i];
            acc.x += wi * v.x;
            acc.y += wi * v.y;
        }
        atomicAdd(&tf[2 * cur], acc.x);
        atomicAdd(&tf[2 * cur + 1], acc.y);
    }
    __syncthreads();
    float2* dst = h1 + (size_t)f * ny * G;
    if constexpr (G == 512) {
        // the tile's columns into registers, the register-resident four-step
        // inverse transform, the image rows straight out of registers
        const int c = threadIdx.x & 15, tq = threadIdx.x >> 4;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) x[m] = tile[(tq + 16 * m) * kTile + c];
        __syncthreads();                                // every read of the tile before it is reused
        float2 out[2][16];
        col512<true>(x, tile, tw, out);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int iy = centred<G>((2 * tq + j) + 32 * k2) + ny / 2;
                if (iy >= 0 && iy < ny) dst[(size_t)iy * G + c0 + c] = out[j][k2];
            }
    } else {
        fft_batch<G, kTile, kColThreads, true>(tile, kTile, 1, tw);
        for (int idx = threadIdx.x; idx < ny * kTile; idx += kColThreads) {
            const int iy = idx / kTile, c = idx & (kTile - 1);
            const int gy = wrapg<G>(iy - ny / 2);
            dst[(size_t)iy * G + c0 + c] = tile[gy * kTile + c];
        }
    }
}

// Grouped adjoint stage 1 without same-address contention: the contributions
// of every group sample to the oversampled grid are precomputed as
// (grid point, sample, weight) entries sorted by point.  Each thread reduces
// a run of RUN consecutive entries for all K coefficient grids at once and
// adds a partial sum to the grid only where the point changes, so the k-space
// centre (where every interleaf overlaps) costs a few adds instead of
// thousands of same-address atomics.  R: [ngroups * ns][K]; grid: [K][G][G]
// (zeroed by the caller).  The run length and block size are tuned per plan
// (tune_gather): longer runs mean fewer atomics, shorter runs more parallelism.
template <int RUN>
__global__ void k_gather_grid(const float2* __restrict__ R, int K, const int* __restrict__ pt,
                              const int* __restrict__ smp, const float* __restrict__ w, int nent, int GG2,
                              float2* __restrict__ grid) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) * RUN;
    if (b >= nent) return;
    const int e = min(nent, b + RUN);
    float2 acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
    int cur = pt[b];
    for (int i = b; i < e; ++i) {
        const int p = pt[i];
        if (p != cur) {
            // (loops over K unrolled to the 16-entry bound: acc stays in registers)
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (k < K) {
                    atomicAdd(&grid[(size_t)k * GG2 + cur].x, acc[k].x);
                    atomicAdd(&grid[(size_t)k * GG2 + cur].y, acc[k].y);
                }
                acc[k] = make_float2(0.f, 0.f);
            }
            cur = p;
        }
        const float wi = w[i];
        const float2* r = R + (size_t)smp[i] * K;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < K) acc[k] = cadd(acc[k], cscale(r[k], wi));
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k < K) {
            atomicAdd(&grid[(size_t)k * GG2 + cur].x, acc[k].x);
            atomicAdd(&grid[(size_t)k * GG2 + cur].y, acc[k].y);
        }
    }
}

// Warp-cooperative form of the same gather: lane i of a warp takes entry
// 32 w + i (all 32 sample rows are requested at once), the lanes holding the
// same grid point (consecutive, the table being sorted by point) add their
// contributions with a segmented shuffle scan, and the last lane of each
// segment adds the segment's sum to the grid (one float2 atomic per
// coefficient).  Lanes past the table get distinct negative points.
__global__ void __launch_bounds__(512) k_gather_warp(const float2* __restrict__ R, int K, const int* __restrict__ pt,
                                                     const int* __restrict__ smp, const float* __restrict__ w,
                                                     int nent, int GG2, float2* __restrict__ grid) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = e < (size_t)nent;
    const int p = valid ? pt[e] : -1 - lane;
    float2 c[16];
    if (valid) {
        const float wi = w[e];
        const float2* r = R + (size_t)smp[e] * K;
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = k < K ? cscale(r[k], wi) : make_float2(0.f, 0.f);
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int po = __shfl_up_sync(0xffffffffu, p, off);
        const bool take = lane >= off && po == p;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < K) {
                const float ox = __shfl_up_sync(0xffffffffu, c[k].x, off);
                const float oy = __shfl_up_sync(0xffffffffu, c[k].y, off);
                if (take) { c[k].x += ox; c[k].y += oy; }
            }
        }
    }
    const int pn = __shfl_down_sync(0xffffffffu, p, 1);
    if (valid && (lane == 31 || pn != p)) {
#pragma unroll
        for (int k = 0; k < 16; ++k)             // (unrolled: c stays in registers)
            if (k < K) atomicAdd(&grid[(size_t)k * GG2 + p], c[k]);
    }
}

// Inverse FFT of a strip's columns of grid image f, image rows kept (strips
// of TILE columns, TILE * 16 threads, as k_cols_store).
template <int G, int TILE>
__global__ void __launch_bounds__(TILE * 16) k_cols_inv(const float2* __restrict__ grid,
                                                       float2* __restrict__ h1, int ny) {
    constexpr int NT = TILE * 16;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* tile = sm + G;
    const int strip = blockIdx.x, f = blockIdx.y;
    const int c0 = strip * TILE;
    fft_twiddles<G>(tw);
    const float2* src = grid + (size_t)f * G * G;
    float2* dst = h1 + (size_t)f * ny * G;
    if constexpr (G == 512 && TILE == 16) {
        // register-resident four-step inverse transform: the grid's columns
        // straight into registers, the image rows straight out of them
        const int c = threadIdx.x & 15, tq = threadIdx.x >> 4;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) x[m] = src[(size_t)(tq + 16 * m) * G + c0 + c];
        __syncthreads();                                // the twiddle table
        float2 out[2][16];
        col512<true>(x, tile, tw, out);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int iy = centred<G>((2 * tq + j) + 32 * k2) + ny / 2;
                if (iy >= 0 && iy < ny) dst[(size_t)iy * G + c0 + c] = out[j][k2];
            }
    } else {
        stage_block<4>(
            G * TILE, [&](int idx) { return src[(size_t)(idx / TILE) * G + c0 + (idx & (TILE - 1))]; },
            [&](int idx, float2 v) { tile[idx] = v; });
        __syncthreads();
        fft_batch<G, TILE, NT, true>(tile, TILE, 1, tw);
        for (int idx = threadIdx.x; idx < ny * TILE; idx += NT) {
            const int iy = idx / TILE, c = idx & (TILE - 1);
            const int gy = wrapg<G>(iy - ny / 2);
            dst[(size_t)iy * G + c0 + c] = tile[gy * TILE + c];
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint stage 2: inverse FFT along x, crop, deapodise.  DST 0: frames
// x[t][iy][ix]; DST 1: coefficient image k, alpha[iy][ix][K] (times scale).
// ---------------------------------------------------------------------------
template <int G, int DST>
__global__ void __launch_bounds__(kRowThreads) k_rows_adj(const float2* __restrict__ h1, float2* __restrict__ x,
                                                          int K, float scale, const float* __restrict__ inv_dx,
                                                          const float* __restrict__ inv_dy, int nx, int ny) {
    extern __shared__ float2 sm[];
    constexpr int LD = G + 1;
    float2* tw = sm;
    float2* rows = sm + G;
    const int t = blockIdx.y;
    const int iy0 = blockIdx.x * kRowB;
    if constexpr (G == 512) {
        // row r's elements tq + 16 m straight into registers, the four-step
        // inverse transform, the image's columns straight out of them
        const int tq = threadIdx.x & 15, r = threadIdx.x >> 4, iy = iy0 + r;
        row512_twiddles(tw);
        float2 xr[32];
        const float2* src = h1 + ((size_t)t * ny + iy) * G;
#pragma unroll
        for (int m = 0; m < 32; ++m) xr[m] = iy < ny ? src[tq + 16 * m] : make_float2(0.f, 0.f);
        __syncthreads();                                // the twiddle table
        float2 out[2][16];
        row512<true>(xr, rows, tw, out);
        if (iy < ny) {
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) {
                    const int ix = centred<G>((tq + 16 * j) + 32 * k2) + nx / 2;
                    if (ix < 0 || ix >= nx) continue;
                    const float2 v = cscale(out[j][k2], inv_dx[ix] * inv_dy[iy] * scale);
                    if (DST == 0) x[((size_t)t * ny + iy) * nx + ix] = v;
                    else x[((size_t)iy * nx + ix) * K + t] = v;
                }
        }
    } else {
        fft_twiddles<G>(tw);
        stage_block<8>(
            kRowB * G,
            [&](int idx) {
                const int iy = iy0 + idx / G;
                return iy < ny ? h1[((size_t)t * ny + iy) * G + idx % G] : make_float2(0.f, 0.f);
            },
            [&](int idx, float2 v) { rows[(idx / G) * LD + idx % G] = v; });
        __syncthreads();
        fft_batch<G, kRowB, kRowThreads, true>(rows, 1, LD, tw);
        for (int idx = threadIdx.x; idx < kRowB * nx; idx += kRowThreads) {
            const int r = idx / nx, ix = idx - r * nx;
            const int iy = iy0 + r;
            if (iy >= ny) continue;
            const float2 v = cscale(rows[r * LD + (wrapg<G>(ix - nx / 2))], inv_dx[ix] * inv_dy[iy] * scale);
            if (DST == 0) x[((size_t)t * ny + iy) * nx + ix] = v;
            else x[((size_t)iy * nx + ix) * K + t] = v;
        }
    }
}

// Adjoint stage 2 in subspace form: partial[p][iy][ix][k] = sum over the
// frames t of part p of (A^H y)_t[iy][ix] phi[t][k].  Block = one image row,
// 16 frames per inner step.
template <int G>
__global__ void __launch_bounds__(kRowThreads, 2) k_rows_adj_reduce(const float2* __restrict__ h1,
                                                                 const float2* __restrict__ phi, int K, int T,
                                                                 int frames_per_part,
                                                                 float2* __restrict__ partial,
                                                                 const float* __restrict__ inv_dx,
                                                                 const float* __restrict__ inv_dy, int nx,
                                                                 int ny) {
    constexpr int LD = G + 1;
    constexpr int MAXK = 16;               // a thread per image column ix (nx <= 256), all K <= 16 coefficients
    extern __shared__ float2 sm[];
    float2* tw = sm;                       // (grid 512: the four-step table, row512_twiddles)
    float2* rows = sm + G;                 // [kRowB][G + 1]
    float2* ph = rows + row_region(G);     // [kRowB][K]
    const int iy = blockIdx.x, part = blockIdx.y;
    const int tb = part * frames_per_part;
    const int te = min(T, tb + frames_per_part);
    if constexpr (G == 512) row512_twiddles(tw);
    else fft_twiddles<G>(tw);
    float2 acc[MAXK];
#pragma unroll
    for (int q = 0; q < MAXK; ++q) acc[q] = make_float2(0.f, 0.f);
    const int ix = threadIdx.x;
    const int gx = wrapg<G>(ix - nx / 2);
    const float sy = inv_dy[iy];
    for (int t0 = tb; t0 < te; t0 += kRowB) {
        if constexpr (G == 512) {
            // frame row r's elements t + 16 m straight into registers, the
            // four-step inverse transform, the image's columns back into the
            // row tile for the reduction
            static_assert(kRowB == 16 && kRowThreads == 256, "the four-step form maps 256 threads to 16 rows");
            const int t = threadIdx.x & 15, r = threadIdx.x >> 4;
            float2 x[32];
            const float2* src = h1 + ((size_t)(t0 + r) * ny + iy) * G;
#pragma unroll
            for (int m = 0; m < 32; ++m) x[m] = t0 + r < te ? src[t + 16 * m] : make_float2(0.f, 0.f);
            for (int i = threadIdx.x; i < kRowB * K; i += kRowThreads) {
                const int tt = t0 + i / K;
                ph[i] = tt < te ? phi[(size_t)tt * K + (i % K)] : make_float2(0.f, 0.f);
            }
            __syncthreads();                            // the twiddle table (first pass)
            float2 out[2][16];
            row512<true>(x, rows, tw, out);
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) {
                    const int g = (t + 16 * j) + 32 * k2;
                    const int cx = centred<G>(g) + nx / 2;
                    if (cx >= 0 && cx < nx) rows[r * LD + g] = out[j][k2];
                }
            __syncthreads();
        } else {
            stage_block<8>(
                kRowB * G,
                [&](int idx) {
                    const int r = idx / G;
                    return t0 + r < te ? h1[((size_t)(t0 + r) * ny + iy) * G + idx % G] : make_float2(0.f, 0.f);
                },
                [&](int idx, float2 v) { rows[(idx / G) * LD + idx % G] = v; });
            for (int i = threadIdx.x; i < kRowB * K; i += kRowThreads) {
                const int tt = t0 + i / K;
                ph[i] = tt < te ? phi[(size_t)tt * K + (i % K)] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            fft_batch<G, kRowB, kRowThreads, true>(rows, 1, LD, tw);
        }
        const int nf = min(kRowB, te - t0);
        if (ix < nx) {
            // one load of the pixel's value per frame serves all K products;
            // the frame's basis row is a shared-memory broadcast
            for (int f = 0; f < nf; ++f) {
                const float2 rv = rows[f * LD + gx];
#pragma unroll
                for (int k = 0; k < MAXK; ++k)
                    if (k < K) acc[k] = cadd(acc[k], cmul(rv, ph[f * K + k]));
            }
        }
        __syncthreads();
    }
    if (ix < nx) {
        const float sc = inv_dx[ix] * sy;
#pragma unroll
        for (int k = 0; k < MAXK; ++k)
            if (k < K) partial[(((size_t)part * ny + iy) * nx + ix) * K + k] = cscale(acc[k], sc);
    }
}

__global__ void k_sum_parts(const float2* __restrict__ partial, int parts, size_t n, float scale,
                            float2* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int p = 0; p < parts; ++p) s = cadd(s, partial[p * n + i]);
        out[i] = cscale(s, scale);
    }
}

// Grouped subspace form ------------------------------------------------------
// Y[g][j][k] = interp of spectrum k at group g's sample j.
template <int G, int W>
__global__ void k_interp_groups(const float2* __restrict__ spec, int K, const int4* __restrict__ grec,
                                int total, float2* __restrict__ Y, float beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int j, mx0, my0;
    float fx, fy;
    unpack(grec[i], j, mx0, my0, fx, fy);
    float wx[W], wy[W];
    kb_weights<W>(fx, beta, wx);
    kb_weights<W>(fy, beta, wy);
    int col[W];
#pragma unroll
    for (int a = 0; a < W; ++a) col[a] = wrapg<G>(mx0 + a);
    for (int k = 0; k < K; ++k) {
        const float2* s = spec + (size_t)k * G * G;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2* r = s + (size_t)(wrapg<G>(my0 + b)) * G;
            float2 rs = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < W; ++a) rs = cadd(rs, cscale(r[col[a]], wx[a]));
            acc = cadd(acc, cscale(rs, wy[b]));
        }
        Y[(size_t)i * K + k] = acc;
    }
}

// y[t][j] = scale * sum_k conj(phi[t][k]) Y[g(t)][j][k] - b[t][j]
__global__ void k_combine_fwd(const float2* __restrict__ Y, const float2* __restrict__ phi, int K,
                              const int* __restrict__ group_of, int T, int ns, float scale,
                              const float2* __restrict__ bsub, float2* __restrict__ y) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)T * ns) return;
    const int t = (int)(i / ns), j = (int)(i - (size_t)t * ns);
    const float2* yv = Y + ((size_t)group_of[t] * ns + j) * K;
    const float2* p = phi + (size_t)t * K;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) acc = cadd(acc, cmulc(yv[k], p[k]));
    acc = cscale(acc, scale);
    if (bsub) acc = csub(acc, bsub[i]);
    y[i] = acc;
}

// R[g][j][k] = sum_{t in g} phi[t][k] r[t][j]
__global__ void k_combine_adj(const float2* __restrict__ r, const float2* __restrict__ phi, int K,
                              const int* __restrict__ gf_off, const int* __restrict__ gf, int ngroups, int ns,
                              float2* __restrict__ R) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)ngroups * ns) return;
    const int g = (int)(i / ns), j = (int)(i - (size_t)g * ns);
    float2 acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
    // four frames' samples loaded before they are added (in frame order)
    const int q1 = gf_off[g + 1];
    for (int q0 = gf_off[g]; q0 < q1; q0 += 4) {
        float2 v[4];
        int tt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            tt[u] = q0 + u < q1 ? gf[q0 + u] : 0;
            v[u] = q0 + u < q1 ? r[(size_t)tt[u] * ns + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (q0 + u >= q1) break;
            const float2* p = phi + (size_t)tt[u] * K;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < K) acc[k] = cadd(acc[k], cmul(v[u], p[k]));
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k)                 // (unrolled: acc stays in registers)
        if (k < K) R[i * K + k] = acc[k];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static double psi_hat(double f, int W, double beta) {
    const double z2 = beta * beta - (M_PI * W * f) * (M_PI * W * f);
    if (z2 > 0) {
        const double z = std::sqrt(z2);
        return W * std::sinh(z) / z;
    }
    if (z2 < 0) {
        const double z = std::sqrt(-z2);
        return W * std::sin(z) / z;
    }
    return W;
}

template <typename Kern>
static mrf_status set_smem(Kern kernel, size_t bytes) {
    MRF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return MRF_OK;
}

static bool supported_grid(int g) { return g == 64 || g == 128 || g == 256 || g == 384 || g == 512; }

#define MRF_DISPATCH_G(G_, ...)                                                          \
    switch (G_) {                                                                        \
        case 64: { constexpr int GG = 64; __VA_ARGS__; break; }                          \
        case 128: { constexpr int GG = 128; __VA_ARGS__; break; }                        \
        case 256: { constexpr int GG = 256; __VA_ARGS__; break; }                        \
        case 384: { constexpr int GG = 384; __VA_ARGS__; break; }                        \
        case 512: { constexpr int GG = 512; __VA_ARGS__; break; }                        \
        default: MRF_REQUIRE(false, "unsupported grid size %d", G_);                     \
    }

#define MRF_DISPATCH_W(W_, ...)                                                          \
    switch (W_) {                                                                        \
        case 4: { constexpr int WW = 4; __VA_ARGS__; break; }                            \
        case 6: { constexpr int WW = 6; __VA_ARGS__; break; }                            \
        default: MRF_REQUIRE(false, "unsupported kernel width %d", W_);                  \
    }

static size_t rows_smem(int G) { return (size_t)(G + row_region(G)) * sizeof(float2); }
static size_t tile_smem(int G) { return (size_t)(G + G * kTile) * sizeof(float2); }

mrf_status launch_rows_fwd(const mrf_plan_s* p, const float2* src, int src_mode, int K, int nf, float2* h1,
                           cudaStream_t s) {
    const int G = p->gx;
    dim3 grid((p->ny + kRowB - 1) / kRowB, nf);
    const size_t sm = rows_smem(G);
    MRF_DISPATCH_G(G, {
        if (src_mode == 0) {
            MRF_PROPAGATE(set_smem(k_rows_fwd<GG, 0>, sm));
            k_rows_fwd<GG, 0><<<grid, kRowThreads, sm, s>>>(src, K, h1, p->inv_dx, p->inv_dy, p->nx, p->ny);
        } else {
            MRF_PROPAGATE(set_smem(k_rows_fwd<GG, 1>, sm));
            k_rows_fwd<GG, 1><<<grid, kRowThreads, sm, s>>>(src, K, h1, p->inv_dx, p->inv_dy, p->nx, p->ny);
        }
    });
    MRF_LAUNCHED_AS("k_rows_fwd", s);
    return MRF_OK;
}

mrf_status launch_cols_interp(const mrf_plan_s* p, const float2* h1, float2* y, const float2* b, float scale,
                              cudaStream_t s) {
    const int G = p->gy;
    dim3 grid(p->nstrips_f, p->T);
    const size_t sm = tile_smem(G);
    MRF_DISPATCH_G(G, MRF_DISPATCH_W(p->W, {
        MRF_PROPAGATE(set_smem(k_cols_interp<GG, WW>, sm));
        k_cols_interp<GG, WW><<<grid, kColThreads, sm, s>>>(h1, y, b, scale, p->fwd_rec, p->fwd_w, p->fwd_off,
                                                            p->group_of, p->ny, p->ns, p->nstrips_f);
    }));
    MRF_LAUNCHED_AS("k_cols_interp", s);
    return MRF_OK;
}

// The frame-form spread's sorted entries (host, double-precision KB weights as
// the grouped gather table's), built once per plan; skipped (the atomic
// spread then runs) beyond kFspMaxEntries entries.
constexpr size_t kFspMaxEntries = (size_t)1 << 24;

static mrf_status build_frame_spread(mrf_plan_s* p, cudaStream_t s) {
    if (p->fsp_tried) return MRF_OK;
    p->fsp_tried = true;
    const int NG = p->ngroups, ns = p->ns, W = p->W, SAN = p->nstrips_a, G = p->gx;
    if ((size_t)NG * ns * W * W > kFspMaxEntries || G != p->gy) return MRF_OK;
    const double beta = p->beta_d;
    std::vector<int4> grec((size_t)NG * ns);
    MRF_CUDA(cudaMemcpyAsync(grec.data(), p->grec, sizeof(int4) * grec.size(), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    auto kb = [&](double u) {
        const double z = 2.0 * u / W;
        const double arg = std::max(0.0, 1.0 - z * z);
        return std::cyl_bessel_i(0.0, beta * std::sqrt(arg));
    };
    struct Ent { int key, loc, smp; float w; };
    std::vector<int> foff((size_t)NG * SAN + 1, 0);
    std::vector<int> floc, fsmp;
    std::vector<float> fw;
    floc.reserve((size_t)NG * ns * W * W);
    fsmp.reserve(floc.capacity());
    fw.reserve(floc.capacity());
    std::vector<Ent> ents;
    for (int g = 0; g < NG; ++g) {
        ents.clear();
        for (int j = 0; j < ns; ++j) {
            const int4 r = grec[(size_t)g * ns + j];
            const int mxw = r.y & 0xffff, myw = (r.y >> 16) & 0xffff;
            float fxf, fyf;
            std::memcpy(&fxf, &r.z, 4);
            std::memcpy(&fyf, &r.w, 4);
            for (int a = 0; a < W; ++a) {
                const int col = (mxw + a) % G;
                const double wa = kb((double)fxf - a);
                for (int b = 0; b < W; ++b) {
                    const int row = (myw + b) % G;
                    const int loc = row * kTile + (col % kTile);
                    ents.push_back({(col / kTile) * (G * kTile) + loc, loc, j, (float)(wa * kb((double)fyf - b))});
                }
            }
        }
        std::stable_sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) { return x.key < y.key; });
        for (const Ent& e : ents) {
            foff[(size_t)g * SAN + e.key / (G * kTile) + 1]++;
            floc.push_back(e.loc);
            fsmp.push_back(e.smp);
            fw.push_back(e.w);
        }
    }
    for (size_t i = 0; i + 1 < foff.size(); ++i) foff[i + 1] += foff[i];
    MRF_CUDA(cudaMalloc(&p->fsp_loc, sizeof(int) * std::max<size_t>(floc.size(), 1)));
    MRF_CUDA(cudaMalloc(&p->fsp_smp, sizeof(int) * std::max<size_t>(fsmp.size(), 1)));
    MRF_CUDA(cudaMalloc(&p->fsp_w, sizeof(float) * std::max<size_t>(fw.size(), 1)));
    MRF_CUDA(cudaMemcpy(p->fsp_loc, floc.data(), sizeof(int) * floc.size(), cudaMemcpyHostToDevice));
    MRF_CUDA(cudaMemcpy(p->fsp_smp, fsmp.data(), sizeof(int) * fsmp.size(), cudaMemcpyHostToDevice));
    MRF_CUDA(cudaMemcpy(p->fsp_w, fw.data(), sizeof(float) * fw.size(), cudaMemcpyHostToDevice));
    int* off = nullptr;
    MRF_CUDA(cudaMalloc(&off, sizeof(int) * foff.size()));
    MRF_CUDA(cudaMemcpy(off, foff.data(), sizeof(int) * foff.size(), cudaMemcpyHostToDevice));
    p->fsp_off = off;
    return MRF_OK;
}

mrf_status launch_spread_cols(mrf_plan_s* p, const float2* y, int src_mode, int K, int nf, float2* h1,
                              cudaStream_t s) {
    const int G = p->gy;
    dim3 grid(p->nstrips_a, nf);
    const size_t sm = tile_smem(G);
    if (src_mode == 0) {
        MRF_PROPAGATE(build_frame_spread(p, s));
        if (p->fsp_off) {
            MRF_DISPATCH_G(G, {
                MRF_PROPAGATE(set_smem(k_spread_gather<GG>, sm));
                k_spread_gather<GG><<<grid, kColThreads, sm, s>>>(y, h1, p->fsp_loc, p->fsp_smp, p->fsp_w, p->fsp_off,
                                                                 p->group_of, p->ny, p->ns, p->nstrips_a);
            });
            MRF_LAUNCHED_AS("k_spread_gather", s);
            return MRF_OK;
        }
    }
    MRF_DISPATCH_G(G, MRF_DISPATCH_W(p->W, {
        if (src_mode == 0) {
            MRF_PROPAGATE(set_smem(k_spread_cols<GG, WW, 0>, sm));
            k_spread_cols<GG, WW, 0><<<grid, kColThreads, sm, s>>>(y, K, h1, p->adj_rec, p->adj_w, p->adj_off,
                                                                   p->group_of, p->ngroups, p->ny, p->ns,
                                                                   p->nstrips_a);
        } else {
            MRF_PROPAGATE(set_smem(k_spread_cols<GG, WW, 1>, sm));
            k_spread_cols<GG, WW, 1><<<grid, kColThreads, sm, s>>>(y, K, h1, p->adj_rec, p->adj_w, p->adj_off,
                                                                   p->group_of, p->ngroups, p->ny, p->ns,
                                                                   p->nstrips_a);
        }
    }));
    MRF_LAUNCHED_AS("k_spread_cols", s);
    return MRF_OK;
}

mrf_status launch_rows_adj(const mrf_plan_s* p, const float2* h1, float2* dst, int dst_mode, int K, int nf,
                           float scale, cudaStream_t s) {
    const int G = p->gx;
    dim3 grid((p->ny + kRowB - 1) / kRowB, nf);
    const size_t sm = rows_smem(G);
    MRF_DISPATCH_G(G, {
        if (dst_mode == 0) {
            MRF_PROPAGATE(set_smem(k_rows_adj<GG, 0>, sm));
            k_rows_adj<GG, 0><<<grid, kRowThreads, sm, s>>>(h1, dst, K, scale, p->inv_dx, p->inv_dy, p->nx,
                                                            p->ny);
        } else {
            MRF_PROPAGATE(set_smem(k_rows_adj<GG, 1>, sm));
            k_rows_adj<GG, 1><<<grid, kRowThreads, sm, s>>>(h1, dst, K, scale, p->inv_dx, p->inv_dy, p->nx,
                                                            p->ny);
        }
    });
    MRF_LAUNCHED_AS("k_rows_adj", s);
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
static void free_plan(mrf_plan_s* p) {
    if (!p) return;
    void* ptrs[] = {p->inv_dx, p->inv_dy, p->fwd_rec, p->fwd_off, p->adj_rec, p->adj_off, p->fwd_w, p->adj_w,
                    p->fsp_off, p->fsp_loc, p->fsp_smp, p->fsp_w, p->grec,
                    p->group_of, p->gf_off, p->gf, p->h1, p->sub_h1, p->sub_spec, p->sub_Y, p->sub_R,
                    p->sub_partial, p->gat_off, p->gat_pt, p->gat_smp, p->gat_w};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

// Grouped adjoint gather table: every (group sample, tap) contribution,
// sorted by its oversampled-grid point (row * G + column),
// with weights psi(ux - mx) psi(uy - my) evaluated in FP64.  Built on the
// host from the plan's sample records the first time the grouped adjoint
// runs (synchronises the stream).
static mrf_status build_gather(mrf_plan_s* p, cudaStream_t s) {
    if (p->gat_off) return MRF_OK;
    const int NG = p->ngroups, ns = p->ns, W = p->W;
    const double beta = p->beta_d;
    std::vector<int4> grec((size_t)NG * ns);
    MRF_CUDA(cudaMemcpyAsync(grec.data(), p->grec, sizeof(int4) * grec.size(), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    auto kb = [&](double u) {
        const double z = 2.0 * u / W;
        const double arg = std::max(0.0, 1.0 - z * z);
        return std::cyl_bessel_i(0.0, beta * std::sqrt(arg));
    };
    struct Ent { int pt, smp; float w; };
    std::vector<Ent> ents;
    ents.reserve((size_t)NG * ns * W * W);
    for (int g = 0; g < NG; ++g)
        for (int j = 0; j < ns; ++j) {
            const int4 r = grec[(size_t)g * ns + j];
            const int mxw = r.y & 0xffff, myw = (r.y >> 16) & 0xffff;
            float fxf, fyf;
            std::memcpy(&fxf, &r.z, 4);
            std::memcpy(&fyf, &r.w, 4);
            for (int a = 0; a < W; ++a) {
                const int col = (mxw + a) % p->gx;
                const double wa = kb((double)fxf - a);
                for (int b = 0; b < W; ++b) {
                    const int row = (myw + b) % p->gy;
                    ents.push_back({row * p->gx + col, g * ns + j, (float)(wa * kb((double)fyf - b))});
                }
            }
        }
    std::stable_sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) { return x.pt < y.pt; });
    std::vector<int> goff(2, 0), gpt(ents.size()), gsmp(ents.size());
    std::vector<float> gw(ents.size());
    for (size_t i = 0; i < ents.size(); ++i) {
        gpt[i] = ents[i].pt;
        gsmp[i] = ents[i].smp;
        gw[i] = ents[i].w;
    }
    goff[1] = (int)ents.size();
    p->gat_n = (int)ents.size();
    MRF_CUDA(cudaMalloc(&p->gat_pt, sizeof(int) * gpt.size()));
    MRF_CUDA(cudaMalloc(&p->gat_smp, sizeof(int) * gsmp.size()));
    MRF_CUDA(cudaMalloc(&p->gat_w, sizeof(float) * gw.size()));
    MRF_CUDA(cudaMemcpy(p->gat_pt, gpt.data(), sizeof(int) * gpt.size(), cudaMemcpyHostToDevice));
    MRF_CUDA(cudaMemcpy(p->gat_smp, gsmp.data(), sizeof(int) * gsmp.size(), cudaMemcpyHostToDevice));
    MRF_CUDA(cudaMemcpy(p->gat_w, gw.data(), sizeof(float) * gw.size(), cudaMemcpyHostToDevice));
    int* off = nullptr;
    MRF_CUDA(cudaMalloc(&off, sizeof(int) * goff.size()));
    MRF_CUDA(cudaMemcpy(off, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice));
    p->gat_off = off;
    return MRF_OK;
}

static mrf_status launch_gather(const mrf_plan_s* p, int run, int threads, int K, cudaStream_t s) {
    if (run == 0) {                               // warp-cooperative form: one entry per thread
        const unsigned blocks = (unsigned)(((size_t)p->gat_n + threads - 1) / threads);
        k_gather_warp<<<blocks, threads, 0, s>>>(p->sub_R, K, p->gat_pt, p->gat_smp, p->gat_w, p->gat_n,
                                                 p->gy * p->gx, p->sub_spec);
        MRF_LAUNCHED_AS("k_gather_warp", s);
        return MRF_OK;
    }
    const int runs = (p->gat_n + run - 1) / run;
    const unsigned blocks = (unsigned)((runs + threads - 1) / threads);
    const int GG2 = p->gy * p->gx;
#define MRF_GATHER(RV) \
    k_gather_grid<RV><<<blocks, threads, 0, s>>>(p->sub_R, K, p->gat_pt, p->gat_smp, p->gat_w, p->gat_n, GG2, p->sub_spec)
    switch (run) {
        case 8: MRF_GATHER(8); break;
        case 16: MRF_GATHER(16); break;
        case 64: MRF_GATHER(64); break;
        default: MRF_GATHER(32); break;
    }
#undef MRF_GATHER
    MRF_LAUNCHED_AS("k_gather_grid", s);
    return MRF_OK;
}

// Spread tile-shape autotuner: time every (run length, block size) of
// k_gather_grid and every block size of k_gather_warp (run 0) on this plan's
// own gather table and K, keep the fastest.
// Runs once per plan and K, on the first grouped adjoint (which already
// synchronises to build the table); the candidates add into sub_spec, which
// the caller clears afterwards.
// Grouped column FFTs with a strip width chosen per plan: the K coefficient
// spectra are transformed column strip by column strip; wider strips mean
// fewer, larger blocks (more threads per block, fewer blocks per SM).
static size_t col_smem(int G, int tile) { return (size_t)(G + G * tile) * sizeof(float2); }
constexpr size_t kMaxDynSmem = 227 * 1024;

template <int GG, int TT>
static mrf_status cols_pass(mrf_plan_s* p, int K, bool inverse, cudaStream_t s) {
    const size_t sm = col_smem(GG, TT);
    const dim3 grid((unsigned)(p->gx / TT), (unsigned)K);
    if (inverse) {
        MRF_PROPAGATE(set_smem(k_cols_inv<GG, TT>, sm));
        k_cols_inv<GG, TT><<<grid, TT * 16, sm, s>>>(p->sub_spec, p->sub_h1, p->ny);
        MRF_LAUNCHED_AS("k_cols_inv", s);
    } else {
        MRF_PROPAGATE(set_smem(k_cols_store<GG, TT>, sm));
        k_cols_store<GG, TT><<<grid, TT * 16, sm, s>>>(p->sub_h1, p->sub_spec, p->ny);
        MRF_LAUNCHED_AS("k_cols_store", s);
    }
    return MRF_OK;
}

static mrf_status launch_cols(mrf_plan_s* p, int K, int tile, bool inverse, cudaStream_t s) {
    MRF_REQUIRE(col_smem(p->gy, tile) <= kMaxDynSmem, "strip width %d does not fit grid %d", tile, p->gy);
    MRF_DISPATCH_G(p->gy, {
        if (tile == 16) return cols_pass<GG, 16>(p, K, inverse, s);
        if (tile == 32) return cols_pass<GG, 32>(p, K, inverse, s);
        if constexpr (GG <= 384) return cols_pass<GG, 64>(p, K, inverse, s);
    });
    set_error("unsupported strip width %d", tile);
    return MRF_EINVAL;
}

// Strip width of the grouped column FFTs for this plan: each candidate's
// forward and inverse passes timed over three repetitions (after a warm-up)
// on the plan's own buffers, before the operator writes them.
static mrf_status tune_cols(mrf_plan_s* p, int K, cudaStream_t s) {
    if (p->col_tuned_K == K) return MRF_OK;
    static const int tiles[] = {16, 32, 64};
    cudaEvent_t e0, e1;
    MRF_CUDA(cudaEventCreate(&e0));
    MRF_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = 16;
    mrf_status st = MRF_OK;
    for (int t : tiles) {
        if (col_smem(p->gy, t) > kMaxDynSmem) continue;
        st = launch_cols(p, K, t, false, s);
        if (st == MRF_OK) st = launch_cols(p, K, t, true, s);
        if (st == MRF_OK && cudaEventRecord(e0, s) != cudaSuccess) st = MRF_ECUDA;
        for (int rep = 0; st == MRF_OK && rep < 3; ++rep) {
            st = launch_cols(p, K, t, false, s);
            if (st == MRF_OK) st = launch_cols(p, K, t, true, s);
        }
        float ms = 0.f;
        if (st != MRF_OK || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            if (st == MRF_OK) {
                set_error("strip-width autotuner: timing failed");
                st = MRF_ECUDA;
            }
            break;
        }
        if (ms < best) { best = ms; bt = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MRF_OK) return st;
    p->col_tile = bt;
    p->col_tuned_K = K;
    return MRF_OK;
}

static mrf_status tune_gather(mrf_plan_s* p, int K, cudaStream_t s) {
    if (p->gat_tuned_K == K) return MRF_OK;
    static const int runs[] = {0, 8, 16, 32, 64};
    static const int threads[] = {128, 256, 512};
    cudaEvent_t e0, e1;
    MRF_CUDA(cudaEventCreate(&e0));
    MRF_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int brun = 32, bthr = 128;
    mrf_status st = MRF_OK;
    for (int r : runs)
        for (int t : threads) {
            st = launch_gather(p, r, t, K, s);          // warm-up
            for (int rep = 0; st == MRF_OK && rep < 3; ++rep) {
                if (rep == 0 && cudaEventRecord(e0, s) != cudaSuccess) st = MRF_ECUDA;
                if (st == MRF_OK) st = launch_gather(p, r, t, K, s);
            }
            float ms = 0.f;
            if (st != MRF_OK || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                if (st == MRF_OK) {
                    set_error("gather autotuner: timing failed");
                    st = MRF_ECUDA;
                }
                break;
            }
            if (ms < best) { best = ms; brun = r; bthr = t; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MRF_OK) return st;
    p->gat_run = brun;
    p->gat_threads = bthr;
    p->gat_tuned_K = K;
    return MRF_OK;
}

mrf_status ensure_subspace_workspace(mrf_plan_s* p, int K) {
    if (p->sub_K >= K) return MRF_OK;
    const int Kc = 16;
    if (p->sub_h1) {
        cudaFree(p->sub_h1);
        cudaFree(p->sub_spec);
        cudaFree(p->sub_Y);
        cudaFree(p->sub_R);
        cudaFree(p->sub_partial);
    }
    p->sub_h1 = p->sub_spec = p->sub_Y = p->sub_R = p->sub_partial = nullptr;
    MRF_CUDA(cudaMalloc(&p->sub_h1, sizeof(float2) * (size_t)Kc * p->ny * p->gx));
    MRF_CUDA(cudaMalloc(&p->sub_spec, sizeof(float2) * (size_t)Kc * p->gy * p->gx));
    MRF_CUDA(cudaMalloc(&p->sub_Y, sizeof(float2) * (size_t)Kc * p->ngroups * p->ns));
    MRF_CUDA(cudaMalloc(&p->sub_R, sizeof(float2) * (size_t)Kc * p->ngroups * p->ns));
    MRF_CUDA(cudaMalloc(&p->sub_partial, sizeof(float2) * (size_t)Kc * p->parts * p->ny * p->nx));
    p->sub_K = Kc;
    return MRF_OK;
}

}  // namespace mrf

using namespace mrf;

extern "C" mrf_status mrf_nufft_plan(mrf_plan* out, int nx, int ny, int T, int ns, const float* traj, int os,
                                     int W, mrf_stream stream) {
    MRF_REQUIRE(out != nullptr, "mrf_nufft_plan: out is NULL");
    *out = nullptr;
    MRF_REQUIRE(traj != nullptr, "mrf_nufft_plan: traj is NULL");
    MRF_REQUIRE(os == 2, "mrf_nufft_plan: os must be 2 (got %d)", os);
    MRF_REQUIRE(W == 4 || W == 6, "mrf_nufft_plan: kb_width must be 4 or 6 (got %d)", W);
    MRF_REQUIRE(nx > 0 && ny > 0 && nx % 2 == 0 && ny % 2 == 0, "mrf_nufft_plan: nx, ny must be even and > 0");
    MRF_REQUIRE(nx == ny, "mrf_nufft_plan: square images only (nx %d, ny %d)", nx, ny);
    MRF_REQUIRE(supported_grid(os * nx) && supported_grid(os * ny),
                "mrf_nufft_plan: os*nx and os*ny must be in {64,128,256,384,512} (got %d, %d)", os * nx, os * ny);
    MRF_REQUIRE(T >= 1 && ns >= 1 && ns < (1 << 24), "mrf_nufft_plan: bad nframes/ns (%d, %d)", T, ns);
    cudaStream_t s = as_stream(stream);
    auto* p = new mrf_plan_s();
    p->nx = nx; p->ny = ny; p->T = T; p->ns = ns; p->os = os; p->W = W;
    p->gx = os * nx; p->gy = os * ny;
    const double beta = M_PI * std::sqrt((W / (double)os) * (W / (double)os) * (os - 0.5) * (os - 0.5) - 0.8);
    p->beta = (float)beta;
    p->beta_d = beta;
    p->sf = kTile - (W - 1);
    p->nstrips_f = (p->gx + p->sf - 1) / p->sf;
    p->nstrips_a = p->gx / kTile;

    std::vector<float> h((size_t)T * ns * 2);
    cudaError_t e = cudaMemcpyAsync(h.data(), traj, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_plan(p);
        set_error("mrf_nufft_plan: reading traj failed: %s", cudaGetErrorString(e));
        return MRF_ECUDA;
    }
    for (size_t i = 0; i < h.size(); ++i) {
        if (!(std::fabs(h[i]) <= 3.2f)) {
            free_plan(p);
            set_error("mrf_nufft_plan: trajectory value %g at %zu outside [-pi, pi]", (double)h[i], i);
            return MRF_EINVAL;
        }
    }
    // group frames with identical sample positions
    std::vector<int> group_of(T), rep;
    std::unordered_map<uint64_t, std::vector<int>> by_hash;
    const size_t fbytes = (size_t)ns * 2 * sizeof(float);
    for (int t = 0; t < T; ++t) {
        const unsigned char* d = reinterpret_cast<const unsigned char*>(h.data() + (size_t)t * ns * 2);
        uint64_t hv = 1469598103934665603ull;
        for (size_t i = 0; i < fbytes; ++i) hv = (hv ^ d[i]) * 1099511628211ull;
        int found = -1;
        for (int g : by_hash[hv])
            if (std::memcmp(h.data() + (size_t)rep[g] * ns * 2, d, fbytes) == 0) { found = g; break; }
        if (found < 0) {
            found = (int)rep.size();
            rep.push_back(t);
            by_hash[hv].push_back(found);
        }
        group_of[t] = found;
    }
    const int NG = (int)rep.size();
    p->ngroups = NG;
    // per-sample records (host double precision decides the nodes)
    const int SFN = p->nstrips_f, SAN = p->nstrips_a;
    std::vector<int4> grec((size_t)NG * ns);
    std::vector<int> fcount((size_t)NG * SFN, 0), acount((size_t)NG * SAN, 0);
    for (int g = 0; g < NG; ++g) {
        const float* kt = h.data() + (size_t)rep[g] * ns * 2;
        for (int j = 0; j < ns; ++j) {
            double ux = kt[2 * j] * p->gx / (2 * M_PI), uy = kt[2 * j + 1] * p->gy / (2 * M_PI);
            if (ux < 0) ux += p->gx;
            if (uy < 0) uy += p->gy;
            const long mx = (long)std::floor(ux - W / 2.0) + 1, my = (long)std::floor(uy - W / 2.0) + 1;
            const float fx = (float)(ux - mx), fy = (float)(uy - my);
            const int mxw = (int)(((mx % p->gx) + p->gx) % p->gx), myw = (int)(((my % p->gy) + p->gy) % p->gy);
            int4 r;
            r.x = j;
            r.y = mxw | (myw << 16);
            std::memcpy(&r.z, &fx, 4);
            std::memcpy(&r.w, &fy, 4);
            grec[(size_t)g * ns + j] = r;
            fcount[(size_t)g * SFN + mxw / p->sf]++;
            const int a1 = mxw / kTile, a2 = ((mxw + W - 1) % p->gx) / kTile;
            acount[(size_t)g * SAN + a1]++;
            if (a2 != a1) acount[(size_t)g * SAN + a2]++;
        }
    }
    std::vector<int> foff((size_t)NG * SFN + 1, 0), aoff((size_t)NG * SAN + 1, 0);
    for (size_t i = 0; i < (size_t)NG * SFN; ++i) foff[i + 1] = foff[i] + fcount[i];
    for (size_t i = 0; i < (size_t)NG * SAN; ++i) aoff[i + 1] = aoff[i] + acount[i];
    std::vector<int4> frec(foff.back()), arec(aoff.back());
    std::vector<int> fpos(foff.begin(), foff.end() - 1), apos(aoff.begin(), aoff.end() - 1);
    for (int g = 0; g < NG; ++g)
        for (int j = 0; j < ns; ++j) {
            const int4 r = grec[(size_t)g * ns + j];
            const int mxw = r.y & 0xffff;
            frec[fpos[(size_t)g * SFN + mxw / p->sf]++] = r;
            const int a1 = mxw / kTile, a2 = ((mxw + W - 1) % p->gx) / kTile;
            arec[apos[(size_t)g * SAN + a1]++] = r;
            if (a2 != a1) arec[apos[(size_t)g * SAN + a2]++] = r;
        }
    // frames of each group (CSR)
    std::vector<int> gfoff(NG + 1, 0), gf(T);
    for (int t = 0; t < T; ++t) gfoff[group_of[t] + 1]++;
    for (int g = 0; g < NG; ++g) gfoff[g + 1] += gfoff[g];
    {
        std::vector<int> pos(gfoff.begin(), gfoff.end() - 1);
        for (int t = 0; t < T; ++t) gf[pos[group_of[t]]++] = t;
    }
    std::vector<float> idx_(nx), idy_(ny);
    for (int i = 0; i < nx; ++i) idx_[i] = (float)(1.0 / psi_hat((i - nx / 2) / (double)p->gx, W, beta));
    for (int i = 0; i < ny; ++i) idy_[i] = (float)(1.0 / psi_hat((i - ny / 2) / (double)p->gy, W, beta));
    // frame parts of the subspace adjoint reduction (about 4 blocks per SM)
    {
        int parts = std::max(1, (4 * 152 + ny - 1) / ny);
        parts = std::min(parts, (T + kRowB - 1) / kRowB);
        int per = (T + parts - 1) / parts;
        per = (per + kRowB - 1) / kRowB * kRowB;
        p->frames_per_part = per;
        p->parts = (T + per - 1) / per;
    }

#define ALLOC_COPY(dst, vec)                                                                         \
    do {                                                                                             \
        e = cudaMalloc(&dst, sizeof(vec[0]) * std::max<size_t>(vec.size(), 1));                      \
        if (e == cudaSuccess && !vec.empty())                                                        \
            e = cudaMemcpy(dst, vec.data(), sizeof(vec[0]) * vec.size(), cudaMemcpyHostToDevice);    \
        if (e != cudaSuccess) goto fail;                                                             \
    } while (0)
    ALLOC_COPY(p->inv_dx, idx_);
    ALLOC_COPY(p->inv_dy, idy_);
    ALLOC_COPY(p->fwd_rec, frec);
    ALLOC_COPY(p->fwd_off, foff);
    ALLOC_COPY(p->adj_rec, arec);
    ALLOC_COPY(p->adj_off, aoff);
    ALLOC_COPY(p->grec, grec);
    ALLOC_COPY(p->group_of, group_of);
    ALLOC_COPY(p->gf_off, gfoff);
    ALLOC_COPY(p->gf, gf);
#undef ALLOC_COPY
    // the records' KB weights, once (the same expression the kernels used to
    // evaluate per frame, so the operator's values are unchanged)
    e = cudaMalloc(&p->fwd_w, sizeof(float) * 2 * W * std::max<size_t>(frec.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->adj_w, sizeof(float) * 2 * W * std::max<size_t>(arec.size(), 1));
    if (e != cudaSuccess) goto fail;
    {
        const int nf = (int)frec.size(), na = (int)arec.size();
        const float bt = p->beta;
        if (W == 4) {
            if (nf) k_rec_weights<4><<<(nf + 255) / 256, 256>>>(p->fwd_rec, nf, bt, p->fwd_w);
            if (na) k_rec_weights<4><<<(na + 255) / 256, 256>>>(p->adj_rec, na, bt, p->adj_w);
        } else {
            if (nf) k_rec_weights<6><<<(nf + 255) / 256, 256>>>(p->fwd_rec, nf, bt, p->fwd_w);
            if (na) k_rec_weights<6><<<(na + 255) / 256, 256>>>(p->adj_rec, na, bt, p->adj_w);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) goto fail;
    }
    e = cudaMalloc(&p->h1, sizeof(float2) * (size_t)T * ny * p->gx);
    if (e != cudaSuccess) goto fail;
    *out = p;
    return MRF_OK;
fail:
    free_plan(p);
    cudaGetLastError();
    set_error("mrf_nufft_plan: device allocation/copy failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MRF_ENOMEM : MRF_ECUDA;
}

extern "C" mrf_status mrf_nufft_tuning(mrf_plan p, int* gather_run, int* gather_threads, int* strip_width) {
    MRF_REQUIRE(p != nullptr, "mrf_nufft_tuning: NULL plan");
    if (gather_run) *gather_run = p->gat_tuned_K ? p->gat_run : 0;
    if (gather_threads) *gather_threads = p->gat_tuned_K ? p->gat_threads : 0;
    if (strip_width) *strip_width = p->col_tuned_K ? p->col_tile : 0;
    return MRF_OK;
}

extern "C" mrf_status mrf_nufft_gather_tuning(mrf_plan p, int* run, int* threads) {
    MRF_REQUIRE(p && run && threads, "mrf_nufft_gather_tuning: NULL argument");
    *run = p->gat_tuned_K ? p->gat_run : 0;
    *threads = p->gat_tuned_K ? p->gat_threads : 0;
    return MRF_OK;
}

extern "C" mrf_status mrf_nufft_destroy(mrf_plan p) {
    free_plan(p);
    return MRF_OK;
}

extern "C" mrf_status mrf_nufft_forward(mrf_plan p, const mrf_c64* x, mrf_c64* y, mrf_stream stream) {
    MRF_REQUIRE(p && x && y, "mrf_nufft_forward: NULL argument");
    cudaStream_t s = as_stream(stream);
    MRF_PROPAGATE(launch_rows_fwd(p, reinterpret_cast<const float2*>(x), 0, 0, p->T, p->h1, s));
    MRF_PROPAGATE(launch_cols_interp(p, p->h1, reinterpret_cast<float2*>(y), nullptr, 1.0f, s));
    return MRF_OK;
}

extern "C" mrf_status mrf_nufft_adjoint(mrf_plan p, const mrf_c64* y, mrf_c64* x, mrf_stream stream) {
    MRF_REQUIRE(p && x && y, "mrf_nufft_adjoint: NULL argument");
    cudaStream_t s = as_stream(stream);
    MRF_PROPAGATE(launch_spread_cols(p, reinterpret_cast<const float2*>(y), 0, 0, p->T, p->h1, s));
    MRF_PROPAGATE(launch_rows_adj(p, p->h1, reinterpret_cast<float2*>(x), 0, 0, p->T, 1.0f, s));
    return MRF_OK;
}

namespace mrf {
mrf_status subspace_forward(mrf_plan_s* p, const float2* alpha, const float2* phi, int K, float scale,
                            const float2* b, float2* y, int mode, cudaStream_t s) {
    MRF_REQUIRE(K >= 1 && K <= 16, "subspace rank K must be in [1, 16] (got %d)", K);
    MRF_REQUIRE(mode == 0 || mode == 1, "subspace mode must be 0 or 1 (got %d)", mode);
    MRF_REQUIRE(p->nx <= 256, "subspace forms need nx <= 256");
    if (mode == 0) {
        const int G = p->gx;
        dim3 grid(p->ny, (p->T + kRowB - 1) / kRowB);
        const size_t sm = (size_t)(G + row_region(G) + kRowB * K) * sizeof(float2);
        MRF_DISPATCH_G(G, {
            MRF_PROPAGATE(set_smem(k_rows_fwd_expand<GG>, sm));
            k_rows_fwd_expand<GG><<<grid, kRowThreads, sm, s>>>(alpha, phi, K, p->T, p->h1, p->inv_dx, p->inv_dy,
                                                                p->nx, p->ny);
        });
        MRF_LAUNCHED_AS("k_rows_fwd_expand", s);
        return launch_cols_interp(p, p->h1, y, b, scale, s);
    }
    MRF_PROPAGATE(ensure_subspace_workspace(p, K));
    MRF_PROPAGATE(tune_cols(p, K, s));                 // before the buffers hold this call's data
    MRF_PROPAGATE(launch_rows_fwd(p, alpha, 1, K, K, p->sub_h1, s));
    MRF_PROPAGATE(launch_cols(p, K, p->col_tile, false, s));
    {
        const int total = p->ngroups * p->ns;
        MRF_DISPATCH_G(p->gx, MRF_DISPATCH_W(p->W, {
            k_interp_groups<GG, WW><<<(total + 255) / 256, 256, 0, s>>>(p->sub_spec, K, p->grec, total, p->sub_Y,
                                                                        p->beta);
        }));
        MRF_LAUNCHED_AS("k_interp_groups", s);
    }
    const size_t n = (size_t)p->T * p->ns;
    k_combine_fwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->sub_Y, phi, K, p->group_of, p->T, p->ns, scale,
                                                               b, y);
    MRF_LAUNCHED_AS("k_combine_fwd", s);
    return MRF_OK;
}

mrf_status subspace_adjoint(mrf_plan_s* p, const float2* y, const float2* phi, int K, float scale,
                            float2* alpha_out, int mode, cudaStream_t s) {
    MRF_REQUIRE(K >= 1 && K <= 16, "subspace rank K must be in [1, 16] (got %d)", K);
    MRF_REQUIRE(mode == 0 || mode == 1, "subspace mode must be 0 or 1 (got %d)", mode);
    MRF_REQUIRE(p->nx <= 256, "subspace forms need nx <= 256");
    MRF_PROPAGATE(ensure_subspace_workspace(p, K));
    if (mode == 0) {
        MRF_PROPAGATE(launch_spread_cols(p, y, 0, 0, p->T, p->h1, s));
        const int G = p->gx;
        dim3 grid(p->ny, p->parts);
        const size_t sm = (size_t)(G + row_region(G) + kRowB * K) * sizeof(float2);
        MRF_DISPATCH_G(G, {
            MRF_PROPAGATE(set_smem(k_rows_adj_reduce<GG>, sm));
            k_rows_adj_reduce<GG><<<grid, kRowThreads, sm, s>>>(p->h1, phi, K, p->T, p->frames_per_part,
                                                                p->sub_partial, p->inv_dx, p->inv_dy, p->nx,
                                                                p->ny);
        });
        MRF_LAUNCHED_AS("k_rows_adj_reduce", s);
        const size_t n = (size_t)p->ny * p->nx * K;
        k_sum_parts<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(p->sub_partial, p->parts, n,
                                                                                        scale, alpha_out);
        MRF_LAUNCHED_AS("k_sum_parts", s);
        return MRF_OK;
    }
    MRF_PROPAGATE(tune_cols(p, K, s));                 // before the buffers hold this call's data
    {
        const size_t n = (size_t)p->ngroups * p->ns;
        k_combine_adj<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(y, phi, K, p->gf_off, p->gf, p->ngroups, p->ns,
                                                                   p->sub_R);
        MRF_LAUNCHED_AS("k_combine_adj", s);
    }
    MRF_PROPAGATE(build_gather(p, s));
    MRF_PROPAGATE(tune_gather(p, K, s));
    {
        const int G = p->gy;
        MRF_CUDA(cudaMemsetAsync(p->sub_spec, 0, sizeof(float2) * (size_t)K * G * G, s));
        MRF_PROPAGATE(launch_gather(p, p->gat_run, p->gat_threads, K, s));
        MRF_PROPAGATE(launch_cols(p, K, p->col_tile, true, s));
    }
    MRF_PROPAGATE(launch_rows_adj(p, p->sub_h1, alpha_out, 1, K, K, scale, s));
    return MRF_OK;
}
}  // namespace mrf

extern "C" mrf_status mrf_nufft_forward_subspace(mrf_plan p, const mrf_c64* alpha, const mrf_c64* phi, int K,
                                                 float scale, const mrf_c64* b, mrf_c64* y, int mode,
                                                 mrf_stream stream) {
    MRF_REQUIRE(p && alpha && phi && y, "mrf_nufft_forward_subspace: NULL argument");
    return subspace_forward(p, reinterpret_cast<const float2*>(alpha), reinterpret_cast<const float2*>(phi), K,
                            scale, reinterpret_cast<const float2*>(b), reinterpret_cast<float2*>(y), mode,
                            as_stream(stream));
}

extern "C" mrf_status mrf_nufft_adjoint_subspace(mrf_plan p, const mrf_c64* y, const mrf_c64* phi, int K,
                                                 float scale, mrf_c64* alpha_out, int mode, mrf_stream stream) {
    MRF_REQUIRE(p && y && phi && alpha_out, "mrf_nufft_adjoint_subspace: NULL argument");
    return subspace_adjoint(p, reinterpret_cast<const float2*>(y), reinterpret_cast<const float2*>(phi), K, scale,
                            reinterpret_cast<float2*>(alpha_out), mode, as_stream(stream));
}

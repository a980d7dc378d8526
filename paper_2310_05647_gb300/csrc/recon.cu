// Algorithm 1 (MS-LLR) with the iterate held in the temporal subspace,
// X = alpha Phi^H, alpha [N][K] (N = nx * ny voxels, row-major, K contiguous).
//
// Per iteration (all on the stream, no host round trip unless costs are read):
//   grad  = (A/a)^H r                        r = (A/a) X - b~ from the last pass
//   QL    = Q(X) L   per patch, and  Tr     (graph term of Eq. 12)
//   alpha = (alpha - mu (grad + lambda1 Q^*(QL)) + c Q^*(P)) / (1 + c cnt)   (Eq. 12 + 19)
//   r     = (A/a) X - b~                     (data residual of the new iterate)
//   P     = SVT_{1/beta}(Q_i(X)) per patch   (Eq. 18, used by the next pass;
//                                             its singular values give the
//                                             nuclear norms of the cost)
//   cost  = 1/2 ||r||^2 + lambda1 Tr(Q L Q^H) + lambda2 sum ||Q_i||_*
//   maps  = Phi_D(X)                         (Eq. 5, compressed atoms)
//   L     = D - W of the k-nearest-patch graph of the maps (Eq. 7-10),
//   lambda1 = lambda1^0 / max(L)
// P_S is the identity on coefficient images, Q^*(Q(X) L) commutes with P_S,
// and the singular values of Q_i(X) (p^2 x T) equal those of Q_i(alpha)
// (p^2 x K) because Phi has orthonormal columns.
#include <algorithm>
#include <climits>
#include <cstring>
#include <cmath>
#include <vector>

#include "common.h"
#include "knn.h"
#include "match.h"
#include "mlp.h"
#include "nufft_plan.h"

namespace mrf {

struct PatchGeom {
    int n, p, s, cnt;   // square image side, patch side, stride, patches per axis
    __host__ __device__ int origin(int i) const { return min(i * s, n - p); }
    __host__ __device__ int count() const { return cnt * cnt; }
};

static PatchGeom make_geom(int n, int p, int s) {
    PatchGeom g;
    g.n = n; g.p = p; g.s = s;
    g.cnt = (n - p) / s + 1 + (((n - p) % s) ? 1 : 0);
    return g;
}

// --------------------------------------------------------------------------
// small reductions
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block, result valid in thread 0
__device__ double block_sum(double v) {
    __shared__ double red[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
        v = warp_sum(v);
    }
    __syncthreads();
    return v;
}

// *acc += sum |x_i|^2 (x 16-byte aligned).  A grid of kNorm2Blocks blocks
// reads x two values per 16-byte load; each thread sums its ~n / (blocks x
// 256) terms in FP32, the threads and blocks add in FP64 (one atomic per
// block: thousands of FP64 atomics on one word cost more than the read).
constexpr int kNorm2Blocks = 4 * 152;
__global__ void k_norm2_acc(const float2* __restrict__ x, size_t n, double* __restrict__ acc) {
    float s = 0.f;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x) {
        const float4 q = x4[i];
        s += q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) s += cabs2(x[n - 1]);
    const double d = block_sum((double)s);
    if (threadIdx.x == 0) atomicAdd(acc, d);
}

// part[b] = block b's sum of |x_i|^2, the same split of x as k_norm2_acc
// (kNorm2Blocks blocks); k_cost adds the parts in block order, so the sum is
// the same on every run.
__global__ void k_norm2_part(const float2* __restrict__ x, size_t n, double* __restrict__ part) {
    float s = 0.f;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x) {
        const float4 q = x4[i];
        s += q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) s += cabs2(x[n - 1]);
    const double d = block_sum((double)s);
    if (threadIdx.x == 0) part[blockIdx.x] = d;
}

// re/im of sum conj(a) b
__global__ void k_dot_acc(const float2* __restrict__ a, const float2* __restrict__ b, size_t n,
                          double* __restrict__ acc) {
    double re = 0.0, im = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 p = cconjmul(a[i], b[i]);
        re += p.x;
        im += p.y;
    }
    re = block_sum(re);
    im = block_sum(im);
    if (threadIdx.x == 0) { atomicAdd(acc, re); atomicAdd(acc + 1, im); }
}

__global__ void k_scale(float2* __restrict__ x, size_t n, float s) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = cscale(x[i], s);
}

__global__ void k_scale_copy(const float2* __restrict__ x, size_t n, float s, float2* __restrict__ y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = cscale(x[i], s);
}

// y = x / sqrt(*n2) (a power-iteration step's normalisation, read on the
// device; zero when the norm is not positive)
__global__ void k_scale_by_norm(const float2* __restrict__ x, size_t n, const double* __restrict__ n2,
                                float2* __restrict__ y) {
    const double nw = sqrt(*n2);
    const float s = nw > 0.0 ? (float)(1.0 / nw) : 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = cscale(x[i], s);
}

__global__ void k_fill(float2* __restrict__ x, size_t n, float2 v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = v;
}

__global__ void k_max(const float* __restrict__ v, int n, float* __restrict__ out) {
    __shared__ float red[32];
    float m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

static unsigned nblk(size_t n, int t = 256) { return (unsigned)std::min<size_t>((n + t - 1) / t, 4096); }

// --------------------------------------------------------------------------
// patch graph (Eq. 7-10)
// --------------------------------------------------------------------------
// Patch features: F[i][2 (py p + px) + c] = rint(4096 T / Tmax) of the patch's
// voxels (12-bit fixed point of T1 / T1max and T2 / T2max, half to even).
// Squared distances of these integers are exact (< 2^32 for p <= 11), so
// the many exact ties of piecewise-constant maps break to the lower index on
// every device.
constexpr double kQScale = 4096.0;

// rint(t / tmax * 4096) as the FP64 oracle rounds it.  The FP32 quotient
// scaled by 4096 (exact) is within 2^-13 of the exact value for ratios up to
// 1 (2^-12 up to 2) and the FP64 one within 2^-41, so away from a half (more
// than 2^-10) both round to the same integer; near a half, for large ratios
// and for non-finite values the FP64 expression decides.
__device__ __forceinline__ int quantise(float t, double tmax) {
    const float y = __fdiv_rn(t, (float)tmax) * (float)kQScale;
    if (fabsf(y) < 2.f * (float)kQScale && fabsf(y - floorf(y) - 0.5f) > 0x1p-10f) return (int)rintf(y);
    return (int)rint((double)t / tmax * kQScale);
}

__global__ void k_features(const float* __restrict__ t1t2, PatchGeom g, double t1max, double t2max, int FD4,
                           int* __restrict__ F) {
    const int pp = g.p * g.p;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.count() * pp) return;
    const int i = e / pp, q = e - i * pp;
    const int py = q / g.p, px = q - py * g.p;
    const int y = g.origin(i / g.cnt) + py, x = g.origin(i % g.cnt) + px;
    const size_t v = (size_t)y * g.n + x;
    int* f = F + (size_t)i * FD4 + 2 * q;
    f[0] = quantise(t1t2[2 * v], t1max);
    f[1] = quantise(t1t2[2 * v + 1], t2max);
}

// sigma^2 = median of the non-zero kNN squared distances (1 if none) on the
// exact integer distances, reported in units of (T / Tmax)^2 (integer /
// 4096^2).  One block; three sweeps over the distances at most:
//  1. a histogram on a monotone log-scale key (the position of the leading
//     bit and the 6 bits after it: 32 x 64 bins), which also counts them;
//     the bin holding the lower middle rank is found by a block scan;
//  2. that bin's elements are compacted into shared memory (when they fit)
//     and the smallest element of any higher bin is taken;
//  3. the rank inside the bin by an 8-bit radix select over the bits the
//     bin leaves open, on the compacted list (else on the distances again).
// The upper middle rank is the same value when enough elements equal it,
// else the smallest element above it.
constexpr int kMedianThreads = 1024;
constexpr int kMedianBins = 2048;
constexpr int kMedianList = 4096;

__device__ __forceinline__ unsigned median_bin(unsigned b) {       // b > 0
    const int e = 31 - __clz(b);
    const unsigned sub = e >= 6 ? (b >> (e - 6)) & 63u : (b << (6 - e)) & 63u;
    return (unsigned)e * 64u + sub;
}

__global__ void __launch_bounds__(kMedianThreads) k_median_nonzero(const unsigned* __restrict__ v, int n,
                                                                   float* __restrict__ sigma2) {
    __shared__ unsigned hist[kMedianBins];
    __shared__ unsigned list[kMedianList];
    __shared__ unsigned s_warp[32];
    __shared__ unsigned s_bin, s_rank, s_eq, s_prefix, s_cnt, s_above, s_total;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(v) & 15u) == 0;
    const int n4 = vec ? n / 4 : 0;
    const uint4* v4 = reinterpret_cast<const uint4*>(v);
    for (int i = tid; i < kMedianBins; i += kMedianThreads) hist[i] = 0u;
    if (tid == 0) { s_cnt = 0u; s_above = 0xffffffffu; }
    __syncthreads();
    // sweep 1
    auto bin_add = [&](unsigned b) { if (b) atomicAdd(&hist[median_bin(b)], 1u); };
#pragma unroll 4
    for (int i = tid; i < n4; i += kMedianThreads) {
        const uint4 q = v4[i];
        bin_add(q.x); bin_add(q.y); bin_add(q.z); bin_add(q.w);
    }
    for (int i = 4 * n4 + tid; i < n; i += kMedianThreads) bin_add(v[i]);
    __syncthreads();
    // block scan: thread t owns bins 2t and 2t + 1
    const unsigned h0 = hist[2 * tid], h1 = hist[2 * tid + 1], own = h0 + h1;
    unsigned incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned w = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;                              // inclusive over warps
        if (lane == 31) s_total = w;
    }
    __syncthreads();
    const unsigned total = s_total;
    if (total == 0u) {
        if (tid == 0) *sigma2 = 1.0f;
        return;
    }
    const unsigned rank = (total - 1u) / 2u;
    incl += wid ? s_warp[wid - 1] : 0u;
    if (incl - own <= rank && rank < incl) {          // exactly one thread
        const unsigned before = incl - own;
        const bool first = rank < before + h0;
        const unsigned k = 2u * tid + (first ? 0u : 1u);
        s_bin = k;
        s_rank = rank - (first ? before : before + h0);
        s_eq = first ? h0 : h1;
    }
    __syncthreads();
    const unsigned k = s_bin, cnt = s_eq;
    const int e = (int)(k >> 6);
    const unsigned lead = 64u + (k & 63u);
    const unsigned base = e >= 6 ? lead << (e - 6) : lead >> (6 - e);
    const bool compact = cnt <= (unsigned)kMedianList;
    // sweep 2
    auto keep = [&](unsigned b, bool in) {
        if (compact) {
            const unsigned m = __ballot_sync(0xffffffffu, in);
            unsigned at = 0;
            if (lane == 0 && m) at = atomicAdd(&s_cnt, (unsigned)__popc(m));
            at = __shfl_sync(0xffffffffu, at, 0);
            const unsigned slot = at + __popc(m & ((1u << lane) - 1u));
            if (in && slot < (unsigned)kMedianList) list[slot] = b;
        }
    };
    unsigned above = 0xffffffffu;
    for (int i0 = 0; i0 < n4; i0 += kMedianThreads) {        // warp-uniform trip count
        const int i = i0 + tid;
        const uint4 q = i < n4 ? v4[i] : make_uint4(0u, 0u, 0u, 0u);
        const unsigned qs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned b = qs[j];
            const unsigned bn = b ? median_bin(b) : 0u;
            if (b && bn > k) above = min(above, b);
            keep(b, b && bn == k);
        }
    }
    for (int i0 = 4 * n4; i0 < n; i0 += kMedianThreads) {
        const int i = i0 + tid;
        const unsigned b = i < n ? v[i] : 0u;
        const unsigned bn = b ? median_bin(b) : 0u;
        if (b && bn > k) above = min(above, b);
        keep(b, b && bn == k);
    }
    for (int o = 16; o > 0; o >>= 1) above = min(above, __shfl_xor_sync(0xffffffffu, above, o));
    if (lane == 0) atomicMin(&s_above, above);
    if (tid == 0) s_prefix = base;
    __syncthreads();
    // sweep 3: the open low bits of the bin, 8 at a time from the top
    auto in_bin = [&](unsigned b) { return b != 0u && median_bin(b) == k; };
    const int m_list = compact ? (int)cnt : 0;
    int bits = e > 6 ? e - 6 : 0;
    unsigned prefix = base, mask = bits ? ~0u << bits : ~0u;
    while (bits > 0) {
        const int width = bits < 8 ? bits : 8;
        const int shift = bits - width;
        const unsigned dmask = (1u << width) - 1u;
        if (tid < 256) hist[tid] = 0u;
        __syncthreads();
        auto add = [&](unsigned b) { if ((b & mask) == prefix) atomicAdd(&hist[(b >> shift) & dmask], 1u); };
        if (compact) {
            for (int i = tid; i < m_list; i += kMedianThreads) add(list[i]);
        } else {
            for (int i = tid; i < n; i += kMedianThreads) {
                const unsigned b = v[i];
                if (in_bin(b)) add(b);
            }
        }
        __syncthreads();
        if (wid == 0) {
            const unsigned r = s_rank;
            unsigned own8[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) { own8[j] = hist[8 * lane + j]; sum += own8[j]; }
            unsigned inc = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, inc > r);
            if (lane == __ffs(hit) - 1) {                // the digits count every element left
                unsigned c = inc - sum;
                int d = 0;
                for (; d < 7; ++d) {
                    if (c + own8[d] > r) break;
                    c += own8[d];
                }
                s_rank = r - c;
                s_eq = own8[d];
                s_prefix = prefix | ((unsigned)(8 * lane + d) << shift);
            }
        }
        __syncthreads();
        prefix = s_prefix;
        mask |= dmask << shift;
        bits = shift;
    }
    const unsigned lo = s_prefix;                    // value of rank (total - 1) / 2
    // elements <= lo: the ones below it (rank - s_rank) and its copies (s_eq)
    const unsigned le = rank - s_rank + s_eq;
    unsigned hi = lo;
    if (le <= total / 2u) {
        unsigned up = 0xffffffffu;                   // smallest element of the bin above lo
        if (compact) {
            for (int i = tid; i < m_list; i += kMedianThreads) if (list[i] > lo) up = min(up, list[i]);
        } else {
            for (int i = tid; i < n; i += kMedianThreads) {
                const unsigned b = v[i];
                if (in_bin(b) && b > lo) up = min(up, b);
            }
        }
        for (int o = 16; o > 0; o >>= 1) up = min(up, __shfl_xor_sync(0xffffffffu, up, o));
        if (lane == 0) atomicMin(&s_above, up);
        __syncthreads();
        hi = s_above;
    }
    if (tid == 0) *sigma2 = (float)(0.5 * ((double)lo + (double)hi) / (kQScale * kQScale));
}

// w = exp(-d2 / sigma^2) on the kNN edges; in-degree counts of the reverse graph
__global__ void k_edge_weights(const int* __restrict__ nbr, const unsigned* __restrict__ d2, int ne,
                               const float* __restrict__ sigma2, float* __restrict__ w, int* __restrict__ rcnt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    w[e] = expf(-((float)d2[e] * (float)(1.0 / (kQScale * kQScale))) / *sigma2);
    atomicAdd(&rcnt[nbr[e]], 1);
}

// Neighbour lists of the graph term are cut into chunks of kGbSplit entries
// (the knn forward entries, then the reverse list).  The patch's own block
// takes the first chunk; each further chunk is an extra work item whose
// partial sum its own block writes, and the last of the patch's blocks to
// finish adds them to the first chunk's sum in chunk order.  The patches of
// a flat region tie at distance 0, and ties go to the lower index, so they
// all name the region's lowest-index patches: a few patches collect reverse
// lists of a thousand entries or more against a mean list length of 2 knn,
// which one block would otherwise read alone.
constexpr int kGbSplit = 32;
__host__ __device__ inline int gb_extra_chunks(int nq) { return nq > kGbSplit ? (nq - 1) / kGbSplit : 0; }
// an upper bound of the extra chunks of a graph (sum of (nq - 1) / kGbSplit,
// with sum nq = 2 np knn)
inline int gb_max_extra(int np, int knn) { return (int)((2LL * np * knn) / kGbSplit) + 1; }

// Exclusive scans of the reverse counts (off: list offsets) and of the patches'
// extra chunks (xoff), the patch of every extra chunk (xpatch[xoff[n]]), and
// zeroed fold counts (xcnt), in one block.
__global__ void __launch_bounds__(1024) k_scan_graph(const int* __restrict__ cnt, int n, int knn,
                                                     int* __restrict__ off, int* __restrict__ xoff,
                                                     int* __restrict__ xpatch, int* __restrict__ xcnt) {
    __shared__ int part[1024], xpart[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0, xs = 0;
    for (int i = b; i < e; ++i) {
        s += cnt[i];
        xs += gb_extra_chunks(knn + cnt[i]);
    }
    part[threadIdx.x] = s;
    xpart[threadIdx.x] = xs;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        const int xv = threadIdx.x >= (unsigned)o ? xpart[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        xpart[threadIdx.x] += xv;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s, xrun = xpart[threadIdx.x] - xs;
    for (int i = b; i < e; ++i) {
        off[i] = run;
        xoff[i] = xrun;
        xcnt[i] = 0;
        run += cnt[i];
        const int nx = gb_extra_chunks(knn + cnt[i]);
        for (int c = 0; c < nx; ++c) xpatch[xrun + c] = i;
        xrun += nx;
    }
    if (threadIdx.x == blockDim.x - 1) {
        off[n] = part[threadIdx.x];
        xoff[n] = xpart[threadIdx.x];
    }
}

__global__ void k_fill_reverse(const int* __restrict__ nbr, const float* __restrict__ w, int ne, int knn,
                               const int* __restrict__ roff, int* __restrict__ rpos, int* __restrict__ rsrc,
                               float* __restrict__ rw) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int j = nbr[e];
    const int at = roff[j] + atomicAdd(&rpos[j], 1);
    rsrc[at] = e / knn;
    rw[at] = w[e];
}

// Order each reverse list by source index (a fixed summation order) and
// compute the degrees of W = (K + K^T)/2.  One warp per target patch: the
// sources of a list are distinct, so each one's rank is the number of set
// bits below it in the warp's bitmap of the list (prefix popcounts over the
// np / 32 words, a lane per contiguous chunk), which sorts the list in
// O(np / 32 + length) whatever the hub sizes; the degree sums the sorted
// reverse weights and the forward weights in a fixed order.
constexpr int kDegWarps = 8;
__global__ void __launch_bounds__(kDegWarps * 32) k_degree(const float* __restrict__ w, int np, int knn,
                                                           const int* __restrict__ roff,
                                                           const int* __restrict__ rsrc_in,
                                                           const float* __restrict__ rw_in, int* __restrict__ rsrc,
                                                           float* __restrict__ rw, float* __restrict__ deg,
                                                           unsigned* __restrict__ deg_max) {
    extern __shared__ unsigned smd[];                     // per warp: [nw] bitmap, then [nw] prefix counts
    const int nw = (np + 31) >> 5;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kDegWarps + wib;
    if (j >= np) return;                                  // whole warps
    unsigned* bits = smd + (size_t)wib * 2 * nw;
    unsigned* pre = bits + nw;
    const int b = roff[j], n = roff[j + 1] - b;
    for (int i = lane; i < nw; i += 32) bits[i] = 0u;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const int src = rsrc_in[b + i];
        atomicOr(&bits[src >> 5], 1u << (src & 31));
    }
    __syncwarp();
    const int per = (nw + 31) >> 5;
    const int w0 = min(nw, lane * per), w1 = min(nw, w0 + per);
    unsigned acc = 0;
    for (int i = w0; i < w1; ++i) acc += __popc(bits[i]);
    unsigned incl = acc;                                  // inclusive scan over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    unsigned run = incl - acc;
    for (int i = w0; i < w1; ++i) { pre[i] = run; run += __popc(bits[i]); }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const int src = rsrc_in[b + i];
        const unsigned word = bits[src >> 5] & ((1u << (src & 31)) - 1u);
        const int at = b + (int)(pre[src >> 5] + __popc(word));
        rsrc[at] = src;
        rw[at] = rw_in[b + i];
    }
    __syncwarp();                                         // the sorted list, read back by the warp
    double d = 0.0;
    for (int i = lane; i < n; i += 32) d += rw[b + i];
    for (int q = lane; q < knn; q += 32) d += w[(size_t)j * knn + q];
    d = warp_sum(d);
    if (lane == 0) {
        const float dj = (float)(0.5 * d);
        deg[j] = dj;
        atomicMax(deg_max, __float_as_uint(dj));   // degrees are >= 0: their bits order like the values
    }
}

// copies of the forward graph and lambda1 for the cost trace
__global__ void k_graph_snapshot(const int* __restrict__ nbr, const float* __restrict__ w,
                                 const float* __restrict__ deg, const float* __restrict__ lam1, int ne, int np,
                                 int* __restrict__ nbr_c, float* __restrict__ w_c, float* __restrict__ deg_c,
                                 float* __restrict__ lam1_c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) {
        nbr_c[i] = nbr[i];
        w_c[i] = w[i];
    }
    if (i < np) deg_c[i] = deg[i];
    if (i == 0) *lam1_c = *lam1;
}

// lambda1 = lambda1^0 / max(L) (or times max(L) as printed)
__global__ void k_lambda(const float* __restrict__ lmax, float lam1_0, int literal, float* __restrict__ lam1) {
    const float m = *lmax;
    *lam1 = literal ? lam1_0 * m : (m > 0.f ? lam1_0 / m : 0.f);
}

// (Q(X) L)_j = deg_j Q_j - 1/2 sum_{i in N(j)} w_ji Q_i - 1/2 sum_{i: j in N(i)} w_ij Q_i,
// written per patch (QL nullable) and/or accumulated into Tr(Q L Q^H).
// With rev == 0 only the forward kNN entries are read, with weight w instead
// of w / 2: then sum_j <Q_j, v_j> = sum_j deg_j |Q_j|^2 - sum_j sum_{i in N(j)}
// w_ji Re <Q_j, Q_i>, which is Tr(Q L Q^H) too (W = (K + K^T) / 2 and Re <., .>
// is symmetric, so the reverse half of W adds the same sum as the forward
// half), at half the neighbour reads; v_j itself is then not (Q L)_j.
// One block per patch j (plus the cut lists' chunk blocks, below), each
// thread up to kGbElems of its p x p x K coefficients (consecutive threads
// read consecutive coefficients of a neighbour's patch rows).  The neighbour
// list (forward kNN entries, then the reverse list) is staged in shared
// memory kGbChunk entries at a time as
// (offset of the neighbour patch's first coefficient, w / 2), so the inner
// loop is one gather and two FMAs per coefficient and neighbour.  (Pairs of
// coefficients per 16-byte load halve the loads but leave fewer in flight
// per warp; measured slower on this latency-bound kernel.)  With xoff set
// (Q(X)L), a list longer than kGbSplit entries is cut: the patch's block
// reads its first kGbSplit entries, and each further chunk gets a block of
// its own (blocks [0, xoff[np]), ahead of the patches' blocks) that writes
// its partial sum to xpart.  Each of these blocks then counts itself in
// xcnt[j] (after a fence); the last of patch j's blocks adds the partials to
// QL_j in chunk order (the same order whichever block is last) and resets
// the count.  No block waits for another.  Grid: np blocks, plus
// gb_max_extra(np, knn) with xoff.
constexpr int kGbThreads = 128;
constexpr int kGbChunk = 256;
constexpr int kGbElems = 5;      // 8 x 8 x 10 coefficients = 5 per thread: no idle slots, 55 registers
static_assert(kGbChunk >= kGbSplit, "a cut chunk is staged in one round");

// v[u] -= wscale * w_q * (coefficient off[u] of neighbour patch i_q), q in
// [q0, q1) of patch j's list (forward entries q < knn, then the reverse list
// from rb); a block-wide call (stages the list in s_off / s_w).
__device__ __forceinline__ void gb_gather(const float2* __restrict__ alpha, const PatchGeom& g, int K, int j,
                                          const int* __restrict__ nbr, const float* __restrict__ w, int knn,
                                          int rb, const int* __restrict__ rsrc, const float* __restrict__ rw,
                                          float wscale, int q0, int q1, const int (&off)[kGbElems],
                                          float2 (&v)[kGbElems], int* s_off, float* s_w) {
    for (int c0 = q0; c0 < q1; c0 += kGbChunk) {
        const int cn = min(kGbChunk, q1 - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cn; t += kGbThreads) {
            const int q = c0 + t;
            int i;
            float wq;
            if (q < knn) { i = nbr[(size_t)j * knn + q]; wq = w[(size_t)j * knn + q]; }
            else { i = rsrc[rb + q - knn]; wq = rw[rb + q - knn]; }
            s_off[t] = (g.origin(i / g.cnt) * g.n + g.origin(i % g.cnt)) * K;
            s_w[t] = wscale * wq;
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < cn; ++t) {
            const float2* src = alpha + s_off[t];
            const float wt = s_w[t];
#pragma unroll
            for (int u = 0; u < kGbElems; ++u) {
                if (off[u] >= 0) {
                    const float2 b = src[off[u]];
                    v[u].x -= wt * b.x;
                    v[u].y -= wt * b.y;
                }
            }
        }
    }
}

// coefficient offsets (within a patch, relative to its first coefficient in
// the image) of this thread's kGbElems coefficients of pass e0, -1 past ne
__device__ __forceinline__ void gb_offsets(const PatchGeom& g, int K, int pK, int ne, int e0,
                                           int (&off)[kGbElems]) {
#pragma unroll
    for (int u = 0; u < kGbElems; ++u) {
        const int e = e0 + threadIdx.x + u * kGbThreads;
        const int py = e / pK, rem = e - py * pK;      // rem = px * K + k
        off[u] = e < ne ? py * g.n * K + rem : -1;
    }
}

// Block-wide: count this block in xcnt[j] once its writes are visible; the
// last of patch j's nx + 1 blocks folds the chunks' partial sums
// xpart[xoff[j] ..] into QL_j, in chunk order, with L2 reads (other SMs
// wrote them), and resets the count.
__device__ __forceinline__ void gb_count_and_fold(int j, int ne, const int* __restrict__ xoff,
                                                  int* __restrict__ xcnt, float2* __restrict__ xpart,
                                                  float2* __restrict__ QL, int* s_last) {
    __threadfence();
    __syncthreads();
    const int x0 = xoff[j], x1 = xoff[j + 1];
    if (threadIdx.x == 0) *s_last = atomicAdd(&xcnt[j], 1) == x1 - x0;
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (threadIdx.x == 0) xcnt[j] = 0;
    for (int e = threadIdx.x; e < ne; e += kGbThreads) {
        float2 v = __ldcg(QL + (size_t)j * ne + e);
#pragma unroll 4
        for (int x = x0; x < x1; ++x) v = cadd(v, __ldcg(xpart + (size_t)x * ne + e));
        QL[(size_t)j * ne + e] = v;
    }
}

__global__ void __launch_bounds__(kGbThreads, 9) k_graph_blocks(const float2* __restrict__ alpha, PatchGeom g,
                                                                int K, const int* __restrict__ nbr,
                                                                const float* __restrict__ w, int knn,
                                                                const int* __restrict__ roff,
                                                                const int* __restrict__ rsrc,
                                                                const float* __restrict__ rw,
                                                                const float* __restrict__ deg, int rev,
                                                                const int* __restrict__ xoff,
                                                                const int* __restrict__ xpatch,
                                                                float2* __restrict__ xpart, int* __restrict__ xcnt,
                                                                float2* __restrict__ QL, double* __restrict__ trace) {
    __shared__ int s_off[kGbChunk];
    __shared__ float s_w[kGbChunk];
    __shared__ int s_last;
    const int np = g.count();
    const int pK = g.p * K;
    const int ne = g.p * pK;
    const bool cut = rev && xoff;
    const int X = cut ? xoff[np] : 0;
    if ((int)blockIdx.x < X) {
        // extra chunk x of patch j = xpatch[x]: list entries [c kGbSplit,
        // (c + 1) kGbSplit), c = 1 + x - xoff[j]; its partial sum
        // -1/2 sum w Q_i goes to xpart[x][p x p x K].  These blocks come
        // first, so the longest chains start while the patches' blocks run.
        const int x = blockIdx.x;
        const int j = xpatch[x];
        const int rb = roff[j], nq = knn + roff[j + 1] - rb;
        const int q0 = (1 + x - xoff[j]) * kGbSplit, q1 = min(nq, q0 + kGbSplit);
        for (int e0 = 0; e0 < ne; e0 += kGbThreads * kGbElems) {
            int off[kGbElems];
            float2 v[kGbElems];
            gb_offsets(g, K, pK, ne, e0, off);
#pragma unroll
            for (int u = 0; u < kGbElems; ++u) v[u] = make_float2(0.f, 0.f);
            gb_gather(alpha, g, K, j, nbr, w, knn, rb, rsrc, rw, 0.5f, q0, q1, off, v, s_off, s_w);
#pragma unroll
            for (int u = 0; u < kGbElems; ++u)
                if (off[u] >= 0) xpart[(size_t)x * ne + e0 + threadIdx.x + u * kGbThreads] = v[u];
        }
        gb_count_and_fold(j, ne, xoff, xcnt, xpart, QL, &s_last);
        return;
    }
    const int j = (int)blockIdx.x - X;
    if (j >= np) return;
    const int jy = g.origin(j / g.cnt), jx = g.origin(j % g.cnt);
    const float dj = deg[j];
    const int rb = rev ? roff[j] : 0, re = rev ? roff[j + 1] : 0;
    const int nq = knn + (rev ? re - rb : 0);
    const float wscale = rev ? 0.5f : 1.0f;
    const bool split = cut && xoff[j + 1] > xoff[j];
    const int q1 = split ? kGbSplit : nq;           // the list's first chunk, or all of it
    float tr = 0.f;                 // this thread's share (kGbElems terms a pass), in FP32
    for (int e0 = 0; e0 < ne; e0 += kGbThreads * kGbElems) {
        int off[kGbElems];
        float2 a[kGbElems], v[kGbElems];
        gb_offsets(g, K, pK, ne, e0, off);
#pragma unroll
        for (int u = 0; u < kGbElems; ++u) {
            a[u] = off[u] >= 0 ? alpha[((size_t)jy * g.n + jx) * K + off[u]] : make_float2(0.f, 0.f);
            v[u] = cscale(a[u], dj);
        }
        gb_gather(alpha, g, K, j, nbr, w, knn, rb, rsrc, rw, wscale, 0, q1, off, v, s_off, s_w);
#pragma unroll
        for (int u = 0; u < kGbElems; ++u) {
            if (off[u] < 0) continue;
            const int e = e0 + threadIdx.x + u * kGbThreads;
            if (QL) QL[(size_t)j * ne + e] = v[u];
            if (trace) tr += a[u].x * v[u].x + a[u].y * v[u].y;
        }
    }
    if (split) gb_count_and_fold(j, ne, xoff, xcnt, xpart, QL, &s_last);
    if (trace) {
        const double t = block_sum((double)tr);     // the patch's share in FP64
        if (threadIdx.x == 0) trace[j] = t;         // k_cost sums the shares in order
    }
}

// --------------------------------------------------------------------------
// SVT (Eq. 18): k_svt in svt.cuh (Gram matrix + two-sided Jacobi per patch)
// --------------------------------------------------------------------------
}  // namespace mrf
#include "svt.cuh"
namespace mrf {

// --------------------------------------------------------------------------
// Z step + X step (Eq. 12 and 19), gathered per voxel:
//   alpha <- (alpha - mu (grad + lambda1 Q^*(QL)) + c Q^*(P)) / (1 + c cnt)
// --------------------------------------------------------------------------
__device__ __forceinline__ int covering(const PatchGeom& g, int y, int* list) {
    int n = 0;
    const int hi = min(g.cnt - 1, y / g.s);
    const int lo = max(0, hi - (g.p + g.s - 1) / g.s);
    for (int i = lo; i <= hi; ++i) {
        const int o = g.origin(i);
        if (o <= y && y < o + g.p) list[n++] = i;
    }
    const int e = g.cnt - 1;
    if (e > hi) {
        const int o = g.origin(e);
        if (o <= y && y < o + g.p) list[n++] = e;
    }
    return n;
}

__global__ void k_xupdate(float2* __restrict__ alpha, const float2* __restrict__ grad,
                          const float2* __restrict__ QL, const float2* __restrict__ P, PatchGeom g, int K,
                          float mu, float c, const float* __restrict__ lam1, int literal,
                          float* __restrict__ cnt_out) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t N = (size_t)g.n * g.n;
    if (e >= N * K) return;
    const int vox = (int)(e / K), k = (int)(e - (size_t)vox * K);
    const int y = vox / g.n, x = vox - y * g.n;
    int ly[16], lx[16];
    const int ny_ = covering(g, y, ly), nx_ = covering(g, x, lx);
    const int pp = g.p * g.p;
    float2 h = make_float2(0.f, 0.f), qp = make_float2(0.f, 0.f);
    for (int a = 0; a < ny_; ++a)
        for (int b = 0; b < nx_; ++b) {
            const int i = ly[a] * g.cnt + lx[b];
            const int row = (y - g.origin(ly[a])) * g.p + (x - g.origin(lx[b]));
            const size_t o = ((size_t)i * pp + row) * K + k;
            if (QL) h = cadd(h, QL[o]);
            if (P) qp = cadd(qp, P[o]);
        }
    const float cnt = (float)(ny_ * nx_);
    if (cnt_out) {
        if (k == 0) cnt_out[vox] = cnt;
        return;
    }
    const float l1 = *lam1;
    const float2 z = csub(alpha[e], cscale(cadd(grad[e], cscale(h, l1)), mu));
    const float den = literal ? 1.f + c : 1.f + c * cnt;
    alpha[e] = cscale(cadd(z, cscale(qp, c)), 1.f / den);
}

// The cost of Algorithm 1 from its shares, each summed in a fixed order (one
// block), so that it is the same on every run: shares[0, np) the patches'
// shares of Tr(Q L Q^H), shares[np, 2 np) their nuclear norms, shares[2 np,
// 2 np + kNorm2Blocks) the blocks' parts of ||r||^2.  The cost goes to
// cost[*slot], and the slot moves on (the iteration count modulo cap, kept on
// the device so that a recorded iteration replays unchanged).
__global__ void k_cost(const double* __restrict__ shares, int np, const float* __restrict__ lam1, float lam2,
                       double* __restrict__ cost, int* __restrict__ slot, int cap) {
    double t = 0.0, nu = 0.0, r2 = 0.0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        t += shares[j];
        nu += shares[np + j];
    }
    for (int j = threadIdx.x; j < kNorm2Blocks; j += blockDim.x) r2 += shares[2 * np + j];
    t = block_sum(t);
    nu = block_sum(nu);
    r2 = block_sum(r2);
    if (threadIdx.x == 0) {
        const int q = *slot;
        cost[q] = 0.5 * r2 + (double)(*lam1) * t + (double)lam2 * nu;
        *slot = q + 1 == cap ? 0 : q + 1;
    }
}

__global__ void k_maps(const float* __restrict__ t1t2, const float* __restrict__ pd, const int* __restrict__ idx,
                       int N, float inv_gamma, float* __restrict__ t1, float* __restrict__ t2,
                       float* __restrict__ pdo, int* __restrict__ idxo) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    if (t1) t1[v] = t1t2[2 * v];
    if (t2) t2[v] = t1t2[2 * v + 1];
    if (pdo) pdo[v] = pd[v] * inv_gamma;
    if (idxo) idxo[v] = idx[v];
}

}  // namespace mrf

// ----------------------------------------------------------------------------
// recon object
// ----------------------------------------------------------------------------
struct mrf_recon_s {
    mrf_plan_s* plan = nullptr;
    mrf_recon_params prm{};
    int K = 0, m = 0, N = 0, np = 0, pp = 0, mode = 0;
    mrf::PatchGeom g{};
    const float2* phi = nullptr;
    const float2* dict_c = nullptr;
    const float* atom_norm2 = nullptr;
    const float* lut = nullptr;
    float t1max = 1.f, t2max = 1.f;
    double a = 1.0, gamma = 1.0;
    mrf::MatchWorkspace mws;
    // device buffers
    float2 *alpha = nullptr, *grad = nullptr, *r = nullptr, *bs = nullptr, *QL = nullptr, *P = nullptr;
    float* cnt = nullptr;
    float *t1t2 = nullptr, *pd = nullptr;
    int* idx = nullptr;
    int* F = nullptr;
    int* nbr = nullptr;
    unsigned* d2 = nullptr;
    mrf::KnnWorkspace knn;      // kNN scratch (operand tiles, per-partition lists)
    float *w = nullptr, *rw = nullptr, *deg = nullptr;
    int *rcnt = nullptr, *roff = nullptr, *rpos = nullptr, *rsrc = nullptr, *rsrc_tmp = nullptr;
    // the graph term's cut lists: extra-chunk offsets [np + 1], patch of each
    // extra chunk and the chunks' partial sums [gb_max_extra][p x p x K]
    bool graph_built = false;   // nbr holds a graph (the previous one seeds the next kNN search)
    int *xoff = nullptr, *xpatch = nullptr, *xcnt = nullptr;     // xcnt: [np] blocks done per cut patch
    float2* xpart = nullptr;
    float* rw_tmp = nullptr;
    float* scal = nullptr;      // [0] sigma2, [1] lmax, [2] lam1, [3] scratch, [4] lam1 of the cost
    // the forward graph (nbr, w, deg) as the iteration began, read by the
    // cost trace while the rebuild replaces the live copy (concurrent mode)
    int* nbr_c = nullptr;
    float *w_c = nullptr, *deg_c = nullptr;
    double* acc = nullptr;      // [0..1] dot, [2] norm (the power iteration for a)
    // [np] the patches' shares of Tr(Q L Q^H), [np] their nuclear norms,
    // [kNorm2Blocks] the blocks' parts of ||r||^2 (summed by k_cost)
    double* trace = nullptr;
    int* cost_slot = nullptr;   // [1] where the next cost goes (iterations done modulo cost_cap)
    cudaGraphExec_t iter_exec = nullptr;   // one recorded iteration (replayed), or none
    long long iter_kernels = 0;            // kernels in it
    double* cost = nullptr;     // [cap] cost history
    int cost_cap = 0, iters_done = 0;
    float2* svt_v = nullptr;    // [np][svt_kp][svt_kp] right singular vectors of the last SVT
    int svt_kp = 0, svt_warm = 0;
    unsigned long long* svt_stats = nullptr;   // executed Jacobi sweeps and rotations, summed over patches
    double svt_patch_launches = 0.0;           // patches x SVT launches since create
    // learned matcher (MRF_RECON_LEARNED)
    float t1min = 0.f, t2min = 0.f;
    float *mlp_x = nullptr, *mlp_norm = nullptr, *mlp_y = nullptr;
    int *fb_list = nullptr, *fb_count = nullptr;
    float2* fb_x = nullptr;
    mrf::TcSlice* fb_table = nullptr;
    // concurrency inside one iteration: two side streams and their events
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // [2]: where a recorded iteration replays
    cudaEvent_t ev[7] = {};                               // [5], [6]: fork to and join from side[2]
    std::vector<void*> owned;
};

namespace mrf {

template <typename T>
static mrf_status dalloc(mrf_recon_s* R, T** p, size_t n) {
    MRF_CUDA(cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(n, 1)));
    R->owned.push_back(*p);
    return MRF_OK;
}

static void free_recon(mrf_recon_s* R) {
    if (!R) return;
    if (R->iter_exec) cudaGraphExecDestroy(R->iter_exec);
    for (cudaStream_t t : R->side)
        if (t) cudaStreamDestroy(t);
    for (cudaEvent_t e : R->ev)
        if (e) cudaEventDestroy(e);
    for (void* p : R->owned) cudaFree(p);
    delete R;
}

// dynamic shared memory above the default 48 KB needs an opt-in per kernel
template <typename Kern>
static mrf_status svt_smem(Kern k, size_t bytes) {
    if (bytes > 48 * 1024) MRF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return MRF_OK;
}

static mrf_status svt(mrf_recon_s* R, const float2* alpha, float2* P, double* nuc, cudaStream_t s) {
    const int K = R->K;
    const int rows = R->pp;
    const float tau = 1.0f / R->prm.beta;
    const int warm = R->svt_warm;
    const int KP = R->svt_kp;
    // two patches per warp (16 lanes, R = rows / 16) up to 64 rows and KP <= 12;
    // one patch per warp otherwise
    const bool half = rows <= 64 && KP <= 12;
    const int per_block = half ? 8 : 4;
    const unsigned blocks = (unsigned)((R->np + per_block - 1) / per_block);
#define MRF_SVT(RR, KK, LL)                                                                                   \
    do {                                                                                                       \
        const size_t sm = (size_t)(128 / LL) * svt_patch_f2(KK) * sizeof(float2);                              \
        MRF_PROPAGATE(svt_smem(k_svt<RR, KK, LL>, sm));                                                        \
        k_svt<RR, KK, LL><<<blocks, 128, sm, s>>>(alpha, R->g, K, tau, P, nuc, R->svt_v, warm, R->svt_stats); \
    } while (0)
    if (half && rows <= 32) {
        switch (KP) {
            case 4: MRF_SVT(2, 4, 16); break;
            case 8: MRF_SVT(2, 8, 16); break;
            case 10: MRF_SVT(2, 10, 16); break;
            default: MRF_SVT(2, 12, 16); break;
        }
    } else if (half) {
        switch (KP) {
            case 4: MRF_SVT(4, 4, 16); break;
            case 8: MRF_SVT(4, 8, 16); break;
            case 10: MRF_SVT(4, 10, 16); break;
            default: MRF_SVT(4, 12, 16); break;
        }
    } else if (rows <= 64) {
        MRF_SVT(2, 16, 32);
    } else {
        switch (KP) {
            case 4: MRF_SVT(4, 4, 32); break;
            case 8: MRF_SVT(4, 8, 32); break;
            case 10: MRF_SVT(4, 10, 32); break;
            case 12: MRF_SVT(4, 12, 32); break;
            default: MRF_SVT(4, 16, 32); break;
        }
    }
#undef MRF_SVT
    MRF_LAUNCHED_AS("k_svt", s);
    R->svt_warm = 1;
    R->svt_patch_launches += R->np;
    return MRF_OK;
}

// L from the current maps, then lambda1
static mrf_status build_graph(mrf_recon_s* R, cudaStream_t s) {
    const int np = R->np, knn = R->prm.knn, FD = 2 * R->pp;
    k_features<<<(unsigned)(((size_t)np * R->pp + 255) / 256), 256, 0, s>>>(R->t1t2, R->g, (double)R->t1max,
                                                                             (double)R->t2max,
                                                                             (FD + 3) / 4 * 4, R->F);
    MRF_LAUNCHED_AS("k_features", s);
    // from the second build on, the previous graph seeds the search (the
    // result does not depend on it)
    MRF_PROPAGATE(knn_run(R->knn, R->F, np, FD, (FD + 3) / 4 * 4, knn, R->nbr, R->d2, s,
                          R->graph_built ? R->nbr : nullptr));
    R->graph_built = true;
    const int ne = np * knn;
    k_median_nonzero<<<1, kMedianThreads, 0, s>>>(R->d2, ne, R->scal + 0);
    MRF_LAUNCHED_AS("k_median_nonzero", s);
    MRF_CUDA(cudaMemsetAsync(R->rcnt, 0, sizeof(int) * np, s));
    MRF_CUDA(cudaMemsetAsync(R->rpos, 0, sizeof(int) * np, s));
    k_edge_weights<<<(ne + 255) / 256, 256, 0, s>>>(R->nbr, R->d2, ne, R->scal + 0, R->w, R->rcnt);
    MRF_LAUNCHED_AS("k_edge_weights", s);
    k_scan_graph<<<1, 1024, 0, s>>>(R->rcnt, np, knn, R->roff, R->xoff, R->xpatch, R->xcnt);
    MRF_LAUNCHED_AS("k_scan_graph", s);
    k_fill_reverse<<<(ne + 255) / 256, 256, 0, s>>>(R->nbr, R->w, ne, knn, R->roff, R->rpos, R->rsrc_tmp,
                                                   R->rw_tmp);
    MRF_LAUNCHED_AS("k_fill_reverse", s);
    MRF_CUDA(cudaMemsetAsync(R->scal + 1, 0, sizeof(float), s));     // max(L), raised by k_degree
    {
        const size_t smd = sizeof(unsigned) * 2 * (size_t)((np + 31) / 32) * kDegWarps;
        MRF_CUDA(cudaFuncSetAttribute(k_degree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd));
        k_degree<<<(unsigned)((np + kDegWarps - 1) / kDegWarps), kDegWarps * 32, smd, s>>>(
            R->w, np, knn, R->roff, R->rsrc_tmp, R->rw_tmp, R->rsrc, R->rw, R->deg,
            reinterpret_cast<unsigned*>(R->scal + 1));
    }
    MRF_LAUNCHED_AS("k_degree", s);
    k_lambda<<<1, 1, 0, s>>>(R->scal + 1, R->prm.lam1_0, (R->prm.flags & MRF_RECON_LITERAL_LAMBDA1) ? 1 : 0,
                             R->scal + 2);
    MRF_LAUNCHED_AS("k_lambda", s);
    return MRF_OK;
}

static mrf_status match_maps(mrf_recon_s* R, cudaStream_t s) {
    return match_run(R->mws, R->alpha, R->N, R->K, R->dict_c, R->m, R->prm.match_precision, R->lut, R->idx,
                     R->pd, R->t1t2, 1.0f, s, R->mws.cand);
}

// Learned matcher: decode the network outputs into maps; a fingerprint
// mapped outside the dictionary's [T1min, T1max] x [T2min, T2max] box, to
// T1 < T2, or to a non-finite value joins the fallback list (matched
// exhaustively next).  idx = -1 marks a learned (off-grid) map value.
__global__ void k_learned_decode(const float* __restrict__ y, const float* __restrict__ norm, int n, float t1min,
                                 float t1max, float t2min, float t2max, float pd_scale, float lt1, float lt1r,
                                 float lt2, float lt2r, float* __restrict__ t1t2, float* __restrict__ pd,
                                 int* __restrict__ idx, int* __restrict__ list, int* __restrict__ count) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const float t1 = expf(lt1 + 0.5f * (y[3 * v] + 1.f) * lt1r);
    const float t2 = expf(lt2 + 0.5f * (y[3 * v + 1] + 1.f) * lt2r);
    const float r = y[3 * v + 2] * pd_scale * norm[v];
    const bool ok = t1 >= t1min && t1 <= t1max && t2 >= t2min && t2 <= t2max && t1 >= t2 && isfinite(r);
    t1t2[2 * v] = ok ? t1 : 0.f;
    t1t2[2 * v + 1] = ok ? t2 : 0.f;
    pd[v] = ok ? fmaxf(r, 0.f) : 0.f;
    idx[v] = -1;
    if (!ok) list[atomicAdd(count, 1)] = v;
}

// compact the fallback fingerprints and give the matcher's slice its row count
__global__ void k_fallback_gather(const float2* __restrict__ alpha, int K, const int* __restrict__ list,
                                  const int* __restrict__ count, float2* __restrict__ xc, TcSlice* __restrict__ table) {
    const int c = *count;
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e == 0) table->n = c;
    if (e >= (size_t)c * K) return;
    const int i = (int)(e / K), k = (int)(e - (size_t)i * K);
    xc[e] = alpha[(size_t)list[i] * K + k];
}

__global__ void k_fallback_scatter(const int* __restrict__ list, const int* __restrict__ count,
                                   const int* __restrict__ best_idx, const float2* __restrict__ best_ip,
                                   const float* __restrict__ norm2, const float* __restrict__ lut,
                                   float* __restrict__ t1t2, float* __restrict__ pd, int* __restrict__ idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const int v = list[i], k = best_idx[i];
    const float n2 = norm2[k];
    idx[v] = k;
    t1t2[2 * v] = lut[2 * k];
    t1t2[2 * v + 1] = lut[2 * k + 1];
    pd[v] = n2 > 0.f ? fmaxf(best_ip[i].x / n2, 0.f) : 0.f;
}

static mrf_status learned_maps(mrf_recon_s* R, cudaStream_t s) {
    const int N = R->N;
    const float* dec = mlp_decode(R->prm.mlp);
    MRF_PROPAGATE(mlp_features(R->alpha, N, R->mlp_x, R->mlp_norm, s));
    MRF_PROPAGATE(mlp_infer(R->prm.mlp, R->mlp_x, N, R->mlp_y, s));
    MRF_CUDA(cudaMemsetAsync(R->fb_count, 0, sizeof(int), s));
    const float lt1 = logf(dec[0]), lt1r = logf(dec[1]) - lt1, lt2 = logf(dec[2]), lt2r = logf(dec[3]) - lt2;
    k_learned_decode<<<(N + 255) / 256, 256, 0, s>>>(R->mlp_y, R->mlp_norm, N, R->t1min, R->t1max, R->t2min,
                                                     R->t2max, dec[4], lt1, lt1r, lt2, lt2r, R->t1t2, R->pd,
                                                     R->idx, R->fb_list, R->fb_count);
    MRF_LAUNCHED_AS("k_learned_decode", s);
    const size_t NK = (size_t)N * R->K;
    k_fallback_gather<<<(unsigned)((NK + 255) / 256), 256, 0, s>>>(R->alpha, R->K, R->fb_list, R->fb_count,
                                                                    R->fb_x, R->fb_table);
    MRF_LAUNCHED_AS("k_fallback_gather", s);
    // exhaustive matching of the fallback list: a launch sized for all N rows,
    // blocks past the list's (device-side) length return at once
    MRF_PROPAGATE(match_tc_batch(R->mws, R->fb_table, 1, (N + 127) / 128, R->K, R->m,
                                 tc_form(R->prm.match_precision), s));
    k_fallback_scatter<<<(N + 255) / 256, 256, 0, s>>>(R->fb_list, R->fb_count, R->mws.best_idx, R->mws.best_ip,
                                                       R->mws.norm2, R->lut, R->t1t2, R->pd, R->idx);
    MRF_LAUNCHED_AS("k_fallback_scatter", s);
    return MRF_OK;
}

// Q(X) L into QL, or (QL null) each patch's share of Tr(Q L Q^H) from the
// forward kNN entries alone into trace[np], of the live graph or (snap) of
// the copy taken when the iteration began
static mrf_status graph_pass(mrf_recon_s* R, float2* QL, double* trace, cudaStream_t s, bool snap = false) {
    // Q(X)L reads the reverse lists, which only the live graph has, and cuts
    // the long ones (extra chunks first in the grid)
    const int grid = R->np + (QL ? gb_max_extra(R->np, R->prm.knn) : 0);
    k_graph_blocks<<<grid, kGbThreads, 0, s>>>(R->alpha, R->g, R->K, snap ? R->nbr_c : R->nbr, snap ? R->w_c : R->w,
                                               R->prm.knn, R->roff, R->rsrc, R->rw, snap ? R->deg_c : R->deg,
                                               QL ? 1 : 0, QL ? R->xoff : nullptr, R->xpatch, R->xpart, R->xcnt, QL,
                                               trace);
    MRF_LAUNCHED_AS(QL ? "k_graph_blocks" : "k_graph_blocks(trace)", s);
    return MRF_OK;
}

// the steps of one iteration before the matching step (stream-ordered,
// capturable); the cost terms only when cost is set
static mrf_status iteration_pre(mrf_recon_s* R, int it, bool cost, cudaStream_t s) {
    const size_t NK = (size_t)R->N * R->K;
    const float inv_a = (float)(1.0 / R->a);
    MRF_PROPAGATE(graph_pass(R, R->QL, nullptr, s));
    const float c = R->prm.mu * R->prm.lam2 * R->prm.beta;
    k_xupdate<<<(unsigned)((NK + 255) / 256), 256, 0, s>>>(
        R->alpha, R->grad, R->QL, R->P, R->g, R->K, R->prm.mu, c, R->scal + 2,
        (R->prm.flags & MRF_RECON_LITERAL_XUPDATE) ? 1 : 0, nullptr);
    MRF_LAUNCHED_AS("k_xupdate", s);
    MRF_PROPAGATE(subspace_forward(R->plan, R->alpha, R->phi, R->K, inv_a, R->bs, R->r, R->mode, s));
    // the next pass's gradient of the data term, A*(r), from this residual
    MRF_PROPAGATE(subspace_adjoint(R->plan, R->r, R->phi, R->K, inv_a, R->grad, R->mode, s));
    MRF_PROPAGATE(svt(R, R->alpha, R->P, cost ? R->trace + R->np : nullptr, s));
    if (cost) {
        const size_t nr = (size_t)R->plan->T * R->plan->ns;
        k_norm2_part<<<kNorm2Blocks, 256, 0, s>>>(R->r, nr, R->trace + 2 * (size_t)R->np);
        MRF_LAUNCHED_AS("k_norm2_part", s);
        MRF_PROPAGATE(graph_pass(R, nullptr, R->trace, s));
        k_cost<<<1, 1024, 0, s>>>(R->trace, R->np, R->scal + 2, R->prm.lam2, R->cost, R->cost_slot, R->cost_cap);
        MRF_LAUNCHED_AS("k_cost", s);
    }
    return MRF_OK;
}

// One iteration of the loop body, with its independent steps on three
// streams (stream-ordered, ends joined into s):
//   s:       (join) X update -> forward -> |r|^2 -> next A*(r) -> (join) cost
//   side[1]: graph copy, graph term Q(X)L (the previous graph) ^ join
//   side[0]:                     SVT of the new iterate -> P, sum sigma -> cost trace
//   side[1]:                     matching -> graph rebuild
// The forward operator, the SVT and the matching all read only the new
// iterate; the graph rebuild only the new maps; the cost trace reads the copy
// of the graph taken at the start, so the rebuild need not wait for it; the
// shares they write are distinct ranges.  The data term's gradient
// A*(r) for the next pass is computed as soon as this pass's residual is
// (create and restore compute the first one), so it runs beside the matching
// and the graph rebuild instead of beside the next graph term.
static mrf_status iteration(mrf_recon_s* R, int it, cudaStream_t s) {
    const bool cost = !(R->prm.flags & MRF_RECON_NO_COST);
    if (R->prm.flags & MRF_RECON_SERIAL) {
        // the same steps one after another on s
        MRF_PROPAGATE(iteration_pre(R, it, cost, s));
        if (R->prm.flags & MRF_RECON_LEARNED) MRF_PROPAGATE(learned_maps(R, s));
        else MRF_PROPAGATE(match_maps(R, s));
        return build_graph(R, s);
    }
    const size_t NK = (size_t)R->N * R->K;
    const float inv_a = (float)(1.0 / R->a);
    cudaStream_t sb = R->side[0], sc = R->side[1];
    // (profiler marks after each cross-stream wait: a side stream's next kernel
    // is charged from the point its inputs are ready)
    auto mark = [](cudaStream_t t) { mrf_profile_mark(reinterpret_cast<mrf_stream>(t)); };
    MRF_CUDA(cudaEventRecord(R->ev[0], s));
    MRF_CUDA(cudaStreamWaitEvent(sc, R->ev[0], 0));
    mark(sc);
    if (cost) {
        const int ne = R->np * R->prm.knn;
        k_graph_snapshot<<<(unsigned)((ne + 255) / 256), 256, 0, sc>>>(R->nbr, R->w, R->deg, R->scal + 2, ne, R->np,
                                                                    R->nbr_c, R->w_c, R->deg_c, R->scal + 4);
        MRF_LAUNCHED_AS("k_graph_snapshot", sc);
    }
    MRF_PROPAGATE(graph_pass(R, R->QL, nullptr, sc));
    MRF_CUDA(cudaEventRecord(R->ev[1], sc));
    MRF_CUDA(cudaStreamWaitEvent(s, R->ev[1], 0));
    mark(s);
    const float c = R->prm.mu * R->prm.lam2 * R->prm.beta;
    k_xupdate<<<(unsigned)((NK + 255) / 256), 256, 0, s>>>(
        R->alpha, R->grad, R->QL, R->P, R->g, R->K, R->prm.mu, c, R->scal + 2,
        (R->prm.flags & MRF_RECON_LITERAL_XUPDATE) ? 1 : 0, nullptr);
    MRF_LAUNCHED_AS("k_xupdate", s);
    MRF_CUDA(cudaEventRecord(R->ev[2], s));                  // the new iterate
    MRF_CUDA(cudaStreamWaitEvent(sb, R->ev[2], 0));
    MRF_CUDA(cudaStreamWaitEvent(sc, R->ev[2], 0));
    mark(sb);
    mark(sc);
    MRF_PROPAGATE(svt(R, R->alpha, R->P, cost ? R->trace + R->np : nullptr, sb));
    if (cost) MRF_PROPAGATE(graph_pass(R, nullptr, R->trace, sb, true));     // trace with this iteration's graph
    MRF_CUDA(cudaEventRecord(R->ev[3], sb));
    if (R->prm.flags & MRF_RECON_LEARNED) MRF_PROPAGATE(learned_maps(R, sc));
    else MRF_PROPAGATE(match_maps(R, sc));
    MRF_PROPAGATE(build_graph(R, sc));
    MRF_CUDA(cudaEventRecord(R->ev[4], sc));
    MRF_PROPAGATE(subspace_forward(R->plan, R->alpha, R->phi, R->K, inv_a, R->bs, R->r, R->mode, s));
    if (cost) {
        const size_t nr = (size_t)R->plan->T * R->plan->ns;
        k_norm2_part<<<kNorm2Blocks, 256, 0, s>>>(R->r, nr, R->trace + 2 * (size_t)R->np);
        MRF_LAUNCHED_AS("k_norm2_part", s);
    }
    // the next pass's gradient of the data term, A*(r), beside the matching
    // and graph rebuild (it needs only this residual)
    MRF_PROPAGATE(subspace_adjoint(R->plan, R->r, R->phi, R->K, inv_a, R->grad, R->mode, s));
    MRF_CUDA(cudaStreamWaitEvent(s, R->ev[3], 0));
    MRF_CUDA(cudaStreamWaitEvent(s, R->ev[4], 0));
    mark(s);
    if (cost) {
        k_cost<<<1, 1024, 0, s>>>(R->trace, R->np, R->scal + 4, R->prm.lam2, R->cost, R->cost_slot, R->cost_cap);
        MRF_LAUNCHED_AS("k_cost", s);
    }
    return MRF_OK;
}

static mrf_status create(mrf_recon_s* R, const float2* b, cudaStream_t s) {
    mrf_plan_s* p = R->plan;
    const int K = R->K, N = R->N, np = R->np, knn = R->prm.knn;
    const size_t NK = (size_t)N * K, nr = (size_t)p->T * p->ns;
    MRF_PROPAGATE(dalloc(R, &R->alpha, NK));
    MRF_PROPAGATE(dalloc(R, &R->grad, NK));
    MRF_PROPAGATE(dalloc(R, &R->r, nr));
    MRF_PROPAGATE(dalloc(R, &R->bs, nr));
    MRF_PROPAGATE(dalloc(R, &R->QL, (size_t)np * R->pp * K));
    MRF_PROPAGATE(dalloc(R, &R->P, (size_t)np * R->pp * K));
    MRF_PROPAGATE(dalloc(R, &R->cnt, N));
    MRF_PROPAGATE(dalloc(R, &R->t1t2, 2 * (size_t)N));
    MRF_PROPAGATE(dalloc(R, &R->pd, N));
    MRF_PROPAGATE(dalloc(R, &R->idx, N));
    const int FD4 = (2 * R->pp + 3) / 4 * 4;
    MRF_PROPAGATE(dalloc(R, &R->F, (size_t)np * FD4));
    MRF_CUDA(cudaMemsetAsync(R->F, 0, sizeof(int) * (size_t)np * FD4, s));
    MRF_PROPAGATE(R->knn.reserve(np, 2 * R->pp, knn));
    MRF_PROPAGATE(dalloc(R, &R->nbr, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->d2, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->w, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->rw, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->rsrc, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->rsrc_tmp, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->rw_tmp, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->deg, np));
    MRF_PROPAGATE(dalloc(R, &R->nbr_c, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->w_c, (size_t)np * knn));
    MRF_PROPAGATE(dalloc(R, &R->deg_c, np));
    MRF_PROPAGATE(dalloc(R, &R->rcnt, np));
    MRF_PROPAGATE(dalloc(R, &R->rpos, np));
    MRF_PROPAGATE(dalloc(R, &R->roff, np + 1));
    {
        const int xmax = mrf::gb_max_extra(np, knn);
        MRF_PROPAGATE(dalloc(R, &R->xoff, np + 1));
        MRF_PROPAGATE(dalloc(R, &R->xpatch, xmax));
        MRF_PROPAGATE(dalloc(R, &R->xpart, (size_t)xmax * R->pp * K));
        MRF_PROPAGATE(dalloc(R, &R->xcnt, np));
    }
    MRF_PROPAGATE(dalloc(R, &R->scal, 8));
    MRF_PROPAGATE(dalloc(R, &R->acc, 8));
    MRF_PROPAGATE(dalloc(R, &R->trace, 2 * (size_t)np + kNorm2Blocks));
    MRF_PROPAGATE(dalloc(R, &R->cost_slot, 1));
    MRF_CUDA(cudaMemsetAsync(R->cost_slot, 0, sizeof(int), s));
    R->svt_kp = K <= 4 ? 4 : K <= 8 ? 8 : K == 10 ? 10 : K <= 12 ? 12 : 16;
    MRF_PROPAGATE(dalloc(R, &R->svt_v, (size_t)np * R->svt_kp * R->svt_kp));
    MRF_PROPAGATE(dalloc(R, &R->svt_stats, 2));
    MRF_CUDA(cudaMemsetAsync(R->svt_stats, 0, 2 * sizeof(unsigned long long), s));
    R->cost_cap = 1024;
    MRF_PROPAGATE(dalloc(R, &R->cost, R->cost_cap));
    MRF_PROPAGATE(R->mws.reserve(N, R->m));
    // the loop's matching calls score the same N rows every time: each call
    // starts from the previous call's candidates (-1 at first: no seed)
    MRF_CUDA(cudaMemsetAsync(R->mws.cand, 0xff, sizeof(int) * (size_t)N * kTopK, s));
    MRF_PROPAGATE(ensure_subspace_workspace(p, K));
    MRF_PROPAGATE(match_prepare(R->mws, R->dict_c, R->atom_norm2, R->m, K, 0, s));
    if (R->prm.flags & MRF_RECON_LEARNED) {
        // network inputs/outputs and the fallback list with its one-slice table
        const int form = tc_form(R->prm.match_precision);
        MRF_PROPAGATE(tc_prepare_operand(R->mws, R->dict_c, R->m, K, form, s));
        MRF_PROPAGATE(dalloc(R, &R->mlp_x, (size_t)N * kMlpIn));
        MRF_PROPAGATE(dalloc(R, &R->mlp_norm, (size_t)N));
        MRF_PROPAGATE(dalloc(R, &R->mlp_y, (size_t)N * kMlpOut));
        MRF_PROPAGATE(dalloc(R, &R->fb_list, (size_t)N));
        MRF_PROPAGATE(dalloc(R, &R->fb_count, 1));
        MRF_PROPAGATE(dalloc(R, &R->fb_x, (size_t)N * K));
        MRF_PROPAGATE(dalloc(R, &R->fb_table, 1));
        const TcSlice t{R->fb_x, 0, 0, R->mws.best_idx, R->mws.best_ip,
                        static_cast<const unsigned char*>(R->mws.tc_b), R->mws.wscore, R->dict_c};
        MRF_CUDA(cudaMemcpyAsync(R->fb_table, &t, sizeof(t), cudaMemcpyHostToDevice, s));
        MRF_CUDA(cudaStreamSynchronize(s));
    }
    // t1max, t2max of the look-up table
    {
        std::vector<float> lut((size_t)R->m * 2);
        MRF_CUDA(cudaMemcpyAsync(lut.data(), R->lut, lut.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
        MRF_CUDA(cudaStreamSynchronize(s));
        R->t1max = R->t2max = 0.f;
        R->t1min = R->t2min = 3.4e38f;
        for (int i = 0; i < R->m; ++i) {
            R->t1max = std::max(R->t1max, lut[2 * i]);
            R->t2max = std::max(R->t2max, lut[2 * i + 1]);
            R->t1min = std::min(R->t1min, lut[2 * i]);
            R->t2min = std::min(R->t2min, lut[2 * i + 1]);
        }
        if (!(R->t1max > 0.f)) R->t1max = 1.f;
        if (!(R->t2max > 0.f)) R->t2max = 1.f;
    }
    // coverage counts
    k_xupdate<<<(unsigned)((NK + 255) / 256), 256, 0, s>>>(R->alpha, nullptr, nullptr, nullptr, R->g, K, 0.f, 0.f,
                                                          nullptr, 0, R->cnt);
    MRF_LAUNCHED_AS("k_xupdate", s);
    // a = ||A P_S||_2 by power iteration on coefficient images
    if (R->prm.a_norm > 0.f) {
        R->a = R->prm.a_norm;
    } else {
        k_fill<<<nblk(NK), 256, 0, s>>>(R->alpha, NK, make_float2((float)(1.0 / std::sqrt((double)NK)), 0.f));
        MRF_LAUNCHED_AS("k_fill", s);
        // (the steps queue back to back: each normalisation reads its norm on
        // the device; the estimate and the last norm come back once)
        double h[4] = {0.0, 0.0, 0.0, 0.0};
        for (int it = 0; it < R->prm.power_iters; ++it) {
            MRF_PROPAGATE(subspace_forward(p, R->alpha, R->phi, K, 1.0f, nullptr, R->r, R->mode, s));
            MRF_PROPAGATE(subspace_adjoint(p, R->r, R->phi, K, 1.0f, R->grad, R->mode, s));
            MRF_CUDA(cudaMemsetAsync(R->acc, 0, 4 * sizeof(double), s));
            k_dot_acc<<<nblk(NK), 256, 0, s>>>(R->alpha, R->grad, NK, R->acc + 0);
            MRF_LAUNCHED_AS("k_dot_acc", s);
            k_norm2_acc<<<nblk(NK), 256, 0, s>>>(R->grad, NK, R->acc + 2);
            MRF_LAUNCHED_AS("k_norm2_acc", s);
            k_scale_by_norm<<<nblk(NK), 256, 0, s>>>(R->grad, NK, R->acc + 2, R->alpha);
            MRF_LAUNCHED_AS("k_scale_by_norm", s);
        }
        if (R->prm.power_iters > 0) {
            MRF_CUDA(cudaMemcpyAsync(h, R->acc, sizeof(h), cudaMemcpyDeviceToHost, s));
            MRF_CUDA(cudaStreamSynchronize(s));
        }
        const double lam = h[0];
        MRF_REQUIRE(R->prm.power_iters <= 0 || h[2] > 0.0,
                    "mrf_recon_create: the operator maps the start vector to zero");
        MRF_REQUIRE(lam > 0.0, "mrf_recon_create: non-positive operator norm estimate");
        R->a = std::sqrt(lam);
    }
    const float inv_a = (float)(1.0 / R->a);
    // X^0 = P_S((A/a)^H (b/a)), matched for the PD scale gamma
    MRF_PROPAGATE(subspace_adjoint(p, b, R->phi, K, inv_a * inv_a, R->alpha, R->mode, s));
    MRF_PROPAGATE(match_maps(R, s));
    if (R->prm.x_scale > 0.f) {
        R->gamma = R->prm.x_scale;
    } else {
        k_max<<<1, 1024, 0, s>>>(R->pd, N, R->scal + 3);
        MRF_LAUNCHED_AS("k_max", s);
        float mx = 0.f;
        MRF_CUDA(cudaMemcpyAsync(&mx, R->scal + 3, sizeof(float), cudaMemcpyDeviceToHost, s));
        MRF_CUDA(cudaStreamSynchronize(s));
        R->gamma = mx > 0.f ? R->prm.pd_target / (double)mx : 1.0;
    }
    const float gm = (float)R->gamma;
    k_scale<<<nblk(NK), 256, 0, s>>>(R->alpha, NK, gm);
    MRF_LAUNCHED_AS("k_scale", s);
    k_scale_copy<<<nblk(nr), 256, 0, s>>>(b, nr, (float)(R->gamma / R->a), R->bs);
    MRF_LAUNCHED_AS("k_scale_copy", s);
    MRF_PROPAGATE(match_maps(R, s));                     // maps in the scaled units
    MRF_PROPAGATE(build_graph(R, s));
    MRF_PROPAGATE(subspace_forward(p, R->alpha, R->phi, K, inv_a, R->bs, R->r, R->mode, s));
    MRF_PROPAGATE(subspace_adjoint(p, R->r, R->phi, K, inv_a, R->grad, R->mode, s));   // the first pass's A*(r)
    MRF_PROPAGATE(svt(R, R->alpha, R->P, nullptr, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    return MRF_OK;
}

}  // namespace mrf

using namespace mrf;

extern "C" mrf_status mrf_graph_sigma2(const unsigned* d2, int ne, float* sigma2, mrf_stream stream) {
    MRF_REQUIRE(ne >= 0 && sigma2 && (ne == 0 || d2), "mrf_graph_sigma2: ne < 0 or a null pointer");
    cudaStream_t s = as_stream(stream);
    k_median_nonzero<<<1, kMedianThreads, 0, s>>>(d2, ne, sigma2);
    MRF_CUDA(cudaGetLastError());
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_create(mrf_recon* out, mrf_plan plan, const mrf_recon_params* prm,
                                       const mrf_c64* phi, int K, const mrf_c64* dict_c, const float* atom_norm2,
                                       const float* lut, int m, const mrf_c64* b, mrf_stream stream) {
    MRF_REQUIRE(out != nullptr, "mrf_recon_create: out is NULL");
    *out = nullptr;
    MRF_REQUIRE(plan && prm && phi && dict_c && atom_norm2 && lut && b, "mrf_recon_create: NULL argument");
    MRF_REQUIRE(K >= 1 && K <= 16, "mrf_recon_create: K must be in [1, 16] (got %d)", K);
    MRF_REQUIRE(m >= 1, "mrf_recon_create: m must be >= 1");
    MRF_REQUIRE(plan->nx <= 256, "mrf_recon_create: images up to 256 x 256");
    MRF_REQUIRE(prm->patch >= 1 && prm->patch <= 11 && prm->patch <= plan->nx,
                "mrf_recon_create: patch must be in [1, 11] and fit the image (got %d)", prm->patch);
    MRF_REQUIRE(prm->stride >= 1 && prm->stride <= prm->patch, "mrf_recon_create: stride must be in [1, patch]");
    MRF_REQUIRE(prm->knn >= 1 && prm->knn <= 32, "mrf_recon_create: knn must be in [1, 32]");
    MRF_REQUIRE(prm->beta > 0.f && prm->mu > 0.f, "mrf_recon_create: beta and mu must be > 0");
    MRF_REQUIRE(prm->match_precision == MRF_MATCH_FP32 || prm->match_precision == MRF_MATCH_BF16 ||
                    prm->match_precision == MRF_MATCH_BF16X3 || prm->match_precision == MRF_MATCH_FP8,
                "mrf_recon_create: unknown match precision %d", prm->match_precision);
    MRF_REQUIRE(!(prm->flags & MRF_RECON_LEARNED) ||
                    (prm->mlp && K == 10 && mrf::tc_form(prm->match_precision) != 0),
                "mrf_recon_create: the learned matcher needs params.mlp, K = 10 and a tensor-core precision "
                "for its fallback");
    const PatchGeom g = make_geom(plan->nx, prm->patch, prm->stride);
    MRF_REQUIRE(g.count() >= prm->knn + 1, "mrf_recon_create: need at least knn + 1 patches (%d)", g.count());
    auto* R = new mrf_recon_s();
    R->plan = plan;
    R->prm = *prm;
    for (cudaStream_t& t : R->side)
        if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess) t = nullptr;
    for (cudaEvent_t& e : R->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
    bool made = true;
    for (cudaStream_t t : R->side) made = made && t;
    for (cudaEvent_t e : R->ev) made = made && e;
    if (!made) {
        free_recon(R);
        set_error("mrf_recon_create: could not create the loop's streams and events");
        return MRF_ECUDA;
    }
    R->K = K;
    R->m = m;
    R->N = plan->nx * plan->ny;
    R->g = g;
    R->np = g.count();
    R->pp = prm->patch * prm->patch;
    R->mode = (prm->flags & MRF_RECON_GROUPED) ? 1 : 0;
    R->phi = reinterpret_cast<const float2*>(phi);
    R->dict_c = reinterpret_cast<const float2*>(dict_c);
    R->atom_norm2 = atom_norm2;
    R->lut = lut;
    const mrf_status st = create(R, reinterpret_cast<const float2*>(b), as_stream(stream));
    if (st != MRF_OK) {
        free_recon(R);
        return st;
    }
    *out = R;
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_iter(mrf_recon R, int n_iters, double* cost_out, mrf_stream stream) {
    MRF_REQUIRE(R != nullptr, "mrf_recon_iter: NULL recon");
    MRF_REQUIRE(n_iters >= 0 && n_iters <= R->cost_cap, "mrf_recon_iter: n_iters must be in [0, %d]", R->cost_cap);
    cudaStream_t s = as_stream(stream);
    const int first = R->iters_done;
    for (int i = 0; i < n_iters; ++i) {
        // the first iteration runs eagerly (tuners, lazily built operands, the
        // SVT's cold start); the next one is recorded and then replayed
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        MRF_CUDA(cudaStreamIsCapturing(s, &cap));
        const bool graph = !(R->prm.flags & (MRF_RECON_EAGER | MRF_RECON_SERIAL)) && first + i >= 1 &&
                           R->svt_warm && !profiling_enabled() && cap == cudaStreamCaptureStatusNone;
        if (!graph) {
            MRF_PROPAGATE(iteration(R, first + i, s));
            continue;
        }
        // recorded and replayed on an internal stream that follows the
        // caller's (which may be a default stream, which cannot be captured)
        cudaStream_t si = R->side[2];
        MRF_CUDA(cudaEventRecord(R->ev[5], s));
        MRF_CUDA(cudaStreamWaitEvent(si, R->ev[5], 0));
        if (!R->iter_exec) {
            const long long before = launches_so_far();
            const double svt_before = R->svt_patch_launches;
            MRF_CUDA(cudaStreamBeginCapture(si, cudaStreamCaptureModeRelaxed));
            const mrf_status st = iteration(R, first + i, si);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(si, &g);
            if (st != MRF_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                if (st != MRF_OK) return st;
                MRF_CUDA(e);
            }
            const cudaError_t ei = cudaGraphInstantiate(&R->iter_exec, g, 0);
            cudaGraphDestroy(g);
            MRF_CUDA(ei);
            R->iter_kernels = launches_so_far() - before;
            note_replayed_launches(-R->iter_kernels);            // counted again at each replay
            R->svt_patch_launches = svt_before;
        }
        MRF_CUDA(cudaGraphLaunch(R->iter_exec, si));
        MRF_CUDA(cudaEventRecord(R->ev[6], si));
        MRF_CUDA(cudaStreamWaitEvent(s, R->ev[6], 0));
        note_replayed_launches(R->iter_kernels);
        R->svt_patch_launches += R->np;
    }
    R->iters_done += n_iters;
    if (cost_out && n_iters > 0) {
        if (R->prm.flags & MRF_RECON_NO_COST) {
            for (int i = 0; i < n_iters; ++i) cost_out[i] = NAN;
        } else {
            std::vector<double> h(R->cost_cap);
            MRF_CUDA(cudaMemcpyAsync(h.data(), R->cost, sizeof(double) * R->cost_cap, cudaMemcpyDeviceToHost, s));
            MRF_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i < n_iters; ++i) cost_out[i] = h[(first + i) % R->cost_cap];
        }
    }
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_maps(mrf_recon R, float* t1, float* t2, float* pd, int* idx, mrf_stream stream) {
    MRF_REQUIRE(R != nullptr, "mrf_recon_maps: NULL recon");
    k_maps<<<(R->N + 255) / 256, 256, 0, as_stream(stream)>>>(R->t1t2, R->pd, R->idx, R->N, (float)(1.0 / R->gamma),
                                                               t1, t2, pd, idx);
    MRF_LAUNCHED_AS("k_maps", as_stream(stream));
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_alpha(mrf_recon R, mrf_c64* alpha, mrf_stream stream) {
    MRF_REQUIRE(R && alpha, "mrf_recon_alpha: NULL argument");
    MRF_CUDA(cudaMemcpyAsync(alpha, R->alpha, sizeof(float2) * (size_t)R->N * R->K, cudaMemcpyDeviceToDevice,
                             as_stream(stream)));
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_svt_stats(mrf_recon R, double* sweeps, double* rotations, double* patch_svts,
                                          mrf_stream stream) {
    MRF_REQUIRE(R && sweeps && rotations && patch_svts, "mrf_recon_svt_stats: NULL argument");
    cudaStream_t s = as_stream(stream);
    unsigned long long h[2] = {0, 0};
    MRF_CUDA(cudaMemcpyAsync(h, R->svt_stats, sizeof h, cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    *sweeps = (double)h[0];
    *rotations = (double)h[1];
    *patch_svts = R->svt_patch_launches;
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_info(mrf_recon R, double* a_norm, double* x_scale, double* lam1, double* sigma2,
                                     mrf_stream stream) {
    MRF_REQUIRE(R != nullptr, "mrf_recon_info: NULL recon");
    float h[3] = {0.f, 0.f, 0.f};
    cudaStream_t s = as_stream(stream);
    MRF_CUDA(cudaMemcpyAsync(h, R->scal, sizeof(h), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    if (a_norm) *a_norm = R->a;
    if (x_scale) *x_scale = R->gamma;
    if (lam1) *lam1 = h[2];
    if (sigma2) *sigma2 = h[0];
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_destroy(mrf_recon R) {
    free_recon(R);
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume of the loop state.  A checkpoint holds what the next
// iteration reads and the graph cannot be rebuilt without: the coefficient
// images, the residual, the SVT output P and its right singular vectors (warm
// start), the maps, the cost history, the iteration count and the scales a
// and gamma (a header checks that the restoring object has the same shape and
// scales).  The graph, sigma^2 and lambda1 are rebuilt from the restored maps.
// ---------------------------------------------------------------------------
namespace mrf {

struct CkptHeader {
    uint32_t magic, version;
    int32_t N, K, np, pp, kp, m, iters_done, svt_warm, cost_cap, pad;
    int64_t nr;
    double a, gamma;
};
constexpr uint32_t kCkptMagic = 0x4d524643u;   // "MRFC"

struct CkptPart {
    void* dev;
    size_t bytes;
};

static std::vector<CkptPart> ckpt_parts(mrf_recon_s* R) {
    const size_t NK = (size_t)R->N * R->K, nr = (size_t)R->plan->T * R->plan->ns;
    return {{R->alpha, sizeof(float2) * NK},
            {R->r, sizeof(float2) * nr},
            {R->P, sizeof(float2) * (size_t)R->np * R->pp * R->K},
            {R->svt_v, sizeof(float2) * (size_t)R->np * R->svt_kp * R->svt_kp},
            {R->t1t2, sizeof(float) * 2 * (size_t)R->N},
            {R->pd, sizeof(float) * (size_t)R->N},
            {R->idx, sizeof(int) * (size_t)R->N},
            {R->cost, sizeof(double) * (size_t)R->cost_cap}};
}

static size_t ckpt_bytes(mrf_recon_s* R) {
    size_t b = sizeof(CkptHeader);
    for (const CkptPart& p : ckpt_parts(R)) b += p.bytes;
    return b;
}

static CkptHeader ckpt_header(mrf_recon_s* R) {
    CkptHeader h{};
    h.magic = kCkptMagic;
    h.version = 1;
    h.N = R->N; h.K = R->K; h.np = R->np; h.pp = R->pp; h.kp = R->svt_kp; h.m = R->m;
    h.iters_done = R->iters_done; h.svt_warm = R->svt_warm; h.cost_cap = R->cost_cap;
    h.nr = (int64_t)R->plan->T * R->plan->ns;
    h.a = R->a;
    h.gamma = R->gamma;
    return h;
}

}  // namespace mrf

extern "C" mrf_status mrf_recon_checkpoint_size(mrf_recon R, size_t* bytes) {
    MRF_REQUIRE(R && bytes, "mrf_recon_checkpoint_size: NULL argument");
    *bytes = mrf::ckpt_bytes(R);
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_checkpoint(mrf_recon R, void* buf, size_t bytes, mrf_stream stream) {
    using namespace mrf;
    MRF_REQUIRE(R && buf, "mrf_recon_checkpoint: NULL argument");
    MRF_REQUIRE(bytes >= ckpt_bytes(R), "mrf_recon_checkpoint: buffer of %zu bytes, need %zu", bytes,
                ckpt_bytes(R));
    cudaStream_t s = as_stream(stream);
    const CkptHeader h = ckpt_header(R);
    char* out = static_cast<char*>(buf);
    std::memcpy(out, &h, sizeof(h));
    size_t at = sizeof(h);
    for (const CkptPart& p : ckpt_parts(R)) {
        MRF_CUDA(cudaMemcpyAsync(out + at, p.dev, p.bytes, cudaMemcpyDeviceToHost, s));
        at += p.bytes;
    }
    MRF_CUDA(cudaStreamSynchronize(s));
    return MRF_OK;
}

extern "C" mrf_status mrf_recon_restore(mrf_recon R, const void* buf, size_t bytes, mrf_stream stream) {
    using namespace mrf;
    MRF_REQUIRE(R && buf, "mrf_recon_restore: NULL argument");
    MRF_REQUIRE(bytes >= sizeof(CkptHeader), "mrf_recon_restore: buffer too small");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const CkptHeader mine = ckpt_header(R);
    MRF_REQUIRE(h.magic == kCkptMagic && h.version == 1, "mrf_recon_restore: not a checkpoint of this library");
    MRF_REQUIRE(h.N == mine.N && h.K == mine.K && h.np == mine.np && h.pp == mine.pp && h.kp == mine.kp &&
                    h.m == mine.m && h.nr == mine.nr && h.cost_cap == mine.cost_cap,
                "mrf_recon_restore: the checkpoint's shape (N %d, K %d, patches %d, atoms %d) differs from this "
                "object's (N %d, K %d, patches %d, atoms %d)", h.N, h.K, h.np, h.m, mine.N, mine.K, mine.np, mine.m);
    MRF_REQUIRE(std::fabs(h.a - mine.a) <= 1e-6 * std::fabs(h.a) &&
                    std::fabs(h.gamma - mine.gamma) <= 1e-6 * std::fabs(h.gamma),
                "mrf_recon_restore: scales differ (a %g vs %g, gamma %g vs %g); create the object with "
                "params.a_norm and params.x_scale set to the saved a and gamma", h.a, mine.a, h.gamma, mine.gamma);
    MRF_REQUIRE(bytes >= ckpt_bytes(R), "mrf_recon_restore: truncated checkpoint");
    cudaStream_t s = as_stream(stream);
    const char* in = static_cast<const char*>(buf);
    size_t at = sizeof(h);
    for (const CkptPart& p : ckpt_parts(R)) {
        MRF_CUDA(cudaMemcpyAsync(p.dev, in + at, p.bytes, cudaMemcpyHostToDevice, s));
        at += p.bytes;
    }
    R->iters_done = h.iters_done;
    R->svt_warm = h.svt_warm;
    // the next pass's A*(r), from the restored residual
    MRF_PROPAGATE(subspace_adjoint(R->plan, R->r, R->phi, R->K, (float)(1.0 / R->a), R->grad, R->mode, s));
    if (R->iter_exec) {                         // recorded before the restore: record again
        cudaGraphExecDestroy(R->iter_exec);
        R->iter_exec = nullptr;
    }
    {
        const int slot = R->iters_done % R->cost_cap;
        MRF_CUDA(cudaMemcpyAsync(R->cost_slot, &slot, sizeof(int), cudaMemcpyHostToDevice, s));
        MRF_CUDA(cudaStreamSynchronize(s));
    }
    MRF_PROPAGATE(build_graph(R, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    return MRF_OK;
}

// ---------------------------------------------------------------------------
// Batched serving: S independent slices (their own plans and sizes, one
// shared dictionary) advanced together.  One batched iteration forks each
// slice's graph term and X update onto a stream of its own; from the new
// iterate on, the slice's SVT and its forward operator + next gradient run on
// two more streams, while one tensor-core launch matches every slice's
// fingerprints (a slice table maps the launch's blocks to slices) as soon as
// all iterates are new; each slice's matching epilogue and graph rebuild
// follow it, and everything joins at the end.  The first mrf_batch_iter runs one iteration
// eagerly (lazy tables, the spread autotuner, the warm SVT state) and then
// captures the fork/join sequence into a CUDA graph that every later
// iteration replays with one launch.
// ---------------------------------------------------------------------------
struct mrf_batch_s {
    std::vector<mrf_recon_s*> R;
    // per slice: graph term, X update, forward, next gradient (st); SVT (sv);
    // matching epilogue and graph rebuild (sg); the new iterate (ev), and the
    // ends of the three streams (eva, evv, evg)
    std::vector<cudaStream_t> st, sv, sg;
    std::vector<cudaEvent_t> ev, eva, evv, evg;
    cudaEvent_t fork = nullptr, fork2 = nullptr;
    cudaStream_t cs = nullptr;      // the batch's own stream (the one captured; joined to the caller's)
    cudaEvent_t entry = nullptr, exit = nullptr;
    mrf::TcSlice* d_slices = nullptr;
    int total_blocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* d_err = nullptr;           // gathered error words (filled by batch_check)
};

namespace mrf {

static void free_batch(mrf_batch_s* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto* v : {&B->st, &B->sv, &B->sg})
        for (cudaStream_t t : *v) cudaStreamDestroy(t);
    for (auto* v : {&B->ev, &B->eva, &B->evv, &B->evg})
        for (cudaEvent_t e : *v) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->fork2) cudaEventDestroy(B->fork2);
    if (B->entry) cudaEventDestroy(B->entry);
    if (B->exit) cudaEventDestroy(B->exit);
    if (B->cs) cudaStreamDestroy(B->cs);
    cudaFree(B->d_slices);
    delete B;
}

static mrf_status batch_iteration(mrf_batch_s* B, cudaStream_t s) {
    const int S = (int)B->R.size();
    mrf_recon_s* R0 = B->R[0];
    const int form = tc_form(R0->prm.match_precision);
    MRF_CUDA(cudaEventRecord(B->fork, s));
    for (int i = 0; i < S; ++i) {
        mrf_recon_s* R = B->R[i];
        cudaStream_t t = B->st[i], tv = B->sv[i], tg = B->sg[i];
        const size_t NK = (size_t)R->N * R->K;
        const float inv_a = (float)(1.0 / R->a);
        MRF_CUDA(cudaStreamWaitEvent(t, B->fork, 0));
        MRF_PROPAGATE(graph_pass(R, R->QL, nullptr, t));
        const float c = R->prm.mu * R->prm.lam2 * R->prm.beta;
        k_xupdate<<<(unsigned)((NK + 255) / 256), 256, 0, t>>>(
            R->alpha, R->grad, R->QL, R->P, R->g, R->K, R->prm.mu, c, R->scal + 2,
            (R->prm.flags & MRF_RECON_LITERAL_XUPDATE) ? 1 : 0, nullptr);
        MRF_LAUNCHED_AS("k_xupdate", t);
        MRF_CUDA(cudaEventRecord(B->ev[i], t));             // the new iterate
        MRF_CUDA(cudaStreamWaitEvent(tv, B->ev[i], 0));
        MRF_PROPAGATE(svt(R, R->alpha, R->P, nullptr, tv));
        MRF_CUDA(cudaEventRecord(B->evv[i], tv));
        if (!form) {
            // FP32: one exhaustive launch per slice
            MRF_CUDA(cudaStreamWaitEvent(tg, B->ev[i], 0));
            MRF_PROPAGATE(match_maps(R, tg));
            MRF_PROPAGATE(build_graph(R, tg));
            MRF_CUDA(cudaEventRecord(B->evg[i], tg));
        }
        MRF_PROPAGATE(subspace_forward(R->plan, R->alpha, R->phi, R->K, inv_a, R->bs, R->r, R->mode, t));
        MRF_PROPAGATE(subspace_adjoint(R->plan, R->r, R->phi, R->K, inv_a, R->grad, R->mode, t));
        MRF_CUDA(cudaEventRecord(B->eva[i], t));
    }
    if (form) {
        for (int i = 0; i < S; ++i) MRF_CUDA(cudaStreamWaitEvent(s, B->ev[i], 0));
        MRF_PROPAGATE(match_tc_batch(R0->mws, B->d_slices, S, B->total_blocks, R0->K, R0->m, form, s));
        MRF_CUDA(cudaEventRecord(B->fork2, s));
        for (int i = 0; i < S; ++i) {
            mrf_recon_s* R = B->R[i];
            cudaStream_t tg = B->sg[i];
            MRF_CUDA(cudaStreamWaitEvent(tg, B->fork2, 0));
            MRF_PROPAGATE(match_finish(R->mws, R->N, R->lut, R->idx, R->pd, R->t1t2, 1.0f, tg));
            MRF_PROPAGATE(build_graph(R, tg));
            MRF_CUDA(cudaEventRecord(B->evg[i], tg));
        }
    }
    for (int i = 0; i < S; ++i) {
        MRF_CUDA(cudaStreamWaitEvent(s, B->eva[i], 0));
        MRF_CUDA(cudaStreamWaitEvent(s, B->evv[i], 0));
        MRF_CUDA(cudaStreamWaitEvent(s, B->evg[i], 0));
    }
    return MRF_OK;
}

// error words of the batch's bounded device waits and range checks
static mrf_status batch_check(mrf_batch_s* B, cudaStream_t s) {
    std::vector<const int*> src;
    for (mrf_recon_s* R : B->R) {
        if (R->mws.tc_err) src.push_back(R->mws.tc_err);
        if (R->knn.err) src.push_back(R->knn.err);
    }
    std::vector<int> h(src.size(), 0);
    for (size_t i = 0; i < src.size(); ++i)
        MRF_CUDA(cudaMemcpyAsync(&h[i], src[i], sizeof(int), cudaMemcpyDeviceToHost, s));
    MRF_CUDA(cudaStreamSynchronize(s));
    for (int v : h) {
        if (v == 2) {
            set_error("mrf_batch_iter: a bounded device wait gave up");
            return MRF_ETIMEOUT;
        }
        if (v == 1) {
            set_error("mrf_batch_iter: a patch feature left [0, 4096]");
            return MRF_EINVAL;
        }
    }
    return MRF_OK;
}

}  // namespace mrf

extern "C" mrf_status mrf_batch_create(mrf_batch* out, const mrf_recon* recons, int count, mrf_stream stream) {
    MRF_REQUIRE(out && recons, "mrf_batch_create: NULL argument");
    MRF_REQUIRE(count >= 1 && count <= 64, "mrf_batch_create: count must be in [1, 64] (got %d)", count);
    *out = nullptr;
    mrf_recon_s* R0 = recons[0];
    MRF_REQUIRE(R0 != nullptr, "mrf_batch_create: NULL recon 0");
    for (int i = 0; i < count; ++i) {
        mrf_recon_s* R = recons[i];
        MRF_REQUIRE(R != nullptr, "mrf_batch_create: NULL recon %d", i);
        MRF_REQUIRE(R->m == R0->m && R->K == R0->K && R->prm.match_precision == R0->prm.match_precision,
                    "mrf_batch_create: slice %d differs from slice 0 in atoms, K or match precision", i);
        MRF_REQUIRE(!(R->prm.flags & MRF_RECON_LEARNED),
                    "mrf_batch_create: slice %d uses the learned matcher (not batched)", i);
        for (int j = 0; j < i; ++j)
            MRF_REQUIRE(R != recons[j] && R->plan != recons[j]->plan,
                        "mrf_batch_create: slices %d and %d share a recon or a NUFFT plan", j, i);
    }
    cudaStream_t s = as_stream(stream);
    const int form = mrf::tc_form(R0->prm.match_precision);
    for (int i = 0; form && i < count; ++i)
        MRF_PROPAGATE(mrf::tc_prepare_operand(recons[i]->mws, recons[i]->dict_c, R0->m, R0->K, form, s));
    auto* B = new mrf_batch_s();
    std::vector<mrf::TcSlice> table;
    for (int i = 0; i < count; ++i) {
        mrf_recon_s* R = recons[i];
        B->R.push_back(R);
        // each slice's matching is seeded from its previous call's candidates,
        // as in the loop of a single slice
        table.push_back({R->alpha, R->N, B->total_blocks, R->mws.best_idx, R->mws.best_ip,
                         static_cast<const unsigned char*>(R->mws.tc_b), R->mws.wscore, R->dict_c,
                         form == 8 ? nullptr : R->mws.cand});
        B->total_blocks += (R->N + 127) / 128;
    }
    mrf_status st = MRF_OK;
    auto fail = [&](const char* what, cudaError_t e) {
        set_error("mrf_batch_create: %s failed: %s", what, cudaGetErrorString(e));
        st = MRF_ECUDA;
    };
    cudaError_t e = cudaMalloc(&B->d_slices, sizeof(mrf::TcSlice) * table.size());
    if (e != cudaSuccess) fail("cudaMalloc", e);
    if (st == MRF_OK) {
        e = cudaMemcpyAsync(B->d_slices, table.data(), sizeof(mrf::TcSlice) * table.size(), cudaMemcpyHostToDevice,
                            s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) fail("slice table upload", e);
    }
    for (int i = 0; st == MRF_OK && i < count; ++i) {
        for (auto* v : {&B->st, &B->sv, &B->sg}) {
            cudaStream_t t;
            e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
            if (e != cudaSuccess) { fail("cudaStreamCreateWithFlags", e); break; }
            v->push_back(t);
        }
        for (auto* v : {&B->ev, &B->eva, &B->evv, &B->evg}) {
            if (st != MRF_OK) break;
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) { fail("cudaEventCreateWithFlags", e); break; }
            v->push_back(ev);
        }
    }
    if (st == MRF_OK && ((e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming)) != cudaSuccess ||
                         (e = cudaEventCreateWithFlags(&B->fork2, cudaEventDisableTiming)) != cudaSuccess ||
                         (e = cudaEventCreateWithFlags(&B->entry, cudaEventDisableTiming)) != cudaSuccess ||
                         (e = cudaEventCreateWithFlags(&B->exit, cudaEventDisableTiming)) != cudaSuccess))
        fail("cudaEventCreateWithFlags", e);
    if (st == MRF_OK && (e = cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking)) != cudaSuccess)
        fail("cudaStreamCreateWithFlags", e);
    if (st != MRF_OK) {
        free_batch(B);
        return st;
    }
    *out = B;
    return MRF_OK;
}

extern "C" mrf_status mrf_batch_iter(mrf_batch B, int n_iters, mrf_stream stream) {
    MRF_REQUIRE(B != nullptr, "mrf_batch_iter: NULL batch");
    MRF_REQUIRE(n_iters >= 0, "mrf_batch_iter: n_iters must be >= 0");
    if (n_iters == 0) return MRF_OK;
    // the work runs on the batch's own stream (the legacy default stream
    // cannot be captured), ordered after and before the caller's stream
    const cudaStream_t caller = as_stream(stream);
    const cudaStream_t s = B->cs;
    MRF_CUDA(cudaEventRecord(B->entry, caller));
    MRF_CUDA(cudaStreamWaitEvent(s, B->entry, 0));
    const int total = n_iters;
    if (!B->exec) {
        MRF_PROPAGATE(batch_iteration(B, s));           // eager: lazy tables, autotuning, warm SVT state
        --n_iters;
        MRF_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        const mrf_status st = batch_iteration(B, s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != MRF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (st != MRF_OK) return st;
            set_error("mrf_batch_iter: stream capture failed: %s", cudaGetErrorString(e));
            return MRF_ECUDA;
        }
        B->graph = g;
        MRF_CUDA(cudaGraphInstantiate(&B->exec, g, 0));
    }
    for (int i = 0; i < n_iters; ++i) MRF_CUDA(cudaGraphLaunch(B->exec, s));
    for (mrf_recon_s* R : B->R) R->iters_done += total;
    MRF_CUDA(cudaEventRecord(B->exit, s));
    MRF_CUDA(cudaStreamWaitEvent(caller, B->exit, 0));
    return batch_check(B, s);
}

extern "C" mrf_status mrf_batch_destroy(mrf_batch B) {
    mrf::free_batch(B);
    return MRF_OK;
}

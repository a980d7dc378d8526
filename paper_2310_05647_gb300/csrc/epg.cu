// FISP dictionary atoms B(eta; theta) with PD = 1 (Eq. 2-3) by extended phase
// graphs.  One block per atom; the state vector (F+_k, F-_k, Z_k) lives in
// shared memory.  Per repetition t:
//   RF rotation of flip a about x:  F+' = c^2 F+ + s^2 F- - i sin(a) Z
//                                   F-' = s^2 F+ + c^2 F- + i sin(a) Z
//                                   Z'  = -i/2 sin(a) F+ + i/2 sin(a) F- + cos(a) Z
//   relaxation over TE (F *= E2, Z_k *= E1, Z_0 += 1 - E1), signal F+_0,
//   relaxation over TR_t - TE, one dephasing: F+_k <- F+_{k-1},
//   F-_k <- F-_{k+1}, F+_0 <- conj(F-_0).
// States that can no longer reach k = 0 before the train ends (k larger than
// the repetitions left) and states not yet populated (k > t + 1) are skipped:
// they never influence a recorded signal, so the result equals the full
// recursion.
#include "common.h"

namespace mrf {

constexpr int kEpgThreads = 128;
constexpr int kEpgMaxT = 4094;   // T + 2 states fit the shared-memory budget

__global__ void __launch_bounds__(kEpgThreads) k_epg_fisp(const float* __restrict__ t1t2, int m,
                                                          const float* __restrict__ fa_deg,
                                                          const float* __restrict__ tr_ms, int T, float te,
                                                          float ti, int inversion, float2* __restrict__ out) {
    extern __shared__ float2 st[];
    const int S = T + 2;
    float2* Fp = st;
    float2* Fm = st + S;
    float2* Z = st + 2 * S;
    float2* Fp2 = st + 3 * S;        // dephasing writes the shifted states here
    float2* Fm2 = st + 4 * S;
    const int atom = blockIdx.x;
    if (atom >= m) return;
    const float t1 = t1t2[2 * atom], t2 = t1t2[2 * atom + 1];
    const float r1 = t1 > 0.f ? 1.0f / t1 : 0.f, r2 = t2 > 0.f ? 1.0f / t2 : 0.f;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        Fp[k] = Fm[k] = Z[k] = Fp2[k] = Fm2[k] = make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) {
        float z0 = 1.0f;
        if (inversion) {
            const float e1 = expf(-ti * r1);
            z0 = -e1 + (1.0f - e1);
        }
        Z[0] = make_float2(z0, 0.f);
    }
    __syncthreads();
    const float e2te = expf(-te * r2), e1te = expf(-te * r1);
    for (int t = 0; t < T; ++t) {
        const int kmax = min(t + 1, T - t);       // states that matter at this repetition
        float sa, ca, sh, ch;
        sincosf(fa_deg[t] * (3.14159265358979f / 180.0f), &sa, &ca);
        sincosf(fa_deg[t] * (3.14159265358979f / 360.0f), &sh, &ch);
        const float c2 = ch * ch, s2 = sh * sh;
        const float rest = tr_ms[t] - te;
        const float e2r = expf(-rest * r2), e1r = expf(-rest * r1);
        const float e2 = e2te * e2r, e1 = e1te * e1r;
        for (int k = threadIdx.x; k <= kmax; k += blockDim.x) {
            const float2 fp = Fp[k], fm = Fm[k], z = Z[k];
            // RF: -i sa z = (sa z.y, -sa z.x)
            float2 nfp = make_float2(c2 * fp.x + s2 * fm.x + sa * z.y, c2 * fp.y + s2 * fm.y - sa * z.x);
            float2 nfm = make_float2(s2 * fp.x + c2 * fm.x - sa * z.y, s2 * fp.y + c2 * fm.y + sa * z.x);
            // -i/2 sa fp + i/2 sa fm = i/2 sa (fm - fp)
            const float2 d = make_float2(fm.x - fp.x, fm.y - fp.y);
            float2 nz = make_float2(ca * z.x - 0.5f * sa * d.y, ca * z.y + 0.5f * sa * d.x);
            if (k == 0) {
                // relaxation over TE, record, relaxation over the rest
                const float2 sig = make_float2(nfp.x * e2te, nfp.y * e2te);
                out[(size_t)atom * T + t] = sig;
                nfp = cscale(nfp, e2);
                nfm = cscale(nfm, e2);
                nz = make_float2((nz.x * e1te + (1.f - e1te)) * e1r + (1.f - e1r), nz.y * e1);
            } else {
                nfp = cscale(nfp, e2);
                nfm = cscale(nfm, e2);
                nz = cscale(nz, e1);
            }
            Fp[k] = nfp;
            Fm[k] = nfm;
            Z[k] = nz;
        }
        __syncthreads();
        // dephasing by one state: F+_k <- F+_{k-1}, F-_k <- F-_{k+1}, F+_0 <- conj(F-_0)
        const int lim = min(kmax + 1, S - 2);
        for (int k = threadIdx.x; k <= lim; k += blockDim.x) {
            const float2 fm = Fm[k + 1];
            Fm2[k] = fm;
            Fp2[k] = k == 0 ? make_float2(fm.x, -fm.y) : Fp[k - 1];
        }
        __syncthreads();
        float2* tp = Fp; Fp = Fp2; Fp2 = tp;
        float2* tm = Fm; Fm = Fm2; Fm2 = tm;
    }
}

}  // namespace mrf

using namespace mrf;

extern "C" mrf_status mrf_epg_fisp(const float* t1t2, int m, const float* fa_deg, const float* tr_ms, int T,
                                   float te_ms, float ti_ms, int inversion, mrf_c64* out, mrf_stream stream) {
    MRF_REQUIRE(t1t2 && fa_deg && tr_ms && out, "mrf_epg_fisp: NULL argument");
    MRF_REQUIRE(m >= 0 && T >= 1 && T <= kEpgMaxT, "mrf_epg_fisp: bad m or T (%d, %d)", m, T);
    if (m == 0) return MRF_OK;
    const size_t smem = sizeof(float2) * 5 * (size_t)(T + 2);
    MRF_CUDA(cudaFuncSetAttribute(k_epg_fisp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_epg_fisp<<<m, kEpgThreads, smem, as_stream(stream)>>>(t1t2, m, fa_deg, tr_ms, T, te_ms, ti_ms, inversion,
                                                            reinterpret_cast<float2*>(out));
    MRF_LAUNCHED_AS("k_epg_fisp", as_stream(stream));
    return MRF_OK;
}

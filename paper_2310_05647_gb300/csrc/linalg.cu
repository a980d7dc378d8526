// Temporal subspace of a dictionary: the orthonormal basis d of the
// fingerprint-manifold projection P_S(X) = X d^dagger d (Eq. 14), taken as the
// top-K right singular vectors of D (m x T).
//
// Randomised block subspace iteration (Yang et al., cited in Sec. I) on
// D^H D without forming it: every product D V and D^H W runs on the GPU with
// FP64 accumulation (the 10th singular value of an MRF dictionary is ~1e-3 of
// the first, so the squared spectrum must not be rounded in FP32); the
// T x (K + 8) block is orthonormalised (modified Gram-Schmidt, FP64) and the
// Rayleigh-Ritz problem (D V)^H (D V) is solved by cyclic complex Jacobi
// (FP64) in host code of this library.  Each column of Phi is given a fixed phase
// (its largest-magnitude entry real and positive).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "common.h"

namespace mrf {

using cd = std::complex<double>;

// W[m][j] = sum_t D[m][t] V[t][j]  (FP32 inputs, FP64 accumulation; one warp
// per atom, lane j < P)
__global__ void k_dv(const float2* __restrict__ D, int m, int T, const double2* __restrict__ V, int P,
                     double2* __restrict__ W) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int j = threadIdx.x & 31;
    if (row >= m || j >= P) return;
    const float2* d = D + (size_t)row * T;
    double re = 0.0, im = 0.0;
    for (int t = 0; t < T; ++t) {
        const float2 a = d[t];
        const double2 v = V[(size_t)t * P + j];
        re += (double)a.x * v.x - (double)a.y * v.y;
        im += (double)a.x * v.y + (double)a.y * v.x;
    }
    W[(size_t)row * P + j] = make_double2(re, im);
}

// Y[t][j] = sum_m conj(D[m][t]) W[m][j]  (one warp per frame, lane j < P)
__global__ void k_dhw(const float2* __restrict__ D, int m, int T, const double2* __restrict__ W, int P,
                      double2* __restrict__ Y) {
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int j = threadIdx.x & 31;
    if (t >= T || j >= P) return;
    double re = 0.0, im = 0.0;
    for (int r = 0; r < m; ++r) {
        const float2 a = D[(size_t)r * T + t];
        const double2 w = W[(size_t)r * P + j];
        re += (double)a.x * w.x + (double)a.y * w.y;
        im += (double)a.x * w.y - (double)a.y * w.x;
    }
    Y[(size_t)t * P + j] = make_double2(re, im);
}

// compressed[m][k] = sum_t D[m][t] Phi[t][k];  norm2[m] = sum_t |D[m][t]|^2
__global__ void k_compress(const float2* __restrict__ D, int m, int T, const float2* __restrict__ phi, int K,
                           float2* __restrict__ comp, float* __restrict__ norm2) {
    const int a = blockIdx.x;
    if (a >= m) return;
    const float2* d = D + (size_t)a * T;
    for (int k = threadIdx.y; k <= K; k += blockDim.y) {
        double re = 0.0, im = 0.0;
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            if (k < K) {
                const float2 p = cmul(d[t], phi[(size_t)t * K + k]);
                re += p.x;
                im += p.y;
            } else {
                re += (double)cabs2(d[t]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (threadIdx.x == 0) {
            if (k < K) {
                if (comp) comp[(size_t)a * K + k] = make_float2((float)re, (float)im);
            } else if (norm2) {
                norm2[a] = (float)re;
            }
        }
    }
}

static uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// modified Gram-Schmidt on the columns of V [T][P] (FP64)
static void orthonormalise(std::vector<cd>& V, int T, int P) {
    for (int j = 0; j < P; ++j) {
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < j; ++i) {
                cd d = 0.0;
                for (int t = 0; t < T; ++t) d += std::conj(V[(size_t)t * P + i]) * V[(size_t)t * P + j];
                for (int t = 0; t < T; ++t) V[(size_t)t * P + j] -= d * V[(size_t)t * P + i];
            }
        double nn = 0.0;
        for (int t = 0; t < T; ++t) nn += std::norm(V[(size_t)t * P + j]);
        nn = std::sqrt(nn);
        for (int t = 0; t < T; ++t) V[(size_t)t * P + j] = nn > 0 ? V[(size_t)t * P + j] / nn : 0.0;
    }
}

// cyclic Jacobi for a Hermitian P x P matrix H (row-major); eigenvalues in w,
// eigenvectors in the columns of U
static void hermitian_jacobi(std::vector<cd> H, int P, std::vector<double>& w, std::vector<cd>& U) {
    U.assign((size_t)P * P, 0.0);
    for (int i = 0; i < P; ++i) U[(size_t)i * P + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < P; ++i)
            for (int j = 0; j < P; ++j) {
                const double v = std::norm(H[(size_t)i * P + j]);
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < P - 1; ++p)
            for (int q = p + 1; q < P; ++q) {
                const cd h = H[(size_t)p * P + q];
                const double ha = std::abs(h);
                if (ha < 1e-300) continue;
                const double a = H[(size_t)p * P + p].real(), b = H[(size_t)q * P + q].real();
                const cd e = std::conj(h) / ha;                  // exp(-i phi)
                const double tau = (b - a) / (2.0 * ha);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                // U2 = [[c, s], [-s e, c e]] acting on (p, q)
                const cd upp = c, upq = s, uqp = -s * e, uqq = c * e;
                for (int i = 0; i < P; ++i) {                    // H <- H U2
                    const cd hp = H[(size_t)i * P + p], hq = H[(size_t)i * P + q];
                    H[(size_t)i * P + p] = hp * upp + hq * uqp;
                    H[(size_t)i * P + q] = hp * upq + hq * uqq;
                }
                for (int j = 0; j < P; ++j) {                    // H <- U2^H H
                    const cd hp = H[(size_t)p * P + j], hq = H[(size_t)q * P + j];
                    H[(size_t)p * P + j] = std::conj(upp) * hp + std::conj(uqp) * hq;
                    H[(size_t)q * P + j] = std::conj(upq) * hp + std::conj(uqq) * hq;
                }
                for (int i = 0; i < P; ++i) {                    // U <- U U2
                    const cd vp = U[(size_t)i * P + p], vq = U[(size_t)i * P + q];
                    U[(size_t)i * P + p] = vp * upp + vq * uqp;
                    U[(size_t)i * P + q] = vp * upq + vq * uqq;
                }
            }
    }
    w.resize(P);
    for (int i = 0; i < P; ++i) w[i] = H[(size_t)i * P + i].real();
}

}  // namespace mrf

using namespace mrf;

extern "C" mrf_status mrf_dict_subspace(const mrf_c64* dict, int m, int T, int K, mrf_c64* phi_out,
                                        mrf_c64* compressed, float* norm2, mrf_stream stream) {
    MRF_REQUIRE(dict && phi_out, "mrf_dict_subspace: NULL dict or phi");
    MRF_REQUIRE(K >= 1 && K <= 16, "mrf_dict_subspace: K must be in [1, 16] (got %d)", K);
    MRF_REQUIRE(T >= K + 8 && T <= 4096, "mrf_dict_subspace: need K + 8 <= T <= 4096 (T = %d)", T);
    MRF_REQUIRE(m >= K, "mrf_dict_subspace: need m >= K");
    cudaStream_t s = as_stream(stream);
    const float2* D = reinterpret_cast<const float2*>(dict);
    const int P = K + 8, iters = 10;
    double2 *V = nullptr, *W = nullptr, *Y = nullptr;
    float2* phi = reinterpret_cast<float2*>(phi_out);
    mrf_status st = MRF_OK;
    std::vector<cd> Vh((size_t)T * P), Yh((size_t)T * P), Wh((size_t)m * P);
    auto fail = [&](const char* what) {
        set_error("mrf_dict_subspace: %s: %s", what, cudaGetErrorString(cudaGetLastError()));
        st = MRF_ECUDA;
    };
    const int wpb = 4;   // warps per block
    auto dv = [&]() {    // W = D V (device)
        if (cudaMemcpyAsync(V, Vh.data(), sizeof(cd) * Vh.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return false;
        k_dv<<<(m + wpb - 1) / wpb, 32 * wpb, 0, s>>>(D, m, T, V, P, W);
        return cudaGetLastError() == cudaSuccess;
    };
    auto dhdv = [&]() {  // Yh = D^H D Vh
        if (!dv()) return false;
        k_dhw<<<(T + wpb - 1) / wpb, 32 * wpb, 0, s>>>(D, m, T, W, P, Y);
        if (cudaGetLastError() != cudaSuccess) return false;
        if (cudaMemcpyAsync(Yh.data(), Y, sizeof(cd) * Yh.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return false;
        return cudaStreamSynchronize(s) == cudaSuccess;
    };
    if (cudaMalloc(&V, sizeof(double2) * (size_t)T * P) != cudaSuccess ||
        cudaMalloc(&W, sizeof(double2) * (size_t)m * P) != cudaSuccess ||
        cudaMalloc(&Y, sizeof(double2) * (size_t)T * P) != cudaSuccess) {
        fail("allocation");
    }
    if (st == MRF_OK) {
        uint64_t seed = 0x5eed0f5ab5ba5eull;
        for (auto& v : Vh) {
            const double u1 = ((splitmix(seed) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            const double u2 = ((splitmix(seed) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            v = cd(u1 - 0.5, u2 - 0.5);
        }
        orthonormalise(Vh, T, P);
        for (int it = 0; it < iters && st == MRF_OK; ++it) {
            if (!dhdv()) { fail("subspace iteration"); break; }
            Vh = Yh;
            orthonormalise(Vh, T, P);
        }
    }
    // Rayleigh-Ritz on W = D V: H = W^H W
    if (st == MRF_OK) {
        if (!dv() || cudaMemcpyAsync(Wh.data(), W, sizeof(cd) * Wh.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            fail("Rayleigh-Ritz product");
    }
    if (st == MRF_OK) {
        std::vector<cd> H((size_t)P * P);
        for (int i = 0; i < P; ++i)
            for (int j = 0; j < P; ++j) {
                cd acc = 0.0;
                for (int r = 0; r < m; ++r) acc += std::conj(Wh[(size_t)r * P + i]) * Wh[(size_t)r * P + j];
                H[(size_t)i * P + j] = acc;
            }
        for (int i = 0; i < P; ++i)                        // exact Hermitian symmetry
            for (int j = i + 1; j < P; ++j) {
                const cd a = 0.5 * (H[(size_t)i * P + j] + std::conj(H[(size_t)j * P + i]));
                H[(size_t)i * P + j] = a;
                H[(size_t)j * P + i] = std::conj(a);
            }
        std::vector<double> w;
        std::vector<cd> U;
        hermitian_jacobi(H, P, w, U);
        std::vector<int> order(P);
        for (int i = 0; i < P; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
        std::vector<cd> Ph((size_t)T * K);
        for (int k = 0; k < K; ++k) {
            const int c = order[k];
            int arg = 0;
            double best = -1.0;
            for (int t = 0; t < T; ++t) {
                cd v = 0.0;
                for (int i = 0; i < P; ++i) v += Vh[(size_t)t * P + i] * U[(size_t)i * P + c];
                Ph[(size_t)t * K + k] = v;
                if (std::abs(v) > best) { best = std::abs(v); arg = t; }
            }
            const cd ph = std::abs(Ph[(size_t)arg * K + k]) > 0 ? std::conj(Ph[(size_t)arg * K + k]) /
                                                                      std::abs(Ph[(size_t)arg * K + k])
                                                                : cd(1.0);
            for (int t = 0; t < T; ++t) Ph[(size_t)t * K + k] *= ph;
        }
        std::vector<float2> pf((size_t)T * K);
        for (size_t i = 0; i < pf.size(); ++i) pf[i] = make_float2((float)Ph[i].real(), (float)Ph[i].imag());
        if (cudaMemcpyAsync(phi, pf.data(), sizeof(float2) * pf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            fail("upload");
        if (st == MRF_OK && (compressed || norm2)) {
            k_compress<<<m, dim3(32, 8), 0, s>>>(D, m, T, phi, K, reinterpret_cast<float2*>(compressed), norm2);
            if (cudaGetLastError() != cudaSuccess) fail("compress");
        }
        if (st == MRF_OK && cudaStreamSynchronize(s) != cudaSuccess) fail("sync");
    }
    cudaFree(V);
    cudaFree(W);
    cudaFree(Y);
    return st;
}

// Whole-path entry points built from the library's other calls:
//
// * mrf_gridding_match: the plain reconstruction X = A^H b (Eq. 1's adjoint,
//   frame by frame) followed by dictionary matching of every voxel's full
//   T-frame fingerprint (Eq. 5).  The adjoint writes frames [T][ny][nx]; a
//   tiled transpose turns them into fingerprint rows [ny nx][T] for the
//   matcher.
// * mrf_recon_run_host: one reconstruction from host k-space to host maps
//   (Algorithm 1: initialisation and n iterations), with the host <-> device
//   copies inside the call.

#include <vector>

#include "common.h"
#include "nufft_plan.h"

namespace mrf {

constexpr int kTr = 32;   // transpose tile edge

// out[c][r] = in[r][c] for an R x Cn complex matrix, through a shared tile so
// that both the loads and the stores are coalesced
__global__ void k_transpose_c64(const float2* __restrict__ in, int R, int Cn, float2* __restrict__ out) {
    __shared__ float2 tile[kTr][kTr + 1];
    const int c0 = blockIdx.x * kTr, r0 = blockIdx.y * kTr;
    const int tx = threadIdx.x, ty = threadIdx.y;       // 32 x 8 threads
    for (int j = ty; j < kTr; j += 8) {
        const int r = r0 + j, c = c0 + tx;
        if (r < R && c < Cn) tile[j][tx] = in[(size_t)r * Cn + c];
    }
    __syncthreads();
    for (int j = ty; j < kTr; j += 8) {
        const int c = c0 + j, r = r0 + tx;
        if (r < R && c < Cn) out[(size_t)c * R + r] = tile[tx][j];
    }
}

}  // namespace mrf

using namespace mrf;

extern "C" mrf_status mrf_gridding_match(mrf_plan p, const mrf_c64* y, const mrf_c64* dict, const float* atom_norm2,
                                         const float* lut, int m, int precision, int* idx, float* pd, float* t1t2,
                                         mrf_c64* x_rows, mrf_stream stream) {
    MRF_REQUIRE(p && y && dict && lut, "mrf_gridding_match: NULL plan, y, dict or lut");
    MRF_REQUIRE(m >= 1, "mrf_gridding_match: m must be >= 1");
    MRF_REQUIRE(p->T <= 2048, "mrf_gridding_match: at most 2048 frames (got %d)", p->T);
    cudaStream_t s = as_stream(stream);
    const int N = p->nx * p->ny, T = p->T;
    const size_t bytes = sizeof(float2) * (size_t)N * T;
    // stream-ordered scratch: the frames, and the rows when the caller keeps none
    float2* frames = nullptr;
    float2* rows = reinterpret_cast<float2*>(x_rows);
    MRF_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&frames), bytes, s));
    float2* own_rows = nullptr;
    mrf_status st = MRF_OK;
    if (!rows) {
        const cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&own_rows), bytes, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(frames, s);
            set_error("mrf_gridding_match: scratch allocation failed: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? MRF_ENOMEM : MRF_ECUDA;
        }
        rows = own_rows;
    }
    st = mrf_nufft_adjoint(p, y, reinterpret_cast<mrf_c64*>(frames), stream);
    if (st == MRF_OK) {
        const dim3 grid((unsigned)((N + kTr - 1) / kTr), (unsigned)((T + kTr - 1) / kTr));
        k_transpose_c64<<<grid, dim3(kTr, 8), 0, s>>>(frames, T, N, rows);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("mrf_gridding_match: transpose launch failed: %s", cudaGetErrorString(e));
            st = MRF_ECUDA;
        } else {
            note_launch("k_transpose_c64", s);
        }
    }
    if (st == MRF_OK)
        st = mrf_match(reinterpret_cast<const mrf_c64*>(rows), N, T, dict, atom_norm2, lut, m, precision, idx, pd,
                       t1t2, stream);
    cudaFreeAsync(frames, s);
    if (own_rows) cudaFreeAsync(own_rows, s);
    return st;
}

extern "C" mrf_status mrf_recon_run_host(mrf_plan p, const mrf_recon_params* prm, const mrf_c64* phi, int K,
                                         const mrf_c64* dict_c, const float* atom_norm2, const float* lut, int m,
                                         const mrf_c64* b_host, int n_iters, float* t1_host, float* t2_host,
                                         float* pd_host, double* cost_out, mrf_stream stream) {
    MRF_REQUIRE(p && prm && b_host, "mrf_recon_run_host: NULL plan, params or b_host");
    MRF_REQUIRE(n_iters >= 0, "mrf_recon_run_host: n_iters must be >= 0");
    cudaStream_t s = as_stream(stream);
    const int N = p->nx * p->ny;
    const size_t b_bytes = sizeof(float2) * (size_t)p->T * p->ns;
    const size_t map_bytes = sizeof(float) * (size_t)N;
    char* dev = nullptr;
    MRF_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dev), b_bytes + 3 * map_bytes, s));
    mrf_c64* b = reinterpret_cast<mrf_c64*>(dev);
    float* maps = reinterpret_cast<float*>(dev + b_bytes);
    mrf_status st = MRF_OK;
    mrf_recon R = nullptr;
    if (cudaMemcpyAsync(b, b_host, b_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        set_error("mrf_recon_run_host: host-to-device copy of b failed");
        st = MRF_ECUDA;
    }
    if (st == MRF_OK) st = mrf_recon_create(&R, p, prm, phi, K, dict_c, atom_norm2, lut, m, b, stream);
    if (st == MRF_OK) st = mrf_recon_iter(R, n_iters, cost_out, stream);
    if (st == MRF_OK) st = mrf_recon_maps(R, maps, maps + N, maps + 2 * N, nullptr, stream);
    float* host[3] = {t1_host, t2_host, pd_host};
    for (int i = 0; i < 3 && st == MRF_OK; ++i)
        if (host[i] &&
            cudaMemcpyAsync(host[i], maps + (size_t)i * N, map_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            set_error("mrf_recon_run_host: device-to-host copy of a map failed");
            st = MRF_ECUDA;
        }
    if (st == MRF_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("mrf_recon_run_host: %s", cudaGetErrorString(cudaGetLastError()));
        st = MRF_ECUDA;
    }
    if (R) mrf_recon_destroy(R);
    cudaFreeAsync(dev, s);
    return st;
}

// NUFFT plan layout shared by the NUFFT and reconstruction translation units.
#pragma once
#include "common.h"

struct mrf_plan_s {
    int nx = 0, ny = 0, T = 0, ns = 0, os = 2, W = 4;
    int gx = 0, gy = 0;           // oversampled grid
    int sf = 13;                  // grid columns owned by a forward strip (strip width - (W - 1))
    int nstrips_f = 0;            // forward strips: ceil(gx / sf)
    int nstrips_a = 0;            // adjoint strips: gx / strip width
    int ngroups = 0;              // distinct per-frame trajectories
    float beta = 0.f;             // Kaiser-Bessel shape
    double beta_d = 0.0;
    int parts = 1, frames_per_part = 1;  // frame split of the subspace adjoint reduction
    float* inv_dx = nullptr;      // [nx] 1 / psi_hat(x)
    float* inv_dy = nullptr;      // [ny]
    int4* fwd_rec = nullptr;      // samples by (group, forward strip of the first x node)
    int* fwd_off = nullptr;       // [ngroups * nstrips_f + 1]
    int4* adj_rec = nullptr;      // samples by (group, every adjoint strip they touch)
    float* fwd_w = nullptr;       // [fwd_rec entries][2 W] KB weights of each record: W along x, then W along y
    float* adj_w = nullptr;       // [adj_rec entries][2 W] the same for the adjoint records
    // frame-form spread as a sorted gather: every (group sample, tap) entry
    // ordered by (group, adjoint strip, point within the strip); built at the
    // first frame-form adjoint unless too large (then the atomic spread runs)
    int* fsp_off = nullptr;       // [ngroups * nstrips_a + 1] (also marks the table as built)
    int* fsp_loc = nullptr;       // point within the strip: gy * strip width + column
    int* fsp_smp = nullptr;       // sample index within the group's frame
    float* fsp_w = nullptr;       // KB weight of the tap
    bool fsp_tried = false;       // the build was attempted (it may have been skipped)
    int* adj_off = nullptr;       // [ngroups * nstrips_a + 1]
    int4* grec = nullptr;         // samples in (group, index) order
    int* group_of = nullptr;      // [T]
    // grouped adjoint: the (grid point, sample, weight) contributions of every
    // group sample, sorted by grid point (built on the first grouped adjoint)
    int gat_n = 0;                // number of entries
    int* gat_off = nullptr;       // [2] = {0, gat_n} (also marks the table as built)
    int* gat_pt = nullptr;        // grid point gy * G + gx
    int* gat_smp = nullptr;       // group sample g * ns + j
    float* gat_w = nullptr;       // psi(ux - mx) psi(uy - my)
    int gat_run = 32;             // tuned entries per thread of k_gather_grid
    int gat_threads = 128;        // tuned block size of k_gather_grid
    int gat_tuned_K = 0;          // K the tuning was done for (0: not tuned)
    int col_tile = 16;            // tuned strip width of the grouped column FFTs (16, 32 or 64)
    int col_tuned_K = 0;          // K the strip width was tuned for (0: not tuned)
    int* gf_off = nullptr;        // [ngroups + 1] frames of each group (CSR)
    int* gf = nullptr;            // [T]
    float2* h1 = nullptr;         // [T][ny][gx] rows transformed along x
    // subspace workspace (allocated on first use, for K <= 16)
    int sub_K = 0;
    float2* sub_h1 = nullptr;     // [16][ny][gx]
    float2* sub_spec = nullptr;   // [16][gy][gx]
    float2* sub_Y = nullptr;      // [ngroups][ns][16]
    float2* sub_R = nullptr;      // [ngroups][ns][16]
    float2* sub_partial = nullptr;  // [parts][ny][nx][16]
};

namespace mrf {
mrf_status subspace_forward(mrf_plan_s* p, const float2* alpha, const float2* phi, int K, float scale,
                            const float2* b, float2* y, int mode, cudaStream_t s);
mrf_status subspace_adjoint(mrf_plan_s* p, const float2* y, const float2* phi, int K, float scale,
                            float2* alpha_out, int mode, cudaStream_t s);
}  // namespace mrf

namespace mrf {
// allocate the subspace workspace of a plan (idempotent; K <= 16)
mrf_status ensure_subspace_workspace(mrf_plan_s* p, int K);
}  // namespace mrf

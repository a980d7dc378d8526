// Matching workspace and entry points shared by match.cu, match_tc.cu and the
// reconstruction loop.
#pragma once
#include "common.h"

namespace mrf {

constexpr int kTopK = 8;   // candidates kept by the BF16 scorer for the FP32 re-rank

struct MatchWorkspace {
    int* best_idx = nullptr;   // [n] winning atom
    float2* best_ip = nullptr; // [n] <d_k, x> of the winner
    int* cand = nullptr;       // [n][kTopK] tensor-core candidates (seeds of the next call)
    float* norm2 = nullptr;    // [m] ||d_m||^2
    float* wscore = nullptr;   // [m] score weight
    int cap_n = 0, cap_m = 0;
    bool borrowed = false;     // pointers carved from a caller-owned block
    // tensor-core matcher: dictionary operand in the shared-memory tile layout
    void* tc_b = nullptr;
    size_t tc_b_bytes = 0;
    const float2* tc_dict = nullptr;   // dictionary the operand was built from
    int tc_m = 0, tc_len = 0, tc_split = 0;
    int* tc_err = nullptr;     // set by a bounded wait that gave up
    ~MatchWorkspace();
    mrf_status reserve(int n, int m);
    void carve(char* base, int n, int m, size_t tc_bytes = 0);
    void detach();
    void release();
};

// norm2/score weights of the atoms (norm2_in nullable: computed from dict)
mrf_status match_prepare(MatchWorkspace& ws, const float2* dict, const float* norm2_in, int m, int len,
                         int literal, cudaStream_t s);
// winners for n fingerprints; outputs nullable; pd multiplied by pd_scale.
// cand_io (nullable, [n][kTopK], BF16 forms only): each row's seed atoms on
// entry, its tensor-core candidates on return (the winners do not depend on
// the seeds)
mrf_status match_run(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict, int m,
                     int precision, const float* lut, int* idx, float* pd, float* t1t2, float pd_scale,
                     cudaStream_t s, int* cand_io = nullptr);
// bytes of the tensor-core dictionary operand for m atoms of length len
size_t tc_operand_bytes(int m, int len, int prec);
// operand form of a tensor-core precision: 1 BF16, 3 split BF16, 8 FP8 e4m3 (0: FP32 path)
inline int tc_form(int precision) {
    return precision == MRF_MATCH_BF16 ? 1 : precision == MRF_MATCH_BF16X3 ? 3 : precision == MRF_MATCH_FP8 ? 8 : 0;
}
// one slice of a batched tensor-core matching launch: fingerprint blocks
// block0 .. block0 + ceil(n / 128) - 1 of the launch belong to this slice,
// matched against the slice's own dictionary operand (same m, length and
// precision for every slice of a launch)
struct TcSlice {
    const float2* x;
    int n;
    int block0;
    int* best_idx;
    float2* best_ip;
    const unsigned char* Bg;     // tensor-core operand of the slice's dictionary
    const float* wscore;         // score weights
    const float2* dict;          // FP32 dictionary (re-rank)
    int* cand = nullptr;         // [n][kTopK] the previous call's candidates in (seeds, -1: none), this
                                 // call's out; null: no seeding (always null at FP8)
};
// build (or reuse) the tensor-core operand of dict in ws
mrf_status tc_prepare_operand(MatchWorkspace& ws, const float2* dict, int m, int len, int prec, cudaStream_t s);
// winners of every slice of a batch in one launch; every slice's operand must
// have been prepared (tc_prepare_operand); ws supplies the error word
mrf_status match_tc_batch(MatchWorkspace& ws, const TcSlice* d_slices, int nslices, int total_blocks, int len,
                          int m, int prec, cudaStream_t s);
// idx / pd / t1t2 of n fingerprints from ws.best_idx / ws.best_ip
mrf_status match_finish(MatchWorkspace& ws, int n, const float* lut, int* idx, float* pd, float* t1t2,
                        float pd_scale, cudaStream_t s);
// tensor-core candidate search and FP32 re-rank (match_tc.cu)
mrf_status match_tc_candidates(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict, int m,
                               int prec, cudaStream_t s, int* cand_io = nullptr);
mrf_status match_rerank(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict,
                        cudaStream_t s);
// full-length fingerprints (a padded reduction beyond the resident tile of
// k_match_tc): the streamed tensor-core matcher of match_tc_long.cu
bool tc_long(int len, int prec);
size_t tc_long_scratch_bytes(int n, int m, int len, int prec);
mrf_status match_tc_long(MatchWorkspace& ws, const float2* x, int n, int len, const float2* dict, int m, int prec,
                         cudaStream_t s);

}  // namespace mrf

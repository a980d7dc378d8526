// Exact k nearest patches of integer patch vectors (the sparse graph of Eq. 7).
#pragma once
#include "common.h"

namespace mrf {

struct KnnWorkspace {
    void* bop = nullptr;          // tensor-core candidate operand (f16 core-matrix tiles)
    size_t bop_bytes = 0;
    int* nrm = nullptr;           // [np] squared norm of the centred vectors
    unsigned* bound = nullptr;    // [np] seeded bound of each row's knn-th distance
    int* pnbr = nullptr;          // [parts][np][knn] per-partition lists
    unsigned* pd2 = nullptr;
    size_t part_entries = 0;      // capacity of pnbr / pd2
    int np_cap = 0;
    int* err = nullptr;           // set when a feature is outside [0, 4096] or a wait gave up
    ~KnnWorkspace();
    // allocate for np vectors of length fd and knn neighbours (outside any
    // stream capture); knn_run allocates nothing when this was large enough
    mrf_status reserve(int np, int fd, int knn);
    void release();
};

// nbr/d2 [np][knn]: the knn rows j != i of F [np][ld] nearest to row i, by the
// exact squared distance over the first fd entries, ascending, ties to the
// lower j.  Needs np > knn, 1 <= knn <= 32, fd <= 255, ld % 4 == 0 and the
// entries fd <= k < ld zero; the tensor-core path (fd <= 128) needs
// 0 <= F <= 4096 and raises ws.err otherwise.  seed (nullable, [np][knn],
// may be nbr itself): a previous neighbour list; on the tensor-core path the
// distances to a row's seeds bound its search, which leaves the result
// unchanged (seeds that are not knn distinct rows j != i give no bound).
mrf_status knn_run(KnnWorkspace& ws, const int* F, int np, int fd, int ld, int knn, int* nbr, unsigned* d2,
                   cudaStream_t s, const int* seed = nullptr);

}  // namespace mrf

// mst.cuh -- exact Euclidean minimum spanning tree by Boruvka rounds.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace iso {

enum : int { MC_OVERFLOW = 0, MC_NEDGES = 1, MC_NCOMP = 2, MC_ROUNDS = 3, MC_OVF_TOTAL = 4, MC_NCOMP_NEW = 5 };

struct MstScratch {
    int64_t n = 0;
    int splits = 1;                // column splits of the sweep grid
    int32_t *comp, *nxt, *nxt2, *tgt;
    float *b1v, *b2v;              // [splits][n] approximate best / second best
    int32_t *b1j;                  // [splits][n]
    double *rowd2;                 // [n] exact best key per row
    int32_t *rowj;                 // [n] (-1 none, -2 pending rescan)
    unsigned long long *cd2, *cpair;   // [n] per component (root-indexed)
    int32_t *cu, *cv;              // [n] chosen edge per component
    double *cdd;                   // [n]
    int32_t *ovf_rows;             // [n]
    int32_t *counters;             // [8]
    int32_t *eu, *ev;              // [n-1] edges as found
    double *ed2;                   // [n-1]
    uint64_t *skey, *kbuf;         // sort buffers [n]
    int32_t *sval, *vbuf;          // [n]
    unsigned long long *nnbits;    // [n] nearest-neighbour d2 (bits) per vertex

    void carve(Arena &A, int64_t n, int splits);
};

int mst_splits(int64_t n);

// Tensor-core sweep state (mst_tc.cu): centred BF16 hi/lo copies of X padded
// to the 128 x 64 tile grid, their TMA maps, squared norms and the best-8
// candidate lists of every (column split, row).
struct TcScratch {
    int64_t n_pad = 0;
    int32_t d_pad = 0;
    int splits = 1;
    __nv_bfloat16 *xh = nullptr, *xl = nullptr;   // rows in norm order: row r is point perm[r]
    float *nrm = nullptr, *rsq = nullptr;          // |y|^2 and |y| of the represented rows
    float *tmax = nullptr, *tsq = nullptr;         // per 128-row tile: max |y|^2 and its sqrt
    float *mean = nullptr;
    double *part = nullptr;
    unsigned int *nmax_bits = nullptr;
    int32_t *perm = nullptr, *iperm = nullptr, *vbuf = nullptr, *compp = nullptr;
    uint64_t *keys = nullptr, *kbuf = nullptr;
    float *tv = nullptr, *tu = nullptr;            // per (split, row): best-8 tile lower bounds, best upper bound
    int32_t *tj = nullptr;
    uint32_t *err = nullptr;
    CUtensorMap map_h, map_l;
    void carve(Arena &A, int64_t n, int32_t d, int splits);
    static size_t bytes_needed(int64_t n, int32_t d, int splits);
};
int tc_splits(int64_t n);
bool tc_supported();
cudaError_t tc_prepare(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s);
cudaError_t tc_sweep_round(TcScratch &T, MstScratch &S, const float *X, int64_t n, int32_t d, uint32_t *status,
                           cudaStream_t s);

// Builds the MST of X (n x d, dtype F32/F64) into S.eu/ev/ed2 (unsorted).
// tc != nullptr selects the tensor-core sweep (F32 input).
// sweep_fp64: use the exact FP64 sweep instead of FP32 + recheck.
// rounds_out / rescans_out: host copies of the round and rescan counts are
// written after the final stream synchronisation by the caller.
cudaError_t mst_build(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                      uint32_t *status, cudaStream_t s, TcScratch *tc = nullptr);

// Nearest-neighbour d2 of every row (exact key), one Boruvka-style sweep with
// every point its own component.  Result in S.rowd2 / S.rowj.
cudaError_t nn_sweep(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                     uint32_t *status, cudaStream_t s, TcScratch *tc = nullptr);

// Sort S.eu/ev/ed2 by key (d2, u, v) into the output arrays (u < v).
cudaError_t mst_sort_edges(MstScratch &S, int32_t *out_u, int32_t *out_v, double *out_d2, cudaStream_t s);

// nnbits[v] = min d2 over MST edges incident to v (the exact nearest
// neighbour, which is always a tree edge).
cudaError_t nn_from_edges(MstScratch &S, const int32_t *eu, const int32_t *ev, const double *ed2,
                          cudaStream_t s);

}  // namespace iso

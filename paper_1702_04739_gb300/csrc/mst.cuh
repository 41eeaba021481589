// mst.cuh -- exact Euclidean minimum spanning tree by Boruvka rounds.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace iso {

enum : int {
    MC_OVERFLOW = 0, MC_NEDGES = 1, MC_NCOMP = 2, MC_ROUNDS = 3, MC_OVF_TOTAL = 4, MC_NCOMP_NEW = 5,
    MC_TARGET = 6   // components at which the forest is complete: 1, or the number of independent sets
};

struct MstScratch {
    int64_t n = 0;
    int splits = 1;                // column splits of the sweep grid
    int32_t *comp, *nxt, *tgt;
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

// Tensor-core sweep state (mst_tc.cu): centred BF16 hi/lo copies of X in a
// padded row space of 128-row tiles, their TMA maps, squared norms and the
// best-8 candidate lists of every (list, row).  One set: rows in norm order,
// padding after the last point.  Independent sets: each set centred on its
// own mean, in norm order inside its own run of whole tiles.
struct TcScratch {
    int64_t n_pad = 0;                             // padded row space (whole 128-row tiles)
    int32_t d_pad = 0;
    int splits = 1;                                // column splits per row tile (one set)
    int lists = 2;                                 // candidate lists per row (2 per split: tiles of a pair)
    int cw = 64;                                   // columns per candidate block (64 or 32)
    bool resident = true;                          // row block resident in shared memory when d_pad <= 128
    __nv_bfloat16 *xh = nullptr, *xl = nullptr;   // row r is point permp[r] (zero rows at padding)
    float *xs = nullptr;                           // [n_pad][d] the points themselves in the same order
    float *nrm = nullptr, *rsq = nullptr;          // |y|^2 and |y| of the represented rows (0 at padding)
    float *cnrm = nullptr;                         // |y|^2 as a column: +inf at padding
    float *tmax = nullptr, *tsq = nullptr;         // per 128-row tile: max |y|^2 and its sqrt
    float *mean = nullptr;                         // [nmeans][d]
    double *part = nullptr;
    unsigned int *nmax_bits = nullptr;
    int32_t *perm = nullptr, *permp = nullptr, *vbuf = nullptr, *compp = nullptr;
    uint64_t *keys = nullptr, *kbuf = nullptr;
    float *tv = nullptr, *tu = nullptr;            // per (list, row): best-8 candidate-block lower bounds, best upper bound
    int32_t *tj = nullptr;
    int32_t *nsurv = nullptr, *surv = nullptr;     // per row: columns to key in FP64 (padded column indices)
    uint32_t *err = nullptr;
    uint32_t *qctr = nullptr;                      // the sweep's work-item counter (zeroed before each launch)
    // independent sets (null for one set): sweep work items {row tile,
    // first and end column tile, split}, set of each point, set offsets
    // and the first padded row of each set (device arrays)
    const int4 *items = nullptr;
    int64_t nitems = 0;
    int32_t nsets = 1;
    const int32_t *set_of = nullptr;
    const int64_t *offs = nullptr;
    const int64_t *rowbase = nullptr;
    int32_t *setcnt = nullptr;                     // components left in each set (independent sets)
    bool keep_order = false;                       // rows as given instead of norm order
    uint64_t wait_cycles = 0;                      // bound of each sweep wait in SM cycles (0: default)
    int stall_test = 0;                            // test hook: the epilogue's first wait cannot complete
    int shard_rank = 0, shard_world = 1;           // sharded call: this rank sweeps row tiles t = rank mod world
    // Pruned rounds (one set, set before carve): rows in a bisection order
    // whose 128-row tiles are compact, each tile's centroid and radius, and
    // per round the pairs of tiles that can hold a component's lightest
    // outgoing edge (mst_prune.cu)
    bool prune = false;
    bool prune_ready = false;                      // the pruned row order is in place (after the first round)
    float *tcen = nullptr;                         // [ntiles][d] tile centroids
    float *trad = nullptr;                         // [ntiles] radii (rounded up)
    float *tlb2 = nullptr;                         // [ntiles][ntiles] lower bound of d2 between two tiles' points
    unsigned int *cub = nullptr;                   // [n] per component: upper bound of its lightest outgoing d2 (bits)
    float *tmu = nullptr;                          // [ntiles] largest bound over the components of a tile's rows
    int32_t *tcomp = nullptr;                      // [ntiles] the one component of a tile's rows, or -1
    int4 *items_a = nullptr, *items_b = nullptr;   // [ntiles] near items, [ntiles][PRUNE_SLOTS - 1] far items
    unsigned long long *far = nullptr;             // [2][ntiles] order construction: farthest points per node
    unsigned long long *swept = nullptr;           // [1] tile pairs swept by the pruned rounds so far
    int32_t *nlists = nullptr;                     // [ntiles] candidate lists the row tile's items write this round
    CUtensorMap map_h, map_l;
    // n_pad_rows / nmeans / lists: 0 = one set
    void carve(Arena &A, int64_t n, int32_t d, int splits, int64_t n_pad_rows = 0, int nmeans = 1, int lists = 0);
};
int tc_splits(int64_t n);
// Pruned rounds: candidate-list slots per row (slot 0: the near tiles,
// 1..PRUNE_SLOTS-1: the far items of the row tile) and near window (tiles).
constexpr int PRUNE_SLOTS = 16;
constexpr int PRUNE_NEAR = 2;
// Whether a one-set call of n points in d dimensions prunes its rounds
// (isoclust_set_mst_prune: -1 auto, 0 never, 1 whenever supported).
bool prune_wanted(int64_t n, int32_t d);
void prune_set_mode(int mode);
int prune_mode();
// Before the first round: rows re-ordered for the pruned rounds (points whose
// distance to the nearest of 256 sample points is more than 4x the median
// of that distance at the end, the others in bisection order), the sweep's
// row data re-placed, the tile geometry.  rowd2 (n doubles) is scratch here.
cudaError_t prune_reorder(TcScratch &T, double *rowd2, const float *X, int64_t n, int32_t d, cudaStream_t s);
// Re-place the sweep's rows (hi/lo split, norms, tile maxima) in T.perm's order.
cudaError_t tc_place_rows(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s);
// Per round, after the near sweep: component bounds and the far items.
cudaError_t prune_far_items(TcScratch &T, const int32_t *comp, const double *rowd2, const int32_t *rowj, int64_t n,
                            const int32_t *counters, cudaStream_t s);
bool tc_supported();
// place = false: the rows are placed later (tc_place_rows, by the pruned
// rounds' order); only the mean, maps and buffers are prepared.
cudaError_t tc_prepare(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s, bool place = true);
cudaError_t tc_sweep_round(TcScratch &T, MstScratch &S, const float *X, int64_t n, int32_t d, uint32_t *status,
                           cudaStream_t s);
// omega screen on the tensor cores: Xp (n x d, omega's row order) and its
// nearest-neighbour d2 bits; need[I * T64 + J] = 1 for every pair of 64-row
// tiles (I <= J) holding a pair within the cutoff zskip of eq. omega's terms
cudaError_t tc_omega_screen(TcScratch &T, const float *Xp, int64_t n, int32_t d,
                            const unsigned long long *nnbits, double sigma, double zskip, uint8_t *need, int64_t T64,
                            cudaStream_t s);
// Sweep variant (bit 0: 32-column candidate blocks, bit 1: streamed row
// block): forced by tc_force_variant, else the fastest of one timed trial
// round per variant, cached per device and shape class.  Runs on the
// round-1 state before the first round and restores the round counters.
cudaError_t tc_autotune(TcScratch &T, MstScratch &S, const float *X, int64_t n, int32_t d, uint32_t *status,
                        cudaStream_t s);
void tc_force_variant(int variant);     // -1: tune
int tc_forced_variant();                // the setting (-1: tune)
int tc_last_variant();                  // this thread's last variant (-1: none)
void tc_clear_last_variant();           // a build without the tensor-core sweep
// independent sets: recount the components of every set from comp
cudaError_t tc_count_sets(TcScratch &T, const int32_t *comp, int64_t n, const int32_t *counters, cudaStream_t s);

// Builds the MST of X (n x d, dtype F32/F64) into S.eu/ev/ed2 (unsorted).
// tc != nullptr selects the tensor-core sweep (F32 input).
// sweep_fp64: use the exact FP64 sweep instead of FP32 + recheck.
// rounds_out / rescans_out: host copies of the round and rescan counts are
// written after the final stream synchronisation by the caller.
// target: components left when the forest is complete (1 for one point set;
// the number of sets when X holds independent sets, whose pairs the sweep
// never mixes); max_n bounds the rounds (the largest set).
// sh != nullptr (sharded call, tensor-core sweep only): each rank's rows
// give the per-component minima, combined across ranks by the caller's
// all-reduce before the union-find.
cudaError_t mst_build(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                      uint32_t *status, cudaStream_t s, TcScratch *tc = nullptr, int32_t target = 1,
                      int64_t max_n = 0, const Shard *sh = nullptr);

// Nearest-neighbour d2 of every row (exact key), one Boruvka-style sweep with
// every point its own component.  Result in S.rowd2 / S.rowj.
cudaError_t nn_sweep(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                     uint32_t *status, cudaStream_t s, TcScratch *tc = nullptr);

// Sort S.eu/ev/ed2 by key (d2, u, v) into the output arrays (u < v).
cudaError_t mst_sort_edges(MstScratch &S, int32_t *out_u, int32_t *out_v, double *out_d2, cudaStream_t s);

// nnbits[v] = min d2 over MST edges incident to v (the exact nearest
// neighbour, which is always a tree edge).
// m: number of edges (default n - 1; a forest of independent sets has fewer).
cudaError_t nn_from_edges(MstScratch &S, const int32_t *eu, const int32_t *ev, const double *ed2,
                          cudaStream_t s, int64_t m = -1);

}  // namespace iso

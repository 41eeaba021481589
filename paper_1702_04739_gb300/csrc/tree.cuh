// tree.cuh -- rooted-tree preparation and Algorithms 1/2/4 on the device.
#pragma once
#include "common.cuh"

namespace iso {

constexpr int DP_LANES = 32;          // thresholds evaluated per Algorithm-1 pass
constexpr int DP_SEARCH_PASSES = 14;  // 1 bracketing pass + 13 passes of 33-ary search
// One tree: after the bracketing pass, up to DP_CAND_PASSES passes take their
// thresholds from the critical ratios of the vertices (see
// tree_search_and_label), then 33-ary search of the bit patterns finishes
// whatever remains (at most 13 passes).
constexpr int DP_CAND_PASSES = 8;
constexpr int DP_TREE_PASSES = 1 + DP_CAND_PASSES + 13;
constexpr int CAND_BUCKETS = 4096;    // histogram of critical ratios over the bracket's bit patterns
constexpr int CAND_EXACT = 10;        // at most this many left: they are tried exactly (+-1 ulp)
constexpr int CAND_SET_BUCKETS = 64;  // independent sets: buckets per set (a multiple of 32)
enum : uint8_t { DEC_DISCARD = 0, DEC_CUT = 1, DEC_JOIN = 2 };

// Device-resident search state of reading S (bisection to the last bit).
constexpr int STATS_BLOCKS = 128;   // blocks of the statistics' first level (fixed: deterministic sums)

struct SearchState {
    unsigned long long lo_bits, hi_bits;
    int have_lo, have_hi, done, error;
    double thr[DP_LANES];
    int cnt[DP_LANES];
    double beta;
    double stats[8];          // phi*, phi_*, omega*, omega_*, p*, p_*, alpha0, beta0
    int passes;               // Algorithm-1 passes that did work
    int max_depth;
    int nleaves;
    int selected;             // cuts among the first k (must equal k)
    unsigned long long ik_bits;
    int lane_lo;              // lane of the last pass whose threshold is lo (-1: none)
    int mode;                 // 0: thresholds from critical ratios, 1: 33-ary bit search
    int cand_passes;          // passes that took their thresholds from critical ratios
    unsigned int ncand;       // critical ratios inside the bracket (this pass)
    unsigned long long cand[CAND_EXACT];
    int final_lane;           // lane of the last pass whose threshold is beta (-1: none; one tree)
};

// Rooted tree in device scratch.
struct TreeDev {
    int64_t n;
    int32_t root;
    int32_t *parent;     // [n], root -1
    int32_t *edge_of;    // [n], input edge index of the parent edge (-1 at the root)
    int32_t *bfs_pos;    // [n], position in the canonical BFS order
    int32_t *ch_off;     // [n+1]
    int32_t *ch_list;    // [max(n-1,1)], children ascending within each parent
    int32_t *adj_off;    // [n+1] sorted adjacency (directed edges grouped by source)
    uint64_t *adj_key;   // [2(n-1)] (src<<32 | dst), sorted
    int32_t *leaves;     // [n]
    int32_t *depth;      // [n]
    int32_t *pre;        // [n] preorder rank with children in ascending index (set by orient_tree)
    int32_t *slot;       // [n] position in the parent's child list (the root: n - 1), set by orient_tree
};

struct TreeScratchSizes;

// Carves (or measures) the scratch of the tree stage.
struct TreeScratch {
    TreeDev T;
    // orientation temporaries
    uint64_t *kbuf;
    int32_t *vals, *vbuf;
    int32_t *rev, *succ, *succ2, *rnk, *rnk2, *size, *flag, *fpos, *tmp32;
    int64_t *ssz, *sx, *tmp64;
    int32_t *anc, *anc2, *dep2, *pre, *pre2, *ib;
    uint64_t *bkeys;
    // DP
    uint8_t *dec;
    double *wh, *ph, *rat;
    int32_t *done, *head, *head2, *cflag, *cidx;
    uint32_t *hist;      // [CAND_BUCKETS] critical ratios per bucket of the bracket
    double *spart;       // [STATS_BLOCKS][6] partial sums and minima of the statistics
    double *phis;        // [n] phi of each child-list slot's parent edge
    SearchState *search;
    uint32_t *status;
    int32_t *hostinfo;   // small device block read back by the host

    void carve(Arena &A, int64_t n);
};

// Orient the tree given by m = n-1 undirected edges (eu, ev) from `root`.
// Writes T.parent, T.edge_of, T.bfs_pos, T.ch_off/ch_list, T.depth, leaves.
// Flags DEV_BAD_TREE if the edges are not a spanning tree.  If
// expect_parent != nullptr, also flags DEV_BAD_TREE when the orientation
// differs from it.
// vset != nullptr: the tree joins independent sets under a virtual root
// (vertex n - 1, vset[v] = set of each real vertex v); the BFS order is then
// set-major, (depth, preorder) inside each set.
// part 0: the whole orientation, with a host check of the Euler tour (a bad
// tree returns before the tour is used); part 1: the tour and its ranking up
// to that check (no host synchronisation: the caller reads S.status); part
// 2: the rest (call only after the caller has seen no DEV_BAD_TREE).
cudaError_t orient_tree(TreeScratch &S, const int32_t *eu, const int32_t *ev, int64_t n,
                        int32_t root, const int32_t *expect_parent, cudaStream_t s, const int32_t *vset = nullptr,
                        int part = 0);

// Edges (eu, ev) from a parent array (root entry skipped), written into
// S.fpos/S.flag-sized buffers; returns the buffers through out pointers.
cudaError_t edges_from_parent(TreeScratch &S, const int32_t *parent, int64_t n, int32_t *eu,
                              int32_t *ev, cudaStream_t s);

// Algorithms 2 + 1 (search) and the labels of Algorithm 4.
cudaError_t tree_search_and_label(TreeScratch &S, const double *phi_par, const double *omega,
                                  const double *p, int32_t k, int32_t *labels, uint8_t *residual,
                                  double *i_k, cudaStream_t s);

// After orient_tree with vset: every set's first point becomes a root
// (parent -1, no parent edge).
cudaError_t fix_set_roots(TreeScratch &S, int32_t nsets, const int64_t *offs, cudaStream_t s);

// Independent sets on a tree oriented with vset (see orient_tree): each
// set's own roots, statistics, search (state SS[b], k = ks[b]) and labels.
// labels / residual cover the real vertices; i_k and beta (nullable) one
// entry per set.  set_hist: nsets x CAND_SET_BUCKETS + 1 counters (scratch).
cudaError_t tree_search_and_label_sets(TreeScratch &S, int32_t nsets, const int64_t *offs, const int32_t *vset,
                                       const int32_t *ks, SearchState *SS, uint32_t *set_hist, const double *phi_par,
                                       const double *omega, const double *p, int32_t *labels, uint8_t *residual,
                                       double *i_k, double *beta, cudaStream_t s);

// phi of each oriented parent edge from the MST edge d2 (eq. phi).
cudaError_t phi_from_edges(const TreeScratch &S, const double *edge_d2, double sigma, double *phi_par,
                           cudaStream_t s);

// omega in the tree-incident mode: sum of phi over incident tree edges,
// ascending neighbour index.
cudaError_t omega_tree_mode(const TreeScratch &S, const double *phi_par, int32_t include_self,
                            double *omega, cudaStream_t s);

}  // namespace iso

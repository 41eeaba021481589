// tree.cu -- the tree half of the hot path.
//
//  * Orientation (Section 2.2 step 3, "BFS order and parent"): the tree is
//    rooted by an Euler tour over the sorted adjacency plus Wyllie list
//    ranking, so the work takes O(log n) launches whatever the tree depth.
//    Subtree sizes from the tour give the preorder rank with children in
//    ascending index; sorting by (depth, preorder) gives the canonical BFS
//    order (children ascending), which fixes Algorithm 1's visiting order.
//  * Algorithm 1 (decision) is evaluated for 32 thresholds at once, one warp
//    lane per threshold.  Instead of one launch per depth level (Section 3.6)
//    a warp starts at every leaf and walks towards the root; the last child
//    to finish a vertex (an atomic arrival counter) folds all of that
//    vertex's children in descending index order (the order Algorithm 1
//    visits siblings, which replaces the ChildId sequencing) and continues
//    upwards.  Every vertex is decided exactly once per pass, with no
//    barrier and no spin-wait.
//  * Algorithm 2 runs to the last bit as a 33-ary search over the ordered
//    bit patterns of non-negative doubles, kept on the device.
//  * Algorithm 4's labels: head pointers (eta) by pointer jumping, an
//    exclusive scan over Cut in processing order, first k cuts kept.
#include "tree.cuh"

namespace iso {

// ---------------------------------------------------------------- scratch
void TreeScratch::carve(Arena &A, int64_t n) {
    int64_t m = n > 0 ? n - 1 : 0;
    int64_t M = 2 * m;
    int64_t big = (M > n ? M : n) + 1;
    T.n = n;
    T.parent = A.take<int32_t>(n);
    T.edge_of = A.take<int32_t>(n);
    T.bfs_pos = A.take<int32_t>(n);
    T.ch_off = A.take<int32_t>(n + 1);
    T.ch_list = A.take<int32_t>(m > 0 ? m : 1);
    T.adj_off = A.take<int32_t>(n + 1);
    T.adj_key = A.take<uint64_t>(big);
    T.leaves = A.take<int32_t>(n);
    T.depth = A.take<int32_t>(n);
    T.slot = A.take<int32_t>(n);
    kbuf = A.take<uint64_t>(big);
    vals = A.take<int32_t>(big);
    vbuf = A.take<int32_t>(big);
    rev = A.take<int32_t>(big);
    succ = A.take<int32_t>(big);
    succ2 = A.take<int32_t>(big);
    rnk = A.take<int32_t>(big);
    rnk2 = A.take<int32_t>(big);
    flag = A.take<int32_t>(big);
    fpos = A.take<int32_t>(big + 1);
    size = A.take<int32_t>(n);
    tmp32 = A.take<int32_t>(scan_tmp_elems(big + 1));
    ssz = A.take<int64_t>(n);
    sx = A.take<int64_t>(n);
    tmp64 = A.take<int64_t>(scan_tmp_elems(n));
    anc = A.take<int32_t>(n);
    anc2 = A.take<int32_t>(n);
    dep2 = A.take<int32_t>(n);
    pre = A.take<int32_t>(n);
    pre2 = A.take<int32_t>(n);
    ib = A.take<int32_t>(n);
    bkeys = A.take<uint64_t>(n);
    dec = A.take<uint8_t>((size_t)n * DP_LANES);
    wh = A.take<double>((size_t)n * DP_LANES);
    ph = A.take<double>((size_t)n * DP_LANES);
    rat = A.take<double>(n);
    done = A.take<int32_t>(n);
    head = A.take<int32_t>(n);
    head2 = A.take<int32_t>(n);
    cflag = A.take<int32_t>(n + 1);
    cidx = A.take<int32_t>(n + 1);
    hist = A.take<uint32_t>(CAND_BUCKETS);
    spart = A.take<double>(6 * STATS_BLOCKS);
    phis = A.take<double>(n);
    search = A.take<SearchState>(1);
    status = A.take<uint32_t>(1);
    hostinfo = A.take<int32_t>(16);
}

namespace {

constexpr int TPB = 256;
inline unsigned blocks_for(int64_t n) { return (unsigned)(n > 0 ? ceil_div(n, TPB) : 1); }
inline int log2_ceil(int64_t x) {
    int l = 0;
    while ((1LL << l) < x) ++l;
    return l;
}

__device__ __forceinline__ void flag_status(uint32_t *st, uint32_t bit) { atomicOr(st, bit); }

__device__ __forceinline__ uint8_t ld_cg_u8(const uint8_t *p) {
    unsigned short v;
    asm volatile("ld.global.cg.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint8_t)v;
}
__device__ __forceinline__ double ld_cg_f64(const double *p) {
    double v;
    asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

// ------------------------------------------------------------ orientation
__global__ void k_dir_keys(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev, int64_t m,
                           int64_t n, uint64_t *__restrict__ keys, int32_t *__restrict__ vals,
                           uint32_t *st) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int64_t u = eu[e], v = ev[e];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v) {
        flag_status(st, DEV_BAD_TREE);
        u = 0; v = 0;
    }
    keys[2 * e] = ((uint64_t)u << 32) | (uint64_t)v;
    vals[2 * e] = (int32_t)(2 * e);
    keys[2 * e + 1] = ((uint64_t)v << 32) | (uint64_t)u;
    vals[2 * e + 1] = (int32_t)(2 * e + 1);
}

__global__ void k_adj_off(const uint64_t *__restrict__ keys, int64_t M, int64_t n, int32_t *adj_off,
                          uint32_t *st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) adj_off[n] = (int32_t)M;
    if (i >= M) return;
    uint32_t s = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != s) adj_off[s] = (int32_t)i;
    if (i > 0 && keys[i] == keys[i - 1]) flag_status(st, DEV_BAD_TREE);
}

__global__ void k_rev_succ(const uint64_t *__restrict__ keys, const int32_t *__restrict__ adj_off,
                           int64_t M, int64_t n, int32_t *__restrict__ rev, int32_t *__restrict__ succ,
                           uint32_t *st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    uint64_t k = keys[i];
    uint32_t u = (uint32_t)(k >> 32), v = (uint32_t)(k & 0xffffffffu);
    int64_t lo = (v < n) ? adj_off[v] : -1, hi = (v < n) ? adj_off[v + 1] : -1;
    if (lo < 0 || hi < 0 || hi < lo || hi > M) {   // vertex with no edges: not spanning
        flag_status(st, DEV_BAD_TREE);
        rev[i] = (int32_t)i;
        succ[i] = -1;
        return;
    }
    uint64_t target = ((uint64_t)v << 32) | (uint64_t)u;
    int64_t a = lo, b = hi;
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        if (keys[mid] < target) a = mid + 1; else b = mid;
    }
    if (a >= hi || keys[a] != target) {
        flag_status(st, DEV_BAD_TREE);
        rev[i] = (int32_t)i;
        succ[i] = -1;
        return;
    }
    rev[i] = (int32_t)a;
    int64_t nx = a + 1;
    if (nx == hi) nx = lo;
    succ[i] = (int32_t)nx;
}

__global__ void k_check_adj(const int32_t *__restrict__ adj_off, int64_t n, uint32_t *st) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && adj_off[v] < 0) flag_status(st, DEV_BAD_TREE);
}

__global__ void k_break_tour(const int32_t *__restrict__ adj_off, const int32_t *__restrict__ rev,
                             int32_t *succ, int32_t root, int64_t M, uint32_t *st) {
    int32_t a = adj_off[root], b = adj_off[root + 1];
    if (a < 0 || b <= a || b > M) { flag_status(st, DEV_BAD_TREE); return; }
    int32_t last = rev[b - 1];
    if (last >= 0 && last < M) succ[last] = -1;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// one Wyllie step: distance-to-end ranking along succ
__global__ void k_wyllie(const int32_t *__restrict__ sin, const int32_t *__restrict__ rin,
                         int32_t *__restrict__ sout, int32_t *__restrict__ rout, int64_t M) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int32_t s = sin[i];
    if (s >= 0) {
        rout[i] = rin[i] + rin[s];
        sout[i] = sin[s];
    } else {
        rout[i] = rin[i];
        sout[i] = -1;
    }
}

__global__ void k_check_ranked(const int32_t *__restrict__ succ, const int32_t *__restrict__ rnk,
                               int64_t M, uint32_t *st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    if (succ[i] != -1 || rnk[i] < 1 || rnk[i] > M) flag_status(st, DEV_BAD_TREE);
}

__global__ void k_orient(const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals,
                         const int32_t *__restrict__ rev, const int32_t *__restrict__ rnk, int64_t M,
                         int64_t n, int32_t root, int32_t *__restrict__ parent, int32_t *__restrict__ size,
                         int32_t *__restrict__ edge_of, int32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        parent[root] = -1;
        size[root] = (int32_t)n;
        edge_of[root] = -1;
    }
    if (i >= M) return;
    int32_t j = rev[i];
    int32_t pi = (int32_t)M - rnk[i], pj = (int32_t)M - rnk[j];
    if (pi < pj) {
        uint64_t k = keys[i];
        int32_t u = (int32_t)(k >> 32), v = (int32_t)(k & 0xffffffffu);
        parent[v] = u;
        size[v] = (pj - pi + 1) / 2;
        edge_of[v] = vals[i] >> 1;
        flag[i] = 1;
    } else {
        flag[i] = 0;
    }
}

__global__ void k_check_parent(const int32_t *__restrict__ got, const int32_t *__restrict__ want,
                               int64_t n, uint32_t *st) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && got[v] != want[v]) flag_status(st, DEV_BAD_TREE);
}

__global__ void k_scan_total(const int32_t *__restrict__ flag, int32_t *fpos, int64_t M) {
    fpos[M] = M > 0 ? fpos[M - 1] + flag[M - 1] : 0;
}

__global__ void k_children(const uint64_t *__restrict__ keys, const int32_t *__restrict__ flag,
                           const int32_t *__restrict__ fpos, int64_t M, int32_t *__restrict__ ch_list) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && flag[i]) ch_list[fpos[i]] = (int32_t)(keys[i] & 0xffffffffu);
}

// slot[v]: v's position in its parent's child list (the orientation root:
// n - 1), a permutation of [0, n).  Algorithm 1's per-threshold states are
// stored by slot, so a vertex's children are the contiguous slots of its
// child range.
__global__ void k_slots(const int32_t *__restrict__ ch_list, int64_t n, int32_t root, int32_t *__restrict__ slot) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n - 1) slot[ch_list[q]] = (int32_t)q;
    else if (q == n - 1) slot[root] = (int32_t)q;
}

// phi of each child-list entry's parent edge, in child-list order
__global__ void k_phi_slots(const int32_t *__restrict__ ch_list, const double *__restrict__ phi, int64_t m,
                            double *__restrict__ phis) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) phis[q] = phi[ch_list[q]];
}

__global__ void k_ch_off(const int32_t *__restrict__ adj_off, const int32_t *__restrict__ fpos,
                         int64_t n, int32_t *__restrict__ ch_off) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v <= n) ch_off[v] = fpos[adj_off[v]];
}

__global__ void k_child_sizes(const int32_t *__restrict__ ch_list, const int32_t *__restrict__ size,
                              int64_t m, int64_t *__restrict__ ssz) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) ssz[q] = size[ch_list[q]];
}

// preorder weight of each vertex: 1 + total size of its earlier siblings
__global__ void k_pre_init(const int32_t *__restrict__ parent, const int32_t *__restrict__ ch_off,
                           const int32_t *__restrict__ ch_list, const int64_t *__restrict__ sx, int64_t m,
                           int32_t root, int32_t *__restrict__ anc, int32_t *__restrict__ dep,
                           int32_t *__restrict__ pre) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) {
        anc[root] = -1;
        dep[root] = 0;
        pre[root] = 0;
    }
    if (q >= m) return;
    int32_t c = ch_list[q];
    int32_t u = parent[c];
    int64_t off = sx[q] - sx[ch_off[u]];
    anc[c] = u;
    dep[c] = 1;
    pre[c] = (int32_t)(1 + off);
}

__global__ void k_jump_acc(const int32_t *__restrict__ ain, const int32_t *__restrict__ din,
                           const int32_t *__restrict__ pin, int32_t *__restrict__ aout,
                           int32_t *__restrict__ dout, int32_t *__restrict__ pout, int64_t n) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t a = ain[v];
    if (a >= 0) {
        dout[v] = din[v] + din[a];
        pout[v] = pin[v] + pin[a];
        aout[v] = ain[a];
    } else {
        dout[v] = din[v];
        pout[v] = pin[v];
        aout[v] = -1;
    }
}

__global__ void k_bfs_keys(const int32_t *__restrict__ dep, const int32_t *__restrict__ pre, int64_t n,
                           uint64_t *__restrict__ bkeys, int32_t *__restrict__ ib) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    bkeys[v] = ((uint64_t)(uint32_t)dep[v] << 32) | (uint64_t)(uint32_t)pre[v];
    ib[v] = (int32_t)v;
}

__global__ void k_bfs_pos(const int32_t *__restrict__ ib, const uint64_t *__restrict__ bkeys, int64_t n,
                          int32_t *__restrict__ bfs_pos, SearchState *S) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bfs_pos[ib[i]] = (int32_t)i;
    if (i == n - 1) S->max_depth = (int)(bkeys[i] >> 32);
}

__global__ void k_leaf_flags(const int32_t *__restrict__ ch_off, int64_t n, int32_t *__restrict__ flag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flag[v] = ch_off[v + 1] == ch_off[v] ? 1 : 0;
}

__global__ void k_leaf_list(const int32_t *__restrict__ flag, const int32_t *__restrict__ fpos, int64_t n,
                            int32_t *__restrict__ leaves, SearchState *S) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (flag[v]) leaves[fpos[v]] = (int32_t)v;
    if (v == n - 1) S->nleaves = fpos[v] + flag[v];
}

__global__ void k_edges_from_parent(const int32_t *__restrict__ parent, const int32_t *__restrict__ pos,
                                    int64_t n, int32_t *__restrict__ eu, int32_t *__restrict__ ev) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t u = parent[v];
    if (u >= 0) {
        eu[pos[v]] = (int32_t)v;
        ev[pos[v]] = u;
    }
}

__global__ void k_nonroot_flags(const int32_t *__restrict__ parent, int64_t n, int32_t *__restrict__ flag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flag[v] = parent[v] >= 0 ? 1 : 0;
}

// Section 2.2 step 4: alpha_0, beta_0 and the thresholds of the first
// (bracketing) pass: 0, alpha_0, beta_0, beta_0 x 2^(2^j), DBL_MAX and 18
// points between alpha_0 and beta_0 on the bit-pattern scale.
__device__ void init_search(SearchState *S, double phs, double phm, double wsum, double wmin, double psum,
                            double pmin) {
    double alpha0 = (phm + pmin) / wsum;
    double beta0 = (phs + psum) / wmin;
    S->stats[0] = phs; S->stats[1] = phm; S->stats[2] = wsum; S->stats[3] = wmin;
    S->stats[4] = psum; S->stats[5] = pmin; S->stats[6] = alpha0; S->stats[7] = beta0;
    S->have_lo = 0; S->have_hi = 0; S->done = 0; S->error = 0; S->passes = 0;
    S->selected = 0; S->ik_bits = 0ull; S->beta = 0.0;
    S->lane_lo = -1; S->mode = 0; S->cand_passes = 0; S->ncand = 0u;
    const double DMAX = 1.7976931348623157e308;
    double b0 = (isfinite(beta0) && beta0 > 0.0) ? beta0 : 1.0;
    double a0 = (isfinite(alpha0) && alpha0 > 0.0) ? alpha0 : 0.0;
    double t[DP_LANES];
    t[0] = 0.0;
    t[1] = a0;
    t[2] = b0;
    double f = b0;
    const double mult[10] = {2.0, 2.0, 4.0, 16.0, 256.0, 65536.0, 4294967296.0, 1.8446744073709552e19,
                             3.402823669209385e38, 1.157920892373162e77};
    for (int q = 0; q < 10; ++q) {   // b0*2, *4, *16, *256, *2^16, ..., *2^512
        f = f * mult[q];
        t[3 + q] = isfinite(f) ? f : DMAX;
    }
    t[13] = DMAX;
    unsigned long long lb = dbits(a0), hb = dbits(b0);
    if (hb < lb) hb = lb;
    unsigned long long g = hb - lb;
    for (int q = 14; q < DP_LANES; ++q) {
        unsigned long long s = (unsigned long long)(q - 13);
        t[q] = bitsd(lb + (g / 19ull) * s + ((g % 19ull) * s) / 19ull);
    }
    for (int q = 0; q < DP_LANES; ++q) {
        S->thr[q] = t[q];
        S->cnt[q] = 0;
    }
}

// ------------------------------------------------------------ stats + search
// Section 2.2 step 4 / Section 3.5: phi*, phi_* over tree edges, omega*,
// omega_*, p*, p_* over the vertices; fixed reduction order (deterministic):
// STATS_BLOCKS blocks reduce contiguous ranges (coalesced loads, a fixed
// tree per block), then one block reduces their partials in block order.
__global__ void __launch_bounds__(256) k_stats_part(const int32_t *__restrict__ parent, const double *__restrict__ phi,
                                                    const double *__restrict__ omega, const double *__restrict__ p,
                                                    int64_t n, double *__restrict__ spart, uint32_t *st) {
    __shared__ double sh[6][256];
    const int tid = threadIdx.x;
    const int64_t chunk = ceil_div(n, STATS_BLOCKS);
    const int64_t a = (int64_t)blockIdx.x * chunk, b = min((int64_t)n, a + chunk);
    double fs = 0.0, fm = INFINITY, ws = 0.0, wm = INFINITY, ps = 0.0, pm = INFINITY;
    uint32_t bad = 0;
    for (int64_t v = a + tid; v < b; v += 256) {
        double w = omega[v];
        if (!(w > 0.0) || isinf(w)) bad |= (isnan(w) || isinf(w)) ? DEV_NONFINITE : DEV_NEGATIVE;
        ws = ws + w;
        wm = fmin(wm, w);
        double pv = p ? p[v] : 0.0;
        if (!(pv >= 0.0) || isinf(pv)) bad |= (isnan(pv) || isinf(pv)) ? DEV_NONFINITE : DEV_NEGATIVE;
        ps = ps + pv;
        pm = fmin(pm, pv);
        if (parent[v] >= 0) {
            double f = phi[v];
            if (!(f >= 0.0) || isinf(f)) bad |= (isnan(f) || isinf(f)) ? DEV_NONFINITE : DEV_NEGATIVE;
            fs = fs + f;
            fm = fmin(fm, f);
        }
    }
    if (bad) flag_status(st, bad);
    sh[0][tid] = fs; sh[1][tid] = fm; sh[2][tid] = ws; sh[3][tid] = wm; sh[4][tid] = ps; sh[5][tid] = pm;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) {
            sh[0][tid] = sh[0][tid] + sh[0][tid + s];
            sh[1][tid] = fmin(sh[1][tid], sh[1][tid + s]);
            sh[2][tid] = sh[2][tid] + sh[2][tid + s];
            sh[3][tid] = fmin(sh[3][tid], sh[3][tid + s]);
            sh[4][tid] = sh[4][tid] + sh[4][tid + s];
            sh[5][tid] = fmin(sh[5][tid], sh[5][tid + s]);
        }
        __syncthreads();
    }
    if (tid < 6) spart[(int64_t)blockIdx.x * 6 + tid] = sh[tid][0];
}

__global__ void __launch_bounds__(STATS_BLOCKS) k_stats_final(const double *__restrict__ spart, int64_t n,
                                                              SearchState *S) {
    __shared__ double sh[6][STATS_BLOCKS];
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 6; ++k) sh[k][tid] = spart[(int64_t)tid * 6 + k];
    __syncthreads();
    for (int s = STATS_BLOCKS / 2; s > 0; s >>= 1) {
        if (tid < s) {
            sh[0][tid] = sh[0][tid] + sh[0][tid + s];
            sh[1][tid] = fmin(sh[1][tid], sh[1][tid + s]);
            sh[2][tid] = sh[2][tid] + sh[2][tid + s];
            sh[3][tid] = fmin(sh[3][tid], sh[3][tid + s]);
            sh[4][tid] = sh[4][tid] + sh[4][tid + s];
            sh[5][tid] = fmin(sh[5][tid], sh[5][tid + s]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        double phs = sh[0][0], phm = n > 1 ? sh[1][0] : 0.0;
        double wsum = sh[2][0], wmin = sh[3][0], psum = sh[4][0], pmin = sh[5][0];
        init_search(S, phs, phm, wsum, wmin, psum, pmin);
    }
}

// Independent sets: one block per set b (vertices offs[b] .. offs[b+1]-1),
// the same statistics in a fixed reduction order.
__global__ void __launch_bounds__(256) k_stats_sets(const int32_t *__restrict__ parent, const double *__restrict__ phi,
                                                    const double *__restrict__ omega, const double *__restrict__ p,
                                                    const int64_t *__restrict__ offs, SearchState *SS, uint32_t *st) {
    __shared__ double sh[6][256];
    const int tid = threadIdx.x, b = blockIdx.x;
    const int64_t v0 = offs[b], v1 = offs[b + 1];
    double fs = 0.0, fm = INFINITY, ws = 0.0, wm = INFINITY, ps = 0.0, pm = INFINITY;
    uint32_t bad = 0;
    for (int64_t v = v0 + tid; v < v1; v += 256) {
        double w = omega[v];
        if (!(w > 0.0) || isinf(w)) bad |= (isnan(w) || isinf(w)) ? DEV_NONFINITE : DEV_NEGATIVE;
        ws = ws + w;
        wm = fmin(wm, w);
        double pv = p ? p[v] : 0.0;
        if (!(pv >= 0.0) || isinf(pv)) bad |= (isnan(pv) || isinf(pv)) ? DEV_NONFINITE : DEV_NEGATIVE;
        ps = ps + pv;
        pm = fmin(pm, pv);
        if (parent[v] >= 0) {
            double f = phi[v];
            if (!(f >= 0.0) || isinf(f)) bad |= (isnan(f) || isinf(f)) ? DEV_NONFINITE : DEV_NEGATIVE;
            fs = fs + f;
            fm = fmin(fm, f);
        }
    }
    if (bad) flag_status(st, bad);
    sh[0][tid] = fs; sh[1][tid] = fm; sh[2][tid] = ws; sh[3][tid] = wm; sh[4][tid] = ps; sh[5][tid] = pm;
    __syncthreads();
    for (int q = 128; q > 0; q >>= 1) {
        if (tid < q) {
            sh[0][tid] = sh[0][tid] + sh[0][tid + q];
            sh[1][tid] = fmin(sh[1][tid], sh[1][tid + q]);
            sh[2][tid] = sh[2][tid] + sh[2][tid + q];
            sh[3][tid] = fmin(sh[3][tid], sh[3][tid + q]);
            sh[4][tid] = sh[4][tid] + sh[4][tid + q];
            sh[5][tid] = fmin(sh[5][tid], sh[5][tid + q]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double phm = v1 - v0 > 1 ? sh[1][0] : 0.0;
        init_search(SS + b, sh[0][0], phm, sh[2][0], sh[3][0], sh[4][0], sh[5][0]);
    }
}

// The forest of independent sets is oriented as one tree under a virtual
// root; afterwards every set's own root (its first point) becomes a root.
__global__ void k_fix_roots(const int64_t *__restrict__ offs, int32_t nsets, int32_t *__restrict__ parent,
                            int32_t *__restrict__ edge_of) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsets) return;
    const int64_t r = offs[b];
    parent[r] = -1;
    edge_of[r] = -1;
}

// Algorithm 1 for 32 thresholds: one lane per threshold, one warp per walk.
struct DpArgs {
    int64_t n;
    const int32_t *parent, *ch_off, *ch_list, *leaves;
    const double *phi, *omega, *p;
    const int32_t *slot;           // v -> its child-list slot: the index of its states (one tree; null: by vertex)
    const double *phis;            // phi of each slot's parent edge
};

// One warp walks from leaf v towards the root, deciding each vertex for the
// 32 thresholds of its lanes; returns this lane's cuts.
// Folds the children [c0, c1) of a vertex into (w, pv) for this lane's
// threshold, in descending index: a joined child adds its omega-hat and
// p-hat, any other its parent edge's phi.  SLOT (one tree): the children's
// states sit in their slots c0 .. c1 - 1, no child-index round trip;
// otherwise (independent sets) they are indexed by vertex, through the child
// list.  Up to DP_FEW children are loaded in one round (a walk's steps are
// latency-bound), more are folded one by one.
constexpr int DP_FEW = 4;
template <bool SLOT>
__device__ __forceinline__ void dp_fold_children(const DpArgs &A, int32_t c0, int32_t c1, int lane,
                                                 const uint8_t *__restrict__ dec, const double *__restrict__ wh,
                                                 const double *__restrict__ ph, double &w, double &pv) {
    const int32_t nc = c1 - c0;
    if (nc <= DP_FEW) {
        int32_t ch[DP_FEW];
        if constexpr (!SLOT) {
#pragma unroll
            for (int q = 0; q < DP_FEW; ++q) ch[q] = q < nc ? A.ch_list[c0 + q] : 0;
        }
        uint8_t dcv[DP_FEW];
        double cw[DP_FEW], cp[DP_FEW], cf[DP_FEW];
#pragma unroll
        for (int q = 0; q < DP_FEW; ++q) {
            dcv[q] = DEC_DISCARD;
            cw[q] = cp[q] = cf[q] = 0.0;
            if (q < nc) {
                const size_t cl = (size_t)(SLOT ? c0 + q : ch[q]) * DP_LANES + lane;
                dcv[q] = ld_cg_u8(dec + cl);
                cw[q] = ld_cg_f64(wh + cl);
                cp[q] = ld_cg_f64(ph + cl);
                cf[q] = SLOT ? A.phis[c0 + q] : A.phi[ch[q]];
            }
        }
#pragma unroll
        for (int q = DP_FEW - 1; q >= 0; --q) {       // siblings in descending index
            if (q < nc) {
                if (dcv[q] == DEC_JOIN) {
                    w = __dadd_rn(w, cw[q]);
                    pv = __dadd_rn(pv, cp[q]);
                } else {
                    pv = __dadd_rn(pv, cf[q]);          // cut or discarded child: boundary edge
                }
            }
        }
    } else {
        for (int32_t q = c1 - 1; q >= c0; --q) {       // siblings in descending index
            const int32_t c = SLOT ? q : A.ch_list[q];
            const size_t cl = (size_t)c * DP_LANES + lane;
            const uint8_t dc = ld_cg_u8(dec + cl);
            if (dc == DEC_JOIN) {
                w = __dadd_rn(w, ld_cg_f64(wh + cl));
                pv = __dadd_rn(pv, ld_cg_f64(ph + cl));
            } else {
                pv = __dadd_rn(pv, SLOT ? A.phis[q] : A.phi[c]);
            }
        }
    }
}

// The hand-off between the warps of sibling walks is message passing: a
// warp's states are written, then (release fence) its arrival is counted;
// the last arrival (acquire fence) reads them all.  Acquire-release fences at
// GPU scope order exactly that.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// One warp walks from leaf v towards the root, deciding each vertex for the
// 32 thresholds of its lanes; returns this lane's cuts.
__device__ __forceinline__ int dp_walk_tree(const DpArgs &A, int32_t v, double N, int lane, int final_pass,
                                       uint8_t *__restrict__ dec, double *__restrict__ wh, double *__restrict__ ph,
                                       int32_t *__restrict__ done, double *__restrict__ rat) {
    // The walk's critical path is the tree's longest chain of handoffs, and
    // each step's memory round trips are its latency: the children are folded
    // in two rounds of loads (dp_fold_children); the parent's child range is
    // fetched with the vertex's own data.
    int cuts = 0;
    while (true) {
        const int32_t c0 = A.ch_off[v], c1 = A.ch_off[v + 1];
        const int32_t u = A.parent[v];
        const int32_t sv = A.slot[v];
        double w = A.omega[v];
        double pv = A.p ? A.p[v] : 0.0;
        const double phv = A.phi[v];
        const int32_t uc0 = u >= 0 ? A.ch_off[u] : 0, uc1 = u >= 0 ? A.ch_off[u + 1] : 0;
        dp_fold_children<true>(A, c0, c1, lane, dec, wh, ph, w, pv);
        const double fe = u >= 0 ? phv : 0.0;
        const double nw = __dmul_rn(N, w);
        const double fp = __dadd_rn(fe, pv);
        uint8_t d;
        if (fp <= nw) {
            d = DEC_CUT;
            ++cuts;
            if (final_pass && lane == 0) rat[v] = __ddiv_rn(fp, w);
        } else if (u >= 0 && __dsub_rn(pv, fe) < nw) {
            d = DEC_JOIN;
        } else {
            d = DEC_DISCARD;
        }
        const size_t vl = (size_t)sv * DP_LANES + lane;
        dec[vl] = d;
        wh[vl] = w;
        ph[vl] = pv;
        if (u < 0) break;
        const int32_t nu = uc1 - uc0;
        if (nu == 1) { v = u; continue; }          // only child: no one to wait for
        fence_acq_rel_gpu();
        __syncwarp();
        int old = 0;
        if (lane == 0) old = atomicAdd(done + u, 1);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old != nu - 1) break;                  // a sibling is still running
        fence_acq_rel_gpu();
        v = u;
    }
    return cuts;
}

// The same walk for the independent sets' pass, which has millions of short
// walks in flight: a vertex's own data (its child range, parent, omega, p,
// phi of its parent edge) does not change during a pass, so the parent's is
// loaded while the current vertex's children are folded.  (One large tree's
// pass is bound by its longest walk and measured faster with dp_walk_tree.)
__device__ __forceinline__ int dp_walk_sets(const DpArgs &A, int32_t v, double N, int lane, int final_pass,
                                       uint8_t *__restrict__ dec, double *__restrict__ wh, double *__restrict__ ph,
                                       int32_t *__restrict__ done, double *__restrict__ rat) {
    int cuts = 0;
    int32_t c0 = A.ch_off[v], c1 = A.ch_off[v + 1];
    int32_t u = A.parent[v];
    double w0 = A.omega[v];
    double p0 = A.p ? A.p[v] : 0.0;
    double fe = u >= 0 ? A.phi[v] : 0.0;
    while (true) {
        int32_t uc0 = 0, uc1 = 0, uu = -1;
        double uw = 0.0, up = 0.0, ufe = 0.0;
        if (u >= 0) {
            uc0 = A.ch_off[u];
            uc1 = A.ch_off[u + 1];
            uu = A.parent[u];
            uw = A.omega[u];
            up = A.p ? A.p[u] : 0.0;
            ufe = A.phi[u];
        }
        double w = w0, pv = p0;
        dp_fold_children<false>(A, c0, c1, lane, dec, wh, ph, w, pv);
        const double nw = __dmul_rn(N, w);
        const double fp = __dadd_rn(fe, pv);
        uint8_t d;
        if (fp <= nw) {
            d = DEC_CUT;
            ++cuts;
            if (final_pass && lane == 0) rat[v] = __ddiv_rn(fp, w);
        } else if (u >= 0 && __dsub_rn(pv, fe) < nw) {
            d = DEC_JOIN;
        } else {
            d = DEC_DISCARD;
        }
        const size_t vl = (size_t)v * DP_LANES + lane;
        dec[vl] = d;
        wh[vl] = w;
        ph[vl] = pv;
        if (u < 0) break;
        const int32_t nu = uc1 - uc0;
        if (nu != 1) {                             // an only child has no one to wait for
            fence_acq_rel_gpu();
            __syncwarp();
            int old = 0;
            if (lane == 0) old = atomicAdd(done + u, 1);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old != nu - 1) break;              // a sibling is still running
            fence_acq_rel_gpu();
        }
        v = u;
        c0 = uc0;
        c1 = uc1;
        u = uu;
        w0 = uw;
        p0 = up;
        fe = uu >= 0 ? ufe : 0.0;
    }
    return cuts;
}

__global__ void __launch_bounds__(256) k_dp_pass(DpArgs A, SearchState *S, uint8_t *__restrict__ dec,
                                                 double *__restrict__ wh, double *__restrict__ ph,
                                                 int32_t *__restrict__ done, double *__restrict__ rat,
                                                 int final_pass) {
    if (!final_pass && S->done) return;
    if (final_pass && S->final_lane >= 0) return;      // k_final_from_lane serves
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double N = final_pass ? S->beta : S->thr[lane];
    const int nleaves = S->nleaves;
    int cuts = 0;
    for (int64_t li = warp; li < nleaves; li += nwarps)
        cuts += dp_walk_tree(A, A.leaves[li], N, lane, final_pass, dec, wh, ph, done, rat);
    if (cuts) atomicAdd(&S->cnt[lane], cuts);
}

// Independent sets (a forest whose trees are the sets): each set has its own
// search state and thresholds.  A warp takes a contiguous run of leaves, so
// its cut counts change set rarely and are flushed at each change.
__global__ void __launch_bounds__(256) k_dp_pass_sets(DpArgs A, const SearchState *G, SearchState *SS,
                                                      const int32_t *__restrict__ vset, uint8_t *__restrict__ dec,
                                                      double *__restrict__ wh, double *__restrict__ ph,
                                                      int32_t *__restrict__ done, double *__restrict__ rat,
                                                      int final_pass, const uint32_t *__restrict__ left) {
    if (!final_pass && *(const volatile uint32_t *)left == 0u) return;     // every set's search is done
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nleaves = G->nleaves;
    const int64_t chunk = (nleaves + nwarps - 1) / nwarps;
    const int64_t l0 = warp * chunk, l1 = min(nleaves, l0 + chunk);
    int32_t cur = -1;
    int cuts = 0;
    for (int64_t li = l0; li < l1; ++li) {
        const int32_t v = A.leaves[li];
        const int32_t b = vset[v];
        if (b != cur) {
            if (cuts) atomicAdd(&SS[cur].cnt[lane], cuts);
            cuts = 0;
            cur = b;
        }
        const SearchState *S = SS + b;
        if (!final_pass && S->done) continue;
        const double N = final_pass ? S->beta : S->thr[lane];
        cuts += dp_walk_sets(A, v, N, lane, final_pass, dec, wh, ph, done, rat);
    }
    if (cuts) atomicAdd(&SS[cur].cnt[lane], cuts);
}

__device__ void search_update(SearchState *S, int32_t k, int last, uint32_t *st) {
    if (S->done) return;
    const unsigned long long NONE = ~0ull;
    unsigned long long hi = S->have_hi ? S->hi_bits : NONE;
    for (int t = 0; t < DP_LANES; ++t)
        if (S->cnt[t] >= k && dbits(S->thr[t]) < hi) hi = dbits(S->thr[t]);
    S->passes += 1;
    if (hi == NONE) {
        S->error = 1;
        S->done = 1;
        flag_status(st, DEV_NO_SOLUTION);
        return;
    }
    bool have_lo = S->have_lo;
    unsigned long long lo = S->lo_bits;
    int lane_lo = -1;
    for (int t = 0; t < DP_LANES; ++t) {
        unsigned long long b = dbits(S->thr[t]);
        if (S->cnt[t] < k && b < hi && (!have_lo || b > lo)) { lo = b; have_lo = true; lane_lo = t; }
    }
    if (lane_lo < 0 && have_lo)          // lo unchanged: a lane that re-evaluated it
        for (int t = 0; t < DP_LANES; ++t)
            if (S->cnt[t] < k && dbits(S->thr[t]) == lo) { lane_lo = t; break; }
    S->lane_lo = lane_lo;
    S->hi_bits = hi; S->have_hi = 1;
    S->lo_bits = lo; S->have_lo = have_lo ? 1 : 0;
    for (int t = 0; t < DP_LANES; ++t) S->cnt[t] = 0;
    if (hi == 0ull || (have_lo && hi - lo <= 1ull)) {
        S->done = 1;
        S->beta = bitsd(hi);
        return;
    }
    if (!have_lo) {   // 0.0 is always tried in the first pass; cannot happen
        S->error = 1;
        S->done = 1;
        flag_status(st, DEV_INTERNAL);
        return;
    }
    if (last) {
        S->done = 1;
        S->beta = bitsd(hi);
        flag_status(st, DEV_INTERNAL);
        return;
    }
    unsigned long long g = hi - lo;
    for (int t = 1; t <= DP_LANES; ++t) {
        unsigned long long s = (unsigned long long)t;
        S->thr[t - 1] = bitsd(lo + (g / 33ull) * s + ((g % 33ull) * s) / 33ull);
    }
}

__global__ void k_search_update(SearchState *S, int32_t k, int last, uint32_t *st) {
    if (threadIdx.x == 0) search_update(S, k, last, st);
}

// ---- thresholds from critical ratios (one tree).  As N grows from lo, the
// first decision of Algorithm 1 to change is that of a vertex whose
// descendants keep theirs, so it changes where N reaches the vertex's own
// critical ratio in lo's state: (phi(e) + p-hat) / omega-hat for the cut
// test, (p-hat - phi(e)) / omega-hat for the join test.  The ratios inside
// the bracket (lo, hi) of every vertex, read from the lane that evaluated lo
// in the last pass, are counted per bucket of the bracket's bit patterns;
// the next pass splits them into 32 groups of equal count (or, when at most
// CAND_EXACT remain, tries each of them and its neighbouring doubles).  Any
// threshold inside the bracket keeps the search correct (the bracket only
// shrinks); these choices only make it shorter.  lo itself is re-evaluated
// in lane 0 so that its state is always available.
__device__ __forceinline__ int cand_bucket(unsigned long long b, unsigned long long lo, double inv_w) {
    int j = (int)((double)(b - lo) * inv_w);
    return j < 0 ? 0 : (j >= CAND_BUCKETS ? CAND_BUCKETS - 1 : j);
}

__device__ __forceinline__ bool cand_active(const SearchState *S) {
    return !S->done && S->mode == 0 && S->lane_lo >= 0 && S->cand_passes < DP_CAND_PASSES;
}

__global__ void __launch_bounds__(256) k_cand_hist(DpArgs A, SearchState *S, const double *__restrict__ wh,
                                                   const double *__restrict__ ph, uint32_t *__restrict__ hist) {
    if (!cand_active(S)) return;
    const unsigned long long lo = S->lo_bits, hi = S->hi_bits;
    const int L = S->lane_lo;
    const double inv_w = (double)CAND_BUCKETS / (double)(hi - lo);
    auto add = [&](double c) {
        const unsigned long long b = dbits(c);
        if (!(c > 0.0) || b <= lo || b >= hi) return;
        atomicAdd(hist + cand_bucket(b, lo, inv_w), 1u);
        const unsigned q = atomicAdd(&S->ncand, 1u);
        if (q < (unsigned)CAND_EXACT) S->cand[q] = b;
    };
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gs) {
        const size_t vl = (size_t)A.slot[v] * DP_LANES + L;
        const double w = wh[vl], pv = ph[vl];
        const int32_t u = A.parent[v];
        const double fe = u >= 0 ? A.phi[v] : 0.0;
        add(__ddiv_rn(__dadd_rn(fe, pv), w));
        if (u >= 0) add(__ddiv_rn(__dsub_rn(pv, fe), w));
    }
}

// One block: the next pass's thresholds (lane 0 = lo), or the switch to the
// 33-ary bit search already written by k_search_update.
__global__ void __launch_bounds__(1024) k_cand_select(SearchState *S, uint32_t *__restrict__ hist) {
    __shared__ unsigned int pre[CAND_BUCKETS];
    __shared__ unsigned int warp_sum[32];
    __shared__ int active;
    const int tid = threadIdx.x;
    if (tid == 0) active = cand_active(S) ? 1 : 0;
    __syncthreads();
    if (!active) {
        if (tid == 0 && !S->done) S->mode = 1;       // k_search_update's bit-search thresholds stand
        for (int j = tid; j < CAND_BUCKETS; j += blockDim.x) hist[j] = 0u;
        return;
    }
    // inclusive prefix sums of the buckets: 4 per thread, then across threads
    constexpr int PER = CAND_BUCKETS / 1024;
    unsigned int loc[PER], run = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) { run += hist[tid * PER + q]; loc[q] = run; }
    const int lane = tid & 31, wp = tid >> 5;
    unsigned int x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wp] = x;
    __syncthreads();
    if (wp == 0) {
        unsigned int z = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        warp_sum[lane] = z;
    }
    __syncthreads();
    const unsigned int before = (x - run) + (wp > 0 ? warp_sum[wp - 1] : 0u);
#pragma unroll
    for (int q = 0; q < PER; ++q) pre[tid * PER + q] = before + loc[q];
    __syncthreads();
    for (int j = tid; j < CAND_BUCKETS; j += blockDim.x) hist[j] = 0u;     // ready for the next pass
    if (tid != 0) return;
    const unsigned long long lo = S->lo_bits, hi = S->hi_bits;
    const unsigned int m = pre[CAND_BUCKETS - 1];
    const unsigned int nc = S->ncand;
    S->ncand = 0u;
    double t[DP_LANES];
    t[0] = bitsd(lo);
    int used = 1;
    if (hi - lo <= (unsigned long long)DP_LANES) {
        // every double of the bracket
        for (int q = 1; q < DP_LANES; ++q) t[q] = bitsd(lo + (unsigned long long)q < hi ? lo + q : hi);
        used = DP_LANES;
    } else if (m == 0u) {
        S->mode = 1;                                  // nothing to aim at: bit search
        return;
    } else if (nc <= (unsigned)CAND_EXACT) {
        // each remaining critical ratio and its neighbouring doubles
        for (unsigned q = 0; q < nc && used + 3 <= DP_LANES; ++q) {
            const unsigned long long b = S->cand[q];
            const unsigned long long c[3] = {b - 1ull, b, b + 1ull};
            for (int r = 0; r < 3; ++r)
                if (c[r] > lo && c[r] < hi) t[used++] = bitsd(c[r]);
        }
    } else {
        // 31 thresholds splitting the ratios into groups of equal count
        const double wdt = (double)(hi - lo) / (double)CAND_BUCKETS;
        int j = 0;
        for (int q = 1; q < DP_LANES; ++q) {
            const unsigned long long r = ((unsigned long long)m * (unsigned long long)q) / DP_LANES;
            while (j < CAND_BUCKETS - 1 && pre[j] < r) ++j;
            unsigned long long b = lo + (unsigned long long)((double)(j + 1) * wdt);
            if (b <= lo) b = lo + 1ull;
            if (b >= hi) b = hi - 1ull;
            t[used++] = bitsd(b);
        }
    }
    for (int q = used; q < DP_LANES; ++q) t[q] = t[used - 1];
    // a spare lane re-evaluates hi: when the search ends after this pass,
    // beta's state is then among the pass's lanes (no final pass needed)
    if (used < DP_LANES) t[DP_LANES - 1] = bitsd(hi);
    for (int q = 0; q < DP_LANES; ++q) S->thr[q] = t[q];
    S->cand_passes += 1;
}

// After the search (one tree): the lane of the last pass that evaluated beta
// itself, if any.  Its decisions and omega-hat / p-hat are those of the
// final call of Algorithm 1 at beta, so k_final_from_lane copies them to
// lane 0 (and forms the cut ratios) instead of another pass.
__global__ void k_final_lane(SearchState *S) {
    if (threadIdx.x != 0) return;
    S->final_lane = -1;
    if (S->error || !S->done) return;
    const unsigned long long b = dbits(S->beta);
    for (int t = 0; t < DP_LANES; ++t)
        if (dbits(S->thr[t]) == b) { S->final_lane = t; return; }
}

__global__ void k_final_from_lane(const SearchState *__restrict__ S, const int32_t *__restrict__ parent,
                                  const double *__restrict__ phi, const int32_t *__restrict__ slot, int64_t n,
                                  uint8_t *__restrict__ dec, const double *__restrict__ wh,
                                  const double *__restrict__ ph, double *__restrict__ rat) {
    const int L = S->final_lane;
    if (L < 0) return;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const size_t s0 = (size_t)slot[v] * DP_LANES, vl = s0 + L;
    const uint8_t d = dec[vl];
    dec[s0] = d;
    if (d == DEC_CUT) {
        // the same operations as the pass at beta: fp = phi(e) + p-hat, fp / omega-hat
        const int32_t u = parent[v];
        const double fe = u >= 0 ? phi[v] : 0.0;
        rat[v] = __ddiv_rn(__dadd_rn(fe, ph[vl]), wh[vl]);
    }
}

// ---- the same for independent sets: each set in candidate mode counts its
// vertices' critical ratios in CAND_SET_BUCKETS buckets of its own bracket
// (hist [nsets][CAND_SET_BUCKETS]); one warp per set then picks its next
// thresholds exactly as k_cand_select does for one tree.
__global__ void __launch_bounds__(256) k_cand_hist_sets(DpArgs A, SearchState *SS, const int32_t *__restrict__ vset,
                                                        int64_t nv, const double *__restrict__ wh,
                                                        const double *__restrict__ ph, uint32_t *__restrict__ hist,
                                                        const uint32_t *__restrict__ left) {
    if (*(const volatile uint32_t *)left == 0u) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gs) {
        const int32_t b = vset[v];
        SearchState *S = SS + b;
        if (!cand_active(S)) continue;
        const unsigned long long lo = S->lo_bits, hi = S->hi_bits;
        const int L = S->lane_lo;
        const double inv_w = (double)CAND_SET_BUCKETS / (double)(hi - lo);
        uint32_t *hb = hist + (size_t)b * CAND_SET_BUCKETS;
        auto add = [&](double c) {
            const unsigned long long bits = dbits(c);
            if (!(c > 0.0) || bits <= lo || bits >= hi) return;
            int j = (int)((double)(bits - lo) * inv_w);
            j = j < 0 ? 0 : (j >= CAND_SET_BUCKETS ? CAND_SET_BUCKETS - 1 : j);
            atomicAdd(hb + j, 1u);
            const unsigned q = atomicAdd(&S->ncand, 1u);
            if (q < (unsigned)CAND_EXACT) S->cand[q] = bits;
        };
        const size_t vl = (size_t)v * DP_LANES + L;
        const double w = wh[vl], pv = ph[vl];
        const int32_t u = A.parent[v];
        const double fe = u >= 0 ? A.phi[v] : 0.0;
        add(__ddiv_rn(__dadd_rn(fe, pv), w));
        if (u >= 0) add(__ddiv_rn(__dsub_rn(pv, fe), w));
    }
}

__global__ void __launch_bounds__(256) k_cand_select_sets(SearchState *SS, int32_t nsets, uint32_t *__restrict__ hist,
                                                          const uint32_t *__restrict__ left) {
    if (*(const volatile uint32_t *)left == 0u) return;
    __shared__ unsigned int pre_s[8][CAND_SET_BUCKETS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nsets) return;
    SearchState *S = SS + b;
    uint32_t *hb = hist + (size_t)b * CAND_SET_BUCKETS;
    unsigned int *pre = pre_s[wib];
    const bool active = cand_active(S);
    // inclusive prefix sums of the set's buckets: CAND_SET_BUCKETS / 32 per lane
    constexpr int PER = CAND_SET_BUCKETS / 32;
    unsigned int loc[PER], run = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) { run += hb[lane * PER + q]; loc[q] = run; }
    unsigned int x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        pre[lane * PER + q] = (x - run) + loc[q];
        hb[lane * PER + q] = 0u;                      // ready for the next pass
    }
    __syncwarp();
    if (lane != 0) return;
    if (!active) {
        if (!S->done) S->mode = 1;                    // k_search_update_sets's bit-search thresholds stand
        return;
    }
    const unsigned long long lo = S->lo_bits, hi = S->hi_bits;
    const unsigned int m = pre[CAND_SET_BUCKETS - 1];
    const unsigned int nc = S->ncand;
    S->ncand = 0u;
    double t[DP_LANES];
    t[0] = bitsd(lo);
    int used = 1;
    if (hi - lo <= (unsigned long long)DP_LANES) {
        for (int q = 1; q < DP_LANES; ++q) t[q] = bitsd(lo + (unsigned long long)q < hi ? lo + q : hi);
        used = DP_LANES;
    } else if (m == 0u) {
        S->mode = 1;
        return;
    } else if (nc <= (unsigned)CAND_EXACT) {
        for (unsigned q = 0; q < nc && used + 3 <= DP_LANES; ++q) {
            const unsigned long long c0 = S->cand[q];
            const unsigned long long c[3] = {c0 - 1ull, c0, c0 + 1ull};
            for (int r = 0; r < 3; ++r)
                if (c[r] > lo && c[r] < hi) t[used++] = bitsd(c[r]);
        }
    } else {
        const double wdt = (double)(hi - lo) / (double)CAND_SET_BUCKETS;
        int j = 0;
        for (int q = 1; q < DP_LANES; ++q) {
            const unsigned long long r = ((unsigned long long)m * (unsigned long long)q) / DP_LANES;
            while (j < CAND_SET_BUCKETS - 1 && pre[j] < r) ++j;
            unsigned long long c = lo + (unsigned long long)((double)(j + 1) * wdt);
            if (c <= lo) c = lo + 1ull;
            if (c >= hi) c = hi - 1ull;
            t[used++] = bitsd(c);
        }
    }
    for (int q = used; q < DP_LANES; ++q) t[q] = t[used - 1];
    for (int q = 0; q < DP_LANES; ++q) S->thr[q] = t[q];
    S->cand_passes += 1;
}

// independent sets: one thread per set
// (left: the sets whose search is not done; the passes after the last one
// finishes return at once)
__global__ void k_search_update_sets(SearchState *SS, const int32_t *__restrict__ ks, int32_t nsets, int last,
                                     uint32_t *st, uint32_t *left) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsets) return;
    const int was = SS[b].done;
    search_update(SS + b, ks[b], last, st);
    if (!was && SS[b].done) atomicSub(left, 1u);
}

__global__ void k_sets_left_init(uint32_t *left, int32_t nsets) { *left = (uint32_t)nsets; }

// ------------------------------------------------------------ labels
__global__ void k_head_init(const uint8_t *__restrict__ dec, const int32_t *__restrict__ slot,
                            const int32_t *__restrict__ parent, int64_t n, int32_t *__restrict__ head) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) head[v] = dec[(size_t)(slot ? slot[v] : (int32_t)v) * DP_LANES] == DEC_JOIN ? parent[v] : (int32_t)v;
}

__global__ void k_head_jump(const int32_t *__restrict__ hin, int32_t *__restrict__ hout, int64_t n) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) hout[v] = hin[hin[v]];
}

__global__ void k_cut_flags(const uint8_t *__restrict__ dec, const int32_t *__restrict__ slot,
                            const int32_t *__restrict__ bfs_pos, int64_t n, int32_t *__restrict__ cflag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) cflag[n - 1 - bfs_pos[v]] = dec[(size_t)(slot ? slot[v] : (int32_t)v) * DP_LANES] == DEC_CUT ? 1 : 0;
}

__global__ void k_labels(const uint8_t *__restrict__ dec, const int32_t *__restrict__ slot,
                         const int32_t *__restrict__ bfs_pos,
                         const int32_t *__restrict__ head, const int32_t *__restrict__ cidx,
                         const double *__restrict__ rat, int64_t n, int32_t k, int32_t *__restrict__ labels,
                         uint8_t *__restrict__ residual, SearchState *S) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t h = head[v];
    int32_t c = dec[(size_t)slot[h] * DP_LANES] == DEC_CUT ? cidx[n - 1 - bfs_pos[h]] : -1;
    int32_t lab = (c >= 0 && c < k) ? c : -1;
    labels[v] = lab;
    residual[v] = lab < 0 ? 1 : 0;
    if (dec[(size_t)slot[v] * DP_LANES] == DEC_CUT) {
        int32_t cv = cidx[n - 1 - bfs_pos[v]];
        if (cv < k) {
            atomicMax(&S->ik_bits, dbits(rat[v]));
            atomicAdd(&S->selected, 1);
        }
    }
}

__global__ void k_finish(SearchState *S, int32_t k, double *i_k, uint32_t *st) {
    if (threadIdx.x != 0) return;
    if (S->error) return;
    if (S->selected != k) flag_status(st, DEV_INTERNAL);
    i_k[0] = bitsd(S->ik_bits);
}

// Independent sets: processing positions are set-major (sets in descending
// order, the virtual root last), so set b's cuts are counted from position
// nv - offs[b+1] (nv = number of real vertices).
__global__ void k_labels_sets(const uint8_t *__restrict__ dec, const int32_t *__restrict__ bfs_pos,
                              const int32_t *__restrict__ head, const int32_t *__restrict__ cidx,
                              const double *__restrict__ rat, int64_t nv, const int32_t *__restrict__ vset,
                              const int64_t *__restrict__ offs, const int32_t *__restrict__ ks,
                              int32_t *__restrict__ labels, uint8_t *__restrict__ residual, SearchState *SS) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int32_t b = vset[v];
    const int32_t base = cidx[nv - offs[b + 1]];
    const int32_t k = ks[b];
    const int32_t h = head[v];
    const int32_t c = dec[(size_t)h * DP_LANES] == DEC_CUT ? cidx[nv - bfs_pos[h]] - base : -1;
    const int32_t lab = (c >= 0 && c < k) ? c : -1;
    labels[v] = lab;
    residual[v] = lab < 0 ? 1 : 0;
    if (dec[(size_t)v * DP_LANES] == DEC_CUT) {
        const int32_t cv = cidx[nv - bfs_pos[v]] - base;
        if (cv < k) {
            atomicMax(&SS[b].ik_bits, dbits(rat[v]));
            atomicAdd(&SS[b].selected, 1);
        }
    }
}

__global__ void k_finish_sets(SearchState *SS, const int32_t *__restrict__ ks, int32_t nsets, double *i_k,
                              double *beta, uint32_t *st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsets) return;
    const SearchState *S = SS + b;
    if (S->error) return;
    if (S->selected != ks[b]) flag_status(st, DEV_INTERNAL);
    i_k[b] = bitsd(S->ik_bits);
    if (beta) beta[b] = S->beta;
}

// BFS keys of independent sets: a stable second sort by set makes the order
// set-major with (depth, preorder) inside each set; the virtual root first.
__global__ void k_set_keys(const int32_t *__restrict__ ib, const int32_t *__restrict__ vset, int64_t n,
                           int64_t nv, uint64_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = ib[i];
    keys[i] = v < nv ? (uint64_t)(vset[v] + 1) : 0ull;
}

__global__ void k_phi_from_edges(const int32_t *__restrict__ edge_of, const double *__restrict__ ed2,
                                 int64_t n, double sigma, double *__restrict__ phi) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t e = edge_of[v];
    if (e < 0) { phi[v] = 0.0; return; }
    double dist = __dsqrt_rn(ed2[e]);
    double y = __ddiv_rn(dist, sigma);
    phi[v] = exp(-y);
}

__global__ void k_omega_tree(const uint64_t *__restrict__ adj_key, const int32_t *__restrict__ adj_off,
                             const int32_t *__restrict__ parent, const double *__restrict__ phi, int64_t n,
                             int32_t include_self, double *__restrict__ omega) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double s = include_self ? 1.0 : 0.0;
    for (int32_t i = adj_off[v]; i < adj_off[v + 1]; ++i) {
        int32_t w = (int32_t)(adj_key[i] & 0xffffffffu);
        double f = parent[v] == w ? phi[v] : phi[w];
        s = __dadd_rn(s, f);
    }
    omega[v] = s;
}

}  // namespace

// ---------------------------------------------------------------- host side
cudaError_t orient_tree(TreeScratch &S, const int32_t *eu, const int32_t *ev, int64_t n, int32_t root,
                        const int32_t *expect_parent, cudaStream_t s, const int32_t *vset, int part) {
    TreeDev &T = S.T;
    T.n = n;
    T.root = root;
    cudaError_t e;
    if (n == 1) {
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.parent, 1, -1);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.edge_of, 1, -1);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.bfs_pos, 1, 0);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.ch_off, 2, 0);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.adj_off, 2, 0);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.leaves, 1, 0);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.depth, 1, 0);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(T.slot, 1, 0);
        k_fill_i32<<<1, 32, 0, ISO_S(s)>>>(S.pre, 1, 0);
        T.pre = S.pre;
        SearchState *SS = S.search;
        int one = 1, zero = 0;
        if ((e = cudaMemcpyAsync(&SS->nleaves, &one, sizeof(int), cudaMemcpyHostToDevice, s))) return e;
        if ((e = cudaMemcpyAsync(&SS->max_depth, &zero, sizeof(int), cudaMemcpyHostToDevice, s))) return e;
        return cudaStreamSynchronize(s);
    }
    const int64_t m = n - 1, M = 2 * m;
    const int L = log2_ceil(M) + 1;
    // the ranks end in rnk after an even number of Wyllie steps, else rnk2
    int32_t *ra = (L % 2 == 0) ? S.rnk : S.rnk2;
    if (part != 2) {
        k_dir_keys<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(eu, ev, m, n, T.adj_key, S.vals, S.status);
        if ((e = sort_pairs_u64(T.adj_key, S.vals, S.kbuf, S.vbuf, M, s))) return e;
        k_fill_i32<<<blocks_for(n + 1), TPB, 0, ISO_S(s)>>>(T.adj_off, n + 1, -1);
        k_adj_off<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(T.adj_key, M, n, T.adj_off, S.status);
        k_check_adj<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(T.adj_off, n, S.status);
        k_rev_succ<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(T.adj_key, T.adj_off, M, n, S.rev, S.succ, S.status);
        k_break_tour<<<1, 1, 0, ISO_S(s)>>>(T.adj_off, S.rev, S.succ, root, M, S.status);
        k_fill_i32<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(S.rnk, M, 1);
        int32_t *sa = S.succ, *sb = S.succ2, *rk = S.rnk, *rb = S.rnk2;
        for (int it = 0; it < L; ++it) {
            k_wyllie<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(sa, rk, sb, rb, M);
            int32_t *t = sa; sa = sb; sb = t;
            t = rk; rk = rb; rb = t;
        }
        k_check_ranked<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(sa, rk, M, S.status);
        if (part == 1) return cudaGetLastError();
        uint32_t hst = 0;
        if ((e = cudaMemcpyAsync(&hst, S.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        if (hst & DEV_BAD_TREE) return cudaSuccess;   // caller reads the status word
    }

    k_orient<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(T.adj_key, S.vals, S.rev, ra, M, n, root, T.parent, S.size, T.edge_of,
                                           S.flag);
    if (expect_parent) k_check_parent<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(T.parent, expect_parent, n, S.status);
    if ((e = exclusive_scan_i32(S.flag, S.fpos, M, S.tmp32, s))) return e;
    k_scan_total<<<1, 1, 0, ISO_S(s)>>>(S.flag, S.fpos, M);
    k_children<<<blocks_for(M), TPB, 0, ISO_S(s)>>>(T.adj_key, S.flag, S.fpos, M, T.ch_list);
    k_slots<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(T.ch_list, n, root, T.slot);
    k_ch_off<<<blocks_for(n + 1), TPB, 0, ISO_S(s)>>>(T.adj_off, S.fpos, n, T.ch_off);
    k_child_sizes<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(T.ch_list, S.size, m, S.ssz);
    if ((e = exclusive_scan_i64(S.ssz, S.sx, m, S.tmp64, s))) return e;
    k_pre_init<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(T.parent, T.ch_off, T.ch_list, S.sx, m, root, S.anc, T.depth, S.pre);
    int32_t *aa = S.anc, *ab = S.anc2, *da = T.depth, *db = S.dep2, *pa = S.pre, *pb = S.pre2;
    const int Ln = log2_ceil(n) + 1;
    for (int it = 0; it < Ln; ++it) {
        k_jump_acc<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(aa, da, pa, ab, db, pb, n);
        int32_t *t = aa; aa = ab; ab = t;
        t = da; da = db; db = t;
        t = pa; pa = pb; pb = t;
    }
    if (da != T.depth) {
        if ((e = cudaMemcpyAsync(T.depth, da, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s))) return e;
    }
    T.pre = pa;
    k_bfs_keys<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(T.depth, pa, n, S.bkeys, S.ib);
    if ((e = sort_pairs_u64(S.bkeys, S.ib, S.kbuf, S.vbuf, n, s))) return e;
    if (vset) {
        // independent sets under a virtual root (vertex n - 1): set-major order
        k_set_keys<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.ib, vset, n, n - 1, S.bkeys);
        if ((e = sort_pairs_u64(S.bkeys, S.ib, S.kbuf, S.vbuf, n, s))) return e;
    }
    k_bfs_pos<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.ib, S.bkeys, n, T.bfs_pos, S.search);
    k_leaf_flags<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(T.ch_off, n, S.flag);
    if ((e = exclusive_scan_i32(S.flag, S.fpos, n, S.tmp32, s))) return e;
    k_leaf_list<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.flag, S.fpos, n, T.leaves, S.search);
    return cudaGetLastError();
}

cudaError_t edges_from_parent(TreeScratch &S, const int32_t *parent, int64_t n, int32_t *eu, int32_t *ev,
                              cudaStream_t s) {
    cudaError_t e;
    k_nonroot_flags<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(parent, n, S.cflag);
    if ((e = exclusive_scan_i32(S.cflag, S.cidx, n, S.tmp32, s))) return e;
    k_edges_from_parent<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(parent, S.cidx, n, eu, ev);
    return cudaGetLastError();
}

cudaError_t tree_search_and_label(TreeScratch &S, const double *phi_par, const double *omega, const double *p,
                                  int32_t k, int32_t *labels, uint8_t *residual, double *i_k, cudaStream_t s) {
    const TreeDev &T = S.T;
    const int64_t n = T.n;
    cudaError_t e;
    k_stats_part<<<STATS_BLOCKS, 256, 0, ISO_S(s)>>>(T.parent, phi_par, omega, p, n, S.spart, S.status);
    k_stats_final<<<1, STATS_BLOCKS, 0, ISO_S(s)>>>(S.spart, n, S.search);
    k_phi_slots<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(T.ch_list, phi_par, n - 1, S.phis);
    DpArgs A{n, T.parent, T.ch_off, T.ch_list, T.leaves, phi_par, omega, p, T.slot, S.phis};
    const unsigned grid = (unsigned)(num_sms() * 8);
    if ((e = cudaMemsetAsync(S.hist, 0, sizeof(uint32_t) * CAND_BUCKETS, s))) return e;
    for (int pass = 0; pass < DP_TREE_PASSES; ++pass) {
        if ((e = cudaMemsetAsync(S.done, 0, sizeof(int32_t) * n, s))) return e;
        k_dp_pass<<<grid, 256, 0, ISO_S(s)>>>(A, S.search, S.dec, S.wh, S.ph, S.done, S.rat, 0);
        k_search_update<<<1, 32, 0, ISO_S(s)>>>(S.search, k, pass == DP_TREE_PASSES - 1, S.status);
        if (pass + 1 < DP_TREE_PASSES) {
            // the next pass's thresholds from the critical ratios in lo's state
            k_cand_hist<<<grid, 256, 0, ISO_S(s)>>>(A, S.search, S.wh, S.ph, S.hist);
            k_cand_select<<<1, 1024, 0, ISO_S(s)>>>(S.search, S.hist);
        }
    }
    // Final call of Algorithm 1 at beta: Cut, eta and the set ratios (from the
    // last pass's lane at beta when it has one, else one more pass)
    k_final_lane<<<1, 32, 0, ISO_S(s)>>>(S.search);
    k_final_from_lane<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.search, T.parent, phi_par, T.slot, n, S.dec, S.wh, S.ph,
                                                           S.rat);
    if ((e = cudaMemsetAsync(S.done, 0, sizeof(int32_t) * n, s))) return e;
    k_dp_pass<<<grid, 256, 0, ISO_S(s)>>>(A, S.search, S.dec, S.wh, S.ph, S.done, S.rat, 1);
    // Algorithm 4: eta by pointer jumping, exclusive scan over Cut.
    k_head_init<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.dec, T.slot, T.parent, n, S.head);
    int32_t *ha = S.head, *hb = S.head2;
    const int Ln = log2_ceil(n) + 1;
    for (int it = 0; it < Ln; ++it) {
        k_head_jump<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(ha, hb, n);
        int32_t *t = ha; ha = hb; hb = t;
    }
    k_cut_flags<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.dec, T.slot, T.bfs_pos, n, S.cflag);
    if ((e = exclusive_scan_i32(S.cflag, S.cidx, n, S.tmp32, s))) return e;
    k_labels<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.dec, T.slot, T.bfs_pos, ha, S.cidx, S.rat, n, k, labels, residual, S.search);
    k_finish<<<1, 32, 0, ISO_S(s)>>>(S.search, k, i_k, S.status);
    return cudaGetLastError();
}

cudaError_t tree_search_and_label_sets(TreeScratch &S, int32_t nsets, const int64_t *offs, const int32_t *vset,
                                       const int32_t *ks, SearchState *SS, uint32_t *set_hist, const double *phi_par,
                                       const double *omega, const double *p, int32_t *labels, uint8_t *residual,
                                       double *i_k, double *beta, cudaStream_t s) {
    const TreeDev &T = S.T;
    const int64_t n = T.n, nv = n - 1;      // vertex nv is the virtual root
    cudaError_t e;
    // the virtual root is never decided: mark it discarded (its own head)
    if ((e = cudaMemsetAsync(S.dec + (size_t)nv * DP_LANES, DEC_DISCARD, DP_LANES, s))) return e;
    k_stats_sets<<<(unsigned)nsets, 256, 0, ISO_S(s)>>>(T.parent, phi_par, omega, p, offs, SS, S.status);
    // (states by vertex: the sets' many short walks and per-vertex sweeps
    // read them in vertex order)
    DpArgs A{n, T.parent, T.ch_off, T.ch_list, T.leaves, phi_par, omega, p, nullptr, nullptr};
    // one full wave: every warp takes an equal run of leaves, so a partial
    // second wave would leave SMs idle for half its length
    static int dp_occ = 0;
    if (dp_occ == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dp_occ, k_dp_pass_sets, 256, 0) != cudaSuccess ||
                        dp_occ < 1))
        dp_occ = 4;
    const unsigned grid = (unsigned)(num_sms() * dp_occ);
    const unsigned gs = (unsigned)ceil_div(nsets, 128);
    // each set: thresholds from its vertices' critical ratios while that
    // narrows its bracket, else the 33-ary bit search (as for one tree)
    if ((e = cudaMemsetAsync(set_hist, 0, sizeof(uint32_t) * (size_t)nsets * CAND_SET_BUCKETS, s))) return e;
    uint32_t *left = set_hist + (size_t)nsets * CAND_SET_BUCKETS;
    k_sets_left_init<<<1, 1, 0, ISO_S(s)>>>(left, nsets);
    const unsigned gw = (unsigned)ceil_div((int64_t)nsets * 32, 256);
    for (int pass = 0; pass < DP_TREE_PASSES; ++pass) {
        if ((e = cudaMemsetAsync(S.done, 0, sizeof(int32_t) * n, s))) return e;
        k_dp_pass_sets<<<grid, 256, 0, ISO_S(s)>>>(A, S.search, SS, vset, S.dec, S.wh, S.ph, S.done, S.rat, 0, left);
        k_search_update_sets<<<gs, 128, 0, ISO_S(s)>>>(SS, ks, nsets, pass == DP_TREE_PASSES - 1, S.status, left);
        if (pass + 1 < DP_TREE_PASSES) {
            k_cand_hist_sets<<<grid, 256, 0, ISO_S(s)>>>(A, SS, vset, nv, S.wh, S.ph, set_hist, left);
            k_cand_select_sets<<<gw, 256, 0, ISO_S(s)>>>(SS, nsets, set_hist, left);
        }
    }
    if ((e = cudaMemsetAsync(S.done, 0, sizeof(int32_t) * n, s))) return e;
    k_dp_pass_sets<<<grid, 256, 0, ISO_S(s)>>>(A, S.search, SS, vset, S.dec, S.wh, S.ph, S.done, S.rat, 1, left);
    k_head_init<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.dec, nullptr, T.parent, n, S.head);
    int32_t *ha = S.head, *hb = S.head2;
    const int Ln = log2_ceil(n) + 1;
    for (int it = 0; it < Ln; ++it) {
        k_head_jump<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(ha, hb, n);
        int32_t *t = ha; ha = hb; hb = t;
    }
    k_cut_flags<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.dec, nullptr, T.bfs_pos, n, S.cflag);
    if ((e = exclusive_scan_i32(S.cflag, S.cidx, n, S.tmp32, s))) return e;
    k_labels_sets<<<blocks_for(nv), TPB, 0, ISO_S(s)>>>(S.dec, T.bfs_pos, ha, S.cidx, S.rat, nv, vset, offs, ks, labels,
                                                        residual, SS);
    k_finish_sets<<<gs, 128, 0, ISO_S(s)>>>(SS, ks, nsets, i_k, beta, S.status);
    return cudaGetLastError();
}

cudaError_t fix_set_roots(TreeScratch &S, int32_t nsets, const int64_t *offs, cudaStream_t s) {
    k_fix_roots<<<blocks_for(nsets), TPB, 0, ISO_S(s)>>>(offs, nsets, S.T.parent, S.T.edge_of);
    return cudaGetLastError();
}

cudaError_t phi_from_edges(const TreeScratch &S, const double *edge_d2, double sigma, double *phi_par,
                           cudaStream_t s) {
    k_phi_from_edges<<<blocks_for(S.T.n), TPB, 0, ISO_S(s)>>>(S.T.edge_of, edge_d2, S.T.n, sigma, phi_par);
    return cudaGetLastError();
}

cudaError_t omega_tree_mode(const TreeScratch &S, const double *phi_par, int32_t include_self, double *omega,
                            cudaStream_t s) {
    k_omega_tree<<<blocks_for(S.T.n), TPB, 0, ISO_S(s)>>>(S.T.adj_key, S.T.adj_off, S.T.parent, phi_par, S.T.n,
                                                   include_self, omega);
    return cudaGetLastError();
}

}  // namespace iso

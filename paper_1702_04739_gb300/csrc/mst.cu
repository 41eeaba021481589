// mst.cu -- Section 2.2 step 2 / Section 3.5: the exact minimum spanning tree
// of the complete Euclidean graph, without storing the n x n matrix.
//
// The paper builds the dense affinity matrix and runs Prim (Algorithm 3),
// n sequential min-reductions.  Here every round of Boruvka's algorithm is
// one fused tiled sweep: a CTA stages 128-row and 128-column point tiles in
// shared memory, evaluates the 128x128 squared distances in FP32 registers
// (8x8 per thread), drops same-component pairs, and keeps each row's two
// smallest values.  Each row's winner is re-evaluated with the canonical FP64
// key; when the runner-up lies inside the proven FP32 error margin the row
// is rescanned and every candidate inside the margin is keyed in FP64, so
// the edge chosen is exactly the minimum-key edge.  Union-find by hooking
// along the chosen edges (mutual pairs broken by component id) and pointer
// jumping contracts the components; Boruvka at least halves them per round.
#include "mst.cuh"

namespace iso {

namespace {
constexpr int TPB = 256;
constexpr int SW_T = 128;      // rows and columns per tile
constexpr int SW_DC = 16;      // dims per shared-memory chunk
constexpr int SW_PAD = SW_T + 4;
inline unsigned blocks_for(int64_t n) { return (unsigned)(n > 0 ? ceil_div(n, TPB) : 1); }
// grid of the round kernels: at most 8 blocks of 256 per SM, grid-stride
inline unsigned round_grid(int64_t n) {
    const int64_t b = n > 0 ? ceil_div(n, 256) : 1, cap = (int64_t)num_sms() * 8;
    return (unsigned)(b < cap ? b : cap);
}
inline int log2_ceil(int64_t x) {
    int l = 0;
    while ((1LL << l) < x) ++l;
    return l;
}

__device__ __forceinline__ bool active(const int32_t *counters) {
    const volatile int32_t *c = counters;
    return c[MC_NCOMP] > c[MC_TARGET];
}

// ---------------------------------------------------------------- FP32 sweep
// grid: (row tiles) x (column splits).  Writes per (split, row) the smallest
// and second smallest FP32 d2 over columns of another component.
__global__ void __launch_bounds__(TPB, 2)
k_sweep_f32(const float *__restrict__ X, int64_t n, int32_t d, const int32_t *__restrict__ comp,
            const int32_t *__restrict__ counters, int splits, float *__restrict__ b1v, int32_t *__restrict__ b1j,
            float *__restrict__ b2v) {
    if (!active(counters)) return;
    __shared__ __align__(16) float As[SW_DC][SW_PAD];
    __shared__ __align__(16) float Bs[SW_DC][SW_PAD];
    __shared__ int32_t Bc[SW_T];
    __shared__ float m1v[SW_T][17];
    __shared__ float m2v[SW_T][17];
    __shared__ int32_t m1j[SW_T][17];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * SW_T;
    const int split = blockIdx.y;
    const int64_t ntiles = ceil_div(n, SW_T);
    const int64_t tiles_per = ceil_div(ntiles, splits);
    const int64_t ct0 = split * tiles_per, ct1 = min(ntiles, ct0 + tiles_per);

    int32_t rc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int64_t r = row0 + ty * 8 + i;
        rc[i] = r < n ? comp[r] : -1;
    }
    float v1[8], v2[8];
    int32_t j1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { v1[i] = INFINITY; v2[i] = INFINITY; j1[i] = -1; }

    for (int64_t ct = ct0; ct < ct1; ++ct) {
        const int64_t col0 = ct * SW_T;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
        for (int t0 = 0; t0 < d; t0 += SW_DC) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < (SW_T * SW_DC) / TPB; ++q) {
                int idx = tid + q * TPB;
                int r = idx / SW_DC, t = idx % SW_DC;
                int64_t gr = row0 + r, gc = col0 + r;
                int gt = t0 + t;
                As[t][r] = (gr < n && gt < d) ? X[gr * d + gt] : 0.0f;
                Bs[t][r] = (gc < n && gt < d) ? X[gc * d + gt] : 0.0f;
            }
            if (t0 == 0 && tid < SW_T) {
                int64_t gc = col0 + tid;
                Bc[tid] = gc < n ? comp[gc] : -2;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < SW_DC; ++t) {
                float4 a0 = *reinterpret_cast<const float4 *>(&As[t][ty * 8]);
                float4 a1 = *reinterpret_cast<const float4 *>(&As[t][ty * 8 + 4]);
                float4 c0 = *reinterpret_cast<const float4 *>(&Bs[t][tx * 8]);
                float4 c1 = *reinterpret_cast<const float4 *>(&Bs[t][tx * 8 + 4]);
                float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                float b[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float df = __fsub_rn(a[i], b[j]);
                        acc[i][j] = __fmaf_rn(df, df, acc[i][j]);
                    }
            }
        }
        // epilogue: same-component pairs and padding are skipped
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int cl = tx * 8 + j;
            const int32_t cc = Bc[cl];
            const int32_t gcol = (int32_t)(col0 + cl);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float v = acc[i][j];
                if (cc >= 0 && cc != rc[i] && v < v2[i]) {
                    if (v < v1[i]) { v2[i] = v1[i]; v1[i] = v; j1[i] = gcol; }
                    else v2[i] = v;
                }
            }
        }
    }
    // merge the 16 column-threads of each row (fixed order)
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        m1v[ty * 8 + i][tx] = v1[i];
        m2v[ty * 8 + i][tx] = v2[i];
        m1j[ty * 8 + i][tx] = j1[i];
    }
    __syncthreads();
    if (tid < SW_T) {
        int64_t r = row0 + tid;
        float a1 = INFINITY, a2 = INFINITY;
        int32_t aj = -1;
        for (int s = 0; s < 16; ++s) {
            float w1 = m1v[tid][s], w2 = m2v[tid][s];
            int32_t wj = m1j[tid][s];
            if (w1 < a1) { a2 = fminf(a1, w2); a1 = w1; aj = wj; }
            else a2 = fminf(a2, w1);
        }
        if (r < n) {
            size_t o = (size_t)split * n + r;
            b1v[o] = a1; b2v[o] = a2; b1j[o] = aj;
        }
    }
}

// Approximate FP32 d2 in exactly the sweep's operation order.
__device__ __forceinline__ float approx_d2(const float *__restrict__ a, const float *__restrict__ b, int d) {
    float acc = 0.0f;
    for (int t = 0; t < d; ++t) {
        float df = __fsub_rn(a[t], b[t]);
        acc = __fmaf_rn(df, df, acc);
    }
    return acc;
}

// Merge the column splits, then either key the winner in FP64 or queue the
// row for a rescan when the runner-up is inside the FP32 error margin.
__global__ void k_recheck(const float *__restrict__ X, int64_t n, int32_t d, int splits,
                          const float *__restrict__ b1v, const int32_t *__restrict__ b1j,
                          const float *__restrict__ b2v, double margin_mul, double margin_add,
                          double *__restrict__ rowd2, int32_t *__restrict__ rowj, int32_t *__restrict__ ovf,
                          int32_t *counters) {
    if (!active(counters)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a1 = INFINITY, a2 = INFINITY;
    int32_t aj = -1;
    for (int s = 0; s < splits; ++s) {
        size_t o = (size_t)s * n + i;
        float w1 = b1v[o], w2 = b2v[o];
        int32_t wj = b1j[o];
        if (w1 < a1) { a2 = fminf(a1, w2); a1 = w1; aj = wj; }
        else a2 = fminf(a2, w1);
    }
    if (aj < 0) { rowj[i] = -1; return; }
    double tau = (double)a1 * margin_mul + margin_add;
    if (!((double)a2 > tau)) {
        int q = atomicAdd(counters + MC_OVERFLOW, 1);
        ovf[q] = (int32_t)i;
        rowj[i] = -2;
        rowd2[i] = tau;          // rescan threshold
        return;
    }
    rowd2[i] = exact_d2(X + i * d, X + (int64_t)aj * d, d);
    rowj[i] = aj;
}

// One CTA per queued row: every column inside the margin is keyed in FP64.
__global__ void __launch_bounds__(TPB) k_rescan(const float *__restrict__ X, int64_t n, int32_t d,
                                                const int32_t *__restrict__ comp, const int32_t *__restrict__ ovf,
                                                double *__restrict__ rowd2, int32_t *__restrict__ rowj,
                                                int32_t *counters) {
    if (!active(counters)) return;
    __shared__ double sd[TPB];
    __shared__ int32_t sj[TPB];
    const int nq = counters[MC_OVERFLOW];
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const int64_t i = ovf[q];
        const double tau = rowd2[i];
        const int32_t ci = comp[i];
        const float *xi = X + i * d;
        double bd = INFINITY;
        int32_t bj = -1;
        for (int64_t j = threadIdx.x; j < n; j += TPB) {
            if (comp[j] == ci) continue;
            float v = approx_d2(xi, X + j * d, d);
            if ((double)v <= tau) {
                double e = exact_d2(xi, X + j * d, d);
                if (bj < 0 || key_less(e, (int32_t)i, (int32_t)j, bd, (int32_t)i, bj)) { bd = e; bj = (int32_t)j; }
            }
        }
        sd[threadIdx.x] = bd;
        sj[threadIdx.x] = bj;
        __syncthreads();
        for (int s = TPB / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                double od = sd[threadIdx.x + s];
                int32_t oj = sj[threadIdx.x + s];
                if (oj >= 0 && (sj[threadIdx.x] < 0 ||
                                key_less(od, (int32_t)i, oj, sd[threadIdx.x], (int32_t)i, sj[threadIdx.x]))) {
                    sd[threadIdx.x] = od;
                    sj[threadIdx.x] = oj;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            rowd2[i] = sd[0];
            rowj[i] = sj[0];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- FP64 sweep
template <class T>
__global__ void __launch_bounds__(TPB) k_sweep_f64(const T *__restrict__ X, int64_t n, int32_t d,
                                                   const int32_t *__restrict__ comp, const int32_t *counters,
                                                   double *__restrict__ rowd2, int32_t *__restrict__ rowj) {
    if (!active(counters)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t ci = comp[i];
    const T *xi = X + i * d;
    double bd = INFINITY;
    int32_t bj = -1;
    for (int64_t j = 0; j < n; ++j) {
        if (comp[j] == ci) continue;
        double e = exact_d2(xi, X + j * d, d);
        if (bj < 0 || key_less(e, (int32_t)i, (int32_t)j, bd, (int32_t)i, bj)) { bd = e; bj = (int32_t)j; }
    }
    rowd2[i] = bd;
    rowj[i] = bj;
}

// ---------------------------------------------------------------- union-find
__global__ void k_mst_init(int32_t *comp, int64_t n, int32_t target, int32_t *counters) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = (int32_t)v;
    if (v == 0) {
        counters[MC_TARGET] = target;
        counters[MC_OVERFLOW] = 0;
        counters[MC_NEDGES] = 0;
        counters[MC_NCOMP] = (int32_t)n;
        counters[MC_ROUNDS] = 0;
        counters[MC_OVF_TOTAL] = 0;
        counters[MC_NCOMP_NEW] = 0;
    }
}

// The kernels of a round loop over their elements with a grid of a few waves
// (round_grid): once the forest is complete, the rest of the fixed round
// budget costs a handful of blocks per launch.
__global__ void k_round_begin(int32_t *counters, unsigned long long *cd2, unsigned long long *cpair, int64_t n) {
    if (!active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        cd2[v] = ~0ull;
        cpair[v] = ~0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counters[MC_OVF_TOTAL] += counters[MC_OVERFLOW];
        counters[MC_OVERFLOW] = 0;
        counters[MC_ROUNDS] += 1;
        counters[MC_NCOMP_NEW] = 0;
    }
}

__global__ void k_cmin_d2(const int32_t *__restrict__ comp, const double *__restrict__ rowd2,
                          const int32_t *__restrict__ rowj, int64_t n, unsigned long long *cd2,
                          const int32_t *counters) {
    if (!active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        // the lanes of one component fold first (late rounds: few components,
        // so one atomic per component and warp instead of one per row)
        const bool has = rowj[i] >= 0;
        const int32_t c = has ? comp[i] : -1;
        const unsigned long long v = has ? dbits(rowd2[i]) : ~0ull;
        const unsigned peers = __match_any_sync(__activemask(), c);
        const unsigned hi = __reduce_min_sync(peers, (unsigned)(v >> 32));
        const unsigned lo = __reduce_min_sync(peers, (unsigned)(v >> 32) == hi ? (unsigned)v : 0xffffffffu);
        if (c >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1)
            atomicMin(cd2 + c, ((unsigned long long)hi << 32) | lo);
    }
}

__global__ void k_cmin_pair(const int32_t *__restrict__ comp, const double *__restrict__ rowd2,
                            const int32_t *__restrict__ rowj, int64_t n, const unsigned long long *cd2,
                            unsigned long long *cpair, const int32_t *counters) {
    if (!active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        int32_t j = rowj[i];
        if (j < 0) continue;
        int32_t c = comp[i];
        if (dbits(rowd2[i]) != cd2[c]) continue;
        unsigned long long a = (unsigned long long)min((int32_t)i, j), b = (unsigned long long)max((int32_t)i, j);
        atomicMin(cpair + c, (a << 32) | b);
    }
}

__global__ void k_hook_tgt(const int32_t *__restrict__ comp, int64_t n, const unsigned long long *__restrict__ cd2,
                           const unsigned long long *__restrict__ cpair, int32_t *__restrict__ tgt,
                           int32_t *__restrict__ cu, int32_t *__restrict__ cv, double *__restrict__ cdd,
                           const int32_t *counters, uint32_t *st) {
    if (!active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        if (comp[v] != v) continue;
        unsigned long long pr = cpair[v];
        if (pr == ~0ull) { tgt[v] = (int32_t)v; continue; }
        int32_t a = (int32_t)(pr >> 32), b = (int32_t)(pr & 0xffffffffu);
        if (a < 0 || b < 0 || a >= n || b >= n) {
            // not a pair of points (a sharded call's all-reduce returned garbage): no hook
            atomicOr(st, DEV_INTERNAL);
            tgt[v] = (int32_t)v;
            continue;
        }
        int32_t outside = comp[a] == v ? b : a;
        tgt[v] = comp[outside];
        cu[v] = a; cv[v] = b; cdd[v] = bitsd(cd2[v]);
    }
}

__global__ void k_hook_resolve(const int32_t *__restrict__ comp, int64_t n, const int32_t *__restrict__ tgt,
                               const int32_t *__restrict__ cu, const int32_t *__restrict__ cv,
                               const double *__restrict__ cdd, int32_t *__restrict__ nxt, int32_t *__restrict__ eu,
                               int32_t *__restrict__ ev, double *__restrict__ ed2, int32_t *counters, uint32_t *st) {
    if (!active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        if (comp[v] != v) continue;
        int32_t T = tgt[v];
        if (T == v) { nxt[v] = (int32_t)v; continue; }
        bool mutual = tgt[T] == v;
        nxt[v] = (mutual && v < T) ? (int32_t)v : T;
        if (!mutual || v < T) {
            int q = atomicAdd(counters + MC_NEDGES, 1);
            if (q < n - 1) { eu[q] = cu[v]; ev[q] = cv[v]; ed2[q] = cdd[v]; }
            else atomicOr(st, DEV_EDGE_COUNT);
        }
    }
}

// Every root's pointer to the root of its hook tree, in place, in one
// launch: a find with path halving from each root.  An entry only ever holds
// an ancestor of its vertex, and a walk only replaces the entry of a vertex
// it visits by that vertex's grandparent, and only if the entry still holds
// the parent it read (compare-and-swap: an entry that already holds its root
// keeps it), so any interleaving of the walks keeps that true, and the walks
// halve the paths they share (with more roots than resident threads, a later
// walk finds the paths of the earlier ones compressed).  A walk ends within
// the tree's depth; one longer than the number of points is a cycle (the
// hooks never build one), reported as an internal error.
__global__ void k_jump_all(const int32_t *__restrict__ comp, int32_t *nxt, int64_t n, const int32_t *counters,
                           uint32_t *st) {
    if (!active(counters)) return;
    volatile int32_t *vn = nxt;                       // other walks change the entries under us
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        if (comp[v] != v) continue;
        int32_t x = (int32_t)v;
        for (int64_t it = 0;; ++it) {
            const int32_t p = vn[x];
            const int32_t q = (p >= 0 && p < n) ? vn[p] : -1;
            if (q < 0 || q >= n || it > n) {
                atomicOr(st, DEV_INTERNAL);
                break;
            }
            if (q == p) {                             // p is a root
                vn[v] = p;
                break;
            }
            atomicCAS(reinterpret_cast<int *>(nxt) + x, p, q);
            x = q;
        }
    }
}

__global__ void k_relabel(int32_t *comp, const int32_t *__restrict__ nxt, int64_t n, int32_t *counters) {
    if (!active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        int32_t r = nxt[comp[v]];
        comp[v] = r;
        if (r == v) atomicAdd(counters + MC_NCOMP_NEW, 1);
    }
}

__global__ void k_round_end(int32_t *counters) {
    if (!active(counters)) return;
    counters[MC_NCOMP] = counters[MC_NCOMP_NEW];
}

__global__ void k_edge_keys(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev, int64_t m,
                            uint64_t *__restrict__ key, int32_t *__restrict__ val) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    uint64_t a = (uint64_t)min(eu[e], ev[e]), b = (uint64_t)max(eu[e], ev[e]);
    key[e] = (a << 32) | b;
    val[e] = (int32_t)e;
}

__global__ void k_edge_keys_d2(const double *__restrict__ ed2, const int32_t *__restrict__ val, int64_t m,
                               uint64_t *__restrict__ key) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) key[q] = dbits(ed2[val[q]]);
}

__global__ void k_edge_gather(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                              const double *__restrict__ ed2, const int32_t *__restrict__ val, int64_t m,
                              int32_t *__restrict__ ou, int32_t *__restrict__ ov, double *__restrict__ od2) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    int32_t e = val[q];
    ou[q] = min(eu[e], ev[e]);
    ov[q] = max(eu[e], ev[e]);
    od2[q] = ed2[e];
}

__global__ void k_nn_init(unsigned long long *nn, int64_t n) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) nn[v] = ~0ull;
}

__global__ void k_nn_edges(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                           const double *__restrict__ ed2, int64_t m, unsigned long long *nn) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    unsigned long long b = dbits(ed2[e]);
    atomicMin(nn + eu[e], b);
    atomicMin(nn + ev[e], b);
}

__global__ void k_nn_rows(const double *__restrict__ rowd2, const int32_t *__restrict__ rowj, int64_t n,
                          unsigned long long *nn) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) nn[v] = rowj[v] >= 0 ? dbits(rowd2[v]) : ~0ull;
}
}  // namespace

int mst_splits(int64_t n) {
    int64_t tiles = ceil_div(n, SW_T);
    int64_t slots = (int64_t)num_sms() * 2;
    int64_t s = ceil_div(4 * slots, tiles > 0 ? tiles : 1);
    int64_t max_s = tiles / 8 > 1 ? tiles / 8 : 1;
    if (s > max_s) s = max_s;
    if (s < 1) s = 1;
    if (s > 64) s = 64;
    return (int)s;
}

void MstScratch::carve(Arena &A, int64_t n_, int splits_) {
    n = n_;
    splits = splits_;
    int64_t m = n > 1 ? n - 1 : 1;
    comp = A.take<int32_t>(n);
    nxt = A.take<int32_t>(n);
    tgt = A.take<int32_t>(n);
    b1v = A.take<float>((size_t)splits * n);
    b2v = A.take<float>((size_t)splits * n);
    b1j = A.take<int32_t>((size_t)splits * n);
    rowd2 = A.take<double>(n);
    rowj = A.take<int32_t>(n);
    cd2 = A.take<unsigned long long>(n);
    cpair = A.take<unsigned long long>(n);
    cu = A.take<int32_t>(n);
    cv = A.take<int32_t>(n);
    cdd = A.take<double>(n);
    ovf_rows = A.take<int32_t>(n);
    counters = A.take<int32_t>(8);
    eu = A.take<int32_t>(m);
    ev = A.take<int32_t>(m);
    ed2 = A.take<double>(m);
    skey = A.take<uint64_t>(n);
    kbuf = A.take<uint64_t>(n);
    sval = A.take<int32_t>(n);
    vbuf = A.take<int32_t>(n);
    nnbits = A.take<unsigned long long>(n);
}

static cudaError_t sweep_round(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                               cudaStream_t s) {
    if (sweep_fp64) {
        if (dtype == ISOCLUST_F64)
            k_sweep_f64<double><<<blocks_for(n), TPB, 0, ISO_S(s)>>>((const double *)X, n, d, S.comp, S.counters, S.rowd2,
                                                              S.rowj);
        else
            k_sweep_f64<float><<<blocks_for(n), TPB, 0, ISO_S(s)>>>((const float *)X, n, d, S.comp, S.counters, S.rowd2,
                                                             S.rowj);
        return cudaGetLastError();
    }
    const float *Xf = (const float *)X;
    dim3 grid((unsigned)ceil_div(n, SW_T), (unsigned)S.splits);
    k_sweep_f32<<<grid, TPB, 0, ISO_S(s)>>>(Xf, n, d, S.comp, S.counters, S.splits, S.b1v, S.b1j, S.b2v);
    // FP32 error of sum_t fl(fl(a-b)^2 + acc) with FMA: relative <= (d+1)u + O(u^2);
    // padded with 2u and a 1.1 safety factor, plus an absolute term for underflow.
    const double u = 5.9604644775390625e-08;   // 2^-24
    const double e = 1.1 * (double)(d + 3) * u;
    const double mul = (1.0 + e) / (1.0 - e);
    const double add = (double)(d + 1) * 1.401298464324817e-45 * 4.0;
    k_recheck<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(Xf, n, d, S.splits, S.b1v, S.b1j, S.b2v, mul, add, S.rowd2, S.rowj,
                                            S.ovf_rows, S.counters);
    k_rescan<<<(unsigned)(num_sms() * 4), TPB, 0, ISO_S(s)>>>(Xf, n, d, S.comp, S.ovf_rows, S.rowd2, S.rowj, S.counters);
    return cudaGetLastError();
}

__global__ void k_or_err(const uint32_t *src, uint32_t *dst) {
    if (*src) atomicOr(dst, *src);
}

cudaError_t mst_build(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                      uint32_t *status, cudaStream_t s, TcScratch *tc, int32_t target, int64_t max_n,
                      const Shard *sh) {
    k_mst_init<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.comp, n, target, S.counters);
    // Boruvka at least halves every unfinished set's components per round
    const int64_t span = max_n > 0 ? max_n : n;
    const int R = log2_ceil(span) + 1;
    const unsigned rg = round_grid(n);
    cudaError_t e;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cs))) return e;
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if (tc && (e = tc_prepare(*tc, (const float *)X, n, d, s, !tc->prune))) return e;
    if (tc && tc->prune) {
        // pruned rounds (one set): the rows take the pruning's order; no row
        // has a previous round's pair yet
        if ((e = prune_reorder(*tc, S.rowd2, (const float *)X, n, d, s))) return e;
        if ((e = cudaMemsetAsync(S.rowj, 0xff, sizeof(int32_t) * n, s))) return e;
    }
    if (tc && (e = tc_count_sets(*tc, S.comp, n, S.counters, s))) return e;
    if (tc && (e = tc_autotune(*tc, S, (const float *)X, n, d, status, s))) return e;
    if (!tc) tc_clear_last_variant();
    for (int r = 0; r < R; ++r) {
        k_round_begin<<<rg, TPB, 0, ISO_S(s)>>>(S.counters, S.cd2, S.cpair, n);
        if (tc) {
            if ((e = tc_sweep_round(*tc, S, (const float *)X, n, d, status, s))) return e;
        } else if ((e = sweep_round(S, X, n, d, dtype, sweep_fp64, s))) {
            return e;
        }
        k_cmin_d2<<<rg, TPB, 0, ISO_S(s)>>>(S.comp, S.rowd2, S.rowj, n, S.cd2, S.counters);
        // sharded: each rank saw only its own rows; the minima over all rows
        if (sh && (e = shard_allreduce(*sh, S.cd2, n, ISOCLUST_REDUCE_MIN_U64, s))) return e;
        k_cmin_pair<<<rg, TPB, 0, ISO_S(s)>>>(S.comp, S.rowd2, S.rowj, n, S.cd2, S.cpair, S.counters);
        if (sh && (e = shard_allreduce(*sh, S.cpair, n, ISOCLUST_REDUCE_MIN_U64, s))) return e;
        k_hook_tgt<<<rg, TPB, 0, ISO_S(s)>>>(S.comp, n, S.cd2, S.cpair, S.tgt, S.cu, S.cv, S.cdd, S.counters, status);
        k_hook_resolve<<<rg, TPB, 0, ISO_S(s)>>>(S.comp, n, S.tgt, S.cu, S.cv, S.cdd, S.nxt, S.eu, S.ev, S.ed2,
                                                     S.counters, status);
        k_jump_all<<<rg, TPB, 0, ISO_S(s)>>>(S.comp, S.nxt, n, S.counters, status);
        k_relabel<<<rg, TPB, 0, ISO_S(s)>>>(S.comp, S.nxt, n, S.counters);
        if (tc && (e = tc_count_sets(*tc, S.comp, n, S.counters, s))) return e;
        k_round_end<<<1, 1, 0, ISO_S(s)>>>(S.counters);
        // one point set whose tree is complete: the rounds left would only
        // launch kernels that return at once (independent sets keep every
        // round, so a call launches the same kernels as its CUDA graph)
        if (target == 1 && !capturing && r + 1 < R) {
            int32_t h[8];
            if ((e = cudaMemcpyAsync(h, S.counters, sizeof(h), cudaMemcpyDeviceToHost, s))) return e;
            if ((e = cudaStreamSynchronize(s))) return e;
            if (h[MC_NCOMP] <= h[MC_TARGET]) break;
        }
    }
    if (tc) k_or_err<<<1, 1, 0, ISO_S(s)>>>(tc->err, status);
    return cudaGetLastError();
}

cudaError_t nn_sweep(MstScratch &S, const void *X, int64_t n, int32_t d, int dtype, bool sweep_fp64,
                     uint32_t *status, cudaStream_t s, TcScratch *tc) {
    k_mst_init<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.comp, n, 1, S.counters);
    k_round_begin<<<round_grid(n), TPB, 0, ISO_S(s)>>>(S.counters, S.cd2, S.cpair, n);
    cudaError_t e;
    if (tc) {
        if ((e = tc_prepare(*tc, (const float *)X, n, d, s))) return e;
        if ((e = tc_sweep_round(*tc, S, (const float *)X, n, d, status, s))) return e;
        k_or_err<<<1, 1, 0, ISO_S(s)>>>(tc->err, status);
    } else if ((e = sweep_round(S, X, n, d, dtype, sweep_fp64, s))) {
        return e;
    }
    k_nn_rows<<<blocks_for(n), TPB, 0, ISO_S(s)>>>(S.rowd2, S.rowj, n, S.nnbits);
    return cudaGetLastError();
}

cudaError_t mst_sort_edges(MstScratch &S, int32_t *out_u, int32_t *out_v, double *out_d2, cudaStream_t s) {
    const int64_t m = S.n - 1;
    if (m <= 0) return cudaSuccess;
    cudaError_t e;
    k_edge_keys<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(S.eu, S.ev, m, S.skey, S.sval);
    if ((e = sort_pairs_u64(S.skey, S.sval, S.kbuf, S.vbuf, m, s))) return e;
    k_edge_keys_d2<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(S.ed2, S.sval, m, S.skey);
    if ((e = sort_pairs_u64(S.skey, S.sval, S.kbuf, S.vbuf, m, s))) return e;   // stable: ties keep (u, v) order
    k_edge_gather<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(S.eu, S.ev, S.ed2, S.sval, m, out_u, out_v, out_d2);
    return cudaGetLastError();
}

cudaError_t nn_from_edges(MstScratch &S, const int32_t *eu, const int32_t *ev, const double *ed2, cudaStream_t s,
                          int64_t m) {
    if (m < 0) m = S.n - 1;
    k_nn_init<<<blocks_for(S.n), TPB, 0, ISO_S(s)>>>(S.nnbits, S.n);
    if (m > 0) k_nn_edges<<<blocks_for(m), TPB, 0, ISO_S(s)>>>(eu, ev, ed2, m, S.nnbits);
    return cudaGetLastError();
}

}  // namespace iso

// mst_prune.cu -- pruned Boruvka rounds for one point set.
//
// Section 3.5's rounds need, for every component, its lightest outgoing
// edge.  A pair of 128-row tiles (R, C) can hold that edge for a component
// of R's rows only if its pairs can be that light: with tile centroids c and
// radii r (every point of a tile within r of its c),
//     d2(i, j) >= LB(R, C) = max(0, |c_R - c_C| - r_R - r_C)^2  (i in R, j in C).
// Each round first sweeps every row tile against its near tiles (the
// PRUNE_NEAR tiles on either side in a bisection order whose tiles are
// compact); the candidates found there bound each component's lightest
// outgoing d2 from above (UB, rigorous: the sweep's upper bound of the
// represented d2 plus the BF16 representation error, or the exact d2 of a
// row's best pair of the previous round whose points are still apart).  A far tile pair is
// then swept only if LB(R, C) <= max over R's rows of their component's UB,
// and not when both tiles lie wholly inside one component.  Pairs left out
// have every d2 > UB of each component of R's rows, so no component's
// lightest edge is among them: the round joins the same components by the
// same edges as the full sweep.
//
// The order, set up before the first round: points whose distance to the
// nearest of 256 evenly spaced sample points is more than 4x the median of
// that distance (isolated points: a tile holding some would span the space)
// go last; the others in recursive bisection of their tile range.  A node (a range of whole tiles) is split
// at its middle tile after sorting its points by their projection on the
// line through two far-apart points of the node (the farthest point from the
// node's first point, then the farthest from that one), so the two halves
// are the node's two ends along that line.
#include <stddef.h>

#include <atomic>

#include "mst.cuh"

namespace iso {

namespace {
constexpr int PR_BM = 128;                 // rows per tile (the sweep's)
std::atomic<int> g_prune_mode{-1};

// node of tile t after l halvings of [0, T), and its tile range [a, b)
__device__ __forceinline__ uint32_t pr_node(int64_t t, int64_t T, int l, int64_t &a, int64_t &b) {
    a = 0;
    b = T;
    uint32_t id = 0;
    for (int k = 0; k < l; ++k) {
        const int64_t m = a + (b - a) / 2;
        if (t < m) { b = m; id = 2 * id; }
        else { a = m; id = 2 * id + 1; }
    }
    return id;
}

// PASS 0: farthest point of each node from its first point; PASS 1: from
// that point.  far[node] = max (d2 bits, index).  A thread per position (its
// row's loads in flight together); the lanes of a warp that share a node
// fold their keys first, so a node sees one atomic per warp.
template <int PASS>
__global__ void k_pr_far(const float *__restrict__ X, int64_t n, int32_t d, const int32_t *__restrict__ perm,
                         int64_t T, int l, const unsigned long long *__restrict__ far0,
                         unsigned long long *__restrict__ far) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t id = 0xffffffffu;
    unsigned long long key = 0;
    if (p < n) {
        int64_t a, b;
        id = pr_node(p / PR_BM, T, l, a, b);
        if (b - a > 1) {
            const int32_t i = perm[p];
            const int64_t ref = PASS == 0 ? (int64_t)perm[a * PR_BM] : (int64_t)(uint32_t)(far0[id] & 0xffffffffull);
            const float *x = X + (int64_t)i * d, *y = X + ref * d;
            float s2 = 0.0f;
            for (int t = 0; t < d; ++t) {
                const float df = x[t] - y[t];
                s2 = fmaf(df, df, s2);
            }
            key = ((unsigned long long)__float_as_uint(s2) << 32) | (unsigned long long)(uint32_t)i;
        } else {
            id = 0xffffffffu;                                // a single tile: not split further
        }
    }
    // lanes of the same node: the largest key goes to the lowest such lane
    const unsigned same = __match_any_sync(0xffffffffu, id);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long k2 = __shfl_down_sync(0xffffffffu, key, o);
        const int src = lane + o;
        if (src < 32 && ((same >> src) & 1u) && k2 > key) key = k2;
    }
    if (id != 0xffffffffu && lane == __ffs(same) - 1) atomicMax(far + id, key);
}

// sort key of position p: (node, projection on the node's far pair's line)
__global__ void k_pr_keys(const float *__restrict__ X, int64_t n, int32_t d, const int32_t *__restrict__ perm,
                          int64_t T, int l, const unsigned long long *__restrict__ far0,
                          const unsigned long long *__restrict__ far1, uint64_t *__restrict__ keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t a, b;
    const uint32_t id = pr_node(p / PR_BM, T, l, a, b);
    const int32_t i = perm[p];
    float proj = 0.0f;
    if (b - a > 1) {
        const int64_t pb = (int64_t)(uint32_t)(far0[id] & 0xffffffffull);
        const int64_t pc = (int64_t)(uint32_t)(far1[id] & 0xffffffffull);
        const float *xi = X + (int64_t)i * d, *xb = X + pb * d, *xc = X + pc * d;
        for (int t = 0; t < d; ++t) proj = fmaf(xi[t] - xb[t], xc[t] - xb[t], proj);
    }
    uint32_t u = __float_as_uint(proj);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);             // order-preserving bits
    keys[p] = ((uint64_t)id << 32) | (uint64_t)u;
}

// Isolation proxy before any round: each point's FP32 d2 to the nearest of
// PR_SAMPLES evenly spaced sample points (itself excluded).  Points of a
// cluster find a sample nearby; isolated points do not.  A thread per point
// keeps 32 dimensions of its row in registers against 32 samples staged in
// shared memory (broadcast reads).
constexpr int PR_SAMPLES = 256;
__global__ void __launch_bounds__(256) k_pr_sample_nn(const float *__restrict__ X, int64_t n, int32_t d,
                                                      int64_t stride, int nsamp, double *__restrict__ out) {
    extern __shared__ float ss[];                             // [32][d]
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float best = INFINITY;
    for (int s0 = 0; s0 < nsamp; s0 += 32) {                  // nsamp: a multiple of 32
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * d; e += blockDim.x) {
            const int q = e / d, t = e - q * d;
            ss[q * d + t] = X[(int64_t)(s0 + q) * stride * d + t];
        }
        __syncthreads();
        if (i < n) {
            float acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
            int t0 = 0;
            for (; t0 + 32 <= d; t0 += 32) {                  // whole chunks of 32 dimensions
                float xv[32];
#pragma unroll
                for (int t = 0; t < 32; t += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(X + i * d + t0 + t);
                    xv[t] = v.x; xv[t + 1] = v.y; xv[t + 2] = v.z; xv[t + 3] = v.w;
                }
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const float *sq = ss + q * d + t0;
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        const float df = xv[t] - sq[t];
                        acc[q] = fmaf(df, df, acc[q]);
                    }
                }
            }
            for (int t = t0; t < d; ++t) {                    // the tail
                const float xt = X[i * d + t];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const float df = xt - ss[q * d + t];
                    acc[q] = fmaf(df, df, acc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if ((int64_t)(s0 + q) * stride != i) best = fminf(best, acc[q]);
        }
    }
    if (i < n) out[i] = (double)best;
}

__global__ void k_pr_nn_keys(const double *__restrict__ rowd2, int64_t n, uint64_t *__restrict__ keys,
                             int32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint64_t)__double_as_longlong(rowd2[i]);     // non-negative: bits are monotone
    vals[i] = (int32_t)i;
}

// isolated points (nearest neighbour d2 above 16x the median's) after the
// others, each group in index order; counts them
__global__ void k_pr_far_keys(const double *__restrict__ rowd2, int64_t n, const uint64_t *__restrict__ sorted,
                              uint64_t *__restrict__ keys, int32_t *__restrict__ vals,
                              unsigned long long *__restrict__ nfar) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double med = __longlong_as_double((long long)sorted[n / 2]);
    const double tau2 = med > 0.0 ? 16.0 * med : INFINITY;
    const bool far = rowd2[i] > tau2;
    keys[i] = ((uint64_t)(far ? 1 : 0) << 32) | (uint64_t)i;
    vals[i] = (int32_t)i;
    if (far) atomicAdd(nfar, 1ull);
}

// Per tile: centroid (FP64 mean, stored FP32) and radius: the largest FP64
// distance of a real row to the stored centroid, rounded up with a margin
// for the FP64 rounding of that distance.
__global__ void __launch_bounds__(128) k_pr_geom(const float *__restrict__ X, int32_t d,
                                                 const int32_t *__restrict__ permp, float *__restrict__ tcen,
                                                 float *__restrict__ trad) {
    extern __shared__ float sc[];                             // d floats
    __shared__ double sr[128];
    const int64_t t = blockIdx.x;
    const int32_t *pr = permp + t * PR_BM;
    int cnt = 0;
    for (int q = 0; q < PR_BM; ++q) cnt += pr[q] >= 0 ? 1 : 0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < PR_BM; ++q) {
            const int32_t i = pr[q];
            if (i >= 0) s += (double)X[(int64_t)i * d + k];
        }
        const float c = cnt > 0 ? (float)(s / (double)cnt) : 0.0f;
        sc[k] = c;
        tcen[t * d + k] = c;
    }
    __syncthreads();
    double r2 = 0.0;
    const int32_t i = pr[threadIdx.x];
    if (i >= 0) {
        const float *xi = X + (int64_t)i * d;
        for (int k = 0; k < d; ++k) {
            const double df = (double)xi[k] - (double)sc[k];
            r2 = fma(df, df, r2);
        }
    }
    sr[threadIdx.x] = r2;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) trad[t] = __double2float_ru(sqrt(sr[0]) * (1.0 + 1e-12));
}

// LB(R, C) as a float rounded down.  The centroid distance comes from an
// FP32 sum of squared differences (relative error below (d + 2) 2^-24),
// taken (d + 8) 2^-23 short of itself.
__global__ void __launch_bounds__(128) k_pr_lb(const float *__restrict__ tcen, const float *__restrict__ trad,
                                               int64_t T, int32_t d, float *__restrict__ tlb2) {
    extern __shared__ float cr[];                             // d floats: c_R
    const int64_t R = blockIdx.y;
    for (int k = threadIdx.x; k < d; k += blockDim.x) cr[k] = tcen[R * d + k];
    __syncthreads();
    const int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= T) return;
    const float *b = tcen + C * d;
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
        const float df = cr[k] - b[k];
        s = fmaf(df, df, s);
    }
    const double g = sqrt((double)s) * (1.0 - (double)(d + 8) * 1.1920928955078125e-07) - (double)trad[R] -
                     (double)trad[C];
    tlb2[R * T + C] = g > 0.0 ? __double2float_rd(g * g * (1.0 - 1e-9)) : 0.0f;
}

__global__ void k_pr_near(int64_t T, int4 *__restrict__ items_a) {
    const int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (R >= T) return;
    const int64_t c0 = R - PRUNE_NEAR > 0 ? R - PRUNE_NEAR : 0;
    const int64_t c1 = R + PRUNE_NEAR + 1 < T ? R + PRUNE_NEAR + 1 : T;
    items_a[R] = make_int4((int)R, (int)c0, (int)c1, 0);
}

__device__ __forceinline__ bool pr_active(const int32_t *counters) {
    const volatile int32_t *c = counters;
    return c[MC_NCOMP] > c[MC_TARGET];
}

// The rigorous upper bound of each component's lightest outgoing d2 from
// the near sweep: per row, the smallest upper bound of a candidate's
// represented d2 (lists 0 and 1), widened by the representation error as
// the recheck does, then the minimum over the component's rows.
// Also, the row's exact best pair of the previous round (rowd2, rowj), when
// its other point is still in another component: a real outgoing edge, so
// its exact d2 (rounded up) bounds the component's lightest one too; this is
// what keeps the bound tight for large components, whose rows see only
// their own component among their near tiles.
__global__ void k_pr_comp_ub(const float *__restrict__ tu, const int32_t *__restrict__ permp,
                             const int32_t *__restrict__ comp, const float *__restrict__ rsq,
                             const unsigned int *__restrict__ nmax_bits, const double *__restrict__ rowd2,
                             const int32_t *__restrict__ rowj, int64_t n_pad, float eps_rep,
                             unsigned int *__restrict__ cub, const int32_t *counters) {
    if (!pr_active(counters)) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const int32_t i = permp[r];
    if (i < 0) return;
    const int32_t ci = comp[i];
    float ub = INFINITY;
    const float U = fminf(tu[r], tu[n_pad + r]);
    if (U < INFINITY) {
        const float smax = __fsqrt_ru(__uint_as_float(*nmax_bits));
        const float w = __fmul_ru(eps_rep, __fadd_ru(rsq[r], smax));
        const float a1 = __fadd_ru(__fsqrt_ru(fmaxf(U, 0.0f)), w);
        ub = __fmul_ru(__fmul_ru(a1, a1), 1.00001f);
    }
    const int32_t j = rowj[i];
    if (j >= 0 && comp[j] != ci) {
        const double d2 = rowd2[i];
        if (d2 < INFINITY) ub = fminf(ub, __double2float_ru(d2));
    }
    if (ub < INFINITY) atomicMin(cub + ci, __float_as_uint(ub));   // non-negative: bits are monotone
}

// Per tile: the largest bound over its rows' components (+inf when one has
// none) and its single component (-1 when its rows span several).
__global__ void __launch_bounds__(128) k_pr_tile_mu(const int32_t *__restrict__ permp,
                                                    const int32_t *__restrict__ comp,
                                                    const unsigned int *__restrict__ cub, float *__restrict__ tmu,
                                                    int32_t *__restrict__ tcomp, const int32_t *counters) {
    if (!pr_active(counters)) return;
    __shared__ unsigned int smu[4];
    __shared__ int32_t smn[4], smx[4];
    const int64_t t = blockIdx.x;
    const int32_t i = permp[t * PR_BM + threadIdx.x];
    unsigned int u = 0;
    int32_t cmn = INT32_MAX, cmx = INT32_MIN;
    if (i >= 0) {
        const int32_t c = comp[i];
        u = cub[c];
        cmn = cmx = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
        cmn = min(cmn, __shfl_xor_sync(0xffffffffu, cmn, o));
        cmx = max(cmx, __shfl_xor_sync(0xffffffffu, cmx, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { smu[w] = u; smn[w] = cmn; smx[w] = cmx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 4; ++q) { u = max(u, smu[q]); cmn = min(cmn, smn[q]); cmx = max(cmx, smx[q]); }
        tmu[t] = u >= 0x7f800000u ? INFINITY : __uint_as_float(u);
        tcomp[t] = cmn == cmx ? cmn : -1;
    }
}

// Far items of row tile R: the runs of column tiles outside the near window
// that can hold a lightest edge.  Beyond PRUNE_SLOTS - 1 runs, the runs
// separated by the smallest gaps are joined (their gap tiles swept too);
// then, while slots are left, the longest run is halved (balance).  Unused
// slots get empty items (their candidate lists are written empty).
constexpr int PR_RUNCAP = 256;             // runs kept per row tile (more: joined as found)
__global__ void __launch_bounds__(256) k_pr_far_items(const float *__restrict__ tlb2, const float *__restrict__ tmu,
                                                      const int32_t *__restrict__ tcomp, int64_t T,
                                                      int4 *__restrict__ items_b, unsigned long long *swept,
                                                      int32_t *__restrict__ nlists, const int32_t *counters) {
    if (!pr_active(counters)) return;
    extern __shared__ uint32_t keep[];                       // ceil(T / 32) words
    __shared__ int32_t rs[PR_RUNCAP], re[PR_RUNCAP];
    const int64_t R = blockIdx.x;
    const float mu = tmu[R];
    const int32_t cr = tcomp[R];
    const int64_t nw = (T + 31) / 32;
    for (int64_t w = threadIdx.x >> 5; w < nw; w += blockDim.x >> 5) {
        const int64_t C = w * 32 + (threadIdx.x & 31);
        bool k = false;
        if (C < T && (C < R - PRUNE_NEAR || C > R + PRUNE_NEAR))
            k = !(cr >= 0 && tcomp[C] == cr) && tlb2[R * T + C] <= mu;
        const uint32_t m = __ballot_sync(0xffffffffu, k);
        if ((threadIdx.x & 31) == 0) keep[w] = m;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    constexpr int NS = PRUNE_SLOTS - 1;
    // runs of kept tiles
    int nr = 0;
    int64_t C = 0;
    while (C < T) {
        int64_t w = C >> 5;
        uint32_t m = keep[w] & (0xffffffffu << (C & 31));
        while (!m && ++w < nw) m = keep[w];
        if (!m) break;
        const int64_t s0 = w * 32 + (__ffs(m) - 1);
        int64_t e = s0;
        w = e >> 5;
        uint32_t z = ~keep[w] & (0xffffffffu << (e & 31));
        while (!z && ++w < nw) z = ~keep[w];
        e = z ? w * 32 + (__ffs(z) - 1) : nw * 32;
        if (e > T) e = T;
        if (nr == PR_RUNCAP) re[nr - 1] = (int32_t)e;       // (full: joined to the last run)
        else { rs[nr] = (int32_t)s0; re[nr] = (int32_t)e; ++nr; }
        C = e;
    }
    if (nr > NS - 1) {
        // the smallest gap g such that joining every gap <= g leaves <= NS - 1
        // runs (one slot stays free: a joined run may straddle the near window)
        int32_t lo = 0, hi = (int32_t)T;
        while (lo < hi) {
            const int32_t g = lo + (hi - lo) / 2;
            int cnt = 1;
            for (int q = 1; q < nr; ++q) cnt += (rs[q] - re[q - 1] > g) ? 1 : 0;
            if (cnt <= NS - 1) hi = g; else lo = g + 1;
        }
        int k = 0;
        for (int q = 1; q < nr; ++q) {
            if (rs[q] - re[k] > lo) { ++k; rs[k] = rs[q]; re[k] = re[q]; }
            else re[k] = re[q];
        }
        nr = k + 1;
        // the near window is swept already (slot 0): cut it out of the run
        // that straddles it (its columns would be candidates twice)
        const int32_t w0 = (int32_t)(R - PRUNE_NEAR), w1 = (int32_t)(R + PRUNE_NEAR + 1);
        for (int q = 0; q < nr; ++q) {
            if (rs[q] < w0 && re[q] > w1) {
                rs[nr] = w1; re[nr] = re[q]; re[q] = w0;
                ++nr;
                break;
            }
        }
    }
    // balance: halve the longest run while slots are left and it is long
    while (nr < NS) {
        int b = -1;
        int32_t bl = 32;
        for (int q = 0; q < nr; ++q)
            if (re[q] - rs[q] > bl) { bl = re[q] - rs[q]; b = q; }
        if (b < 0) break;
        const int32_t mid = rs[b] + bl / 2;
        rs[nr] = mid; re[nr] = re[b]; re[b] = mid;
        ++nr;
    }
    int4 *out = items_b + R * NS;
    int64_t cnt = (R + PRUNE_NEAR + 1 < T ? R + PRUNE_NEAR + 1 : T) - (R - PRUNE_NEAR > 0 ? R - PRUNE_NEAR : 0);
    for (int q = 0; q < NS; ++q) {
        if (q < nr) {
            out[q] = make_int4((int)R, rs[q], re[q], q + 1);
            cnt += re[q] - rs[q];
        } else {
            out[q] = make_int4((int)R, 0, 0, q + 1);
        }
    }
    // tile pairs this row tile sweeps this round, near window included;
    // its rows' candidates are in the lists of slot 0 and of the nr items
    atomicAdd(swept, (unsigned long long)cnt);
    nlists[R] = 2 * (1 + nr);
}
}  // namespace

void prune_set_mode(int mode) { g_prune_mode.store(mode); }
int prune_mode() { return g_prune_mode.load(); }

bool prune_wanted(int64_t n, int32_t d) {
    const int mode = g_prune_mode.load();
    const int64_t nt = ceil_div(n, PR_BM);
    // supported: rows of at most 256 dimensions, a multiple of 4 (the
    // order's sample search stages 32 rows in shared memory and reads rows by
    // 16 bytes), at least 64 points
    if (mode == 0 || nt > 16384 || n < 64 || d > 256 || d % 4) return false;
    if (mode == 1) return true;
    // tile bounds separate little in many dimensions; below ~64k points the
    // order and bounds cost more than the pruned tile pairs save
    return d <= 256 && n >= 65536;
}

static cudaError_t prune_geometry(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s);

// recursive bisection of positions [0, m) of T.perm (whole tiles from 0)
static cudaError_t prune_bisect(TcScratch &T, const float *X, int64_t m, int32_t d, cudaStream_t s) {
    const int64_t nt = ceil_div(m, PR_BM);
    const unsigned g = (unsigned)ceil_div(m, 256);                 // a thread per position
    int levels = 0;
    while (((int64_t)1 << levels) < nt) ++levels;
    cudaError_t e;
    unsigned long long *far0 = T.far, *far1 = T.far + 2 * nt;
    for (int l = 0; l < levels; ++l) {
        if ((e = cudaMemsetAsync(T.far, 0, sizeof(unsigned long long) * 4 * nt, s))) return e;
        k_pr_far<0><<<g, 256, 0, ISO_S(s)>>>(X, m, d, T.perm, nt, l, nullptr, far0);
        k_pr_far<1><<<g, 256, 0, ISO_S(s)>>>(X, m, d, T.perm, nt, l, far0, far1);
        k_pr_keys<<<g, 256, 0, ISO_S(s)>>>(X, m, d, T.perm, nt, l, far0, far1, T.keys);
        // stable: ties keep the previous level's order
        if ((e = sort_pairs_u64(T.keys, T.perm, T.kbuf, T.vbuf, m, s))) return e;
    }
    return cudaGetLastError();
}

cudaError_t prune_reorder(TcScratch &T, double *rowd2, const float *X, int64_t n, int32_t d, cudaStream_t s) {
    cudaError_t e;
    const unsigned g = (unsigned)ceil_div(n, 256);
    // the isolation proxy (into rowd2, free before the first round)
    const int nsamp = (int)((n < PR_SAMPLES ? n : PR_SAMPLES) & ~(int64_t)31);
    if (nsamp < 32) return cudaErrorInvalidValue;           // (prune_wanted: n >= 64)
    if (d % 4) return cudaErrorInvalidValue;                  // (prune_wanted: rows of 4k floats)
    k_pr_sample_nn<<<g, 256, sizeof(float) * 32 * d, ISO_S(s)>>>(X, n, d, n / nsamp, nsamp, rowd2);
    // the median nearest-neighbour d2, then isolated points last
    k_pr_nn_keys<<<g, 256, 0, ISO_S(s)>>>(rowd2, n, T.keys, T.perm);
    if ((e = sort_pairs_u64(T.keys, T.perm, T.kbuf, T.vbuf, n, s))) return e;
    if ((e = cudaMemsetAsync(T.far, 0, sizeof(unsigned long long), s))) return e;
    k_pr_far_keys<<<g, 256, 0, ISO_S(s)>>>(rowd2, n, T.keys, T.kbuf, T.perm, T.far);
    if ((e = cudaMemcpyAsync(T.keys, T.kbuf, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s))) return e;
    unsigned long long nfar = 0;
    if ((e = cudaMemcpyAsync(&nfar, T.far, sizeof(nfar), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = sort_pairs_u64(T.keys, T.perm, T.kbuf, T.vbuf, n, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    const int64_t m = n - (int64_t)nfar;
    if (m > 1 && (e = prune_bisect(T, X, m, d, s))) return e;
    if ((e = tc_place_rows(T, X, n, d, s))) return e;
    if ((e = prune_geometry(T, X, n, d, s))) return e;
    T.prune_ready = true;
    return cudaGetLastError();
}

static cudaError_t prune_geometry(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s) {
    const int64_t nt = T.n_pad / PR_BM;
    (void)n;
    k_pr_geom<<<(unsigned)nt, 128, sizeof(float) * d, ISO_S(s)>>>(X, d, T.permp, T.tcen, T.trad);
    k_pr_lb<<<dim3((unsigned)ceil_div(nt, 128), (unsigned)nt), 128, sizeof(float) * d, ISO_S(s)>>>(T.tcen, T.trad, nt,
                                                                                                 d, T.tlb2);
    k_pr_near<<<(unsigned)ceil_div(nt, 128), 128, 0, ISO_S(s)>>>(nt, T.items_a);
    return cudaGetLastError();
}

cudaError_t prune_far_items(TcScratch &T, const int32_t *comp, const double *rowd2, const int32_t *rowj, int64_t n,
                            const int32_t *counters, cudaStream_t s) {
    const int64_t nt = T.n_pad / PR_BM;
    (void)n;
    cudaError_t e;
    if ((e = cudaMemsetAsync(T.cub, 0xff, sizeof(unsigned int) * n, s))) return e;
    const double eps_rep = 1.25 * (3.814697265625e-06 + 5.9604644775390625e-08);
    k_pr_comp_ub<<<(unsigned)ceil_div(T.n_pad, 256), 256, 0, ISO_S(s)>>>(T.tu, T.permp, comp, T.rsq, T.nmax_bits,
                                                                        rowd2, rowj, T.n_pad,
                                                                        (float)(eps_rep * 1.0001), T.cub, counters);
    k_pr_tile_mu<<<(unsigned)nt, 128, 0, ISO_S(s)>>>(T.permp, comp, T.cub, T.tmu, T.tcomp, counters);
    k_pr_far_items<<<(unsigned)nt, 256, sizeof(uint32_t) * ceil_div(nt, 32), ISO_S(s)>>>(T.tlb2, T.tmu, T.tcomp, nt,
                                                                                       T.items_b, T.swept, T.nlists,
                                                                                       counters);
    return cudaGetLastError();
}

}  // namespace iso

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

// The lanes of an 8-lane group hold parts of one sum.
__device__ __forceinline__ float group8_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

__device__ __forceinline__ float4 f4sub(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}

// order-preserving bits of a float
__device__ __forceinline__ uint32_t pr_fbits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The levels whose nodes hold more than PR_LOC_TILES tiles run over all
// positions at once (PR_GB positions per block; a block meets at most two
// nodes, which hold more than PR_LOC positions each); the nodes of the first
// level below that are finished one per block, every further level inside
// shared memory.
constexpr int PR_LOC_TILES = 16;
constexpr int PR_LOC = PR_LOC_TILES * PR_BM;             // positions of a node finished by one block
constexpr int PR_LOC_THREADS = 512;
constexpr int PR_GB = 256;

// PASS 0: farthest point of each node from its first point; PASS 1: from
// that point.  far[node] = max (d2 bits, index).  8 lanes per position
// (16-byte loads of its row split over the lanes), 4 positions per lane
// group in flight; the block's nodes fold in shared memory, then one atomic
// per node.
template <int PASS>
__global__ void __launch_bounds__(256) k_pr_far(const float *__restrict__ X, int64_t n, int32_t d,
                                                const int32_t *__restrict__ perm, int64_t T, int l,
                                                const unsigned long long *__restrict__ far0,
                                                unsigned long long *__restrict__ far) {
    __shared__ unsigned long long sm[2];
    const int64_t p0 = (int64_t)blockIdx.x * PR_GB;
    int64_t a0, b0;
    const uint32_t id0 = pr_node(p0 / PR_BM, T, l, a0, b0);
    if (threadIdx.x < 2) sm[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 3, sub = lane & 7, warp = threadIdx.x >> 5;
    const int d4 = d >> 2;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    for (int h = 0; h < 2; ++h) {                            // warp w: positions p0 + 32 w + 16 h + g + 4 u
        int64_t ii[4], ref[4];
        uint32_t id[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + 32 * warp + 16 * h + g + 4 * u;
            ok[u] = p < n;
            id[u] = id0;
            ii[u] = 0;
            ref[u] = 0;
            if (ok[u]) {
                int64_t a, b;
                id[u] = pr_node(p / PR_BM, T, l, a, b);
                ok[u] = b - a > 1;
                ii[u] = perm[p];
                ref[u] = PASS == 0 ? (int64_t)perm[a * PR_BM] : (int64_t)(uint32_t)(far0[id[u]] & 0xffffffffull);
            }
        }
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int t = sub; t < d4; t += 8) {
            float4 x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = X4[ii[u] * d4 + t];
                y[u] = X4[ref[u] * d4 + t];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 df = f4sub(x[u], y[u]);
                acc[u] = dot4(df, df, acc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = group8_sum(acc[u]);
        if (sub == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!ok[u]) continue;
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(acc[u]) << 32) | (unsigned long long)(uint32_t)ii[u];
                if (id[u] - id0 < 2) atomicMax(&sm[id[u] - id0], key);
                else atomicMax(far + id[u], key);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 && sm[threadIdx.x]) atomicMax(far + id0 + threadIdx.x, sm[threadIdx.x]);
}

// sort key of position p: (node, projection on the node's far pair's line)
__global__ void __launch_bounds__(256) k_pr_keys(const float *__restrict__ X, int64_t n, int32_t d,
                                                 const int32_t *__restrict__ perm, int64_t T, int l,
                                                 const unsigned long long *__restrict__ far0,
                                                 const unsigned long long *__restrict__ far1,
                                                 uint64_t *__restrict__ keys) {
    const int64_t p0 = (int64_t)blockIdx.x * PR_GB;
    const int lane = threadIdx.x & 31, g = lane >> 3, sub = lane & 7, warp = threadIdx.x >> 5;
    const int d4 = d >> 2;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    for (int h = 0; h < 2; ++h) {
        int64_t ii[4], rb[4], rc[4];
        uint32_t id[4];
        bool ok[4], split[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + 32 * warp + 16 * h + g + 4 * u;
            ok[u] = p < n;
            split[u] = false;
            id[u] = 0;
            ii[u] = rb[u] = rc[u] = 0;
            if (ok[u]) {
                int64_t a, b;
                id[u] = pr_node(p / PR_BM, T, l, a, b);
                ii[u] = perm[p];
                split[u] = b - a > 1;
                if (split[u]) {
                    rb[u] = (int64_t)(uint32_t)(far0[id[u]] & 0xffffffffull);
                    rc[u] = (int64_t)(uint32_t)(far1[id[u]] & 0xffffffffull);
                }
            }
        }
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int t = sub; t < d4; t += 8) {
            float4 x[4], xb[4], xc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = X4[ii[u] * d4 + t];
                xb[u] = X4[rb[u] * d4 + t];
                xc[u] = X4[rc[u] * d4 + t];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = dot4(f4sub(x[u], xb[u]), f4sub(xc[u], xb[u]), acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = group8_sum(acc[u]);
        if (sub == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!ok[u]) continue;
                const int64_t p = p0 + 32 * warp + 16 * h + g + 4 * u;
                keys[p] = ((uint64_t)id[u] << 32) | (uint64_t)pr_fbits(split[u] ? acc[u] : 0.0f);
            }
        }
    }
}

// tile range [a, b) of node s `depth` halvings below [a, b)
__device__ __forceinline__ void pr_sub(int64_t &a, int64_t &b, int depth, uint32_t s) {
    for (int k = depth - 1; k >= 0; --k) {
        const int64_t m = a + (b - a) / 2;
        if ((s >> k) & 1u) a = m;
        else b = m;
    }
}

// bitonic sort of P2 (a power of two) keys in shared memory by the block
__device__ void pr_bitonic(uint64_t *sk, int P2) {
    for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int x = i ^ j;
                if (x > i) {
                    const uint64_t a = sk[i], b = sk[x];
                    if ((a > b) == ((i & k) == 0)) {
                        sk[i] = b;
                        sk[x] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// The levels L0 .. levels-1 of the node of level L0 with index blockIdx.x
// (at most PR_LOC_TILES tiles, so at most 4 levels and 8 sub-nodes), in
// shared memory: per level the two far-point passes and the projections,
// then a sort by (sub-node, projection, previous position) - the stable
// order of the global levels' sort.
__global__ void __launch_bounds__(PR_LOC_THREADS) k_pr_local(const float *__restrict__ X, int64_t m, int32_t d,
                                                             int32_t *__restrict__ perm, int64_t T, int L0,
                                                             int levels) {
    extern __shared__ __align__(16) unsigned char pr_sm[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(pr_sm);                            // [PR_LOC]
    int32_t *sva = reinterpret_cast<int32_t *>(skey + PR_LOC);                        // [PR_LOC]
    int32_t *svb = sva + PR_LOC;                                                       // [PR_LOC]
    unsigned long long *sfar = reinterpret_cast<unsigned long long *>(svb + PR_LOC);  // [2][PR_LOC_TILES]
    float *srow = reinterpret_cast<float *>(sfar + 2 * PR_LOC_TILES);                 // [2][PR_LOC_TILES][d]
    int64_t na = 0, nb = T;
    pr_sub(na, nb, L0, blockIdx.x);
    const int64_t base = na * PR_BM;
    const int64_t end = nb * PR_BM < m ? nb * PR_BM : m;
    const int cnt = end > base ? (int)(end - base) : 0;
    if (cnt == 0) return;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) sva[q] = perm[base + q];
    int P2 = 1;
    while (P2 < cnt) P2 <<= 1;
    const int lane = threadIdx.x & 31, g = lane >> 3, sub = lane & 7, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5, d4 = d >> 2;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    const float4 *R4 = reinterpret_cast<const float4 *>(srow);
    __syncthreads();
    for (int l = L0; l < levels; ++l) {
        const int depth = l - L0, nsub = 1 << depth;
        // pass 0: d2 to the sub-node's first point (reference row in slot 0);
        // pass 1: to its farthest (slot 1); pass 2: the projection on the
        // line from the pass-1 point (slot 1) to the pass-2 point (slot 0)
        for (int pass = 0; pass < 3; ++pass) {
            const int slot = pass == 1 ? 1 : 0;
            for (int e = threadIdx.x; e < nsub * d; e += blockDim.x) {
                const int sn = e / d, t = e - sn * d;
                int64_t sa = na, sb = nb;
                pr_sub(sa, sb, depth, (uint32_t)sn);
                int64_t ref = -1;
                if (sb - sa > 1 && sa * PR_BM < end)
                    ref = pass == 0 ? (int64_t)sva[(sa - na) * PR_BM]
                                    : (int64_t)(uint32_t)(sfar[(pass - 1) * PR_LOC_TILES + sn] & 0xffffffffull);
                srow[(slot * PR_LOC_TILES + sn) * d + t] = ref >= 0 ? X[ref * d + t] : 0.0f;
            }
            if (pass < 2)
                for (int sn = threadIdx.x; sn < nsub; sn += blockDim.x) sfar[pass * PR_LOC_TILES + sn] = 0;
            __syncthreads();
            for (int q0 = warp * 16; q0 < cnt; q0 += nwarps * 16) {     // (warp-uniform)
                int64_t ii[4];
                int ss[4];
                bool ok[4], split[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + g + 4 * u;
                    ok[u] = q < cnt;
                    ii[u] = ok[u] ? sva[q] : sva[0];
                    int64_t sa = na, sb = nb;
                    uint32_t sn = 0;
                    const int64_t t = na + (ok[u] ? q : 0) / PR_BM;
                    for (int k = 0; k < depth; ++k) {
                        const int64_t mid = sa + (sb - sa) / 2;
                        if (t < mid) { sb = mid; sn = 2 * sn; }
                        else { sa = mid; sn = 2 * sn + 1; }
                    }
                    ss[u] = (int)sn;
                    split[u] = sb - sa > 1;
                }
                float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                for (int t = sub; t < d4; t += 8) {
                    float4 x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) x[u] = X4[ii[u] * d4 + t];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 r = R4[(slot * PR_LOC_TILES + ss[u]) * d4 + t];
                        if (pass < 2) {
                            const float4 df = f4sub(x[u], r);
                            acc[u] = dot4(df, df, acc[u]);
                        } else {
                            const float4 xb = R4[(PR_LOC_TILES + ss[u]) * d4 + t];
                            acc[u] = dot4(f4sub(x[u], xb), f4sub(r, xb), acc[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = group8_sum(acc[u]);
                if (sub == 0) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (!ok[u]) continue;
                        const int q = q0 + g + 4 * u;
                        if (pass < 2) {
                            if (split[u])
                                atomicMax(&sfar[pass * PR_LOC_TILES + ss[u]],
                                          ((unsigned long long)__float_as_uint(acc[u]) << 32) |
                                              (unsigned long long)(uint32_t)ii[u]);
                        } else {
                            skey[q] = ((uint64_t)ss[u] << 44) | ((uint64_t)pr_fbits(split[u] ? acc[u] : 0.0f) << 12) |
                                      (uint64_t)q;
                        }
                    }
                }
            }
            __syncthreads();
        }
        for (int q = cnt + threadIdx.x; q < P2; q += blockDim.x) skey[q] = ~0ull;
        __syncthreads();
        pr_bitonic(skey, P2);
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) svb[q] = sva[skey[q] & 0xfffu];
        __syncthreads();
        int32_t *tmp = sva; sva = svb; svb = tmp;
    }
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) perm[base + q] = sva[q];
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

// The isolation threshold: 16x the median of the proxy over an evenly
// spaced subsample of at most PR_MED points (a bitonic sort in shared
// memory by one block); +inf when that median is 0.
constexpr int PR_MED = 4096;
__global__ void __launch_bounds__(1024) k_pr_median(const double *__restrict__ rowd2, int64_t n,
                                                    unsigned long long *__restrict__ tau_bits) {
    __shared__ uint64_t sk[PR_MED];
    const int S = (int)(n < PR_MED ? n : PR_MED);
    int P2 = 1;
    while (P2 < S) P2 <<= 1;
    for (int q = threadIdx.x; q < P2; q += blockDim.x)             // non-negative: bits are monotone
        sk[q] = q < S ? (uint64_t)__double_as_longlong(rowd2[(int64_t)q * n / S]) : ~0ull;
    __syncthreads();
    pr_bitonic(sk, P2);
    if (threadIdx.x == 0) {
        const double med = __longlong_as_double((long long)sk[S / 2]);
        *tau_bits = (unsigned long long)__double_as_longlong(med > 0.0 ? 16.0 * med : INFINITY);
    }
}

__global__ void k_pr_flags(const double *__restrict__ rowd2, int64_t n, const unsigned long long *__restrict__ tau_bits,
                           int32_t *__restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keep[i] = rowd2[i] > __longlong_as_double((long long)*tau_bits) ? 0 : 1;
}

// points kept first, isolated ones after them, each group in index order;
// m_out = the number kept
__global__ void k_pr_partition(const int32_t *__restrict__ keep, const int32_t *__restrict__ pos, int64_t n,
                               int32_t *__restrict__ perm, unsigned long long *__restrict__ m_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t m = (int64_t)pos[n - 1] + keep[n - 1];
    perm[keep[i] ? (int64_t)pos[i] : m + (i - pos[i])] = (int32_t)i;
    if (i == 0) *m_out = (unsigned long long)m;
}

// Per tile: centroid c (FP32 mean; any c serves) and radius: an upper
// bound of every real row's distance to c, in FP32 with upward rounding
// throughout (|x - c| bounded by the larger magnitude of its two directed
// roundings, squares and sums rounded up, square root rounded up).  Warp w
// sums rows 32w .. 32w+31 (lanes over dimensions: coalesced), then a warp per
// row for the radius.
__global__ void __launch_bounds__(128) k_pr_geom(const float *__restrict__ X, int32_t d,
                                                 const int32_t *__restrict__ permp, float *__restrict__ tcen,
                                                 float *__restrict__ trad) {
    extern __shared__ float gsum[];                           // [4][d] partial sums, then [d] the centroid
    __shared__ float sr[4];
    const int64_t t = blockIdx.x;
    const int32_t *pr = permp + t * PR_BM;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cnt = __syncthreads_count(pr[threadIdx.x] >= 0);
    for (int k = lane; k < d; k += 32) {
        float sum = 0.0f;
#pragma unroll 8
        for (int q = 32 * warp; q < 32 * warp + 32; ++q) {
            const int32_t i = pr[q];
            if (i >= 0) sum += X[(int64_t)i * d + k];
        }
        gsum[warp * d + k] = sum;
    }
    __syncthreads();
    float *sc = gsum + 4 * d;
    const float inv = cnt > 0 ? 1.0f / (float)cnt : 0.0f;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        const float c = (((gsum[k] + gsum[d + k]) + gsum[2 * d + k]) + gsum[3 * d + k]) * inv;
        sc[k] = c;
        tcen[t * d + k] = c;
    }
    __syncthreads();
    float r2max = 0.0f;
    for (int q = 32 * warp; q < 32 * warp + 32; ++q) {
        const int32_t i = pr[q];
        if (i < 0) continue;                                  // (warp-uniform)
        float r2 = 0.0f;
        for (int k = lane; k < d; k += 32) {
            const float x = X[(int64_t)i * d + k], c = sc[k];
            const float df = fmaxf(fabsf(__fsub_ru(x, c)), fabsf(__fsub_rd(x, c)));
            r2 = __fmaf_ru(df, df, r2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r2 = __fadd_ru(r2, __shfl_xor_sync(0xffffffffu, r2, o));
        r2max = fmaxf(r2max, r2);
    }
    if (lane == 0) sr[warp] = r2max;
    __syncthreads();
    if (threadIdx.x == 0) trad[t] = __fsqrt_ru(fmaxf(fmaxf(sr[0], sr[1]), fmaxf(sr[2], sr[3])));
}

// LB(R, C) as a float rounded down.  The centroid distance comes from an
// FP32 sum of squared differences in dimension order (relative error below
// (d + 2) 2^-24), taken (d + 8) 2^-23 short of itself.  A block takes 32 x 32
// tile pairs, the centroids staged 64 dimensions at a time (padded rows).
constexpr int PR_LBT = 32;
__global__ void __launch_bounds__(256) k_pr_lb(const float *__restrict__ tcen, const float *__restrict__ trad,
                                               int64_t T, int32_t d, float *__restrict__ tlb2) {
    __shared__ float cr[PR_LBT][65], cc[PR_LBT][65];
    const int64_t R0 = (int64_t)blockIdx.y * PR_LBT, C0 = (int64_t)blockIdx.x * PR_LBT;
    const int r = threadIdx.x >> 3, c0 = threadIdx.x & 7;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k0 = 0; k0 < d; k0 += 64) {
        const int kc = d - k0 < 64 ? d - k0 : 64;
        __syncthreads();
        for (int e = threadIdx.x; e < PR_LBT * 64; e += blockDim.x) {
            const int q = e >> 6, k = e & 63;
            cr[q][k] = (R0 + q < T && k < kc) ? tcen[(R0 + q) * d + k0 + k] : 0.0f;
            cc[q][k] = (C0 + q < T && k < kc) ? tcen[(C0 + q) * d + k0 + k] : 0.0f;
        }
        __syncthreads();
        for (int k = 0; k < kc; ++k) {
            const float a = cr[r][k];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float df = a - cc[c0 + 8 * j][k];
                acc[j] = fmaf(df, df, acc[j]);
            }
        }
    }
    const int64_t R = R0 + r;
    if (R >= T) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t C = C0 + c0 + 8 * j;
        if (C >= T) continue;
        const double g = sqrt((double)acc[j]) * (1.0 - (double)(d + 8) * 1.1920928955078125e-07) - (double)trad[R] -
                         (double)trad[C];
        tlb2[R * T + C] = g > 0.0 ? __double2float_rd(g * g * (1.0 - 1e-9)) : 0.0f;
    }
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
    const int32_t i = r < n_pad ? permp[r] : -1;
    const int32_t ci = i >= 0 ? comp[i] : -1;
    // the lanes of one component fold first: one atomic per component and warp
    const unsigned peers = __match_any_sync(0xffffffffu, ci);
    if (i < 0) return;
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
    // non-negative: bits are monotone (+inf: 0x7f800000 leaves cub as it is)
    const unsigned m = __reduce_min_sync(peers, __float_as_uint(ub));
    if ((threadIdx.x & 31) == __ffs(peers) - 1 && m < 0x7f800000u) atomicMin(cub + ci, m);
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
    int levels = 0;
    while (((int64_t)1 << levels) < nt) ++levels;
    // L0: the first level whose nodes hold at most PR_LOC_TILES tiles (the
    // largest node of level l holds ceil(nt / 2^l) tiles)
    int L0 = 0;
    while (ceil_div(nt, (int64_t)1 << L0) > PR_LOC_TILES) ++L0;
    cudaError_t e;
    const unsigned g = (unsigned)ceil_div(m, PR_GB);
    unsigned long long *far0 = T.far, *far1 = T.far + 2 * nt;
    for (int l = 0; l < L0 && l < levels; ++l) {
        if ((e = cudaMemsetAsync(T.far, 0, sizeof(unsigned long long) * 4 * nt, s))) return e;
        k_pr_far<0><<<g, 256, 0, ISO_S(s)>>>(X, m, d, T.perm, nt, l, nullptr, far0);
        k_pr_far<1><<<g, 256, 0, ISO_S(s)>>>(X, m, d, T.perm, nt, l, far0, far1);
        k_pr_keys<<<g, 256, 0, ISO_S(s)>>>(X, m, d, T.perm, nt, l, far0, far1, T.keys);
        // stable: ties keep the previous level's order
        if ((e = sort_pairs_u64(T.keys, T.perm, T.kbuf, T.vbuf, m, s))) return e;
    }
    if (L0 < levels) {
        const size_t smem = sizeof(uint64_t) * PR_LOC + 2 * sizeof(int32_t) * PR_LOC +
                            2 * sizeof(unsigned long long) * PR_LOC_TILES + 2 * sizeof(float) * PR_LOC_TILES * d;
        if ((e = cudaFuncSetAttribute(k_pr_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_pr_local<<<1u << L0, PR_LOC_THREADS, smem, ISO_S(s)>>>(X, m, d, T.perm, nt, L0, levels);
    }
    return cudaGetLastError();
}

cudaError_t prune_reorder(TcScratch &T, double *rowd2, const float *X, int64_t n, int32_t d, cudaStream_t s) {
    cudaError_t e;
    const unsigned g = (unsigned)ceil_div(n, 256);
    // the isolation proxy (into rowd2, free before the first round)
    const int nsamp = (int)((n < PR_SAMPLES ? n : PR_SAMPLES) & ~(int64_t)31);
    if (nsamp < 32) return cudaErrorInvalidValue;           // (prune_wanted: n >= 64)
    if (d % 4 || (reinterpret_cast<uintptr_t>(X) & 15)) return cudaErrorInvalidValue;   // rows of 16-byte units
    k_pr_sample_nn<<<g, 256, sizeof(float) * 32 * d, ISO_S(s)>>>(X, n, d, n / nsamp, nsamp, rowd2);
    // isolated points last: a stable partition by the threshold (an
    // exclusive scan of the kept flags gives each kept point its position)
    k_pr_median<<<1, 1024, 0, ISO_S(s)>>>(rowd2, n, T.far);
    int32_t *keep = T.vbuf;
    int32_t *pos = reinterpret_cast<int32_t *>(T.keys);        // (keys, kbuf: 2n int32 each)
    int32_t *tmp = reinterpret_cast<int32_t *>(T.kbuf);
    k_pr_flags<<<g, 256, 0, ISO_S(s)>>>(rowd2, n, T.far, keep);
    if ((e = exclusive_scan_i32(keep, pos, n, tmp, s))) return e;
    k_pr_partition<<<g, 256, 0, ISO_S(s)>>>(keep, pos, n, T.perm, T.far + 1);
    unsigned long long mkept = 0;
    if ((e = cudaMemcpyAsync(&mkept, T.far + 1, sizeof(mkept), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    const int64_t m = (int64_t)mkept;
    if (m < 0 || m > n) return cudaErrorUnknown;
    if (m > 1 && (e = prune_bisect(T, X, m, d, s))) return e;
    if ((e = tc_place_rows(T, X, n, d, s))) return e;
    if ((e = prune_geometry(T, X, n, d, s))) return e;
    T.prune_ready = true;
    return cudaGetLastError();
}

static cudaError_t prune_geometry(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s) {
    const int64_t nt = T.n_pad / PR_BM;
    (void)n;
    const size_t gsm = sizeof(float) * 5 * d;
    k_pr_geom<<<(unsigned)nt, 128, gsm, ISO_S(s)>>>(X, d, T.permp, T.tcen, T.trad);
    const unsigned gl = (unsigned)ceil_div(nt, PR_LBT);
    k_pr_lb<<<dim3(gl, gl), 256, 0, ISO_S(s)>>>(T.tcen, T.trad, nt, d, T.tlb2);
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

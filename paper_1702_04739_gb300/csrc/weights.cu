// weights.cu -- eq. omega and eq. potential on all pairs, FP64-grade.
//
// omega_i = sum_{j != i} exp(-||x_i - x_j|| / sigma) needs every term to
// ~1e-14 relative, because i_k inherits omega's error.  GB300's FP64 pipe
// runs at a small fraction of its FP32 rate, so for FP32 input every pair is
// evaluated in double-word ("double-float") FP32 arithmetic:
//   * the difference a - b is made exact by TwoSum (Knuth), its square by
//     TwoProd with FMA (Dekker), and the d2 sum is a renormalised
//     double-word accumulation (Joldes, Muller, Popescu 2017);
//   * sqrt by one Newton correction of the correctly rounded FP32 root;
//   * exp by table-driven argument reduction (Tang 1989): z = k ln2/64 + r
//     with a three-part ln2/64, |r| <= ln2/128, a degree-5 Taylor polynomial
//     whose r^2/2 term is double-word, and a 64-entry 2^(-j/64) table.
// Each row is shifted by its nearest-neighbour distance, so the terms of a
// row are exp(-(y_ij - y_i,nn)) <= 1 and the row sum stays inside FP32's
// range; omega_i = exp(-y_i,nn) * sum is formed in FP64 at the end.
// Rows are owned by threads (4x4 pairs per thread, 64x64 tiles), so each
// row's sum has a fixed order: the result is deterministic.
// FP64 input uses a plain FP64 kernel with the reference summation order.
#include <math.h>

#include "common.cuh"
#include "dwmath.cuh"

namespace iso {


ExpTable make_exp_table() {
    ExpTable T;
    for (int j = 0; j < 64; ++j) {
        double v = exp2(-(double)j / 64.0);
        float hi = (float)v;
        float lo = (float)(v - (double)hi);
        T.t[j] = make_float2(hi, lo);
    }
    return T;
}

namespace {
constexpr int TPB = 256;
constexpr int WT = 64;        // rows / columns per tile
constexpr int WDC = 32;       // dims per shared-memory chunk
constexpr int WPAD = WT + 4;
constexpr int GR_DCH = (WDC * WPAD) / 2;    // dimensions of D per chunk (a double-word each, in As)
constexpr int GR_FCAP = (WDC * WPAD) / 2;   // cancelling pairs per round (indices in Bs, results in As)

struct RowAcc {
    float wh, wl, ph, pl;
};

// SCREEN: before the double-word pass, each 64x64 tile pair is evaluated in
// plain FP32; if no pair can have a term above e^-zskip of its row's
// largest term (a rigorous lower bound on z from the FP32 error bound), the
// tile pair is skipped.  Skipped terms total < n e^-zskip relative.
template <bool WITH_P, bool SCREEN>
__global__ void __launch_bounds__(TPB, 2)
k_weights_dw(const float *__restrict__ X, int64_t n, int32_t d, const unsigned long long *__restrict__ nnbits,
             float is_h, float is_l, double inv_sigma, ExpTable tabv, double alpha, int include_self,
             float zskip, float scr_shrink, double *__restrict__ omega, double *__restrict__ pout,
             unsigned long long *__restrict__ tile_counts) {
    __shared__ __align__(16) float As[WDC][WPAD];
    __shared__ __align__(16) float Bs[WDC][WPAD];
    __shared__ float2 tab[64];
    __shared__ float mw[WT][17][2];
    __shared__ float mp[WITH_P ? WT : 1][17][2];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * WT;
    if (tid < 64) tab[tid] = tabv.t[tid];

    float sh_h[4], sh_l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = row0 + ty * 4 + i;
        double sh = 0.0;
        if (r < n) {
            double nd2 = bitsd(nnbits[r]);
            sh = isfinite(nd2) ? __dmul_rn(__dsqrt_rn(nd2), inv_sigma) : 0.0;
        }
        sh_h[i] = (float)sh;
        sh_l[i] = (float)(sh - (double)sh_h[i]);
    }
    RowAcc acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = RowAcc{0.f, 0.f, 0.f, 0.f};

    const int64_t ntiles = ceil_div(n, WT);
    unsigned long long dw_tiles = 0;
    for (int64_t ct = 0; ct < ntiles; ++ct) {
        const int64_t col0 = ct * WT;
        if (SCREEN) {
            float A32[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) A32[i][j] = 0.f;
            for (int t0 = 0; t0 < d; t0 += WDC) {
                __syncthreads();
#pragma unroll
                for (int q = 0; q < (WT * WDC) / TPB; ++q) {
                    int idx = tid + q * TPB;
                    int r = idx / WDC, t = idx % WDC;
                    int64_t gr = row0 + r, gc = col0 + r;
                    int gt = t0 + t;
                    As[t][r] = (gr < n && gt < d) ? X[gr * d + gt] : 0.0f;
                    Bs[t][r] = (gc < n && gt < d) ? X[gc * d + gt] : 0.0f;
                }
                __syncthreads();
                const int tl = min(WDC, d - t0);
                for (int t = 0; t < tl; ++t) {
                    float4 a4 = *reinterpret_cast<const float4 *>(&As[t][ty * 4]);
                    float4 b4 = *reinterpret_cast<const float4 *>(&Bs[t][tx * 4]);
                    float a[4] = {a4.x, a4.y, a4.z, a4.w};
                    float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float df = __fsub_rn(a[i], b[j]);
                            A32[i][j] = __fmaf_rn(df, df, A32[i][j]);
                        }
                }
            }
            int need = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t gr = row0 + ty * 4 + i;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t gc = col0 + tx * 4 + j;
                    if (gr >= n || gc >= n || gc == gr) continue;
                    // d >= sqrt(d2_fp32 * (1 - e)): z >= d / sigma - y_nn
                    float zlo = __fmul_rn(__fsqrt_rn(__fmul_rn(A32[i][j], scr_shrink)), is_h) - sh_h[i];
                    if (!(zlo > zskip)) need = 1;
                }
            }
            if (!__syncthreads_or(need)) continue;
            ++dw_tiles;
        }
        float S[4][4], E[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { S[i][j] = 0.f; E[i][j] = 0.f; }
        for (int t0 = 0; t0 < d; t0 += WDC) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < (WT * WDC) / TPB; ++q) {
                int idx = tid + q * TPB;
                int r = idx / WDC, t = idx % WDC;
                int64_t gr = row0 + r, gc = col0 + r;
                int gt = t0 + t;
                As[t][r] = (gr < n && gt < d) ? X[gr * d + gt] : 0.0f;
                Bs[t][r] = (gc < n && gt < d) ? X[gc * d + gt] : 0.0f;
            }
            __syncthreads();
            const int tl = min(WDC, d - t0);
            for (int t = 0; t < tl; ++t) {
                float4 a4 = *reinterpret_cast<const float4 *>(&As[t][ty * 4]);
                float4 b4 = *reinterpret_cast<const float4 *>(&Bs[t][tx * 4]);
                float a[4] = {a4.x, a4.y, a4.z, a4.w};
                float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float s, e;
                        two_sum(a[i], -b[j], s, e);               // exact a - b
                        float p = __fmul_rn(s, s);
                        float q2 = __fmaf_rn(s, s, -p);             // exact s^2 = p + q2
                        q2 = __fmaf_rn(__fadd_rn(s, s), e, q2);     // + 2 s e
                        float hs, he;
                        two_sum(S[i][j], p, hs, he);
                        he = __fadd_rn(he, __fadd_rn(E[i][j], q2));
                        fast_two_sum(hs, he, S[i][j], E[i][j]);
                    }
            }
        }
        // epilogue: sqrt, /sigma, shift, exp, row accumulation
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t gr = row0 + ty * 4 + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t gc = col0 + tx * 4 + j;
                if (gr >= n || gc >= n || gc == gr) continue;
                const float Sh = S[i][j], El = E[i][j];
                float r = __fsqrt_rn(Sh);
                float dl = 0.0f;
                if (r > 0.0f) {
                    float res = __fadd_rn(__fmaf_rn(-r, r, Sh), El);
                    dl = __fmul_rn(res, __frcp_rn(__fadd_rn(r, r)));
                }
                if (WITH_P) dw_add(acc[i].ph, acc[i].pl, r, dl);
                float yh, yl;
                two_prod(r, is_h, yh, yl);
                yl = __fmaf_rn(r, is_l, yl);
                yl = __fmaf_rn(dl, is_h, yl);
                fast_two_sum(yh, yl, yh, yl);
                float zh, zl;
                two_sum(yh, -sh_h[i], zh, zl);
                zl = __fadd_rn(zl, __fsub_rn(yl, sh_l[i]));
                fast_two_sum(zh, zl, zh, zl);
                if (zh > zskip) continue;      // < e^-zskip of the row's largest term
                float th, tl2;
                dw_exp_neg(zh, zl, tab, th, tl2);
                dw_add(acc[i].wh, acc[i].wl, th, tl2);
            }
        }
    }
    if (SCREEN && tid == 0) {
        atomicAdd(tile_counts + 0, (unsigned long long)ntiles);
        atomicAdd(tile_counts + 1, dw_tiles);
    }
    // merge the 16 column-threads of each row in fixed order
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        mw[ty * 4 + i][tx][0] = acc[i].wh;
        mw[ty * 4 + i][tx][1] = acc[i].wl;
        if (WITH_P) {
            mp[ty * 4 + i][tx][0] = acc[i].ph;
            mp[ty * 4 + i][tx][1] = acc[i].pl;
        }
    }
    __syncthreads();
    if (tid < WT) {
        const int64_t r = row0 + tid;
        if (r < n) {
            float h = 0.f, l = 0.f, qh = 0.f, ql = 0.f;
            for (int s = 0; s < 16; ++s) {
                dw_add(h, l, mw[tid][s][0], mw[tid][s][1]);
                if (WITH_P) dw_add(qh, ql, mp[tid][s][0], mp[tid][s][1]);
            }
            // the shift actually applied to this row's terms was the
            // double-word (fh, fl) of sh; fh + fl is exact in FP64
            double nd2 = bitsd(nnbits[r]);
            double sh = isfinite(nd2) ? __dmul_rn(__dsqrt_rn(nd2), inv_sigma) : 0.0;
            const float fh = (float)sh;
            const float fl = (float)(sh - (double)fh);
            double scale = exp(-__dadd_rn((double)fh, (double)fl));
            double w = __dmul_rn(scale, __dadd_rn((double)h, (double)l));
            if (include_self) w = __dadd_rn(w, 1.0);
            omega[r] = w;
            if (WITH_P && pout) pout[r] = __dmul_rn(alpha, __dadd_rn((double)qh, (double)ql));
        }
    }
}

// exp(-(d / sigma - shift)) for a double-word distance (r, dl); false when
// the term is below e^-zskip of the row's largest term (dropped).
__device__ __forceinline__ bool dw_term(float r, float dl, float is_h, float is_l, float sh_h, float sh_l, float zskip,
                                        const float2 *__restrict__ tab, float &th, float &tl) {
    float yh, yl;
    two_prod(r, is_h, yh, yl);
    yl = __fmaf_rn(r, is_l, yl);
    yl = __fmaf_rn(dl, is_h, yl);
    fast_two_sum(yh, yl, yh, yl);
    float zh, zl;
    two_sum(yh, -sh_h, zh, zl);
    zl = __fadd_rn(zl, __fsub_rn(yl, sh_l));
    fast_two_sum(zh, zl, zh, zl);
    if (zh > zskip) return false;
    dw_exp_neg(zh, zl, tab, th, tl);
    return true;
}

__device__ __forceinline__ void split_shift(const unsigned long long *nnbits, int64_t r, int64_t n, double inv_sigma,
                                            float &h, float &l) {
    double sh = 0.0;
    if (r < n) {
        const double nd2 = bitsd(nnbits[r]);
        sh = isfinite(nd2) ? __dmul_rn(__dsqrt_rn(nd2), inv_sigma) : 0.0;
    }
    h = (float)sh;
    l = (float)(sh - (double)h);
}

// Unordered 64x64 tile pair w = (I, J), I <= J, of the upper triangle in
// row-major order.
__device__ __forceinline__ void tri_item(int64_t w, int64_t T, int64_t &I, int64_t &J) {
    const double b = 2.0 * (double)T + 1.0;
    int64_t i = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)w)) * 0.5);
    if (i < 0) i = 0;
    while (i > 0 && i * T - i * (i - 1) / 2 > w) --i;
    while ((i + 1) * T - (i + 1) * i / 2 <= w) ++i;
    I = i;
    J = i + (w - (i * T - i * (i - 1) / 2));
}

// Per 64-row tile: centroid c (FP64 mean, stored FP32), radius r >= the
// distance of every real row to the stored c (FP64, rounded up), and the
// largest nearest-neighbour shift of its rows (rounded up).  By the triangle
// inequality every pair of tiles I, J has distances >= |c_I - c_J| - r_I - r_J.
__global__ void __launch_bounds__(64) k_tile_bounds(const float *__restrict__ X, int64_t n, int32_t d,
                                                    const float2 *__restrict__ shdw,
                                                    const int32_t *__restrict__ tile_valid, float *__restrict__ cen,
                                                    float *__restrict__ rad, float *__restrict__ msh) {
    __shared__ double red[64];
    const int64_t I = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t r0 = I * WT;
    const int nv = tile_valid ? tile_valid[I] : (int)(n - r0 < WT ? n - r0 : WT);
    for (int32_t t = tid; t < d; t += 64) {
        double sum = 0.0;
        for (int q = 0; q < nv; ++q) sum += (double)X[(r0 + q) * d + t];
        cen[I * d + t] = nv > 0 ? (float)(sum / (double)nv) : 0.0f;
    }
    __syncthreads();
    double dist = 0.0, sh = 0.0;
    if (tid < nv) {
        double acc = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            const double df = (double)X[(r0 + tid) * d + t] - (double)cen[I * d + t];
            acc += df * df;
        }
        dist = sqrt(acc);
        const float2 y = shdw[r0 + tid];
        sh = (double)y.x + (double)y.y;
    }
    red[tid] = dist;
    __syncthreads();
    for (int q = 32; q > 0; q >>= 1) {
        if (tid < q) red[tid] = fmax(red[tid], red[tid + q]);
        __syncthreads();
    }
    if (tid == 0) rad[I] = (float)(red[0] * (1.0 + 1e-6)) * 1.000001f;
    __syncthreads();
    red[tid] = sh;
    __syncthreads();
    for (int q = 32; q > 0; q >>= 1) {
        if (tid < q) red[tid] = fmax(red[tid], red[tid + q]);
        __syncthreads();
    }
    if (tid == 0) msh[I] = (float)(red[0] * (1.0 + 1e-6)) * 1.000001f;
}

// One thread per tile pair w = (I, J): every distance is >= |c_I - c_J| -
// r_I - r_J; when even that is beyond zskip of both tiles' largest shift, no
// term of the pair of tiles can matter and the pair is skipped before the
// per-pair screen.  The FP32 sum carries the pair screen's relative error,
// hence its shrink; every other step rounds towards the safe side.
// With the tensor-core screen (need != null) the pair is skipped unless it
// found a pair of points within the cutoff.
template <bool SETS>
__global__ void k_tile_pair_skip(const float *__restrict__ cen, const float *__restrict__ rad,
                                 const float *__restrict__ msh, int32_t d, int64_t T, int64_t nitems,
                                 const int2 *__restrict__ witems, float is_h, float zskip, float scr_shrink,
                                 const uint8_t *__restrict__ need, uint8_t *__restrict__ tskip) {
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nitems; w += gs) {
        int64_t I, J;
        if constexpr (SETS) {
            I = witems[w].x;
            J = witems[w].y;
        } else {
            tri_item(w, T, I, J);
        }
        uint8_t skip = 0;
        if (need) {
            skip = (I != J && !need[I * T + J]) ? 1 : 0;
        } else if (I != J) {
            float tot = 0.0f;
            for (int32_t t = 0; t < d; ++t) {
                const float df = __fsub_rn(cen[I * d + t], cen[J * d + t]);
                tot = __fmaf_rn(df, df, tot);
            }
            const float lb = __fsub_rd(__fsqrt_rd(__fmul_rd(tot, scr_shrink)), __fadd_ru(rad[I], rad[J]));
            const float ylb = __fmul_rd(__fmul_rd(lb, is_h), 0.999999f);
            skip = ylb - fmaxf(msh[I], msh[J]) > zskip ? 1 : 0;
        }
        tskip[w] = skip;
    }
}

// d2 of rows of the omega order from the tensor-core Gram (omega_tc.cu).
struct GramArgs {
    const float2 *gbuf;          // [blocks][128][64] G in units of 2^(E_i + E_j - 14)
    const int32_t *item_slot;    // per item: 2 x block + half
    const float *yh, *yl;        // y = x - c_T, double-word
    const int32_t *rexp;         // E of each row
    const float2 *rnorm;         // |y|^2, double-word
    const float *cen;            // tile centroids c_T
    int one_centre;              // 1: every row was centred on the same point (D = 0)
};

// 16-byte asynchronous global -> shared copies (the Gram tile of an item,
// landing while the item's cross terms are computed)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
constexpr int GR_GTILE_BYTES = WT * WT * (int)sizeof(float2);      // one item's Gram tile (32 KB)

// Symmetric omega sweep: each unordered tile pair is screened in FP32 and,
// if any of its terms can matter in either direction, evaluated once in
// double-word arithmetic; the pair's d2 serves both omega_i and omega_j.
// Row partials (rows of I) and column partials (rows of J) go to fixed slots
// of item w, so the final sums do not depend on scheduling.
// Independent sets: the tile pairs come from a list (both tiles of one set)
// and tile_valid[I] counts the real rows of tile I (padding follows them).
template <bool SETS, bool GRAM = false>
__global__ void __launch_bounds__(TPB, 2)
k_weights_sym(const float *__restrict__ X, int64_t n, int32_t d, const float2 *__restrict__ shdw,
              float is_h, float is_l, ExpTable tabv, float zskip, float scr_shrink, int64_t T,
              int64_t nitems, const int2 *__restrict__ witems, const int32_t *__restrict__ tile_valid,
              const uint8_t *__restrict__ tskip, int prescreened, uint8_t *__restrict__ flags,
              float2 *__restrict__ rpart, float2 *__restrict__ cpart, unsigned long long *__restrict__ tile_counts,
              int shard_rank, int shard_world, GramArgs ga) {
    __shared__ __align__(16) float As[WDC][WPAD];
    __shared__ __align__(16) float Bs[WDC][WPAD];
    __shared__ float2 tab[64];
    __shared__ float2 mr[WT][17];
    __shared__ float2 mc[WT][17];
    __shared__ int64_t sIJ[5];
    __shared__ float sred[TPB / 32][2];        // per warp: smallest and largest shift of its real rows
    __shared__ float2 sUV[GRAM ? 2 * WT : 1];  // GRAM: |y|^2 +- 2 <y, D> of the rows of I, then of J
    __shared__ float sSc[GRAM ? 2 * WT : 1];   // GRAM: 2^(E - 7) of the rows of I, 2^(E - 6) of J
    __shared__ float2 sC;                      // GRAM: |D|^2
    __shared__ float sMg[GRAM ? 2 * WT : 1];   // GRAM: |y|^2 + 2 |<y, D>| (+ |D|^2 for I): the parts' size
    __shared__ int sFb;                        // GRAM: cancelling pairs of the item
    extern __shared__ __align__(16) float2 sG[];   // GRAM: the item's Gram tile, [WT][WT] double-words
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    if (tid < 64) tab[tid] = tabv.t[tid];
    unsigned long long dw_items = 0, screened = 0, fallbacks = 0;
    // a sharded call evaluates the items w with w mod world == rank
    for (int64_t w = (int64_t)blockIdx.x * shard_world + shard_rank; w < nitems;
         w += (int64_t)gridDim.x * shard_world) {
        ++screened;
        __syncthreads();                       // previous item's readers of sIJ are done
        if (tid == 0) {
            if constexpr (SETS) {
                const int2 it = witems[w];
                sIJ[0] = it.x;
                sIJ[1] = it.y;
                sIJ[2] = tile_valid[it.x];
                sIJ[3] = tile_valid[it.y];
            } else {
                tri_item(w, T, sIJ[0], sIJ[1]);
            }
            sIJ[4] = tskip[w];
            if (sIJ[4]) flags[w] = 0;
        }
        __syncthreads();
        if (sIJ[4]) continue;             // the tile bound already rules the pair of tiles out
        const int64_t I = sIJ[0], J = sIJ[1];
        const int64_t row0 = I * WT, col0 = J * WT;
        const bool diag = I == J;
        // real rows of the two tiles (padding follows them): local row lr of
        // tile I is real iff rok(lr)
        const int nI = SETS ? (int)sIJ[2] : 0, nJ = SETS ? (int)sIJ[3] : 0;
        auto rok = [&](int lr) { return SETS ? lr < nI : row0 + lr < n; };
        auto cok = [&](int lc) { return SETS ? lc < nJ : col0 + lc < n; };
        float rs_h[4], rs_l[4], cs_h[4], cs_l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int lr = ty * 4 + q, lc = tx * 4 + q;
            const float2 a = rok(lr) ? shdw[row0 + lr] : make_float2(0.f, 0.f);
            const float2 b = cok(lc) ? shdw[col0 + lc] : make_float2(0.f, 0.f);
            rs_h[q] = a.x; rs_l[q] = a.y;
            cs_h[q] = b.x; cs_l[q] = b.y;
        }
        {
            // the tile pair's range of shifts (read after the next barrier)
            float mn = INFINITY, mx = -INFINITY;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (rok(ty * 4 + q)) { mn = fminf(mn, rs_h[q]); mx = fmaxf(mx, rs_h[q]); }
                if (cok(tx * 4 + q)) { mn = fminf(mn, cs_h[q]); mx = fmaxf(mx, cs_h[q]); }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if ((tid & 31) == 0) { sred[tid >> 5][0] = mn; sred[tid >> 5][1] = mx; }
        }
        // ---- FP32 screen, both directions (unless the tensor-core screen
        //      already decided this pair of tiles)
        if (!prescreened) {
            // ---- FP32 screen, both directions
            float A32[4][4];
    #pragma unroll
            for (int i = 0; i < 4; ++i)
    #pragma unroll
                for (int j = 0; j < 4; ++j) A32[i][j] = 0.f;
            for (int t0 = 0; t0 < d; t0 += WDC) {
                __syncthreads();
    #pragma unroll
                for (int q = 0; q < (WT * WDC) / TPB; ++q) {
                    int idx = tid + q * TPB;
                    int r = idx / WDC, t = idx % WDC;
                    int64_t gr = row0 + r, gc = col0 + r;
                    int gt = t0 + t;
                    As[t][r] = (rok(r) && gt < d) ? X[gr * d + gt] : 0.0f;
                    Bs[t][r] = (cok(r) && gt < d) ? X[gc * d + gt] : 0.0f;
                }
                __syncthreads();
                const int tl = min(WDC, d - t0);
                for (int t = 0; t < tl; ++t) {
                    float4 a4 = *reinterpret_cast<const float4 *>(&As[t][ty * 4]);
                    float4 b4 = *reinterpret_cast<const float4 *>(&Bs[t][tx * 4]);
                    float a[4] = {a4.x, a4.y, a4.z, a4.w};
                    float b[4] = {b4.x, b4.y, b4.z, b4.w};
    #pragma unroll
                    for (int i = 0; i < 4; ++i)
    #pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float df = __fsub_rn(a[i], b[j]);
                            A32[i][j] = __fmaf_rn(df, df, A32[i][j]);
                        }
                }
            }
            int need = 0;
    #pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int lr = ty * 4 + i;
    #pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int lc = tx * 4 + j;
                    if (!rok(lr) || !cok(lc) || (diag && lc == lr)) continue;
                    const float y = __fmul_rn(__fsqrt_rn(__fmul_rn(A32[i][j], scr_shrink)), is_h);
                    if (!(y - rs_h[i] > zskip) || !(y - cs_h[j] > zskip)) need = 1;
                }
            }
            if (!__syncthreads_or(need)) {
                if (tid == 0) flags[w] = 0;
                continue;
            }
        }
        ++dw_items;
        if constexpr (GRAM) {
            // the item's Gram tile into shared memory (it lands during the
            // cross terms; every reader of the previous tile is past the
            // item's first barrier)
            const int32_t gslot = ga.item_slot[w];
            if (gslot >= 0) {
                const float4 *src = reinterpret_cast<const float4 *>(
                    ga.gbuf + ((size_t)(gslot >> 1) * (2 * WT) + (size_t)(gslot & 1) * WT) * WT);
                float4 *dst = reinterpret_cast<float4 *>(sG);
#pragma unroll
                for (int q = 0; q < GR_GTILE_BYTES / 16 / TPB; ++q) cp_async16(dst + tid + q * TPB, src + tid + q * TPB);
            }
            cp_async_commit();
        }
        // ---- double-word pass
        float S[4][4], E[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { S[i][j] = 0.f; E[i][j] = 0.f; }
        if constexpr (GRAM) {
            // d2 = (|y_i|^2 + 2 <y_i, D> + |D|^2) + (|y_j|^2 - 2 <y_j, D>) - 2 G_ij, y = x - c_T,
            // D = c_I - c_J (zero on the diagonal and when every row shares one centre)
            const int lane = tid & 31, wq = tid >> 5;
            const bool cross = !diag && !ga.one_centre;
            float2 *sD = reinterpret_cast<float2 *>(&As[0][0]);          // D chunk, double-word
            float2 *sX = reinterpret_cast<float2 *>(&Bs[0][0]);          // upper half's partial products
            {
                // products p = 0..63 (rows of I) and 64..127 (rows of J), one
                // thread each; the two halves of the block take alternate
                // dimensions of every chunk of D
                const int pr = tid & 127, hh = tid >> 7;
                const int64_t gr = pr < WT ? row0 + pr : col0 + (pr - WT);
                float xh = 0.f, xl = 0.f, ch = 0.f, cl = 0.f;
                if (cross) {
                    const float *cI = ga.cen + I * d, *cJ = ga.cen + J * d;
                    const float *ryh = ga.yh + gr * d, *ryl = ga.yl + gr * d;
                    for (int t0 = 0; t0 < d; t0 += GR_DCH) {
                        const int tl = min(GR_DCH, d - t0);
                        __syncthreads();                       // previous chunk's readers are done
                        for (int t = tid; t < tl; t += TPB) {
                            float Dh, Dl;
                            two_sum(cI[t0 + t], -cJ[t0 + t], Dh, Dl);
                            sD[t] = make_float2(Dh, Dl);
                            float p, e;
                            two_prod(Dh, Dh, p, e);
                            e = __fmaf_rn(__fadd_rn(Dh, Dh), Dl, e);
                            dw_add(ch, cl, p, e);
                        }
                        __syncthreads();
                        // the lower half of the block takes the chunk's first
                        // h4 dimensions, the upper half the rest (4 at a time
                        // when rows are 16-byte aligned)
                        const int h4 = ((tl + 7) >> 3) << 2;
                        const int ta = hh ? min(h4, tl) : 0, tb = hh ? tl : min(h4, tl);
                        auto term = [&](float a, float al, float2 D) {
                            float p, e;
                            two_prod(a, D.x, p, e);
                            e = __fmaf_rn(a, D.y, __fmaf_rn(al, D.x, e));
                            dw_add(xh, xl, p, e);
                        };
                        if ((d & 3) == 0) {
                            for (int t = ta; t < tb; t += 4) {
                                const float4 a4 = *reinterpret_cast<const float4 *>(ryh + t0 + t);
                                const float4 l4 = *reinterpret_cast<const float4 *>(ryl + t0 + t);
                                const float4 d01 = *reinterpret_cast<const float4 *>(sD + t);
                                const float4 d23 = *reinterpret_cast<const float4 *>(sD + t + 2);
                                term(a4.x, l4.x, make_float2(d01.x, d01.y));
                                term(a4.y, l4.y, make_float2(d01.z, d01.w));
                                term(a4.z, l4.z, make_float2(d23.x, d23.y));
                                term(a4.w, l4.w, make_float2(d23.z, d23.w));
                            }
                        } else {
                            for (int t = ta; t < tb; ++t) term(ryh[t0 + t], ryl[t0 + t], sD[t]);
                        }
                    }
                    // |D|^2: the threads' chunk partials, folded in a fixed order
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float oh = __shfl_xor_sync(0xffffffffu, ch, o);
                        const float ol = __shfl_xor_sync(0xffffffffu, cl, o);
                        dw_add(ch, cl, oh, ol);
                    }
                    if (hh) sX[pr] = make_float2(xh, xl);
                }
                __syncthreads();
                if (cross && lane == 0) sX[128 + wq] = make_float2(ch, cl);
                __syncthreads();
                if (tid < 2 * WT) {
                    const float2 rn = ga.rnorm[gr];
                    float uh = rn.x, ul = rn.y;
                    float mg = rn.x;
                    if (cross) {
                        const float2 o = sX[pr];
                        dw_add(xh, xl, o.x, o.y);
                        const float sg = pr < WT ? 2.0f : -2.0f;
                        dw_add(uh, ul, __fmul_rn(sg, xh), __fmul_rn(sg, xl));
                        mg = __fadd_rn(rn.x, fabsf(__fmul_rn(2.0f, xh)));
                    }
                    sUV[pr] = make_float2(uh, ul);
                    sMg[pr] = mg;
                    sSc[pr] = ldexpf(1.0f, ga.rexp[gr] - (pr < WT ? 7 : 6));
                }
                if (tid == 0) {
                    float h = 0.f, l = 0.f;
                    if (cross)
                        for (int q = 0; q < TPB / 32; ++q) dw_add(h, l, sX[128 + q].x, sX[128 + q].y);
                    sC = make_float2(h, l);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            const int32_t slot = ga.item_slot[w];
            // (every kept item has a Gram block; should one lack it, its pairs
            // take the direct sums below)
            const float2 *Gp = sG;
            const float2 C = sC;
            unsigned fb = 0u;                  // pairs whose Gram form cancels (bit 4i + j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int lr = ty * 4 + i;
                float uh = sUV[lr].x, ul = sUV[lr].y;
                dw_add(uh, ul, C.x, C.y);
                const float mi = sMg[lr] + C.x, si = sSc[lr];
                float4 g01 = make_float4(0.f, 0.f, 0.f, 0.f), g23 = g01;
                if (slot >= 0) {
                    g01 = *reinterpret_cast<const float4 *>(Gp + lr * WT + tx * 4);
                    g23 = *reinterpret_cast<const float4 *>(Gp + lr * WT + tx * 4 + 2);
                }
                const float gv[4][2] = {{g01.x, g01.y}, {g01.z, g01.w}, {g23.x, g23.y}, {g23.z, g23.w}};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int lc = tx * 4 + j;
                    const float sc = __fmul_rn(si, sSc[WT + lc]);      // 2^(E_i + E_j - 13), exact
                    const float gh = __fmul_rn(gv[j][0], sc), gl = __fmul_rn(gv[j][1], sc);
                    const float2 V = sUV[WT + lc];
                    float h = uh, l = ul;
                    dw_add(h, l, V.x, V.y);
                    dw_add(h, l, -gh, -gl);
                    // the Gram form's error is about 2^-46 of the addends'
                    // size M: where they cancel to under half of it, the
                    // pair takes the direct sum of squared differences
                    const float M = mi + sMg[WT + lc] + fabsf(gh);
                    const bool real = rok(lr) && cok(lc) && !(diag && lc == lr);
                    if (real && (slot < 0 || !(__fmul_rn(h, 2.0f) >= M))) fb |= 1u << (4 * i + j);
                    S[i][j] = h;
                    E[i][j] = l;
                }
            }
            fallbacks += (unsigned)__popc(fb);
            // the cancelling pairs go to a block-wide list (pair index lr * 64
            // + lc), evaluated by groups of GL lanes (a lane per GL-th
            // dimension, the group's double-word partials folded in a fixed
            // tree); results come back through shared memory
            uint16_t *flist = reinterpret_cast<uint16_t *>(&Bs[0][0]);
            float2 *fres = reinterpret_cast<float2 *>(&As[0][0]);
            if (tid == 0) sFb = 0;
            __syncthreads();
            const int nmine = __popc(fb);
            const int fbase = nmine ? atomicAdd(&sFb, nmine) : 0;
            __syncthreads();
            const int ftotal = sFb;
            const int GL = d >= 256 ? 32 : 8;
            const int ngroups = (TPB / 32) * (32 / GL);      // groups in the block
            for (int r0 = 0; r0 < ftotal; r0 += GR_FCAP) {
                const int rn = min(GR_FCAP, ftotal - r0);
                {
                    unsigned m = fb;
                    for (int q = 0; m; ++q) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1u;
                        const int e = fbase + q - r0;
                        if (e >= 0 && e < rn) flist[e] = (uint16_t)((ty * 4 + (b >> 2)) * WT + tx * 4 + (b & 3));
                    }
                }
                __syncthreads();
                {
                    // warp-uniform trip count: the groups of a warp take
                    // consecutive entries, the whole warp shuffles
                    const int gpw = 32 / GL, wg = lane / GL, gl = lane % GL;
                    for (int eb = wq * gpw; eb < rn; eb += ngroups) {
                        const int e = eb + wg;
                        float ph = 0.f, pl = 0.f;
                        if (e < rn) {
                            const int pi = flist[e];
                            const float *xa = X + (row0 + (pi >> 6)) * d, *xb = X + (col0 + (pi & 63)) * d;
                            auto sq = [&](float a, float b) {
                                float s1, e1;
                                two_sum(a, -b, s1, e1);
                                const float p = __fmul_rn(s1, s1);
                                float q2 = __fmaf_rn(s1, s1, -p);
                                q2 = __fmaf_rn(__fadd_rn(s1, s1), e1, q2);
                                dw_add(ph, pl, p, q2);
                            };
                            if ((d & 3) == 0) {
                                // 4 consecutive dimensions per lane and step
                                for (int t = 4 * gl; t < d; t += 4 * GL) {
                                    const float4 a = *reinterpret_cast<const float4 *>(xa + t);
                                    const float4 b = *reinterpret_cast<const float4 *>(xb + t);
                                    sq(a.x, b.x);
                                    sq(a.y, b.y);
                                    sq(a.z, b.z);
                                    sq(a.w, b.w);
                                }
                            } else {
                                for (int t = gl; t < d; t += GL) sq(xa[t], xb[t]);
                            }
                        }
                        for (int o = GL >> 1; o > 0; o >>= 1) {
                            const float oh = __shfl_xor_sync(0xffffffffu, ph, o);
                            const float ol = __shfl_xor_sync(0xffffffffu, pl, o);
                            dw_add(ph, pl, oh, ol);
                        }
                        if (e < rn && gl == 0) fres[e] = make_float2(ph, pl);
                    }
                }
                __syncthreads();
                {
                    unsigned m = fb;
                    for (int q = 0; m; ++q) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1u;
                        const int e = fbase + q - r0;
                        if (e >= 0 && e < rn) {
                            const float2 v = fres[e];
#pragma unroll
                            for (int kk = 0; kk < 16; ++kk)
                                if (kk == b) {
                                    S[kk >> 2][kk & 3] = v.x;
                                    E[kk >> 2][kk & 3] = v.y;
                                }
                        }
                    }
                }
                __syncthreads();
            }
        } else
        for (int t0 = 0; t0 < d; t0 += WDC) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < (WT * WDC) / TPB; ++q) {
                int idx = tid + q * TPB;
                int r = idx / WDC, t = idx % WDC;
                int64_t gr = row0 + r, gc = col0 + r;
                int gt = t0 + t;
                As[t][r] = (rok(r) && gt < d) ? X[gr * d + gt] : 0.0f;
                Bs[t][r] = (cok(r) && gt < d) ? X[gc * d + gt] : 0.0f;
            }
            __syncthreads();
            const int tl = min(WDC, d - t0);
            // S takes each square's high part by TwoSum; the rounding errors
            // and the squares' low parts gather in E, renormalised every 4
            // dimensions (E stays below 2^-21 of S between renormalisations)
#pragma unroll 4
            for (int t = 0; t < tl; ++t) {
                float4 a4 = *reinterpret_cast<const float4 *>(&As[t][ty * 4]);
                float4 b4 = *reinterpret_cast<const float4 *>(&Bs[t][tx * 4]);
                float a[4] = {a4.x, a4.y, a4.z, a4.w};
                float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float s1, e1;
                        two_sum(a[i], -b[j], s1, e1);
                        float p = __fmul_rn(s1, s1);
                        float q2 = __fmaf_rn(s1, s1, -p);
                        q2 = __fmaf_rn(__fadd_rn(s1, s1), e1, q2);
                        float hs, he;
                        two_sum(S[i][j], p, hs, he);
                        S[i][j] = hs;
                        E[i][j] = __fadd_rn(E[i][j], __fadd_rn(he, q2));
                    }
                if ((t & 3) == 3) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) fast_two_sum(S[i][j], E[i][j], S[i][j], E[i][j]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) fast_two_sum(S[i][j], E[i][j], S[i][j], E[i][j]);
        }
        float rh[4] = {0.f, 0.f, 0.f, 0.f}, rl[4] = {0.f, 0.f, 0.f, 0.f};
        float ch[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
        // One exponential per pair for both of its rows: terms are taken
        // against a shift sref shared by the tile pair, exp(-(y - sref)), and
        // each row's partial is scaled by exp(sh - sref) in the merge.  sref
        // keeps every kept term's exponent in [-75, 70] (double-word FP32
        // stays normal and the partials finite); otherwise each direction
        // takes its own shift as on the diagonal.
        float smin = INFINITY, smax = -INFINITY;
#pragma unroll
        for (int q = 0; q < TPB / 32; ++q) { smin = fminf(smin, sred[q][0]); smax = fmaxf(smax, sred[q][1]); }
        const float sref = fmaxf(smin, smax + zskip - 70.0f);
        const bool one_exp = !diag && sref - smin <= 75.0f;
        float ar[4], ac[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { ar[q] = rs_h[q] - sref; ac[q] = cs_h[q] - sref; }
        if (one_exp) {
            // off the diagonal with one shift: the 16 pairs without branches
            // (a dropped or padding pair adds an exact zero, which leaves the
            // double-word sums unchanged), so their dependent double-word
            // chains can interleave
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int lr = ty * 4 + i;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int lc = tx * 4 + j;
                    const bool real = rok(lr) && cok(lc);
                    const float Sh = real ? S[i][j] : 1.0f, El = real ? E[i][j] : 0.0f;
                    const float r = __fsqrt_rn(Sh);
                    float dl = 0.0f;
                    if (r > 0.0f) {
                        const float res = __fadd_rn(__fmaf_rn(-r, r, Sh), El);
                        dl = __fmul_rn(res, __frcp_rn(__fadd_rn(r, r)));
                    }
                    float yh, yl;
                    two_prod(r, is_h, yh, yl);
                    yl = __fmaf_rn(r, is_l, yl);
                    yl = __fmaf_rn(dl, is_h, yl);
                    fast_two_sum(yh, yl, yh, yl);
                    float zh, zl;
                    two_sum(yh, -sref, zh, zl);
                    zl = __fadd_rn(zl, yl);
                    fast_two_sum(zh, zl, zh, zl);
                    // below e^-zskip of the largest term of both rows (the
                    // margin covers the FP32 shift differences): dropped
                    const bool keep = real && !(zh > zskip + fmaxf(ar[i], ac[j]) + 0.01f);
                    float th, tl2;
                    dw_exp_neg(keep ? zh : 0.0f, keep ? zl : 0.0f, tab, th, tl2);
                    th = keep ? th : 0.0f;
                    tl2 = keep ? tl2 : 0.0f;
                    dw_add(rh[i], rl[i], th, tl2);
                    dw_add(ch[j], cl[j], th, tl2);
                }
            }
        } else
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int lr = ty * 4 + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int lc = tx * 4 + j;
                if (!rok(lr) || !cok(lc) || (diag && lc == lr)) continue;
                const float Sh = S[i][j], El = E[i][j];
                const float r = __fsqrt_rn(Sh);
                float dl = 0.0f;
                if (r > 0.0f) {
                    const float res = __fadd_rn(__fmaf_rn(-r, r, Sh), El);
                    dl = __fmul_rn(res, __frcp_rn(__fadd_rn(r, r)));
                }
                float th, tl2;
                if (one_exp) {
                    float yh, yl;
                    two_prod(r, is_h, yh, yl);
                    yl = __fmaf_rn(r, is_l, yl);
                    yl = __fmaf_rn(dl, is_h, yl);
                    fast_two_sum(yh, yl, yh, yl);
                    float zh, zl;
                    two_sum(yh, -sref, zh, zl);
                    zl = __fadd_rn(zl, yl);
                    fast_two_sum(zh, zl, zh, zl);
                    // below e^-zskip of the largest term of both rows (the
                    // margin covers the FP32 shift differences): dropped
                    if (zh > zskip + fmaxf(ar[i], ac[j]) + 0.01f) continue;
                    dw_exp_neg(zh, zl, tab, th, tl2);
                    dw_add(rh[i], rl[i], th, tl2);
                    dw_add(ch[j], cl[j], th, tl2);
                } else {
                    if (dw_term(r, dl, is_h, is_l, rs_h[i], rs_l[i], zskip, tab, th, tl2))
                        dw_add(rh[i], rl[i], th, tl2);
                    if (!diag && dw_term(r, dl, is_h, is_l, cs_h[j], cs_l[j], zskip, tab, th, tl2))
                        dw_add(ch[j], cl[j], th, tl2);
                }
            }
        }
        // rows of I: merge the 16 column-threads; columns of J: merge the 16 row-threads
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            mr[ty * 4 + q][tx] = make_float2(rh[q], rl[q]);
            mc[tx * 4 + q][ty] = make_float2(ch[q], cl[q]);
        }
        __syncthreads();
        // partials leave in each row's own shift: sum exp(-(y - sh))
        auto to_own_shift = [&](float &h, float &l, float2 sh) {
            float zh, zl, fh, fl;
            two_sum(sref, -sh.x, zh, zl);          // sref - sh as a double-word
            zl = __fsub_rn(zl, sh.y);
            fast_two_sum(zh, zl, zh, zl);
            dw_exp_neg(zh, zl, tab, fh, fl);       // exp(sh - sref)
            float p, e;
            two_prod(h, fh, p, e);
            e = __fmaf_rn(h, fl, e);
            e = __fmaf_rn(l, fh, e);
            fast_two_sum(p, e, h, l);
        };
        if (tid < WT) {
            float h = 0.f, l = 0.f;
            for (int k = 0; k < 16; ++k) dw_add(h, l, mr[tid][k].x, mr[tid][k].y);
            if (one_exp && rok(tid)) to_own_shift(h, l, shdw[row0 + tid]);
            rpart[w * WT + tid] = make_float2(h, l);
        } else if (tid < 2 * WT) {
            const int c = tid - WT;
            float h = 0.f, l = 0.f;
            if (!diag) {
                for (int k = 0; k < 16; ++k) dw_add(h, l, mc[c][k].x, mc[c][k].y);
                if (one_exp && cok(c)) to_own_shift(h, l, shdw[col0 + c]);
            }
            cpart[w * WT + c] = make_float2(h, l);
        }
        if (tid == 0) flags[w] = 1;
    }
    if (tid == 0) {
        atomicAdd(tile_counts + 0, screened);
        atomicAdd(tile_counts + 1, dw_items);
    }
    if constexpr (GRAM) {
        // pairs that took the direct sums (tile_counts[2])
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, o);
        if ((tid & 31) == 0 && fallbacks) atomicAdd(tile_counts + 2, fallbacks);
    }
}

// Per row: the shift y_nn = |x - x_nn| / sigma as a double-word (once per call).
__global__ void k_shift_dw(const unsigned long long *__restrict__ nnbits, int64_t n, double inv_sigma,
                           float2 *__restrict__ shdw) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float h, l;
    split_shift(nnbits, r, n, inv_sigma, h, l);
    shdw[r] = make_float2(h, l);
}

// omega_r = exp(-y_nn,r) * (sum over the items of row r's tile, in item
// order, of the row or column partial), formed in FP64.
__global__ void k_weights_reduce(const unsigned long long *__restrict__ nnbits, int64_t n, int64_t T,
                                 double inv_sigma, int include_self, const uint8_t *__restrict__ flags,
                                 const float2 *__restrict__ rpart, const float2 *__restrict__ cpart,
                                 double *__restrict__ omega, double *__restrict__ part64) {
    // a warp is 32 rows of one 64-row tile I (blocks of 256 rows): its lanes
    // read the flags of 32 tile pairs at once; the kept pairs' partials are
    // then added in ascending J, the order of a plain loop over J
    const int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    if (r0 >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t r = r0 + lane;
    const int64_t I = r0 / WT, c = r - I * WT;
    auto item = [&](int64_t J) {
        return J < I ? J * T - J * (J - 1) / 2 + (I - J)      // item (J, I): r is a column
                     : I * T - I * (I - 1) / 2 + (J - I);     // item (I, J): r is a row
    };
    // 64 tile pairs' flags per step (two loads in flight), then the kept
    // pairs' partials RB at a time (their loads in flight together), added
    // in ascending J as they come
    constexpr int RB = 16;
    float h = 0.f, l = 0.f;
    for (int64_t J0 = 0; J0 < T; J0 += 64) {
        const int64_t Ja = J0 + lane, Jb = J0 + 32 + lane;
        const bool ka = Ja < T && flags[item(Ja)];
        const bool kb = Jb < T && flags[item(Jb)];
        unsigned ma = __ballot_sync(0xffffffffu, ka), mb = __ballot_sync(0xffffffffu, kb);
        while (ma | mb) {                                   // (warp-uniform)
            float2 v[RB];
            int nv = 0;
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                if (ma | mb) {
                    int64_t J;
                    if (ma) { J = J0 + (__ffs(ma) - 1); ma &= ma - 1u; }
                    else { J = J0 + 32 + (__ffs(mb) - 1); mb &= mb - 1u; }
                    const int64_t w = item(J);
                    v[q] = J < I ? cpart[w * WT + c] : rpart[w * WT + c];
                    nv = q + 1;
                }
            }
#pragma unroll
            for (int q = 0; q < RB; ++q)
                if (q < nv) dw_add(h, l, v[q].x, v[q].y);
        }
    }
    if (r >= n) return;
    if (part64) {                 // sharded call: this rank's share, combined across ranks first
        part64[r] = __dadd_rn((double)h, (double)l);
        return;
    }
    float fh, fl;
    split_shift(nnbits, r, n, inv_sigma, fh, fl);
    double w2 = __dmul_rn(exp(-__dadd_rn((double)fh, (double)fl)), __dadd_rn((double)h, (double)l));
    if (include_self) w2 = __dadd_rn(w2, 1.0);
    omega[r] = w2;
}

// Sharded call: omega_r from the sum over the ranks of their shares.
__global__ void k_weights_finish(const unsigned long long *__restrict__ nnbits, int64_t n, double inv_sigma,
                                 int include_self, const double *__restrict__ part64, double *__restrict__ omega) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float fh, fl;
    split_shift(nnbits, r, n, inv_sigma, fh, fl);
    double w2 = __dmul_rn(exp(-__dadd_rn((double)fh, (double)fl)), part64[r]);
    if (include_self) w2 = __dadd_rn(w2, 1.0);
    omega[r] = w2;
}

// Independent sets: padded row r of tile I (set b = tile_set[I], tiles
// [tile0[b], tile0[b] + ntl[b]), items from item0[b] in upper-triangle row
// order); padding rows get 0.
__global__ void k_weights_reduce_sets(const unsigned long long *__restrict__ nnbits, int64_t n_pad,
                                      const int32_t *__restrict__ tile_valid, const int32_t *__restrict__ tile_set,
                                      const int64_t *__restrict__ tile0, const int64_t *__restrict__ ntl,
                                      const int64_t *__restrict__ item0, double inv_sigma, int include_self,
                                      const uint8_t *__restrict__ flags, const float2 *__restrict__ rpart,
                                      const float2 *__restrict__ cpart, double *__restrict__ omega) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const int64_t I = r / WT, c = r - I * WT;
    if (c >= tile_valid[I]) {
        omega[r] = 0.0;
        return;
    }
    const int32_t b = tile_set[I];
    const int64_t T = ntl[b], base = item0[b], Il = I - tile0[b];
    float h = 0.f, l = 0.f;
    for (int64_t Jl = 0; Jl < T; ++Jl) {
        if (Jl < Il) {
            const int64_t w = base + Jl * T - Jl * (Jl - 1) / 2 + (Il - Jl);    // item (J, I): r is a column
            if (flags[w]) dw_add(h, l, cpart[w * WT + c].x, cpart[w * WT + c].y);
        } else {
            const int64_t w = base + Il * T - Il * (Il - 1) / 2 + (Jl - Il);    // item (I, J): r is a row
            if (flags[w]) dw_add(h, l, rpart[w * WT + c].x, rpart[w * WT + c].y);
        }
    }
    float fh, fl;
    split_shift(nnbits, r, n_pad, inv_sigma, fh, fl);
    double w2 = __dmul_rn(exp(-__dadd_rn((double)fh, (double)fl)), __dadd_rn((double)h, (double)l));
    if (include_self) w2 = __dadd_rn(w2, 1.0);
    omega[r] = w2;
}

// FP64 input: canonical FP64 terms, j ascending (the oracle's order).
template <class T>
__global__ void __launch_bounds__(TPB) k_weights_f64(const T *__restrict__ X, int64_t n, int32_t d, double sigma,
                                                     double alpha, int include_self, double *__restrict__ omega,
                                                     double *__restrict__ pout) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T *xi = X + i * d;
    double sw = 0.0, sd = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) {
            if (include_self) sw = __dadd_rn(sw, 1.0);
            continue;
        }
        double d2 = exact_d2(xi, X + j * d, d);
        double dist = __dsqrt_rn(d2);
        sw = __dadd_rn(sw, exp(-__ddiv_rn(dist, sigma)));
        if (alpha != 0.0) sd = __dadd_rn(sd, dist);
    }
    omega[i] = sw;
    if (pout) pout[i] = alpha != 0.0 ? __dmul_rn(alpha, sd) : 0.0;
}
}  // namespace

// part: row partials, column partials [items][64] float2, shifts [rows]
// float2, flags [items], then (256-aligned) tile centroids [T][d], radii [T]
// and largest shifts [T]
struct SymParts {
    float2 *rpart, *cpart, *shdw;
    uint8_t *flags, *tskip;
    float *cen, *rad, *msh;
};
static SymParts sym_parts(void *part, int64_t items, int64_t rows, int64_t T, int32_t d) {
    SymParts P;
    P.rpart = (float2 *)part;
    P.cpart = P.rpart + items * WT;
    P.shdw = P.cpart + items * WT;
    P.flags = (uint8_t *)(P.shdw + rows);
    uintptr_t c = ((uintptr_t)(P.flags + items) + 255) & ~(uintptr_t)255;
    P.cen = (float *)c;
    P.rad = P.cen + T * d;
    P.msh = P.rad + T;
    P.tskip = (uint8_t *)(P.msh + T);
    return P;
}
static size_t sym_bytes(int64_t items, int64_t rows, int64_t T, int32_t d) {
    return (size_t)items * (2 + 2 * WT * sizeof(float2)) + (size_t)rows * sizeof(float2) + 256 +
           (size_t)T * (d + 2) * sizeof(float) + 4096;
}

// the omega cutoff of a problem with n points per set: terms below
// e^-zskip of a row's largest term are dropped (total < e^-36 of the row)
float omega_zskip(int64_t n) { return (float)(36.0 + log((double)(n > 2 ? n : 2))); }

size_t weights_sym_bytes(int64_t n, int32_t d) {
    const int64_t T = ceil_div(n, WT);
    return sym_bytes(T * (T + 1) / 2, n, T, d);
}

// Symmetric screened omega (F32 input, p not needed).  part must hold
// weights_sym_bytes(n) bytes.
cudaError_t weights_launch_sym(const float *X, int64_t n, int32_t d, double sigma, int include_self,
                               const unsigned long long *nnbits, double *omega, void *part,
                               unsigned long long *tile_counts, const uint8_t *need, cudaEvent_t *kev,
                               cudaStream_t s, const Shard *sh, double *part64, OmegaGram *og, uint32_t *status,
                               uint64_t wait_cycles) {
    static const ExpTable tab = make_exp_table();
    const double is = 1.0 / sigma;
    const float is_h = (float)is;
    const float is_l = (float)(is - (double)is_h);
    const float zskip = omega_zskip(n);
    const double e = 1.1 * (double)(d + 3) * 5.9604644775390625e-08;
    const float shrink = (float)((1.0 - e) * (1.0 - 1e-6));
    const int64_t T = ceil_div(n, WT);
    const int64_t items = T * (T + 1) / 2;
    const SymParts P = sym_parts(part, items, n, T, d);
    const unsigned grid = (unsigned)(num_sms() * 2);
    k_shift_dw<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(nnbits, n, is, P.shdw);
    k_tile_bounds<<<(unsigned)T, 64, 0, ISO_S(s)>>>(X, n, d, P.shdw, nullptr, P.cen, P.rad, P.msh);
    k_tile_pair_skip<false><<<(unsigned)(num_sms() * 8), 256, 0, ISO_S(s)>>>(P.cen, P.rad, P.msh, d, T, items, nullptr,
                                                                            is_h, zskip, shrink, need, P.tskip);
    cudaError_t err;
    // sharded: the items of other ranks hold nothing here
    if (sh && (err = cudaMemsetAsync(P.flags, 0, (size_t)items, s))) return err;
    if (kev) record_event(kev[0], s);
    if (og && need) {
        // the kept tile pairs' Gram on the tensor cores, then the terms
        if ((err = omega_gram_launch(*og, X, n, d, P.cen, P.tskip, status, wait_cycles, s, kev ? kev + 2 : nullptr)))
            return err;
        const GramArgs ga{og->gbuf, og->item_slot, og->yh, og->yl, og->rexp, og->rnorm, P.cen, og->one_centre};
        static bool gattr = false;
        if (!gattr) {
            if ((err = cudaFuncSetAttribute(k_weights_sym<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            GR_GTILE_BYTES)))
                return err;
            gattr = true;
        }
        k_weights_sym<false, true><<<grid, TPB, GR_GTILE_BYTES, ISO_S(s)>>>(X, n, d, P.shdw, is_h, is_l, tab, zskip, shrink, T,
                                                               items, nullptr, nullptr, P.tskip, 1, P.flags, P.rpart,
                                                               P.cpart, tile_counts, sh ? sh->rank : 0,
                                                               sh ? sh->world : 1, ga);
    } else {
        k_weights_sym<false><<<grid, TPB, 0, ISO_S(s)>>>(X, n, d, P.shdw, is_h, is_l, tab, zskip, shrink, T, items,
                                                         nullptr, nullptr, P.tskip, need ? 1 : 0, P.flags, P.rpart,
                                                         P.cpart, tile_counts, sh ? sh->rank : 0, sh ? sh->world : 1,
                                                         GramArgs{});
    }
    if (kev) record_event(kev[1], s);
    k_weights_reduce<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(nnbits, n, T, is, include_self, P.flags,
                                                                      P.rpart, P.cpart, omega, sh ? part64 : nullptr);
    if (sh) {
        if ((err = shard_allreduce(*sh, part64, n, ISOCLUST_REDUCE_SUM_F64, s))) return err;
        k_weights_finish<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(nnbits, n, is, include_self, part64, omega);
    }
    return cudaGetLastError();
}

size_t weights_sym_sets_bytes(int64_t n_pad, int64_t nitems, int32_t d) {
    return sym_bytes(nitems, n_pad, ceil_div(n_pad, WT), d);
}

// Symmetric screened omega over independent sets.  Xp / nnbits / omega are
// in the padded row space (n_pad rows, sets in whole 64-row tiles); the
// items are the upper triangles of the sets' tile grids; max_n is the
// largest set (it bounds the number of terms per row).
cudaError_t weights_launch_sym_sets(const float *Xp, int64_t n_pad, int32_t d, double sigma, int include_self,
                                    const unsigned long long *nnbits, double *omega, void *part, const int2 *witems,
                                    int64_t nitems, const int32_t *tile_valid, const int32_t *tile_set,
                                    const int64_t *tile0, const int64_t *ntl, const int64_t *item0, int64_t max_n,
                                    unsigned long long *tile_counts, cudaEvent_t *kev, cudaStream_t s) {
    static const ExpTable tab = make_exp_table();
    const double is = 1.0 / sigma;
    const float is_h = (float)is;
    const float is_l = (float)(is - (double)is_h);
    const float zskip = omega_zskip(max_n);
    const double e = 1.1 * (double)(d + 3) * 5.9604644775390625e-08;
    const float shrink = (float)((1.0 - e) * (1.0 - 1e-6));
    const int64_t T = ceil_div(n_pad, WT);
    const SymParts P = sym_parts(part, nitems, n_pad, T, d);
    const unsigned grid = (unsigned)(num_sms() * 2);
    k_shift_dw<<<(unsigned)ceil_div(n_pad, 256), 256, 0, ISO_S(s)>>>(nnbits, n_pad, is, P.shdw);
    k_tile_bounds<<<(unsigned)T, 64, 0, ISO_S(s)>>>(Xp, n_pad, d, P.shdw, tile_valid, P.cen, P.rad, P.msh);
    if (nitems > 0) {
        k_tile_pair_skip<true><<<(unsigned)(num_sms() * 8), 256, 0, ISO_S(s)>>>(
            P.cen, P.rad, P.msh, d, T, nitems, witems, is_h, zskip, shrink, nullptr, P.tskip);
        if (kev) record_event(kev[0], s);
        // independent sets: the tile bound is the only screen; tile pairs it
        // keeps go straight to the double-word pass (for sets of a few
        // thousand points nearly every pair of tiles holds terms, so the FP32
        // pair screen would cost more than the double-word work it saves)
        k_weights_sym<true><<<grid, TPB, 0, ISO_S(s)>>>(Xp, n_pad, d, P.shdw, is_h, is_l, tab, zskip, shrink, 0, nitems,
                                                        witems, tile_valid, P.tskip, 1, P.flags, P.rpart, P.cpart,
                                                        tile_counts, 0, 1, GramArgs{});
        if (kev) record_event(kev[1], s);
    }
    k_weights_reduce_sets<<<(unsigned)ceil_div(n_pad, 256), 256, 0, ISO_S(s)>>>(
        nnbits, n_pad, tile_valid, tile_set, tile0, ntl, item0, is, include_self, P.flags, P.rpart, P.cpart, omega);
    return cudaGetLastError();
}

cudaError_t weights_launch(const void *X, int64_t n, int32_t d, int dtype, bool fp64_path, double sigma,
                           double alpha, int include_self, const unsigned long long *nnbits, double *omega,
                           double *p, unsigned long long *tile_counts, cudaStream_t s) {
    if (fp64_path || dtype == ISOCLUST_F64) {
        unsigned g = (unsigned)ceil_div(n, TPB);
        if (dtype == ISOCLUST_F64)
            k_weights_f64<double><<<g, TPB, 0, ISO_S(s)>>>((const double *)X, n, d, sigma, alpha, include_self, omega, p);
        else
            k_weights_f64<float><<<g, TPB, 0, ISO_S(s)>>>((const float *)X, n, d, sigma, alpha, include_self, omega, p);
        return cudaGetLastError();
    }
    static const ExpTable tab = make_exp_table();
    const double is = 1.0 / sigma;
    const float is_h = (float)is;
    const float is_l = (float)(is - (double)is_h);
    // Terms below e^-zskip of a row's largest term are dropped: their total
    // is below n e^-zskip = e^-36 ~ 2.3e-16 of the row sum.
    const float zskip = omega_zskip(n);
    // FP32 d2 relative error <= (d+1)u (+ underflow): shrink by 1.1(d+3)u
    // plus the rounding of the screen's own sqrt/multiply/subtract.
    const double e = 1.1 * (double)(d + 3) * 5.9604644775390625e-08;
    const float shrink = (float)((1.0 - e) * (1.0 - 1e-6));
    unsigned g = (unsigned)ceil_div(n, WT);
    const bool with_p = alpha != 0.0 && p;
    const bool screen = !with_p && tile_counts != nullptr;
    if (with_p)
        k_weights_dw<true, false><<<g, TPB, 0, ISO_S(s)>>>((const float *)X, n, d, nnbits, is_h, is_l, is, tab, alpha,
                                                          include_self, zskip, shrink, omega, p, tile_counts);
    else if (screen)
        k_weights_dw<false, true><<<g, TPB, 0, ISO_S(s)>>>((const float *)X, n, d, nnbits, is_h, is_l, is, tab, alpha,
                                                          include_self, zskip, shrink, omega, p, tile_counts);
    else
        k_weights_dw<false, false><<<g, TPB, 0, ISO_S(s)>>>((const float *)X, n, d, nnbits, is_h, is_l, is, tab,
                                                           alpha, include_self, zskip, shrink, omega, p, tile_counts);
    if (!with_p && p) {
        cudaError_t e2 = cudaMemsetAsync(p, 0, sizeof(double) * n, s);
        if (e2 != cudaSuccess) return e2;
    }
    return cudaGetLastError();
}

}  // namespace iso

// adjoint.cu -- the derivative of i_k through the fixed tree and subpartition.
//
// With alpha = 0 the cost of a k-subpartition (Section 2.1) is
// max_j phi(dA_j) / omega(A_j): dA_j the tree edges with exactly one end in
// A_j, phi of eq. phi on each, omega(A_j) the sum of eq. omega over A_j.  The
// points enter as z = s (.) x (a per-feature scale) and the bandwidth sigma
// enters eq. phi and eq. omega.  Holding the tree and the subpartition found
// by the forward pass fixed, i_k = R = Phi / Omega for the set A* of the
// largest ratio and dR = (dPhi - R dOmega) / Omega, with
//   d phi(e) / d z_u = -phi (z_u - z_v) / (sigma r_e) = -d phi(e) / d z_v,
//   d phi(e) / d sigma = phi r_e / sigma^2,
//   Omega = sum_{i in A*} sum_{j != i} w_ij: an ordered pair (i in A*, j)
//   adds -w (z_i - z_j) / (sigma r) to d/dz_i, the opposite to d/dz_j and
//   w r / sigma^2 to d/dsigma.
// Everything is FP64 (the derivative is compared with FP64 finite
// differences).  The pair sums run in 64 x 64 tiles with 4 x 4 register
// blocks: squared distances from dot products, the pair coefficients in
// shared memory, then applied to the column points as a small matrix
// product; partial sums per work item are added in a fixed order, so the
// result is deterministic.  Rows of A* pair with every point, the other rows
// with the points of A* only.
#include <vector>

#include "common.cuh"
#include "dwmath.cuh"

namespace iso {
cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s);

namespace {
constexpr int TPB = 256;

inline unsigned grid_for(int64_t n) {
    const int64_t b = n > 0 ? ceil_div(n, TPB) : 1, cap = (int64_t)num_sms() * 16;
    return (unsigned)(b < cap ? b : cap);
}

template <class T>
__device__ __forceinline__ double zv(const T *__restrict__ X, const double *__restrict__ s, int64_t i, int32_t t,
                                     int32_t d) {
    return __dmul_rn(s[t], (double)X[i * d + t]);
}

// Phi_j and Omega_j of every label from the forward's phi / omega: only to
// pick A* (the largest ratio; the smallest label among equal ratios).
__global__ void k_label_sums(const int32_t *__restrict__ parent, const int32_t *__restrict__ labels,
                             const double *__restrict__ phi, const double *__restrict__ omega, int64_t n,
                             int32_t k, double *phik, double *omk) {
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        const int32_t a = labels[v];
        if (a >= 0 && a < k) atomicAdd(omk + a, omega[v]);
        const int32_t u = parent[v];
        if (u < 0) continue;
        const int32_t b = labels[u];
        if (a == b) continue;
        if (a >= 0 && a < k) atomicAdd(phik + a, phi[v]);
        if (b >= 0 && b < k) atomicAdd(phik + b, phi[v]);
    }
}

__global__ void k_pick_set(const double *__restrict__ phik, const double *__restrict__ omk, int32_t k,
                           int32_t *jstar, uint32_t *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t best = 0;
    for (int32_t j = 0; j < k; ++j) {
        if (!(omk[j] > 0.0)) {                 // an empty label or a non-positive omega
            atomicOr(st, DEV_NEGATIVE);
            *jstar = 0;
            return;
        }
        if (j > 0 && phik[j] / omk[j] > phik[best] / omk[best]) best = j;
    }
    *jstar = best;
}

// membership of A*, boundary flags (v's parent edge has one end in A*)
__global__ void k_set_flags(const int32_t *__restrict__ parent, const int32_t *__restrict__ labels, int64_t n,
                            const int32_t *__restrict__ jstar, int32_t *__restrict__ fa, int32_t *__restrict__ fb,
                            int32_t *__restrict__ fe) {
    const int32_t js = *jstar;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        const int in = labels[v] == js;
        fa[v] = in;
        fb[v] = 1 - in;
        const int32_t u = parent[v];
        fe[v] = (u >= 0 && in != (labels[u] == js)) ? 1 : 0;
    }
}

__global__ void k_compact(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int64_t n,
                          int32_t *__restrict__ list, int32_t *count) {
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs) {
        if (flag[v]) list[pos[v]] = (int32_t)v;
        if (v == n - 1) *count = pos[v] + flag[v];
    }
}

// Boundary edges of A*, in vertex order, one block: Phi, dPhi/dsigma and
// dPhi/dz at both ends (threads over the dimensions).
template <class T>
__global__ void __launch_bounds__(TPB) k_phi_grad(const T *__restrict__ X, const double *__restrict__ s, int32_t d,
                                                  const int32_t *__restrict__ parent, const int32_t *__restrict__ elist,
                                                  const int32_t *__restrict__ ecount, double sigma,
                                                  double *__restrict__ gphi, double *out2) {
    __shared__ double red[TPB];
    const int tid = threadIdx.x;
    const int32_t m = *ecount;
    double Phi = 0.0, Psig = 0.0;
    for (int32_t e = 0; e < m; ++e) {
        const int64_t v = elist[e], u = parent[v];
        double acc = 0.0;
        for (int32_t t = tid; t < d; t += TPB) {
            const double dz = __dsub_rn(zv(X, s, v, t, d), zv(X, s, u, t, d));
            acc = __fma_rn(dz, dz, acc);
        }
        red[tid] = acc;
        __syncthreads();
        for (int q = TPB / 2; q > 0; q >>= 1) {
            if (tid < q) red[tid] = __dadd_rn(red[tid], red[tid + q]);
            __syncthreads();
        }
        const double r = sqrt(red[0]);
        __syncthreads();
        const double f = exp(-r / sigma);
        Phi = Phi + f;
        Psig = Psig + f * r / (sigma * sigma);
        if (r > 0.0) {
            const double c = -f / (sigma * r);
            for (int32_t t = tid; t < d; t += TPB) {
                const double dz = __dsub_rn(zv(X, s, v, t, d), zv(X, s, u, t, d));
                gphi[v * d + t] = __fma_rn(c, dz, gphi[v * d + t]);
                gphi[u * d + t] = __fma_rn(-c, dz, gphi[u * d + t]);
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        out2[0] = Phi;
        out2[1] = Psig;
    }
}

// Omega's pair sums.  Work item = (row group, 64-row
// tile of the group's list, chunk of GC columns): group 0 = rows of A*
// against every point, group 1 = the other rows against A*.  Per 64 x 64
// pair tile (all of a point's first 128 dimensions in shared memory at
// once): squared distances from dot products, |z_i|^2 + |z_j|^2 - 2 z_i.z_j
// (4 x 4 pairs per thread), with a direct FP64 recomputation where that
// cancels (d2 < 2^-20 (|z_i|^2 + |z_j|^2)); the coefficients
// c_ij = -m w / (sigma r), w = exp(-r / sigma), in shared memory; then
// V_i += sum_j c_ij z_j (512 threads, 2 rows x 8 dimensions each).  Everything
// runs in double-word FP32, where GB300's FP32 pipe has 64 times the FP64
// rate: the two d-long sums on z's double-word copy (exact products by FMA,
// TwoSum of the high parts, low parts summed in FP32 and renormalised every
// 16 dimensions or 64 columns: relative error ~ d 2^-48), the root and
// reciprocal by one correction of their FP32 values, the exp by the
// table-driven double-word exp of the omega sweep.  A pair whose r / sigma
// exceeds 80 (past FP32's exponent range) takes the FP64 path; omega's own
// sums (w and w r / sigma^2) are added in FP64.  Each item writes its
// partial sums to its own slot; k_pair_reduce adds the slots of a row in
// chunk order.
constexpr int GT = 64;              // rows / columns per pair tile
constexpr int GK = 128;             // dimensions per shared-memory block (and of V per pass)
constexpr int GS = GT + 1;          // padded stride of the shared-memory blocks (bank-conflict free)
constexpr int GP = 512;             // threads of the pair kernel: 32 x 16
constexpr int GR = GT / (GP / 16);  // rows per thread (2)
constexpr int GC = 4096;            // columns per work item

struct PairItem {
    int32_t group, tile, chunk, pad;
};

// (sh, sl) += (ah + al)(bh + bl): the product's error by FMA, the cross
// terms rounded (the lo.lo term is below 2^-48 of the product), the high
// parts added by TwoSum, everything else gathered in sl (renormalised by
// the caller)
__device__ __forceinline__ void dw_mac(float ah, float al, float bh, float bl, float &sh, float &sl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float t = __fadd_rn(sh, p);
    const float bb = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}
__device__ __forceinline__ void dw_norm(float &h, float &l) {
    const float t = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(t, h));
    h = t;
}
__device__ __forceinline__ float2 dw_of(double z) {
    const float h = __double2float_rn(z);
    return make_float2(h, __double2float_rn(__dsub_rn(z, (double)h)));
}
// (ah + al)(bh + bl) as a double-word (the lo.lo term dropped)
__device__ __forceinline__ void dw_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    fast_two_sum(p, e, ph, pl);
}

// z = s (.) x of every point as double-words, once per call
template <class T>
__global__ void k_z_dw(const T *__restrict__ X, const double *__restrict__ s, int64_t n, int32_t d,
                       float2 *__restrict__ Zd) {
    const int64_t tot = n * (int64_t)d, gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gs) {
        const int32_t t = (int32_t)(e % d);
        Zd[e] = dw_of(__dmul_rn(s[t], (double)X[e]));
    }
}

template <class T>
__global__ void __launch_bounds__(GP, 1)
k_pair_grad(const T *__restrict__ X, const double *__restrict__ s, int64_t n, int32_t d,
            const double *__restrict__ N2, const int32_t *__restrict__ inA, const int32_t *__restrict__ alist,
            const int32_t *__restrict__ blist, const int32_t *__restrict__ cnt, const PairItem *__restrict__ items,
            int64_t nitems, double sigma, const float2 *__restrict__ Zd, ExpTable tabv, double *__restrict__ Vp,
            double *__restrict__ Cp, double *__restrict__ Op, double *__restrict__ Sp) {
    extern __shared__ __align__(16) float2 gsm[];
    const double isg = 1.0 / sigma, isg2 = isg * isg;
    const float2 isw = dw_of(isg);                     // 1/sigma as a double-word
    __shared__ float2 tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = tabv.t[threadIdx.x];
    float2 *Zr = gsm;                                  // [GK][GS] double-word z of the rows (dimension-major)
    float2 *Zc = Zr + GK * GS;                         // [GK][GS] of the columns
    float2 *Cm = Zc + GK * GS;                         // [GT][GS] double-word coefficients
    __shared__ int32_t ri[GT], ci[GT], rin[GT], cin[GT];
    __shared__ float2 rn[GT], cn[GT];                  // |z|^2 as double-words
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int32_t na = cnt[1], nb = cnt[2];
    const float2 zero2 = make_float2(0.f, 0.f);
    // dimensions [k0, k0 + GK) of the 64 listed points idx[] into Z (GS-strided rows of dims)
    auto load_block = [&](float2 *Z, const int32_t *idx, int32_t k0) {
        const int32_t kl = min(GK, d - k0);
        for (int e = tid; e < GK * GT; e += GP) {
            const int c = e / GK, t = e % GK;
            Z[t * GS + c] = (t < kl && idx[c] >= 0) ? Zd[(int64_t)idx[c] * d + k0 + t] : zero2;
        }
    };
    for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {
        const PairItem it = items[w];
        const int32_t *rlist = it.group == 0 ? alist : blist;
        const int64_t nr = it.group == 0 ? na : nb;
        const int64_t ncol = it.group == 0 ? n : na;
        const int64_t q0 = (int64_t)it.chunk * GC, q1 = min(ncol, q0 + GC);
        __syncthreads();
        if (tid < GT) {
            const int64_t q = (int64_t)it.tile * GT + tid;
            ri[tid] = q < nr ? rlist[q] : -1;
            rin[tid] = ri[tid] >= 0 ? inA[ri[tid]] : 0;
            rn[tid] = ri[tid] >= 0 ? dw_of(N2[ri[tid]]) : zero2;
        }
        __syncthreads();
        int32_t zr_k0 = -1;                            // chunk of dimensions held in Zr
        double csum[GR], osum[GR], ssum[GR];
#pragma unroll
        for (int i = 0; i < GR; ++i) { csum[i] = 0.0; osum[i] = 0.0; ssum[i] = 0.0; }
        for (int32_t v0 = 0; v0 < d; v0 += GK) {
            // thread (ty, tx): rows ty*GR+i, dimensions v0 + hh*16 + tx
            float Vh[GR][GK / 16], Vl[GR][GK / 16];
#pragma unroll
            for (int i = 0; i < GR; ++i)
#pragma unroll
                for (int c = 0; c < GK / 16; ++c) { Vh[i][c] = 0.f; Vl[i][c] = 0.f; }
            for (int64_t c0 = q0; c0 < q1; c0 += GT) {
                __syncthreads();                       // readers of ci, Zc and Cm of the last tile are done
                if (tid < GT) {
                    const int64_t q = c0 + tid;
                    const int64_t j = q < q1 ? (it.group == 0 ? q : (int64_t)alist[q]) : -1;
                    ci[tid] = (int32_t)j;
                    cin[tid] = j >= 0 ? inA[j] : 0;
                    cn[tid] = j >= 0 ? dw_of(N2[j]) : zero2;
                }
                __syncthreads();
                // ---- dot products z_i . z_j (double-word): thread (ty, tx) takes
                //      rows ty*GR+i and columns j*16+tx (conflict-free loads)
                float gh[GR][4], gl[GR][4];
#pragma unroll
                for (int i = 0; i < GR; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) { gh[i][j] = 0.f; gl[i][j] = 0.f; }
                int32_t zc_k0 = -1;
                for (int32_t k0 = 0; k0 < d; k0 += GK) {
                    if (k0 > 0) __syncthreads();
                    if (zr_k0 != k0) load_block(Zr, ri, k0);
                    load_block(Zc, ci, k0);
                    zr_k0 = k0;
                    zc_k0 = k0;
                    __syncthreads();
                    const int32_t kl = min(GK, d - k0);
                    for (int32_t t0 = 0; t0 < kl; t0 += 16) {
                        const int32_t tl = min(16, kl - t0);
#pragma unroll 4
                        for (int t = t0; t < t0 + tl; ++t) {
                            float2 a[GR], b[4];
#pragma unroll
                            for (int i = 0; i < GR; ++i) a[i] = Zr[t * GS + ty * GR + i];
#pragma unroll
                            for (int j = 0; j < 4; ++j) b[j] = Zc[t * GS + j * 16 + tx];
#pragma unroll
                            for (int i = 0; i < GR; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) dw_mac(a[i].x, a[i].y, b[j].x, b[j].y, gh[i][j], gl[i][j]);
                        }
#pragma unroll
                        for (int i = 0; i < GR; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) dw_norm(gh[i][j], gl[i][j]);
                    }
                }
                // ---- pair coefficients c_ij = -m w / (sigma r) with w = exp(-r / sigma),
                //      in double-word FP32; omega's sums (w, w r / sigma^2) in FP64
#pragma unroll
                for (int i = 0; i < GR; ++i) {
                    const int r = ty * GR + i;
                    float csh = 0.f, csl = 0.f;
                    double os = 0.0, ss = 0.0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = j * 16 + tx;
                        const int32_t gi = ri[r], gj = ci[c];
                        const int mult = rin[r] + cin[c];
                        float cch = 0.f, ccl = 0.f;
                        if (gi >= 0 && gj >= 0 && gi != gj && mult > 0) {
                            float nh = rn[r].x, nl = rn[r].y;
                            dw_add(nh, nl, cn[c].x, cn[c].y);              // |z_i|^2 + |z_j|^2
                            float r2h = nh, r2l = nl;
                            dw_add(r2h, r2l, -2.0f * gh[i][j], -2.0f * gl[i][j]);
                            if (r2h < nh * 9.5367431640625e-07f) {      // cancellation: direct FP64 differences
                                double dd = 0.0;
                                for (int32_t t = 0; t < d; ++t) {
                                    const double df = __dsub_rn(zv(X, s, gi, t, d), zv(X, s, gj, t, d));
                                    dd = __fma_rn(df, df, dd);
                                }
                                const float2 q = dw_of(dd);
                                r2h = q.x;
                                r2l = q.y;
                            }
                            if (!(r2h > 0.f)) { r2h = 0.f; r2l = 0.f; }
                            // r by one correction of the FP32 root; 1/r likewise
                            const float rh = __fsqrt_rn(r2h);
                            float rl = 0.f, qh = 0.f, ql = 0.f;
                            if (rh > 0.f) {
                                rl = __fmul_rn(__fadd_rn(__fmaf_rn(-rh, rh, r2h), r2l), __frcp_rn(__fadd_rn(rh, rh)));
                                qh = __frcp_rn(rh);
                                float t = __fmaf_rn(-rh, qh, 1.0f);
                                t = __fmaf_rn(-rl, qh, t);
                                ql = __fmul_rn(t, qh);
                            }
                            float zh, zl;
                            dw_mul(rh, rl, isw.x, isw.y, zh, zl);          // r / sigma
                            double wwd;
                            if (zh <= 80.0f) {
                                float wh, wl, ah, al, bh, bl;
                                dw_exp_neg(zh, zl, tab, wh, wl);
                                dw_mul(isw.x, isw.y, qh, ql, ah, al);     // 1 / (sigma r)
                                dw_mul(wh, wl, ah, al, bh, bl);
                                if (rh > 0.f) {
                                    cch = -(float)mult * bh;                // mult is 1 or 2: exact
                                    ccl = -(float)mult * bl;
                                }
                                wwd = __dadd_rn((double)wh, (double)wl);
                            } else {
                                // past FP32's exponent range: the pair in FP64
                                const double rd = __dadd_rn((double)rh, (double)rl);
                                wwd = exp(-rd * isg);
                                const float2 q = dw_of(-(double)mult * wwd * (isg / rd));
                                cch = q.x;
                                ccl = q.y;
                            }
                            if (rin[r] && v0 == 0) {
                                os = os + wwd;
                                ss = ss + wwd * __dadd_rn((double)rh, (double)rl) * isg2;
                            }
                        }
                        Cm[r * GS + c] = make_float2(cch, ccl);
                        dw_add(csh, csl, cch, ccl);
                    }
                    // rows' sums over this tile's 64 columns: the 16 threads of a row, in order
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) {
                        const float oh = __shfl_down_sync(0xffffffffu, csh, o, 16);
                        const float ol = __shfl_down_sync(0xffffffffu, csl, o, 16);
                        dw_add(csh, csl, oh, ol);
                        os = os + __shfl_down_sync(0xffffffffu, os, o, 16);
                        ss = ss + __shfl_down_sync(0xffffffffu, ss, o, 16);
                    }
                    if (v0 == 0) {
                        csum[i] = csum[i] + __dadd_rn((double)csh, (double)csl);
                        osum[i] = osum[i] + os;
                        ssum[i] = ssum[i] + ss;
                    }
                }
                // ---- V[r][t] += sum_c C[r][c] z_c[t], t in [v0, v0 + GK): the
                //      columns' chunk v0 is in Zc unless d > GK moved past it
                if (zc_k0 != v0) {
                    __syncthreads();
                    load_block(Zc, ci, v0);
                }
                __syncthreads();                       // Cm (and Zc) complete
#pragma unroll 2
                for (int c = 0; c < GT; ++c) {
                    float2 zc[GK / 16], cf[GR];
#pragma unroll
                    for (int hh = 0; hh < GK / 16; ++hh) zc[hh] = Zc[(hh * 16 + tx) * GS + c];
#pragma unroll
                    for (int i = 0; i < GR; ++i) cf[i] = Cm[(ty * GR + i) * GS + c];
#pragma unroll
                    for (int i = 0; i < GR; ++i)
#pragma unroll
                        for (int hh = 0; hh < GK / 16; ++hh)
                            dw_mac(cf[i].x, cf[i].y, zc[hh].x, zc[hh].y, Vh[i][hh], Vl[i][hh]);
                }
#pragma unroll
                for (int i = 0; i < GR; ++i)
#pragma unroll
                    for (int hh = 0; hh < GK / 16; ++hh) dw_norm(Vh[i][hh], Vl[i][hh]);
            }
            // partial V of this item: rows ty*GR+i, dimension v0 + hh*16 + tx
#pragma unroll
            for (int i = 0; i < GR; ++i)
#pragma unroll
                for (int hh = 0; hh < GK / 16; ++hh) {
                    const int32_t t = v0 + hh * 16 + tx;
                    if (t < d) Vp[(w * GT + ty * GR + i) * (int64_t)d + t] = __dadd_rn((double)Vh[i][hh], (double)Vl[i][hh]);
                }
        }
        if (tx == 0) {
#pragma unroll
            for (int i = 0; i < GR; ++i) {
                const int r = ty * GR + i;
                Cp[w * GT + r] = csum[i];
                Op[w * GT + r] = osum[i];
                Sp[w * GT + r] = ssum[i];
            }
        }
    }
}

// gom[i] = C_i z_i - V_i, omega_i and the sigma term of every listed row:
// the item slots of its row tile added in chunk order.
template <class T>
__global__ void k_pair_reduce(const T *__restrict__ X, const double *__restrict__ s, int64_t n, int32_t d,
                              const int32_t *__restrict__ alist, const int32_t *__restrict__ blist,
                              const int32_t *__restrict__ cnt, int64_t itemsA, int64_t chunksA, int64_t chunksB,
                              const double *__restrict__ Vp, const double *__restrict__ Cp,
                              const double *__restrict__ Op, const double *__restrict__ Sp, double *__restrict__ gom,
                              double *__restrict__ rowom, double *__restrict__ rowsig) {
    const int32_t na = cnt[1], nb = cnt[2];
    const int64_t total = (int64_t)na + nb;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total * (int64_t)d; e += gs) {
        const int64_t q = e / d;
        const int32_t t = (int32_t)(e - q * d);
        const bool ga = q < na;
        const int64_t qq = ga ? q : q - na;
        const int32_t i = ga ? alist[qq] : blist[qq];
        const int64_t tile = qq / GT, r = qq - tile * GT;
        const int64_t nch = ga ? chunksA : chunksB;
        const int64_t w0 = ga ? tile * chunksA : itemsA + tile * chunksB;
        double cs = 0.0, vs = 0.0;
        for (int64_t k = 0; k < nch; ++k) {
            cs = cs + Cp[(w0 + k) * GT + r];
            vs = vs + Vp[((w0 + k) * GT + r) * (int64_t)d + t];
        }
        gom[(int64_t)i * d + t] = __fma_rn(cs, zv(X, s, i, t, d), -vs);
        if (t == 0) {
            double os = 0.0, ss = 0.0;
            for (int64_t k = 0; k < nch; ++k) {
                os = os + Op[(w0 + k) * GT + r];
                ss = ss + Sp[(w0 + k) * GT + r];
            }
            rowom[i] = os;
            rowsig[i] = ss;
        }
    }
}

__global__ void k_row_norms(const float *__restrict__ Xf, const double *__restrict__ Xd, const double *__restrict__ s,
                            int64_t n, int32_t d, double *__restrict__ N2) {
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        double acc = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            const double z = Xf ? zv(Xf, s, i, t, d) : zv(Xd, s, i, t, d);
            acc = __fma_rn(z, z, acc);
        }
        N2[i] = acc;
    }
}

// Omega = sum of rowom over A*, Omega_sigma likewise (fixed order, one block)
__global__ void __launch_bounds__(TPB) k_omega_total(const int32_t *__restrict__ alist, const int32_t *__restrict__ acount,
                                                     const double *__restrict__ rowom, const double *__restrict__ rowsig,
                                                     double *out2) {
    __shared__ double a[TPB], b[TPB];
    const int tid = threadIdx.x;
    const int32_t m = *acount;
    double x = 0.0, y = 0.0;
    for (int32_t q = tid; q < m; q += TPB) {
        x = __dadd_rn(x, rowom[alist[q]]);
        y = __dadd_rn(y, rowsig[alist[q]]);
    }
    a[tid] = x;
    b[tid] = y;
    __syncthreads();
    for (int q = TPB / 2; q > 0; q >>= 1) {
        if (tid < q) {
            a[tid] = __dadd_rn(a[tid], a[tid + q]);
            b[tid] = __dadd_rn(b[tid], b[tid + q]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        out2[0] = a[0];
        out2[1] = b[0];
    }
}

// dX = g s (dPhi - R dOmega) / Omega; per feature dscale (rows in order); dsigma
template <class T>
__global__ void k_grad_out(const T *__restrict__ X, const double *__restrict__ s, int64_t n, int32_t d,
                           const double *__restrict__ gphi, const double *__restrict__ gom,
                           const double *__restrict__ phi2, const double *__restrict__ om2, double g,
                           double *__restrict__ dX) {
    const double Omega = om2[0], R = phi2[0] / Omega;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += gs) {
        const int32_t t = (int32_t)(e % d);
        const double gz = (gphi[e] - R * gom[e]) / Omega;
        dX[e] = g * gz * s[t];
    }
}

// d i_k / d scale_t = g / Omega sum_i (gphi_it - R gom_it) x_it: rows in
// GS_CHUNKS chunks (block (t-group, chunk), 32 dimensions x 8 row lanes,
// lanes added in order), then the chunks added in order by k_grad_scale.
constexpr int GS_CHUNKS = 64;
template <class T>
__global__ void __launch_bounds__(256) k_grad_scale_part(const T *__restrict__ X, int64_t n, int32_t d,
                                                         const double *__restrict__ gphi,
                                                         const double *__restrict__ gom,
                                                         const double *__restrict__ phi2,
                                                         const double *__restrict__ om2, double *__restrict__ part) {
    __shared__ double red[8][33];
    const double R = phi2[0] / om2[0];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int32_t t = blockIdx.x * 32 + tx;
    const int64_t per = (n + GS_CHUNKS - 1) / GS_CHUNKS;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(n, i0 + per);
    double acc = 0.0;
    if (t < d)
        for (int64_t i = i0 + ty; i < i1; i += 8)
            acc = __fma_rn(__fma_rn(-R, gom[i * d + t], gphi[i * d + t]), (double)X[i * d + t], acc);
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && t < d) {
        double sum = 0.0;
        for (int q = 0; q < 8; ++q) sum = sum + red[q][tx];
        part[(int64_t)blockIdx.y * d + t] = sum;
    }
}

__global__ void k_grad_scale(int32_t d, const double *__restrict__ part, const double *__restrict__ phi2,
                             const double *__restrict__ om2, double g, double *__restrict__ dscale,
                             double *__restrict__ dsigma, double *__restrict__ ik) {
    const double Omega = om2[0], R = phi2[0] / Omega;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < d) {
        double acc = 0.0;
        for (int c = 0; c < GS_CHUNKS; ++c) acc = acc + part[(int64_t)c * d + t];
        dscale[t] = g * acc / Omega;
    }
    if (t == 0) {
        dsigma[0] = g * (phi2[1] - R * om2[1]) / Omega;
        if (ik) ik[0] = R;
    }
}

template <class T>
__global__ void k_scale_rows(const T *__restrict__ X, const double *__restrict__ s, int64_t n, int32_t d,
                             T *__restrict__ Z) {
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += gs)
        Z[e] = (T)__dmul_rn(s[e % d], (double)X[e]);
}
}  // namespace

static int64_t pair_items_bound(int64_t n) {
    return 2 * ceil_div(n, GT) * ceil_div(n, GC) + 2;
}

size_t adjoint_bytes(int64_t n, int32_t d, int32_t k) {
    Arena A;
    const int64_t mi = pair_items_bound(n);
    A.take<double>(n);
    A.take<PairItem>(mi);
    A.take<double>((size_t)mi * GT * d);
    A.take<double>((size_t)mi * GT * 3);
    A.take<double>((size_t)n * d);
    A.take<double>((size_t)n * d);
    A.take<float2>((size_t)n * d);
    A.take<double>(n);
    A.take<double>(n);
    A.take<int32_t>(n);
    A.take<int32_t>(n);
    A.take<int32_t>(n);
    A.take<int32_t>(n);
    A.take<int32_t>(n);
    A.take<int32_t>(n);
    A.take<int32_t>(n + 1);
    A.take<int32_t>(n + 1);
    A.take<int32_t>(n + 1);
    A.take<int32_t>(scan_tmp_elems(n + 1));
    A.take<double>(k);
    A.take<double>(k);
    A.take<double>(4);
    A.take<int32_t>(8);
    A.take<double>((size_t)GS_CHUNKS * d);
    return A.off;
}

// Work space carved from `ws` (adjoint_bytes); outputs on the stream.
cudaError_t adjoint_launch(const void *X, int32_t dtype, int64_t n, int32_t d, const double *scale, double sigma,
                           const int32_t *parent, const int32_t *labels, int32_t k, const double *phi_par,
                           const double *omega, double grad, double *dX, double *dscale, double *dsigma, double *ik,
                           void *ws, uint32_t *status, cudaEvent_t *kev, cudaStream_t s) {
    Arena A{(char *)ws, adjoint_bytes(n, d, k) + 4096, 0, false};
    const int64_t mi = pair_items_bound(n);
    double *N2 = A.take<double>(n);
    PairItem *pitems = A.take<PairItem>(mi);
    double *Vp = A.take<double>((size_t)mi * GT * d);
    double *Cp = A.take<double>((size_t)mi * GT * 3);
    double *Op = Cp + mi * GT, *Sp = Op + mi * GT;
    double *gphi = A.take<double>((size_t)n * d);
    double *gom = A.take<double>((size_t)n * d);
    float2 *Zd = A.take<float2>((size_t)n * d);
    double *rowom = A.take<double>(n);
    double *rowsig = A.take<double>(n);
    int32_t *fa = A.take<int32_t>(n);
    int32_t *fb = A.take<int32_t>(n);
    int32_t *fe = A.take<int32_t>(n);
    int32_t *alist = A.take<int32_t>(n);
    int32_t *blist = A.take<int32_t>(n);
    int32_t *elist = A.take<int32_t>(n);
    int32_t *pa = A.take<int32_t>(n + 1);
    int32_t *pb = A.take<int32_t>(n + 1);
    int32_t *pe = A.take<int32_t>(n + 1);
    int32_t *tmp = A.take<int32_t>(scan_tmp_elems(n + 1));
    double *phik = A.take<double>(k);
    double *omk = A.take<double>(k);
    double *sums = A.take<double>(4);      // Phi, Phi_sigma, Omega, Omega_sigma
    int32_t *cnt = A.take<int32_t>(8);     // jstar, |A*|, |rest|, |boundary|
    double *gpart = A.take<double>((size_t)GS_CHUNKS * d);
    if (A.overflow) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(gphi, 0, sizeof(double) * n * d, s))) return e;
    if ((e = cudaMemsetAsync(phik, 0, sizeof(double) * k, s))) return e;
    if ((e = cudaMemsetAsync(omk, 0, sizeof(double) * k, s))) return e;
    if ((e = cudaMemsetAsync(rowom, 0, sizeof(double) * n, s))) return e;
    if ((e = cudaMemsetAsync(rowsig, 0, sizeof(double) * n, s))) return e;
    const unsigned g = grid_for(n);
    k_label_sums<<<g, TPB, 0, ISO_S(s)>>>(parent, labels, phi_par, omega, n, k, phik, omk);
    k_pick_set<<<1, 32, 0, ISO_S(s)>>>(phik, omk, k, cnt, status);
    k_set_flags<<<g, TPB, 0, ISO_S(s)>>>(parent, labels, n, cnt, fa, fb, fe);
    if ((e = exclusive_scan_i32(fa, pa, n, tmp, s))) return e;
    k_compact<<<g, TPB, 0, ISO_S(s)>>>(fa, pa, n, alist, cnt + 1);
    if ((e = exclusive_scan_i32(fb, pb, n, tmp, s))) return e;
    k_compact<<<g, TPB, 0, ISO_S(s)>>>(fb, pb, n, blist, cnt + 2);
    if ((e = exclusive_scan_i32(fe, pe, n, tmp, s))) return e;
    k_compact<<<g, TPB, 0, ISO_S(s)>>>(fe, pe, n, elist, cnt + 3);
    // list sizes on the host: they shape the work items of the pair sums
    int32_t hc[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    const int64_t na = hc[1], nb = hc[2];
    const int64_t chunksA = ceil_div(n, GC), chunksB = na > 0 ? ceil_div(na, GC) : 0;
    const int64_t tilesA = ceil_div(na, GT), tilesB = na > 0 ? ceil_div(nb, GT) : 0;
    std::vector<PairItem> items;
    for (int64_t t = 0; t < tilesA; ++t)
        for (int64_t c = 0; c < chunksA; ++c) items.push_back(PairItem{0, (int32_t)t, (int32_t)c, 0});
    for (int64_t t = 0; t < tilesB; ++t)
        for (int64_t c = 0; c < chunksB; ++c) items.push_back(PairItem{1, (int32_t)t, (int32_t)c, 0});
    const int64_t nit = (int64_t)items.size();
    if (nit > mi) return cudaErrorInvalidValue;
    if (nit > 0 &&
        (e = cudaMemcpyAsync(pitems, items.data(), sizeof(PairItem) * nit, cudaMemcpyHostToDevice, s)))
        return e;
    const size_t gsm = sizeof(float2) * (2 * GK * GS + GT * GS);
    static const ExpTable tab = make_exp_table();
    const unsigned gp = (unsigned)(nit < num_sms() ? (nit > 0 ? nit : 1) : num_sms());
    const unsigned gr = grid_for((na + nb) * d);
    static bool attr = false;
    if (!attr) {
        if ((e = cudaFuncSetAttribute(k_pair_grad<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm)))
            return e;
        if ((e = cudaFuncSetAttribute(k_pair_grad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm)))
            return e;
        attr = true;
    }
    if (dtype == ISOCLUST_F64) {
        const double *Xd = (const double *)X;
        k_phi_grad<double><<<1, TPB, 0, ISO_S(s)>>>(Xd, scale, d, parent, elist, cnt + 3, sigma, gphi, sums);
        k_row_norms<<<g, TPB, 0, ISO_S(s)>>>(nullptr, Xd, scale, n, d, N2);
        k_z_dw<double><<<grid_for(n * d), TPB, 0, ISO_S(s)>>>(Xd, scale, n, d, Zd);
        if (kev) record_event(kev[0], s);
        if (nit > 0)
            k_pair_grad<double><<<gp, GP, gsm, ISO_S(s)>>>(Xd, scale, n, d, N2, fa, alist, blist, cnt, pitems, nit,
                                                             sigma, Zd, tab, Vp, Cp, Op, Sp);
        if (kev) record_event(kev[1], s);
        k_pair_reduce<double><<<gr, TPB, 0, ISO_S(s)>>>(Xd, scale, n, d, alist, blist, cnt, tilesA * chunksA, chunksA,
                                                         chunksB, Vp, Cp, Op, Sp, gom, rowom, rowsig);
        k_omega_total<<<1, TPB, 0, ISO_S(s)>>>(alist, cnt + 1, rowom, rowsig, sums + 2);
        k_grad_out<double><<<grid_for(n * d), TPB, 0, ISO_S(s)>>>(Xd, scale, n, d, gphi, gom, sums, sums + 2, grad, dX);
        k_grad_scale_part<double><<<dim3((unsigned)ceil_div(d, 32), GS_CHUNKS), 256, 0, ISO_S(s)>>>(
            Xd, n, d, gphi, gom, sums, sums + 2, gpart);
        k_grad_scale<<<(unsigned)ceil_div(d, 128), 128, 0, ISO_S(s)>>>(d, gpart, sums, sums + 2, grad, dscale, dsigma,
                                                                      ik);
    } else {
        const float *Xf = (const float *)X;
        k_phi_grad<float><<<1, TPB, 0, ISO_S(s)>>>(Xf, scale, d, parent, elist, cnt + 3, sigma, gphi, sums);
        k_row_norms<<<g, TPB, 0, ISO_S(s)>>>(Xf, nullptr, scale, n, d, N2);
        k_z_dw<float><<<grid_for(n * d), TPB, 0, ISO_S(s)>>>(Xf, scale, n, d, Zd);
        if (kev) record_event(kev[0], s);
        if (nit > 0)
            k_pair_grad<float><<<gp, GP, gsm, ISO_S(s)>>>(Xf, scale, n, d, N2, fa, alist, blist, cnt, pitems, nit,
                                                            sigma, Zd, tab, Vp, Cp, Op, Sp);
        if (kev) record_event(kev[1], s);
        k_pair_reduce<float><<<gr, TPB, 0, ISO_S(s)>>>(Xf, scale, n, d, alist, blist, cnt, tilesA * chunksA, chunksA,
                                                        chunksB, Vp, Cp, Op, Sp, gom, rowom, rowsig);
        k_omega_total<<<1, TPB, 0, ISO_S(s)>>>(alist, cnt + 1, rowom, rowsig, sums + 2);
        k_grad_out<float><<<grid_for(n * d), TPB, 0, ISO_S(s)>>>(Xf, scale, n, d, gphi, gom, sums, sums + 2, grad, dX);
        k_grad_scale_part<float><<<dim3((unsigned)ceil_div(d, 32), GS_CHUNKS), 256, 0, ISO_S(s)>>>(
            Xf, n, d, gphi, gom, sums, sums + 2, gpart);
        k_grad_scale<<<(unsigned)ceil_div(d, 128), 128, 0, ISO_S(s)>>>(d, gpart, sums, sums + 2, grad, dscale, dsigma,
                                                                      ik);
    }
    return cudaGetLastError();
}

cudaError_t scale_rows_launch(const void *X, int32_t dtype, int64_t n, int32_t d, const double *scale, void *Z,
                              cudaStream_t s) {
    const unsigned g = grid_for(n * d);
    if (dtype == ISOCLUST_F64)
        k_scale_rows<double><<<g, TPB, 0, ISO_S(s)>>>((const double *)X, scale, n, d, (double *)Z);
    else
        k_scale_rows<float><<<g, TPB, 0, ISO_S(s)>>>((const float *)X, scale, n, d, (float *)Z);
    return cudaGetLastError();
}

}  // namespace iso

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
// differences).  The pair sums are tiled: 32 rows x 32 columns per step, the
// pair coefficients in shared memory, then applied to the column points as a
// small matrix product; every row's sums run in a fixed order, so the result
// is deterministic.  Rows of A* pair with every point, the other rows with
// the points of A* only.
#include "common.cuh"

namespace iso {
cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s);

namespace {
constexpr int TPB = 256;
constexpr int AT = 32;        // rows and columns per pair tile
constexpr int ADC = 32;       // dimensions per shared-memory chunk (static shared memory < 48 KB)

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

// Omega's pair sums for the rows in rlist (32 per block-step) against the
// columns in clist (all points when clist is null).  A pair (i, j) counts
// once per end in A* (in_i + in_j); rows of A* also sum w (-> omega_i) and
// w r / sigma^2.  gom[i] = C_i z_i - V_i with C_i = sum_j c_ij,
// V_i = sum_j c_ij z_j, c_ij = -(in_i + in_j) w / (sigma r).  V is held in
// registers for 128 dimensions at a time (larger d: the pairs are revisited
// per 128-dimension chunk).
template <class T>
__global__ void __launch_bounds__(TPB) k_omega_grad(const T *__restrict__ X, const double *__restrict__ s, int64_t n,
                                                    int32_t d, const int32_t *__restrict__ rlist,
                                                    const int32_t *__restrict__ rcount,
                                                    const int32_t *__restrict__ clist,
                                                    const int32_t *__restrict__ ccount,
                                                    const int32_t *__restrict__ inA, double sigma,
                                                    double *__restrict__ gom, double *__restrict__ rowom,
                                                    double *__restrict__ rowsig) {
    constexpr int VQ = (AT * 128) / TPB;      // accumulators per thread: (row, dimension) pairs
    __shared__ double Zr[AT][ADC + 1];
    __shared__ double Zc[AT][ADC + 1];
    __shared__ double C[AT][AT + 1];          // squared distances, then the pair coefficients
    __shared__ double W[AT][AT + 1];
    __shared__ double WR[AT][AT + 1];
    __shared__ int32_t ri[AT], ci[AT], rin[AT], cin[AT];
    __shared__ double Cs[AT];
    const int tid = threadIdx.x;
    const int64_t nr = *rcount, nc = clist ? (int64_t)*ccount : n;
    const int64_t ntr = (nr + AT - 1) / AT, ntc = (nc + AT - 1) / AT;
    const int32_t dchunks = (d + 127) / 128;
    for (int64_t tr = blockIdx.x; tr < ntr; tr += gridDim.x) {
        __syncthreads();
        if (tid < AT) {
            const int64_t q = tr * AT + tid;
            ri[tid] = q < nr ? rlist[q] : -1;
            rin[tid] = q < nr ? inA[ri[tid]] : 0;
        }
        double cs = 0.0, os = 0.0, ss = 0.0;   // row tid < AT: C_i, omega_i, sigma term
        for (int32_t dc = 0; dc < dchunks; ++dc) {
            const int32_t t0 = dc * 128, tl = min(128, d - t0);
            double vacc[VQ];
#pragma unroll
            for (int q = 0; q < VQ; ++q) vacc[q] = 0.0;
            for (int64_t tc = 0; tc < ntc; ++tc) {
                __syncthreads();
                if (tid < AT) {
                    const int64_t q = tc * AT + tid;
                    const int64_t j = q < nc ? (clist ? (int64_t)clist[q] : q) : -1;
                    ci[tid] = (int32_t)j;
                    cin[tid] = j >= 0 ? inA[j] : 0;
                }
                for (int e = tid; e < AT * AT; e += TPB) C[e / AT][e % AT] = 0.0;
                __syncthreads();
                // squared distances of the 32 x 32 pairs over all dimensions
                for (int32_t u0 = 0; u0 < d; u0 += ADC) {
                    const int ul = min(ADC, d - u0);
                    for (int e = tid; e < AT * ADC; e += TPB) {
                        const int r = e / ADC, t = e % ADC;
                        Zr[r][t] = (t < ul && ri[r] >= 0) ? zv(X, s, ri[r], u0 + t, d) : 0.0;
                        Zc[r][t] = (t < ul && ci[r] >= 0) ? zv(X, s, ci[r], u0 + t, d) : 0.0;
                    }
                    __syncthreads();
                    for (int e = tid; e < AT * AT; e += TPB) {
                        const int r = e / AT, c = e % AT;
                        double acc = C[r][c];
                        for (int t = 0; t < ul; ++t) {
                            const double dz = __dsub_rn(Zr[r][t], Zc[c][t]);
                            acc = __fma_rn(dz, dz, acc);
                        }
                        C[r][c] = acc;
                    }
                    __syncthreads();
                }
                // pair coefficients
                for (int e = tid; e < AT * AT; e += TPB) {
                    const int r = e / AT, c = e % AT;
                    const int32_t i = ri[r], j = ci[c];
                    double cc = 0.0, w = 0.0, wr = 0.0;
                    const int mult = rin[r] + cin[c];
                    if (i >= 0 && j >= 0 && i != j && mult > 0) {
                        const double rr = sqrt(C[r][c]);
                        const double ww = exp(-rr / sigma);
                        if (rr > 0.0) cc = -(double)mult * ww / (sigma * rr);
                        if (rin[r]) {
                            w = ww;
                            wr = ww * rr / (sigma * sigma);
                        }
                    }
                    C[r][c] = cc;
                    W[r][c] = w;
                    WR[r][c] = wr;
                }
                __syncthreads();
                if (dc == 0 && tid < AT) {
                    for (int c = 0; c < AT; ++c) {
                        cs = __dadd_rn(cs, C[tid][c]);
                        os = __dadd_rn(os, W[tid][c]);
                        ss = __dadd_rn(ss, WR[tid][c]);
                    }
                }
                // V[r][t] += sum_c C[r][c] z_c[t] over this chunk's dimensions
                for (int32_t h = 0; h < tl; h += ADC) {
                    const int hl = min(ADC, tl - h);
                    __syncthreads();
                    for (int e = tid; e < AT * ADC; e += TPB) {
                        const int c = e / ADC, t = e % ADC;
                        Zc[c][t] = (t < hl && ci[c] >= 0) ? zv(X, s, ci[c], t0 + h + t, d) : 0.0;
                    }
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < VQ; ++q) {
                        const int e = tid + q * TPB;
                        const int r = e / 128, t = e % 128;
                        if (t >= h && t < h + hl) {
                            double a = vacc[q];
                            for (int c = 0; c < AT; ++c) a = __fma_rn(C[r][c], Zc[c][t - h], a);
                            vacc[q] = a;
                        }
                    }
                }
            }
            // gom[i][t] = C_i z_i[t] - V_i[t]
            __syncthreads();
            if (tid < AT) Cs[tid] = cs;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < VQ; ++q) {
                const int e = tid + q * TPB;
                const int r = e / 128, t = e % 128;
                const int32_t i = ri[r];
                if (i >= 0 && t < tl)
                    gom[(int64_t)i * d + t0 + t] = __fma_rn(Cs[r], zv(X, s, i, t0 + t, d), -vacc[q]);
            }
        }
        if (tid < AT && ri[tid] >= 0) {
            rowom[ri[tid]] = os;
            rowsig[ri[tid]] = ss;
        }
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

template <class T>
__global__ void k_grad_scale(const T *__restrict__ X, const double *__restrict__ s, int64_t n, int32_t d,
                             const double *__restrict__ gphi, const double *__restrict__ gom,
                             const double *__restrict__ phi2, const double *__restrict__ om2, double g,
                             double *__restrict__ dscale, double *__restrict__ dsigma, double *__restrict__ ik) {
    const double Omega = om2[0], R = phi2[0] / Omega;
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < d) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double gz = (gphi[i * d + t] - R * gom[i * d + t]) / Omega;
            acc = __fma_rn(gz, (double)X[i * d + t], acc);
        }
        dscale[t] = g * acc;
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

size_t adjoint_bytes(int64_t n, int32_t d, int32_t k) {
    Arena A;
    A.take<double>((size_t)n * d);
    A.take<double>((size_t)n * d);
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
    return A.off;
}

// Work space carved from `ws` (adjoint_bytes); outputs on the stream.
cudaError_t adjoint_launch(const void *X, int32_t dtype, int64_t n, int32_t d, const double *scale, double sigma,
                           const int32_t *parent, const int32_t *labels, int32_t k, const double *phi_par,
                           const double *omega, double grad, double *dX, double *dscale, double *dsigma, double *ik,
                           void *ws, uint32_t *status, cudaStream_t s) {
    Arena A{(char *)ws, adjoint_bytes(n, d, k) + 4096, 0, false};
    double *gphi = A.take<double>((size_t)n * d);
    double *gom = A.take<double>((size_t)n * d);
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
    const unsigned gp = (unsigned)(num_sms() * 2);
    if (dtype == ISOCLUST_F64) {
        const double *Xd = (const double *)X;
        k_phi_grad<double><<<1, TPB, 0, ISO_S(s)>>>(Xd, scale, d, parent, elist, cnt + 3, sigma, gphi, sums);
        k_omega_grad<double><<<gp, TPB, 0, ISO_S(s)>>>(Xd, scale, n, d, alist, cnt + 1, nullptr, nullptr, fa, sigma,
                                                        gom, rowom, rowsig);
        k_omega_grad<double><<<gp, TPB, 0, ISO_S(s)>>>(Xd, scale, n, d, blist, cnt + 2, alist, cnt + 1, fa, sigma,
                                                        gom, rowom, rowsig);
        k_omega_total<<<1, TPB, 0, ISO_S(s)>>>(alist, cnt + 1, rowom, rowsig, sums + 2);
        k_grad_out<double><<<grid_for(n * d), TPB, 0, ISO_S(s)>>>(Xd, scale, n, d, gphi, gom, sums, sums + 2, grad, dX);
        k_grad_scale<double><<<(unsigned)ceil_div(d, 128), 128, 0, ISO_S(s)>>>(Xd, scale, n, d, gphi, gom, sums,
                                                                               sums + 2, grad, dscale, dsigma, ik);
    } else {
        const float *Xf = (const float *)X;
        k_phi_grad<float><<<1, TPB, 0, ISO_S(s)>>>(Xf, scale, d, parent, elist, cnt + 3, sigma, gphi, sums);
        k_omega_grad<float><<<gp, TPB, 0, ISO_S(s)>>>(Xf, scale, n, d, alist, cnt + 1, nullptr, nullptr, fa, sigma,
                                                       gom, rowom, rowsig);
        k_omega_grad<float><<<gp, TPB, 0, ISO_S(s)>>>(Xf, scale, n, d, blist, cnt + 2, alist, cnt + 1, fa, sigma,
                                                       gom, rowom, rowsig);
        k_omega_total<<<1, TPB, 0, ISO_S(s)>>>(alist, cnt + 1, rowom, rowsig, sums + 2);
        k_grad_out<float><<<grid_for(n * d), TPB, 0, ISO_S(s)>>>(Xf, scale, n, d, gphi, gom, sums, sums + 2, grad, dX);
        k_grad_scale<float><<<(unsigned)ceil_div(d, 128), 128, 0, ISO_S(s)>>>(Xf, scale, n, d, gphi, gom, sums,
                                                                              sums + 2, grad, dscale, dsigma, ik);
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

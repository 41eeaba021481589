// omega_tc.cu -- the Gram tiles of eq. omega on the tensor cores, exactly.
//
// eq. omega needs every term exp(-||x_i - x_j|| / sigma) to about 1e-14
// relative, so d2 must carry about 2^-46 relative error.  With y = x - c_T
// (c_T the centroid of the point's 64-row tile T) and D = c_I - c_J,
//     d2(i, j) = |y_i|^2 + |y_j|^2 + |D|^2 - 2 <y_i, y_j> + 2 <y_i, D> - 2 <y_j, D>.
// The Gram <y_i, y_j> of a pair of tiles is the O(rows x cols x d) part; it
// runs on tcgen05 in an error-free form (the splitting idea of Ozaki, Ogita,
// Oishi and Rump): every row is scaled by a power of two to a 55-bit signed
// integer vector Y_i = y_i 2^(55 - E_i) (|y_i,t| < 2^E_i) and written as 7
// balanced base-256 digits, Y_i = sum_s a_s 2^(8 (6 - s)), |a_s| <= 129, each
// exact in BF16.  A product of two digits is an integer below 2^14.03, so a
// sum of at most 8 x 64 of them stays below 2^24 and the FP32 accumulator of
// kind::f16 holds it exactly.  The digit pairs of equal weight s + t = m
// (m = 0..7, 34 pairs) are summed in one TMEM accumulator each (8 x 64
// columns: all 512), 64 dimensions at a time; the pairs with s + t >= 8
// weigh below 2^-53 of |y_i| |y_j| and are dropped.  The epilogue folds the 8
// exact sums into a double-word FP32 value per pair,
//     G = sum_m 2^(-8m) Q_m  (in units of 2^(E_i + E_j - 14)),
// which the symmetric omega sweep (weights.cu) reads instead of forming the
// d-long double-word sums itself.
//
// Work: blocks of 128 rows (two 64-row tiles 2P, 2P+1) by 64 columns (tile
// J), the upper-triangle tile pairs the screen keeps.  Per CTA: warp 0 TMA
// producer (digit planes, 128-byte swizzle), warp 1 TMEM allocation and MMA
// issue, warps 2..9 epilogue (two per TMEM lane quadrant, 32 columns each).
// With d <= 64 the block's 7 row planes stay resident while its column
// planes stream through a 2-stage ring; wider rows stream both per 64-wide
// chunk.  Every wait is bounded; a CTA drains its copies and MMAs before it
// frees its tensor memory.
#include <cuda_bf16.h>
#include <stddef.h>

#include "common.cuh"
#include "dwmath.cuh"
#include "tcgen05.cuh"

namespace iso {
using namespace tcx;

namespace {
constexpr int OZ_S = 7;                                   // digit planes per row
constexpr int OZ_G = 8;                                   // accumulators: s + t = 0..7
constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64;
constexpr int OZ_APLANE = OZ_BM * OZ_BK * 2;              // 16 KB
constexpr int OZ_BPLANE = OZ_BN * OZ_BK * 2;              // 8 KB
constexpr int OZ_A = OZ_S * OZ_APLANE;                    // 112 KB
constexpr int OZ_B = OZ_S * OZ_BPLANE;                    // 56 KB
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr long long OZ_WAIT_CYCLES = 4000000000LL;

struct __align__(16) OzShared {
    uint64_t full[2], empty[2];
    uint64_t acc_full, acc_empty;
    uint64_t a_full, a_empty;
    uint64_t drain;
    uint32_t tmem_base;
    uint32_t pad;
};
__host__ __device__ constexpr int oz_nst(bool ares) { return ares ? 2 : 1; }
__host__ __device__ constexpr int oz_sb(bool ares) { return ares ? OZ_B : OZ_A + OZ_B; }
__host__ __device__ constexpr int oz_smem(bool ares) {
    return (ares ? OZ_A : 0) + oz_nst(ares) * oz_sb(ares) + 1024 + (int)sizeof(OzShared);
}
static_assert(oz_smem(true) <= 227 * 1024 && oz_smem(false) <= 227 * 1024, "shared memory budget");
static_assert(OZ_APLANE % 1024 == 0 && OZ_BPLANE % 1024 == 0, "planes on 1024-byte boundaries");

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// ---- digits: one warp per padded row r of the omega order (rows past n and
// dimensions past d are zero).  Also the row's y = x - c_T as a double-word,
// its exponent E and |y|^2 as a double-word.  cen_stride = 0: every row is
// centred on the same point cen[0 .. d).
// The mean of the tile centroids (the single centre of long rows).
__global__ void k_oz_centre(const float *__restrict__ cen, int64_t T64, int32_t d, float *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d) return;
    double s = 0.0;
    for (int64_t T = 0; T < T64; ++T) s += (double)cen[T * d + t];
    out[t] = (float)(s / (double)T64);
}

__global__ void __launch_bounds__(256) k_oz_digits(const float *__restrict__ X, int64_t n, int32_t d, int32_t d_pad,
                                                   int64_t n_pad, const float *__restrict__ cen, int64_t cen_stride,
                                                   __nv_bfloat16 *__restrict__ planes, float *__restrict__ yh_out,
                                                   float *__restrict__ yl_out, int32_t *__restrict__ rexp,
                                                   float2 *__restrict__ rnorm) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n_pad) return;
    const int64_t T = r / 64;
    const bool real = r < n;
    // pass 1: exponent and norm
    int emax = -1000;
    float nh = 0.f, nl = 0.f;
    for (int t = lane; t < d; t += 32) {
        float yh = 0.f, yl = 0.f;
        if (real) two_sum(X[r * d + t], -cen[T * cen_stride + t], yh, yl);
        if (yh != 0.f) emax = max(emax, ilogbf(yh) + 1);         // |yh| < 2^(ilogb + 1)
        float p, e;
        two_prod(yh, yh, p, e);
        e = __fmaf_rn(__fadd_rn(yh, yh), yl, e);
        dw_add(nh, nl, p, e);
        yh_out[r * d + t] = yh;
        yl_out[r * d + t] = yl;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        const float oh = __shfl_xor_sync(0xffffffffu, nh, o), ol = __shfl_xor_sync(0xffffffffu, nl, o);
        dw_add(nh, nl, oh, ol);
    }
    const int E = emax > -1000 ? emax : 0;
    if (lane == 0) {
        rexp[r] = E;
        rnorm[r] = make_float2(nh, nl);
    }
    // pass 2: Y = round(y 2^(55 - E)) as 7 balanced base-256 digits
    const int k = 55 - E;
    const size_t plane = (size_t)n_pad * d_pad;
    for (int t = lane; t < d_pad; t += 32) {
        long long Y = 0;
        if (real && t < d) {
            const float yh = yh_out[r * d + t], yl = yl_out[r * d + t];
            Y = __float2ll_rn(ldexpf(yh, k)) + __float2ll_rn(ldexpf(yl, k));
        }
        int a[OZ_S];
#pragma unroll
        for (int s = OZ_S - 1; s >= 1; --s) {
            a[s] = (int)((Y + 128) & 255) - 128;
            Y = (Y - a[s]) >> 8;
        }
        a[0] = (int)Y;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) planes[s * plane + (size_t)r * d_pad + t] = __float2bfloat16_rn((float)a[s]);
    }
}

__device__ __forceinline__ int64_t oz_item(int64_t I, int64_t J, int64_t T) {
    return I * T - I * (I - 1) / 2 + (J - I);          // upper-triangle item (I, J), I <= J
}

// candidate block (P, J), J in [2P, T64): bit 0 = item (2P, J) kept, bit 1 =
// item (2P + 1, J) kept (2P + 1 <= J)
__global__ void k_oz_flags(const uint8_t *__restrict__ tskip, int64_t T64, int32_t *__restrict__ flag,
                           int32_t *__restrict__ bits) {
    const int64_t P = blockIdx.y;
    const int64_t J = 2 * P + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= T64) return;
    const int64_t c = P * T64 - P * (P - 1) + (J - 2 * P);
    int b = tskip[oz_item(2 * P, J, T64)] ? 0 : 1;
    if (2 * P + 1 <= J && !tskip[oz_item(2 * P + 1, J, T64)]) b |= 2;
    flag[c] = b ? 1 : 0;
    bits[c] = b;
}

__global__ void k_oz_compact(const int32_t *__restrict__ pos, const int32_t *__restrict__ bits, int64_t T64,
                             int4 *__restrict__ blocks, int32_t *__restrict__ item_slot) {
    const int64_t P = blockIdx.y;
    const int64_t J = 2 * P + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= T64) return;
    const int64_t c = P * T64 - P * (P - 1) + (J - 2 * P);
    const int b = bits[c];
    if (!b) return;
    const int32_t q = pos[c];
    blocks[q] = make_int4((int)P, (int)J, b, 0);
    if (b & 1) item_slot[oz_item(2 * P, J, T64)] = 2 * q;
    if (b & 2) item_slot[oz_item(2 * P + 1, J, T64)] = 2 * q + 1;
}

// G = sum_m 2^(-8m) Q_m as a double-word: Q_5 + 2^-8 Q_6 + 2^-16 Q_7 in
// FP32 (its rounding, one unit of group 5, is 2^-40 of a group-0 unit, below
// 2^-52 of |y_i| |y_j| >= 2^12 group-0 units), then Horner in double-word.
__device__ __forceinline__ void oz_fold(const float (&Q)[OZ_G], float &h, float &l) {
    const float c8 = 0.00390625f;     // 2^-8
    float t = __fmaf_rn(__fmaf_rn(Q[7], c8, Q[6]), c8, Q[5]);
    h = t;
    l = 0.0f;
#pragma unroll
    for (int m = 4; m >= 0; --m) {
        h = __fmul_rn(h, c8);
        l = __fmul_rn(l, c8);
        float s, e;
        two_sum(Q[m], h, s, e);
        e = __fadd_rn(e, l);
        fast_two_sum(s, e, h, l);
    }
}

template <bool ARES>
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_gram(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t n_pad,
          int kchunks, const int4 *__restrict__ blocks, int64_t nblocks, float2 *__restrict__ gout,
          uint32_t *err, long long wait_limit) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int NST = oz_nst(ARES);
    constexpr int SB = oz_sb(ARES);
    unsigned char *areg = base;                                  // resident row planes (ARES)
    unsigned char *ring = base + (ARES ? OZ_A : 0);
    OzShared *sh = (OzShared *)(ring + NST * SB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t IDESC = tc_idesc(OZ_BN, OZ_BM);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->acc_full, 1);
        mbar_init(&sh->acc_empty, OZ_EPI_WARPS);
        mbar_init(&sh->a_full, 1);
        mbar_init(&sh->a_empty, 1);
        mbar_init(&sh->drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "n"(OZ_G * OZ_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    // a contiguous run of blocks per CTA: the list is sorted by P, so the
    // resident row planes change rarely
    const int64_t per = (nblocks + gridDim.x - 1) / gridDim.x;
    const int64_t w0 = (int64_t)blockIdx.x * per, w1 = min(nblocks, w0 + per);

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, a_phase = 0, fills = 0, a_fills = 0;
            int curP = -1;
            bool ok = true;
            for (int64_t w = w0; w < w1 && ok; ++w) {
                const int4 b = blocks[w];
                const int P = b.x, J = b.y;
                if (ARES && P != curP) {
                    if (!(ok = mbar_wait(&sh->a_empty, a_phase ^ 1u, err, wait_limit))) break;
                    mbar_expect_tx(&sh->a_full, (uint32_t)OZ_A);
                    for (int s = 0; s < OZ_S; ++s)
                        tma_load_2d(areg + s * OZ_APLANE, &mapA, 0, (int)(s * n_pad) + P * OZ_BM, &sh->a_full);
                    ++a_fills;
                    a_phase ^= 1u;
                    curP = P;
                }
                for (int kc = 0; kc < kchunks; ++kc) {
                    if (!(ok = mbar_wait(&sh->empty[stage], phase ^ 1u, err, wait_limit))) break;
                    unsigned char *st = ring + stage * SB;
                    mbar_expect_tx(&sh->full[stage], (uint32_t)SB);
                    if (!ARES)
                        for (int s = 0; s < OZ_S; ++s)
                            tma_load_2d(st + s * OZ_APLANE, &mapA, kc * OZ_BK, (int)(s * n_pad) + P * OZ_BM,
                                        &sh->full[stage]);
                    unsigned char *sbp = st + (ARES ? 0 : OZ_A);
                    for (int t = 0; t < OZ_S; ++t)
                        tma_load_2d(sbp + t * OZ_BPLANE, &mapB, kc * OZ_BK, (int)(t * n_pad) + J * OZ_BN,
                                    &sh->full[stage]);
                    ++fills;
                    if (++stage == NST) { stage = 0; phase ^= 1u; }
                }
            }
            // the copies this CTA issued land before it exits
            for (uint32_t st = 0; st < (uint32_t)NST && st < fills; ++st) {
                const uint32_t f = (fills - 1u) - ((fills - 1u - st) % (uint32_t)NST);
                mbar_drain(&sh->full[st], (f / (uint32_t)NST) & 1u, err, OZ_WAIT_CYCLES);
            }
            if (ARES && a_fills > 0) mbar_drain(&sh->a_full, (a_fills - 1u) & 1u, err, OZ_WAIT_CYCLES);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, acc_phase = 0, a_phase = 0;
            int curP = -1;
            bool ok = true;
            for (int64_t w = w0; w < w1 && ok; ++w) {
                const int P = blocks[w].x;
                if (ARES && P != curP) {
                    if (curP >= 0) mma_commit(&sh->a_empty);      // the previous row planes are free after its MMAs
                    if (!(ok = mbar_wait(&sh->a_full, a_phase, err, wait_limit))) break;
                    tc_fence_after();
                    a_phase ^= 1u;
                    curP = P;
                }
                for (int kc = 0; kc < kchunks && ok; ++kc) {
                    if (!(ok = mbar_wait(&sh->acc_empty, acc_phase ^ 1u, err, wait_limit))) break;
                    tc_fence_after();
                    if (!(ok = mbar_wait(&sh->full[stage], phase, err, wait_limit))) break;
                    tc_fence_after();
                    const uint32_t sst = smem_u32(ring + stage * SB);
                    const uint32_t sa = ARES ? smem_u32(areg) : sst;
                    const uint32_t sbp = sst + (ARES ? 0 : OZ_A);
#pragma unroll 1
                    for (int kk = 0; kk < OZ_BK / 16; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 32) >> 4;      // 16 bf16 = 32 bytes
#pragma unroll
                        for (int m = 0; m < OZ_G; ++m) {
                            const int s0 = m > OZ_S - 1 ? m - (OZ_S - 1) : 0, s1 = m < OZ_S - 1 ? m : OZ_S - 1;
#pragma unroll
                            for (int s = s0; s <= s1; ++s) {
                                const uint64_t ad = make_sw128_desc(sa + s * OZ_APLANE) + o;
                                const uint64_t bd = make_sw128_desc(sbp + (m - s) * OZ_BPLANE) + o;
                                mma_bf16(tmem + m * OZ_BN, ad, bd, IDESC, (kk > 0 || s > s0) ? 1u : 0u);
                            }
                        }
                    }
                    mma_commit(&sh->empty[stage]);
                    if (++stage == NST) { stage = 0; phase ^= 1u; }
                    mma_commit(&sh->acc_full);
                    acc_phase ^= 1u;
                }
            }
            // every MMA this thread issued completes before TMEM is freed
            mma_commit(&sh->drain);
            mbar_drain(&sh->drain, 0u, err, OZ_WAIT_CYCLES);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..9)
        const int quad = warp & 3;                      // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;               // columns half * 32 .. + 31
        const int row = quad * 32 + lane;               // row of the block = TMEM lane
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int64_t w = w0; w < w1; ++w) {
            const int4 b = blocks[w];
            const bool mine = (quad < 2) ? (b.z & 1) : (b.z & 2);      // warp-uniform
            float gh[32], gl[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) { gh[c] = 0.f; gl[c] = 0.f; }
            for (int kc = 0; kc < kchunks; ++kc) {
                if (ok) ok = mbar_wait(&sh->acc_full, acc_phase, err, wait_limit);
                ok = __all_sync(0xffffffffu, ok);
                tc_fence_after();
                if (ok && mine) {
#pragma unroll
                    for (int cg = 0; cg < 4; ++cg) {
                        uint32_t q[OZ_G][8];
#pragma unroll
                        for (int m = 0; m < OZ_G; ++m) tmem_ld8(tq + m * OZ_BN + cg * 8, q[m]);
                        tmem_ld_wait();
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            float Q[OZ_G];
#pragma unroll
                            for (int m = 0; m < OZ_G; ++m) Q[m] = __uint_as_float(q[m][c]);
                            float h, l;
                            oz_fold(Q, h, l);
                            if (kc == 0) {          // (h, l) is normalised: the same as adding it to zero
                                gh[cg * 8 + c] = h;
                                gl[cg * 8 + c] = l;
                            } else {
                                dw_add(gh[cg * 8 + c], gl[cg * 8 + c], h, l);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->acc_empty);
                acc_phase ^= 1u;
            }
            if (ok && mine) {
                float2 *dst = gout + ((size_t)w * OZ_BM + row) * OZ_BN + half * 32;
#pragma unroll
                for (int c = 0; c < 32; c += 2)
                    *reinterpret_cast<float4 *>(dst + c) = make_float4(gh[c], gl[c], gh[c + 1], gl[c + 1]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(OZ_G * OZ_BN)
                     : "memory");
    }
}
}  // namespace

// ---- host
size_t omega_gram_bytes(int64_t n, int32_t d) {
    const int64_t T64 = ceil_div(n, 64), T128 = ceil_div(n, 128);
    const int64_t n_pad = T128 * 128;
    const int64_t d_pad = ceil_div(d, OZ_BK) * OZ_BK;
    const int64_t ncand = T128 * T64;               // >= the candidate blocks
    const int64_t items = T64 * (T64 + 1) / 2;
    return (size_t)OZ_S * n_pad * d_pad * 2 + 2 * (size_t)n_pad * d * 4 + (size_t)n_pad * (4 + 8) +
           (size_t)ncand * (4 + 4 + 4 + 16) + (size_t)items * 4 + (size_t)scan_tmp_elems(ncand + 1) * 4 +
           (size_t)d * 4 + 9 * 1024;
}

cudaError_t omega_gram_launch(OmegaGram &G, const float *Xp, int64_t n, int32_t d, const float *cen,
                              const uint8_t *tskip, uint32_t *err, uint64_t wait_cycles, cudaStream_t s,
                              cudaEvent_t *kev) {
    cudaError_t e;
    const int64_t T64 = ceil_div(n, 64), T128 = ceil_div(n, 128);
    const int64_t n_pad = T128 * 128;
    const int32_t d_pad = (int32_t)(ceil_div(d, OZ_BK) * OZ_BK);
    const int64_t ncand = T128 * T64;
    const int64_t items = T64 * (T64 + 1) / 2;
    // carve the scratch
    Arena A{(char *)G.scratch, G.scratch_bytes, 0, false};
    __nv_bfloat16 *planes = A.take<__nv_bfloat16>((size_t)OZ_S * n_pad * d_pad, 1024);
    G.yh = A.take<float>((size_t)n_pad * d);
    G.yl = A.take<float>((size_t)n_pad * d);
    G.rexp = A.take<int32_t>(n_pad);
    G.rnorm = A.take<float2>(n_pad);
    int32_t *flag = A.take<int32_t>(ncand + 1);
    int32_t *pos = A.take<int32_t>(ncand + 1);
    int32_t *bits = A.take<int32_t>(ncand);
    int4 *blocks = A.take<int4>(ncand);
    G.item_slot = A.take<int32_t>(items);
    int32_t *tmp = A.take<int32_t>(scan_tmp_elems(ncand + 1));
    float *one = A.take<float>(d);
    if (A.overflow) return cudaErrorInvalidValue;

    // long rows share one centre: their tile-centred cross terms <y, c_I -
    // c_J> would cost O(d) per row and tile pair
    G.one_centre = d >= OMEGA_ONE_CENTRE_MIN_D ? 1 : 0;
    if (G.one_centre) k_oz_centre<<<(unsigned)ceil_div(d, 128), 128, 0, ISO_S(s)>>>(cen, T64, d, one);
    k_oz_digits<<<(unsigned)ceil_div(n_pad * 32, 256), 256, 0, ISO_S(s)>>>(
        Xp, n, d, d_pad, n_pad, G.one_centre ? one : cen, G.one_centre ? 0 : d, planes, G.yh, G.yl, G.rexp, G.rnorm);
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int32_t) * (ncand + 1), s))) return e;
    if ((e = cudaMemsetAsync(bits, 0, sizeof(int32_t) * ncand, s))) return e;
    if ((e = cudaMemsetAsync(G.item_slot, 0xff, sizeof(int32_t) * items, s))) return e;
    const dim3 fg((unsigned)ceil_div(T64, 256), (unsigned)T128);
    k_oz_flags<<<fg, 256, 0, ISO_S(s)>>>(tskip, T64, flag, bits);
    if ((e = exclusive_scan_i32(flag, pos, ncand + 1, tmp, s))) return e;
    k_oz_compact<<<fg, 256, 0, ISO_S(s)>>>(pos, bits, T64, blocks, G.item_slot);
    int32_t nb = 0;
    if ((e = cudaMemcpyAsync(&nb, pos + ncand, sizeof(int32_t), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    G.nblocks = nb;
    // the Gram buffer: 128 x 64 double-words per block
    const size_t gbytes = (size_t)(nb > 0 ? nb : 1) * OZ_BM * OZ_BN * sizeof(float2);
    if (!(G.gbuf = (float2 *)gram_acquire(gbytes))) return cudaErrorMemoryAllocation;
    if (nb == 0) {
        if (kev) { record_event(kev[0], s); record_event(kev[1], s); }
        return cudaGetLastError();
    }
    CUtensorMap mapA, mapB;
    if ((e = tc_map_bf16(&mapA, planes, (int64_t)OZ_S * n_pad, d_pad, OZ_BM))) return e;
    if ((e = tc_map_bf16(&mapB, planes, (int64_t)OZ_S * n_pad, d_pad, OZ_BN))) return e;
    const bool ares = d_pad == OZ_BK;
    static bool attr = false;
    if (!attr) {
        if ((e = cudaFuncSetAttribute(k_oz_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz_smem(true))))
            return e;
        if ((e = cudaFuncSetAttribute(k_oz_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz_smem(false))))
            return e;
        attr = true;
    }
    const int64_t nsm = (int64_t)num_sms();
    const unsigned grid = (unsigned)(nb < nsm ? nb : nsm);
    const long long lim = wait_cycles > 0 ? (long long)(wait_cycles < (1ull << 62) ? wait_cycles : (1ull << 62))
                                          : OZ_WAIT_CYCLES;
    if (kev) record_event(kev[0], s);
    if (ares)
        k_oz_gram<true><<<grid, OZ_THREADS, oz_smem(true), ISO_S(s)>>>(mapA, mapB, n_pad, d_pad / OZ_BK, blocks, nb,
                                                                       G.gbuf, err, lim);
    else
        k_oz_gram<false><<<grid, OZ_THREADS, oz_smem(false), ISO_S(s)>>>(mapA, mapB, n_pad, d_pad / OZ_BK, blocks, nb,
                                                                         G.gbuf, err, lim);
    if (kev) record_event(kev[1], s);
    return cudaGetLastError();
}

}  // namespace iso

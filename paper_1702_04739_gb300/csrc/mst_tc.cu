// mst_tc.cu -- Boruvka sweep on the 5th-generation tensor cores (tcgen05).
//
// Section 3.5's minimum spanning tree, one Boruvka round per launch: for
// every row i, the candidates for its nearest point of another component.
// The squared distance is taken from the Gram matrix,
//     d2(i, j) = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j>,
// whose dense <x_i, x_j> tiles are the only tensor-core work: the centred
// points are split into BF16 hi + lo parts and each 128-row tile against a
// pair of 128-column tiles is hi.hi + hi.lo + lo.hi (three kind::f16 MMAs of
// N = 256 per 16-wide K step) with FP32 accumulation in tensor memory.  Per CTA:
//   warp 0      TMA producer: 128x64 BF16 tiles (128-byte swizzle) of the
//               column blocks (and of the row block when it streams) into
//               a 2-stage ring,
//   warp 1      allocates TMEM and issues the MMAs (one elected lane),
//   warps 2..9  epilogue: tcgen05.ld of the FP32 accumulator (warp w reads
//               TMEM lane quadrant w mod 4 and one 128-column tile of the
//               pair, one row per thread), d2 = n_i + n_j - 2g, same-component
//               mask, and a running best-8 of 32-column blocks per row.
// Two TMEM accumulators (2 x 256 columns) let the MMAs of the next pair of
// column tiles run ahead of the epilogue of the current one.  Every mbarrier
// wait is bounded; on timeout the kernel raises an error flag and stops.
// The candidates are exact-keyed in FP64 by k_recheck_tc inside a rigorous
// error margin; rows whose margin is not closed by the best 8 are rescanned.
#include <cuda.h>
#include <stddef.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mst.cuh"
#include "tcgen05.cuh"

namespace iso {

using namespace tcx;

namespace {
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;      // BK bf16 = 128 bytes (one swizzle row)
constexpr int TC_NP = 2;                                  // column tiles per MMA (N = 256)
constexpr int TC_BNP = TC_NP * TC_BN;
constexpr int TC_NST = 2;                                 // ring depth
constexpr int TC_MAXST = TC_NST;                          // barrier slots for the ring
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;         // 16 KB: 128 rows x one K chunk
constexpr int TC_EPI_WARPS = 8;                           // two per TMEM lane quadrant
constexpr int TC_NACC = 2;                                // TMEM accumulators (2 x 256 columns = all 512)
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_TOPK = 8;                                // best candidate blocks kept per (list, row)
// Columns per candidate block: 64 (one set, d_pad <= 64: the epilogue is
// the sweep's limit) or 32 (independent sets or wider rows: the recheck's
// column reads are the limit).
constexpr int TC_SURV = 8;                                // FP64-keyed columns per row (more: rescan)
constexpr int TC_QD = 4;                                  // work-item queue slots (producer -> MMA, epilogue)
constexpr long long TC_WAIT_CYCLES = 4000000000LL;         // default bound of one wait (about 2 s)

// Column metadata first: the epilogue reads it with 16-byte vector loads.
struct __align__(16) TcShared {
    float cnorm[TC_NACC][TC_BNP];
    int32_t ccomp[TC_NACC][TC_BNP];
    uint64_t full[TC_MAXST], empty[TC_MAXST];
    uint64_t acc_full[TC_NACC], acc_empty[TC_NACC];
    uint64_t a_full, a_empty;
    uint64_t drain;                                       // completion of the issued MMAs at exit
    uint64_t stall;                                       // test hook: a barrier nothing arrives at
    uint64_t q_full[TC_QD], q_empty[TC_QD];               // work-item queue
    int32_t q_item[TC_QD];
    uint32_t tmem_base;
    uint32_t pad;
};
static_assert(offsetof(TcShared, cnorm) % 16 == 0, "cnorm must be 16-byte aligned");
static_assert(offsetof(TcShared, ccomp) % 16 == 0, "ccomp must be 16-byte aligned");
static_assert(offsetof(TcShared, full) % 8 == 0, "mbarriers must be 8-byte aligned");
// AK = K chunks of a resident row block (0: A and B stream together).  A
// ring stage holds one K chunk of a pair of column tiles, hi and lo (B hi
// 256 rows, B lo 256 rows), preceded by the row tile's chunk (A hi, A lo)
// when A streams.
static_assert(TC_BNP % 16 == 0 && TC_BNP <= 256, "N of one MMA");
__host__ __device__ constexpr int tc_areg_bytes(int AK) { return AK * 2 * TC_TILE_BYTES; }
__host__ __device__ constexpr int tc_sb(int AK) { return (AK > 0 ? 2 * TC_NP : 2 + 2 * TC_NP) * TC_TILE_BYTES; }
__host__ __device__ constexpr int tc_smem(int AK) {
    return tc_areg_bytes(AK) + TC_NST * tc_sb(AK) + 1024 + (int)sizeof(TcShared);
}
static_assert(tc_sb(0) % 1024 == 0 && tc_sb(1) % 1024 == 0, "TcShared follows 1024-aligned tiles");
static_assert(tc_smem(0) <= 227 * 1024 && tc_smem(1) <= 227 * 1024 && tc_smem(2) <= 227 * 1024,
              "shared memory budget");


// The bound of every wait in the sweep: the caller's spin limit (SM cycles),
// or the default.
static long long tc_wait_limit(const TcScratch &T) {
    return T.wait_cycles > 0 ? (long long)(T.wait_cycles < (1ull << 62) ? T.wait_cycles : (1ull << 62))
                             : TC_WAIT_CYCLES;
}

// m = min(m, v) unless the column's component is the row's (a predicated
// min: compare + min per element)
__device__ __forceinline__ void min_foreign(float &m, float v, int32_t ccol, int32_t crow) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ne.s32 p, %1, %2;\n\t"
        "@p min.f32 %0, %0, %3;\n\t}"
        : "+f"(m)
        : "r"(ccol), "r"(crow), "f"(v));
}

__device__ __forceinline__ void top_insert(float (&v)[TC_TOPK], int32_t (&j)[TC_TOPK], float x, int32_t c) {
    v[TC_TOPK - 1] = x;
    j[TC_TOPK - 1] = c;
#pragma unroll
    for (int q = TC_TOPK - 1; q > 0; --q) {
        if (v[q] < v[q - 1]) {
            float tv = v[q]; v[q] = v[q - 1]; v[q - 1] = tv;
            int32_t tj = j[q]; j[q] = j[q - 1]; j[q - 1] = tj;
        }
    }
}

__device__ __forceinline__ bool mst_active(const int32_t *counters) {
    const volatile int32_t *c = counters;
    return c[MC_NCOMP] > c[MC_TARGET];
}

// ARES: the row block's A tiles (hi, lo, every K chunk) stay resident in
// shared memory for a whole work item and only the column blocks stream
// through the ring (used when d_pad <= 128); otherwise A and B chunks
// stream together.
// SCREEN: the same Gram tiles decide, for omega, which pairs of 64-row tiles
// hold a pair (i, j) within the cutoff: d2 <= max(A_i, A_j) with A the
// squared cutoff distance of each row (rowA; -inf at padding) tested
// against the rigorous lower bound of d2; need[I64 * T64 + J64] = 1.
struct ScreenArgs {
    const float *rowA;
    uint8_t *need;
    int64_t T64;
};

template <int AK, bool SCREEN, int CW>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_sweep_tc(const __grid_constant__ CUtensorMap tmh, const __grid_constant__ CUtensorMap tml,
           const float *__restrict__ rnorm, const float *__restrict__ cnorm, const float *__restrict__ rsq,
           const float *__restrict__ tmax, const float *__restrict__ tsq, float acoef, float bcoef,
           const int32_t *__restrict__ comp, int64_t nrows, int ntiles, int kchunks, int splits,
           const int4 *__restrict__ witems, int64_t nwitems, const int32_t *__restrict__ setcnt,
           const int32_t *counters, float *__restrict__ out_v, int32_t *__restrict__ out_j, float *__restrict__ out_u,
           uint32_t *err, ScreenArgs scr, long long wait_limit, int stall_test, int rt_stride, int rt_off,
           uint32_t *__restrict__ qctr) {
    if (!SCREEN && !mst_active(counters)) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr bool ARES = AK > 0;
    constexpr int NST = TC_NST;                                         // ring depth
    constexpr int SB = tc_sb(AK);                                       // bytes per ring stage
    unsigned char *areg = base;                                         // resident A (ARES)
    unsigned char *ring = base + tc_areg_bytes(AK);
    TcShared *sh = (TcShared *)(ring + NST * SB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int a = 0; a < TC_NACC; ++a) {
            mbar_init(&sh->acc_full[a], 1);
            mbar_init(&sh->acc_empty[a], TC_EPI_WARPS);
        }
        mbar_init(&sh->a_full, 1);
        mbar_init(&sh->a_empty, 1);
        mbar_init(&sh->drain, 1);
        mbar_init(&sh->stall, 1);
        for (int q = 0; q < TC_QD; ++q) {
            mbar_init(&sh->q_full[q], 1);
            mbar_init(&sh->q_empty[q], 1 + TC_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "n"(TC_NACC * TC_BNP)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    // work item w: row tile rt against column tiles [c0, c1), candidate list
    // pair sp; either from the item list (sp in the low 4 bits, the set
    // above: items of a set whose forest is complete are skipped) or row tile
    // x column split.  Items are handed out in order by the launch's counter
    // (qctr, zero at launch): the producer takes the next one when it is
    // ready for it and publishes it to the MMA issuer and the epilogue warps
    // through a TC_QD-slot queue (-1: none left), so a CTA with long items
    // takes fewer of them.
    // (a sharded call: only the row tiles rt_off, rt_off + rt_stride, ... of this rank)
    const int64_t own_tiles = rt_off < ntiles ? ((int64_t)ntiles - rt_off + rt_stride - 1) / rt_stride : 0;
    const int64_t items = witems ? nwitems : own_tiles * splits;
    const int tiles_per_split = (ntiles + splits - 1) / splits;
    auto item = [&](int64_t w, int &rt, int &c0, int &c1, int &sp) {
        if (witems) {
            const int4 it = witems[w];
            rt = it.x; c0 = it.y; c1 = it.z; sp = it.w & 15;
            if (setcnt && setcnt[it.w >> 4] <= 1) c1 = c0;      // nothing left to join in this set
        } else {
            rt = (int)(w / splits) * rt_stride + rt_off;      // row tiles of this rank (sharded calls)
            sp = (int)(w % splits);
            c0 = sp * tiles_per_split;
            c1 = min(ntiles, c0 + tiles_per_split);
        }
    };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, a_phase = 0;
            uint32_t fills = 0, a_fills = 0;         // ring stages / A blocks whose copies were issued
            uint32_t qs = 0, qph = 0;
            bool ok = true;
            while (ok) {
                if (!(ok = mbar_wait(&sh->q_empty[qs], qph ^ 1u, err, wait_limit))) break;
                const uint32_t wq = atomicAdd(qctr, 1u);
                const int64_t w = (int64_t)wq < items ? (int64_t)wq : -1;
                sh->q_item[qs] = (int32_t)w;
                mbar_arrive(&sh->q_full[qs]);
                if (++qs == TC_QD) { qs = 0; qph ^= 1u; }
                if (w < 0) break;
                int rt, c0, c1, sp;
                item(w, rt, c0, c1, sp);
                if (ARES && c0 < c1) {          // (an empty item only writes its rows' empty lists)
                    if (!(ok = mbar_wait(&sh->a_empty, a_phase ^ 1u, err, wait_limit))) break;
                    mbar_expect_tx(&sh->a_full, (uint32_t)(kchunks * 2 * TC_TILE_BYTES));
                    for (int kc = 0; kc < kchunks; ++kc) {
                        tma_load_2d(areg + (2 * kc) * TC_TILE_BYTES, &tmh, kc * TC_BK, rt * TC_BM, &sh->a_full);
                        tma_load_2d(areg + (2 * kc + 1) * TC_TILE_BYTES, &tml, kc * TC_BK, rt * TC_BM, &sh->a_full);
                    }
                    ++a_fills;
                    a_phase ^= 1u;
                }
                for (int ct = c0; ct < c1 && ok; ct += TC_NP) {
                    const int nct = min(TC_NP, c1 - ct);
                    for (int kc = 0; kc < kchunks; ++kc) {
                        if (!(ok = mbar_wait(&sh->empty[stage], phase ^ 1u, err, wait_limit))) break;
                        unsigned char *st = ring + stage * SB;
                        // stage: [A hi][A lo] (streaming A) then [B hi: NP tiles][B lo: NP tiles]
                        unsigned char *sbh = st + (ARES ? 0 : 2 * TC_TILE_BYTES);
                        unsigned char *sbl = sbh + TC_NP * TC_TILE_BYTES;
                        mbar_expect_tx(&sh->full[stage], (uint32_t)((ARES ? 0 : 2) + 2 * nct) * TC_TILE_BYTES);
                        if (!ARES) {
                            tma_load_2d(st, &tmh, kc * TC_BK, rt * TC_BM, &sh->full[stage]);
                            tma_load_2d(st + TC_TILE_BYTES, &tml, kc * TC_BK, rt * TC_BM, &sh->full[stage]);
                        }
                        for (int q = 0; q < nct; ++q) {
                            tma_load_2d(sbh + q * TC_TILE_BYTES, &tmh, kc * TC_BK, (ct + q) * TC_BN, &sh->full[stage]);
                            tma_load_2d(sbl + q * TC_TILE_BYTES, &tml, kc * TC_BK, (ct + q) * TC_BN, &sh->full[stage]);
                        }
                        ++fills;
                        if (++stage == NST) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            // before the CTA exits (also after a timeout), the copies it
            // issued land: the last fill of each ring stage and of the A block
            for (uint32_t st = 0; st < (uint32_t)NST && st < fills; ++st) {
                const uint32_t f = (fills - 1u) - ((fills - 1u - st) % (uint32_t)NST);   // last fill of stage st
                mbar_drain(&sh->full[st], (f / (uint32_t)NST) & 1u, err);
            }
            if (ARES && a_fills > 0) mbar_drain(&sh->a_full, (a_fills - 1u) & 1u, err);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0, a_phase = 0;
            uint32_t qs = 0, qph = 0;
            bool ok = true;
            while (ok) {
                if (!(ok = mbar_wait(&sh->q_full[qs], qph, err, wait_limit))) break;
                const int64_t w = *(volatile int32_t *)&sh->q_item[qs];
                mbar_arrive(&sh->q_empty[qs]);
                if (++qs == TC_QD) { qs = 0; qph ^= 1u; }
                if (w < 0) break;
                int rt, c0, c1, sp;
                item(w, rt, c0, c1, sp);
                (void)rt;
                if (ARES && c0 < c1) {
                    if (!(ok = mbar_wait(&sh->a_full, a_phase, err, wait_limit))) break;
                    tc_fence_after();
                }
                for (int ct = c0; ct < c1 && ok; ct += TC_NP) {
                    const uint32_t idesc = tc_idesc(min(TC_NP, c1 - ct) * TC_BN);
                    if (!(ok = mbar_wait(&sh->acc_empty[acc], acc_phase ^ 1u, err, wait_limit))) break;
                    tc_fence_after();
                    const uint32_t dt = tmem + acc * TC_BNP;
                    for (int kc = 0; kc < kchunks; ++kc) {
                        if (!(ok = mbar_wait(&sh->full[stage], phase, err, wait_limit))) break;
                        tc_fence_after();
                        const uint32_t sb = smem_u32(ring + stage * SB);
                        const uint32_t sbh = sb + (ARES ? 0 : 2 * TC_TILE_BYTES), sbl = sbh + TC_NP * TC_TILE_BYTES;
                        const uint32_t sa = ARES ? smem_u32(areg + (2 * kc) * TC_TILE_BYTES) : sb;
                        const uint64_t ah = make_sw128_desc(sa), al = make_sw128_desc(sa + TC_TILE_BYTES);
                        const uint64_t bh = make_sw128_desc(sbh), bl = make_sw128_desc(sbl);
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk) {
                            const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 bf16 = 32 bytes
                            mma_bf16(dt, ah + o, bh + o, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16(dt, ah + o, bl + o, idesc, 1u);
                            mma_bf16(dt, al + o, bh + o, idesc, 1u);
                        }
                        mma_commit(&sh->empty[stage]);
                        if (++stage == NST) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    mma_commit(&sh->acc_full[acc]);
                    if (++acc == TC_NACC) { acc = 0; acc_phase ^= 1u; }
                }
                if (ARES && ok && c0 < c1) {
                    mma_commit(&sh->a_empty);     // A region free once this item's MMAs are done
                    a_phase ^= 1u;
                }
            }
            // every MMA this thread issued completes before TMEM is freed
            // (also after a timeout): one more commit, and its arrival
            mma_commit(&sh->drain);
            mbar_drain(&sh->drain, 0u, err);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..9)
        // warps 2..5 take the first column tile of a pair, 6..9 the second;
        // each warp covers its tile's 128 columns as two 64-column candidate
        // blocks, for the 32 rows of its TMEM lane quadrant
        const int et = threadIdx.x - 64;               // 0..255
        const int h = et >> 7;                         // column tile of the pair
        const int quad = warp & 3;                     // TMEM lane quadrant of this warp
        const int trow = quad * 32 + lane;             // row within the tile = TMEM lane
        const int cm = et;                             // column of the pair whose metadata this thread stages
        uint32_t acc = 0, acc_phase = 0;
        uint32_t qs = 0, qph = 0;
        bool ok = true;
        for (;;) {
            if (ok) ok = mbar_wait(&sh->q_full[qs], qph, err, wait_limit);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;                            // (a wait ran out: the call reports it)
            const int64_t w = *(volatile int32_t *)&sh->q_item[qs];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->q_empty[qs]);
            if (++qs == TC_QD) { qs = 0; qph ^= 1u; }
            if (w < 0) break;
            int rt, c0, c1, sp;
            item(w, rt, c0, c1, sp);
            const int64_t row = (int64_t)rt * TC_BM + trow;      // < nrows: whole tiles
            const float nrow = rnorm[row];
            const float srow = rsq[row];
            const int32_t crow = SCREEN ? 0 : comp[row];
            const float arow = SCREEN ? scr.rowA[row] : 0.0f;
            float ubest = INFINITY;        // smallest upper bound of a candidate's d2
            float bv[TC_TOPK];
            int32_t bj[TC_TOPK];
#pragma unroll
            for (int q = 0; q < TC_TOPK; ++q) { bv[q] = INFINITY; bj[q] = -1; }
            // column metadata, prefetched one pair of tiles ahead (columns of
            // a missing second tile: +inf norm, no component)
            float pn = INFINITY;
            int32_t pc = -2;
            if (c0 < c1 && cm < min(TC_NP, c1 - c0) * TC_BN) {
                const int64_t pcol = (int64_t)c0 * TC_BN + cm;
                pn = cnorm[pcol];
                pc = SCREEN ? __float_as_int(scr.rowA[pcol]) : comp[pcol];
            }
            float ptsq = 0.f, ptmax = 0.f;
            if (c0 + h < c1) { ptsq = __ldg(tsq + c0 + h); ptmax = __ldg(tmax + c0 + h); }
            for (int ct = c0; ct < c1; ct += TC_NP) {
                sh->cnorm[acc][cm] = pn;
                sh->ccomp[acc][cm] = pc;
                const float ctsq = ptsq, ctmax = ptmax;
                const bool mine = ct + h < c1;          // this warp's column tile exists (warp-uniform)
                const int cn2 = ct + TC_NP;
                if (cn2 < c1) {
                    pn = INFINITY;
                    pc = -2;
                    if (cm < min(TC_NP, c1 - cn2) * TC_BN) {
                        const int64_t pcol = (int64_t)cn2 * TC_BN + cm;
                        pn = cnorm[pcol];
                        pc = SCREEN ? __float_as_int(scr.rowA[pcol]) : comp[pcol];
                    }
                    if (cn2 + h < c1) { ptsq = __ldg(tsq + cn2 + h); ptmax = __ldg(tmax + cn2 + h); }
                }
                asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_EPI_WARPS) : "memory");
                // test hook: the epilogue first waits for a barrier that no
                // role arrives at, so the bounded wait runs out (timeout path)
                if (stall_test && ok) ok = mbar_wait(&sh->stall, 0u, err, wait_limit);
                if (ok) ok = mbar_wait(&sh->acc_full[acc], acc_phase, err, wait_limit);
                // lanes may part on a wait that runs out; the warp-collective
                // TMEM loads below need one answer for the whole warp
                ok = __all_sync(0xffffffffu, ok);
                tc_fence_after();
                // SCREEN: d2 >= v + n_i - dlt with v = n_j - 2g; near if that
                // bound <= max(A_i, A_j), i.e. v <= max(A_i, A_j) + (dlt - n_i)
                const float dlt = acoef * srow * ctsq + bcoef * (nrow + ctmax);
                // (padding rows: arow = -inf makes both thresholds -inf; the
                // warp-collective TMEM loads stay unconditional within a warp)
                const bool rvalid = arow > -INFINITY;
                const float Ci = SCREEN ? (rvalid ? __fadd_ru(__fadd_ru(dlt, 1e-5f * (nrow + ctmax)), -nrow) : -INFINITY)
                                        : 0.0f;
                const float Bi = SCREEN ? (rvalid ? __fadd_ru(arow, Ci) : -INFINITY) : 0.0f;
                // two 64-column halves of the warp's tile; each half is one
                // TMEM load pair and 64 / CW candidate blocks
                static_assert(CW == 32 || CW == 64, "candidate block width");
                constexpr int NB = 64 / CW;
#pragma unroll 1
                for (int hf = 0; hf < 2; ++hf) {
                    float m0 = INFINITY, m1 = INFINITY;   // min over each block of n_j - 2 g (foreign columns)
                    // (four independent chains per 32 columns, folded after: min is exact)
                    float ma[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
                    float mb[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
                    bool near = false;                   // SCREEN: a pair of this half within the cutoff
                    if (ok && mine) {
                        const int cofs = h * TC_BN + hf * 64;
                        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + acc * TC_BNP + cofs;
                        uint32_t g0[32], g1[32];
                        tmem_ld32(tbase, g0);
                        tmem_ld32(tbase + 32, g1);
                        tmem_ld_wait();
                        const float *cn = &sh->cnorm[acc][cofs];
                        const int32_t *cc = &sh->ccomp[acc][cofs];
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            const float4 nc = *reinterpret_cast<const float4 *>(cn + q);
                            const int4 cmv4 = *reinterpret_cast<const int4 *>(cc + q);
                            const float ncv[4] = {nc.x, nc.y, nc.z, nc.w};
                            const int32_t cmv[4] = {cmv4.x, cmv4.y, cmv4.z, cmv4.w};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float v = __fmaf_rn(-2.0f, __uint_as_float(g0[q + u]), ncv[u]);
                                if constexpr (SCREEN)
                                    near |= v <= fmaxf(Bi, __fadd_ru(__int_as_float(cmv[u]), Ci));
                                else
                                    min_foreign(ma[u], v, cmv[u], crow);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            const float4 nc = *reinterpret_cast<const float4 *>(cn + 32 + q);
                            const int4 cmv4 = *reinterpret_cast<const int4 *>(cc + 32 + q);
                            const float ncv[4] = {nc.x, nc.y, nc.z, nc.w};
                            const int32_t cmv[4] = {cmv4.x, cmv4.y, cmv4.z, cmv4.w};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float v = __fmaf_rn(-2.0f, __uint_as_float(g1[q + u]), ncv[u]);
                                if constexpr (SCREEN)
                                    near |= v <= fmaxf(Bi, __fadd_ru(__int_as_float(cmv[u]), Ci));
                                else
                                    min_foreign(NB == 2 ? mb[u] : ma[u], v, cmv[u], crow);
                            }
                        }
                        if constexpr (!SCREEN) {
                            m0 = fminf(fminf(ma[0], ma[1]), fminf(ma[2], ma[3]));
                            m1 = fminf(fminf(mb[0], mb[1]), fminf(mb[2], mb[3]));
                        }
                    }
                    if constexpr (SCREEN) {
                        // rows of this warp are one 64-row half of the row tile
                        if (__ballot_sync(0xffffffffu, near) && lane == 0) {
                            const int64_t I64 = 2 * (int64_t)rt + (quad >> 1), J64 = 2 * (int64_t)(ct + h) + hf;
                            if (I64 < scr.T64 && J64 < scr.T64) scr.need[I64 * scr.T64 + J64] = 1;
                        }
                    } else if (mine) {
                        // rigorous bounds of each block's smallest d2 of the
                        // represented points: accumulation + dropped lo.lo
                        // (A s_i s_j) and FP32 norm/epilogue rounding
                        const int blk = (TC_BN / CW) * (ct + h) + NB * hf;
                        m0 = __fadd_rn(m0, nrow);
                        if constexpr (NB == 2) {
                            m1 = __fadd_rn(m1, nrow);
                            ubest = fminf(ubest, fminf(m0, m1) + dlt);
#pragma unroll 1
                            for (int e = 0; e < NB; ++e) {
                                const float lb = (e ? m1 : m0) - dlt;
                                if (lb < bv[TC_TOPK - 1]) top_insert(bv, bj, lb, blk + e);
                            }
                        } else {
                            ubest = fminf(ubest, m0 + dlt);
                            const float lb = m0 - dlt;
                            if (lb < bv[TC_TOPK - 1]) top_insert(bv, bj, lb, blk);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->acc_empty[acc]);
                if (++acc == TC_NACC) { acc = 0; acc_phase ^= 1u; }
            }
            if (!SCREEN) {
                const size_t o = ((size_t)(2 * sp + h) * nrows + row) * TC_TOPK;   // (32-byte aligned)
                static_assert(TC_TOPK == 8, "two 16-byte stores per list");
                float4 *ov = reinterpret_cast<float4 *>(out_v + o);
                int4 *oj = reinterpret_cast<int4 *>(out_j + o);
                ov[0] = make_float4(bv[0], bv[1], bv[2], bv[3]);
                ov[1] = make_float4(bv[4], bv[5], bv[6], bv[7]);
                oj[0] = make_int4(bj[0], bj[1], bj[2], bj[3]);
                oj[1] = make_int4(bj[4], bj[5], bj[6], bj[7]);
                out_u[(size_t)(2 * sp + h) * nrows + row] = ubest;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_NACC * TC_BNP)
                     : "memory");
    }
}

// Centre, split into BF16 hi + lo (zero rows at padding) and the squared
// norms of the represented points.
// Partial column sums of rows [r0, r1): warp w sums every 8th row from
// r0 + w in FP32 (four chains, 32 columns per warp), the block's warps are
// added in FP64.  Any centre serves (it only shrinks the represented
// magnitudes); this one is deterministic.
__global__ void __launch_bounds__(256) k_tc_mean_partial(const float *__restrict__ X, int64_t n, int32_t d,
                                                         int64_t rows_per, double *__restrict__ part) {
    __shared__ float acc[8][33];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int t = blockIdx.y * 32 + lane;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    if (t < d) {
        int64_t r = r0 + wp;
#pragma unroll 2
        for (; r + 24 < r1; r += 32) {
            s0 += X[r * d + t];
            s1 += X[(r + 8) * d + t];
            s2 += X[(r + 16) * d + t];
            s3 += X[(r + 24) * d + t];
        }
        for (; r < r1; r += 8) s0 += X[r * d + t];
    }
    acc[wp][lane] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (wp == 0 && t < d) {
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += (double)acc[w][lane];
        part[(int64_t)blockIdx.x * d + t] = sum;
    }
}

__global__ void k_tc_mean_final(const double *__restrict__ part, int nparts, int64_t n, int32_t d,
                                float *__restrict__ mean) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d) return;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * d + t];
    mean[t] = (float)(s / (double)n);
}

// One block per set: the set's mean (any centre serves; it only shrinks the
// represented magnitudes).  8 warps x 32 dimensions per pass.
__global__ void __launch_bounds__(256) k_tc_set_mean(const float *__restrict__ X, const int64_t *__restrict__ offs,
                                                     int32_t d, float *__restrict__ mean) {
    __shared__ double acc[8][33];
    const int b = blockIdx.x, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t r0 = offs[b], r1 = offs[b + 1];
    for (int t0 = 0; t0 < d; t0 += 32) {
        const int t = t0 + lane;
        float s0 = 0.0f, s1 = 0.0f;                         // FP32 chains; the warps add in FP64
        if (t < d) {
            int64_t r = r0 + wp;
            for (; r + 8 < r1; r += 16) {
                s0 += X[r * d + t];
                s1 += X[(r + 8) * d + t];
            }
            if (r < r1) s0 += X[r * d + t];
        }
        acc[wp][lane] = (double)(s0 + s1);
        __syncthreads();
        if (wp == 0 && t < d) {
            double tot = 0.0;
            for (int q = 0; q < 8; ++q) tot += acc[q][lane];
            mean[(int64_t)b * d + t] = r1 > r0 ? (float)(tot / (double)(r1 - r0)) : 0.0f;
        }
        __syncthreads();
    }
}

// Sort keys: norm order (one set), or (set, norm) for independent sets.
__global__ void k_tc_prenorm_keys(const float *__restrict__ X, const float *__restrict__ mean,
                                  const int32_t *__restrict__ set_of, int64_t n, int32_t d,
                                  uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = set_of ? set_of[i] : 0;
    const float *mu = mean + (int64_t)b * d;
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        const double y = (double)__fsub_rn(X[i * d + t], mu[t]);
        s += y * y;
    }
    const uint64_t nb = (uint64_t)__float_as_uint((float)s);     // non-negative: bits are monotone
    keys[i] = set_of ? (((uint64_t)(uint32_t)b << 32) | nb) : ((nb << 32) | (uint64_t)i);
    vals[i] = (int32_t)i;
}

// Padded row of sorted position q: q itself (one set), or the set's first
// padded row plus the rank inside the set.
__global__ void k_tc_place(const int32_t *__restrict__ perm, int64_t n, const int32_t *__restrict__ set_of,
                           const int64_t *__restrict__ offs, const int64_t *__restrict__ rowbase,
                           int32_t *__restrict__ permp) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t i = perm[q];
    int64_t r = q;
    if (set_of) {
        const int32_t b = set_of[i];
        r = rowbase[b] + (q - offs[b]);
    }
    permp[r] = i;
}

// Also writes xs, the points themselves in the same row order (zero rows at
// padding): the recheck reads candidate columns as contiguous blocks.
__global__ void k_tc_split(const float *__restrict__ X, const float *__restrict__ mean,
                           const int32_t *__restrict__ set_of, const int32_t *__restrict__ permp, int32_t d,
                           int64_t n_pad, int32_t d_pad, __nv_bfloat16 *__restrict__ xh,
                           __nv_bfloat16 *__restrict__ xl, float *__restrict__ xs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_pad * d_pad) return;
    const int64_t r = idx / d_pad, t = idx - r * d_pad;
    const int32_t i = permp[r];
    float y = 0.0f;
    if (t < d) {
        const float x = i >= 0 ? X[(int64_t)i * d + t] : 0.0f;
        xs[r * d + t] = x;
        if (i >= 0) {
            const int64_t b = set_of ? set_of[i] : 0;
            y = __fsub_rn(x, mean[b * d + t]);
        }
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(y);
    const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(y, __bfloat162float(h)));
    xh[idx] = h;
    xl[idx] = l;
}

__global__ void k_tc_norms(const __nv_bfloat16 *__restrict__ xh, const __nv_bfloat16 *__restrict__ xl,
                           const int32_t *__restrict__ permp, int64_t n_pad, int32_t d_pad,
                           float *__restrict__ nrm, float *__restrict__ cnrm, float *__restrict__ sq,
                           unsigned int *__restrict__ nmax_bits) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    double s = 0.0;
    for (int t = 0; t < d_pad; ++t) {
        const double v = (double)__bfloat162float(xh[r * d_pad + t]) + (double)__bfloat162float(xl[r * d_pad + t]);
        s += v * v;
    }
    const float f = (float)s;
    nrm[r] = f;
    cnrm[r] = permp[r] >= 0 ? f : INFINITY;
    sq[r] = (float)sqrt(s);
    atomicMax(nmax_bits, __float_as_uint(f));
}

// per 128-row tile: the largest squared norm and its square root
__global__ void k_tc_tile_max(const float *__restrict__ nrm, int64_t n_pad, float *__restrict__ tmax,
                              float *__restrict__ tsq) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t * TC_BM >= n_pad) return;
    float m = 0.0f;
    for (int r = 0; r < TC_BM; ++r) m = fmaxf(m, nrm[t * TC_BM + r]);
    tmax[t] = m;
    tsq[t] = sqrtf(m) * 1.0000002f;       // rounded up
}

__global__ void k_tc_gather_comp(const int32_t *__restrict__ comp, const int32_t *__restrict__ permp,
                                 int64_t n_pad, int32_t *__restrict__ compp, const int32_t *counters) {
    if (!mst_active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_pad; r += gs) {
        const int32_t i = permp[r];
        compp[r] = i >= 0 ? comp[i] : -2;
    }
}

// components of each set: the roots of comp counted per set
__global__ void k_tc_set_roots(const int32_t *__restrict__ comp, const int32_t *__restrict__ set_of, int64_t n,
                               int32_t *__restrict__ setcnt, const int32_t *counters) {
    if (!mst_active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gs)
        if (comp[v] == v) atomicAdd(setcnt + set_of[v], 1);
}

__global__ void k_tc_identity(int32_t *__restrict__ permp, int64_t n, int64_t n_pad) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_pad) permp[r] = r < n ? (int32_t)r : -1;
}

// omega screen: squared cutoff distance of row r, (sigma (zskip + y_r) + w_r)^2
// with y_r = d_nn(r) / sigma and w_r the representation error bound of the
// BF16 split, computed in FP64 and rounded up; -inf at padding
__global__ void k_screen_rows(const unsigned long long *__restrict__ nnbits, const float *__restrict__ rsq,
                              const unsigned int *__restrict__ nmax_bits, int64_t n, int64_t n_pad, double sigma,
                              double zskip, double eps_rep, float *__restrict__ rowA) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    if (r >= n) {
        rowA[r] = -INFINITY;
        return;
    }
    const double nd2 = __longlong_as_double((long long)nnbits[r]);
    const double y = isfinite(nd2) ? sqrt(nd2) / sigma : 0.0;
    const double smax = sqrt((double)__uint_as_float(*nmax_bits));
    const double a = sigma * (zskip + y) * (1.0 + 1e-9) + eps_rep * ((double)rsq[r] + smax);
    rowA[r] = __double2float_ru(a * a * (1.0 + 1e-6));
}

__global__ void k_tc_fill_lists(float *__restrict__ tv, int32_t *__restrict__ tj, float *__restrict__ tu,
                                int64_t nv, int64_t nu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) {
        tv[i] = INFINITY;
        tj[i] = -1;
    }
    if (i < nu) tu[i] = INFINITY;
}

// One warp per padded row r, the point i = permp[r] (none at padding).
// Candidate columns are read from xs (rows in the sweep's order) with their
// components from compp, so a candidate block is 32 contiguous rows of xs;
// only the survivors of the FP32 filter are mapped back to point indices.
// The lists (column split x tile of the pair) hold each split's best-8
// block lower bounds and their best upper bound U.
// The epilogue's bounds hold for the BF16-represented points; the exact
// points differ by the representation error rep, so a block can hold the
// nearest foreign point only if its lower bound is <= U + 2 rep.  Those
// blocks' columns are filtered with FP32 direct differences and the
// survivors keyed in FP64.  If 8 or more blocks qualify (a list may have
// dropped more), the row is queued for a rescan.
__device__ __forceinline__ float approx_d2_f32(const float *__restrict__ a, const float *__restrict__ b, int d) {
    float acc = 0.0f;
    for (int t = 0; t < d; ++t) {
        const float df = __fsub_rn(a[t], b[t]);
        acc = __fmaf_rn(df, df, acc);
    }
    return acc;
}

// FP32 squared differences of row r against the columns of the NU first
// slots (dimension order, one FMA chain per column; a dead slot reads the
// row itself and is ignored), unrolled so that fewer columns keep more loads
// in flight.
template <int NU>
__device__ __forceinline__ void rc_dist(const float *__restrict__ xs, int64_t r, int32_t d, bool vec,
                                        const int32_t (&jp)[4], const bool (&live)[4], float (&acc)[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = 0.0f;
    const float *xi = xs + r * d;
    if (vec) {
        constexpr int UNR = NU == 1 ? 4 : (NU == 2 ? 2 : 1);
        const float4 *xi4 = reinterpret_cast<const float4 *>(xi);
        const float4 *b4[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) b4[u] = reinterpret_cast<const float4 *>(xs + (live[u] ? (int64_t)jp[u] : r) * d);
        const int d4 = d / 4;
        int t = 0;
#pragma unroll 1
        for (; t + UNR <= d4; t += UNR) {
            float4 a[UNR], b[UNR][NU];
#pragma unroll
            for (int v = 0; v < UNR; ++v) {
                a[v] = xi4[t + v];
#pragma unroll
                for (int u = 0; u < NU; ++u) b[v][u] = b4[u][t + v];
            }
#pragma unroll
            for (int v = 0; v < UNR; ++v) {
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    float df = __fsub_rn(a[v].x, b[v][u].x); acc[u] = __fmaf_rn(df, df, acc[u]);
                    df = __fsub_rn(a[v].y, b[v][u].y); acc[u] = __fmaf_rn(df, df, acc[u]);
                    df = __fsub_rn(a[v].z, b[v][u].z); acc[u] = __fmaf_rn(df, df, acc[u]);
                    df = __fsub_rn(a[v].w, b[v][u].w); acc[u] = __fmaf_rn(df, df, acc[u]);
                }
            }
        }
#pragma unroll 1
        for (; t < d4; ++t) {
            const float4 a = xi4[t];
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const float4 b = b4[u][t];
                float df = __fsub_rn(a.x, b.x); acc[u] = __fmaf_rn(df, df, acc[u]);
                df = __fsub_rn(a.y, b.y); acc[u] = __fmaf_rn(df, df, acc[u]);
                df = __fsub_rn(a.z, b.z); acc[u] = __fmaf_rn(df, df, acc[u]);
                df = __fsub_rn(a.w, b.w); acc[u] = __fmaf_rn(df, df, acc[u]);
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < NU; ++u)
            if (live[u]) acc[u] = approx_d2_f32(xi, xs + (int64_t)jp[u] * d, d);
    }
}

template <int EPL, int CW>
__device__ __forceinline__ void recheck_row(int64_t r, int lane, const float *__restrict__ xs, int64_t n, int32_t d,
                                            int lists, const float *__restrict__ tv, const int32_t *__restrict__ tj,
                                            const float *__restrict__ tu, const float *__restrict__ rsq,
                                            const int32_t *__restrict__ perm, const int32_t *__restrict__ compp,
                                            const unsigned int *__restrict__ nmax_bits, float eps_rep, float mul32,
                                            float add32, int32_t *__restrict__ nsurv, int32_t *__restrict__ surv,
                                            int32_t *__restrict__ rowj, int32_t *__restrict__ ovf,
                                            const int32_t *__restrict__ set_of, const int32_t *__restrict__ setcnt,
                                            int32_t *counters, int32_t *__restrict__ bj_s, int shard_rank,
                                            int shard_world,
                                            const int32_t *__restrict__ row_lists) {
    if (lane == 0) nsurv[r] = 0;           // every row, padding included: k_exact_tc reads them all
    const int64_t i = perm[r];
    if (i < 0) return;                     // padding row
    if (shard_world > 1 && (int)((r / TC_BM) % shard_world) != shard_rank) {
        if (lane == 0) rowj[i] = -1;       // another rank's row (sharded calls)
        return;
    }
    if (setcnt && setcnt[set_of[i]] <= 1) {     // the row's set is one component already
        if (lane == 0) rowj[i] = -1;
        return;
    }
    // ---- the cut: U, the smallest upper bound over the lists of the
    //      row's nearest foreign d2; each lane holds EPL of the lists x 8
    //      block entries (lists x 8 <= 32 EPL)
    if (row_lists) lists = row_lists[r / TC_BM];
    const int ne = lists * TC_TOPK;
    float U = lane < lists ? tu[(size_t)lane * n + r] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) U = fminf(U, __shfl_xor_sync(0xffffffffu, U, o));
    if (!(U < INFINITY)) {
        if (lane == 0) rowj[i] = -1;
        return;
    }
    // representation error: distances move by at most w = eps (|y_i| + |y_max|).
    // FP32 bounds rounded upwards at every step, then inflated by 1e-5.
    const float si = rsq[r], smax = __fsqrt_ru(__uint_as_float(*nmax_bits));
    const float w = __fmul_ru(eps_rep, __fadd_ru(si, smax));
    const float a1 = __fadd_ru(__fsqrt_ru(fmaxf(U, 0.0f)), w);
    const float hi_true = __fmul_ru(__fmul_ru(a1, a1), 1.00001f);     // exact nearest foreign d2 <= this
    const float a2 = __fadd_ru(__fsqrt_ru(hi_true), w);
    const float tile_cut = __fmul_ru(__fmul_ru(a2, a2), 1.00001f);   // represented d2 of any candidate <= this
    // ---- the blocks whose lower bound is within the cut, compacted (their
    //      order does not matter).  TC_TOPK of them or more: a list may have
    //      dropped more, so the row is queued for a rescan.
    int cnt = 0;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
        const int e = lane + 32 * q;
        bool qual = false;
        int32_t blk = -1;
        if (e < ne) {
            const int sidx = e / TC_TOPK, k = e - sidx * TC_TOPK;
            const size_t o = ((size_t)sidx * n + r) * TC_TOPK + k;
            blk = tj[o];
            qual = blk >= 0 && tv[o] <= tile_cut;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, qual);
        const int slot = cnt + __popc(bal & below);
        if (qual && slot < TC_TOPK) bj_s[slot] = blk;
        cnt += __popc(bal);
    }
    if (cnt >= TC_TOPK) {
        if (lane == 0) {
            const int q = atomicAdd(counters + MC_OVERFLOW, 1);
            ovf[q] = (int32_t)i;
            rowj[i] = -2;
        }
        return;
    }
    if (cnt == 0) {
        if (lane == 0) rowj[i] = -1;
        return;
    }
    __syncwarp();
    int32_t bj[TC_TOPK];
#pragma unroll
    for (int k = 0; k < TC_TOPK; ++k) bj[k] = k < cnt ? bj_s[k] : -1;
    __syncwarp();                           // (bj_s is rewritten by the warp's next row)
    // FP32 direct differences over the qualifying blocks (up to four columns
    // per lane per pass, only as many as there are).  Pass 1: the row's FP32
    // minimum m32; the exact best has FP32 value <= m32 * mul32 + add32.
    // Pass 2 filters the first pass's distances and records those columns.
    const int32_t ci = compp[r];
    const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(xs) & 15) == 0;
    // a pass covers up to four columns per lane: SPB of each of BPP blocks
    constexpr int SPB = CW / 32, BPP = 4 / SPB;
    auto slots = [&](int k, int nu, int32_t (&jp)[4], bool (&live)[4]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = k + u / SPB;
            const int cand = (u < nu && q < TC_TOPK) ? bj[q < TC_TOPK ? q : 0] : -1;
            jp[u] = cand < 0 ? -1 : cand * CW + lane + 32 * (u % SPB);   // padded column (< n_pad <= 2^31)
            int32_t cj = -2;
            if (jp[u] >= 0 && jp[u] < n) cj = compp[jp[u]];
            live[u] = cj >= 0 && cj != ci;                                 // padding: -2
        }
    };
    auto scan = [&](int k, int32_t (&jp)[4], bool (&live)[4], float (&acc)[4]) {
        const int nu = min(4, (cnt - k) * SPB);                           // (warp-uniform)
        slots(k, nu, jp, live);
        if (nu == 1) rc_dist<1>(xs, r, d, vec, jp, live, acc);
        else if (nu == 2) rc_dist<2>(xs, r, d, vec, jp, live, acc);
        else rc_dist<4>(xs, r, d, vec, jp, live, acc);
    };
    // pass 1 keeps the distances of its first KEEP passes in registers; pass
    // 2 filters those against the threshold without reading the columns
    // again (later passes, rare, are scanned again).
    constexpr int NPASS = TC_TOPK / BPP, KEEP = NPASS < 2 ? NPASS : 2;
    float pmin[NPASS];
    float accs[KEEP][4];
    int32_t jps[KEEP][4];
    uint32_t livem = 0;                 // bit 4p + u: slot u of kept pass p is a live foreign point
    float m32 = INFINITY;
#pragma unroll
    for (int p = 0; p < NPASS; ++p) {
        pmin[p] = INFINITY;
        if (BPP * p >= cnt) continue;
        int32_t jp[4];
        bool live[4];
        float acc[4];
        scan(BPP * p, jp, live, acc);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (live[u]) pmin[p] = fminf(pmin[p], acc[u]);
            if (p < KEEP) {
                accs[p < KEEP ? p : 0][u] = acc[u];
                jps[p < KEEP ? p : 0][u] = jp[u];
                if (live[u]) livem |= 1u << (4 * p + u);
            }
        }
        m32 = fminf(m32, pmin[p]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m32 = fminf(m32, __shfl_xor_sync(0xffffffffu, m32, o));
    if (!(m32 < INFINITY)) {
        if (lane == 0) rowj[i] = -1;
        return;
    }
    const float thr = __fadd_ru(__fmul_ru(m32, mul32), add32);
    int ns = 0;
#pragma unroll
    for (int p = 0; p < NPASS; ++p) {
        if (!__any_sync(0xffffffffu, pmin[p] <= thr)) continue;
        int32_t jp[4];
        bool live[4];
        float acc[4];
        if (p < KEEP) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[u] = accs[p < KEEP ? p : 0][u];
                jp[u] = jps[p < KEEP ? p : 0][u];
                live[u] = (livem >> (4 * p + u)) & 1u;
            }
        } else {
            scan(BPP * p, jp, live, acc);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool sv = live[u] && acc[u] <= thr;
            const unsigned bal = __ballot_sync(0xffffffffu, sv);
            const int slot = ns + __popc(bal & below);
            if (sv && slot < TC_SURV) surv[r * TC_SURV + slot] = jp[u];
            ns += __popc(bal);
        }
    }
    if (lane == 0) {
        if (ns > TC_SURV) {                     // many near-ties: exact rescan of the row
            const int q = atomicAdd(counters + MC_OVERFLOW, 1);
            ovf[q] = (int32_t)i;
            rowj[i] = -2;
        } else {
            nsurv[r] = ns;
        }
    }
}

// Exact keys of the recorded columns, one thread per row: the FP64 pipe sees
// full warps (a warp per row would run each key on a single lane).
__global__ void __launch_bounds__(256) k_exact_tc(const float *__restrict__ xs, int64_t n, int32_t d,
                                                  const int32_t *__restrict__ perm, const int32_t *__restrict__ nsurv,
                                                  const int32_t *__restrict__ surv, double *__restrict__ rowd2,
                                                  int32_t *__restrict__ rowj, const int32_t *counters) {
    if (!mst_active(counters)) return;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gs) {
        const int c = nsurv[r];
        const int32_t i = perm[r];
        if (c <= 0 || c > TC_SURV || i < 0) continue;
        const float *xi = xs + r * d;
        double best = INFINITY;
        int32_t bestj = -1;
        for (int q = 0; q < c; ++q) {
            const int64_t jp = surv[r * TC_SURV + q];
            if (jp < 0 || jp >= n) continue;
            const int32_t j = perm[jp];
            if (j < 0) continue;
            const double e = exact_d2(xi, xs + jp * d, d);
            if (bestj < 0 || key_less(e, i, j, best, i, bestj)) {
                best = e;
                bestj = j;
            }
        }
        rowd2[i] = best;
        rowj[i] = bestj;
    }
}

template <int EPL, int CW>
__global__ void __launch_bounds__(256, 4) k_recheck_tc(const float *__restrict__ xs, int64_t n, int32_t d, int lists,
                                                       const float *__restrict__ tv, const int32_t *__restrict__ tj,
                                                       const float *__restrict__ tu, const float *__restrict__ rsq,
                                                       const int32_t *__restrict__ perm,
                                                       const int32_t *__restrict__ compp,
                                                       const unsigned int *__restrict__ nmax_bits, float eps_rep,
                                                       float mul32, float add32, int32_t *__restrict__ nsurv,
                                                       int32_t *__restrict__ surv, int32_t *__restrict__ rowj,
                                                       int32_t *__restrict__ ovf, const int32_t *__restrict__ set_of,
                                                       const int32_t *__restrict__ setcnt, int32_t *counters,
                                                       int shard_rank, int shard_world,
                                                       const int32_t *__restrict__ row_lists) {
    if (!mst_active(counters)) return;
    __shared__ int32_t bj_s[8][TC_TOPK];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw)
        recheck_row<EPL, CW>(r, lane, xs, n, d, lists, tv, tj, tu, rsq, perm, compp, nmax_bits, eps_rep, mul32, add32, nsurv,
                             surv, rowj, ovf, set_of, setcnt, counters, bj_s[wib], shard_rank,
                             shard_world, row_lists);
}

// Self-contained rescan of a queued row: FP32 direct differences give the
// minimum m; every column within the FP32 error margin of m is keyed in FP64.
// With independent sets only the row's own set is scanned.
__global__ void __launch_bounds__(256) k_rescan_tc(const float *__restrict__ X, int64_t n, int32_t d,
                                                   const int32_t *__restrict__ comp, const int32_t *__restrict__ ovf,
                                                   const int32_t *__restrict__ set_of, const int64_t *__restrict__ offs,
                                                   double mul, double add, double *__restrict__ rowd2,
                                                   int32_t *__restrict__ rowj, int32_t *counters) {
    if (!mst_active(counters)) return;
    __shared__ float smin[256];
    __shared__ double sd[256];
    __shared__ int32_t sj[256];
    const int nq = counters[MC_OVERFLOW];
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const int64_t i = ovf[q];
        const int32_t ci = comp[i];
        const float *xi = X + i * d;
        const int64_t j0 = set_of ? offs[set_of[i]] : 0, j1 = set_of ? offs[set_of[i] + 1] : n;
        float m = INFINITY;
        for (int64_t j = j0 + threadIdx.x; j < j1; j += 256) {
            if (comp[j] == ci) continue;
            float acc = 0.0f;
            for (int t = 0; t < d; ++t) {
                const float df = __fsub_rn(xi[t], X[j * d + t]);
                acc = __fmaf_rn(df, df, acc);
            }
            m = fminf(m, acc);
        }
        smin[threadIdx.x] = m;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + s]);
            __syncthreads();
        }
        const double tau = (double)smin[0] * mul + add;
        double bd = INFINITY;
        int32_t bjj = -1;
        for (int64_t j = j0 + threadIdx.x; j < j1; j += 256) {
            if (comp[j] == ci) continue;
            float acc = 0.0f;
            for (int t = 0; t < d; ++t) {
                const float df = __fsub_rn(xi[t], X[j * d + t]);
                acc = __fmaf_rn(df, df, acc);
            }
            if ((double)acc <= tau) {
                const double e = exact_d2(xi, X + j * d, d);
                if (bjj < 0 || key_less(e, (int32_t)i, (int32_t)j, bd, (int32_t)i, bjj)) { bd = e; bjj = (int32_t)j; }
            }
        }
        sd[threadIdx.x] = bd;
        sj[threadIdx.x] = bjj;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double od = sd[threadIdx.x + s];
                const int32_t oj = sj[threadIdx.x + s];
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

cudaError_t make_map_rows(CUtensorMap *m, const void *base, int64_t n_pad, int32_t d_pad, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)d_pad, (cuuint64_t)n_pad};
    cuuint64_t strides[1] = {(cuuint64_t)d_pad * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t n_pad, int32_t d_pad) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)d_pad, (cuuint64_t)n_pad};
    cuuint64_t strides[1] = {(cuuint64_t)d_pad * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

cudaError_t tc_map_bf16(CUtensorMap *m, const void *base, int64_t rows, int32_t cols, int box_rows) {
    return make_map_rows(m, base, rows, cols, box_rows);
}

void TcScratch::carve(Arena &A, int64_t n, int32_t d, int splits_, int64_t n_pad_rows, int nmeans, int lists_) {
    splits = splits_;
    lists = lists_ > 0 ? lists_ : 2 * splits;
    n_pad = n_pad_rows > 0 ? n_pad_rows : ceil_div(n, TC_BM) * TC_BM;
    d_pad = (int32_t)(ceil_div(d, TC_BK) * TC_BK);
    const int64_t nt = n_pad / TC_BM;
    xh = A.take<__nv_bfloat16>((size_t)n_pad * d_pad, 1024);
    xl = A.take<__nv_bfloat16>((size_t)n_pad * d_pad, 1024);
    xs = A.take<float>((size_t)n_pad * d, 256);
    nrm = A.take<float>(n_pad);
    cnrm = A.take<float>(n_pad);
    rsq = A.take<float>(n_pad);
    tmax = A.take<float>(nt);
    tsq = A.take<float>(nt);
    mean = A.take<float>((size_t)(nmeans > 0 ? nmeans : 1) * d);
    part = A.take<double>((size_t)64 * d);
    nmax_bits = A.take<unsigned int>(4);
    perm = A.take<int32_t>(n);
    permp = A.take<int32_t>(n_pad);
    vbuf = A.take<int32_t>(n);
    keys = A.take<uint64_t>(n);
    kbuf = A.take<uint64_t>(n);
    compp = A.take<int32_t>(n_pad);
    nsurv = A.take<int32_t>(n_pad);
    surv = A.take<int32_t>((size_t)n_pad * TC_SURV);
    tv = A.take<float>((size_t)lists * n_pad * TC_TOPK);
    tj = A.take<int32_t>((size_t)lists * n_pad * TC_TOPK);
    tu = A.take<float>((size_t)lists * n_pad);
    err = A.take<uint32_t>(4);
    qctr = A.take<uint32_t>(4);
    setcnt = nmeans > 1 || n_pad_rows > 0 ? A.take<int32_t>((size_t)(nmeans > 0 ? nmeans : 1)) : nullptr;
    if (prune) {
        tcen = A.take<float>((size_t)nt * d);
        trad = A.take<float>(nt);
        tlb2 = A.take<float>((size_t)nt * nt);
        cub = A.take<unsigned int>(n);
        tmu = A.take<float>(nt);
        tcomp = A.take<int32_t>(nt);
        items_a = A.take<int4>(nt);
        items_b = A.take<int4>((size_t)nt * (PRUNE_SLOTS - 1));
        far = A.take<unsigned long long>((size_t)4 * nt);
        swept = A.take<unsigned long long>(1);
        nlists = A.take<int32_t>(nt);
    }
}

namespace {
struct TuneKey {
    int dev, sets, d_pad, lg_rows, lg_items;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, sets, d_pad, lg_rows, lg_items) < std::tie(o.dev, o.sets, o.d_pad, o.lg_rows, o.lg_items);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;           // shape class -> fastest variant
std::atomic<int> g_force{-1};
thread_local int g_last_variant = -1;
int ilog2(int64_t x) {
    int l = 0;
    while (x > 1) { x >>= 1; ++l; }
    return l;
}
void apply_variant(TcScratch &T, int v) {
    T.cw = (v & 1) ? 32 : 64;
    T.resident = (v & 2) == 0;
}
}  // namespace

void tc_force_variant(int variant) { g_force.store(variant); }
int tc_forced_variant() { return g_force.load(); }
int tc_last_variant() { return g_last_variant; }
void tc_clear_last_variant() { g_last_variant = -1; }

cudaError_t tc_autotune(TcScratch &T, MstScratch &S, const float *X, int64_t n, int32_t d, uint32_t *status,
                        cudaStream_t s) {
    const int heuristic = (T.cw == 32 ? 1 : 0) | (T.resident ? 0 : 2);
    const int forced = g_force.load();
    if (forced >= 0) {
        apply_variant(T, forced);
        g_last_variant = forced;
        return cudaSuccess;
    }
    const int kchunks = T.d_pad / TC_BK;
    const int64_t items = T.items ? T.nitems : (T.n_pad / TC_BM) * T.splits;
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    const TuneKey key{dev, (T.set_of != nullptr ? 1 : 0) | (T.prune ? 2 : 0), T.d_pad, ilog2(T.n_pad),
                      ilog2(items > 0 ? items : 1)};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply_variant(T, it->second);
            g_last_variant = it->second;
            return cudaSuccess;
        }
    }
    // small problems: a trial round costs more than any difference
    if (T.n_pad < 8192) {
        g_last_variant = heuristic;
        return cudaSuccess;
    }
    int cand[4], nc = 0;
    cand[nc++] = 0;
    cand[nc++] = 1;
    if (kchunks <= 2) {
        cand[nc++] = 2;
        cand[nc++] = 3;
    }
    int32_t saved[8];
    if ((e = cudaMemcpyAsync(saved, S.counters, sizeof(saved), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
        if (e0) cudaEventDestroy(e0);
        return e;
    }
    int best = heuristic;
    float best_ms = INFINITY;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        apply_variant(T, cand[c]);
        // two trial rounds on the round-1 state, the second timed; the
        // rescan queue is emptied before each (it indexes by its count)
        float ms = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            if ((e = cudaMemsetAsync(S.counters + MC_OVERFLOW, 0, sizeof(int32_t), s))) break;
            if ((e = cudaEventRecord(e0, s))) break;
            if ((e = tc_sweep_round(T, S, X, n, d, status, s))) break;
            if ((e = cudaEventRecord(e1, s))) break;
            if ((e = cudaEventSynchronize(e1))) break;
            if ((e = cudaEventElapsedTime(&ms, e0, e1))) break;
        }
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return e;
    // restore the round counters (the trials only touched the rescan queue)
    if ((e = cudaMemcpy(S.counters, saved, sizeof(saved), cudaMemcpyHostToDevice))) return e;
    if (T.swept && (e = cudaMemsetAsync(T.swept, 0, sizeof(unsigned long long), s))) return e;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[key] = best;
    }
    apply_variant(T, best);
    g_last_variant = best;
    return cudaSuccess;
}

cudaError_t tc_count_sets(TcScratch &T, const int32_t *comp, int64_t n, const int32_t *counters, cudaStream_t s) {
    if (!T.set_of || !T.setcnt) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemsetAsync(T.setcnt, 0, sizeof(int32_t) * T.nsets, s))) return e;
    const int64_t b = ceil_div(n, 256), cap = (int64_t)num_sms() * 8;
    k_tc_set_roots<<<(unsigned)(b < cap ? b : cap), 256, 0, ISO_S(s)>>>(comp, T.set_of, n, T.setcnt, counters);
    return cudaGetLastError();
}

cudaError_t tc_omega_screen(TcScratch &T, const float *Xp, int64_t n, int32_t d,
                            const unsigned long long *nnbits, double sigma, double zskip, uint8_t *need, int64_t T64,
                            cudaStream_t s) {
    cudaError_t e;
    T.keep_order = true;
    T.set_of = nullptr;
    T.items = nullptr;
    if ((e = tc_prepare(T, Xp, n, d, s))) return e;
    float *rowA = T.tu;                                     // >= n_pad floats
    const double eps_rep = 1.25 * (3.814697265625e-06 + 5.9604644775390625e-08);
    k_screen_rows<<<(unsigned)ceil_div(T.n_pad, 256), 256, 0, ISO_S(s)>>>(nnbits, T.rsq, T.nmax_bits, n, T.n_pad, sigma,
                                                                          zskip, eps_rep, rowA);
    if ((e = cudaMemsetAsync(need, 0, (size_t)T64 * T64, s))) return e;
    // the upper triangle of 128-row tiles, row tile I against [I, T) in
    // chunks of 16 column tiles
    const int ntiles = (int)(T.n_pad / TC_BM);
    std::vector<int4> items;
    for (int I = 0; I < ntiles; ++I)
        for (int c0 = I; c0 < ntiles; c0 += 16) items.push_back(make_int4(I, c0, c0 + 16 < ntiles ? c0 + 16 : ntiles, 0));
    int4 *ditems = reinterpret_cast<int4 *>(T.tj);          // lists x n_pad x 8 int32 >> items
    if ((size_t)items.size() * sizeof(int4) > (size_t)T.lists * T.n_pad * TC_TOPK * sizeof(int32_t))
        return cudaErrorInvalidValue;
    if ((e = cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s))) return e;
    const int kchunks = T.d_pad / TC_BK;
    const int64_t nsm = (int64_t)num_sms(), nit = (int64_t)items.size();
    const unsigned grid = (unsigned)(nit < nsm ? nit : nsm);
    const double u = 1.1920928955078125e-07;
    const float acoef = (float)(1.25 * 2.0 * (3.0 * T.d_pad * u + 3.814697265625e-06));
    const float bcoef = (float)(1.25 * 8.0 * 5.9604644775390625e-08);
    const ScreenArgs scr{rowA, need, T64};
#define ISO_SCREEN_LAUNCH(AKV)                                                                                    \
    k_sweep_tc<AKV, true, 64><<<grid, TC_THREADS, tc_smem(AKV), ISO_S(s)>>>(                                          \
        T.map_h, T.map_l, T.nrm, T.cnrm, T.rsq, T.tmax, T.tsq, acoef, bcoef, nullptr, T.n_pad, ntiles, kchunks, 1,   \
        ditems, nit, nullptr, nullptr, nullptr, nullptr, nullptr, T.err, scr, tc_wait_limit(T), T.stall_test, 1, 0,  \
        T.qctr)
    if ((e = cudaMemsetAsync(T.qctr, 0, sizeof(uint32_t), s))) return e;
    if (kchunks == 1)
        ISO_SCREEN_LAUNCH(1);
    else if (kchunks == 2)
        ISO_SCREEN_LAUNCH(2);
    else
        ISO_SCREEN_LAUNCH(0);
#undef ISO_SCREEN_LAUNCH
    return cudaGetLastError();
}

// At most 16 splits: the recheck merges 2 x splits candidate lists in one warp.
int tc_splits(int64_t n) {
    const int64_t rt = ceil_div(n, TC_BM);
    int64_t s = ceil_div((int64_t)num_sms() * 16, rt > 0 ? rt : 1);
    const int64_t max_s = rt / 4 > 1 ? rt / 4 : 1;
    if (s > max_s) s = max_s;
    if (s > 16) s = 16;
    if (s < 1) s = 1;
    return (int)s;
}

bool tc_supported() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

cudaError_t tc_prepare(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s, bool place) {
    cudaError_t e;
    const bool sets = T.set_of != nullptr;
    if (sets) {
        k_tc_set_mean<<<(unsigned)T.nsets, 256, 0, ISO_S(s)>>>(X, T.offs, d, T.mean);
    } else {
        const int64_t rows_per = ceil_div(n, 64);
        dim3 gm(64, (unsigned)ceil_div(d, 32));
        k_tc_mean_partial<<<gm, 256, 0, ISO_S(s)>>>(X, n, d, rows_per, T.part);
        k_tc_mean_final<<<(unsigned)ceil_div(d, 128), 128, 0, ISO_S(s)>>>(T.part, 64, n, d, T.mean);
    }
    T.prune_ready = false;           // (pruned rounds start after the first, in their own row order)
    if (T.keep_order) {
        // rows as given (the omega screen works in omega's row order)
        k_tc_identity<<<(unsigned)ceil_div(T.n_pad, 256), 256, 0, ISO_S(s)>>>(T.permp, n, T.n_pad);
    } else if (place) {
        // norm order: tiles of points with similar |x - c| give tight tile bounds
        k_tc_prenorm_keys<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(X, T.mean, T.set_of, n, d, T.keys, T.perm);
        if ((e = sort_pairs_u64(T.keys, T.perm, T.kbuf, T.vbuf, n, s))) return e;
        if ((e = cudaMemsetAsync(T.permp, 0xff, sizeof(int32_t) * T.n_pad, s))) return e;     // -1: padding
        k_tc_place<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(T.perm, n, T.set_of, T.offs, T.rowbase,
                                                                    T.permp);
    }
    T.cw = (sets || T.d_pad > 64) ? 32 : 64;      // heuristic variant (see tc_autotune)
    T.resident = true;
    if (place || T.keep_order) {
        const int64_t tot = T.n_pad * T.d_pad;
        k_tc_split<<<(unsigned)ceil_div(tot, 256), 256, 0, ISO_S(s)>>>(X, T.mean, T.set_of, T.permp, d, T.n_pad,
                                                                      T.d_pad, T.xh, T.xl, T.xs);
        if ((e = cudaMemsetAsync(T.nmax_bits, 0, sizeof(unsigned int), s))) return e;
        k_tc_norms<<<(unsigned)ceil_div(T.n_pad, 256), 256, 0, ISO_S(s)>>>(T.xh, T.xl, T.permp, T.n_pad, T.d_pad,
                                                                          T.nrm, T.cnrm, T.rsq, T.nmax_bits);
        k_tc_tile_max<<<(unsigned)ceil_div(T.n_pad / TC_BM, 128), 128, 0, ISO_S(s)>>>(T.nrm, T.n_pad, T.tmax,
                                                                                      T.tsq);
    }
    if (T.swept && (e = cudaMemsetAsync(T.swept, 0, sizeof(unsigned long long), s))) return e;
    if (sets) {
        // lists that no item writes (sets with fewer splits) stay empty
        const int64_t nv = (int64_t)T.lists * T.n_pad * TC_TOPK, nu = (int64_t)T.lists * T.n_pad;
        k_tc_fill_lists<<<(unsigned)ceil_div(nv, 256), 256, 0, ISO_S(s)>>>(T.tv, T.tj, T.tu, nv, nu);
    }
    if ((e = cudaMemsetAsync(T.err, 0, sizeof(uint32_t), s))) return e;
    if ((e = make_map(&T.map_h, T.xh, T.n_pad, T.d_pad))) return e;
    if ((e = make_map(&T.map_l, T.xl, T.n_pad, T.d_pad))) return e;
    static bool attr = false;
    if (!attr) {
#define ISO_SMEM_ATTR(AKV, SCR, CWV)                                                                              \
    if ((e = cudaFuncSetAttribute(k_sweep_tc<AKV, SCR, CWV>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                  tc_smem(AKV))))                                                                 \
        return e;
        ISO_SMEM_ATTR(0, false, 32)
        ISO_SMEM_ATTR(1, false, 32)
        ISO_SMEM_ATTR(2, false, 32)
        ISO_SMEM_ATTR(0, false, 64)
        ISO_SMEM_ATTR(1, false, 64)
        ISO_SMEM_ATTR(2, false, 64)
        ISO_SMEM_ATTR(0, true, 64)
        ISO_SMEM_ATTR(1, true, 64)
        ISO_SMEM_ATTR(2, true, 64)
#undef ISO_SMEM_ATTR
        attr = true;
    }
    return cudaGetLastError();
}

cudaError_t tc_place_rows(TcScratch &T, const float *X, int64_t n, int32_t d, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(T.permp, 0xff, sizeof(int32_t) * T.n_pad, s))) return e;     // -1: padding
    k_tc_place<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(T.perm, n, nullptr, nullptr, nullptr, T.permp);
    const int64_t tot = T.n_pad * T.d_pad;
    k_tc_split<<<(unsigned)ceil_div(tot, 256), 256, 0, ISO_S(s)>>>(X, T.mean, nullptr, T.permp, d, T.n_pad, T.d_pad,
                                                                  T.xh, T.xl, T.xs);
    if ((e = cudaMemsetAsync(T.nmax_bits, 0, sizeof(unsigned int), s))) return e;
    k_tc_norms<<<(unsigned)ceil_div(T.n_pad, 256), 256, 0, ISO_S(s)>>>(T.xh, T.xl, T.permp, T.n_pad, T.d_pad, T.nrm,
                                                                      T.cnrm, T.rsq, T.nmax_bits);
    k_tc_tile_max<<<(unsigned)ceil_div(T.n_pad / TC_BM, 128), 128, 0, ISO_S(s)>>>(T.nrm, T.n_pad, T.tmax, T.tsq);
    return cudaGetLastError();
}

cudaError_t tc_sweep_round(TcScratch &T, MstScratch &S, const float *X, int64_t n, int32_t d, uint32_t *status,
                           cudaStream_t s) {
    const int ntiles = (int)(T.n_pad / TC_BM);
    const int kchunks = T.d_pad / TC_BK;
    // a sharded call sweeps the row tiles t with t mod world == rank
    const int64_t own_tiles = T.shard_rank < ntiles
                                  ? ((int64_t)ntiles - T.shard_rank + T.shard_world - 1) / T.shard_world : 0;
    const int64_t nsm = (int64_t)num_sms();
    const bool pruned = T.prune && T.prune_ready && !T.items && T.shard_world == 1;
    const int64_t gblocks = ceil_div(T.n_pad, 256), gcap = (int64_t)num_sms() * 8;
    k_tc_gather_comp<<<(unsigned)(gblocks < gcap ? gblocks : gcap), 256, 0, ISO_S(s)>>>(S.comp, T.permp, T.n_pad,
                                                                                       T.compp, S.counters);
    // d2 = n_i + n_j - 2g against d2 of the represented points: tensor-core
    // FP32 accumulation of 3 d_pad products (worst case: one rounding of the
    // running magnitude per addition, 2^-23) and the dropped lo.lo term
    // (2^-18), both times 2|y_i||y_j|; FP32 rounding of the norms (2^-24
    // (n_i + n_j)) and of the epilogue's fl(fl(n_j - 2g) + n_i) (at most
    // 2^-24 (4 n_i + 5 n_j)): 8 x 2^-24 (n_i + n_j).  25 % headroom.
    const double u = 1.1920928955078125e-07;   // 2^-23
    const float acoef = (float)(1.25 * 2.0 * (3.0 * T.d_pad * u + 3.814697265625e-06));
    const float bcoef = (float)(1.25 * 8.0 * 5.9604644775390625e-08);
    // one sweep launch over an item list (null: row tile x column split)
    auto sweep = [&](const int4 *wit, int64_t nwit) {
        const int64_t items = wit ? nwit : own_tiles * T.splits;
        const unsigned grid = (unsigned)(items < nsm ? (items > 0 ? items : 1) : nsm);
#define ISO_SWEEP_LAUNCH(AKV, CWV)                                                                                \
    k_sweep_tc<AKV, false, CWV><<<grid, TC_THREADS, tc_smem(AKV), ISO_S(s)>>>(                                         \
        T.map_h, T.map_l, T.nrm, T.cnrm, T.rsq, T.tmax, T.tsq, acoef, bcoef, T.compp, T.n_pad, ntiles, kchunks,      \
        T.splits, wit, nwit, T.setcnt, S.counters, T.tv, T.tj, T.tu, T.err, ScreenArgs{},                        \
        tc_wait_limit(T), T.stall_test, wit ? 1 : T.shard_world, wit ? 0 : T.shard_rank, T.qctr)
        const cudaError_t me = cudaMemsetAsync(T.qctr, 0, sizeof(uint32_t), s);
        if (me != cudaSuccess) return me;
        if (kchunks == 1 && T.resident) {
            if (T.cw == 32) ISO_SWEEP_LAUNCH(1, 32);
            else ISO_SWEEP_LAUNCH(1, 64);
        } else if (kchunks == 2 && T.resident) {
            if (T.cw == 32) ISO_SWEEP_LAUNCH(2, 32);
            else ISO_SWEEP_LAUNCH(2, 64);
        } else {
            if (T.cw == 32) ISO_SWEEP_LAUNCH(0, 32);
            else ISO_SWEEP_LAUNCH(0, 64);
        }
#undef ISO_SWEEP_LAUNCH
        return cudaGetLastError();
    };
    if (pruned) {
        // near tiles first (candidate list slot 0); their candidates bound
        // each component's lightest edge, which decides the far items
        // (slots 1 .. PRUNE_SLOTS - 1)
        cudaError_t pe = sweep(T.items_a, ntiles);
        if (pe == cudaSuccess) pe = prune_far_items(T, S.comp, S.rowd2, S.rowj, n, S.counters, s);
        if (pe == cudaSuccess) pe = sweep(T.items_b, (int64_t)ntiles * (PRUNE_SLOTS - 1));
        if (pe != cudaSuccess) return pe;
    } else {
        const cudaError_t pe = sweep(T.items, T.nitems);
        if (pe != cudaSuccess) return pe;
    }
    // representation error of a centred point by BF16 hi + lo: 2^-18 relative
    // per element, plus the FP32 rounding of x - c (2^-24); 25 % headroom
    const double eps_rep = 1.25 * (3.814697265625e-06 + 5.9604644775390625e-08);
    // FP32 direct differences: relative error <= e (and an underflow term);
    // any column within m32 * (1+e)/(1-e) + 2 add of the row's FP32 minimum
    // can hold the exact best
    const double e = 1.1 * (double)(d + 3) * 5.9604644775390625e-08;
    const double mul = (1.0 + e) / (1.0 - e);
    const double add = (double)(d + 1) * 1.401298464324817e-45 * 4.0;
    const float mul32 = (float)(mul * (1.0 + 1e-6)), add32 = (float)(2.01 * add) + 1.401298464324817e-45f;
    const int64_t rblocks = ceil_div(T.n_pad * 32, 256), rcap = (int64_t)num_sms() * 16;
    // entries per lane of the list merge: lists x 8 <= 32 EPL (lists <= 32)
#define ISO_RECHECK_LAUNCH(EPLV, CWV)                                                                                \
    k_recheck_tc<EPLV, CWV><<<(unsigned)(rblocks < rcap ? rblocks : rcap), 256, 0, ISO_S(s)>>>(                        \
        T.xs, T.n_pad, d, T.lists, T.tv, T.tj, T.tu, T.rsq, T.permp, T.compp, T.nmax_bits, (float)(eps_rep * 1.0001),  \
        mul32, add32, T.nsurv, T.surv, S.rowj, S.ovf_rows, T.set_of, T.setcnt, S.counters, T.shard_rank,           \
        T.shard_world, pruned ? T.nlists : nullptr)
    if (T.lists <= 4)
        {
        if (T.cw == 32) ISO_RECHECK_LAUNCH(1, 32);
        else ISO_RECHECK_LAUNCH(1, 64);
    }
    else if (T.lists <= 8)
        {
        if (T.cw == 32) ISO_RECHECK_LAUNCH(2, 32);
        else ISO_RECHECK_LAUNCH(2, 64);
    }
    else if (T.lists <= 16)
        {
        if (T.cw == 32) ISO_RECHECK_LAUNCH(4, 32);
        else ISO_RECHECK_LAUNCH(4, 64);
    }
    else
        {
        if (T.cw == 32) ISO_RECHECK_LAUNCH(8, 32);
        else ISO_RECHECK_LAUNCH(8, 64);
    }
#undef ISO_RECHECK_LAUNCH
    const int64_t xblocks = ceil_div(T.n_pad, 256), xcap = (int64_t)num_sms() * 8;
    k_exact_tc<<<(unsigned)(xblocks < xcap ? xblocks : xcap), 256, 0, ISO_S(s)>>>(T.xs, T.n_pad, d, T.permp, T.nsurv,
                                                                                  T.surv, S.rowd2, S.rowj,
                                                                                  S.counters);
    k_rescan_tc<<<(unsigned)(num_sms() * 4), 256, 0, ISO_S(s)>>>(X, n, d, S.comp, S.ovf_rows, T.set_of, T.offs, mul,
                                                                 add, S.rowd2, S.rowj, S.counters);
    (void)status;
    return cudaGetLastError();
}

}  // namespace iso

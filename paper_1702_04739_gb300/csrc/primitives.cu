// primitives.cu -- exclusive scan and stable merge sort.
#include "common.cuh"

namespace iso {

namespace {
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles(const T *__restrict__ in, T *__restrict__ out,
                                                          int64_t n, T *__restrict__ sums) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : T(0);
        acc += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;   // exclusive warp offsets
    }
    __syncthreads();
    T run = warp_tot[warp] + incl - acc;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = run;
}

template <class T>
__global__ void add_tile_offsets(T *__restrict__ out, int64_t n, const T *__restrict__ offs) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += offs[idx / SCAN_TILE];
}

template <class T>
cudaError_t scan_impl(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t nb = ceil_div(n, SCAN_TILE);
    T *sums = tmp;
    T *sums_scanned = tmp + nb;
    scan_tiles<T><<<(unsigned)nb, SCAN_THREADS, 0, ISO_S(s)>>>(in, out, n, sums);
    if (nb > 1) {
        cudaError_t e = scan_impl<T>(sums, sums_scanned, nb, tmp + 2 * nb, s);
        if (e != cudaSuccess) return e;
        add_tile_offsets<T><<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(out, n, sums_scanned);
    }
    return cudaGetLastError();
}
}  // namespace

size_t scan_tmp_elems(int64_t n) {
    size_t tot = 0;
    while (n > 1) {
        int64_t nb = ceil_div(n, SCAN_TILE);
        tot += 2 * (size_t)nb;
        n = nb;
    }
    return tot + 2;
}

cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, tmp, s);
}
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, tmp, s);
}

// ---------------------------------------------------------------- merge sort
namespace {
// One merge pass: runs of width w are merged pairwise.  Each element finds
// its output slot from its rank in its own run plus a binary search in the
// partner run (A-elements go before equal B-elements: stable).
__global__ void merge_pass(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
                           uint64_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int64_t w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t run = i / w;
    int64_t start = (run & ~1LL) * w;
    uint64_t key = kin[i];
    int64_t pos_in_run = i - run * w;
    int64_t out;
    if ((run & 1) == 0) {
        int64_t b0 = start + w, b1 = min(start + 2 * w, n);
        int64_t lo = b0, hi = b1;   // first B element with key >= key
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (kin[mid] < key) lo = mid + 1; else hi = mid;
        }
        out = start + pos_in_run + (lo - b0);
    } else {
        int64_t a0 = start, a1 = start + w;
        int64_t lo = a0, hi = a1;   // first A element with key > key
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (kin[mid] <= key) lo = mid + 1; else hi = mid;
        }
        out = start + pos_in_run + (lo - a0);
    }
    kout[out] = key;
    vout[out] = vin[i];
}

// The first passes in shared memory: each block sorts its chunk of
// SORT_CHUNK elements with the same stable rank merge, run widths 1 to
// SORT_CHUNK / 2, then the global passes continue from SORT_CHUNK.
constexpr int SORT_CHUNK = 2048, SORT_THREADS = 1024;
__global__ void __launch_bounds__(SORT_THREADS) chunk_sort(const uint64_t *__restrict__ kin,
                                                           const int32_t *__restrict__ vin,
                                                           uint64_t *__restrict__ kout, int32_t *__restrict__ vout,
                                                           int64_t n) {
    __shared__ uint64_t sk[2][SORT_CHUNK];
    __shared__ int32_t sv[2][SORT_CHUNK];
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    const int cnt = (int)(n - base < SORT_CHUNK ? n - base : SORT_CHUNK);
    for (int i = threadIdx.x; i < cnt; i += SORT_THREADS) {
        sk[0][i] = kin[base + i];
        sv[0][i] = vin[base + i];
    }
    __syncthreads();
    int b = 0;
    for (int w = 1; w < cnt; w <<= 1, b ^= 1) {
        const uint64_t *ka = sk[b];
        for (int i = threadIdx.x; i < cnt; i += SORT_THREADS) {
            const int run = i / w, start = (run & ~1) * w, pos = i - run * w;
            const uint64_t key = ka[i];
            int out;
            if ((run & 1) == 0) {
                int lo = start + w < cnt ? start + w : cnt, hi = start + 2 * w < cnt ? start + 2 * w : cnt;
                const int b0 = lo;
                while (lo < hi) {                    // first B element with key >= key
                    const int mid = (lo + hi) >> 1;
                    if (ka[mid] < key) lo = mid + 1; else hi = mid;
                }
                out = start + pos + (lo - b0);
            } else {
                int lo = start, hi = start + w;
                while (lo < hi) {                    // first A element with key > key
                    const int mid = (lo + hi) >> 1;
                    if (ka[mid] <= key) lo = mid + 1; else hi = mid;
                }
                out = start + pos + (lo - start);
            }
            sk[b ^ 1][out] = key;
            sv[b ^ 1][out] = sv[b][i];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < cnt; i += SORT_THREADS) {
        kout[base + i] = sk[b][i];
        vout[base + i] = sv[b][i];
    }
}
}  // namespace

cudaError_t sort_pairs_u64(uint64_t *keys, int32_t *vals, uint64_t *kbuf, int32_t *vbuf, int64_t n,
                           cudaStream_t s) {
    if (n <= 1) return cudaSuccess;
    uint64_t *ka = keys, *kb = kbuf;
    int32_t *va = vals, *vb = vbuf;
    chunk_sort<<<(unsigned)ceil_div(n, SORT_CHUNK), SORT_THREADS, 0, ISO_S(s)>>>(ka, va, kb, vb, n);
    {
        uint64_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    for (int64_t w = SORT_CHUNK; w < n; w <<= 1) {
        merge_pass<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(ka, va, kb, vb, n, w);
        uint64_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace iso

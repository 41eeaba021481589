// noalloc.cu -- isoclust_tree_isoperimetric_noalloc: the tree stage with its
// scratch in a file-scope device array, for callers that cannot allocate.
//
// Some callers of this library cannot call cudaMalloc: a host application
// that hands the whole device to its own memory pool (an inference server or
// a framework allocator that reserves all free memory up front), where a
// foreign cudaMalloc fails or breaks the pool's accounting; or a real-time
// loop on one stream that cannot afford cudaMalloc/cudaFree, which may
// synchronise the whole device.  The regular entry points grow a cached
// scratch buffer with cudaMalloc; this one never does.  Its scratch is the
// array below, which bounds the tree it accepts to ISOCLUST_NOALLOC_MAX_N
// vertices.  The array lives in this file's own device module, which the
// CUDA runtime loads lazily: it takes its place in a device's memory when
// the first call on that device looks up its address, and stays there until
// the process exits.  So that first call (any small tree) belongs before the
// caller's pool reserves the device's free memory, and before any stream
// capture; loading the module may synchronise the device.
#include <mutex>

#include "common.cuh"
#include "tree.cuh"

namespace iso {

// Scratch of the tree stage for n <= ISOCLUST_NOALLOC_MAX_N (12.2 MiB measured,
// 13 MiB reserved).  Host code must not pass this name to a kernel: on the
// host it is only a stand-in for the symbol.  Its device address is looked
// up with cudaGetSymbolAddress below.
constexpr size_t NOALLOC_BYTES = size_t(13) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
constexpr int NA_MAX_DEV = 64;
std::mutex g_na_mu[NA_MAX_DEV];
void *g_na_ptr[NA_MAX_DEV] = {nullptr};

__global__ void k_na_init(int32_t *info, uint32_t *st) {
    info[0] = 0;
    info[1] = 2147483647;
    st[0] = 0u;
}

__global__ void k_na_tree_input(const int32_t *__restrict__ parent, int64_t n, int32_t *info, uint32_t *st) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t p = parent[v];
    if (p == -1) {
        atomicAdd(info + 0, 1);
        atomicMin(info + 1, (int32_t)v);
    } else if (p < 0 || p >= n || p == v) {
        atomicOr(st, DEV_BAD_TREE);
    }
}

}  // namespace

}  // namespace iso

using namespace iso;

extern "C" isoclust_status isoclust_tree_isoperimetric_noalloc(int64_t n, const int32_t *parent,
                                                               const double *phi_par, const double *omega,
                                                               const double *p, int32_t k,
                                                               const isoclust_opts *opts, int32_t *labels,
                                                               uint8_t *residual, double *i_k, void *stream) {
    (void)opts;
    if (!parent || !phi_par || !omega || !labels || !residual || !i_k)
        return fail(ISOCLUST_ERR_INVALID_ARG, "a required pointer is NULL");
    if (n < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "n = %lld must be >= 1", (long long)n);
    if (n > ISOCLUST_NOALLOC_MAX_N)
        return fail(ISOCLUST_ERR_INVALID_ARG,
                    "n = %lld exceeds ISOCLUST_NOALLOC_MAX_N = %d of the allocation-free entry point", (long long)n,
                    ISOCLUST_NOALLOC_MAX_N);
    if (k < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "k = %d must be >= 1", k);
    if (k > n) return fail(ISOCLUST_ERR_K_GT_N, "k = %d exceeds n = %lld", k, (long long)n);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    ISO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEV) return fail(ISOCLUST_ERR_INVALID_ARG, "device %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_na_mu[dev]);

    // Set-up, once per device, with that device current: the device address
    // of the static array (the host-side name is not a device pointer).  This
    // loads the module that holds the array, placing it in device memory.
    if (!g_na_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                        "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_na_ptr[dev] = ptr;
    }

    // Carve the tree-stage scratch out of the static array.
    const int64_t m = n > 1 ? n - 1 : 1;
    Arena A{(char *)g_na_ptr[dev], NOALLOC_BYTES, 0, false};
    TreeScratch TS;
    TS.carve(A, n);
    int32_t *eu = A.take<int32_t>(m);
    int32_t *ev = A.take<int32_t>(m);
    if (A.overflow) return fail(ISOCLUST_ERR_INTERNAL, "static scratch too small for n = %lld", (long long)n);

    // The array keeps the previous call's contents: the status word and
    // counters that must start at zero are cleared here; every other array
    // is fully written before it is read.
    k_na_init<<<1, 1, 0, ISO_S(s)>>>(TS.hostinfo, TS.status);
    k_na_tree_input<<<(unsigned)ceil_div(n, 256), 256, 0, ISO_S(s)>>>(parent, n, TS.hostinfo, TS.status);
    int32_t info[2] = {0, 0};
    uint32_t hst = 0;
    ISO_CUDA(cudaMemcpyAsync(info, TS.hostinfo, sizeof(info), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaMemcpyAsync(&hst, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    if (hst) return map_status(hst, true);
    if (info[0] != 1) return fail(ISOCLUST_ERR_INVALID_ARG, "parent[] has %d roots (need exactly 1)", info[0]);
    if (n > 1) ISO_CUDA(edges_from_parent(TS, parent, n, eu, ev, s));
    ISO_CUDA(orient_tree(TS, eu, ev, n, info[1], parent, s));
    ISO_CUDA(cudaMemcpyAsync(&hst, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    if (hst) return map_status(hst, true);
    ISO_CUDA(tree_search_and_label(TS, phi_par, omega, p, k, labels, residual, i_k, s));
    ISO_CUDA(cudaMemcpyAsync(&hst, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    return map_status(hst, true);
}

// api.cu -- the C ABI (include/isoclust.h): validation, scratch, orchestration.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <vector>
#include <mutex>

#include "common.cuh"
#include "mst.cuh"
#include "tree.cuh"

namespace iso {
cudaError_t weights_launch(const void *X, int64_t n, int32_t d, int dtype, bool fp64_path, double sigma,
                           double alpha, int include_self, const unsigned long long *nnbits, double *omega,
                           double *p, unsigned long long *tile_counts, cudaStream_t s);
size_t weights_sym_bytes(int64_t n, int32_t d);
cudaError_t weights_launch_sym(const float *X, int64_t n, int32_t d, double sigma, int include_self,
                               const unsigned long long *nnbits, double *omega, void *part,
                               unsigned long long *tile_counts, const uint8_t *need, cudaEvent_t *kev,
                               cudaStream_t s, const Shard *sh = nullptr, double *part64 = nullptr,
                               OmegaGram *og = nullptr, uint32_t *status = nullptr, uint64_t wait_cycles = 0);
float omega_zskip(int64_t n);
constexpr size_t SYM_PART_LIMIT = size_t(16) << 30;   // symmetric sweep up to 16 GiB of partials
// the omega Gram goes to the tensor cores by default for rows at least this
// long (measured on GB300: 1.23x faster at d = 64, 1.3x at d = 128, 5x at
// d = 4,096 than the double-word CUDA-core sums)
constexpr int32_t OMEGA_GRAM_MIN_D = 64;
size_t weights_sym_sets_bytes(int64_t n_pad, int64_t nitems, int32_t d);
cudaError_t weights_launch_sym_sets(const float *Xp, int64_t n_pad, int32_t d, double sigma, int include_self,
                                    const unsigned long long *nnbits, double *omega, void *part, const int2 *witems,
                                    int64_t nitems, const int32_t *tile_valid, const int32_t *tile_set,
                                    const int64_t *tile0, const int64_t *ntl, const int64_t *item0, int64_t max_n,
                                    unsigned long long *tile_counts, cudaEvent_t *kev, cudaStream_t s);

size_t adjoint_bytes(int64_t n, int32_t d, int32_t k);
cudaError_t adjoint_launch(const void *X, int32_t dtype, int64_t n, int32_t d, const double *scale, double sigma,
                           const int32_t *parent, const int32_t *labels, int32_t k, const double *phi_par,
                           const double *omega, double grad, double *dX, double *dscale, double *dsigma, double *ik,
                           void *ws, uint32_t *status, cudaEvent_t *kev, cudaStream_t s);
cudaError_t scale_rows_launch(const void *X, int32_t dtype, int64_t n, int32_t d, const double *scale, void *Z,
                              cudaStream_t s);

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = "";
static thread_local double g_prof_ms[6] = {0, 0, 0, 0, 0, 0};
static thread_local int64_t g_prof_cnt[4] = {0, 0, 0, 0};
static thread_local int64_t g_prof_mst_tiles[2] = {0, 0};     // tile pairs swept, and a full sweep's
static thread_local unsigned long long g_prof_tiles[3] = {0, 0, 0};
static thread_local int g_prof_sym = 0;
static thread_local double g_prof_omega_kernel_ms = 0.0;
static thread_local double g_prof_omega_gram_ms = 0.0;
static thread_local int64_t g_prof_omega_gram_blocks = 0;

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

isoclust_status fail(isoclust_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

static thread_local int g_comm_rc = 0;            // a failed all-reduce callback (sharded calls)

isoclust_status cuda_fail(cudaError_t e, const char *what) {
    if (g_comm_rc) {
        const int rc = g_comm_rc;
        g_comm_rc = 0;
        return fail(ISOCLUST_ERR_COMM, "the all-reduce callback returned %d", rc);
    }
    snprintf(g_err, sizeof(g_err), "CUDA error %d (%s) at %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? ISOCLUST_ERR_OOM : ISOCLUST_ERR_CUDA;
}

cudaError_t shard_allreduce(const Shard &sh, void *buf, int64_t count, int32_t op, cudaStream_t s) {
    const cudaError_t pending = cudaGetLastError();     // launches queued before the collective
    if (pending != cudaSuccess) return pending;
    const int32_t rc = sh.fn(sh.ctx, buf, count, op, (void *)s);
    if (rc != 0) {
        g_comm_rc = rc;
        cudaStreamSynchronize(s);         // the call returns with none of its work in flight
        cudaGetLastError();
        return cudaErrorUnknown;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- device info
static std::mutex g_dev_mu;
constexpr int MAX_DEV = 64;
static int g_sms[MAX_DEV] = {0};
static std::mutex g_call_mu[MAX_DEV];
static void *g_scratch[MAX_DEV] = {nullptr};
static size_t g_scratch_cap[MAX_DEV] = {0};

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    return dev < MAX_DEV ? dev : 0;
}

int num_sms() {
    int dev = current_device();
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (g_sms[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        g_sms[dev] = v;
    }
    return g_sms[dev];
}

// Caller holds g_call_mu[dev]; no work from an earlier call is in flight
// (every call synchronises its stream before returning).
void *scratch_acquire(size_t bytes, cudaStream_t stream, isoclust_status *st) {
    (void)stream;
    int dev = current_device();
    if (g_scratch_cap[dev] >= bytes && g_scratch[dev]) return g_scratch[dev];
    if (g_scratch[dev]) {
        cudaDeviceSynchronize();
        cudaFree(g_scratch[dev]);
        g_scratch[dev] = nullptr;
        g_scratch_cap[dev] = 0;
    }
    size_t want = bytes + bytes / 4 + (1u << 20);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *st = fail(ISOCLUST_ERR_OOM, "cannot allocate %zu bytes of device scratch", bytes);
            return nullptr;
        }
        want = bytes;
    }
    g_scratch[dev] = p;
    g_scratch_cap[dev] = want;
    return p;
}

static void *g_gram[MAX_DEV] = {nullptr};
static size_t g_gram_cap[MAX_DEV] = {0};

// Caller holds g_call_mu[dev] (one call per device at a time).
void *gram_acquire(size_t bytes) {
    int dev = current_device();
    if (g_gram_cap[dev] >= bytes && g_gram[dev]) return g_gram[dev];
    if (g_gram[dev]) {
        cudaDeviceSynchronize();
        cudaFree(g_gram[dev]);
        g_gram[dev] = nullptr;
        g_gram_cap[dev] = 0;
    }
    size_t want = bytes + bytes / 8 + (1u << 20);
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        want = bytes;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate %zu bytes for the omega Gram tiles", bytes);
            return nullptr;
        }
    }
    g_gram[dev] = p;
    g_gram_cap[dev] = want;
    return p;
}

void scratch_release() {
    int dev = current_device();
    if (g_scratch[dev]) {
        cudaFree(g_scratch[dev]);
        g_scratch[dev] = nullptr;
        g_scratch_cap[dev] = 0;
    }
}

// ---------------------------------------------------------------- validation kernels
namespace {
constexpr int TPB = 256;

template <class T>
__global__ void k_check_finite(const T *__restrict__ X, int64_t count, uint32_t *st) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite((double)X[i])) bad = true;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(st, DEV_NONFINITE);
}

__global__ void k_tree_input(const int32_t *__restrict__ parent, int64_t n, int32_t *info, uint32_t *st) {
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

__global__ void k_check_edges(const int32_t *counters, int64_t n, uint32_t *st) {
    if (counters[MC_NEDGES] != n - 1 || counters[MC_NCOMP] != 1) atomicOr(st, DEV_EDGE_COUNT);
}

__global__ void k_copy_beta(const SearchState *S, double *beta) { beta[0] = S->beta; }

__global__ void k_or_err_api(const uint32_t *src, uint32_t *dst) {
    if (*src) atomicOr(dst, *src);
}

// Row order of the omega sweep: MST preorder (spatially coherent runs),
// with rows whose nearest neighbour is far (y_nn > 16) moved to the front:
// they need double-word work against most columns, so their CTAs start
// first instead of forming the tail of the grid.
__global__ void k_order_keys(const int32_t *__restrict__ pre, const unsigned long long *__restrict__ nnbits,
                             int64_t n, double inv_sigma, uint64_t *__restrict__ key, int32_t *__restrict__ val) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    double y = sqrt(__longlong_as_double((long long)nnbits[v])) * inv_sigma;
    uint64_t far = (y > 16.0) ? 0ull : 1ull;
    key[v] = (far << 32) | (uint64_t)(uint32_t)pre[v];
    val[v] = (int32_t)v;
}

__global__ void k_gather_rows(const float *__restrict__ X, const int32_t *__restrict__ perm,
                              const unsigned long long *__restrict__ nnbits, int64_t n, int32_t d,
                              float *__restrict__ Xp, unsigned long long *__restrict__ nnp) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * (int64_t)d) return;
    int64_t r = idx / d, t = idx - r * d;
    int64_t src = perm[r];
    Xp[idx] = X[src * d + t];
    if (t == 0) nnp[r] = nnbits[src];
}

__global__ void k_scatter_rows(const double *__restrict__ vp, const int32_t *__restrict__ perm, int64_t n,
                               double *__restrict__ v) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) v[perm[r]] = vp[r];
}
}  // namespace

cudaError_t check_finite(const void *X, int64_t count, int dtype, uint32_t *status, double *absmax, cudaStream_t s) {
    (void)absmax;
    int64_t gb = ceil_div(count, TPB), gmax = (int64_t)num_sms() * 16;
    unsigned g = (unsigned)(gb < gmax ? gb : gmax);
    if (g == 0) g = 1;
    if (dtype == ISOCLUST_F64)
        k_check_finite<double><<<g, TPB, 0, ISO_S(s)>>>((const double *)X, count, status);
    else
        k_check_finite<float><<<g, TPB, 0, ISO_S(s)>>>((const float *)X, count, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- helpers
isoclust_status map_status(uint32_t st, bool user_tree) {
    if (st & DEV_NONFINITE) return fail(ISOCLUST_ERR_NONFINITE, "non-finite value in an input array");
    // a wait that ran out leaves the stages after it without their input:
    // it is reported before anything that follows from it
    if (st & DEV_TIMEOUT) return fail(ISOCLUST_ERR_TIMEOUT, "a bounded device wait ran out");
    if (st & DEV_BAD_TREE)
        return user_tree ? fail(ISOCLUST_ERR_INVALID_ARG, "parent[] does not describe a rooted tree")
                         : fail(ISOCLUST_ERR_INTERNAL, "internal: the spanning tree is malformed");
    if (st & DEV_NEGATIVE)
        return user_tree ? fail(ISOCLUST_ERR_INVALID_ARG, "omega must be > 0, phi and p >= 0")
                         : fail(ISOCLUST_ERR_INTERNAL, "internal: a vertex weight is not positive");
    if (st & DEV_NO_SOLUTION) return fail(ISOCLUST_ERR_NO_SOLUTION, "no finite threshold gives k sets");
    if (st) return fail(ISOCLUST_ERR_INTERNAL, "internal consistency check failed (0x%x)", st);
    return ISOCLUST_OK;
}

static isoclust_opts resolve_opts(const isoclust_opts *o) { return o ? *o : isoclust_opts_default(); }

static isoclust_status check_opts(const isoclust_opts &o, int64_t n, int dtype) {
    if (!(o.alpha >= 0.0) || !isfinite(o.alpha)) return fail(ISOCLUST_ERR_INVALID_ARG, "alpha must be finite and >= 0");
    if (o.omega_mode != ISOCLUST_OMEGA_FULL && o.omega_mode != ISOCLUST_OMEGA_TREE)
        return fail(ISOCLUST_ERR_INVALID_ARG, "unknown omega_mode %d", o.omega_mode);
    if (o.precision < ISOCLUST_PREC_AUTO || o.precision > ISOCLUST_PREC_BF16_TC)
        return fail(ISOCLUST_ERR_INVALID_ARG, "unknown precision %d", o.precision);
    if ((o.precision == ISOCLUST_PREC_FP32 || o.precision == ISOCLUST_PREC_BF16_TC) && dtype != ISOCLUST_F32)
        return fail(ISOCLUST_ERR_INVALID_ARG, "precision FP32 / BF16_TC needs F32 input");
    if (o.root < 0 || o.root >= n) return fail(ISOCLUST_ERR_INVALID_ARG, "root %d out of range", o.root);
    if (o.include_self != 0 && o.include_self != 1) return fail(ISOCLUST_ERR_INVALID_ARG, "include_self must be 0 or 1");
    return ISOCLUST_OK;
}

static isoclust_status check_points(const void *X, int64_t n, int32_t d, int32_t dtype, int64_t min_n) {
    if (!X) return fail(ISOCLUST_ERR_INVALID_ARG, "X is NULL");
    if (n < min_n) return fail(ISOCLUST_ERR_INVALID_ARG, "n = %lld is below %lld", (long long)n, (long long)min_n);
    if (n > 2147483646LL) return fail(ISOCLUST_ERR_INVALID_ARG, "n = %lld is too large", (long long)n);
    if (d < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "d = %d must be >= 1", d);
    if (dtype != ISOCLUST_F32 && dtype != ISOCLUST_F64) return fail(ISOCLUST_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    if ((double)n * (double)d > 9.0e15) return fail(ISOCLUST_ERR_INVALID_ARG, "n*d too large");
    return ISOCLUST_OK;
}

struct Events {
    cudaEvent_t e[12] = {};
    bool ok = false;
    Events() {
        ok = true;
        for (auto &x : e) ok = ok && cudaEventCreate(&x) == cudaSuccess;
    }
    ~Events() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    void rec(int i, cudaStream_t s) {
        if (ok) record_event(e[i], s);
    }
    double ms(int a, int b) {
        float t = 0.f;
        if (!ok) return 0.0;
        if (cudaEventElapsedTime(&t, e[a], e[b]) != cudaSuccess) {
            cudaGetLastError();              // a pair never recorded: no time, no pending error
            return 0.0;
        }
        return (double)t;
    }
};

// ---- CUDA graphs of repeated batched calls.  A batched call whose
// arguments (pointers, sizes, the plan's offsets and ks, sigma, options),
// scratch base and sweep-variant setting all match the previous batched call
// on this device replays the two graphs captured from that call's device
// work (before and after the host check of the trees) instead of launching
// every kernel again.  The first call of a signature runs eagerly (the sweep
// variant is tuned there), the second is captured, later ones replay.  The
// graphs run on a library-owned stream; the call stays synchronous.
// isoclust_set_batched_graphs(0) keeps every call eager.
struct SetsGraph {
    uint64_t key = 0;
    int seen = 0;                                  // consecutive calls with this key
    bool broken = false;                           // capture failed for this key: eager
    cudaGraphExec_t g[2] = {nullptr, nullptr};
    long long nk[2] = {0, 0};                      // kernels in each graph
    Events *ev = nullptr;                          // the events the graphs record
    void reset(uint64_t k) {
        for (auto &x : g)
            if (x) { cudaGraphExecDestroy(x); x = nullptr; }
        delete ev;
        ev = nullptr;
        key = k;
        seen = 0;
        broken = false;
        nk[0] = nk[1] = 0;
    }
};
static SetsGraph g_sets_graph[MAX_DEV];
static cudaStream_t g_graph_stream[MAX_DEV] = {nullptr};
static int g_last_graph_mode = 0;                  // 0 eager, 1 captured, 2 replayed (last batched call)

static std::atomic<int> g_graphs_on{1};          // isoclust_set_batched_graphs
static std::atomic<int> g_stall_test{0};         // isoclust_set_test_stalled_wait
static std::atomic<int> g_omega_gram{-1};        // isoclust_set_omega_gram (-1: by row length)
static bool graphs_enabled() { return g_graphs_on.load(std::memory_order_relaxed) != 0; }

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    }
    template <class T> void val(const T &v) { add(&v, sizeof(v)); }
};

static bool use_fp64_sweep(const isoclust_opts &o, int dtype) {
    if (o.precision == ISOCLUST_PREC_FP64) return true;
    if (o.precision == ISOCLUST_PREC_FP32 || o.precision == ISOCLUST_PREC_BF16_TC) return false;
    return dtype == ISOCLUST_F64;
}

// Tensor-core sweep: requested, or AUTO on F32 input on an sm_103 device.
static isoclust_status use_tc_sweep(const isoclust_opts &o, int dtype, bool *out) {
    *out = false;
    if (dtype != ISOCLUST_F32) return ISOCLUST_OK;
    if (o.precision == ISOCLUST_PREC_BF16_TC) {
        if (!tc_supported()) return fail(ISOCLUST_ERR_INVALID_ARG, "precision BF16_TC needs an sm_103 device");
        *out = true;
    } else if (o.precision == ISOCLUST_PREC_AUTO) {
        *out = tc_supported();
    }
    return ISOCLUST_OK;
}

// ---------------------------------------------------------------- the pipeline
static isoclust_status cluster_impl(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t k, double sigma,
                                    const isoclust_opts *opts_in, int32_t *labels, uint8_t *residual, double *i_k,
                                    int32_t *out_parent, double *out_phi, double *out_omega, double *out_p,
                                    double *out_beta, int32_t *out_eu, int32_t *out_ev, double *out_ed2,
                                    cudaStream_t s, bool need_labels, const Shard *sh = nullptr) {
    isoclust_status st;
    g_comm_rc = 0;
    if ((st = check_points(X, n, d, dtype, 2))) return st;
    isoclust_opts o = resolve_opts(opts_in);
    if ((st = check_opts(o, n, dtype))) return st;
    if (need_labels) {
        if (!labels || !residual || !i_k) return fail(ISOCLUST_ERR_INVALID_ARG, "labels, residual and i_k are required");
        if (k < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "k = %d must be >= 1", k);
        if (k > n) return fail(ISOCLUST_ERR_K_GT_N, "k = %d exceeds n = %lld", k, (long long)n);
        if (!(sigma > 0.0) || !isfinite(sigma)) return fail(ISOCLUST_ERR_INVALID_ARG, "sigma must be finite and > 0");
    }
    const bool fp64_sweep = use_fp64_sweep(o, dtype);
    const int splits = mst_splits(n);
    bool use_tc = false;
    if ((st = use_tc_sweep(o, dtype, &use_tc))) return st;
    TcScratch TC;
    TC.wait_cycles = o.spin_limit;
    TC.stall_test = g_stall_test.load(std::memory_order_relaxed);
    const int tsplits = use_tc ? tc_splits(n) : 1;
    if (sh) {
        // the sharded work: the tensor-core sweep and the symmetric omega sweep
        if (!use_tc || fp64_sweep || o.alpha != 0.0 || o.omega_mode != ISOCLUST_OMEGA_FULL || !need_labels ||
            weights_sym_bytes(n, d) > SYM_PART_LIMIT)
            return fail(ISOCLUST_ERR_INVALID_ARG, "a sharded call needs F32 input on an sm_103 device, alpha = 0, "
                                                  "full-graph omega and precision AUTO or BF16_TC");
        TC.shard_rank = sh->rank;
        TC.shard_world = sh->world;
    }
    // pruned Boruvka rounds (one set, not sharded); their candidate lists
    // (2 per slot) are all written by the first, full round too, which then
    // sweeps PRUNE_SLOTS column splits
    // (the order's kernels read rows by 16 bytes)
    TC.prune = use_tc && !sh && prune_wanted(n, d) && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    const int tlists = TC.prune ? 2 * PRUNE_SLOTS : 0;
    const int tsplits_used = TC.prune ? PRUNE_SLOTS : tsplits;

    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_call_mu[dev]);

    // scratch layout (measured, then carved)
    struct Perm {
        int32_t *perm = nullptr, *vbuf = nullptr;
        uint64_t *key = nullptr, *kbuf = nullptr;
        float *Xp = nullptr;
        unsigned long long *nnp = nullptr, *tiles = nullptr;
        double *omp = nullptr, *pp = nullptr;
        void *sym = nullptr;
        uint8_t *need = nullptr;
        double *part64 = nullptr;
        void *gram = nullptr;
    } P;
    const bool permuted = need_labels && dtype == ISOCLUST_F32 && !fp64_sweep;
    const bool symmetric = permuted && o.alpha == 0.0 && o.omega_mode == ISOCLUST_OMEGA_FULL &&
                           weights_sym_bytes(n, d) <= SYM_PART_LIMIT;
    // eq. omega's Gram on the tensor cores (with the tensor-core screen)
    int64_t gram_blocks = 0;
    const int gram_mode = g_omega_gram.load(std::memory_order_relaxed);
    const bool gram = symmetric && use_tc && ceil_div(n, 128) <= 65535 &&
                      (gram_mode == 1 || (gram_mode < 0 && d >= OMEGA_GRAM_MIN_D));
    auto carve = [&](Arena &A, MstScratch &M, TreeScratch &TS, double **phi, double **om, double **pp, double **omtmp,
                     uint32_t **status) {
        *status = A.take<uint32_t>(4);
        M.carve(A, n, splits);
        if (use_tc) TC.carve(A, n, d, tsplits_used, 0, 1, tlists);
        if (need_labels) {
            TS.carve(A, n);
            *phi = A.take<double>(n);
            *om = A.take<double>(n);
            *pp = A.take<double>(n);
            *omtmp = A.take<double>(n);
        }
        if (permuted) {
            P.perm = A.take<int32_t>(n);
            P.vbuf = A.take<int32_t>(n);
            P.key = A.take<uint64_t>(n);
            P.kbuf = A.take<uint64_t>(n);
            P.Xp = A.take<float>((size_t)n * d);
            P.nnp = A.take<unsigned long long>(n);
            P.tiles = A.take<unsigned long long>(3);
            P.omp = A.take<double>(n);
            P.pp = A.take<double>(n);
            if (symmetric) P.sym = (void *)A.take<unsigned char>(weights_sym_bytes(n, d));
            if (symmetric && use_tc) P.need = A.take<uint8_t>((size_t)ceil_div(n, 64) * ceil_div(n, 64));
            if (sh) P.part64 = A.take<double>(n);
            if (gram) P.gram = (void *)A.take<unsigned char>(omega_gram_bytes(n, d), 1024);
        }
    };
    MstScratch M;
    TreeScratch TS;
    double *phi = nullptr, *om = nullptr, *pp = nullptr, *omtmp = nullptr;
    uint32_t *status = nullptr;
    Arena meas;
    carve(meas, M, TS, &phi, &om, &pp, &omtmp, &status);
    void *base = scratch_acquire(meas.off, s, &st);
    if (!base) return st;
    Arena A{(char *)base, meas.off + 4096, 0, false};
    carve(A, M, TS, &phi, &om, &pp, &omtmp, &status);
    if (A.overflow) return fail(ISOCLUST_ERR_INTERNAL, "scratch carve overflow");
    if (out_phi) phi = out_phi;
    if (out_omega) om = out_omega;
    if (out_p) pp = out_p;

    Events ev;
    ev.rec(0, s);
    ISO_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t) * 4, s));
    if (need_labels) ISO_CUDA(cudaMemsetAsync(TS.status, 0, sizeof(uint32_t), s));
    ISO_CUDA(check_finite(X, n * (int64_t)d, dtype, status, nullptr, s));
    uint32_t hst = 0;
    ISO_CUDA(cudaMemcpyAsync(&hst, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    if (hst) return map_status(hst, false);
    ev.rec(1, s);

    // Section 2.2 steps 1-2: minimum spanning tree
    ISO_CUDA(mst_build(M, X, n, d, dtype, fp64_sweep, status, s, use_tc ? &TC : nullptr, 1, 0, sh));
    const bool mst_pruned = TC.prune && TC.prune_ready;     // (the omega screen re-prepares TC later)
    unsigned long long mst_swept = 0;
    if (mst_pruned) {
        ISO_CUDA(cudaMemcpyAsync(&mst_swept, TC.swept, sizeof(mst_swept), cudaMemcpyDeviceToHost, s));
        ISO_CUDA(cudaStreamSynchronize(s));
    }
    k_check_edges<<<1, 1, 0, ISO_S(s)>>>(M.counters, n, status);
    if (out_eu || out_ev || out_ed2) {
        if (!(out_eu && out_ev && out_ed2)) return fail(ISOCLUST_ERR_INVALID_ARG, "edge outputs must be all or none");
        ISO_CUDA(mst_sort_edges(M, out_eu, out_ev, out_ed2, s));
    }
    ev.rec(2, s);

    if (need_labels) {
        // the tree is complete (no wait ran out, n - 1 edges) before anything walks it
        {
            uint32_t h1 = 0;
            ISO_CUDA(cudaMemcpyAsync(&h1, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            ISO_CUDA(cudaStreamSynchronize(s));
            if (h1) return map_status(h1, false);
        }
        // Section 2.2 step 3: root the tree, BFS order
        ISO_CUDA(orient_tree(TS, M.eu, M.ev, n, o.root, nullptr, s));
        {
            uint32_t h2 = 0;
            ISO_CUDA(cudaMemcpyAsync(&h2, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            ISO_CUDA(cudaStreamSynchronize(s));
            uint32_t h3 = 0;
            ISO_CUDA(cudaMemcpy(&h3, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
            if (h2 | h3) return map_status(h2 | h3, false);
        }
        ev.rec(3, s);
        // eq. omega / eq. potential
        const bool full = o.omega_mode == ISOCLUST_OMEGA_FULL;
        if (full || o.alpha != 0.0) {
            ISO_CUDA(nn_from_edges(M, M.eu, M.ev, M.ed2, s));
            double *om_out = full ? om : omtmp;
            if (permuted) {
                const unsigned gb = (unsigned)ceil_div(n, TPB);
                k_order_keys<<<gb, TPB, 0, ISO_S(s)>>>(TS.T.pre, M.nnbits, n, 1.0 / sigma, P.key, P.perm);
                ISO_CUDA(sort_pairs_u64(P.key, P.perm, P.kbuf, P.vbuf, n, s));
                k_gather_rows<<<(unsigned)ceil_div(n * (int64_t)d, TPB), TPB, 0, ISO_S(s)>>>(
                    (const float *)X, P.perm, M.nnbits, n, d, P.Xp, P.nnp);
                ISO_CUDA(cudaMemsetAsync(P.tiles, 0, 3 * sizeof(unsigned long long), s));
                if (symmetric) {
                    // the tensor cores decide which pairs of 64-row tiles can hold a term
                    if (use_tc) {
                        ISO_CUDA(tc_omega_screen(TC, P.Xp, n, d, P.nnp, sigma, (double)omega_zskip(n), P.need,
                                                 ceil_div(n, 64), s));
                        k_or_err_api<<<1, 1, 0, ISO_S(s)>>>(TC.err, status);
                    }
                    OmegaGram og;
                    og.scratch = P.gram;
                    og.scratch_bytes = gram ? omega_gram_bytes(n, d) : 0;
                    ISO_CUDA(weights_launch_sym(P.Xp, n, d, sigma, o.include_self, P.nnp, P.omp, P.sym, P.tiles,
                                                use_tc ? P.need : nullptr, ev.ok ? ev.e + 8 : nullptr, s, sh,
                                                P.part64, gram ? &og : nullptr, status, o.spin_limit));
                    gram_blocks = og.nblocks;
                }
                else
                    ISO_CUDA(weights_launch(P.Xp, n, d, dtype, false, sigma, o.alpha, o.include_self, P.nnp, P.omp,
                                            P.pp, P.tiles, s));
                k_scatter_rows<<<gb, TPB, 0, ISO_S(s)>>>(P.omp, P.perm, n, om_out);
                if (symmetric)
                    ISO_CUDA(cudaMemsetAsync(pp, 0, sizeof(double) * n, s));
                else
                    k_scatter_rows<<<gb, TPB, 0, ISO_S(s)>>>(P.pp, P.perm, n, pp);
            } else {
                ISO_CUDA(weights_launch(X, n, d, dtype, false, sigma, o.alpha, o.include_self, M.nnbits, om_out, pp,
                                        nullptr, s));
            }
        }
        ev.rec(4, s);
        ISO_CUDA(phi_from_edges(TS, M.ed2, sigma, phi, s));
        if (!full) ISO_CUDA(omega_tree_mode(TS, phi, o.include_self, om, s));
        // Algorithm 2 (search) + Algorithm 1, then Algorithm 4's labels
        ISO_CUDA(tree_search_and_label(TS, phi, om, o.alpha != 0.0 ? pp : nullptr, k, labels, residual, i_k, s));
        ev.rec(5, s);
        if (out_parent) ISO_CUDA(cudaMemcpyAsync(out_parent, TS.T.parent, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        if (out_beta) k_copy_beta<<<1, 1, 0, ISO_S(s)>>>(TS.search, out_beta);
        if (out_p && o.alpha == 0.0) ISO_CUDA(cudaMemsetAsync(out_p, 0, sizeof(double) * n, s));
    } else {
        ev.rec(3, s);
        ev.rec(4, s);
        ev.rec(5, s);
    }
    ev.rec(6, s);
    ISO_CUDA(cudaGetLastError());
    ISO_CUDA(cudaStreamSynchronize(s));
    uint32_t fin = 0;
    ISO_CUDA(cudaMemcpy(&fin, status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    int32_t cnt[8] = {0};
    ISO_CUDA(cudaMemcpy(cnt, M.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    SearchState ss;
    memset(&ss, 0, sizeof(ss));
    if (need_labels) {
        uint32_t tf = 0;
        ISO_CUDA(cudaMemcpy(&tf, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        fin |= tf;
        ISO_CUDA(cudaMemcpy(&ss, TS.search, sizeof(ss), cudaMemcpyDeviceToHost));
    }
    g_prof_ms[0] = ev.ms(0, 1);
    g_prof_ms[1] = ev.ms(3, 4);
    g_prof_ms[2] = ev.ms(1, 2);
    g_prof_ms[3] = ev.ms(2, 3);
    g_prof_ms[4] = ev.ms(4, 5);
    g_prof_ms[5] = ev.ms(5, 6);
    g_prof_cnt[0] = cnt[MC_ROUNDS];
    g_prof_cnt[1] = cnt[MC_OVF_TOTAL] + cnt[MC_OVERFLOW];
    g_prof_cnt[2] = ss.passes + (need_labels ? 1 : 0);
    g_prof_cnt[3] = ss.max_depth;
    g_prof_mst_tiles[0] = g_prof_mst_tiles[1] = 0;
    if (use_tc) {
        const int64_t nt = TC.n_pad / 128;
        g_prof_mst_tiles[1] = (int64_t)cnt[MC_ROUNDS] * nt * nt;
        g_prof_mst_tiles[0] = g_prof_mst_tiles[1];
        if (mst_pruned) g_prof_mst_tiles[0] = (int64_t)mst_swept;     // every round pruned
    }
    g_prof_tiles[0] = g_prof_tiles[1] = g_prof_tiles[2] = 0;
    if (permuted) ISO_CUDA(cudaMemcpy(g_prof_tiles, P.tiles, sizeof(g_prof_tiles), cudaMemcpyDeviceToHost));
    g_prof_sym = symmetric ? (gram ? 3 : (use_tc ? 2 : 1)) : 0;
    // the symmetric sweep kernel (after the Gram kernel when that ran), and the Gram kernel
    g_prof_omega_kernel_ms = symmetric ? (gram ? ev.ms(11, 9) : ev.ms(8, 9)) : 0.0;
    g_prof_omega_gram_ms = (symmetric && gram) ? ev.ms(10, 11) : 0.0;
    g_prof_omega_gram_blocks = (symmetric && gram) ? gram_blocks : 0;
    return map_status(fin, false);
}

// ---------------------------------------------------------------- independent sets
namespace {
// upper bound search: the b with base[b] <= w < base[b + 1]
__device__ __forceinline__ int32_t find_set(const int64_t *__restrict__ base, int32_t nsets, int64_t w) {
    int32_t lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (base[mid] <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_set_of(const int64_t *__restrict__ offs, int32_t *__restrict__ set_of) {
    const int32_t b = blockIdx.x;
    for (int64_t v = offs[b] + threadIdx.x; v < offs[b + 1]; v += blockDim.x) set_of[v] = b;
}

// tensor-core sweep items: set b's row tiles against the set's column tiles
__global__ void k_tc_items(const int64_t *__restrict__ tcbase, const int64_t *__restrict__ rowbase, int32_t nsets,
                           int4 *__restrict__ items) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= tcbase[nsets]) return;
    const int32_t b = find_set(tcbase, nsets, w);
    const int32_t t0 = (int32_t)(rowbase[b] / 128), nt = (int32_t)(tcbase[b + 1] - tcbase[b]);
    items[w] = make_int4(t0 + (int32_t)(w - tcbase[b]), t0, t0 + nt, b << 4);   // list pair 0, set b
}

// omega items: the upper triangle of set b's 64-row tile grid, row-major
__global__ void k_omega_items(const int64_t *__restrict__ item0, const int64_t *__restrict__ tile0,
                              const int64_t *__restrict__ ntl, int32_t nsets, int2 *__restrict__ items) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= item0[nsets]) return;
    const int32_t b = find_set(item0, nsets, w);
    const int64_t T = ntl[b], q = w - item0[b];
    int64_t i = 0;
    while ((i + 1) * T - (i + 1) * i / 2 <= q) ++i;     // at most T steps (T <= max set / 64)
    const int64_t j = i + (q - (i * T - i * (i - 1) / 2));
    items[w] = make_int2((int32_t)(tile0[b] + i), (int32_t)(tile0[b] + j));
}

__global__ void k_omega_tiles(const int64_t *__restrict__ tile0, const int64_t *__restrict__ offs, int32_t nsets,
                              int64_t ntiles, int32_t *__restrict__ tile_valid, int32_t *__restrict__ tile_set) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int32_t b = find_set(tile0, nsets, t);
    const int64_t nb = offs[b + 1] - offs[b], lo = (t - tile0[b]) * 64;
    const int64_t left = nb - lo;
    tile_valid[t] = (int32_t)(left < 64 ? (left > 0 ? left : 0) : 64);
    tile_set[t] = b;
}

// the forest's edges plus one virtual edge (nv, first point of b) per set
__global__ void k_virtual_edges(const int64_t *__restrict__ offs, int32_t nsets, int64_t m_mst, int64_t nv,
                                int32_t *__restrict__ eu, int32_t *__restrict__ ev, double *__restrict__ ed2) {
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsets) return;
    eu[m_mst + b] = (int32_t)nv;
    ev[m_mst + b] = (int32_t)offs[b];
    ed2[m_mst + b] = 0.0;
}

__global__ void k_check_edges_sets(const int32_t *counters, int64_t n, int32_t nsets, uint32_t *st) {
    if (counters[MC_NEDGES] != n - nsets || counters[MC_NCOMP] != nsets) atomicOr(st, DEV_EDGE_COUNT);
}

// padded omega row of point v: its set's first tile, plus its preorder rank
// inside the set (the sets' subtrees are consecutive in the preorder)
__global__ void k_pos64(const int32_t *__restrict__ pre, const int32_t *__restrict__ set_of,
                        const int64_t *__restrict__ offs, const int64_t *__restrict__ tile0, int64_t n,
                        int64_t *__restrict__ pos) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t b = set_of[v];
    pos[v] = tile0[b] * 64 + (int64_t)(pre[v] - pre[offs[b]]);
}

__global__ void k_gather_pad(const float *__restrict__ X, const int64_t *__restrict__ pos,
                             const unsigned long long *__restrict__ nnbits, int64_t n, int32_t d,
                             float *__restrict__ Xp, unsigned long long *__restrict__ nnp) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * (int64_t)d) return;
    const int64_t v = idx / d, t = idx - v * d;
    const int64_t r = pos[v];
    Xp[r * d + t] = X[idx];
    if (t == 0) nnp[r] = nnbits[v];
}

__global__ void k_scatter_pad(const double *__restrict__ omp, const int64_t *__restrict__ pos, int64_t n,
                              double *__restrict__ om) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) om[v] = omp[pos[v]];
    if (v == n) om[n] = 1.0;         // the virtual root (never read)
}
}  // namespace

static isoclust_status cluster_sets_impl(const void *X, const int64_t *offsets, int32_t nsets, int32_t d,
                                         int32_t dtype, const int32_t *ks, double sigma, const isoclust_opts *opts_in,
                                         int32_t *labels, uint8_t *residual, double *i_k, double *beta,
                                         int32_t *out_parent, double *out_phi, double *out_omega, cudaStream_t s) {
    if (!X || !offsets || !ks || !labels || !residual || !i_k)
        return fail(ISOCLUST_ERR_INVALID_ARG, "a required pointer is NULL");
    if (nsets < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "nsets = %d must be >= 1", nsets);
    if (dtype != ISOCLUST_F32) return fail(ISOCLUST_ERR_INVALID_ARG, "independent sets need F32 input");
    if (d < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "d = %d must be >= 1", d);
    if (!(sigma > 0.0) || !isfinite(sigma)) return fail(ISOCLUST_ERR_INVALID_ARG, "sigma must be finite and > 0");
    if (offsets[0] != 0) return fail(ISOCLUST_ERR_INVALID_ARG, "offsets[0] must be 0");
    int64_t max_n = 0;
    for (int32_t b = 0; b < nsets; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        if (nb < 2) return fail(ISOCLUST_ERR_INVALID_ARG, "set %d has %lld points (need >= 2)", b, (long long)nb);
        if (ks[b] < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "ks[%d] = %d must be >= 1", b, ks[b]);
        if (ks[b] > nb) return fail(ISOCLUST_ERR_K_GT_N, "ks[%d] = %d exceeds the set's %lld points", b, ks[b], (long long)nb);
        if (nb > max_n) max_n = nb;
    }
    const int64_t N = offsets[nsets];
    isoclust_status st;
    if ((st = check_points(X, N, d, dtype, 2))) return st;
    isoclust_opts o = resolve_opts(opts_in);
    if ((st = check_opts(o, N, dtype))) return st;
    if (o.alpha != 0.0 || o.omega_mode != ISOCLUST_OMEGA_FULL || o.root != 0 ||
        (o.precision != ISOCLUST_PREC_AUTO && o.precision != ISOCLUST_PREC_BF16_TC))
        return fail(ISOCLUST_ERR_INVALID_ARG,
                    "independent sets support alpha = 0, omega_mode FULL, root 0 and precision AUTO / BF16_TC");
    if (!tc_supported()) return fail(ISOCLUST_ERR_INVALID_ARG, "independent sets need an sm_103 device");

    // ---- plan (host): per-set tile runs of the two padded row spaces
    const int64_t P = nsets;
    std::vector<int64_t> plan((size_t)(6 * P + 3));
    int64_t *h_offs = plan.data();                  // [P + 1]
    int64_t *h_rowbase = h_offs + (P + 1);          // [P]      first 128-row of each set (TC sweep)
    int64_t *h_tcbase = h_rowbase + P;              // [P + 1]  first sweep item of each set
    int64_t *h_tile0 = h_tcbase + (P + 1);          // [P]      first 64-row tile of each set (omega)
    int64_t *h_ntl = h_tile0 + P;                   // [P]      64-row tiles of each set
    int64_t *h_item0 = h_ntl + P;                   // [P + 1]  first omega item of each set
    int64_t rb = 0, tc = 0, t64 = 0, it = 0;
    for (int32_t b = 0; b < nsets; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        h_offs[b] = offsets[b];
        h_rowbase[b] = rb;
        h_tcbase[b] = tc;
        const int64_t t128 = ceil_div(nb, 128);
        rb += t128 * 128;
        tc += t128;
        const int64_t T = ceil_div(nb, 64);
        h_tile0[b] = t64;
        h_ntl[b] = T;
        h_item0[b] = it;
        t64 += T;
        it += T * (T + 1) / 2;
    }
    h_offs[P] = N;
    h_tcbase[P] = tc;
    h_item0[P] = it;
    const int64_t n_pad128 = rb, ntc = tc, n_pad64 = t64 * 64, ntile64 = t64, nitems = it;
    // the sweep addresses padded rows with 32-bit column indices
    if (n_pad128 > 2147483648LL)
        return fail(ISOCLUST_ERR_INVALID_ARG, "the sets' padded rows (%lld) exceed 2^31", (long long)n_pad128);

    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_call_mu[dev]);
    MstScratch M;
    TcScratch TC;
    TreeScratch TS;
    struct {
        uint32_t *status;
        int64_t *plan;
        int32_t *ks, *set_of, *eu, *ev, *tile_valid, *tile_set;
        int4 *titems;
        int2 *witems;
        double *ed2, *phi, *om, *omp;
        SearchState *SS;
        uint32_t *set_hist;
        int64_t *pos;
        float *Xp;
        unsigned long long *nnp, *tiles;
        void *sym;
    } B;
    auto carve = [&](Arena &A) {
        B.status = A.take<uint32_t>(4);
        B.plan = A.take<int64_t>(plan.size());
        B.ks = A.take<int32_t>(P);
        B.set_of = A.take<int32_t>(N);
        B.titems = A.take<int4>(ntc);
        B.witems = A.take<int2>(nitems > 0 ? nitems : 1);
        B.tile_valid = A.take<int32_t>(ntile64);
        B.tile_set = A.take<int32_t>(ntile64);
        M.carve(A, N, 1);
        TC.carve(A, N, d, 1, n_pad128, nsets, 2);
        TS.carve(A, N + 1);
        B.eu = A.take<int32_t>(N);
        B.ev = A.take<int32_t>(N);
        B.ed2 = A.take<double>(N);
        B.phi = A.take<double>(N + 1);
        B.om = A.take<double>(N + 1);
        B.SS = A.take<SearchState>(P);
        B.set_hist = A.take<uint32_t>((size_t)P * CAND_SET_BUCKETS + 1);
        B.pos = A.take<int64_t>(N);
        B.Xp = A.take<float>((size_t)n_pad64 * d);
        B.nnp = A.take<unsigned long long>(n_pad64);
        B.omp = A.take<double>(n_pad64);
        B.tiles = A.take<unsigned long long>(3);
        B.sym = (void *)A.take<unsigned char>(weights_sym_sets_bytes(n_pad64, nitems, d));
    };
    Arena meas;
    carve(meas);
    void *base = scratch_acquire(meas.off, s, &st);
    if (!base) return st;
    Arena A{(char *)base, meas.off + 4096, 0, false};
    carve(A);
    if (A.overflow) return fail(ISOCLUST_ERR_INTERNAL, "scratch carve overflow");
    const int64_t *d_offs = B.plan, *d_rowbase = d_offs + (P + 1), *d_tcbase = d_rowbase + P;
    const int64_t *d_tile0 = d_tcbase + (P + 1), *d_ntl = d_tile0 + P, *d_item0 = d_ntl + P;

    TC.wait_cycles = o.spin_limit;
    TC.stall_test = g_stall_test.load(std::memory_order_relaxed);
    Events ev;
    ev.rec(0, s);
    ISO_CUDA(cudaMemcpyAsync(B.plan, plan.data(), plan.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    ISO_CUDA(cudaMemcpyAsync(B.ks, ks, (size_t)P * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    ISO_CUDA(cudaMemsetAsync(B.status, 0, sizeof(uint32_t) * 4, s));
    ISO_CUDA(cudaMemsetAsync(TS.status, 0, sizeof(uint32_t), s));
    ISO_CUDA(check_finite(X, N * (int64_t)d, dtype, B.status, nullptr, s));
    k_set_of<<<(unsigned)P, 256, 0, ISO_S(s)>>>(d_offs, B.set_of);
    k_tc_items<<<(unsigned)ceil_div(ntc, TPB), TPB, 0, ISO_S(s)>>>(d_tcbase, d_rowbase, nsets, B.titems);
    if (nitems > 0)
        k_omega_items<<<(unsigned)ceil_div(nitems, TPB), TPB, 0, ISO_S(s)>>>(d_item0, d_tile0, d_ntl, nsets, B.witems);
    k_omega_tiles<<<(unsigned)ceil_div(ntile64, TPB), TPB, 0, ISO_S(s)>>>(d_tile0, d_offs, nsets, ntile64,
                                                                          B.tile_valid, B.tile_set);
    uint32_t hst = 0;
    ISO_CUDA(cudaMemcpyAsync(&hst, B.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));       // also retires the pageable plan upload
    if (hst) return map_status(hst, false);
    ev.rec(1, s);

    // Section 2.2 steps 1-3 up to the host check of the trees (phase 0),
    // then steps 3-4 and Algorithms 1, 2 and 4 (phase 1)
    const bool mid_check = o.spin_limit != 0 || TC.stall_test != 0;
    auto phase0 = [&](cudaStream_t q, Events &E) -> cudaError_t {
        cudaError_t e;
        E.rec(1, q);
        // one Boruvka forest for every set
        TC.items = B.titems;
        TC.nitems = ntc;
        TC.nsets = nsets;
        TC.set_of = B.set_of;
        TC.offs = d_offs;
        TC.rowbase = d_rowbase;
        if ((e = mst_build(M, X, N, d, dtype, false, B.status, q, &TC, nsets, max_n))) return e;
        k_check_edges_sets<<<1, 1, 0, ISO_S(q)>>>(M.counters, N, nsets, B.status);
        E.rec(2, q);
        if (mid_check) {
            // a caller's spin limit can run out: the forest is checked before
            // anything walks it (kernel by kernel only, no graphs then)
            uint32_t h1 = 0;
            if ((e = cudaMemcpyAsync(&h1, B.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, q))) return e;
            if ((e = cudaStreamSynchronize(q))) return e;
            if (h1) return cudaSuccess;            // the host check after this phase reports it
        }
        // the sets' trees under a virtual root (vertex N)
        const int64_t m_mst = N - nsets;
        if ((e = cudaMemcpyAsync(B.eu, M.eu, sizeof(int32_t) * m_mst, cudaMemcpyDeviceToDevice, q))) return e;
        if ((e = cudaMemcpyAsync(B.ev, M.ev, sizeof(int32_t) * m_mst, cudaMemcpyDeviceToDevice, q))) return e;
        if ((e = cudaMemcpyAsync(B.ed2, M.ed2, sizeof(double) * m_mst, cudaMemcpyDeviceToDevice, q))) return e;
        k_virtual_edges<<<(unsigned)ceil_div(P, TPB), TPB, 0, ISO_S(q)>>>(d_offs, nsets, m_mst, N, B.eu, B.ev, B.ed2);
        return orient_tree(TS, B.eu, B.ev, N + 1, (int32_t)N, nullptr, q, B.set_of, 1);
    };
    auto phase1 = [&](cudaStream_t q, Events &E) -> cudaError_t {
        cudaError_t e;
        const int64_t m_mst = N - nsets;
        if ((e = orient_tree(TS, B.eu, B.ev, N + 1, (int32_t)N, nullptr, q, B.set_of, 2))) return e;
        if ((e = fix_set_roots(TS, nsets, d_offs, q))) return e;
        E.rec(3, q);
        // eq. omega per set, symmetric tile pairs in each set's MST preorder
        if ((e = nn_from_edges(M, M.eu, M.ev, M.ed2, q, m_mst))) return e;
        k_pos64<<<(unsigned)ceil_div(N, TPB), TPB, 0, ISO_S(q)>>>(TS.T.pre, B.set_of, d_offs, d_tile0, N, B.pos);
        if ((e = cudaMemsetAsync(B.nnp, 0xff, sizeof(unsigned long long) * n_pad64, q))) return e;
        k_gather_pad<<<(unsigned)ceil_div(N * (int64_t)d, TPB), TPB, 0, ISO_S(q)>>>((const float *)X, B.pos, M.nnbits, N,
                                                                                    d, B.Xp, B.nnp);
        if ((e = cudaMemsetAsync(B.tiles, 0, 3 * sizeof(unsigned long long), q))) return e;
        if ((e = weights_launch_sym_sets(B.Xp, n_pad64, d, sigma, o.include_self, B.nnp, B.omp, B.sym, B.witems,
                                         nitems, B.tile_valid, B.tile_set, d_tile0, d_ntl, d_item0, max_n, B.tiles,
                                         E.ok ? E.e + 8 : nullptr, q)))
            return e;
        k_scatter_pad<<<(unsigned)ceil_div(N + 1, TPB), TPB, 0, ISO_S(q)>>>(B.omp, B.pos, N, B.om);
        E.rec(4, q);
        if ((e = phi_from_edges(TS, B.ed2, sigma, B.phi, q))) return e;
        // Algorithm 2 + Algorithm 1 per set, then Algorithm 4's labels
        if ((e = tree_search_and_label_sets(TS, nsets, d_offs, B.set_of, B.ks, B.SS, B.set_hist, B.phi, B.om, nullptr, labels,
                                            residual, i_k, beta, q)))
            return e;
        E.rec(5, q);
        if (out_parent &&
            (e = cudaMemcpyAsync(out_parent, TS.T.parent, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, q)))
            return e;
        if (out_phi && (e = cudaMemcpyAsync(out_phi, B.phi, sizeof(double) * N, cudaMemcpyDeviceToDevice, q)))
            return e;
        if (out_omega && (e = cudaMemcpyAsync(out_omega, B.om, sizeof(double) * N, cudaMemcpyDeviceToDevice, q)))
            return e;
        E.rec(6, q);
        return cudaGetLastError();
    };

    SetsGraph &G = g_sets_graph[dev];
    bool replay = false, capture = false;
    if (graphs_enabled() && !mid_check) {
        Fnv f;
        f.val(X); f.val(N); f.val(d); f.val(dtype); f.val(nsets); f.val(sigma);
        f.val(o.alpha); f.val(o.omega_mode); f.val(o.precision); f.val(o.root); f.val(o.include_self);
        f.add(offsets, sizeof(int64_t) * (size_t)(P + 1));
        f.add(ks, sizeof(int32_t) * (size_t)P);
        f.val(labels); f.val(residual); f.val(i_k); f.val(beta);
        f.val(out_parent); f.val(out_phi); f.val(out_omega);
        f.val(base); f.val(meas.off);
        const int fv = tc_forced_variant();
        f.val(fv);
        if (G.key != f.h) G.reset(f.h);
        ++G.seen;
        replay = !G.broken && G.g[0] && G.g[1];
        capture = !G.broken && !replay && G.seen >= 2;
        if ((replay || capture) && !g_graph_stream[dev] &&
            cudaStreamCreateWithFlags(&g_graph_stream[dev], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            replay = capture = false;
        }
        if ((replay || capture) && !G.ev) G.ev = new Events;
    }
    cudaStream_t q = (replay || capture) ? g_graph_stream[dev] : s;
    Events &E = (replay || capture) ? *G.ev : ev;
    for (int ph = 0; ph < 2; ++ph) {
        if (replay) {
            ISO_CUDA(cudaGraphLaunch(G.g[ph], q));
            note_launches(G.nk[ph]);
        } else if (capture && !G.broken) {
            const long long c0 = g_launches.load();
            ISO_CUDA(cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = ph == 0 ? phase0(q, E) : phase1(q, E);
            cudaGraph_t graph = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(q, &graph);
            if (e == cudaSuccess) e = ee;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&G.g[ph], graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e == cudaSuccess) {
                G.nk[ph] = g_launches.load() - c0;
                ISO_CUDA(cudaGraphLaunch(G.g[ph], q));
            } else {
                // not capturable: this call from here on, and later calls
                // with this signature, run kernel by kernel
                cudaGetLastError();
                G.broken = true;
                ISO_CUDA(ph == 0 ? phase0(q, E) : phase1(q, E));
            }
        } else {
            ISO_CUDA(ph == 0 ? phase0(q, E) : phase1(q, E));
        }
        if (ph == 0) {
            // the trees are checked before anything walks them
            uint32_t h2 = 0, h3 = 0;
            ISO_CUDA(cudaMemcpyAsync(&h2, B.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, q));
            ISO_CUDA(cudaMemcpyAsync(&h3, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, q));
            ISO_CUDA(cudaStreamSynchronize(q));
            if (h2 | h3) return map_status(h2 | h3, false);
        }
    }
    g_last_graph_mode = replay ? 2 : (capture && !G.broken ? 1 : 0);
    ISO_CUDA(cudaGetLastError());
    ISO_CUDA(cudaStreamSynchronize(q));
    uint32_t fin = 0, tf = 0;
    ISO_CUDA(cudaMemcpy(&fin, B.status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    ISO_CUDA(cudaMemcpy(&tf, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    fin |= tf;
    int32_t cnt[8] = {0};
    ISO_CUDA(cudaMemcpy(cnt, M.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    g_prof_ms[0] = ev.ms(0, 1);
    g_prof_ms[1] = E.ms(3, 4);
    g_prof_ms[2] = E.ms(1, 2);
    g_prof_ms[3] = E.ms(2, 3);
    g_prof_ms[4] = E.ms(4, 5);
    g_prof_ms[5] = E.ms(5, 6);
    g_prof_cnt[0] = cnt[MC_ROUNDS];
    g_prof_cnt[1] = cnt[MC_OVF_TOTAL] + cnt[MC_OVERFLOW];
    g_prof_cnt[2] = DP_TREE_PASSES + 1;
    g_prof_cnt[3] = 0;
    ISO_CUDA(cudaMemcpy(g_prof_tiles, B.tiles, sizeof(g_prof_tiles), cudaMemcpyDeviceToHost));
    g_prof_sym = 1;
    g_prof_omega_kernel_ms = nitems > 0 ? E.ms(8, 9) : 0.0;
    g_prof_omega_gram_ms = 0.0;
    g_prof_omega_gram_blocks = 0;
    return map_status(fin, false);
}

}  // namespace iso

using namespace iso;

extern "C" {

isoclust_opts isoclust_opts_default(void) {
    isoclust_opts o;
    o.alpha = 0.0;
    o.omega_mode = ISOCLUST_OMEGA_FULL;
    o.precision = ISOCLUST_PREC_AUTO;
    o.root = 0;
    o.include_self = 0;
    o.spin_limit = 0;
    return o;
}

const char *isoclust_last_error(void) { return g_err; }

const char *isoclust_status_string(isoclust_status s) {
    switch (s) {
        case ISOCLUST_OK: return "ISOCLUST_OK";
        case ISOCLUST_ERR_INVALID_ARG: return "ISOCLUST_ERR_INVALID_ARG";
        case ISOCLUST_ERR_K_GT_N: return "ISOCLUST_ERR_K_GT_N";
        case ISOCLUST_ERR_NONFINITE: return "ISOCLUST_ERR_NONFINITE";
        case ISOCLUST_ERR_OOM: return "ISOCLUST_ERR_OOM";
        case ISOCLUST_ERR_CUDA: return "ISOCLUST_ERR_CUDA";
        case ISOCLUST_ERR_TIMEOUT: return "ISOCLUST_ERR_TIMEOUT";
        case ISOCLUST_ERR_NO_SOLUTION: return "ISOCLUST_ERR_NO_SOLUTION";
        case ISOCLUST_ERR_INTERNAL: return "ISOCLUST_ERR_INTERNAL";
    }
    return "ISOCLUST_UNKNOWN";
}

int32_t isoclust_abi_version(void) { return ISOCLUST_ABI_VERSION; }

int64_t isoclust_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void isoclust_last_mst_tiles(int64_t *tiles2) {
    if (tiles2) {
        tiles2[0] = g_prof_mst_tiles[0];
        tiles2[1] = g_prof_mst_tiles[1];
    }
}

void isoclust_last_profile(double *t_ms6, int64_t *counts4) {
    if (t_ms6) for (int i = 0; i < 6; ++i) t_ms6[i] = g_prof_ms[i];
    if (counts4) for (int i = 0; i < 4; ++i) counts4[i] = g_prof_cnt[i];
}

double isoclust_last_omega_kernel_ms(void) { return g_prof_omega_kernel_ms; }

double isoclust_last_omega_gram_ms(int64_t *blocks, int64_t *direct_pairs) {
    if (blocks) *blocks = g_prof_omega_gram_blocks;
    if (direct_pairs) *direct_pairs = g_prof_omega_gram_blocks ? (int64_t)g_prof_tiles[2] : 0;
    return g_prof_omega_gram_ms;
}

isoclust_status isoclust_set_sweep_variant(int32_t variant) {
    if (variant < -1 || variant > 3) return fail(ISOCLUST_ERR_INVALID_ARG, "sweep variant %d is not in -1..3", variant);
    tc_force_variant(variant);
    return ISOCLUST_OK;
}

int32_t isoclust_last_sweep_variant(void) { return tc_last_variant(); }

int32_t isoclust_last_batched_graph_mode(void) { return g_last_graph_mode; }

isoclust_status isoclust_set_mst_prune(int32_t mode) {
    if (mode < -1 || mode > 1) return fail(ISOCLUST_ERR_INVALID_ARG, "mst prune mode %d is not -1, 0 or 1", mode);
    prune_set_mode(mode);
    return ISOCLUST_OK;
}

isoclust_status isoclust_set_omega_gram(int32_t mode) {
    if (mode < -1 || mode > 1) return fail(ISOCLUST_ERR_INVALID_ARG, "mode must be -1, 0 or 1");
    g_omega_gram.store(mode, std::memory_order_relaxed);
    return ISOCLUST_OK;
}

isoclust_status isoclust_set_test_stalled_wait(int32_t on) {
    if (on != 0 && on != 1) return fail(ISOCLUST_ERR_INVALID_ARG, "on must be 0 or 1");
    g_stall_test.store(on, std::memory_order_relaxed);
    return ISOCLUST_OK;
}

isoclust_status isoclust_set_batched_graphs(int32_t enable) {
    if (enable != 0 && enable != 1) return fail(ISOCLUST_ERR_INVALID_ARG, "enable must be 0 or 1");
    g_graphs_on.store(enable, std::memory_order_relaxed);
    return ISOCLUST_OK;
}

void isoclust_last_omega_tiles(int64_t *tiles3) {
    if (tiles3) {
        tiles3[0] = (int64_t)g_prof_tiles[0];
        tiles3[1] = (int64_t)g_prof_tiles[1];
        tiles3[2] = g_prof_sym;
    }
}

isoclust_status isoclust_cluster_mst(const void *X, int64_t n, int32_t d, int32_t dtype, const isoclust_opts *opts,
                                     int32_t *edge_u, int32_t *edge_v, double *edge_d2, void *stream) {
    if (!edge_u || !edge_v || !edge_d2) return fail(ISOCLUST_ERR_INVALID_ARG, "edge outputs are required");
    return cluster_impl(X, n, d, dtype, 1, 1.0, opts, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                        nullptr, edge_u, edge_v, edge_d2, (cudaStream_t)stream, false);
}

isoclust_status isoclust_cluster(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t k, double sigma,
                                 const isoclust_opts *opts, int32_t *labels, uint8_t *residual, double *i_k,
                                 void *stream) {
    return cluster_impl(X, n, d, dtype, k, sigma, opts, labels, residual, i_k, nullptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream, true);
}

isoclust_status isoclust_cluster_sharded(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t k, double sigma,
                                         const isoclust_opts *opts, const isoclust_comm *comm, int32_t *labels,
                                         uint8_t *residual, double *i_k, void *stream) {
    if (!comm || !comm->allreduce) return fail(ISOCLUST_ERR_INVALID_ARG, "comm and comm->allreduce are required");
    if (comm->world < 1 || comm->rank < 0 || comm->rank >= comm->world)
        return fail(ISOCLUST_ERR_INVALID_ARG, "rank %d of world %d", comm->rank, comm->world);
    Shard sh;
    sh.rank = comm->rank;
    sh.world = comm->world;
    sh.fn = comm->allreduce;
    sh.ctx = comm->ctx;
    return cluster_impl(X, n, d, dtype, k, sigma, opts, labels, residual, i_k, nullptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream, true, &sh);
}

isoclust_status isoclust_cluster_detail(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t k, double sigma,
                                        const isoclust_opts *opts, int32_t *labels, uint8_t *residual, double *i_k,
                                        int32_t *parent, double *phi_par, double *omega, double *p, double *beta,
                                        int32_t *edge_u, int32_t *edge_v, double *edge_d2, void *stream) {
    return cluster_impl(X, n, d, dtype, k, sigma, opts, labels, residual, i_k, parent, phi_par, omega, p, beta,
                        edge_u, edge_v, edge_d2, (cudaStream_t)stream, true);
}

isoclust_status isoclust_cluster_batched(const void *X, const int64_t *offsets, int32_t nsets, int32_t d,
                                         int32_t dtype, const int32_t *ks, double sigma, const isoclust_opts *opts,
                                         int32_t *labels, uint8_t *residual, double *i_k, double *beta, void *stream) {
    return cluster_sets_impl(X, offsets, nsets, d, dtype, ks, sigma, opts, labels, residual, i_k, beta, nullptr, nullptr,
                             nullptr, (cudaStream_t)stream);
}

isoclust_status isoclust_cluster_batched_detail(const void *X, const int64_t *offsets, int32_t nsets, int32_t d,
                                                int32_t dtype, const int32_t *ks, double sigma,
                                                const isoclust_opts *opts, int32_t *labels, uint8_t *residual,
                                                double *i_k, double *beta, int32_t *parent, double *phi_par,
                                                double *omega, void *stream) {
    return cluster_sets_impl(X, offsets, nsets, d, dtype, ks, sigma, opts, labels, residual, i_k, beta, parent, phi_par,
                             omega, (cudaStream_t)stream);
}

isoclust_status isoclust_scale_features(const void *X, int64_t n, int32_t d, int32_t dtype, const double *scale,
                                        void *Z, void *stream) {
    isoclust_status st;
    if ((st = check_points(X, n, d, dtype, 1))) return st;
    if (!scale || !Z) return fail(ISOCLUST_ERR_INVALID_ARG, "scale and Z are required");
    cudaStream_t s = (cudaStream_t)stream;
    ISO_CUDA(scale_rows_launch(X, dtype, n, d, scale, Z, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    return ISOCLUST_OK;
}

isoclust_status isoclust_ik_backward(const void *X, int64_t n, int32_t d, int32_t dtype, const double *scale,
                                     double sigma, const int32_t *parent, const int32_t *labels, int32_t k,
                                     const double *phi_par, const double *omega, double grad_ik, double *dX,
                                     double *dscale, double *dsigma, double *i_k, void *stream) {
    isoclust_status st;
    if ((st = check_points(X, n, d, dtype, 2))) return st;
    if (!scale || !parent || !labels || !phi_par || !omega || !dX || !dscale || !dsigma)
        return fail(ISOCLUST_ERR_INVALID_ARG, "a required pointer is NULL");
    if (k < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "k = %d must be >= 1", k);
    if (k > n) return fail(ISOCLUST_ERR_K_GT_N, "k = %d exceeds n = %lld", k, (long long)n);
    if (!(sigma > 0.0) || !isfinite(sigma)) return fail(ISOCLUST_ERR_INVALID_ARG, "sigma must be finite and > 0");
    if (!isfinite(grad_ik)) return fail(ISOCLUST_ERR_INVALID_ARG, "grad_ik must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_call_mu[dev]);
    const size_t ws_bytes = adjoint_bytes(n, d, k) + 4096;
    void *base = scratch_acquire(ws_bytes + 256, s, &st);
    if (!base) return st;
    uint32_t *status = (uint32_t *)base;
    void *ws = (char *)base + 256;
    Events ev;
    ev.rec(0, s);
    ISO_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    ISO_CUDA(adjoint_launch(X, dtype, n, d, scale, sigma, parent, labels, k, phi_par, omega, grad_ik, dX, dscale,
                            dsigma, i_k, ws, status, ev.ok ? ev.e + 8 : nullptr, s));
    ev.rec(1, s);
    ISO_CUDA(cudaStreamSynchronize(s));
    uint32_t hst = 0;
    ISO_CUDA(cudaMemcpy(&hst, status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 6; ++i) g_prof_ms[i] = 0.0;
    g_prof_ms[4] = ev.ms(0, 1);
    g_prof_omega_kernel_ms = ev.ms(8, 9);
    g_prof_omega_gram_ms = 0.0;
    g_prof_omega_gram_blocks = 0;
    if (hst & DEV_NEGATIVE) return fail(ISOCLUST_ERR_INVALID_ARG, "a label 0..k-1 has no points or no positive omega");
    return map_status(hst, true);
}

isoclust_status isoclust_vertex_weights(const void *X, int64_t n, int32_t d, int32_t dtype, double sigma,
                                        const isoclust_opts *opts_in, double *omega, double *p, void *stream) {
    isoclust_status st;
    if ((st = check_points(X, n, d, dtype, 2))) return st;
    if (!omega) return fail(ISOCLUST_ERR_INVALID_ARG, "omega is NULL");
    if (!(sigma > 0.0) || !isfinite(sigma)) return fail(ISOCLUST_ERR_INVALID_ARG, "sigma must be finite and > 0");
    isoclust_opts o = resolve_opts(opts_in);
    if ((st = check_opts(o, n, dtype))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool fp64 = use_fp64_sweep(o, dtype);
    const int splits = mst_splits(n);
    bool use_tc = false;
    if ((st = use_tc_sweep(o, dtype, &use_tc))) return st;
    TcScratch TC;
    TC.wait_cycles = o.spin_limit;
    TC.stall_test = g_stall_test.load(std::memory_order_relaxed);
    const int tsplits = use_tc ? tc_splits(n) : 1;
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_call_mu[dev]);
    MstScratch M;
    uint32_t *status = nullptr;
    Arena meas;
    status = meas.take<uint32_t>(4);
    M.carve(meas, n, splits);
    if (use_tc) TC.carve(meas, n, d, tsplits);
    void *base = scratch_acquire(meas.off, s, &st);
    if (!base) return st;
    Arena A{(char *)base, meas.off + 4096, 0, false};
    status = A.take<uint32_t>(4);
    M.carve(A, n, splits);
    if (use_tc) TC.carve(A, n, d, tsplits);
    ISO_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t) * 4, s));
    ISO_CUDA(check_finite(X, n * (int64_t)d, dtype, status, nullptr, s));
    uint32_t hst = 0;
    ISO_CUDA(cudaMemcpyAsync(&hst, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    if (hst) return map_status(hst, false);
    if (!fp64) ISO_CUDA(nn_sweep(M, X, n, d, dtype, fp64, status, s, use_tc ? &TC : nullptr));
    ISO_CUDA(weights_launch(X, n, d, dtype, fp64, sigma, o.alpha, o.include_self, M.nnbits, omega, p, nullptr, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    ISO_CUDA(cudaMemcpy(&hst, status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return map_status(hst, false);
}

isoclust_status isoclust_tree_isoperimetric(int64_t n, const int32_t *parent, const double *phi_par,
                                            const double *omega, const double *p, int32_t k,
                                            const isoclust_opts *opts, int32_t *labels, uint8_t *residual,
                                            double *i_k, void *stream) {
    (void)opts;
    if (!parent || !phi_par || !omega || !labels || !residual || !i_k)
        return fail(ISOCLUST_ERR_INVALID_ARG, "a required pointer is NULL");
    if (n < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "n = %lld must be >= 1", (long long)n);
    if (n > 2147483646LL) return fail(ISOCLUST_ERR_INVALID_ARG, "n too large");
    if (k < 1) return fail(ISOCLUST_ERR_INVALID_ARG, "k = %d must be >= 1", k);
    if (k > n) return fail(ISOCLUST_ERR_K_GT_N, "k = %d exceeds n = %lld", k, (long long)n);
    cudaStream_t s = (cudaStream_t)stream;
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_call_mu[dev]);
    TreeScratch TS;
    int32_t *eu = nullptr, *ev = nullptr;
    const int64_t m = n > 1 ? n - 1 : 1;
    Arena meas;
    TS.carve(meas, n);
    eu = meas.take<int32_t>(m);
    ev = meas.take<int32_t>(m);
    isoclust_status st;
    void *base = scratch_acquire(meas.off, s, &st);
    if (!base) return st;
    Arena A{(char *)base, meas.off + 4096, 0, false};
    TS.carve(A, n);
    eu = A.take<int32_t>(m);
    ev = A.take<int32_t>(m);

    Events evs;
    evs.rec(0, s);
    ISO_CUDA(cudaMemsetAsync(TS.status, 0, sizeof(uint32_t), s));
    int32_t init[2] = {0, 2147483647};
    ISO_CUDA(cudaMemcpyAsync(TS.hostinfo, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_tree_input<<<(unsigned)ceil_div(n, TPB), TPB, 0, ISO_S(s)>>>(parent, n, TS.hostinfo, TS.status);
    int32_t info[2] = {0, 0};
    uint32_t hst = 0;
    ISO_CUDA(cudaMemcpyAsync(info, TS.hostinfo, sizeof(info), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaMemcpyAsync(&hst, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    if (hst) return map_status(hst, true);
    if (info[0] != 1) return fail(ISOCLUST_ERR_INVALID_ARG, "parent[] has %d roots (need exactly 1)", info[0]);
    const int32_t root = info[1];
    if (n > 1) ISO_CUDA(edges_from_parent(TS, parent, n, eu, ev, s));
    ISO_CUDA(orient_tree(TS, eu, ev, n, root, parent, s));
    ISO_CUDA(cudaMemcpyAsync(&hst, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    ISO_CUDA(cudaStreamSynchronize(s));
    if (hst) return map_status(hst, true);
    evs.rec(1, s);
    ISO_CUDA(tree_search_and_label(TS, phi_par, omega, p, k, labels, residual, i_k, s));
    evs.rec(2, s);
    ISO_CUDA(cudaStreamSynchronize(s));
    ISO_CUDA(cudaMemcpy(&hst, TS.status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    SearchState ss;
    ISO_CUDA(cudaMemcpy(&ss, TS.search, sizeof(ss), cudaMemcpyDeviceToHost));
    g_prof_ms[0] = 0; g_prof_ms[1] = 0; g_prof_ms[2] = 0;
    g_prof_ms[3] = evs.ms(0, 1);
    g_prof_ms[4] = evs.ms(1, 2);
    g_prof_ms[5] = 0;
    g_prof_cnt[0] = 0; g_prof_cnt[1] = 0;
    g_prof_cnt[2] = ss.passes + 1;
    g_prof_cnt[3] = ss.max_depth;
    return map_status(hst, true);
}

}  // extern "C"

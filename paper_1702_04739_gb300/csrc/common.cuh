// common.cuh -- shared internals of the isoclust CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "isoclust.h"

namespace iso {

// ---------------------------------------------------------------- status
// Device status word bits (one 32-bit word per call, OR-ed by kernels).
enum : uint32_t {
    DEV_NONFINITE = 1u << 0,    // NaN/Inf in an input array
    DEV_BAD_TREE = 1u << 1,     // parent[] / edge list does not form a tree
    DEV_NEGATIVE = 1u << 2,     // a weight that must be >= 0 (or > 0) is not
    DEV_NO_SOLUTION = 1u << 3,  // no threshold answers YES
    DEV_INTERNAL = 1u << 4,     // a consistency check failed
    DEV_TIMEOUT = 1u << 5,      // a bounded wait ran out
    DEV_EDGE_COUNT = 1u << 6,   // Boruvka did not produce n-1 edges
};

// A sharded call's collectives (isoclust_comm): rank r of world processes
// and the caller's all-reduce.  A null Shard pointer: nothing is sharded.
struct Shard {
    int32_t rank = 0, world = 1;
    isoclust_allreduce_fn fn = nullptr;
    void *ctx = nullptr;
};
// Runs the caller's all-reduce; a failure is reported as ISOCLUST_ERR_COMM
// by the next cuda_fail of this thread (the returned error is cudaErrorUnknown).
cudaError_t shard_allreduce(const Shard &sh, void *buf, int64_t count, int32_t op, cudaStream_t s);

void set_error(const char *fmt, ...);
isoclust_status fail(isoclust_status s, const char *fmt, ...);
isoclust_status cuda_fail(cudaError_t e, const char *what);
// Status word of a call's device checks -> its status code (and message);
// user_tree: the tree came from the caller (a malformed one is INVALID_ARG).
isoclust_status map_status(uint32_t st, bool user_tree);

#define ISO_CUDA(expr)                                              \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return ::iso::cuda_fail(_e, #expr);  \
    } while (0)

#define ISO_LAUNCH_CHECK(what)                                      \
    do {                                                            \
        cudaError_t _e = cudaGetLastError();                        \
        if (_e != cudaSuccess) return ::iso::cuda_fail(_e, what);   \
    } while (0)

// ---------------------------------------------------------------- launch count
// Every kernel launch passes its stream through ISO_S(), which bumps a
// process-wide counter (isoclust_kernel_launches()).
void note_launch();
#define ISO_S(s) (::iso::note_launch(), (s))

// Timing event on s.  Under stream capture a plain record only orders work
// inside the graph; the external flag makes the graph record the event
// itself when it runs, so its time can be read afterwards.
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    return cudaEventRecord(e, s);
}

// ---------------------------------------------------------------- arena
// Bump allocator over one device buffer.  In measure mode (base == nullptr)
// it only adds up the bytes a stage needs, so the same carving code both
// sizes and lays out the scratch.
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    bool overflow = false;

    template <class T>
    T *take(size_t count, size_t align = 256) {
        size_t a = (off + align - 1) / align * align;
        size_t bytes = count * sizeof(T);
        off = a + bytes;
        if (base == nullptr) return nullptr;
        if (off > cap) { overflow = true; return nullptr; }
        return reinterpret_cast<T *>(base + a);
    }
};

// Per-device cached scratch (grow-only).  Returns nullptr on failure.
void *scratch_acquire(size_t bytes, cudaStream_t stream, isoclust_status *st);
void scratch_release();
// A second per-device cached buffer (grow-only) for the omega Gram tiles,
// whose size is known only after the screen.  nullptr on failure.
void *gram_acquire(size_t bytes);

// The Gram of eq. omega's tile pairs on the tensor cores (omega_tc.cu).
// scratch / scratch_bytes: omega_gram_bytes(n, d) bytes of the call's
// scratch; the launch fills the rest (rows of the omega order padded to 128).
struct OmegaGram {
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    float *yh = nullptr, *yl = nullptr;   // [n_pad][d] y = x - c_T as a double-word
    int32_t *rexp = nullptr;              // [n_pad] E of each row
    float2 *rnorm = nullptr;              // [n_pad] |y|^2 as a double-word
    int32_t *item_slot = nullptr;         // [items] 2 x block + half, -1 when the screen drops the item
    float2 *gbuf = nullptr;               // [blocks][128][64] G in units of 2^(E_i + E_j - 14)
    int64_t nblocks = 0;
    int one_centre = 0;                   // every row centred on one point instead of its tile's centroid
};
// Rows at least this long are centred on one point for the Gram (no cross terms).
constexpr int32_t OMEGA_ONE_CENTRE_MIN_D = 1024;
size_t omega_gram_bytes(int64_t n, int32_t d);
// kev (may be null): two events recorded around the Gram kernel
cudaError_t omega_gram_launch(OmegaGram &G, const float *Xp, int64_t n, int32_t d, const float *cen,
                              const uint8_t *tskip, uint32_t *err, uint64_t wait_cycles, cudaStream_t s,
                              cudaEvent_t *kev = nullptr);

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms();

// exclusive scans (primitives.cu).  tmp must hold scan_tmp_elems(n) elements.
size_t scan_tmp_elems(int64_t n);
cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp,
                               cudaStream_t s);
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                               cudaStream_t s);

// Stable sort of (key, value) pairs by 64-bit key (merge sort, primitives.cu).
// keys/vals are sorted in place; kbuf/vbuf are ping-pong buffers of size n.
cudaError_t sort_pairs_u64(uint64_t *keys, int32_t *vals, uint64_t *kbuf, int32_t *vbuf,
                           int64_t n, cudaStream_t s);

// Non-finite scan of an input array (validation.cu): ORs DEV_NONFINITE.
cudaError_t check_finite(const void *X, int64_t count, int dtype, uint32_t *status,
                         double *absmax, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(uint64_t u) { return __longlong_as_double((long long)u); }

// Canonical FP64 distance key (reading K): ascending t, separately rounded
// subtract / multiply / add, no FMA.  Both rows are converted exactly.
template <class T>
__device__ __forceinline__ double exact_d2(const T *__restrict__ a, const T *__restrict__ b, int d) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double df = __dsub_rn((double)a[t], (double)b[t]);
        s = __dadd_rn(s, __dmul_rn(df, df));
    }
    return s;
}

// (d2, min, max) strict order
__device__ __forceinline__ bool key_less(double da, int32_t ua, int32_t va, double db, int32_t ub,
                                         int32_t vb) {
    int32_t a0 = min(ua, va), a1 = max(ua, va), b0 = min(ub, vb), b1 = max(ub, vb);
    if (da != db) return da < db;
    if (a0 != b0) return a0 < b0;
    return a1 < b1;
}

}  // namespace iso

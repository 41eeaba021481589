/*
 * isoclust.h -- C ABI of the GB300 (sm_103a) isoperimetric clustering hot path.
 *
 * Method: Javadi & Ashkboos, "An Efficient Parallel Data Clustering Algorithm
 * Using Isoperimetric Number of Trees" (arXiv 1702.04739):
 *   Section 2.1, eq. phi / eq. omega / eq. potential / eq. cost / eq. MISO,
 *   Section 2.2 (Algorithm 1: decision, Algorithm 2: bisection, pipeline
 *   steps 1-5), Section 3.5 (minimum spanning tree, global min/sum
 *   reductions), Section 3.6 (Cut / eta arrays, Algorithm 4: labels by an
 *   exclusive scan over Cut).
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers owned by the caller, row-major and
 *     densely packed, unless stated otherwise.  The library reads inputs,
 *     writes outputs, and never frees or retains either.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is queued on it; every call synchronises `stream`
 *     once before it returns so that the status it returns is final.
 *   - Internal scratch memory is allocated by the library on the current
 *     device, cached per device and reused by later calls (grow-only).  Calls
 *     on the same device from several host threads are serialised.
 *   - No call throws.  On a non-OK status the outputs are unspecified and
 *     isoclust_last_error() holds a one-line reason (per host thread).
 *   - Indices are 0-based.  n is limited to 2^31 - 2 points.
 *
 * Readings of the paper fixed by this library (each is applied identically by
 * every entry point):
 *   K  distance key: d2(i,j) = sum_t (x_it - x_jt)^2 evaluated in FP64 with
 *      t ascending and separately rounded subtract, multiply, add (no FMA);
 *      edges are ordered by (d2, min(i,j), max(i,j)), a strict total order,
 *      so the minimum spanning tree (Section 2.2 step 2) is unique.
 *   W  phi(e) = exp(-sqrt(d2)/sigma) (eq. phi); omega_i sums phi(x_i,x_j)
 *      over all j != i (eq. omega; `include_self` adds the j = i term);
 *      p_i = alpha * sum_{j != i} ||x_i - x_j|| (eq. potential).
 *   B  the tree is rooted at `root`; Algorithm 1 visits the reverse of the
 *      breadth-first order whose children are taken in ascending index, so
 *      siblings fold into their parent in descending index order.
 *   S  the bisection of Algorithm 2 is run to the last bit: beta is the
 *      smallest non-negative double N at which Algorithm 1 answers YES.
 *   L  cluster j (0-based) is the (j+1)-th cut vertex of Algorithm 1 at beta
 *      together with every vertex joined into it; vertices in none of the k
 *      sets are residual (label -1, residual flag 1).  i_k = cost of the k
 *      sets (eq. cost) = MISO_k of the weighted tree.
 */
#ifndef ISOCLUST_H
#define ISOCLUST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISOCLUST_ABI_VERSION 1

/* Status codes returned by every entry point. */
typedef enum {
    ISOCLUST_OK = 0,
    ISOCLUST_ERR_INVALID_ARG = 1,   /* bad size, pointer, option or malformed tree */
    ISOCLUST_ERR_K_GT_N = 2,        /* more clusters requested than points      */
    ISOCLUST_ERR_NONFINITE = 3,     /* NaN or Inf in X (found on the device)    */
    ISOCLUST_ERR_OOM = 4,           /* scratch allocation failed                */
    ISOCLUST_ERR_CUDA = 5,          /* a CUDA runtime call failed               */
    ISOCLUST_ERR_TIMEOUT = 6,       /* a bounded device wait ran out            */
    ISOCLUST_ERR_NO_SOLUTION = 7,   /* no finite N makes Algorithm 1 answer YES */
    ISOCLUST_ERR_INTERNAL = 8,      /* an internal consistency check failed     */
    ISOCLUST_ERR_COMM = 9           /* a sharded call's all-reduce callback failed */
} isoclust_status;

/* Element type of X. */
enum { ISOCLUST_F32 = 0, ISOCLUST_F64 = 1 };

/* omega_mode values. */
enum {
    ISOCLUST_OMEGA_FULL = 0,   /* eq. omega: sum over all j != i (default)          */
    ISOCLUST_OMEGA_TREE = 1    /* sum of phi over the tree edges incident to x_i    */
};

/* precision values: arithmetic of the Boruvka candidate sweep.  Every path
 * ends in the same FP64 key comparison, so all give the identical tree. */
enum {
    ISOCLUST_PREC_AUTO = 0,    /* F64 input: FP64 sweep; F32 input: tensor-core sweep    */
    ISOCLUST_PREC_FP64 = 1,    /* FP64 sweep (exact keys directly)                       */
    ISOCLUST_PREC_FP32 = 2,    /* FP32 SIMT candidates, FP64 recheck in a proven margin  */
    ISOCLUST_PREC_BF16_TC = 3  /* BF16 hi+lo Gram tiles on tcgen05 tensor cores with FP32
                                  accumulation, FP64 recheck in a proven margin (F32
                                  input, sm_103 only)                                    */
};

typedef struct {
    double alpha;               /* eq. potential scale; 0 (default) means p == 0       */
    int32_t omega_mode;         /* ISOCLUST_OMEGA_*, default FULL                       */
    int32_t precision;          /* ISOCLUST_PREC_*, default AUTO                        */
    int32_t root;               /* root vertex of the tree (default 0)                  */
    int32_t include_self;       /* 1: omega and p include the j = i term (default 0)   */
    uint64_t spin_limit;        /* bound of every device-side wait, SM clock cycles
                                   (0 = default, 4e9: about 2 s); see below         */
} isoclust_opts;

/* spin_limit: the library's only device-side waits are the mbarrier waits
 * of the tensor-core Boruvka sweep (and of the omega screen, which reuses
 * it), between its copy, MMA and epilogue roles.  Each wait gives up after
 * spin_limit SM clock cycles: the kernel raises a timeout flag, lets the
 * copies and MMAs it already issued finish, frees its tensor memory and
 * returns; the call then returns ISOCLUST_ERR_TIMEOUT without walking the
 * unfinished tree, and the device stays usable.  A small value can make
 * calls fail on a healthy device.  Calls without the tensor-core sweep
 * never wait. */

/* Test hook of the timeout path (no paper counterpart): while on (1), the
 * epilogue of every tensor-core sweep launch first waits for a barrier that
 * nothing arrives at, so that wait runs out after spin_limit cycles and the
 * call returns ISOCLUST_ERR_TIMEOUT through the same teardown as a real
 * timeout (in-flight copies and MMAs drained, tensor memory freed).  0 (the
 * default) turns it off.  Process-wide; other values -> INVALID_ARG. */
isoclust_status isoclust_set_test_stalled_wait(int32_t on);

/* Default options (alpha 0, full-graph omega, AUTO precision, root 0). */
isoclust_opts isoclust_opts_default(void);

/* One-line description of the last non-OK status on this host thread. */
const char *isoclust_last_error(void);

/* Static name of a status code. */
const char *isoclust_status_string(isoclust_status s);

/* ABI version of the loaded library (ISOCLUST_ABI_VERSION). */
int32_t isoclust_abi_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all devices, all threads).  Differences between two reads count the
 * kernels of the calls made in between. */
int64_t isoclust_kernel_launches(void);

/*
 * isoclust_cluster_mst -- Section 2.2 steps 1-2 (and Section 3.5): the exact
 * Euclidean minimum spanning tree of the n points under key K, found by a
 * fused tiled distance + Boruvka min-outgoing-edge sweep and GPU union-find;
 * the n x n matrix is never stored.
 *   X       n x d points, dtype ISOCLUST_F32 or ISOCLUST_F64 (device).
 *   edge_u, edge_v  [n-1] int32 (device, written): edge endpoints with
 *           edge_u < edge_v.
 *   edge_d2 [n-1] double (device, written): d2 of the edge (reading K).
 *   Edges are written in increasing key order (d2, edge_u, edge_v).
 * Errors: n < 2, d < 1, NULL pointers, bad dtype/options -> INVALID_ARG;
 *         NaN/Inf in X -> NONFINITE.
 */
isoclust_status isoclust_cluster_mst(const void *X, int64_t n, int32_t d, int32_t dtype,
                                     const isoclust_opts *opts,
                                     int32_t *edge_u, int32_t *edge_v, double *edge_d2,
                                     void *stream);

/*
 * isoclust_vertex_weights -- eq. omega and eq. potential (reading W) for all
 * n points: omega[i] = sum_{j != i} exp(-||x_i - x_j|| / sigma) and
 * p[i] = alpha * sum_{j != i} ||x_i - x_j||, in FP64-grade arithmetic.
 *   omega [n] double (device, written); p [n] double (device, written) or
 *   NULL when alpha == 0 is not needed.  opts->omega_mode is ignored here
 *   (this is the full-graph form).
 * Errors: as isoclust_cluster_mst, plus sigma <= 0 or non-finite -> INVALID_ARG.
 */
isoclust_status isoclust_vertex_weights(const void *X, int64_t n, int32_t d, int32_t dtype,
                                        double sigma, const isoclust_opts *opts,
                                        double *omega, double *p, void *stream);

/*
 * isoclust_tree_isoperimetric -- Algorithm 2 around Algorithm 1 (Section
 * 2.2) computed as in Algorithm 4 (Section 3.6) on a rooted weighted tree:
 * the exact k-th isoperimetric number MISO_k(T) and its minimising
 * k-subpartition (readings B, S, L).
 *   parent  [n] int32 (device): parent vertex; exactly one entry is -1 (the
 *           root).  Must describe a tree, else INVALID_ARG.
 *   phi_par [n] double (device): phi of the edge (v, parent[v]); the root's
 *           entry is ignored.  Must be >= 0 and finite.
 *   omega   [n] double (device): vertex weights, > 0 and finite.
 *   p       [n] double (device) or NULL (p == 0): potentials, >= 0.
 *   k       number of sets, 1 <= k <= n.
 *   labels  [n] int32 (device, written): cluster 0..k-1 or -1 (residual).
 *   residual[n] uint8 (device, written): 1 iff labels == -1.
 *   i_k     [1] double (device, written): MISO_k(T) = cost of the k sets.
 *   opts    may be NULL (defaults); opts->root is ignored (the tree's own
 *           root is used).
 * Errors: n < 1, k < 1, NULL pointers, malformed tree -> INVALID_ARG;
 *         k > n -> K_GT_N; NaN/Inf or negative weights -> NONFINITE /
 *         INVALID_ARG; no finite threshold -> NO_SOLUTION.
 */
isoclust_status isoclust_tree_isoperimetric(int64_t n, const int32_t *parent,
                                            const double *phi_par, const double *omega,
                                            const double *p, int32_t k,
                                            const isoclust_opts *opts,
                                            int32_t *labels, uint8_t *residual, double *i_k,
                                            void *stream);

/*
 * isoclust_tree_isoperimetric_noalloc -- the same computation and the same
 * results as isoclust_tree_isoperimetric, for callers that cannot allocate
 * device memory.  The paper has no counterpart; it exists for embedding.
 *
 * Who needs it: a host application that hands the whole device to its own
 * memory pool (an inference server, or a framework whose allocator reserves
 * all free memory up front), where a foreign cudaMalloc fails or breaks the
 * pool's accounting; or a latency-bound loop that cannot afford cudaMalloc /
 * cudaFree, which may synchronise the whole device.  This entry point calls
 * neither, nor any other allocating routine: its scratch is a fixed 13 MiB
 * array in the library's device code.  The caller still provides every
 * input and output buffer.
 *
 * Limits and behaviour:
 *   - n <= ISOCLUST_NOALLOC_MAX_N; larger trees are rejected with
 *     ISOCLUST_ERR_INVALID_ARG and a message naming the limit.
 *   - The array is placed in a device's memory when the first call on that
 *     device sets up (the CUDA runtime loads the module holding it lazily,
 *     and this call looks up the array's device address with
 *     cudaGetSymbolAddress, that device current); from then on it stays
 *     there until the process exits.  Make that first call (any small tree
 *     will do) on each device before a memory pool reserves the device's
 *     free memory and before any stream capture; it may synchronise the
 *     device.
 *   - All calls share the one array, which keeps the previous call's
 *     contents (the call clears what must start at zero).  Calls from this
 *     process are serialised and each completes before it returns; work that
 *     overlapped on the GPU would race on the array.
 *   - Arguments, errors and outputs are those of isoclust_tree_isoperimetric.
 */
#define ISOCLUST_NOALLOC_MAX_N 16384
isoclust_status isoclust_tree_isoperimetric_noalloc(int64_t n, const int32_t *parent,
                                                    const double *phi_par, const double *omega,
                                                    const double *p, int32_t k,
                                                    const isoclust_opts *opts,
                                                    int32_t *labels, uint8_t *residual, double *i_k,
                                                    void *stream);

/*
 * isoclust_cluster -- the whole hot path (Section 2.2 steps 1-5, Section 3):
 * minimum spanning tree of X, phi on its edges, omega (and p), the rooted
 * tree's global min/sum statistics, the bisection of Algorithm 2 with the
 * level-parallel Algorithm 1, and the labels of Algorithm 4.
 *   X       n x d points (device), dtype ISOCLUST_F32 or ISOCLUST_F64.
 *   k       number of clusters, 1 <= k <= n.  sigma > 0 (eq. phi).
 *   labels  [n] int32, residual [n] uint8, i_k [1] double (device, written)
 *           as in isoclust_tree_isoperimetric.
 * Errors: as isoclust_cluster_mst and isoclust_vertex_weights; k > n -> K_GT_N.
 */
isoclust_status isoclust_cluster(const void *X, int64_t n, int32_t d, int32_t dtype,
                                 int32_t k, double sigma, const isoclust_opts *opts,
                                 int32_t *labels, uint8_t *residual, double *i_k,
                                 void *stream);

/*
 * isoclust_cluster_detail -- isoclust_cluster that also returns the
 * intermediate results of the path (every output pointer may be NULL):
 *   parent [n] int32, phi_par [n] double   the MST rooted at opts->root
 *   omega [n] double, p [n] double         the vertex weights used
 *   beta [1] double                        the threshold of reading S
 *   edge_u, edge_v [n-1] int32, edge_d2 [n-1] double  the MST edges (key order)
 */
isoclust_status isoclust_cluster_detail(const void *X, int64_t n, int32_t d, int32_t dtype,
                                        int32_t k, double sigma, const isoclust_opts *opts,
                                        int32_t *labels, uint8_t *residual, double *i_k,
                                        int32_t *parent, double *phi_par, double *omega,
                                        double *p, double *beta,
                                        int32_t *edge_u, int32_t *edge_v, double *edge_d2,
                                        void *stream);

/*
 * isoclust_cluster_batched -- independent point sets in one call: set b is
 * rows offsets[b] .. offsets[b+1]-1 of X and is clustered into ks[b] sets
 * exactly as isoclust_cluster would cluster it alone (its own MST, omega
 * over its own pairs, phi, statistics, threshold search and labels; the
 * paper defines the method per point set, Section 2.2).  The sets share each
 * launch: one Boruvka forest whose sweep never pairs points of different
 * sets, one omega sweep over the sets' own tile pairs, and one tree pass with
 * a search state per set.
 *   X        N x d points, N = offsets[nsets] (device, F32 only).
 *   offsets  [nsets+1] int64 HOST array, offsets[0] = 0, every set >= 2 points.
 *   ks       [nsets] int32 HOST array, 1 <= ks[b] <= points of set b.
 *   labels   [N] int32, residual [N] uint8 (device, written): row v of set b
 *            gets its label within set b, 0 .. ks[b]-1, or -1 (residual), as
 *            isoclust_cluster would give it on that set alone.
 *   i_k      [nsets] double (device, written); beta [nsets] (device, may be
 *            NULL).
 *   opts     alpha = 0, omega_mode FULL, root 0 (each set's first point),
 *            precision AUTO or BF16_TC; others -> ISOCLUST_ERR_INVALID_ARG.
 * Needs an sm_103 device (tensor-core sweep).  The plan of the launch is
 * built on the host from offsets, hence host arrays.  Errors: as
 * isoclust_cluster, per set; a set with fewer than 2 points or ks[b] < 1 ->
 * ISOCLUST_ERR_INVALID_ARG, ks[b] above the set's size -> ISOCLUST_ERR_K_GT_N;
 * more than 2^31 rows once every set is rounded up to a multiple of 128 ->
 * ISOCLUST_ERR_INVALID_ARG.
 */
isoclust_status isoclust_cluster_batched(const void *X, const int64_t *offsets, int32_t nsets,
                                         int32_t d, int32_t dtype, const int32_t *ks, double sigma,
                                         const isoclust_opts *opts, int32_t *labels,
                                         uint8_t *residual, double *i_k, double *beta,
                                         void *stream);

/* isoclust_cluster_batched that also returns, for all N points (device,
 * NULL to skip): parent [N] int32 in global point indices (-1 at each set's
 * first point), phi_par [N] double, omega [N] double. */
isoclust_status isoclust_cluster_batched_detail(const void *X, const int64_t *offsets, int32_t nsets,
                                                int32_t d, int32_t dtype, const int32_t *ks,
                                                double sigma, const isoclust_opts *opts,
                                                int32_t *labels, uint8_t *residual, double *i_k,
                                                double *beta, int32_t *parent, double *phi_par,
                                                double *omega, void *stream);

/*
 * isoclust_scale_features -- Z = scale (.) X per feature (z_it = scale_t x_it,
 * formed in FP64 and stored in X's dtype): the points of a forward call with
 * a per-feature scale.  X, Z: n x d device arrays of dtype; scale: [d]
 * double (device).  Synchronous on `stream`.
 */
isoclust_status isoclust_scale_features(const void *X, int64_t n, int32_t d, int32_t dtype,
                                        const double *scale, void *Z, void *stream);

/*
 * isoclust_ik_backward -- the derivative of i_k (alpha = 0) through the
 * tree and the subpartition of a forward call on z = scale (.) x, held fixed
 * (eq. phi, eq. omega; the cost of Section 2.1).  A* is the label of the
 * largest ratio phi(dA_j) / omega(A_j), picked from the forward's phi_par /
 * omega; everything else is recomputed from X, scale and sigma (results in
 * FP64; Omega's pair sums in double-word FP32, relative error ~ d 2^-48,
 * with FP64 past FP32's exponent range):
 *   i_k = Phi / Omega,  Phi = sum of phi over the tree edges with one end in
 *   A*,  Omega = sum over A* of eq. omega,  dR = (dPhi - i_k dOmega) / Omega.
 *   X        n x d points (device, F32 or F64) before scaling.
 *   scale    [d] double (device); sigma > 0 (host).
 *   parent, labels, phi_par, omega: [n] from isoclust_cluster_detail on the
 *            scaled points (device); k as in that call.
 *   grad_ik  upstream gradient of i_k (host scalar).
 *   dX [n x d] double, dscale [d] double, dsigma [1] double (device, written):
 *            grad_ik times the derivative; i_k [1] double (device, may be
 *            NULL): the FP64 value of i_k on the fixed structure.
 * Coincident points (zero distance) contribute no direction.  Errors:
 * INVALID_ARG for a NULL pointer, sigma <= 0, a label in 0..k-1 without
 * points; K_GT_N for k > n.  Synchronous on `stream`.
 */
isoclust_status isoclust_ik_backward(const void *X, int64_t n, int32_t d, int32_t dtype,
                                     const double *scale, double sigma, const int32_t *parent,
                                     const int32_t *labels, int32_t k, const double *phi_par,
                                     const double *omega, double grad_ik, double *dX,
                                     double *dscale, double *dsigma, double *i_k, void *stream);

/*
 * isoclust_cluster_sharded -- isoclust_cluster on one point set whose
 * pairwise work is split across `comm->world` processes, one GPU each
 * (Section 3.5's MST rounds and eq. omega are sums and minima over the rows
 * of X, so rows shard; the tree stage is O(n) and runs on every rank).
 * Every rank calls it with the same X (replicated in its own device memory),
 * sizes, k, sigma and options, and gets the same labels, residual and i_k.
 *   - Boruvka rounds: rank r sweeps the 128-row tiles t of the norm-ordered
 *     rows with t mod world == r (tensor-core sweep, FP64 recheck of its own
 *     rows); the per-component minimum keys are combined by two all-reduce
 *     MIN calls per round (the d2 bits, then the packed (min, max) pair among
 *     the rows that reach that d2), each over n uint64 values; the
 *     union-find that follows is identical on every rank.
 *   - eq. omega: rank r evaluates the 64-row tile pairs w of the symmetric
 *     sweep with w mod world == r; each rank's per-row partial sums (FP64)
 *     are combined by one all-reduce SUM over n doubles.
 * comm->allreduce(ctx, buf, count, op, stream) must reduce the `count`
 * elements at device address `buf` in place across all ranks with `op`
 * (ISOCLUST_REDUCE_MIN_U64: unsigned 64-bit minimum - all ones marks "no
 * key", so a signed minimum needs the sign bit flipped before and after;
 * ISOCLUST_REDUCE_SUM_F64)
 * ordered on `stream` (a cudaStream_t): it is called from the host between
 * kernel launches, with earlier work queued, not finished; the library's
 * kernels that follow are queued after it returns.  It returns 0 on success;
 * anything else makes the call return ISOCLUST_ERR_COMM.  rank in [0,
 * world), world >= 1; world == 1 runs the single-GPU work through the same
 * path.  The omega sums of different ranks are added in FP64 after the
 * double-word per-rank sums, so omega (and i_k) can differ from
 * isoclust_cluster's in the last bits, within its error bound; the tree is
 * the same unique MST.
 * Needs F32 input, an sm_103 device, alpha = 0, full-graph omega and the
 * AUTO or BF16_TC precision; other options -> ISOCLUST_ERR_INVALID_ARG.
 */
enum { ISOCLUST_REDUCE_MIN_U64 = 0, ISOCLUST_REDUCE_SUM_F64 = 1 };
typedef int32_t (*isoclust_allreduce_fn)(void *ctx, void *buf, int64_t count, int32_t op, void *stream);
typedef struct {
    int32_t rank;                     /* this process, 0 .. world-1       */
    int32_t world;                    /* processes sharing the work       */
    isoclust_allreduce_fn allreduce;  /* the caller's collective          */
    void *ctx;                        /* passed back to allreduce         */
} isoclust_comm;

isoclust_status isoclust_cluster_sharded(const void *X, int64_t n, int32_t d, int32_t dtype,
                                         int32_t k, double sigma, const isoclust_opts *opts,
                                         const isoclust_comm *comm,
                                         int32_t *labels, uint8_t *residual, double *i_k,
                                         void *stream);

/* Per-stage device times (milliseconds, CUDA events on the call's stream)
 * of the last isoclust_cluster / _detail / _batched call on this host thread:
 * t[0] validation, t[1] weights, t[2] MST, t[3] tree orientation + stats,
 * t[4] bisection, t[5] labels (after isoclust_ik_backward: t[4] is the
 * backward's time, the others 0).  counts[0] = Boruvka rounds, counts[1] =
 * rows rescanned after a candidate-margin overflow, counts[2] = Algorithm-1
 * passes, counts[3] = tree depth.  Either pointer may be NULL. */
void isoclust_last_profile(double *t_ms6, int64_t *counts4);

/* The last one-set call's tensor-core sweep on this host thread: tiles2[0]
 * = pairs of 128-row tiles swept over all Boruvka rounds (row tile x column
 * tile; the pruned rounds' near and far tiles), tiles2[1] = the pairs a full
 * sweep of every round takes (rounds x tiles^2); both 0 without that sweep. */
void isoclust_last_mst_tiles(int64_t *tiles2);

/* Tile pairs of the omega sweep in the last isoclust_cluster / _detail call
 * on this host thread: tiles3[0] = 64x64 tile pairs screened, tiles3[1] =
 * tile pairs evaluated in double-word arithmetic (the rest held only terms
 * below e^-(36 + ln n) of their row's largest term), tiles3[2] = 0 when the
 * pairs were ordered, 1 when unordered (symmetric sweep, each pair once for
 * both rows) and screened in FP32, 2 when unordered and screened on the
 * tensor cores (the FP32 screen did not run), 3 as 2 with the kept pairs'
 * Gram on the tensor cores (isoclust_set_omega_gram).  Zero counts when the screen did not run (F64 input,
 * alpha > 0, or the FP64 precision option). */
void isoclust_last_omega_tiles(int64_t *tiles3);

/* Device time (milliseconds, CUDA events on the call's stream around its
 * launch) of the dominant pair kernel of the last call on this host thread:
 * the symmetric omega kernel after isoclust_cluster / _detail / _batched (0
 * when it did not run; with the Gram on the tensor cores, the sweep that
 * reads it), the pair-sum kernel of dOmega after isoclust_ik_backward. */
double isoclust_last_omega_kernel_ms(void);

/* Device time (milliseconds, CUDA events on the call's stream) of the
 * tensor-core Gram kernel of omega in the last one-set call on this host
 * thread (isoclust_set_omega_gram), 0 when it did not run; *blocks (may be
 * NULL) gets its number of 128 x 64 blocks (each 34 BF16 digit-plane MMA
 * products of 2 x 128 x 64 x d_pad flop, d_pad = d rounded up to 64), and
 * *direct_pairs (may be NULL) the number of pairs whose Gram form cancelled
 * and which took the direct sum of squared differences instead. */
double isoclust_last_omega_gram_ms(int64_t *blocks, int64_t *direct_pairs);

/* Tile variant of the tensor-core Boruvka sweep (Section 3.5's MST step
 * with the tiled Gram sweep): bit 0 set = 32-column candidate blocks (else
 * 64), bit 1 set = the row block streams with the column blocks (else it
 * stays resident in shared memory when the padded row length is <= 128).
 * variant -1 (the default) lets the library pick: on the first call of a
 * shape class (device, one set or independent sets, padded row length, and
 * the powers of two of the padded rows and work items) it times one trial
 * round of each variant on the round-1 state and caches the fastest; small
 * problems take a fixed rule.  0..3 force a variant for every later call of
 * the process.  Results do not depend on the variant (the minimum spanning
 * tree under the edge key is unique); only the speed does.  Other values ->
 * ISOCLUST_ERR_INVALID_ARG.  Process-wide setting; no device work. */
isoclust_status isoclust_set_sweep_variant(int32_t variant);

/* The sweep variant of the last minimum-spanning-tree build on this host
 * thread (0..3), or -1 when none ran (FP32/FP64 sweep, F64 input). */
int32_t isoclust_last_sweep_variant(void);

/* How the last isoclust_cluster_batched / _batched_detail call on this
 * process ran its device work: 0 launched kernel by kernel, 1 captured into
 * CUDA graphs and launched them, 2 replayed the graphs of the previous call.
 * A call replays when its arguments (pointers, sizes, offsets and ks
 * contents, sigma, options) match the previous batched call on the device
 * (the first call of a signature runs kernel by kernel, the second is
 * captured).  Results are identical in every mode. */
int32_t isoclust_last_batched_graph_mode(void);

/* Arithmetic of eq. omega's pair sums in one-set calls (F32 input, sm_103,
 * alpha = 0, full-graph omega).  Tensor-core Gram: each kept tile pair's
 * Gram <y_i, y_j> of the tile-centred points is formed exactly on the tensor
 * cores (7 balanced base-256 digit planes per row, BF16 products summed
 * exactly in FP32 accumulators), the rest of d2 and the terms in double-word
 * FP32, and pairs whose Gram form cancels (its parts more than twice d2)
 * take the double-word sum of squared differences.  Otherwise every pair's
 * d2 is that double-word sum.  Both keep d2 to about 2^-46 relative; omega
 * agrees to within the library's error bound, not bit for bit.
 * Rows of 1,024 dimensions or more are centred on one point for the Gram
 * (the mean of the 64-row tiles' centroids), shorter ones on their tile's
 * centroid.
 * mode -1 (the default): the Gram on the tensor cores for rows of 64
 * dimensions or more; 1: always; 0: never.  Process-wide; other values ->
 * INVALID_ARG. */
isoclust_status isoclust_set_omega_gram(int32_t mode);

/* Pruned Boruvka rounds for one-set calls (Section 3.5's minimum spanning
 * tree): rows in a recursive-bisection order whose 128-row tiles are
 * compact; each round first sweeps every tile against its near tiles, which
 * bounds each component's lightest outgoing edge from above, and then sweeps
 * only the pairs of tiles whose distance lower bound (centroid distance less
 * both radii) is within the bound of some component of the row tile, and
 * never two tiles wholly inside one component.  The tree is the same edge
 * for edge.  mode -1 (the default): pruned for n >= 65,536 and d <= 256;
 * 1: whenever the tensor-core sweep runs a one-set call of 64 points or
 * more and at most 256 dimensions, a multiple of 4; 0: never.  Either way
 * X must start on a 16-byte boundary (the order's kernels read rows by 16
 * bytes); otherwise the call runs unpruned.  Not for sharded calls.
 * Process-wide; other values -> INVALID_ARG. */
isoclust_status isoclust_set_mst_prune(int32_t mode);

/* Whether repeated batched calls may capture and replay CUDA graphs: 1 (the
 * default) allows it, 0 keeps every later batched call kernel by kernel.
 * Process-wide setting, no device work; other values -> INVALID_ARG.  A
 * batched call with a non-zero opts->spin_limit never uses graphs. */
isoclust_status isoclust_set_batched_graphs(int32_t enable);

#ifdef __cplusplus
}
#endif

#endif /* ISOCLUST_H */

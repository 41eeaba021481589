/*
 * isoclust_oracle.c -- plain, slow, FP64 CPU oracle for the isoperimetric
 * clustering hot path of Javadi & Ashkboos, "An Efficient Parallel Data
 * Clustering Algorithm Using Isoperimetric Number of Trees" (arXiv 1702.04739).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Everything is FP64 (the paper states no precision).  Each function follows
 * the paper's definition or algorithm in the paper's order; where the paper
 * is silent or ambiguous the reading taken is written beside the code:
 *
 *   R1  distance key: d2(i,j) = sum_t (x_it - x_jt)^2, t ascending, one
 *       rounded subtraction, multiplication and addition per term (no FMA:
 *       build with -ffp-contract=off).  Edges compare by (d2, min, max), a
 *       strict total order, so the minimum spanning tree is unique.
 *   R2  omega (eq. omega) and p (eq. potential) sum over every j != i in
 *       ascending j (phi is only defined for i != j, eq. phi); an option adds
 *       the j = i term.  An option replaces omega by the sum of phi over the
 *       tree edges incident to x_i.
 *   R3  the root is vertex `root` (default 0); "BFS order" is the breadth-
 *       first order with the children of every vertex taken in ascending
 *       index, and Algorithm 1 walks it backwards (root last, x_n = v).
 *   R4  the else-branch of Algorithm 1 adds phi of the parent edge e to p(u).
 *   R5  the search of Algorithm 2 is run to the last bit: beta is the
 *       smallest non-negative double N for which Algorithm 1 answers YES
 *       (bisection on the ordered bit patterns of non-negative doubles,
 *       started from [alpha_0, beta_0] as Algorithm 2 prescribes).
 *   R6  A_j is the j-th cut made by Algorithm 1; its label is j-1; vertices
 *       in no A_j are residual (label -1).  MISO_k = cost of {A_1..A_k}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void oracle_set_threads(int t) { g_threads = t > 0 ? t : 1; }
int oracle_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------ */
/* Section 2.2 step 1: edge weights d(x_i,x_j) = ||x_i - x_j||_2, kept
 * squared (reading R1).  X is row-major n x d in FP64. */
double oracle_d2(const double *X, int64_t n, int32_t d, int64_t i, int64_t j)
{
    (void)n;
    const double *a = X + i * (int64_t)d;
    const double *b = X + j * (int64_t)d;
    double s = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double diff = a[t] - b[t];
        double sq = diff * diff;
        s = s + sq;
    }
    return s;
}

/* strict total order on edges: (d2, min index, max index) */
static int key_less(double d2a, int64_t ua, int64_t va, double d2b, int64_t ub, int64_t vb)
{
    int64_t a0 = ua < va ? ua : va, a1 = ua < va ? va : ua;
    int64_t b0 = ub < vb ? ub : vb, b1 = ub < vb ? vb : ub;
    if (d2a != d2b) return d2a < d2b;
    if (a0 != b0) return a0 < b0;
    return a1 < b1;
}

typedef struct { double d2; int32_t u, v; } edge_t;

static int edge_cmp(const void *pa, const void *pb)
{
    const edge_t *a = (const edge_t *)pa, *b = (const edge_t *)pb;
    if (key_less(a->d2, a->u, a->v, b->d2, b->u, b->v)) return -1;
    if (key_less(b->d2, b->u, b->v, a->d2, a->u, a->v)) return 1;
    return 0;
}

static void sort_edges_out(edge_t *E, int64_t m, int32_t *eu, int32_t *ev, double *ed2)
{
    qsort(E, (size_t)m, sizeof(edge_t), edge_cmp);
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = E[e].u, v = E[e].v;
        eu[e] = u < v ? u : v;
        ev[e] = u < v ? v : u;
        ed2[e] = E[e].d2;
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 3 (Section 3.5): Prim's algorithm from `root`.  Each step adds
 * the outside vertex whose best edge to the tree is smallest, records its
 * Parent and Depth, then updates every outside vertex's best edge with the
 * new vertex.  Loop bound read as |T| < n.  Outputs: the n-1 edges sorted by
 * key, and parent[] (root: -1) / depth[] of the tree rooted at `root`. */
int oracle_mst_prim(const double *X, int64_t n, int32_t d, int64_t root,
                    int32_t *eu, int32_t *ev, double *ed2,
                    int32_t *parent, int32_t *depth)
{
    if (n < 1 || root < 0 || root >= n) return -1;
    double *bd2 = (double *)malloc(sizeof(double) * n);
    int64_t *bfrom = (int64_t *)malloc(sizeof(int64_t) * n);
    char *in = (char *)calloc((size_t)n, 1);
    edge_t *E = (edge_t *)malloc(sizeof(edge_t) * (n > 1 ? n - 1 : 1));
    if (!bd2 || !bfrom || !in || !E) { free(bd2); free(bfrom); free(in); free(E); return -2; }

    for (int64_t v = 0; v < n; ++v) { bd2[v] = INFINITY; bfrom[v] = -1; }
    in[root] = 1;
    parent[root] = -1;
    depth[root] = 0;
    int64_t last = root;
    for (int64_t added = 1; added < n; ++added) {
        /* update all distances with the vertex added last */
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int64_t w = 0; w < n; ++w) {
            if (in[w]) continue;
            double c = oracle_d2(X, n, d, last, w);
            if (bfrom[w] < 0 || key_less(c, last, w, bd2[w], bfrom[w], w)) {
                bd2[w] = c;
                bfrom[w] = last;
            }
        }
        /* min-reduction: outside vertex with the smallest best edge */
        int64_t best = -1;
        for (int64_t w = 0; w < n; ++w) {
            if (in[w]) continue;
            if (best < 0 || key_less(bd2[w], bfrom[w], w, bd2[best], bfrom[best], best)) best = w;
        }
        in[best] = 1;
        parent[best] = (int32_t)bfrom[best];
        depth[best] = depth[bfrom[best]] + 1;
        E[added - 1].d2 = bd2[best];
        E[added - 1].u = (int32_t)bfrom[best];
        E[added - 1].v = (int32_t)best;
        last = best;
    }
    if (n > 1) sort_edges_out(E, n - 1, eu, ev, ed2);
    free(bd2); free(bfrom); free(in); free(E);
    return 0;
}

/* Kruskal over all pairs (self-check of Prim for small n). */
static int64_t uf_find(int64_t *p, int64_t x)
{
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

int oracle_mst_kruskal(const double *X, int64_t n, int32_t d,
                       int32_t *eu, int32_t *ev, double *ed2)
{
    if (n < 1) return -1;
    int64_t m = n * (n - 1) / 2;
    edge_t *all = (edge_t *)malloc(sizeof(edge_t) * (m > 0 ? m : 1));
    int64_t *p = (int64_t *)malloc(sizeof(int64_t) * n);
    edge_t *E = (edge_t *)malloc(sizeof(edge_t) * (n > 1 ? n - 1 : 1));
    if (!all || !p || !E) { free(all); free(p); free(E); return -2; }
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            all[c].d2 = oracle_d2(X, n, d, i, j);
            all[c].u = (int32_t)i;
            all[c].v = (int32_t)j;
            ++c;
        }
    qsort(all, (size_t)m, sizeof(edge_t), edge_cmp);
    for (int64_t i = 0; i < n; ++i) p[i] = i;
    int64_t taken = 0;
    for (int64_t e = 0; e < m && taken < n - 1; ++e) {
        int64_t a = uf_find(p, all[e].u), b = uf_find(p, all[e].v);
        if (a == b) continue;
        p[a] = b;
        E[taken++] = all[e];
    }
    if (n > 1) sort_edges_out(E, n - 1, eu, ev, ed2);
    free(all); free(p); free(E);
    return taken == n - 1 ? 0 : -3;
}

/* Exact nearest neighbour (smallest key) of each listed row. */
int oracle_nn_rows(const double *X, int64_t n, int32_t d, const int64_t *rows, int64_t nrows,
                   int32_t *nn, double *nn_d2)
{
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        int64_t best = -1;
        double bd = INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double c = oracle_d2(X, n, d, i, j);
            if (best < 0 || key_less(c, i, j, bd, i, best)) { best = j; bd = c; }
        }
        nn[r] = (int32_t)best;
        nn_d2[r] = bd;
    }
    return 0;
}

/* One step of Boruvka's method (Section 3.5's MST, the rounds that replace
 * Prim's loop): for each listed row i, its smallest-key edge (d2, min, max)
 * to a point of another component (comp[j] != comp[i]); -1 / INFINITY when
 * every point is in i's component. */
int oracle_min_foreign(const double *X, int64_t n, int32_t d, const int32_t *comp,
                       const int64_t *rows, int64_t nrows, int32_t *out_j, double *out_d2)
{
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        int64_t best = -1;
        double bd = INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            if (comp[j] == comp[i]) continue;
            double c = oracle_d2(X, n, d, i, j);
            if (best < 0 || key_less(c, i, j, bd, i, best)) { best = j; bd = c; }
        }
        out_j[r] = (int32_t)best;
        out_d2[r] = bd;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* eq. phi: phi(x_i,x_j) = exp(-||x_i - x_j||_2 / sigma)                */
static double flow_of_d2(double d2, double sigma)
{
    double dist = sqrt(d2);
    double y = dist / sigma;
    return exp(-y);
}

double oracle_flow(double d2, double sigma) { return flow_of_d2(d2, sigma); }

/* eq. phi on the parent edge of every vertex: phi_par[v] = phi(x_v,
 * x_parent[v]) (0 at the root), as the pipeline of oracle_cluster forms it. */
int oracle_parent_flow(const double *X, int64_t n, int32_t d, const int32_t *parent, double sigma,
                       double *phi_par)
{
    for (int64_t v = 0; v < n; ++v) {
        if (parent[v] >= n) return -1;
        phi_par[v] = parent[v] >= 0 ? flow_of_d2(oracle_d2(X, n, d, v, parent[v]), sigma) : 0.0;
    }
    return 0;
}

/* eq. omega and eq. potential for the listed rows (all rows when rows is
 * NULL): omega_i = sum_j phi(x_i,x_j), p_i = alpha * sum_j ||x_i - x_j||,
 * j ascending, j = i skipped unless include_self (reading R2). */
int oracle_weights(const double *X, int64_t n, int32_t d, double sigma, double alpha,
                   int32_t include_self, const int64_t *rows, int64_t nrows,
                   double *omega, double *p)
{
    int64_t cnt = rows ? nrows : n;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 16)
    for (int64_t r = 0; r < cnt; ++r) {
        int64_t i = rows ? rows[r] : r;
        double sw = 0.0, sd = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) {
                if (include_self) { sw = sw + 1.0; sd = sd + 0.0; }
                continue;
            }
            double d2 = oracle_d2(X, n, d, i, j);
            sw = sw + flow_of_d2(d2, sigma);
            if (alpha != 0.0) sd = sd + sqrt(d2);
        }
        omega[r] = sw;
        p[r] = alpha != 0.0 ? alpha * sd : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Section 2.2 step 3: BFS order from the root with children in ascending
 * index (reading R3).  parent[v] = -1 marks the root.  Writes order[0..n-1]
 * (order[0] = root).  Returns 0, or -1 if parent[] is not a rooted tree. */
int oracle_bfs_order(int64_t n, const int32_t *parent, int32_t *order)
{
    int64_t root = -1;
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *kids = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    if (!cnt || !kids || !fill) { free(cnt); free(kids); free(fill); return -2; }
    for (int64_t v = 0; v < n; ++v) {
        if (parent[v] < 0) { if (root >= 0) { root = -2; } else if (root == -1) root = v; continue; }
        if (parent[v] >= n) { root = -2; break; }
        cnt[parent[v] + 1]++;
    }
    if (root < 0) { free(cnt); free(kids); free(fill); return -1; }
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    memcpy(fill, cnt, sizeof(int64_t) * (n + 1));
    for (int64_t v = 0; v < n; ++v)          /* ascending v => ascending children */
        if (parent[v] >= 0) kids[fill[parent[v]]++] = (int32_t)v;
    int64_t head = 0, tail = 0;
    order[tail++] = (int32_t)root;
    while (head < tail) {
        int32_t u = order[head++];
        for (int64_t c = cnt[u]; c < cnt[u + 1]; ++c) {
            if (tail >= n) { free(cnt); free(kids); free(fill); return -1; }
            order[tail++] = kids[c];
        }
    }
    free(cnt); free(kids); free(fill);
    return tail == n ? 0 : -1;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: decide whether some k-subpartition has cost <= N.
 * Walks x_1..x_n = reversed BFS order (root last), on working copies of
 * omega and p.  eta(x) is kept as linked lists so A_j = eta(x_i) can be read
 * out at the cut.  Stops when j = k (the while condition).  Returns j (the
 * number of cuts made, <= k).  If labels != NULL, writes label j-1 for the
 * members of A_j and -1 elsewhere; ratio[j-1] = (phi(e)+p(x_i))/omega(x_i). */
typedef struct {
    int64_t n;
    const int32_t *parent;
    const double *phi_par;   /* phi of the parent edge; ignored at the root */
    const double *omega;
    const double *p;         /* may be NULL: p == 0 */
    const int32_t *order;    /* BFS order, order[0] = root */
} tree_t;

static int64_t decision(const tree_t *T, int64_t k, double N,
                        double *w, double *pp, int32_t *lhead, int32_t *lnext, int32_t *ltail,
                        int32_t *labels, double *ratio)
{
    int64_t n = T->n;
    for (int64_t v = 0; v < n; ++v) {
        w[v] = T->omega[v];
        pp[v] = T->p ? T->p[v] : 0.0;
        lhead[v] = (int32_t)v; lnext[v] = -1; ltail[v] = (int32_t)v;   /* eta(x) = {x} */
    }
    if (labels) for (int64_t v = 0; v < n; ++v) labels[v] = -1;
    int64_t j = 0;
    int64_t i = 0;                            /* x_{i+1} = order[n-1-i] */
    while (j < k && i < n) {
        int32_t x = T->order[n - 1 - i];
        int32_t u = T->parent[x];
        double fe = u >= 0 ? T->phi_par[x] : 0.0;   /* the root has no parent edge */
        double pv = pp[x], wv = w[x];
        double nw = N * wv;
        if (fe + pv <= nw) {
            /* x is a cut vertex: A_j = eta(x), phi(dA_j) = phi(e) + p(x) */
            j = j + 1;
            if (labels) {
                for (int32_t m = lhead[x]; m >= 0; m = lnext[m]) labels[m] = (int32_t)(j - 1);
            }
            if (ratio) ratio[j - 1] = (fe + pv) / wv;
            if (u >= 0) pp[u] = pp[u] + fe;
        } else if (pv - fe < nw) {
            /* join x to its parent */
            if (u >= 0) {
                lnext[ltail[u]] = lhead[x];
                ltail[u] = ltail[x];
                w[u] = w[u] + wv;
                pp[u] = pp[u] + pv;
            }
        } else {
            /* discard: the parent edge becomes boundary of u's set (R4) */
            if (u >= 0) pp[u] = pp[u] + fe;
        }
        i = i + 1;
    }
    return j;
}

/* Public form of Algorithm 1: returns the number of cuts (<= k) made at
 * threshold N; YES iff the return value equals k. */
int64_t oracle_decision(int64_t n, const int32_t *parent, const double *phi_par,
                        const double *omega, const double *p, int64_t k, double N)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * n);
    double *w = (double *)malloc(sizeof(double) * n), *pp = (double *)malloc(sizeof(double) * n);
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * n), *b = (int32_t *)malloc(sizeof(int32_t) * n),
            *c = (int32_t *)malloc(sizeof(int32_t) * n);
    int64_t r = -1;
    if (order && w && pp && a && b && c && oracle_bfs_order(n, parent, order) == 0) {
        tree_t T = {n, parent, phi_par, omega, p, order};
        r = decision(&T, k, N, w, pp, a, b, c, NULL, NULL);
    }
    free(order); free(w); free(pp); free(a); free(b); free(c);
    return r;
}

/* Algorithm 1 at threshold N, reporting how close each decision was.
 * Same walk and early stop as decision() (x_1..x_n = reversed BFS order,
 * stop after the k-th cut).  For every vertex x visited, with e its parent
 * edge and omega-hat, p-hat the working values at x's turn:
 *   code[x]  = 0 cut, 1 join, 2 discard (the branch Algorithm 1 took);
 *   ncut[x]  = (phi(e) + p-hat(x)) / omega-hat(x): the cut test holds iff
 *              N reaches this value (up to the rounding of N * omega-hat);
 *   njoin[x] = (p-hat(x) - phi(e)) / omega-hat(x): the join test holds iff
 *              N exceeds it.
 * Vertices not visited (after the k-th cut) get code -1 and NaN ratios.
 * Returns the number of cuts made, or -1 if parent[] is not a rooted tree. */
int64_t oracle_decision_detail(int64_t n, const int32_t *parent, const double *phi_par,
                               const double *omega, const double *p, int64_t k, double N,
                               int8_t *code, double *ncut, double *njoin)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    double *w = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *pp = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int64_t j = -1;
    if (!order || !w || !pp || oracle_bfs_order(n, parent, order) != 0) goto out;
    for (int64_t v = 0; v < n; ++v) {
        w[v] = omega[v];
        pp[v] = p ? p[v] : 0.0;
        code[v] = -1;
        ncut[v] = NAN;
        njoin[v] = NAN;
    }
    j = 0;
    for (int64_t i = 0; j < k && i < n; ++i) {
        int32_t x = order[n - 1 - i];
        int32_t u = parent[x];
        double fe = u >= 0 ? phi_par[x] : 0.0;
        double pv = pp[x], wv = w[x];
        double nw = N * wv;
        ncut[x] = (fe + pv) / wv;
        njoin[x] = (pv - fe) / wv;
        if (fe + pv <= nw) {
            code[x] = 0;
            j = j + 1;
            if (u >= 0) pp[u] = pp[u] + fe;
        } else if (pv - fe < nw) {
            code[x] = 1;
            if (u >= 0) { w[u] = w[u] + wv; pp[u] = pp[u] + pv; }
        } else {
            code[x] = 2;
            if (u >= 0) pp[u] = pp[u] + fe;
        }
    }
out:
    free(order); free(w); free(pp);
    return j;
}

static uint64_t dbits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double bitsd(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

/* Algorithm 2 with reading R5, then the final call of Algorithm 1 at beta.
 * stats[0..5] = phi*, phi_*, omega*, omega_*, p*, p_*; stats[6] = alpha_0,
 * stats[7] = beta_0; info[0] = number of Algorithm-1 calls.
 * Returns 0, -1 (bad tree) or -3 (no finite threshold answers YES). */
int oracle_tree_stage(int64_t n, const int32_t *parent, const double *phi_par,
                      const double *omega, const double *p, int64_t k,
                      int32_t *labels, uint8_t *residual, double *i_k, double *beta_out,
                      double *stats, int64_t *info)
{
    if (n < 1 || k < 1 || k > n) return -1;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * n);
    double *w = (double *)malloc(sizeof(double) * n), *pp = (double *)malloc(sizeof(double) * n);
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * n), *b = (int32_t *)malloc(sizeof(int32_t) * n),
            *c = (int32_t *)malloc(sizeof(int32_t) * n);
    double *ratio = (double *)malloc(sizeof(double) * (size_t)k);
    int rc = 0;
    if (!order || !w || !pp || !a || !b || !c || !ratio) { rc = -2; goto out; }
    if (oracle_bfs_order(n, parent, order) != 0) { rc = -1; goto out; }
    {
        tree_t T = {n, parent, phi_par, omega, p, order};
        /* Section 2.2 step 4: phi*, phi_* over the tree edges; omega*, omega_*, p*, p_* over X */
        double phs = 0.0, phm = INFINITY, ws = 0.0, wm = INFINITY, ps = 0.0, pm = INFINITY;
        for (int64_t v = 0; v < n; ++v) {
            if (parent[v] >= 0) { phs = phs + phi_par[v]; if (phi_par[v] < phm) phm = phi_par[v]; }
            ws = ws + omega[v]; if (omega[v] < wm) wm = omega[v];
            double pv = p ? p[v] : 0.0;
            ps = ps + pv; if (pv < pm) pm = pv;
        }
        if (n == 1) phm = 0.0;
        double alpha0 = (phm + pm) / ws;
        double beta0 = (phs + ps) / wm;
        int64_t calls = 0;
        double beta;
        if (decision(&T, k, 0.0, w, pp, a, b, c, NULL, NULL) == k) {
            beta = 0.0;
            ++calls;
        } else {
            ++calls;
            double lo = 0.0;
            double hi = isfinite(beta0) && beta0 > 0.0 ? beta0 : 1.0;
            int ok = 0;
            for (int t = 0; t < 2100; ++t) {
                ++calls;
                if (decision(&T, k, hi, w, pp, a, b, c, NULL, NULL) == k) { ok = 1; break; }
                lo = hi;
                if (hi >= 1.0e308) break;
                hi = hi * 2.0;
                if (!isfinite(hi)) hi = 1.7976931348623157e308;
            }
            if (!ok) { rc = -3; goto out; }
            if (alpha0 > lo && alpha0 < hi) {
                ++calls;
                if (decision(&T, k, alpha0, w, pp, a, b, c, NULL, NULL) == k) hi = alpha0;
                else lo = alpha0;
            }
            uint64_t lb = dbits(lo), hb = dbits(hi);
            while (hb - lb > 1) {
                uint64_t mb = lb + (hb - lb) / 2;
                ++calls;
                if (decision(&T, k, bitsd(mb), w, pp, a, b, c, NULL, NULL) == k) hb = mb;
                else lb = mb;
            }
            beta = bitsd(hb);
        }
        /* Final call of Algorithm 1 at beta: the minimising subpartition */
        int64_t j = decision(&T, k, beta, w, pp, a, b, c, labels, ratio);
        ++calls;
        if (j != k) { rc = -3; goto out; }
        double cost = ratio[0];
        for (int64_t q = 1; q < k; ++q) if (ratio[q] > cost) cost = ratio[q];
        *i_k = cost;
        *beta_out = beta;
        for (int64_t v = 0; v < n; ++v) residual[v] = labels[v] < 0 ? 1 : 0;
        if (stats) {
            stats[0] = phs; stats[1] = phm; stats[2] = ws; stats[3] = wm;
            stats[4] = ps; stats[5] = pm; stats[6] = alpha0; stats[7] = beta0;
        }
        if (info) info[0] = calls;
    }
out:
    free(order); free(w); free(pp); free(a); free(b); free(c); free(ratio);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Section 2.2 steps 1-5 end to end.  omega_mode 0 = eq. omega over all
 * pairs, 1 = sum of phi over the incident tree edges (reading R2).
 * Outputs the tree (parent, phi_par), omega, p, labels, residual, i_k, beta
 * and the n-1 MST edges sorted by key. */
int oracle_cluster(const double *X, int64_t n, int32_t d, int64_t k, double sigma,
                   double alpha, int32_t omega_mode, int32_t include_self, int64_t root,
                   int32_t *eu, int32_t *ev, double *ed2,
                   int32_t *parent, double *phi_par, double *omega, double *p,
                   int32_t *labels, uint8_t *residual, double *i_k, double *beta,
                   double *stats, int64_t *info)
{
    if (n < 2 || d < 1 || k < 1 || k > n || !(sigma > 0.0)) return -1;
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!depth) return -2;
    int rc = oracle_mst_prim(X, n, d, root, eu, ev, ed2, parent, depth);
    free(depth);
    if (rc) return rc;
    /* phi of each tree edge, stored at the child vertex (parent list A, W) */
    for (int64_t v = 0; v < n; ++v)
        phi_par[v] = parent[v] >= 0 ? flow_of_d2(oracle_d2(X, n, d, v, parent[v]), sigma) : 0.0;
    if (omega_mode == 0) {
        oracle_weights(X, n, d, sigma, alpha, include_self, NULL, 0, omega, p);
    } else {
        double *om_dummy = (double *)malloc(sizeof(double) * n);
        if (!om_dummy) return -2;
        oracle_weights(X, n, d, sigma, alpha, include_self, NULL, 0, om_dummy, p);
        free(om_dummy);
        /* omega_i = sum of phi over tree edges incident to i, ascending neighbour */
        for (int64_t v = 0; v < n; ++v) omega[v] = include_self ? 1.0 : 0.0;
        edge_t *E = (edge_t *)malloc(sizeof(edge_t) * 2 * (n - 1));
        if (!E) return -2;
        for (int64_t e = 0; e < n - 1; ++e) {
            E[2 * e].u = eu[e]; E[2 * e].v = ev[e]; E[2 * e].d2 = ed2[e];
            E[2 * e + 1].u = ev[e]; E[2 * e + 1].v = eu[e]; E[2 * e + 1].d2 = ed2[e];
        }
        {
            /* counting sort by owner, then neighbours ascending within owner */
            int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
            int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * 2 * (n - 1));
            double *nd = (double *)malloc(sizeof(double) * 2 * (n - 1));
            if (!cnt || !nb || !nd) { free(cnt); free(nb); free(nd); free(E); return -2; }
            for (int64_t e = 0; e < 2 * (n - 1); ++e) cnt[E[e].u + 1]++;
            for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
            int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
            memcpy(fill, cnt, sizeof(int64_t) * (n + 1));
            for (int64_t e = 0; e < 2 * (n - 1); ++e) { nb[fill[E[e].u]] = E[e].v; nd[fill[E[e].u]++] = E[e].d2; }
            for (int64_t v = 0; v < n; ++v) {
                /* insertion sort of v's neighbour list by index */
                for (int64_t x = cnt[v] + 1; x < cnt[v + 1]; ++x) {
                    int32_t kb = nb[x]; double kd = nd[x]; int64_t y = x - 1;
                    while (y >= cnt[v] && nb[y] > kb) { nb[y + 1] = nb[y]; nd[y + 1] = nd[y]; --y; }
                    nb[y + 1] = kb; nd[y + 1] = kd;
                }
                double s = omega[v];
                for (int64_t x = cnt[v]; x < cnt[v + 1]; ++x) s = s + flow_of_d2(nd[x], sigma);
                omega[v] = s;
            }
            free(cnt); free(nb); free(nd); free(fill);
        }
        free(E);
    }
    return oracle_tree_stage(n, parent, phi_par, omega, alpha != 0.0 ? p : NULL, k,
                             labels, residual, i_k, beta, stats, info);
}

/* ------------------------------------------------------------------ */
/* i_k through a fixed structure, and its derivative.
 *
 * With alpha = 0 (p = 0) the cost of a k-subpartition (Section 2.1) is
 * max_j phi(dA_j) / omega(A_j): dA_j are the tree edges with exactly one
 * end in A_j (phi of eq. phi on each), omega(A_j) is the sum of eq. omega
 * over A_j.  The points enter as z_i = s (.) x_i, a per-feature scale s, and
 * the bandwidth sigma enters eq. phi and eq. omega.  Holding the tree
 * (parent) and the subpartition (labels; A_j = {v : labels[v] == j}) fixed,
 * i_k = R = Phi / Omega for the set A* of the largest ratio, and
 *   dR = (dPhi - R dOmega) / Omega,
 *   phi(e) = exp(-r_e / sigma), r_e = ||z_u - z_v||,
 *     d phi / d z_u = -phi (z_u - z_v) / (sigma r_e) = -d phi / d z_v,
 *     d phi / d sigma = phi r_e / sigma^2,
 *   Omega = sum_{i in A*} sum_{j != i} w_ij, w_ij = exp(-r_ij / sigma): each
 *     ordered pair (i in A*, j) adds -w (z_i - z_j) / (sigma r) to d/dz_i,
 *     the opposite to d/dz_j, and w r / sigma^2 to d/dsigma.
 * Chain rule to the inputs: dR/dx_it = s_t dR/dz_it, dR/ds_t = sum_i x_it dR/dz_it.
 * Coincident points (r = 0) are not differentiable; their terms are taken
 * as 0 (the direction is undefined). */
static double zdist(const double *X, const double *s, int32_t d, int64_t i, int64_t j)
{
    double acc = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double dz = s[t] * X[i * (int64_t)d + t] - s[t] * X[j * (int64_t)d + t];
        acc = acc + dz * dz;
    }
    return sqrt(acc);
}

/* Phi_j, Omega_j of every label 0..k-1 and R = the largest ratio; jstar is
 * the smallest label with that ratio. */
int oracle_ik_fixed(const double *X, int64_t n, int32_t d, const double *s, double sigma,
                    const int32_t *parent, const int32_t *labels, int64_t k,
                    double *phi_k, double *omega_k, int32_t *jstar, double *R)
{
    if (n < 1 || d < 1 || k < 1 || !(sigma > 0.0)) return -1;
    for (int64_t j = 0; j < k; ++j) { phi_k[j] = 0.0; omega_k[j] = 0.0; }
    for (int64_t v = 0; v < n; ++v) {           /* boundary edges: one end in A_j */
        int64_t u = parent[v];
        if (u < 0) continue;
        int32_t a = labels[v], b = labels[u];
        if (a == b) continue;
        double f = exp(-zdist(X, s, d, v, u) / sigma);
        if (a >= 0 && a < k) phi_k[a] = phi_k[a] + f;
        if (b >= 0 && b < k) phi_k[b] = phi_k[b] + f;
    }
    double *om = (double *)malloc(sizeof(double) * n);
    if (!om) return -2;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {            /* eq. omega of each labelled point */
        om[i] = 0.0;
        if (labels[i] < 0 || labels[i] >= k) continue;
        double w = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) w = w + exp(-zdist(X, s, d, i, j) / sigma);
        om[i] = w;
    }
    for (int64_t i = 0; i < n; ++i)
        if (labels[i] >= 0 && labels[i] < k) omega_k[labels[i]] = omega_k[labels[i]] + om[i];
    free(om);
    int32_t best = 0;
    for (int64_t j = 1; j < k; ++j)
        if (phi_k[j] / omega_k[j] > phi_k[best] / omega_k[best]) best = (int32_t)j;
    *jstar = best;
    *R = phi_k[best] / omega_k[best];
    return 0;
}

/* dR/dX (n x d), dR/ds (d), dR/dsigma for the set jstar, and R itself. */
int oracle_ik_grad(const double *X, int64_t n, int32_t d, const double *s, double sigma,
                   const int32_t *parent, const int32_t *labels, int32_t jstar,
                   double *dX, double *ds, double *dsigma, double *R)
{
    if (n < 1 || d < 1 || !(sigma > 0.0)) return -1;
    double *gphi = (double *)calloc((size_t)n * d, sizeof(double));   /* dPhi/dz */
    double *gom = (double *)calloc((size_t)n * d, sizeof(double));    /* dOmega/dz */
    double *rowsig = (double *)calloc((size_t)n, sizeof(double));
    double *rowom = (double *)calloc((size_t)n, sizeof(double));
    if (!gphi || !gom || !rowsig || !rowom) { free(gphi); free(gom); free(rowsig); free(rowom); return -2; }
    double Phi = 0.0, dPhi_sig = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t u = parent[v];
        if (u < 0) continue;
        if ((labels[v] == jstar) == (labels[u] == jstar)) continue;     /* not in dA* */
        double r = zdist(X, s, d, v, u);
        double f = exp(-r / sigma);
        Phi = Phi + f;
        dPhi_sig = dPhi_sig + f * r / (sigma * sigma);
        if (r > 0.0) {
            double c = -f / (sigma * r);
            for (int32_t t = 0; t < d; ++t) {
                double dz = s[t] * X[v * (int64_t)d + t] - s[t] * X[u * (int64_t)d + t];
                gphi[v * (int64_t)d + t] = gphi[v * (int64_t)d + t] + c * dz;
                gphi[u * (int64_t)d + t] = gphi[u * (int64_t)d + t] - c * dz;
            }
        }
    }
    /* Omega: rows of A* collect their own terms; every row collects the
     * terms where it is the partner j (two passes keep each row's sum in a
     * fixed order) */
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double *g = gom + i * (int64_t)d;
        double sw = 0.0, sg = 0.0;
        const int in_i = labels[i] == jstar;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const int in_j = labels[j] == jstar;
            if (!in_i && !in_j) continue;
            double r = zdist(X, s, d, i, j);
            double w = exp(-r / sigma);
            if (in_i) { sw = sw + w; sg = sg + w * r / (sigma * sigma); }
            if (r > 0.0) {
                /* (i in A*, j): -w/(sigma r) (z_i - z_j) on z_i;
                 * (j in A*, i): -w/(sigma r) (z_j - z_i) on z_i as the partner */
                double c = -w / (sigma * r) * (double)(in_i + in_j);
                for (int32_t t = 0; t < d; ++t) {
                    double dz = s[t] * X[i * (int64_t)d + t] - s[t] * X[j * (int64_t)d + t];
                    g[t] = g[t] + c * dz;
                }
            }
        }
        rowom[i] = sw;
        rowsig[i] = sg;
    }
    double Omega = 0.0, dOm_sig = 0.0;
    for (int64_t i = 0; i < n; ++i) { Omega = Omega + rowom[i]; dOm_sig = dOm_sig + rowsig[i]; }
    double Rv = Phi / Omega;
    for (int32_t t = 0; t < d; ++t) ds[t] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = 0; t < d; ++t) {
            double gz = (gphi[i * (int64_t)d + t] - Rv * gom[i * (int64_t)d + t]) / Omega;
            dX[i * (int64_t)d + t] = gz * s[t];
            ds[t] = ds[t] + gz * X[i * (int64_t)d + t];
        }
    *dsigma = (dPhi_sig - Rv * dOm_sig) / Omega;
    *R = Rv;
    free(gphi); free(gom); free(rowsig); free(rowom);
    return 0;
}

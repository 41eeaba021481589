"""Pins of the FP64 oracle against things other than itself.

Each test targets a plausible mistake (dropped term, wrong sign or index,
transposed operand, wrong order) and checks the oracle against a closed form,
brute force over the paper's definitions, an independent library routine,
higher precision, or an invariant of the method.
"""
import json
import math
import os

import numpy as np
import pytest

from _brute import edge_flow_map, miso_bruteforce, phi_for_parent, random_tree, reroot

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- distance key
def test_d2_integer_points_exact(oracle_lib):
    """Integer coordinates: d2 is an exact integer, computed here with Python ints."""
    rng = np.random.default_rng(3)
    X = rng.integers(-1000, 1000, size=(20, 7))
    for i in range(20):
        for j in range(20):
            want = sum((int(a) - int(b)) ** 2 for a, b in zip(X[i], X[j]))
            assert oracle_lib.d2(X, i, j) == float(want)


def test_d2_f32_inputs_same_as_f64(oracle_lib):
    """f32 -> f64 is exact, so f32 inputs give the same keys as their f64 copy."""
    rng = np.random.default_rng(4)
    X32 = rng.normal(size=(10, 5)).astype(np.float32)
    X64 = X32.astype(np.float64)
    for i in range(10):
        for j in range(10):
            assert oracle_lib.d2(X32, i, j) == oracle_lib.d2(X64, i, j)


# ---------------------------------------------------------------- MST
def _cut_property_ok(X, eu, ev, ed2, d2fn):
    """Every tree edge is the minimum-key edge across the cut it defines."""
    n = X.shape[0]
    adj = [[] for _ in range(n)]
    for a, b in zip(eu, ev):
        adj[a].append(b); adj[b].append(a)
    for e, (a, b) in enumerate(zip(eu, ev)):
        side = np.zeros(n, bool)
        stack = [a]; side[a] = True
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if (u, w) in ((a, b), (b, a)):
                    continue
                if not side[w]:
                    side[w] = True; stack.append(w)
        best = None
        for i in np.nonzero(side)[0]:
            for j in np.nonzero(~side)[0]:
                k = (d2fn(i, j), min(i, j), max(i, j))
                if best is None or k < best:
                    best = k
        if best != (ed2[e], min(a, b), max(a, b)):
            return False
    return True


@pytest.mark.parametrize("seed", range(4))
def test_prim_equals_kruskal_and_cut_property(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    X = rng.normal(size=(n, 3))
    eu, ev, ed2, parent, depth = oracle_lib.mst_prim(X)
    ku, kv, kd = oracle_lib.mst_kruskal(X)
    assert (eu == ku).all() and (ev == kv).all() and (ed2 == kd).all()
    assert _cut_property_ok(X, eu, ev, ed2, lambda i, j: oracle_lib.d2(X, i, j))


def test_mst_with_exact_ties_tie_break(oracle_lib):
    """Integer grid points have many equal d2: the (d2, min, max) order decides."""
    rng = np.random.default_rng(11)
    X = rng.integers(-2, 3, size=(30, 2)).astype(np.float64)
    X = np.unique(X, axis=0)
    rng.shuffle(X)
    eu, ev, ed2, _, _ = oracle_lib.mst_prim(X)
    ku, kv, kd = oracle_lib.mst_kruskal(X)
    assert (eu == ku).all() and (ev == kv).all()
    assert _cut_property_ok(X, eu, ev, ed2, lambda i, j: oracle_lib.d2(X, i, j))


def test_mst_matches_scipy(oracle_lib):
    """Independent library MST (scipy.sparse.csgraph) on distinct distances."""
    sp = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(5)
    X = rng.normal(size=(120, 6))
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    T = sp.minimum_spanning_tree(D).tocoo()
    want = sorted((min(a, b), max(a, b)) for a, b in zip(T.row, T.col))
    eu, ev, ed2, _, _ = oracle_lib.mst_prim(X)
    got = sorted(zip(eu.tolist(), ev.tolist()))
    assert got == want
    assert math.isclose(float(np.sqrt(ed2).sum()), float(T.data.sum()), rel_tol=1e-12)


def test_mst_on_a_line_is_the_chain(oracle_lib):
    rng = np.random.default_rng(6)
    xs = np.cumsum(rng.uniform(0.1, 2.0, size=30))
    perm = rng.permutation(30)
    X = xs[perm][:, None]
    eu, ev, ed2, parent, depth = oracle_lib.mst_prim(X, root=0)
    pos = np.argsort(xs[perm])
    want = sorted((min(pos[i], pos[i + 1]), max(pos[i], pos[i + 1])) for i in range(29))
    assert sorted(zip(eu.tolist(), ev.tolist())) == want


def test_prim_parent_depth_consistent(oracle_lib):
    rng = np.random.default_rng(7)
    X = rng.normal(size=(60, 4))
    for root in (0, 17, 59):
        eu, ev, ed2, parent, depth = oracle_lib.mst_prim(X, root=root)
        assert parent[root] == -1 and depth[root] == 0
        es = set(zip(eu.tolist(), ev.tolist()))
        for v in range(60):
            if v != root:
                assert (min(v, parent[v]), max(v, parent[v])) in es
                assert depth[v] == depth[parent[v]] + 1


def test_nn_rows_is_min_key(oracle_lib):
    rng = np.random.default_rng(8)
    X = rng.integers(-3, 4, size=(50, 2)).astype(np.float64)
    rows = np.arange(50)
    nn, nd = oracle_lib.nn_rows(X, rows)
    for i in rows:
        cands = [(oracle_lib.d2(X, i, j), min(i, j), max(i, j), j) for j in range(50) if j != i]
        best = min(cands)
        assert nn[i] == best[3] and nd[i] == best[0]


# ---------------------------------------------------------------- weights
def test_omega_closed_form_on_equally_spaced_line(oracle_lib):
    """x_i = i*h: omega_i = sum_{m=1}^{i} r^m + sum_{m=1}^{n-1-i} r^m, r = exp(-h/sigma)."""
    n, h, sigma = 40, 0.37, 1.3
    X = (np.arange(n) * h)[:, None]
    om, p = oracle_lib.weights(X, sigma, alpha=0.5)
    r = math.exp(-h / sigma)
    for i in range(n):
        a, b = i, n - 1 - i
        want = r * (1 - r ** a) / (1 - r) + r * (1 - r ** b) / (1 - r)
        assert math.isclose(om[i], want, rel_tol=1e-13)
        want_p = 0.5 * h * (a * (a + 1) / 2 + b * (b + 1) / 2)
        assert math.isclose(p[i], want_p, rel_tol=1e-13)


def test_omega_two_points_and_self_term(oracle_lib):
    X = np.array([[0.0, 0.0], [3.0, 4.0]])
    om, p = oracle_lib.weights(X, 2.0, alpha=1.0)
    assert math.isclose(om[0], math.exp(-2.5), rel_tol=1e-15) and om[0] == om[1]
    assert p[0] == 5.0 and p[1] == 5.0
    om2, p2 = oracle_lib.weights(X, 2.0, alpha=1.0, include_self=True)
    assert math.isclose(om2[0], 1.0 + math.exp(-2.5), rel_tol=1e-15)
    assert p2[0] == 5.0


def test_omega_against_long_double(oracle_lib):
    rng = np.random.default_rng(9)
    X = rng.normal(size=(64, 5)).astype(np.float32)
    om, _ = oracle_lib.weights(X, 0.7)
    Xl = X.astype(np.longdouble)
    for i in range(64):
        diff = Xl - Xl[i]
        dist = np.sqrt((diff * diff).sum(axis=1))
        terms = np.exp(-dist / np.longdouble(0.7))
        want = terms.sum() - terms[i]
        assert abs(float(om[i]) - float(want)) <= 1e-14 * float(want)


def test_omega_row_subset_matches_full(oracle_lib):
    rng = np.random.default_rng(10)
    X = rng.normal(size=(80, 3))
    om, p = oracle_lib.weights(X, 1.0, alpha=0.3)
    rows = np.array([5, 0, 79, 33])
    om_s, p_s = oracle_lib.weights(X, 1.0, alpha=0.3, rows=rows)
    assert (om_s == om[rows]).all() and (p_s == p[rows]).all()


# ---------------------------------------------------------------- tree stage
def _random_weights(rng, parent, with_p):
    n = parent.size
    phi = np.where(parent >= 0, rng.uniform(0.05, 1.0, n), 0.0)
    om = rng.uniform(0.5, 3.0, n)
    p = rng.uniform(0.0, 0.5, n) if with_p else None
    return phi, om, p


@pytest.mark.parametrize("shape", ["random", "path", "star", "caterpillar"])
@pytest.mark.parametrize("with_p", [False, True])
def test_tree_stage_equals_bruteforce_miso(oracle_lib, shape, with_p):
    rng = np.random.default_rng(hash((shape, with_p)) % 2**32)
    for _ in range(25):
        n = int(rng.integers(1, 9))
        kmax = max(k for k in range(1, n + 1) if (k + 1) ** n <= 400_000)
        k = int(rng.integers(1, kmax + 1))
        parent = random_tree(rng, n, shape)
        phi, om, p = _random_weights(rng, parent, with_p)
        r = oracle_lib.tree_stage(parent, phi, om, p, k)
        b = miso_bruteforce(parent, phi, om, p, k)
        assert math.isclose(r["i_k"], b, rel_tol=1e-12, abs_tol=1e-300), (n, k, r["i_k"], b)


def test_tree_stage_bruteforce_n11(oracle_lib):
    rng = np.random.default_rng(123)
    for k in (2, 3):
        parent = random_tree(rng, 11, "random")
        phi, om, p = _random_weights(rng, parent, True)
        r = oracle_lib.tree_stage(parent, phi, om, p, k)
        assert math.isclose(r["i_k"], miso_bruteforce(parent, phi, om, p, k), rel_tol=1e-12)


def test_hand_derived_golden_trees(oracle_lib):
    with open(os.path.join(HERE, "golden", "hand_trees.json")) as f:
        g = json.load(f)
    for c in g["cases"]:
        for k, want in c["miso"].items():
            r = oracle_lib.tree_stage(c["parent"], c["phi_par"], c["omega"], None, int(k))
            assert math.isclose(r["i_k"], want, rel_tol=1e-15, abs_tol=1e-300), (c["name"], k)


def test_path_closed_form_k2(oracle_lib):
    """Uniform path P_n, p = 0: MISO_2 = phi / (floor(n/2) * w)."""
    for n in (2, 3, 10, 101, 1000):
        parent = np.arange(-1, n - 1, dtype=np.int32)
        phi = np.full(n, 0.3); phi[0] = 0.0
        om = np.full(n, 1.7)
        r = oracle_lib.tree_stage(parent, phi, om, None, 2)
        assert math.isclose(r["i_k"], 0.3 / ((n // 2) * 1.7), rel_tol=1e-12)


def test_star_closed_forms(oracle_lib):
    """Uniform star, m leaves: MISO_k = phi/w_leaf (2<=k<=m), MISO_{m+1} = max(phi/w_leaf, m phi/w_c)."""
    m, f, wl, wc = 9, 0.4, 1.5, 2.0
    parent = np.array([-1] + [0] * m, dtype=np.int32)
    phi = np.array([0.0] + [f] * m)
    om = np.array([wc] + [wl] * m)
    for k in range(2, m + 1):
        assert math.isclose(oracle_lib.tree_stage(parent, phi, om, None, k)["i_k"], f / wl, rel_tol=1e-12)
    r = oracle_lib.tree_stage(parent, phi, om, None, m + 1)
    assert math.isclose(r["i_k"], max(f / wl, m * f / wc), rel_tol=1e-12)


def test_k1_whole_set_and_k_eq_n_singletons(oracle_lib):
    rng = np.random.default_rng(12)
    parent = random_tree(rng, 30, "random")
    phi, om, _ = _random_weights(rng, parent, False)
    r1 = oracle_lib.tree_stage(parent, phi, om, None, 1)
    assert r1["i_k"] == 0.0 and (r1["labels"] == 0).all()
    rn = oracle_lib.tree_stage(parent, phi, om, None, 30)
    bnd = np.zeros(30)
    for v in range(30):
        if parent[v] >= 0:
            bnd[v] += phi[v]; bnd[parent[v]] += phi[v]
    assert math.isclose(rn["i_k"], float((bnd / om).max()), rel_tol=1e-12)
    assert sorted(rn["labels"].tolist()) == list(range(30))


def test_miso_is_root_independent(oracle_lib):
    rng = np.random.default_rng(13)
    for _ in range(10):
        parent = random_tree(rng, 40, "random")
        phi, om, p = _random_weights(rng, parent, True)
        emap = edge_flow_map(parent, phi)
        k = int(rng.integers(1, 8))
        base = oracle_lib.tree_stage(parent, phi, om, p, k)["i_k"]
        for new_root in rng.choice(40, size=3, replace=False):
            par2 = reroot(parent, int(new_root))
            r = oracle_lib.tree_stage(par2, phi_for_parent(par2, emap), om, p, k)
            assert math.isclose(r["i_k"], base, rel_tol=1e-12)


def test_decision_monotone_and_beta_is_the_boundary(oracle_lib):
    rng = np.random.default_rng(14)
    for _ in range(20):
        n = int(rng.integers(2, 60))
        parent = random_tree(rng, n, "random")
        phi, om, p = _random_weights(rng, parent, bool(rng.integers(0, 2)))
        k = int(rng.integers(1, n + 1))
        r = oracle_lib.tree_stage(parent, phi, om, p, k)
        beta = r["beta"]
        assert oracle_lib.decision(parent, phi, om, p, k, beta) == k
        if beta > 0:
            assert oracle_lib.decision(parent, phi, om, p, k, np.nextafter(beta, 0.0)) < k
        grid = np.sort(np.concatenate([rng.uniform(0, 2 * beta + 1e-9, 40), [beta]]))
        yes = [oracle_lib.decision(parent, phi, om, p, k, float(N)) == k for N in grid]
        first = yes.index(True)
        assert all(yes[first:])


def test_returned_sets_are_a_valid_subpartition(oracle_lib):
    """Labels give k disjoint non-empty sets whose ratios (from the definitions) are <= beta."""
    rng = np.random.default_rng(15)
    for _ in range(15):
        n = int(rng.integers(3, 80))
        parent = random_tree(rng, n, "random")
        phi, om, p = _random_weights(rng, parent, True)
        k = int(rng.integers(1, min(n, 8) + 1))
        r = oracle_lib.tree_stage(parent, phi, om, p, k)
        lab = r["labels"]
        assert ((lab >= -1) & (lab < k)).all()
        assert (r["residual"] == (lab < 0)).all()
        worst = 0.0
        for j in range(k):
            A = lab == j
            assert A.any()
            bnd = sum(phi[v] for v in range(n) if parent[v] >= 0 and A[v] != A[parent[v]])
            ratio = (bnd + p[A].sum()) / om[A].sum()
            assert ratio <= r["beta"] * (1 + 1e-12)
            worst = max(worst, ratio)
        assert math.isclose(worst, r["i_k"], rel_tol=1e-12)


def test_cluster_pipeline_consistent_with_stages(oracle_lib):
    rng = np.random.default_rng(16)
    X = rng.normal(size=(150, 4))
    c = oracle_lib.cluster(X, 4, 0.8)
    eu, ev, ed2, parent, _ = oracle_lib.mst_prim(X)
    assert (c["edge_u"] == eu).all() and (c["parent"] == parent).all()
    om, _ = oracle_lib.weights(X, 0.8)
    assert (c["omega"] == om).all()
    phi = np.array([oracle_lib.flow(oracle_lib.d2(X, v, parent[v]), 0.8) if parent[v] >= 0 else 0.0
                    for v in range(150)])
    assert (c["phi_par"] == phi).all()
    t = oracle_lib.tree_stage(parent, phi, om, None, 4)
    assert t["i_k"] == c["i_k"] and (t["labels"] == c["labels"]).all()


def test_cluster_scale_invariance_bitwise(oracle_lib):
    """X -> 2X and sigma -> 2 sigma scale d2 by 4 exactly: identical outputs."""
    rng = np.random.default_rng(17)
    X = rng.normal(size=(120, 3))
    a = oracle_lib.cluster(X, 3, 0.9)
    b = oracle_lib.cluster(2 * X, 3, 1.8)
    assert a["i_k"] == b["i_k"] and (a["labels"] == b["labels"]).all()


def test_cluster_permutation_invariance(oracle_lib):
    rng = np.random.default_rng(18)
    X = rng.normal(size=(100, 3))
    perm = rng.permutation(100)
    a = oracle_lib.cluster(X, 3, 1.0, root=int(np.argmin(perm)))  # same root point
    b = oracle_lib.cluster(X[perm], 3, 1.0, root=0)
    assert math.isclose(a["i_k"], b["i_k"], rel_tol=1e-12)
    la, lb = a["labels"][perm], b["labels"]
    assert ((la < 0) == (lb < 0)).all()
    pairs = {(int(x), int(y)) for x, y in zip(la, lb) if x >= 0}
    assert len(pairs) == len({x for x, _ in pairs}) == len({y for _, y in pairs})


def test_tree_omega_mode(oracle_lib):
    rng = np.random.default_rng(19)
    X = rng.normal(size=(50, 3))
    c = oracle_lib.cluster(X, 3, 1.0, omega_mode=1)
    deg_sum = np.zeros(50)
    for v in range(50):
        if c["parent"][v] >= 0:
            deg_sum[v] += c["phi_par"][v]; deg_sum[c["parent"][v]] += c["phi_par"][v]
    assert np.allclose(c["omega"], deg_sum, rtol=1e-14, atol=0)


def test_malformed_tree_rejected(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.bfs_order([1, 0, -1])          # cycle 0 <-> 1 disconnected from root 2
    with pytest.raises(ValueError):
        oracle_lib.bfs_order([-1, -1, 0])         # two roots


# ---------------------------------------------------------------- label order (readings A5-A8)
def _label_order_cases():
    with open(os.path.join(HERE, "golden", "label_order_trees.json")) as f:
        return json.load(f)


def test_bfs_order_hand_written(oracle_lib):
    """A hand-written breadth-first order (children ascending) on an unsorted
    tree: a depth-first order or descending children fail it."""
    for c in _label_order_cases()["bfs_cases"]:
        assert oracle_lib.bfs_order(c["parent"]).tolist() == c["bfs"], c["name"]


@pytest.mark.parametrize("case", [c["name"] for c in _label_order_cases()["label_cases"]])
def test_label_order_hand_derived(oracle_lib, case):
    """Which k sets Algorithm 1 returns and how they are numbered: ascending
    children in the BFS, the reversed walk, the first k cuts numbered j-1,
    and the descending-index fold of omega-hat (hand-derived expectations)."""
    c = next(x for x in _label_order_cases()["label_cases"] if x["name"] == case)
    r = oracle_lib.tree_stage(c["parent"], c["phi_par"], c["omega"], None, c["k"])
    assert r["labels"].tolist() == c["labels"]
    assert r["i_k"] == c["i_k"]
    if "beta" in c:
        assert r["beta"] == c["beta"]


# ---------------------------------------------------------------- decision margins
def _set_ratio(parent, phi, om, p, A):
    n = parent.size
    bnd = sum(phi[v] for v in range(n) if parent[v] >= 0 and A[v] != A[parent[v]])
    return (bnd + (p[A].sum() if p is not None else 0.0)) / om[A].sum()


@pytest.mark.parametrize("with_p", [False, True])
def test_decision_detail_agrees_with_definitions(oracle_lib, with_p):
    """At beta: the cut vertices, in walking order, head the sets 0..k-1; a
    cut vertex's critical ratio is its set's ratio from the definitions
    (eq. cost); every branch taken agrees with its critical ratios; some
    vertex sits at beta (beta is the YES/NO boundary)."""
    rng = np.random.default_rng(20 + with_p)
    for _ in range(20):
        n = int(rng.integers(2, 70))
        parent = random_tree(rng, n, "random")
        phi, om, p = _random_weights(rng, parent, with_p)
        k = int(rng.integers(1, min(n, 9) + 1))
        r = oracle_lib.tree_stage(parent, phi, om, p, k)
        beta, lab = r["beta"], r["labels"]
        det = oracle_lib.decision_detail(parent, phi, om, p, k, beta)
        assert det["cuts"] == k
        order = oracle_lib.bfs_order(parent)[::-1]
        visited = [int(x) for x in order if det["code"][x] >= 0]
        cuts = [x for x in visited if det["code"][x] == 0]
        assert len(cuts) == k
        for j, x in enumerate(cuts):
            assert lab[x] == j
            want = _set_ratio(parent, phi, om, p, lab == j)
            assert math.isclose(det["ncut"][x], want, rel_tol=1e-13)
        eps = 4e-16
        closest = np.inf
        for x in visited:
            c, nc, nj = det["code"][x], det["ncut"][x], det["njoin"][x]
            if c == 0:
                assert nc <= beta * (1 + eps)
            elif c == 1:
                assert nc > beta * (1 - eps) and nj < beta * (1 + eps)
                assert parent[x] >= 0 and lab[x] == lab[parent[x]]
            else:
                assert nc > beta * (1 - eps) and nj >= beta * (1 - eps)
            if beta > 0:
                closest = min(closest, abs(nc - beta) / beta, abs(nj - beta) / beta)
        if beta > 0:
            assert closest <= 1e-15
        assert (det["code"][[v for v in range(n) if v not in visited]] == -1).all()


def test_decision_detail_hand_trees(oracle_lib):
    """The two-level hand tree at beta = 1/2: leaves 6, 5, 4 cut with ratio
    exactly 1/2 (phi 1 over omega 2); the walk stops after the third cut."""
    c = next(x for x in _label_order_cases()["label_cases"] if x["name"] == "two_levels_bfs_not_dfs")
    det = oracle_lib.decision_detail(c["parent"], c["phi_par"], c["omega"], None, c["k"], c["beta"])
    assert det["cuts"] == 3
    assert det["code"].tolist() == [-1, -1, -1, -1, 0, 0, 0]
    assert det["ncut"][4] == det["ncut"][5] == det["ncut"][6] == 0.5
    assert det["njoin"][6] == -0.5


def test_parent_flow_matches_the_pipeline(oracle_lib):
    """phi on parent edges equals the per-pair flow of the same d2 and the
    pipeline's own phi_par."""
    rng = np.random.default_rng(22)
    X = rng.normal(size=(90, 5)).astype(np.float32)
    c = oracle_lib.cluster(X, 3, 0.7)
    pf = oracle_lib.parent_flow(X, c["parent"], 0.7)
    assert (pf == c["phi_par"]).all()
    v = int(np.nonzero(c["parent"] >= 0)[0][0])
    assert pf[v] == math.exp(-math.sqrt(oracle_lib.d2(X, v, int(c["parent"][v]))) / 0.7)


def test_min_foreign_is_nearest_neighbour_then_boruvka_equals_prim(oracle_lib):
    """With every point its own component the step gives the nearest
    neighbours; Boruvka rounds built on it give Prim's tree."""
    rng = np.random.default_rng(23)
    X = rng.normal(size=(70, 3))
    n = X.shape[0]
    rows = np.arange(n)
    j, d2 = oracle_lib.min_foreign(X, np.arange(n), rows)
    nn, nd = oracle_lib.nn_rows(X, rows)
    assert (j == nn).all() and (d2 == nd).all()
    comp = np.arange(n)
    edges = set()
    while len(set(comp.tolist())) > 1:
        j, d2 = oracle_lib.min_foreign(X, comp, rows)
        best = {}
        for i in range(n):
            key = (d2[i], min(i, j[i]), max(i, j[i]))
            if comp[i] not in best or key < best[comp[i]]:
                best[comp[i]] = key
        for _, a, b in best.values():
            edges.add((a, b))
        # merge along the chosen edges
        p = {c: c for c in set(comp.tolist())}

        def f(x):
            while p[x] != x:
                x = p[x]
            return x
        for _, a, b in best.values():
            ra, rb = f(comp[a]), f(comp[b])
            if ra != rb:
                p[max(ra, rb)] = min(ra, rb)
        comp = np.array([f(c) for c in comp])
    eu, ev, _, _, _ = oracle_lib.mst_prim(X)
    assert edges == set(zip(eu.tolist(), ev.tolist()))

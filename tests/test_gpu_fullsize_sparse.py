"""Full-size parity on the 50,000-point, d = 4,096 sparse-like workload
(non-negative log-normal values at 1% density, 10 groups, rows
L2-normalised), through isoclust_cluster_detail with default options.  The
tensor-core sweep streams both operands here (64 K-chunks of 64).  Sampled
outputs against the oracle plus properties that hold at any size."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1702_04739_gb300 import isoclust, workloads
    oracle.build()
    oracle.set_threads(16)
    X, k, sigma = workloads.make("sparse_n50k_d4096", seed=0)
    out = isoclust.cluster_detail(torch.from_numpy(X).cuda(), k, sigma)
    host = {key: v.cpu().numpy() for key, v in out.items()}
    return dict(X=X, k=k, sigma=sigma, out=host, oracle=oracle)


def test_mst_structure_and_nearest_neighbours(run):
    o, X, orc = run["out"], run["X"], run["oracle"]
    n = X.shape[0]
    eu, ev, ed = o["edge_u"], o["edge_v"], o["edge_d2"]
    assert eu.size == n - 1 and (eu < ev).all()
    keys = list(zip(ed.tolist(), eu.tolist(), ev.tolist()))
    assert keys == sorted(keys)
    edges = {(int(a), int(b)): float(c) for a, b, c in zip(eu, ev, ed)}
    rows = np.random.default_rng(0).choice(n, size=48, replace=False)
    nn, nd2 = orc.nn_rows(X, rows)
    for i, j, dd in zip(rows, nn, nd2):
        key = (min(int(i), int(j)), max(int(i), int(j)))
        assert key in edges and edges[key] == dd
    # every tree edge's d2 is the canonical key of its endpoints
    for e in np.random.default_rng(1).choice(n - 1, size=48, replace=False):
        assert orc.d2(X, int(eu[e]), int(ev[e])) == ed[e]


def test_omega_sampled_rows(run):
    o, X, orc, sigma = run["out"], run["X"], run["oracle"], run["sigma"]
    rows = np.random.default_rng(2).choice(X.shape[0], size=24, replace=False)
    om, _ = orc.weights(X, sigma, rows=rows)
    nn, nd2 = orc.nn_rows(X, rows)
    # the renormalised double-word sum of d squares carries ~2^-48 sqrt(d)
    # relative error, so the d = 64 bound scales by sqrt(d / 64)
    tol = 2.0 ** -45 * math.sqrt(X.shape[1] / 64.0) * (np.sqrt(nd2) / sigma + 4.0)
    rel = np.abs(o["omega"][rows] - om) / om
    assert (rel <= tol).all(), rel.max()


def test_labels_valid_and_cost(run):
    o, k = run["out"], run["k"]
    lab, parent, phi, om = o["labels"], o["parent"], o["phi_par"], o["omega"]
    beta, ik = float(o["beta"][0]), float(o["i_k"][0])
    assert ((lab >= -1) & (lab < k)).all()
    nonroot = parent >= 0
    ratios = []
    for j in range(k):
        A = lab == j
        assert A.any()
        tops = np.nonzero(A & ~(nonroot & A[np.maximum(parent, 0)]))[0]
        assert tops.size == 1
        cross = nonroot & (A != A[np.maximum(parent, 0)])
        ratios.append(phi[cross].sum() / om[A].sum())
    assert max(ratios) <= beta * (1 + 1e-12)
    assert math.isclose(max(ratios), ik, rel_tol=1e-12)

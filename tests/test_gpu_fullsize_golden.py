"""Full-size parity: the CUDA path against the FP64 oracle on every benchmark
workload at its full size, element by element.

The oracle's results are stored under tests/golden/fullsize/ by
tests/golden/make_fullsize.py (oracle only; the largest runs take minutes to
tens of minutes of CPU time).  Each test regenerates the seeded input, checks
that it is byte-identical to the input the oracle saw, runs the library in the
benchmark's launch configuration and compares:
  * MST edges (u, v, d2) and parent: bit-exact (Section 2.2 step 2, the
    unique tree under the key (d2, min, max));
  * labels and residual: bit-exact (Algorithm 1 at beta, readings A5-A8);
  * i_k and beta: within 1e-12 relative (eq. MISO);
  * phi on the tree edges: within 4e-16 relative (one exp rounding);
  * omega: per row within the double-word bound of the parity tests, and the
    largest relative error is reported;
  * the decision margin: the smallest relative distance between beta and the
    critical threshold of any decision Algorithm 1 takes before its k-th cut
    (those at beta itself, which decide beta, are counted apart), reported
    beside the omega error it has to exceed for the labels to be stable.
The independent-set workload compares every set's tree and labels through
digests of the oracle's arrays, every set's i_k and beta, and the omega of 16
sets spread over the size range.
"""
import hashlib
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize")
SINGLE = ["blobs_n2000_d8", "moons_n20k_d128", "blobs_n100k_d64", "sparse_n50k_d4096"]
IK_RTOL = 1e-12
PHI_RTOL = 4e-16


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def golden(name):
    path = os.path.join(GOLD, name + ".npz")
    assert os.path.exists(path), f"missing golden {path} (tests/golden/make_fullsize.py writes it)"
    return dict(np.load(path, allow_pickle=False))


def omega_bound(n, d, eu, ev, ed2, sigma):
    """Per-row bound of the double-word omega (see test_gpu_parity.omega_tol),
    with each row's nearest-neighbour distance read from the tree's edges
    (every nearest-neighbour edge is a tree edge)."""
    nn = np.full(n, np.inf)
    np.minimum.at(nn, eu, ed2)
    np.minimum.at(nn, ev, ed2)
    y = np.sqrt(nn) / sigma
    return 2.0 ** -45 * max(1.0, math.sqrt(d / 64.0)) * (y + 4.0)


def decision_margin(orc, parent, phi, omega, k, beta):
    """(smallest relative margin of a decision not at beta, decisions at beta)."""
    det = orc.decision_detail(parent, phi, omega, None, k, beta)
    vis = det["code"] >= 0
    if beta <= 0:
        return math.inf, 0
    rel = np.minimum(np.abs(det["ncut"][vis] - beta), np.abs(det["njoin"][vis] - beta)) / beta
    at_beta = rel <= 1e-15
    return (float(rel[~at_beta].min()) if (~at_beta).any() else math.inf), int(at_beta.sum())


@pytest.fixture(scope="module")
def iso():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04739_gb300 import isoclust
    isoclust.load()
    return isoclust


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    oracle.set_threads(max(1, min(16, os.cpu_count() or 1)))
    return oracle


@pytest.mark.parametrize("name", SINGLE)
def test_single_set_against_oracle(iso, orc, parity_report, name):
    from paper_1702_04739_gb300 import workloads
    g = golden(name)
    X, k, sigma = workloads.make(name, seed=0)
    assert sha(X) == str(g["x_sha256"]), "the seeded input differs from the one the oracle saw"
    n, d = X.shape
    Xd = torch.from_numpy(X).cuda()
    if name.startswith("moons"):
        # the differentiable path's forward: z = scale (.) x with scale 1
        Xd = iso.scale_features(Xd, torch.ones(d, dtype=torch.float64, device="cuda"))
        assert torch.equal(Xd.cpu(), torch.from_numpy(X))
    out = {key: v.cpu().numpy() for key, v in iso.cluster_detail(Xd, k, sigma).items()}
    lab, res, ik = iso.cluster(Xd, k, sigma)
    # MST: bit-exact edge list in key order, and the rooted tree
    assert (out["edge_u"] == g["edge_u"]).all() and (out["edge_v"] == g["edge_v"]).all(), "MST edges differ"
    assert (out["edge_d2"] == g["edge_d2"]).all(), "MST d2 differ"
    assert (out["parent"] == g["parent"]).all(), "parent differs"
    # phi on the tree edges
    phi_o = orc.parent_flow(X, g["parent"], sigma)
    nz = g["parent"] >= 0
    phi_err = float((np.abs(out["phi_par"][nz] - phi_o[nz]) / phi_o[nz]).max())
    assert phi_err <= PHI_RTOL
    # omega per row
    rel = np.abs(out["omega"] - g["omega"]) / g["omega"]
    bound = omega_bound(n, d, g["edge_u"], g["edge_v"], g["edge_d2"], sigma)
    worst = int(np.argmax(rel / bound))
    assert (rel <= bound).all(), (worst, rel[worst], bound[worst])
    # labels, i_k, beta
    assert (out["labels"] == g["labels"].astype(np.int32)).all(), "labels differ"
    assert (out["residual"] == (g["labels"] < 0)).all()
    ik_err = abs(float(out["i_k"][0]) - float(g["i_k"])) / float(g["i_k"])
    beta_err = abs(float(out["beta"][0]) - float(g["beta"])) / float(g["beta"])
    assert ik_err <= IK_RTOL and beta_err <= IK_RTOL
    # the benchmark's call gives the same result
    assert (lab.cpu().numpy() == out["labels"]).all() and float(ik.cpu()[0]) == float(out["i_k"][0])
    margin, at_beta = decision_margin(orc, g["parent"], phi_o, g["omega"], k, float(g["beta"]))
    parity_report(f"{name}: n={n} d={d} MST+parent+labels bit-exact; i_k rel err {ik_err:.2e}, beta {beta_err:.2e}; "
                  f"phi max rel err {phi_err:.2e}; omega max rel err {float(rel.max()):.2e} "
                  f"(largest share of its row bound {float((rel / bound).max()):.3f}); decision margin "
                  f"{margin:.2e} ({at_beta} decision(s) at beta)")


def test_independent_sets_against_oracle(iso, orc, parity_report):
    from paper_1702_04739_gb300 import workloads
    g = golden("batched_4096_d32")
    X, offs, ks, sigma = workloads.make_batched("batched_4096_d32", seed=0)
    assert sha(X, offs, ks) == str(g["x_sha256"]), "the seeded input differs from the one the oracle saw"
    nsets = ks.size
    Xd = torch.from_numpy(X).cuda()
    out = iso.cluster_batched(Xd, offs, ks, sigma, detail=True)
    plain = iso.cluster_batched(Xd, offs, ks, sigma)          # the benchmark's entry point
    assert torch.equal(plain["labels"], out["labels"]) and torch.equal(plain["i_k"], out["i_k"])
    parent = out["parent"].cpu().numpy()
    labels = out["labels"].cpu().numpy()
    omega = out["omega"].cpu().numpy()
    ik = out["i_k"].cpu().numpy()
    beta = out["beta"].cpu().numpy()
    bad = []
    for b in range(nsets):
        lo, hi = int(offs[b]), int(offs[b + 1])
        pl = parent[lo:hi].copy()
        pl[pl >= 0] -= lo
        if (sha(pl.astype(np.int32)) != g["digests"][b][1].decode()
                or sha(labels[lo:hi].astype(np.int32)) != g["digests"][b][2].decode()):
            bad.append(b)
    if bad:
        b = bad[0]
        r = orc.cluster(np.ascontiguousarray(X[offs[b]:offs[b + 1]]), int(ks[b]), sigma)
        pl = parent[offs[b]:offs[b + 1]].copy()
        pl[pl >= 0] -= offs[b]
        raise AssertionError(f"{len(bad)} sets differ, first {b}: parent diffs at "
                             f"{np.nonzero(pl != r['parent'])[0][:5]}, labels diffs at "
                             f"{np.nonzero(labels[offs[b]:offs[b + 1]] != r['labels'])[0][:5]}")
    ik_err = float((np.abs(ik - g["i_k"]) / g["i_k"]).max())
    beta_err = float((np.abs(beta - g["beta"]) / g["beta"]).max())
    assert ik_err <= IK_RTOL and beta_err <= IK_RTOL
    # omega of the sampled sets
    worst_rel, worst_share, pos = 0.0, 0.0, 0
    for b in g["omega_sets"]:
        lo, hi = int(offs[b]), int(offs[b + 1])
        want = g["omega"][pos:pos + hi - lo]
        pos += hi - lo
        Xb = X[lo:hi]
        pl = parent[lo:hi].copy()
        pl[pl >= 0] -= lo
        v = np.nonzero(pl >= 0)[0]
        d2 = ((Xb[v].astype(np.float64) - Xb[pl[v]].astype(np.float64)) ** 2).sum(1)
        bound = omega_bound(hi - lo, X.shape[1], v, pl[v], d2, sigma)
        rel = np.abs(omega[lo:hi] - want) / want
        assert (rel <= bound).all(), (int(b), float(rel.max()))
        worst_rel = max(worst_rel, float(rel.max()))
        worst_share = max(worst_share, float((rel / bound).max()))
    assert pos == g["omega"].size
    parity_report(f"batched_4096_d32: {nsets} sets, {X.shape[0]} points; every set's parent and labels bit-exact; "
                  f"i_k max rel err {ik_err:.2e}, beta {beta_err:.2e}; omega of {len(g['omega_sets'])} sets max rel "
                  f"err {worst_rel:.2e} (largest share of its row bound {worst_share:.3f})")

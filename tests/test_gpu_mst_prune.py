"""Pruned Boruvka rounds (isoclust_set_mst_prune) against the full sweep and
the oracle's Prim tree: the same edges, bit for bit, on clustered, uniform,
duplicated and ragged inputs, with the pruning forced on for small sets and
off for large ones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def iso():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04739_gb300 import isoclust
    isoclust.load()
    yield isoclust
    isoclust.set_mst_prune(-1)


def _cases():
    from paper_1702_04739_gb300 import workloads
    rng = np.random.default_rng(41)
    out = []
    X, _ = workloads.blobs_anisotropic(seed=42, n=9000, k=12)
    out.append(("blobs_d64", X))
    X = workloads.blobs_isotropic(seed=43, n_per=1500, k=6, d=8, dtype=np.float32)[0]
    X[17] = X[3]                                              # duplicates across the order
    X[2000:2040] = X[100]
    out.append(("blobs_d8_dups", X))
    out.append(("uniform_d3_ragged", rng.uniform(-1, 1, size=(7001, 3)).astype(np.float32)))
    X, _ = workloads.moons_embedded(seed=44, n=8000)
    out.append(("moons_d128", X))
    grid = np.stack(np.meshgrid(np.arange(60), np.arange(60)), -1).reshape(-1, 2).astype(np.float32)
    out.append(("grid_ties_d2", grid))
    return out


def _mst(iso, X):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    u, v, d2 = iso.cluster_mst(Xd)
    return u.cpu().numpy(), v.cpu().numpy(), d2.cpu().numpy()


@pytest.mark.parametrize("case", range(5))
def test_pruned_rounds_give_the_full_sweeps_tree(iso, oracle_lib, case):
    name, X = _cases()[case]
    iso.set_mst_prune(1)
    pu, pv, pd = _mst(iso, X)
    iso.set_mst_prune(0)
    fu, fv, fd = _mst(iso, X)
    iso.set_mst_prune(-1)
    assert (pu == fu).all() and (pv == fv).all() and (pd == fd).all(), name
    ru, rv, rd = oracle_lib.mst_prim(X)[:3]
    assert (pu == ru).all() and (pv == rv).all() and (pd == rd).all(), name


def test_pruned_after_a_full_call_the_same(iso):
    from paper_1702_04739_gb300 import workloads
    X, _ = workloads.blobs_anisotropic(seed=45, n=40000, k=20)
    # a full call on other points first leaves its data in the library's
    # scratch: every candidate list a round reads must be one it wrote
    Y, _ = workloads.blobs_anisotropic(seed=46, n=30000, k=9)
    iso.cluster(torch.from_numpy(Y).cuda(), 9, 1.0)
    iso.set_mst_prune(1)
    au, av, ad = _mst(iso, X)
    assert iso.last_profile()["mst_tiles_swept"] < iso.last_profile()["mst_tiles_full"]
    iso.set_mst_prune(0)
    fu, fv, fd = _mst(iso, X)
    iso.set_mst_prune(-1)
    assert (au == fu).all() and (av == fv).all() and (ad == fd).all()


@pytest.mark.parametrize("prune", [0, 1])
def test_hook_chain_is_the_path(iso, oracle_lib, prune):
    """Points on a line with strictly shrinking gaps: in the first round every
    point hooks to its right neighbour, so the hooks form one chain through
    all the points (the deepest tree the root finding can meet); the tree is
    the path.  Coordinates and squared gaps are integers below 2^24, exact in
    FP32."""
    N = 4000
    x = np.concatenate([[0], np.cumsum(N - np.arange(N - 1))]).astype(np.float64)
    X = np.zeros((N, 4), np.float32)
    X[:, 0] = x
    iso.set_mst_prune(prune)
    u, v, d2 = _mst(iso, X)
    iso.set_mst_prune(-1)
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    assert sorted(zip(lo.tolist(), hi.tolist())) == [(k, k + 1) for k in range(N - 1)]
    ru, rv, rd = oracle_lib.mst_prim(X)[:3]
    assert (u == ru).all() and (v == rv).all() and (d2 == rd).all()

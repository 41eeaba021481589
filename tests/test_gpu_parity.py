"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (fixed here, derived in the design notes):
  * MST edge set and d2: bit-exact (integer/index work + canonical FP64 key).
  * tree stage fed identical inputs: labels, residual and i_k bit-exact.
  * omega: per-row relative error <= omega_tol(y_i) = 2^-45 max(1, sqrt(d/64))
    (y_i + 4), with y_i = ||x_i - x_nn(i)|| / sigma.  Each term is evaluated in double-word
    FP32: d2 carries ~2^-46 relative error, so the term's exponent
    y = d / sigma carries ~2^-47 * y absolute error, and so does the term's
    relative value; the bound keeps a factor ~4 of headroom over that.
  * end to end: i_k within 1e-12 relative; labels bit-exact.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IK_RTOL = 1e-12


def omega_tol(orc, X, sigma):
    """Per-row bound on the double-word omega error (see module docstring);
    the d2 sum's error grows like sqrt(d), so the d = 64 constant scales."""
    nn, nd2 = orc.nn_rows(X, np.arange(X.shape[0]))
    y = np.sqrt(nd2) / sigma
    return 2.0 ** -45 * max(1.0, math.sqrt(X.shape[1] / 64.0)) * (y + 4.0)


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
    oracle.set_threads(max(1, min(16, (torch.get_num_threads() or 1))))
    return oracle


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ------------------------------------------------------------------ tree stage
TREE_CASES = [
    (1, "random", 1), (2, "path", 1), (2, "path", 2), (5, "star", 3), (37, "random", 4), (64, "caterpillar", 7),
    (300, "binary", 10), (1000, "deep", 5), (1000, "star", 20), (5000, "random", 20), (4097, "path", 2),
    (20000, "random", 50),
]


@pytest.mark.parametrize("n,shape,k", TREE_CASES)
@pytest.mark.parametrize("with_p", [False, True])
def test_tree_stage_bit_exact(iso, orc, n, shape, k, with_p):
    from paper_1702_04739_gb300 import workloads
    parent, phi, om, p = workloads.random_rooted_tree(seed=n * 7 + k, n=n, shape=shape)
    if not with_p:
        p = None
    ref = orc.tree_stage(parent, phi, om, p, k)
    lab, res, ik = iso.tree_isoperimetric(_cuda(parent), _cuda(phi), _cuda(om), _cuda(p) if p is not None else None, k)
    assert float(ik.cpu()[0]) == ref["i_k"]
    assert (lab.cpu().numpy() == ref["labels"]).all()
    assert (res.cpu().numpy() == ref["residual"]).all()


def test_tree_stage_golden_and_k_range(iso, orc):
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_trees.json")) as f:
        g = json.load(f)
    for c in g["cases"]:
        for k, want in c["miso"].items():
            lab, res, ik = iso.tree_isoperimetric(_cuda(np.array(c["parent"], np.int32)),
                                                  _cuda(np.array(c["phi_par"])), _cuda(np.array(c["omega"])),
                                                  None, int(k))
            assert math.isclose(float(ik.cpu()[0]), want, rel_tol=1e-15, abs_tol=1e-300)


def test_tree_stage_full_size(iso, orc):
    """100,000-vertex random tree, the size of the 100k-point workload."""
    from paper_1702_04739_gb300 import workloads
    parent, phi, om, p = workloads.random_rooted_tree(seed=2024, n=100_000, shape="deep")
    for k in (1, 20, 3000):
        ref = orc.tree_stage(parent, phi, om, p, k)
        lab, res, ik = iso.tree_isoperimetric(_cuda(parent), _cuda(phi), _cuda(om), _cuda(p), k)
        assert float(ik.cpu()[0]) == ref["i_k"]
        assert (lab.cpu().numpy() == ref["labels"]).all()


@pytest.mark.parametrize("bad", ["two_roots", "cycle", "out_of_range", "self_loop", "no_root", "triangle"])
def test_tree_stage_rejects_malformed(iso, bad):
    n = 5
    parent = {"two_roots": [-1, 0, -1, 2, 2], "cycle": [1, 0, -1, 2, 2], "out_of_range": [-1, 0, 9, 0, 0],
              "self_loop": [-1, 1, 0, 0, 0], "no_root": [1, 2, 3, 4, 0], "triangle": [1, 2, 0, -1, 3]}[bad]
    phi = np.full(n, 0.5)
    om = np.ones(n)
    with pytest.raises(iso.IsoclustError) as e:
        iso.tree_isoperimetric(_cuda(np.array(parent, np.int32)), _cuda(phi), _cuda(om), None, 2)
    assert e.value.code == 1


def test_tree_stage_rejects_bad_weights(iso):
    parent = np.array([-1, 0, 0], np.int32)
    for om, code in ((np.array([1.0, 0.0, 1.0]), 1), (np.array([1.0, np.nan, 1.0]), 3), (np.array([1.0, -1.0, 1.0]), 1)):
        with pytest.raises(iso.IsoclustError) as e:
            iso.tree_isoperimetric(_cuda(parent), _cuda(np.array([0.0, 0.5, 0.5])), _cuda(om), None, 2)
        assert e.value.code == code
    with pytest.raises(iso.IsoclustError) as e:
        iso.tree_isoperimetric(_cuda(parent), _cuda(np.array([0.0, 0.5, 0.5])), _cuda(np.ones(3)), None, 4)
    assert e.value.code == 2


# ------------------------------------------------------------------ MST
def _mst_inputs():
    from paper_1702_04739_gb300 import workloads as W
    rng = np.random.default_rng(77)
    yield "blobs_f64", W.blobs_isotropic(seed=1, n_per=100, k=5, d=8)[0]
    yield "blobs_f32", W.blobs_isotropic(seed=2, n_per=150, k=4, d=8, dtype=np.float32)[0]
    yield "aniso_f32_d64", W.blobs_anisotropic(seed=3, n=1500, k=6, d=64)[0]
    yield "uniform_f32_d3", W.uniform_points(seed=4, n=777, d=3)
    yield "grid_ties_f32", W.integer_grid_points(seed=5, n=600, d=2, span=12)
    yield "duplicates_f32", np.repeat(W.uniform_points(seed=6, n=40, d=5), 3, axis=0)
    yield "line_d1_f32", rng.normal(size=(300, 1)).astype(np.float32)
    yield "n2_f64", np.array([[0.0, 1.0], [2.0, 3.0]])
    yield "n3_f32", np.array([[0, 0], [1, 0], [0, 1]], np.float32)
    yield "d130_f32", rng.normal(size=(260, 130)).astype(np.float32)
    yield "sparse_d512_f32", W.sparse_groups(seed=7, n_per=60, k=4, d=512)[0]


@pytest.mark.parametrize("name,X", list(_mst_inputs()), ids=[c[0] for c in _mst_inputs()])
def test_mst_bit_exact(iso, orc, name, X):
    eu, ev, ed, _, _ = orc.mst_prim(X)
    gu, gv, gd = iso.cluster_mst(_cuda(X))
    assert (gu.cpu().numpy() == eu).all() and (gv.cpu().numpy() == ev).all()
    assert (gd.cpu().numpy() == ed).all()


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mst_precision_paths_agree(iso, orc, prec):
    from paper_1702_04739_gb300 import workloads as W
    X = W.blobs_anisotropic(seed=9, n=2000, k=5, d=64)[0]
    eu, ev, ed, _, _ = orc.mst_prim(X)
    gu, gv, gd = iso.cluster_mst(_cuda(X), iso.opts(precision=prec))
    assert (gu.cpu().numpy() == eu).all() and (gv.cpu().numpy() == ev).all() and (gd.cpu().numpy() == ed).all()


# ------------------------------------------------------------------ omega / p
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("alpha,sigma", [(0.0, 1.0), (0.7, 0.35), (0.0, 3.0)])
def test_vertex_weights(iso, orc, dtype, alpha, sigma):
    from paper_1702_04739_gb300 import workloads as W
    X = W.blobs_anisotropic(seed=11, n=1300, k=5, d=64)[0].astype(dtype)
    om, p = orc.weights(X, sigma, alpha=alpha)
    gom, gp = iso.vertex_weights(_cuda(X), sigma, iso.opts(alpha=alpha))
    tol = omega_tol(orc, X, sigma) if dtype == np.float32 else 1e-14
    rel = np.abs(gom.cpu().numpy() - om) / om
    assert (rel <= tol).all(), (rel.max(), (rel / tol).max())
    if alpha:
        relp = np.abs(gp.cpu().numpy() - p) / p
        assert relp.max() <= 1e-13, relp.max()
    else:
        assert (gp.cpu().numpy() == 0).all()


def test_vertex_weights_include_self_and_ragged(iso, orc):
    rng = np.random.default_rng(12)
    for n, d in ((2, 1), (65, 3), (129, 33), (300, 70)):
        X = rng.normal(size=(n, d)).astype(np.float32)
        om, _ = orc.weights(X, 0.9, include_self=True)
        gom, _ = iso.vertex_weights(_cuda(X), 0.9, iso.opts(include_self=True), want_p=False)
        assert (np.abs(gom.cpu().numpy() - om) / om <= omega_tol(orc, X, 0.9)).all()


# ------------------------------------------------------------------ end to end
def _e2e_cases():
    from paper_1702_04739_gb300 import workloads as W
    yield "blobs_n2000_d8_f64", W.blobs_isotropic(seed=0)[0], 5, 1.0
    yield "blobs_f32_k3", W.blobs_isotropic(seed=3, n_per=200, k=3, d=8, dtype=np.float32)[0], 3, 1.0
    yield "aniso_d64", W.blobs_anisotropic(seed=4, n=3000, k=8, d=64)[0], 8, 1.0
    yield "uniform_k1", W.uniform_points(seed=5, n=500, d=4), 1, 0.5
    yield "uniform_k_eq_n", W.uniform_points(seed=6, n=40, d=2), 40, 0.5
    yield "grid_ties", W.integer_grid_points(seed=7, n=400, d=3, span=6), 6, 2.0
    yield "table1_wine_shape", W.table1_shape(seed=8, n=178, k=3, d=13)[0], 3, 1.0


@pytest.mark.parametrize("name,X,k,sigma", list(_e2e_cases()), ids=[c[0] for c in _e2e_cases()])
def test_cluster_end_to_end(iso, orc, name, X, k, sigma):
    ref = orc.cluster(X, k, sigma)
    out = iso.cluster_detail(_cuda(X), k, sigma)
    assert (out["edge_u"].cpu().numpy() == ref["edge_u"]).all()
    assert (out["edge_v"].cpu().numpy() == ref["edge_v"]).all()
    assert (out["parent"].cpu().numpy() == ref["parent"]).all()
    assert np.allclose(out["phi_par"].cpu().numpy(), ref["phi_par"], rtol=4e-16, atol=0)
    tol = omega_tol(orc, X, sigma) if X.dtype == np.float32 else 1e-14
    assert (np.abs(out["omega"].cpu().numpy() - ref["omega"]) / ref["omega"] <= tol).all()
    assert math.isclose(float(out["i_k"].cpu()[0]), ref["i_k"], rel_tol=IK_RTOL)
    assert (out["labels"].cpu().numpy() == ref["labels"]).all()
    lab, res, ik = iso.cluster(_cuda(X), k, sigma)
    assert (lab.cpu().numpy() == out["labels"].cpu().numpy()).all()
    assert float(ik.cpu()[0]) == float(out["i_k"].cpu()[0])


def test_cluster_options(iso, orc):
    from paper_1702_04739_gb300 import workloads as W
    X = W.blobs_isotropic(seed=21, n_per=80, k=4, d=5, dtype=np.float32)[0]
    for kw in (dict(alpha=0.01), dict(omega_mode=1), dict(root=17), dict(include_self=True),
               dict(omega_mode=1, alpha=0.002)):
        ref = orc.cluster(X, 4, 1.0, **kw)
        lab, res, ik = iso.cluster(_cuda(X), 4, 1.0, iso.opts(**kw))
        assert math.isclose(float(ik.cpu()[0]), ref["i_k"], rel_tol=IK_RTOL), kw
        assert (lab.cpu().numpy() == ref["labels"]).all(), kw


def test_cluster_deterministic(iso):
    from paper_1702_04739_gb300 import workloads as W
    X = _cuda(W.blobs_anisotropic(seed=31, n=4000, k=6, d=64)[0])
    a = iso.cluster_detail(X, 6, 1.0)
    b = iso.cluster_detail(X, 6, 1.0)
    for key in a:
        assert torch.equal(a[key], b[key]), key


def test_cluster_errors(iso):
    X = np.random.default_rng(0).normal(size=(50, 3)).astype(np.float32)
    Xn = X.copy(); Xn[7, 1] = np.nan
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster(_cuda(Xn), 2, 1.0)
    assert e.value.code == 3
    Xi = X.copy(); Xi[3, 0] = np.inf
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster_mst(_cuda(Xi))
    assert e.value.code == 3
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster(_cuda(X), 51, 1.0)
    assert e.value.code == 2
    for args in ((0, 1.0), (2, 0.0), (2, float("nan")), (2, -1.0)):
        with pytest.raises(iso.IsoclustError) as e:
            iso.cluster(_cuda(X), *args)
        assert e.value.code == 1
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster(_cuda(X[:1]), 1, 1.0)
    assert e.value.code == 1
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster(_cuda(X), 2, 1.0, iso.opts(root=50))
    assert e.value.code == 1
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster(_cuda(X.astype(np.float64)), 2, 1.0, iso.opts(precision=2))
    assert e.value.code == 1
    # the library stays usable after errors
    lab, res, ik = iso.cluster(_cuda(X), 2, 1.0)
    assert np.isfinite(float(ik.cpu()[0]))

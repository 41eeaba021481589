"""Pins of the oracle's derivative of i_k through a fixed structure (CPU).

The oracle's analytic gradient (oracle_ik_grad) is checked against what the
mathematics fixes, not against itself:
  * central finite differences (h = 1e-6, FP64) of the oracle's own i_k on the
    same fixed tree and subpartition, for X, the per-feature scale and sigma;
  * exact identities: i_k is invariant to (X, sigma) -> (cX, c sigma), to
    (scale, sigma) -> (c scale, c sigma) and to translating all points, so
    sum X.dX + sigma dsigma = 0, sum scale.dscale + sigma dsigma = 0 and
    sum_i dX_i = 0 (Euler's theorem for degree-0 homogeneous functions);
  * the fixed-structure value equals the forward's i_k, and the structure
    does not change under the finite-difference perturbations.
A dropped term (the partner pairs of omega, the boundary edges, the sigma
terms) or a sign error fails at least one of these."""
import numpy as np
import pytest

import oracle
from paper_1702_04739_gb300 import workloads as W

H = 1e-6


def _case(name):
    if name == "blobs":
        X = W.blobs_isotropic(seed=11, n_per=45, k=3, d=5)[0]
        return X, np.linspace(0.8, 1.25, 5), 1.0, 3
    X = W.moons_embedded(seed=2, n=180, d=8, noise=0.05)[0].astype(np.float64)
    return X, np.linspace(1.1, 0.9, 8), 0.4, 3


@pytest.fixture(scope="module", params=["blobs", "moons"])
def case(request):
    oracle.build()
    X, s, sigma, k = _case(request.param)
    fwd = oracle.cluster(X * s, k, sigma)
    fx = oracle.ik_fixed(X, s, sigma, fwd["parent"], fwd["labels"], k)
    g = oracle.ik_grad(X, s, sigma, fwd["parent"], fwd["labels"], fx["jstar"])
    return dict(X=X, s=s, sigma=sigma, k=k, fwd=fwd, fx=fx, g=g)


def _R(c, X=None, s=None, sigma=None):
    return oracle.ik_fixed(c["X"] if X is None else X, c["s"] if s is None else s,
                           c["sigma"] if sigma is None else sigma,
                           c["fwd"]["parent"], c["fwd"]["labels"], c["k"])["R"]


def test_fixed_value_is_the_forward_i_k(case):
    assert np.isclose(case["fx"]["R"], case["fwd"]["i_k"], rtol=1e-12, atol=0)
    assert np.isclose(case["g"]["R"], case["fwd"]["i_k"], rtol=1e-12, atol=0)


def test_central_differences(case):
    c, g = case, case["g"]
    gs = g["dscale"]
    for t in range(c["s"].size):
        sp, sm = c["s"].copy(), c["s"].copy()
        sp[t] += H
        sm[t] -= H
        fd = (_R(c, s=sp) - _R(c, s=sm)) / (2 * H)
        assert abs(fd - gs[t]) <= 1e-6 * np.abs(gs).max(), (t, fd, gs[t])
    fd = (_R(c, sigma=c["sigma"] + H) - _R(c, sigma=c["sigma"] - H)) / (2 * H)
    assert abs(fd - g["dsigma"]) <= 1e-6 * abs(g["dsigma"])
    gx = g["dX"]
    flat = np.argsort(-np.abs(gx).ravel())[:12]          # the largest entries, where FD noise is small
    rng = np.random.default_rng(0)
    flat = np.concatenate([flat, rng.choice(gx.size, 8, replace=False)])
    for q in flat:
        i, t = divmod(int(q), gx.shape[1])
        Xp, Xm = c["X"].copy(), c["X"].copy()
        Xp[i, t] += H
        Xm[i, t] -= H
        fd = (_R(c, X=Xp) - _R(c, X=Xm)) / (2 * H)
        assert abs(fd - gx[i, t]) <= 1e-6 * np.abs(gx).max(), (i, t, fd, gx[i, t])


def test_invariance_identities(case):
    c, g = case, case["g"]
    a = (g["dX"] * c["X"]).sum() + c["sigma"] * g["dsigma"]
    assert abs(a) <= 1e-10 * (np.abs(g["dX"] * c["X"]).sum() + abs(c["sigma"] * g["dsigma"]))
    b = (g["dscale"] * c["s"]).sum() + c["sigma"] * g["dsigma"]
    assert abs(b) <= 1e-10 * (np.abs(g["dscale"] * c["s"]).sum() + abs(c["sigma"] * g["dsigma"]))
    tr = g["dX"].sum(axis=0)
    assert (np.abs(tr) <= 1e-10 * np.abs(g["dX"]).sum(axis=0) + 1e-300).all()


def test_structure_is_stable_under_the_perturbations(case):
    c = case
    rng = np.random.default_rng(1)
    for _ in range(3):
        i, t = int(rng.integers(c["X"].shape[0])), int(rng.integers(c["X"].shape[1]))
        Xp = c["X"].copy()
        Xp[i, t] += H
        f2 = oracle.cluster(Xp * c["s"], c["k"], c["sigma"])
        assert (f2["parent"] == c["fwd"]["parent"]).all()
        assert (f2["labels"] == c["fwd"]["labels"]).all()
    f3 = oracle.cluster(c["X"] * c["s"], c["k"], c["sigma"] + H)
    assert (f3["labels"] == c["fwd"]["labels"]).all()


def test_moons_recipe():
    X, y = W.moons_embedded(seed=0, n=300, d=16)
    assert X.shape == (300, 16) and X.dtype == np.float32
    assert np.bincount(y).tolist() == [100, 100, 100]
    X2, _ = W.moons_embedded(seed=0, n=300, d=16, noise=0.0)
    # noise-free points lie in a 2-D subspace at distance <= 3 from the origin
    assert np.linalg.matrix_rank(X2.astype(np.float64), tol=1e-4) == 2

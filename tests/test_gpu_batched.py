"""GPU parity of independent point sets in one call (isoclust_cluster_batched)
against the FP64 oracle run on each set alone.

Bars, per set (those of the one-set path): the MST (parent array, global
indices) bit-exact, phi within 4e-16, omega within the double-word bound,
labels bit-exact, i_k and beta within 1e-12 relative.  The batched call also
agrees with the library's own one-set call on every set (identical trees and
labels).  The full 4,096-set workload is checked on sampled sets and by
properties that hold for every set."""
import math

import numpy as np
import pytest

from test_gpu_parity import IK_RTOL, omega_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# ragged sizes on both sides of the 64- and 128-row tile boundaries, tiny sets
SMALL_SIZES = [2, 3, 5, 17, 63, 64, 65, 127, 128, 129, 191, 200, 255, 256, 257, 383, 511, 700]


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
    oracle.set_threads(16)
    return oracle


def _small_batch(seed=0):
    from paper_1702_04739_gb300 import workloads as W
    rng = np.random.default_rng(seed + 100)
    sizes = SMALL_SIZES + [int(v) for v in rng.integers(6, 420, size=14)]
    return W.batched_sets(seed=seed, d=32, sizes=sizes)


def _check_set(orc, X, offs, ks, out, b, sigma=1.0, ref=None):
    lo, hi = int(offs[b]), int(offs[b + 1])
    Xb = X[lo:hi]
    if ref is None:
        ref = orc.cluster(Xb, int(ks[b]), sigma)
    par = out["parent"][lo:hi]
    want = np.where(ref["parent"] >= 0, ref["parent"] + lo, -1)
    assert (par == want).all(), b
    assert np.allclose(out["phi_par"][lo:hi], ref["phi_par"], rtol=4e-16, atol=0), b
    tol = omega_tol(orc, Xb, sigma)
    assert (np.abs(out["omega"][lo:hi] - ref["omega"]) / ref["omega"] <= tol).all(), b
    assert (out["labels"][lo:hi] == ref["labels"]).all(), b
    assert (out["residual"][lo:hi] == ref["residual"]).all(), b
    assert math.isclose(float(out["i_k"][b]), ref["i_k"], rel_tol=IK_RTOL), b
    assert math.isclose(float(out["beta"][b]), ref["beta"], rel_tol=IK_RTOL), b


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_small_batch_against_oracle(iso, orc):
    X, offs, ks = _small_batch(0)
    out = _host(iso.cluster_batched(torch.from_numpy(X).cuda(), offs, ks, 1.0, detail=True))
    for b in range(len(ks)):
        _check_set(orc, X, offs, ks, out, b)


def test_batched_equals_single_calls(iso):
    X, offs, ks = _small_batch(1)
    Xd = torch.from_numpy(X).cuda()
    out = _host(iso.cluster_batched(Xd, offs, ks, 1.0, detail=True))
    for b in range(len(ks)):
        lo, hi = int(offs[b]), int(offs[b + 1])
        one = _host(iso.cluster_detail(Xd[lo:hi].contiguous(), int(ks[b]), 1.0))
        par = np.where(one["parent"] >= 0, one["parent"] + lo, -1)
        assert (out["parent"][lo:hi] == par).all(), b
        assert (out["phi_par"][lo:hi] == one["phi_par"]).all(), b
        assert (out["labels"][lo:hi] == one["labels"]).all(), b
        assert math.isclose(float(out["i_k"][b]), float(one["i_k"][0]), rel_tol=IK_RTOL), b


def test_batched_options_and_errors(iso):
    X, offs, ks = _small_batch(2)
    Xd = torch.from_numpy(X).cuda()
    a = _host(iso.cluster_batched(Xd, offs, ks, 1.0))
    b = _host(iso.cluster_batched(Xd, offs, ks, 1.0, iso.opts(precision=iso.PREC_BF16_TC)))
    c = _host(iso.cluster_batched(Xd, offs, ks, 1.0))
    for key in ("labels", "residual", "i_k", "beta"):
        assert (a[key] == b[key]).all() and (a[key] == c[key]).all(), key   # deterministic
    # include_self shifts every omega by exactly one term of 1
    s = _host(iso.cluster_batched(Xd, offs, ks, 1.0, iso.opts(include_self=True), detail=True))
    d = _host(iso.cluster_batched(Xd, offs, ks, 1.0, detail=True))
    assert np.allclose(s["omega"], d["omega"] + 1.0, rtol=1e-15, atol=0)
    with pytest.raises(iso.IsoclustError):
        iso.cluster_batched(Xd, offs, [int(ks[0]) + 10**6] + [int(v) for v in ks[1:]], 1.0)
    with pytest.raises(iso.IsoclustError):
        iso.cluster_batched(Xd, offs, ks, 1.0, iso.opts(alpha=0.1))
    with pytest.raises(iso.IsoclustError):
        iso.cluster_batched(Xd.double(), offs, ks, 1.0)
    bad = offs.copy()
    bad[1] = 1                     # a one-point set
    with pytest.raises(iso.IsoclustError):
        iso.cluster_batched(Xd, bad, ks, 1.0)
    Xn = X.copy()
    Xn[int(offs[5]) + 1, 3] = np.nan
    with pytest.raises(iso.IsoclustError):
        iso.cluster_batched(torch.from_numpy(Xn).cuda(), offs, ks, 1.0)


@pytest.fixture(scope="module")
def full(iso):
    from paper_1702_04739_gb300 import workloads as W
    X, offs, ks, sigma = W.make_batched("batched_4096_d32", seed=0)
    out = _host(iso.cluster_batched(torch.from_numpy(X).cuda(), offs, ks, sigma, detail=True))
    return X, offs, ks, sigma, out


def test_full_batch_sampled_sets(orc, full):
    X, offs, ks, sigma, out = full
    sizes = np.diff(offs)
    rng = np.random.default_rng(5)
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))} | {int(v) for v in rng.choice(len(ks), 6, replace=False)}
    for b in sorted(pick):
        _check_set(orc, X, offs, ks, out, b, sigma)


def test_full_batch_properties(full):
    X, offs, ks, sigma, out = full
    lab, par, phi, om = out["labels"], out["parent"], out["phi_par"], out["omega"]
    assert np.isfinite(out["i_k"]).all() and (out["i_k"] > 0).all()
    assert (out["i_k"] <= out["beta"] * (1 + 1e-12)).all()
    for b in range(len(ks)):
        lo, hi = int(offs[b]), int(offs[b + 1])
        L, Pa = lab[lo:hi], par[lo:hi]
        assert Pa[0] == -1 and ((Pa[1:] >= lo) & (Pa[1:] < hi)).all()
        assert ((L >= -1) & (L < ks[b])).all()
        assert np.unique(L[L >= 0]).size == ks[b]
        assert (om[lo:hi] > 0).all()


def test_repeated_calls_replay_cuda_graphs(iso):
    """Identical batched calls: the first launches kernel by kernel, the
    second captures CUDA graphs, the third replays them; every output is
    bit-identical and each call launches the same number of kernels."""
    X, offs, ks = _small_batch(3)
    Xd = torch.from_numpy(X).cuda()
    plan = iso.BatchPlan(offs, ks)
    n = X.shape[0]
    outs, modes, launches = [], [], []
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    residual = torch.empty(n, dtype=torch.uint8, device="cuda")
    ik = torch.empty(len(ks), dtype=torch.float64, device="cuda")
    for _ in range(4):
        l0 = iso.kernel_launches()
        iso.cluster_batched_into(Xd, plan, 1.0, labels, residual, ik)
        launches.append(iso.kernel_launches() - l0)
        modes.append(iso.last_batched_graph_mode())
        outs.append((labels.cpu().numpy().copy(), residual.cpu().numpy().copy(), ik.cpu().numpy().copy()))
    assert modes == [0, 1, 2, 2], modes
    assert len(set(launches)) == 1, launches
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert (a == b).all()
    # another signature (different ks) starts again kernel by kernel
    ks2 = np.maximum(1, np.asarray(ks) - 1).astype(np.int32)
    iso.cluster_batched_into(Xd, iso.BatchPlan(offs, ks2), 1.0, labels, residual, ik)
    assert iso.last_batched_graph_mode() == 0

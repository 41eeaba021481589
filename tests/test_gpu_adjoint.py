"""GPU parity of the derivative of i_k (isoclust_ik_backward and the
autograd Function) against the oracle's FP64 gradient on the same fixed
structure; the oracle's gradient is itself pinned by finite differences and
exact invariances (test_oracle_grad.py).

Bars: i_k of the fixed structure within 1e-12 relative; dX within 1e-10 of
max |dX| (FP64 on both sides, sums in different orders; the difference
dPhi - i_k dOmega cancels to about 1e-4 of its terms, so 1e-10 keeps a wide
margin over the ~1e-16 rounding of the sums); dscale and dsigma likewise.
The forward runs on the scaled FP32 points (the differentiation workload
stores FP32); its tree and labels equal the oracle's on the same points."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RT = 1e-10


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


def _run(iso, orc, X, s, sigma, k):
    Xd = torch.from_numpy(X).cuda()
    sd = torch.from_numpy(s).cuda()
    Z = iso.scale_features(Xd, sd)
    out = iso.cluster_detail(Z, k, sigma)
    g = iso.ik_backward(Xd, sd, sigma, out["parent"], out["labels"], k, out["phi_par"], out["omega"], 1.0)
    h = {key: v.cpu().numpy() for key, v in out.items()}
    gh = {key: v.cpu().numpy() for key, v in g.items()}
    Zh = Z.cpu().numpy()
    return Xd, sd, h, gh, Zh


def _compare(orc, X, s, sigma, k, h, gh):
    X64 = X.astype(np.float64)
    fx = orc.ik_fixed(X64, s, sigma, h["parent"], h["labels"], k)
    ref = orc.ik_grad(X64, s, sigma, h["parent"], h["labels"], fx["jstar"])
    assert math.isclose(float(gh["i_k"][0]), ref["R"], rel_tol=1e-12)
    # the forward clustered the FP32-rounded points fl(s x) (relative change
    # <= 2^-24 per coordinate); the derivative is of the exact z = s x
    assert math.isclose(float(gh["i_k"][0]), float(h["i_k"][0]), rel_tol=1e-6)
    assert np.abs(gh["dX"] - ref["dX"]).max() <= RT * np.abs(ref["dX"]).max()
    assert np.abs(gh["dscale"] - ref["dscale"]).max() <= RT * np.abs(ref["dscale"]).max()
    assert abs(gh["dsigma"][0] - ref["dsigma"]) <= RT * abs(ref["dsigma"])
    return ref


@pytest.mark.parametrize("seed,n,d,k,sigma", [(1, 400, 16, 3, 0.5), (2, 257, 7, 4, 1.0), (3, 130, 130, 2, 2.0)])
def test_backward_small(iso, orc, seed, n, d, k, sigma):
    from paper_1702_04739_gb300 import workloads as W
    X = W.moons_embedded(seed=seed, n=n, d=d, noise=0.05)[0]
    s = np.linspace(0.85, 1.2, d)
    Xd, sd, h, gh, Zh = _run(iso, orc, X, s, sigma, k)
    fwd = orc.cluster(Zh.astype(np.float64), k, sigma)
    assert (fwd["parent"] == h["parent"]).all() and (fwd["labels"] == h["labels"]).all()
    _compare(orc, X, s, sigma, k, h, gh)


def test_autograd_function(iso):
    from paper_1702_04739_gb300 import workloads as W
    X = torch.from_numpy(W.moons_embedded(seed=4, n=300, d=12, noise=0.05)[0]).cuda().requires_grad_(True)
    s = torch.linspace(0.9, 1.1, 12, dtype=torch.float64, device="cuda").requires_grad_(True)
    sig = torch.tensor(0.7, dtype=torch.float64, device="cuda", requires_grad=True)
    ik, labels = iso.IsoperimetricNumber.apply(X, s, sig, 3)
    (ik * 3.0).backward()
    Z = iso.scale_features(X.detach(), s.detach())
    out = iso.cluster_detail(Z, 3, 0.7)
    g = iso.ik_backward(X.detach(), s.detach(), 0.7, out["parent"], out["labels"], 3, out["phi_par"],
                        out["omega"], 3.0)
    assert torch.equal(labels, out["labels"])
    assert float(ik.detach()) == float(out["i_k"][0])
    assert torch.allclose(X.grad.double(), g["dX"], rtol=1e-6, atol=1e-7 * float(g["dX"].abs().max()))
    assert torch.equal(s.grad, g["dscale"])
    assert float(sig.grad) == float(g["dsigma"][0])


def test_backward_errors(iso):
    from paper_1702_04739_gb300 import workloads as W
    X = torch.from_numpy(W.moons_embedded(seed=5, n=100, d=4)[0]).cuda()
    s = torch.ones(4, dtype=torch.float64, device="cuda")
    out = iso.cluster_detail(iso.scale_features(X, s), 3, 1.0)
    args = (out["parent"], out["labels"], 3, out["phi_par"], out["omega"])
    with pytest.raises(iso.IsoclustError):
        iso.ik_backward(X, s, 0.0, *args)
    with pytest.raises(iso.IsoclustError):
        iso.ik_backward(X, s, 1.0, out["parent"], out["labels"], 101, out["phi_par"], out["omega"])
    with pytest.raises(iso.IsoclustError):   # label 3 has no points
        iso.ik_backward(X, s, 1.0, out["parent"], out["labels"], 4, out["phi_par"], out["omega"])
    with pytest.raises(ValueError):
        iso.scale_features(X, torch.ones(5, dtype=torch.float64, device="cuda"))


@pytest.fixture(scope="module")
def full(iso, orc):
    from paper_1702_04739_gb300 import workloads as W
    X, k, sigma = W.make("moons_n20k_d128", seed=0)
    s = np.ones(X.shape[1])
    Xd, sd, h, gh, Zh = _run(iso, orc, X, s, sigma, k)
    return X, s, k, sigma, Xd, sd, h, gh


def test_full_size_backward_against_oracle(orc, full):
    X, s, k, sigma, Xd, sd, h, gh = full
    ref = _compare(orc, X, s, sigma, k, h, gh)
    # central difference of the oracle's fixed-structure i_k in sigma (FP64, h = 1e-6)
    H = 1e-6
    X64 = X.astype(np.float64)
    rp = orc.ik_fixed(X64, s, sigma + H, h["parent"], h["labels"], k)["R"]
    rm = orc.ik_fixed(X64, s, sigma - H, h["parent"], h["labels"], k)["R"]
    assert abs((rp - rm) / (2 * H) - gh["dsigma"][0]) <= 1e-6 * abs(ref["dsigma"])


def test_full_size_structure_stable(iso, full):
    X, s, k, sigma, Xd, sd, h, gh = full
    rng = np.random.default_rng(3)
    for _ in range(3):
        i, t = int(rng.integers(X.shape[0])), int(rng.integers(X.shape[1]))
        Xp = X.copy()
        Xp[i, t] = np.float32(Xp[i, t] + np.float32(1e-6))      # the finite-difference step
        out = iso.cluster_detail(iso.scale_features(torch.from_numpy(Xp).cuda(), sd), k, sigma)
        assert (out["labels"].cpu().numpy() == h["labels"]).all()
        assert (out["parent"].cpu().numpy() == h["parent"]).all()

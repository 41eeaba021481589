"""eq. omega with the kept tile pairs' Gram on the tensor cores (the default
for F32 one-set calls on sm_103) against the FP64 oracle and against the
double-word CUDA-core sums (isoclust_set_omega_gram(0)): per-row omega within
the library's bound, the MST unchanged, labels equal.  Cases cover the
resident-row kernel (d <= 64) and the streamed one (d > 64, several 64-wide
chunks), ragged tiles, exact duplicates and near-duplicates (where the Gram
form cancels and the direct sums take over, by groups of 8 lanes for short
rows and of 32 for long ones), and rows long enough (d >= 1024) to be centred
on one point instead of their tile's centroid."""
import math

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
    isoclust.set_omega_gram(-1)


def _bound(orc, X, sigma):
    nn, nd2 = orc.nn_rows(X, np.arange(X.shape[0]))
    return 2.0 ** -45 * max(1.0, math.sqrt(X.shape[1] / 64.0)) * (np.sqrt(nd2) / sigma + 4.0)


def _cases():
    from paper_1702_04739_gb300 import workloads
    rng = np.random.default_rng(31)
    out = []
    X, _ = workloads.blobs_anisotropic(seed=21, n=5000, k=7)
    out.append(("blobs_d64", X, 7, 1.0))
    X = workloads.blobs_isotropic(seed=22, n_per=700, k=3, d=130, dtype=np.float32)[0]
    out.append(("blobs_d130", X, 3, 2.0))
    X = workloads.blobs_isotropic(seed=23, n_per=450, k=4, d=8, dtype=np.float32)[0]
    X[100] = X[5]                                         # an exact duplicate
    X[200] = X[7] + np.float32(1e-6)                      # a near-duplicate
    out.append(("blobs_d8_dups", X, 4, 1.0))
    X = (rng.normal(size=(3001, 37)) * np.exp(rng.uniform(-4, 4, size=37))).astype(np.float32)
    out.append(("scaled_d37_ragged", X, 5, 3.0))
    X = workloads.blobs_isotropic(seed=24, n_per=500, k=3, d=1100, dtype=np.float32)[0]
    X[10] = X[3]                                          # an exact duplicate of a long row
    X[400] = X[401] + np.float32(1e-5)                    # and a near-duplicate
    out.append(("blobs_d1100_one_centre_dups", X, 3, 4.0))
    return out


@pytest.mark.parametrize("case", range(5))
def test_gram_omega_against_oracle_and_cuda_cores(iso, oracle_lib, parity_report, case):
    name, X, k, sigma = _cases()[case]
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    iso.set_omega_gram(True)
    g = {key: v.cpu().numpy() for key, v in iso.cluster_detail(Xd, k, sigma).items()}
    prof = iso.last_profile()
    assert prof["omega_symmetric"] == 3
    if "dups" in name:
        assert prof["omega_gram_direct_pairs"] > 0         # the duplicates took the direct sums
    iso.set_omega_gram(False)
    c = {key: v.cpu().numpy() for key, v in iso.cluster_detail(Xd, k, sigma).items()}
    assert iso.last_profile()["omega_symmetric"] == 2
    iso.set_omega_gram(-1)
    om, _ = oracle_lib.weights(X, sigma)
    bound = _bound(oracle_lib, X, sigma)
    rel_g = np.abs(g["omega"] - om) / om
    rel_c = np.abs(c["omega"] - om) / om
    assert (rel_g <= bound).all(), (int(np.argmax(rel_g / bound)), float(rel_g.max()))
    assert (rel_c <= bound).all()
    assert (g["edge_u"] == c["edge_u"]).all() and (g["edge_d2"] == c["edge_d2"]).all()
    ref = oracle_lib.cluster(X, k, sigma)
    assert (g["labels"] == ref["labels"]).all()
    assert abs(float(g["i_k"][0]) - ref["i_k"]) <= 1e-12 * ref["i_k"]
    parity_report(f"omega Gram on tensor cores, {name}: max rel err {rel_g.max():.2e} (share of bound "
                  f"{(rel_g / bound).max():.3f}); double-word CUDA cores {rel_c.max():.2e}")

"""The bounded-wait (timeout) path of the tensor-core Boruvka sweep.

The library's only device-side waits are the sweep's mbarrier waits; each
gives up after opts.spin_limit SM cycles (default about 2 s), raises a flag,
lets the copies and MMAs its CTA issued finish, frees its tensor memory and
returns, and the call reports ISOCLUST_ERR_TIMEOUT without walking the
unfinished tree.  The test hook isoclust_set_test_stalled_wait makes the
epilogue wait for a barrier nothing arrives at, so the wait runs out for
certain; afterwards the device and the library must work as before (results
bit-identical to a call made before the timeouts, and to the oracle).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 6


@pytest.fixture(scope="module")
def iso():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04739_gb300 import isoclust
    isoclust.load()
    return isoclust


def _timed_out(fn):
    from paper_1702_04739_gb300 import isoclust
    with pytest.raises(isoclust.IsoclustError) as e:
        fn()
    assert e.value.code == TIMEOUT, str(e.value)
    return str(e.value)


def test_stalled_wait_times_out_and_the_library_recovers(iso, oracle_lib):
    from paper_1702_04739_gb300 import workloads
    X = workloads.blobs_anisotropic(seed=5, n=3000, k=6)[0]
    k, sigma = 6, 1.0
    ref = oracle_lib.cluster(X, k, sigma)
    Xd = torch.from_numpy(X).cuda()
    before = {key: v.cpu().numpy() for key, v in iso.cluster_detail(Xd, k, sigma).items()}
    Xb, offs, ks = workloads.batched_sets(seed=2, d=16, sizes=[300, 900, 200])
    Xbd = torch.from_numpy(Xb).cuda()
    bat_before = iso.cluster_batched(Xbd, offs, ks, sigma)
    short = iso.opts(spin_limit=2_000_000)          # about 1 ms per wait
    iso.set_test_stalled_wait(True)
    try:
        _timed_out(lambda: iso.cluster(Xd, k, sigma, short))
        _timed_out(lambda: iso.cluster_mst(Xd, short))
        _timed_out(lambda: iso.cluster_batched(Xbd, offs, ks, sigma, short))
        _timed_out(lambda: iso.cluster(Xd, k, sigma))   # the default bound (about 2 s) runs out too
    finally:
        iso.set_test_stalled_wait(False)
    torch.cuda.synchronize()
    after = {key: v.cpu().numpy() for key, v in iso.cluster_detail(Xd, k, sigma).items()}
    for key in ("edge_u", "edge_v", "edge_d2", "parent", "labels", "omega", "i_k", "beta"):
        assert (after[key] == before[key]).all(), key
    assert (after["edge_u"] == ref["edge_u"]).all() and (after["edge_d2"] == ref["edge_d2"]).all()
    assert (after["labels"] == ref["labels"]).all()
    bat_after = iso.cluster_batched(Xbd, offs, ks, sigma)
    assert torch.equal(bat_after["labels"], bat_before["labels"]) and torch.equal(bat_after["i_k"],
                                                                                  bat_before["i_k"])
    # a generous caller limit behaves like the default
    ok = iso.cluster(Xd, k, sigma, iso.opts(spin_limit=10 ** 10))
    assert (ok[0].cpu().numpy() == ref["labels"]).all()

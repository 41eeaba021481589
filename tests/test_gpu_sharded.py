"""The sharded call (isoclust_cluster_sharded) on the GPU.

world = 1 runs the sharded code path (row-tile split, per-component minima
and omega shares through the caller's all-reduce, here the identity) and must
give isoclust_cluster's results bit for bit.  world = 2 runs as two processes
that both use cuda:0 and exchange through gloo on host copies (the kernels of
the two ranks never wait on each other; each rank's all-reduce is a host
call between its own launches): both ranks must agree, the labels must be the
oracle's and i_k within 1e-12 (the two ranks' omega shares are added in FP64,
so omega can differ from the one-GPU sum in the last bits).  A failing
callback gives ISOCLUST_ERR_COMM and leaves the library usable.
"""
import os
import time
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import _sharded_ranks  # noqa: E402


@pytest.fixture(scope="module")
def iso():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04739_gb300 import isoclust
    isoclust.load()
    return isoclust


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_world_one_equals_the_unsharded_call(iso):
    from paper_1702_04739_gb300 import workloads
    X, _ = workloads.blobs_anisotropic(seed=3, n=12000, k=10)
    Xd = torch.from_numpy(X).cuda()
    calls = []

    def identity(buf, count, op, stream):
        calls.append(op)
    lab1, res1, ik1 = iso.cluster_sharded(Xd, 10, 1.0, 0, 1, identity)
    lab0, res0, ik0 = iso.cluster(Xd, 10, 1.0)
    assert torch.equal(lab1, lab0) and torch.equal(res1, res0) and torch.equal(ik1, ik0)
    assert iso.REDUCE_SUM_F64 in calls and calls.count(iso.REDUCE_MIN_U64) >= 2


def test_failing_collective_is_reported(iso):
    from paper_1702_04739_gb300 import workloads
    X, _ = workloads.blobs_anisotropic(seed=4, n=3000, k=5)
    Xd = torch.from_numpy(X).cuda()

    def broken(buf, count, op, stream):
        raise RuntimeError("peer lost")
    with pytest.raises(iso.IsoclustError) as e:
        iso.cluster_sharded(Xd, 5, 1.0, 0, 2, broken)
    assert e.value.code == 9 and "peer lost" in str(e.value)
    torch.cuda.synchronize()
    lab, _, _ = iso.cluster(Xd, 5, 1.0)
    assert (lab.cpu().numpy() >= -1).all()


def test_two_ranks_on_one_gpu_through_gloo(iso, oracle_lib, tmp_path):
    import torch.multiprocessing as mp
    from paper_1702_04739_gb300 import workloads
    n = 6000
    ctx = mp.start_processes(_sharded_ranks.gpu_cluster_rank, args=(2, _free_port(), str(tmp_path), n), nprocs=2,
                             join=False, start_method="spawn")
    deadline = time.monotonic() + 300.0
    for p in ctx.processes:
        p.join(max(1.0, deadline - time.monotonic()))
    for p in ctx.processes:
        if p.is_alive():
            p.terminate()
            p.join(30.0)
    codes = [p.exitcode for p in ctx.processes]
    if codes != [0, 0]:
        def read(name):
            f = os.path.join(tmp_path, name)
            return open(f).read()[-3000:] if os.path.exists(f) else "(none)"
        report = "\n".join(f"rank {r}: exit {codes[r]}\n log:\n{read(f'gpu{r}.log')}\n error:\n{read(f'gpu{r}.err')}"
                           f"\n fault trace:\n{read(f'gpu{r}.trace')}" for r in range(2))
        raise AssertionError("a rank failed\n" + report)
    r0, r1 = (np.load(os.path.join(tmp_path, f"gpu{r}.npy")) for r in range(2))
    assert (r0 == r1).all()
    lab, res, ik = r0[:n].astype(np.int32), r0[n:2 * n].astype(np.uint8), float(r0[2 * n])
    X, _ = workloads.blobs_anisotropic(seed=11, n=n, k=8)
    ref = oracle_lib.cluster(X, 8, 1.0)
    assert (lab == ref["labels"]).all() and (res == ref["residual"]).all()
    assert abs(ik - ref["i_k"]) <= 1e-12 * ref["i_k"]
    Xd = torch.from_numpy(X).cuda()
    lab0, _, ik0 = iso.cluster(Xd, 8, 1.0)
    assert (lab0.cpu().numpy() == lab).all()
    assert abs(float(ik0.cpu()[0]) - ik) <= 1e-12 * ik

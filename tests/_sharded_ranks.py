"""Rank bodies of the sharded tests (world_size 2, gloo on 127.0.0.1), run as
spawned processes by tests/test_sharded_cpu.py and tests/test_gpu_sharded.py."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def _init(rank, world, port):
    import datetime
    import torch.distributed as dist
    # a rank that leaves early ends the other's next collective within a minute
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    return dist


def adapter_rank(rank, world, port, out):
    """The all-reduce adapter on host buffers: MIN of uint64 keys, SUM of doubles."""
    import torch  # noqa: F401
    from paper_1702_04739_gb300 import isoclust, sharded
    dist = _init(rank, world, port)
    ar = sharded.torch_allreduce(device_buffers=False)
    none = np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = np.array([5 + rank, 2 ** 62 - rank, none >> np.uint64(1), 7 * (1 - rank)], dtype=np.uint64)
    keys = np.concatenate([keys, np.array([none, none if rank else np.uint64(2 ** 63 + 5)], dtype=np.uint64)])
    vals = np.array([0.5 * (rank + 1), -1.25, 1e300, 3.0], dtype=np.float64)
    ar(keys.ctypes.data, keys.size, isoclust.REDUCE_MIN_U64, 0)
    ar(vals.ctypes.data, vals.size, isoclust.REDUCE_SUM_F64, 0)
    np.save(os.path.join(out, f"adapter{rank}.npy"), np.concatenate([keys.view(np.float64), vals]))
    dist.destroy_process_group()


def boruvka_rank(rank, world, port, out, tile_rows):
    """Boruvka rounds split by row tiles (t mod world == rank): each rank
    keys its own rows (the oracle's step), the per-component minima are
    combined by the adapter's all-reduce MIN (d2 bits, then the packed pair
    among the rows at that d2), and every rank merges the same components."""
    import torch  # noqa: F401
    import oracle
    from paper_1702_04739_gb300 import isoclust, sharded
    dist = _init(rank, world, port)
    ar = sharded.torch_allreduce(device_buffers=False)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(300, 4))
    n = X.shape[0]
    ntiles = -(-n // tile_rows)
    mine = np.concatenate([np.arange(t * tile_rows, min(n, (t + 1) * tile_rows))
                           for t in sharded.row_tiles_of(ntiles, rank, world)])
    comp = np.arange(n)
    edges = []
    NONE = np.uint64(0xFFFFFFFFFFFFFFFF)
    while len(np.unique(comp)) > 1:
        j, d2 = oracle.min_foreign(X, comp, mine)
        cd2 = np.full(n, NONE, dtype=np.uint64)
        bits = d2.view(np.uint64)
        for r, i in enumerate(mine):
            if j[r] >= 0:
                cd2[comp[i]] = min(cd2[comp[i]], bits[r])
        ar(cd2.ctypes.data, n, isoclust.REDUCE_MIN_U64, 0)
        cpair = np.full(n, NONE, dtype=np.uint64)
        for r, i in enumerate(mine):
            if j[r] >= 0 and bits[r] == cd2[comp[i]]:
                a, b = min(i, j[r]), max(i, j[r])
                cpair[comp[i]] = min(cpair[comp[i]], np.uint64((int(a) << 32) | int(b)))
        ar(cpair.ctypes.data, n, isoclust.REDUCE_MIN_U64, 0)
        p = {int(c): int(c) for c in np.unique(comp)}

        def f(x):
            while p[x] != x:
                x = p[x]
            return x
        for c in np.unique(comp):
            pr = int(cpair[c])
            a, b = pr >> 32, pr & 0xFFFFFFFF
            ra, rb = f(int(comp[a])), f(int(comp[b]))
            if ra != rb:
                p[max(ra, rb)] = min(ra, rb)
                edges.append((a, b))
        comp = np.array([f(int(c)) for c in comp])
    np.save(os.path.join(out, f"edges{rank}.npy"), np.array(sorted(edges), dtype=np.int64))
    dist.destroy_process_group()


def gpu_cluster_rank(rank, world, port, out, n):
    """isoclust_cluster_sharded on one GPU per rank (here both ranks share
    cuda:0), the exchange through gloo on host copies.  Each rank logs its
    collectives (op, count) and keeps its own error, so a failure names the
    rank that caused it (the other rank only sees the lost peer)."""
    import faulthandler
    import traceback
    import torch
    from paper_1702_04739_gb300 import isoclust, sharded, workloads
    trace = open(os.path.join(out, f"gpu{rank}.trace"), "w")
    faulthandler.enable(file=trace)
    log = open(os.path.join(out, f"gpu{rank}.log"), "w")
    try:
        dist = _init(rank, world, port)
        torch.cuda.set_device(0)
        X, _ = workloads.blobs_anisotropic(seed=11, n=n, k=8)
        Xd = torch.from_numpy(X).cuda()
        inner = sharded.torch_allreduce(device_buffers=True, device=Xd.device)

        def logged(ptr, count, op, stream):
            log.write(f"{op} {count}\n")
            log.flush()
            inner(ptr, count, op, stream)
        lab, res, ik = isoclust.cluster_sharded(Xd, 8, 1.0, rank, world, logged)
        np.save(os.path.join(out, f"gpu{rank}.npy"), np.concatenate([lab.cpu().numpy().astype(np.float64),
                                                                     res.cpu().numpy().astype(np.float64),
                                                                     ik.cpu().numpy()]))
        log.write("done\n")
        log.flush()
        dist.barrier()
        dist.destroy_process_group()
    except BaseException:
        with open(os.path.join(out, f"gpu{rank}.err"), "w") as f:
            f.write(traceback.format_exc())
        raise

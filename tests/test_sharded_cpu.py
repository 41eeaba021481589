"""The sharded call's host side on CPU ranks (world_size 2, gloo): the
row split, the all-reduce adapter, and the Boruvka exchange protocol (each
rank keys its own row tiles, per-component minima combined by all-reduce MIN,
the same merge everywhere) against the single-process tree of the oracle."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import _sharded_ranks  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(fn, *args):
    mp.start_processes(fn, args=(2, _free_port()) + args, nprocs=2, join=True, start_method="spawn")


def test_row_split_is_a_partition():
    from paper_1702_04739_gb300 import sharded
    for ntiles in (1, 2, 7, 782):
        for world in (1, 2, 3, 8):
            got = sorted(t for r in range(world) for t in sharded.row_tiles_of(ntiles, r, world))
            assert got == list(range(ntiles))


def test_allreduce_adapter_on_two_ranks(tmp_path):
    _spawn(_sharded_ranks.adapter_rank, str(tmp_path))
    a, b = (np.load(tmp_path / f"adapter{r}.npy") for r in range(2))
    assert (a.view(np.uint64) == b.view(np.uint64)).all()       # the keys' bits may read as NaN
    keys = a[:6].view(np.uint64)
    # unsigned minima, the all-ones "none" key included
    assert keys.tolist() == [5, 2 ** 62 - 1, 2 ** 63 - 1, 0, 2 ** 64 - 1, 2 ** 63 + 5]
    assert a[6:].tolist() == [1.5, -2.5, 2e300, 6.0]


def test_boruvka_exchange_on_two_ranks_gives_the_oracle_tree(tmp_path, oracle_lib):
    _spawn(_sharded_ranks.boruvka_rank, str(tmp_path), 16)
    e0, e1 = (np.load(tmp_path / f"edges{r}.npy") for r in range(2))
    assert (e0 == e1).all()
    rng = np.random.default_rng(7)
    X = rng.normal(size=(300, 4))
    eu, ev, _, _, _ = oracle_lib.mst_prim(X)
    assert sorted(map(tuple, e0.tolist())) == sorted(zip(eu.tolist(), ev.tolist()))

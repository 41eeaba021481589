"""Host side of the sharded call (isoclust_cluster_sharded): the all-reduce
callback over torch.distributed, and the rule that splits the rows.

The library splits the row-pairwise work of one point set across W
processes, one GPU each, and calls back for the exchange steps (Section
3.5's Boruvka rounds need the minimum key of every component over all rows;
eq. omega needs each row's sum over all tile pairs).  This module only
marshals those calls onto a torch.distributed process group: NCCL reduces the
device buffers in place on the caller's stream; any other backend (gloo)
reduces a host copy.
"""
from __future__ import annotations

import torch

from . import isoclust

TILE_ROWS = 128        # rows per tile of the tensor-core sweep


def row_tiles_of(ntiles: int, rank: int, world: int) -> range:
    """The 128-row tiles (of the sweep's norm-ordered rows) that `rank`
    sweeps: t with t mod world == rank, so every rank gets tiles from the
    whole norm range."""
    return range(rank, ntiles, world)


class _DeviceBuffer:
    """A device address as a tensor view (no copy), via __cuda_array_interface__."""

    def __init__(self, ptr: int, count: int, typestr: str, stream: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": stream or None}


SIGN = -(2 ** 63)      # int64 with only the sign bit set


def _view(ptr: int, count: int, op: int, stream: int, device_buffers: bool, device):
    if op == isoclust.REDUCE_MIN_U64:
        # uint64 keys (all ones = none) reduced as int64 with the sign bit
        # flipped: that maps the unsigned order onto the signed one
        typestr, dtype = "<i8", torch.int64
    elif op == isoclust.REDUCE_SUM_F64:
        typestr, dtype = "<f8", torch.float64
    else:
        raise ValueError(f"unknown reduction {op}")
    if device_buffers:
        t = torch.as_tensor(_DeviceBuffer(ptr, count, typestr, stream), device=device)
        if t.data_ptr() != ptr:
            raise RuntimeError("the device buffer was copied, not viewed")
        return t
    import ctypes
    import numpy as np
    buf = (ctypes.c_byte * (8 * count)).from_address(ptr)
    return torch.from_numpy(np.frombuffer(buf, dtype=np.int64 if dtype == torch.int64 else np.float64))


def torch_allreduce(group=None, device_buffers: bool = True, device=None):
    """An `allreduce` for isoclust.cluster_sharded over a torch.distributed
    group.  device_buffers=False treats the addresses as host memory (tests
    of the exchange on CPU ranks)."""
    import torch.distributed as dist
    backend = dist.get_backend(group)

    def allreduce(ptr: int, count: int, op: int, stream: int) -> None:
        t = _view(ptr, count, op, stream, device_buffers, device)
        umin = op == isoclust.REDUCE_MIN_U64
        rop = dist.ReduceOp.MIN if umin else dist.ReduceOp.SUM
        if umin:
            t.bitwise_xor_(SIGN)
        if not device_buffers or backend == "nccl":
            dist.all_reduce(t, op=rop, group=group)
        else:
            # a CPU backend: reduce a host copy (synchronous) and copy it back
            h = t.cpu()
            dist.all_reduce(h, op=rop, group=group)
            t.copy_(h)
        if umin:
            t.bitwise_xor_(SIGN)
    return allreduce

"""The allocation-free tree-stage entry point, through the C ABI.

isoclust_tree_isoperimetric_noalloc serves callers that cannot call
cudaMalloc (an application whose own pool owns the device memory, or a loop
that cannot take cudaMalloc's device-wide synchronisation).  Its scratch is a
fixed array in the library; these checks call it twice in a row on different
trees and compare each result with the allocating entry point under the tree
stage's bar (bit-exact labels, residual flags and i_k).  Collected last on
purpose, so that a stop-at-first-failure run has run everything else first.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOALLOC_MAX_N = 16384


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04739_gb300 import isoclust
    L = isoclust.load()
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.isoclust_tree_isoperimetric_noalloc.restype = ctypes.c_int
    L.isoclust_tree_isoperimetric_noalloc.argtypes = [I64, P, P, P, P, I32, P, P, P, P, P]
    return L


def _call(fn, parent, phi, om, p, k):
    n = parent.numel()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    residual = torch.empty(n, dtype=torch.uint8, device="cuda")
    ik = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = fn(n, parent.data_ptr(), phi.data_ptr(), om.data_ptr(), p.data_ptr() if p is not None else None, k, None,
            labels.data_ptr(), residual.data_ptr(), ik.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, labels.cpu().numpy(), residual.cpu().numpy(), float(ik.cpu()[0])


def test_noalloc_matches_allocating_entry_two_calls(lib):
    from paper_1702_04739_gb300 import workloads
    cases = [(3000, "random", 7, True), (NOALLOC_MAX_N, "deep", 20, False)]
    for seed, (n, shape, k, with_p) in enumerate(cases):
        parent, phi, om, p = workloads.random_rooted_tree(seed=100 + seed, n=n, shape=shape)
        c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        args = (c(parent), c(phi), c(om), c(p) if with_p else None, k)
        rc0, lab0, res0, ik0 = _call(lib.isoclust_tree_isoperimetric, *args)
        rc1, lab1, res1, ik1 = _call(lib.isoclust_tree_isoperimetric_noalloc, *args)
        assert rc0 == 0 and rc1 == 0, (rc0, rc1, lib.isoclust_last_error())
        assert ik1 == ik0
        assert (lab1 == lab0).all() and (res1 == res0).all()


def test_noalloc_rejects_trees_beyond_its_limit(lib):
    n = NOALLOC_MAX_N + 1
    parent = torch.full((n,), 0, dtype=torch.int32, device="cuda")
    dummy = torch.ones(n, dtype=torch.float64, device="cuda")
    rc, *_ = _call(lib.isoclust_tree_isoperimetric_noalloc, parent, dummy, dummy, None, 2)
    assert rc == 1
    assert b"ISOCLUST_NOALLOC_MAX_N" in lib.isoclust_last_error()

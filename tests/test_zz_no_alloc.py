"""The allocation-free tree-stage entry point, through the C ABI.

isoclust_tree_isoperimetric_noalloc serves callers that cannot call
cudaMalloc (an application whose own pool owns the device memory, or a loop
that cannot take cudaMalloc's device-wide synchronisation).  Its scratch is a
fixed array in the library; these checks call it several times in a row on
different trees - a small tree after the largest one, so stale scratch of a
bigger tree sits under a smaller one - and compare each result with the
allocating entry point under the tree stage's bar (bit-exact labels, residual
flags and i_k).  After one set-up call the device's free memory must not move.
Collected last on purpose, so that a stop-at-first-failure run has run
everything else first.
"""
import ctypes
import os
import re

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "isoclust.h")


def header_max_n() -> int:
    with open(HEADER) as f:
        m = re.search(r"#define\s+ISOCLUST_NOALLOC_MAX_N\s+(\d+)", f.read())
    assert m, "ISOCLUST_NOALLOC_MAX_N is not defined in include/isoclust.h"
    return int(m.group(1))


NOALLOC_MAX_N = header_max_n()


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


def _tree(seed, n, shape, with_p):
    from paper_1702_04739_gb300 import workloads
    parent, phi, om, p = workloads.random_rooted_tree(seed=seed, n=n, shape=shape)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return c(parent), c(phi), c(om), (c(p) if with_p else None)


def _call(fn, tree, k, out):
    parent, phi, om, p = tree
    n = parent.numel()
    labels, residual, ik = out
    rc = fn(n, parent.data_ptr(), phi.data_ptr(), om.data_ptr(), p.data_ptr() if p is not None else None, k, None,
            labels.data_ptr(), residual.data_ptr(), ik.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc


def _outputs(n):
    return (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"))


def _host(out, n):
    labels, residual, ik = out
    return labels[:n].cpu().numpy().copy(), residual[:n].cpu().numpy().copy(), float(ik.cpu()[0])


def test_header_limit_is_the_tested_limit():
    assert NOALLOC_MAX_N == 16384


def test_noalloc_matches_allocating_entry_and_allocates_nothing(lib):
    cases = [(3000, "random", 7, True), (NOALLOC_MAX_N, "deep", 20, False), (700, "binary", 5, True)]
    trees = [_tree(100 + q, n, shape, with_p) for q, (n, shape, _, with_p) in enumerate(cases)]
    out = _outputs(NOALLOC_MAX_N)
    # expected results from the allocating entry point (its scratch is
    # allocated here, before the free-memory reading)
    want = []
    for tree, (n, _, k, _) in zip(trees, cases):
        rc = _call(lib.isoclust_tree_isoperimetric, tree, k, out)
        assert rc == 0, lib.isoclust_last_error()
        want.append(_host(out, n))
    # set-up call: loads the module holding the static array, looks up its address
    assert _call(lib.isoclust_tree_isoperimetric_noalloc, trees[2], cases[2][2], out) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for tree, (n, _, k, _), (lab0, res0, ik0) in zip(trees, cases, want):
        rc = _call(lib.isoclust_tree_isoperimetric_noalloc, tree, k, out)
        assert rc == 0, lib.isoclust_last_error()
        lab1, res1, ik1 = _host(out, n)
        assert ik1 == ik0
        assert (lab1 == lab0).all() and (res1 == res0).all()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the allocation-free entry point changed the free device memory"


def test_noalloc_rejects_trees_beyond_its_limit(lib):
    n = NOALLOC_MAX_N + 1
    parent = torch.full((n,), 0, dtype=torch.int32, device="cuda")
    dummy = torch.ones(n, dtype=torch.float64, device="cuda")
    rc = _call(lib.isoclust_tree_isoperimetric_noalloc, (parent, dummy, dummy, None), 2, _outputs(n))
    assert rc == 1
    assert b"ISOCLUST_NOALLOC_MAX_N" in lib.isoclust_last_error()

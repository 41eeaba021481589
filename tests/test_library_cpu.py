"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol declared in include/isoclust.h, and rejects bad arguments on the
host before any device work (no GPU needed, no compute call made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1702_04739_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "isoclust.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isoclust_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("isoclust_cluster_mst", "isoclust_tree_isoperimetric", "isoclust_cluster",
                 "isoclust_vertex_weights", "isoclust_last_error", "isoclust_opts_default"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_library_is_sm103a_only():
    from paper_1702_04739_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_defaults_and_strings(lib):
    from paper_1702_04739_gb300 import isoclust
    L = isoclust.load()
    o = L.isoclust_opts_default()
    assert o.alpha == 0.0 and o.omega_mode == 0 and o.precision == 0 and o.root == 0 and o.include_self == 0
    assert L.isoclust_abi_version() == 1
    assert L.isoclust_status_string(2) == b"ISOCLUST_ERR_K_GT_N"
    assert L.isoclust_status_string(0) == b"ISOCLUST_OK"


def test_host_side_validation_without_device_work():
    """Each of these calls returns before any CUDA call (argument checks only)."""
    from paper_1702_04739_gb300 import isoclust
    L = isoclust.load()
    fake = ctypes.c_void_p(16)          # never dereferenced on these paths
    n, d = 10, 3
    assert L.isoclust_cluster(None, n, d, 0, 2, 1.0, None, fake, fake, fake, None) == 1
    assert L.isoclust_cluster(fake, 1, d, 0, 1, 1.0, None, fake, fake, fake, None) == 1
    assert L.isoclust_cluster(fake, n, 0, 0, 2, 1.0, None, fake, fake, fake, None) == 1
    assert L.isoclust_cluster(fake, n, d, 7, 2, 1.0, None, fake, fake, fake, None) == 1
    assert L.isoclust_cluster(fake, n, d, 0, 11, 1.0, None, fake, fake, fake, None) == 2
    assert L.isoclust_cluster(fake, n, d, 0, 0, 1.0, None, fake, fake, fake, None) == 1
    assert L.isoclust_cluster(fake, n, d, 0, 2, 0.0, None, fake, fake, fake, None) == 1
    assert L.isoclust_cluster(fake, n, d, 0, 2, float("inf"), None, fake, fake, fake, None) == 1
    bad = isoclust.opts(root=10)
    assert L.isoclust_cluster(fake, n, d, 0, 2, 1.0, ctypes.byref(bad), fake, fake, fake, None) == 1
    bad = isoclust.opts(alpha=-1.0)
    assert L.isoclust_cluster(fake, n, d, 0, 2, 1.0, ctypes.byref(bad), fake, fake, fake, None) == 1
    bad = isoclust.opts(precision=2)
    assert L.isoclust_cluster(fake, n, d, 1, 2, 1.0, ctypes.byref(bad), fake, fake, fake, None) == 1
    assert L.isoclust_cluster_mst(fake, n, d, 0, None, None, fake, fake, None) == 1
    assert L.isoclust_vertex_weights(fake, n, d, 0, -1.0, None, fake, None, None) == 1
    assert L.isoclust_tree_isoperimetric(0, fake, fake, fake, None, 1, None, fake, fake, fake, None) == 1
    assert L.isoclust_tree_isoperimetric(5, fake, fake, fake, None, 6, None, fake, fake, fake, None) == 2
    assert L.isoclust_tree_isoperimetric(5, None, fake, fake, None, 2, None, fake, fake, fake, None) == 1
    assert b"exceeds" in L.isoclust_last_error() or b"NULL" in L.isoclust_last_error()
    # the sweep-variant setting is host state only
    assert L.isoclust_set_sweep_variant(4) == 1 and L.isoclust_set_sweep_variant(-2) == 1
    assert L.isoclust_set_sweep_variant(2) == 0 and L.isoclust_set_sweep_variant(-1) == 0


def test_binding_requires_cuda_tensors():
    torch = pytest.importorskip("torch")
    from paper_1702_04739_gb300 import isoclust
    with pytest.raises(TypeError):
        isoclust.cluster(torch.zeros(10, 3), 2, 1.0)


def test_batched_host_side_validation():
    """isoclust_cluster_batched checks its host plan arrays before any CUDA call."""
    from paper_1702_04739_gb300 import isoclust
    L = isoclust.load()
    fake = ctypes.c_void_p(16)
    offs = (ctypes.c_int64 * 4)(0, 5, 9, 20)
    ks = (ctypes.c_int32 * 3)(2, 3, 4)

    def call(X=fake, o=offs, nsets=3, d=3, dtype=0, k=ks, sigma=1.0, opts=None):
        return L.isoclust_cluster_batched(X, o, nsets, d, dtype, k, ctypes.c_double(sigma), opts,
                                          fake, fake, fake, None, None)

    assert call(X=None) == 1
    assert call(nsets=0) == 1
    assert call(dtype=1) == 1                                   # F32 only
    assert call(sigma=0.0) == 1
    assert call(o=(ctypes.c_int64 * 4)(1, 5, 9, 20)) == 1        # offsets[0] != 0
    assert call(o=(ctypes.c_int64 * 4)(0, 1, 9, 20)) == 1        # a one-point set
    assert call(k=(ctypes.c_int32 * 3)(2, 0, 4)) == 1            # k < 1
    assert call(k=(ctypes.c_int32 * 3)(2, 5, 4)) == 2            # k above the set's size
    bad = isoclust.opts(alpha=0.5)
    assert call(opts=ctypes.byref(bad)) == 1
    bad = isoclust.opts(omega_mode=1)
    assert call(opts=ctypes.byref(bad)) == 1
    bad = isoclust.opts(precision=1)
    assert call(opts=ctypes.byref(bad)) == 1


def test_batched_workload_recipe():
    import numpy as np
    from paper_1702_04739_gb300 import workloads as W
    X, offs, ks = W.batched_sets(seed=3, nsets=64, d=32)
    sizes = np.diff(offs)
    assert X.dtype == np.float32 and X.shape == (offs[-1], 32)
    assert offs[0] == 0 and (sizes >= 64).all() and (sizes <= 8192).all()
    assert ((ks >= 2) & (ks <= 8)).all()
    X2, offs2, ks2 = W.batched_sets(seed=3, nsets=64, d=32)
    assert (X == X2).all() and (offs == offs2).all() and (ks == ks2).all()
    Xs, offs_s, ks_s = W.batched_sets(seed=1, d=4, sizes=[2, 3, 70])
    assert list(np.diff(offs_s)) == [2, 3, 70] and (ks_s <= np.diff(offs_s)).all()


def test_process_settings_validate_their_argument():
    """The graph and test-hook switches take 0 or 1 (no device work)."""
    from paper_1702_04739_gb300 import isoclust
    L = isoclust.load()
    assert L.isoclust_set_batched_graphs(2) == 1 and L.isoclust_set_test_stalled_wait(-1) == 1
    assert L.isoclust_set_batched_graphs(1) == 0 and L.isoclust_set_test_stalled_wait(0) == 0
    assert L.isoclust_set_omega_gram(2) == 1 and L.isoclust_set_omega_gram(-1) == 0
    assert L.isoclust_set_mst_prune(-2) == 1 and L.isoclust_set_mst_prune(-1) == 0

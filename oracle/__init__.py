"""FP64 CPU oracle for the isoperimetric clustering hot path (arXiv 1702.04739).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA path.  The arithmetic lives in
``isoclust_oracle.c`` (plain C, FP64, no FMA contraction); this module only
compiles it with gcc and marshals numpy arrays.

Functions and the passages they follow:
  d2           Section 2.2 step 1 (edge weight ||x_i - x_j||, kept squared)
  mst_prim     Algorithm 3 (Prim with min-reduction), key (d2, min, max)
  mst_kruskal  textbook Kruskal over all pairs (self-check of mst_prim)
  nn_rows      exact nearest neighbour (smallest key) of sampled rows
  min_foreign  one Boruvka step: each row's smallest-key edge to another component
  weights      eq. omega and eq. potential
  flow         eq. phi
  parent_flow  eq. phi on the parent edge of every vertex of a rooted tree
  bfs_order    Section 2.2 step 3 (BFS order, children ascending)
  decision     Algorithm 1
  decision_detail  Algorithm 1 with each visited vertex's branch and the
               two critical thresholds of its tests (decision margins)
  tree_stage   Algorithm 2 (bisection to the last bit) + final Algorithm 1
  cluster      Section 2.2 steps 1-5 end to end
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isoclust_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_d2.restype = _dbl
            lib.oracle_d2.argtypes = [_ptr, _i64, _i32, _i64, _i64]
            lib.oracle_flow.restype = _dbl
            lib.oracle_flow.argtypes = [_dbl, _dbl]
            lib.oracle_parent_flow.restype = ctypes.c_int
            lib.oracle_parent_flow.argtypes = [_ptr, _i64, _i32, _ptr, _dbl, _ptr]
            lib.oracle_mst_prim.restype = ctypes.c_int
            lib.oracle_mst_prim.argtypes = [_ptr, _i64, _i32, _i64, _ptr, _ptr, _ptr, _ptr, _ptr]
            lib.oracle_mst_kruskal.restype = ctypes.c_int
            lib.oracle_mst_kruskal.argtypes = [_ptr, _i64, _i32, _ptr, _ptr, _ptr]
            lib.oracle_nn_rows.restype = ctypes.c_int
            lib.oracle_nn_rows.argtypes = [_ptr, _i64, _i32, _ptr, _i64, _ptr, _ptr]
            lib.oracle_min_foreign.restype = ctypes.c_int
            lib.oracle_min_foreign.argtypes = [_ptr, _i64, _i32, _ptr, _ptr, _i64, _ptr, _ptr]
            lib.oracle_weights.restype = ctypes.c_int
            lib.oracle_weights.argtypes = [_ptr, _i64, _i32, _dbl, _dbl, _i32, _ptr, _i64, _ptr, _ptr]
            lib.oracle_bfs_order.restype = ctypes.c_int
            lib.oracle_bfs_order.argtypes = [_i64, _ptr, _ptr]
            lib.oracle_decision.restype = _i64
            lib.oracle_decision.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _i64, _dbl]
            lib.oracle_decision_detail.restype = _i64
            lib.oracle_decision_detail.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _i64, _dbl, _ptr, _ptr, _ptr]
            lib.oracle_tree_stage.restype = ctypes.c_int
            lib.oracle_tree_stage.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _i64,
                                              _ptr, _ptr, _ptr, _ptr, _ptr, _ptr]
            lib.oracle_cluster.restype = ctypes.c_int
            lib.oracle_cluster.argtypes = [_ptr, _i64, _i32, _i64, _dbl, _dbl, _i32, _i32, _i64,
                                           _ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr,
                                           _ptr, _ptr, _ptr, _ptr, _ptr, _ptr]
            lib.oracle_ik_fixed.restype = ctypes.c_int
            lib.oracle_ik_fixed.argtypes = [_ptr, _i64, _i32, _ptr, _dbl, _ptr, _ptr, _i64, _ptr, _ptr, _ptr, _ptr]
            lib.oracle_ik_grad.restype = ctypes.c_int
            lib.oracle_ik_grad.argtypes = [_ptr, _i64, _i32, _ptr, _dbl, _ptr, _ptr, _i32, _ptr, _ptr, _ptr, _ptr]
            lib.oracle_set_threads.restype = None
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_get_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _X(X):
    # f32 -> f64 conversion is exact, so the oracle sees the same values.
    return np.ascontiguousarray(np.asarray(X, dtype=np.float64))


def d2(X, i: int, j: int) -> float:
    X = _X(X)
    return float(_load().oracle_d2(_p(X), X.shape[0], X.shape[1], int(i), int(j)))


def flow(d2v: float, sigma: float) -> float:
    return float(_load().oracle_flow(float(d2v), float(sigma)))


def parent_flow(X, parent, sigma: float):
    """phi of every vertex's parent edge (eq. phi), 0 at the root."""
    X = _X(X)
    parent = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    out = np.zeros(parent.size, np.float64)
    if _load().oracle_parent_flow(_p(X), X.shape[0], X.shape[1], _p(parent), float(sigma), _p(out)):
        raise ValueError("parent index out of range")
    return out


def mst_prim(X, root: int = 0):
    """Returns (eu, ev, ed2, parent, depth); edges sorted by (d2, min, max)."""
    X = _X(X)
    n, d = X.shape
    m = max(n - 1, 0)
    eu = np.zeros(m, np.int32); ev = np.zeros(m, np.int32); ed2 = np.zeros(m, np.float64)
    parent = np.zeros(n, np.int32); depth = np.zeros(n, np.int32)
    rc = _load().oracle_mst_prim(_p(X), n, d, int(root), _p(eu), _p(ev), _p(ed2), _p(parent), _p(depth))
    if rc:
        raise RuntimeError(f"oracle_mst_prim failed: {rc}")
    return eu, ev, ed2, parent, depth


def mst_kruskal(X):
    X = _X(X)
    n, d = X.shape
    m = max(n - 1, 0)
    eu = np.zeros(m, np.int32); ev = np.zeros(m, np.int32); ed2 = np.zeros(m, np.float64)
    rc = _load().oracle_mst_kruskal(_p(X), n, d, _p(eu), _p(ev), _p(ed2))
    if rc:
        raise RuntimeError(f"oracle_mst_kruskal failed: {rc}")
    return eu, ev, ed2


def nn_rows(X, rows):
    X = _X(X)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    nn = np.zeros(rows.size, np.int32); nd = np.zeros(rows.size, np.float64)
    _load().oracle_nn_rows(_p(X), X.shape[0], X.shape[1], _p(rows), rows.size, _p(nn), _p(nd))
    return nn, nd


def min_foreign(X, comp, rows):
    """For each row, (j, d2) of its smallest-key edge to another component."""
    X = _X(X)
    comp = np.ascontiguousarray(np.asarray(comp, dtype=np.int32))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    j = np.zeros(rows.size, np.int32); d2v = np.zeros(rows.size, np.float64)
    _load().oracle_min_foreign(_p(X), X.shape[0], X.shape[1], _p(comp), _p(rows), rows.size, _p(j), _p(d2v))
    return j, d2v


def weights(X, sigma: float, alpha: float = 0.0, include_self: bool = False, rows=None):
    """(omega, p) for all rows, or for the listed rows only."""
    X = _X(X)
    n, d = X.shape
    if rows is None:
        cnt, rp = n, None
    else:
        rp = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        cnt = rp.size
    om = np.zeros(cnt, np.float64); p = np.zeros(cnt, np.float64)
    _load().oracle_weights(_p(X), n, d, float(sigma), float(alpha), int(bool(include_self)),
                           _p(rp), cnt, _p(om), _p(p))
    return om, p


def bfs_order(parent):
    parent = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    order = np.zeros(parent.size, np.int32)
    rc = _load().oracle_bfs_order(parent.size, _p(parent), _p(order))
    if rc:
        raise ValueError("parent[] is not a rooted tree")
    return order


def _tree_args(parent, phi_par, omega, p):
    parent = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    phi_par = np.ascontiguousarray(np.asarray(phi_par, dtype=np.float64))
    omega = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    p = None if p is None else np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    return parent, phi_par, omega, p


def decision(parent, phi_par, omega, p, k: int, N: float) -> int:
    """Algorithm 1: number of cuts made (== k means YES)."""
    parent, phi_par, omega, p = _tree_args(parent, phi_par, omega, p)
    r = _load().oracle_decision(parent.size, _p(parent), _p(phi_par), _p(omega), _p(p), int(k), float(N))
    if r < 0:
        raise ValueError("parent[] is not a rooted tree")
    return int(r)


def decision_detail(parent, phi_par, omega, p, k: int, N: float) -> dict:
    """Algorithm 1 at N with its early stop: per vertex the branch taken
    (0 cut, 1 join, 2 discard, -1 not visited) and the thresholds at which
    its cut test ((phi(e) + p-hat) / omega-hat) and join test
    ((p-hat - phi(e)) / omega-hat) change; cuts = the number of cuts made."""
    parent, phi_par, omega, p = _tree_args(parent, phi_par, omega, p)
    n = parent.size
    code = np.zeros(n, np.int8)
    ncut = np.zeros(n, np.float64)
    njoin = np.zeros(n, np.float64)
    r = _load().oracle_decision_detail(n, _p(parent), _p(phi_par), _p(omega), _p(p), int(k), float(N),
                                       _p(code), _p(ncut), _p(njoin))
    if r < 0:
        raise ValueError("parent[] is not a rooted tree")
    return dict(code=code, ncut=ncut, njoin=njoin, cuts=int(r))


def tree_stage(parent, phi_par, omega, p, k: int) -> dict:
    """Algorithm 2 + final Algorithm 1 on a rooted weighted tree."""
    parent, phi_par, omega, p = _tree_args(parent, phi_par, omega, p)
    n = parent.size
    labels = np.zeros(n, np.int32); residual = np.zeros(n, np.uint8)
    ik = np.zeros(1, np.float64); beta = np.zeros(1, np.float64)
    stats = np.zeros(8, np.float64); info = np.zeros(1, np.int64)
    rc = _load().oracle_tree_stage(n, _p(parent), _p(phi_par), _p(omega), _p(p), int(k),
                                   _p(labels), _p(residual), _p(ik), _p(beta), _p(stats), _p(info))
    if rc:
        raise RuntimeError(f"oracle_tree_stage failed: {rc}")
    return dict(labels=labels, residual=residual, i_k=float(ik[0]), beta=float(beta[0]),
                stats=stats, calls=int(info[0]))


def cluster(X, k: int, sigma: float, alpha: float = 0.0, omega_mode: int = 0,
            include_self: bool = False, root: int = 0) -> dict:
    """Section 2.2 steps 1-5 end to end."""
    X = _X(X)
    n, d = X.shape
    m = n - 1
    eu = np.zeros(m, np.int32); ev = np.zeros(m, np.int32); ed2 = np.zeros(m, np.float64)
    parent = np.zeros(n, np.int32); phi = np.zeros(n, np.float64)
    om = np.zeros(n, np.float64); p = np.zeros(n, np.float64)
    labels = np.zeros(n, np.int32); residual = np.zeros(n, np.uint8)
    ik = np.zeros(1, np.float64); beta = np.zeros(1, np.float64)
    stats = np.zeros(8, np.float64); info = np.zeros(1, np.int64)
    rc = _load().oracle_cluster(_p(X), n, d, int(k), float(sigma), float(alpha), int(omega_mode),
                                int(bool(include_self)), int(root),
                                _p(eu), _p(ev), _p(ed2), _p(parent), _p(phi), _p(om), _p(p),
                                _p(labels), _p(residual), _p(ik), _p(beta), _p(stats), _p(info))
    if rc:
        raise RuntimeError(f"oracle_cluster failed: {rc}")
    return dict(edge_u=eu, edge_v=ev, edge_d2=ed2, parent=parent, phi_par=phi, omega=om, p=p,
                labels=labels, residual=residual, i_k=float(ik[0]), beta=float(beta[0]),
                stats=stats, calls=int(info[0]))


def ik_fixed(X, scale, sigma: float, parent, labels, k: int) -> dict:
    """i_k on a fixed tree and subpartition (alpha = 0): the ratio
    phi(dA_j)/omega(A_j) of every label j < k from z = scale * x, the largest
    (R) and its label (jstar)."""
    X = _X(X)
    n, d = X.shape
    s = np.ascontiguousarray(np.asarray(scale, dtype=np.float64).reshape(d))
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    phk = np.zeros(k, np.float64); omk = np.zeros(k, np.float64)
    js = np.zeros(1, np.int32); R = np.zeros(1, np.float64)
    rc = _load().oracle_ik_fixed(_p(X), n, d, _p(s), float(sigma), _p(parent), _p(labels), int(k),
                                 _p(phk), _p(omk), _p(js), _p(R))
    if rc:
        raise RuntimeError(f"oracle_ik_fixed failed: {rc}")
    return dict(R=float(R[0]), jstar=int(js[0]), phi=phk, omega=omk)


def ik_grad(X, scale, sigma: float, parent, labels, jstar: int) -> dict:
    """dR/dX, dR/dscale, dR/dsigma of R = phi(dA*)/omega(A*) for the set jstar
    on a fixed tree and subpartition."""
    X = _X(X)
    n, d = X.shape
    s = np.ascontiguousarray(np.asarray(scale, dtype=np.float64).reshape(d))
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    dX = np.zeros((n, d), np.float64); ds = np.zeros(d, np.float64)
    dsig = np.zeros(1, np.float64); R = np.zeros(1, np.float64)
    rc = _load().oracle_ik_grad(_p(X), n, d, _p(s), float(sigma), _p(parent), _p(labels), int(jstar),
                                _p(dX), _p(ds), _p(dsig), _p(R))
    if rc:
        raise RuntimeError(f"oracle_ik_grad failed: {rc}")
    return dict(dX=dX, dscale=ds, dsigma=float(dsig[0]), R=float(R[0]))

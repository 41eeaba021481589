"""Thin Python binding of the isoclust C ABI (include/isoclust.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library libisoclust.so.  Inputs are torch CUDA tensors (device memory);
outputs are allocated with torch on the same device; the call is queued on
torch's current stream.  There is no CPU fallback: if the library cannot be
loaded, or a tensor is not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

F32, F64 = 0, 1
OMEGA_FULL, OMEGA_TREE = 0, 1
PREC_AUTO, PREC_FP64, PREC_FP32, PREC_BF16_TC = 0, 1, 2, 3

STATUS = {
    0: "ISOCLUST_OK", 1: "ISOCLUST_ERR_INVALID_ARG", 2: "ISOCLUST_ERR_K_GT_N", 3: "ISOCLUST_ERR_NONFINITE",
    4: "ISOCLUST_ERR_OOM", 5: "ISOCLUST_ERR_CUDA", 6: "ISOCLUST_ERR_TIMEOUT", 7: "ISOCLUST_ERR_NO_SOLUTION",
    8: "ISOCLUST_ERR_INTERNAL", 9: "ISOCLUST_ERR_COMM",
}
REDUCE_MIN_U64, REDUCE_SUM_F64 = 0, 1
# int32 allreduce(void *ctx, void *buf, int64 count, int32 op, void *stream)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_void_p)


class Comm(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("world", ctypes.c_int32), ("allreduce", ALLREDUCE_FN),
                ("ctx", ctypes.c_void_p)]


class IsoclustError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("omega_mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("root", ctypes.c_int32), ("include_self", ctypes.c_int32), ("spin_limit", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libisoclust.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libisoclust.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        lib.isoclust_opts_default.restype = Opts
        lib.isoclust_last_error.restype = ctypes.c_char_p
        lib.isoclust_status_string.restype = ctypes.c_char_p
        lib.isoclust_status_string.argtypes = [ctypes.c_int]
        lib.isoclust_abi_version.restype = _I32
        lib.isoclust_kernel_launches.restype = _I64
        lib.isoclust_cluster_mst.restype = ctypes.c_int
        lib.isoclust_cluster_mst.argtypes = [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P]
        lib.isoclust_vertex_weights.restype = ctypes.c_int
        lib.isoclust_vertex_weights.argtypes = [_P, _I64, _I32, _I32, _D, _P, _P, _P, _P]
        lib.isoclust_tree_isoperimetric.restype = ctypes.c_int
        lib.isoclust_tree_isoperimetric.argtypes = [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P]
        lib.isoclust_cluster.restype = ctypes.c_int
        lib.isoclust_cluster.argtypes = [_P, _I64, _I32, _I32, _I32, _D, _P, _P, _P, _P, _P]
        lib.isoclust_cluster_sharded.restype = ctypes.c_int
        lib.isoclust_cluster_sharded.argtypes = [_P, _I64, _I32, _I32, _I32, _D, _P, _P, _P, _P, _P, _P]
        lib.isoclust_cluster_detail.restype = ctypes.c_int
        lib.isoclust_cluster_detail.argtypes = [_P, _I64, _I32, _I32, _I32, _D, _P, _P, _P, _P,
                                                _P, _P, _P, _P, _P, _P, _P, _P, _P]
        lib.isoclust_cluster_batched.restype = ctypes.c_int
        lib.isoclust_cluster_batched.argtypes = [_P, _P, _I32, _I32, _I32, _P, _D, _P, _P, _P, _P, _P, _P]
        lib.isoclust_cluster_batched_detail.restype = ctypes.c_int
        lib.isoclust_cluster_batched_detail.argtypes = [_P, _P, _I32, _I32, _I32, _P, _D, _P, _P, _P, _P, _P,
                                                        _P, _P, _P, _P]
        lib.isoclust_scale_features.restype = ctypes.c_int
        lib.isoclust_scale_features.argtypes = [_P, _I64, _I32, _I32, _P, _P, _P]
        lib.isoclust_ik_backward.restype = ctypes.c_int
        lib.isoclust_ik_backward.argtypes = [_P, _I64, _I32, _I32, _P, _D, _P, _P, _I32, _P, _P, _D, _P, _P, _P, _P,
                                             _P]
        lib.isoclust_last_profile.restype = None
        lib.isoclust_last_profile.argtypes = [_P, _P]
        lib.isoclust_last_omega_kernel_ms.restype = _D
        lib.isoclust_last_omega_kernel_ms.argtypes = []
        lib.isoclust_last_omega_gram_ms.restype = _D
        lib.isoclust_last_omega_gram_ms.argtypes = [_P, _P]
        lib.isoclust_set_sweep_variant.restype = ctypes.c_int
        lib.isoclust_set_sweep_variant.argtypes = [ctypes.c_int32]
        lib.isoclust_last_sweep_variant.restype = ctypes.c_int32
        lib.isoclust_last_sweep_variant.argtypes = []
        lib.isoclust_last_batched_graph_mode.restype = ctypes.c_int32
        lib.isoclust_last_batched_graph_mode.argtypes = []
        lib.isoclust_set_batched_graphs.restype = ctypes.c_int
        lib.isoclust_set_batched_graphs.argtypes = [ctypes.c_int32]
        lib.isoclust_set_omega_gram.restype = ctypes.c_int
        lib.isoclust_set_omega_gram.argtypes = [ctypes.c_int32]
        lib.isoclust_set_mst_prune.restype = ctypes.c_int
        lib.isoclust_set_mst_prune.argtypes = [ctypes.c_int32]
        lib.isoclust_set_test_stalled_wait.restype = ctypes.c_int
        lib.isoclust_set_test_stalled_wait.argtypes = [ctypes.c_int32]
        lib.isoclust_last_mst_tiles.restype = None
        lib.isoclust_last_mst_tiles.argtypes = [_P]
        lib.isoclust_last_omega_tiles.restype = None
        lib.isoclust_last_omega_tiles.argtypes = [_P]
        _lib = lib
        return lib


def opts(alpha: float = 0.0, omega_mode: int = OMEGA_FULL, precision: int = PREC_AUTO, root: int = 0,
         include_self: bool = False, spin_limit: int = 0) -> Opts:
    return Opts(float(alpha), int(omega_mode), int(precision), int(root), int(bool(include_self)), int(spin_limit))


def _check(code: int):
    if code != 0:
        raise IsoclustError(code, (load().isoclust_last_error() or b"").decode())


def _dev_ptr(t: torch.Tensor, dtype=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("isoclust takes CUDA tensors (device memory)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _points(X: torch.Tensor):
    if X.dim() != 2:
        raise ValueError("X must be 2-D (n, d)")
    if X.dtype == torch.float32:
        dt = F32
    elif X.dtype == torch.float64:
        dt = F64
    else:
        raise TypeError("X must be float32 or float64")
    return _dev_ptr(X), X.shape[0], X.shape[1], dt


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _opts_ptr(o):
    return ctypes.byref(o) if o is not None else None


def cluster_mst(X: torch.Tensor, o: Opts | None = None):
    """(edge_u, edge_v, edge_d2) of the exact MST, in key order."""
    lib = load()
    xp, n, d, dt = _points(X)
    m = max(n - 1, 0)
    eu = torch.empty(m, dtype=torch.int32, device=X.device)
    ev = torch.empty(m, dtype=torch.int32, device=X.device)
    ed = torch.empty(m, dtype=torch.float64, device=X.device)
    _check(lib.isoclust_cluster_mst(xp, n, d, dt, _opts_ptr(o), eu.data_ptr(), ev.data_ptr(), ed.data_ptr(),
                                    _stream(X.device)))
    return eu, ev, ed


def vertex_weights(X: torch.Tensor, sigma: float, o: Opts | None = None, want_p: bool = True):
    """(omega, p) of eq. omega / eq. potential."""
    lib = load()
    xp, n, d, dt = _points(X)
    om = torch.empty(n, dtype=torch.float64, device=X.device)
    p = torch.empty(n, dtype=torch.float64, device=X.device) if want_p else None
    _check(lib.isoclust_vertex_weights(xp, n, d, dt, float(sigma), _opts_ptr(o), om.data_ptr(),
                                       p.data_ptr() if p is not None else None, _stream(X.device)))
    return om, p


def tree_isoperimetric(parent: torch.Tensor, phi_par: torch.Tensor, omega: torch.Tensor, p, k: int,
                       o: Opts | None = None):
    """(labels, residual, i_k) of Algorithms 2 + 1 + 4 on a rooted weighted tree."""
    lib = load()
    n = parent.numel()
    dev = parent.device
    pp = _dev_ptr(parent, torch.int32)
    fp = _dev_ptr(phi_par, torch.float64)
    wp = _dev_ptr(omega, torch.float64)
    qp = _dev_ptr(p, torch.float64) if p is not None else None
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    residual = torch.empty(n, dtype=torch.uint8, device=dev)
    ik = torch.empty(1, dtype=torch.float64, device=dev)
    _check(lib.isoclust_tree_isoperimetric(n, pp, fp, wp, qp, int(k), _opts_ptr(o), labels.data_ptr(),
                                           residual.data_ptr(), ik.data_ptr(), _stream(dev)))
    return labels, residual, ik


def cluster(X: torch.Tensor, k: int, sigma: float, o: Opts | None = None):
    """(labels, residual, i_k) of the whole hot path."""
    lib = load()
    xp, n, d, dt = _points(X)
    labels = torch.empty(n, dtype=torch.int32, device=X.device)
    residual = torch.empty(n, dtype=torch.uint8, device=X.device)
    ik = torch.empty(1, dtype=torch.float64, device=X.device)
    _check(lib.isoclust_cluster(xp, n, d, dt, int(k), float(sigma), _opts_ptr(o), labels.data_ptr(),
                                residual.data_ptr(), ik.data_ptr(), _stream(X.device)))
    return labels, residual, ik


def cluster_into(X: torch.Tensor, k: int, sigma: float, labels, residual, ik, o: Opts | None = None):
    """cluster() writing into caller-provided device tensors."""
    lib = load()
    xp, n, d, dt = _points(X)
    _check(lib.isoclust_cluster(xp, n, d, dt, int(k), float(sigma), _opts_ptr(o), labels.data_ptr(),
                                residual.data_ptr(), ik.data_ptr(), _stream(X.device)))


def cluster_sharded(X: torch.Tensor, k: int, sigma: float, rank: int, world: int, allreduce,
                    o: Opts | None = None):
    """isoclust_cluster_sharded: the pairwise work split across `world`
    processes (this one is `rank`); every rank passes the same X and gets the
    same (labels, residual, i_k).  allreduce(buf, count, op, stream) reduces
    `count` elements at device address `buf` in place across the ranks
    (op REDUCE_MIN_U64 or REDUCE_SUM_F64), ordered on `stream`; it raises
    on failure.  See sharded.torch_allreduce for one over torch.distributed."""
    lib = load()
    xp, n, d, dt = _points(X)
    dev = X.device
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    residual = torch.empty(n, dtype=torch.uint8, device=dev)
    ik = torch.empty(1, dtype=torch.float64, device=dev)
    failure = []

    def cb(ctx, buf, count, op, stream):
        try:
            allreduce(int(buf), int(count), int(op), int(stream or 0))
            return 0
        except Exception as e:      # reported as ISOCLUST_ERR_COMM; the exception is re-raised below
            failure.append(e)
            return 1
    fn = ALLREDUCE_FN(cb)
    comm = Comm(int(rank), int(world), fn, None)
    code = lib.isoclust_cluster_sharded(xp, n, d, dt, int(k), float(sigma), _opts_ptr(o), ctypes.byref(comm),
                                        labels.data_ptr(), residual.data_ptr(), ik.data_ptr(), _stream(dev))
    if failure:
        raise IsoclustError(code, f"all-reduce callback failed: {failure[0]!r}") from failure[0]
    _check(code)
    return labels, residual, ik


def cluster_detail(X: torch.Tensor, k: int, sigma: float, o: Opts | None = None) -> dict:
    lib = load()
    xp, n, d, dt = _points(X)
    dev = X.device
    out = dict(
        labels=torch.empty(n, dtype=torch.int32, device=dev),
        residual=torch.empty(n, dtype=torch.uint8, device=dev),
        i_k=torch.empty(1, dtype=torch.float64, device=dev),
        parent=torch.empty(n, dtype=torch.int32, device=dev),
        phi_par=torch.empty(n, dtype=torch.float64, device=dev),
        omega=torch.empty(n, dtype=torch.float64, device=dev),
        p=torch.empty(n, dtype=torch.float64, device=dev),
        beta=torch.empty(1, dtype=torch.float64, device=dev),
        edge_u=torch.empty(max(n - 1, 0), dtype=torch.int32, device=dev),
        edge_v=torch.empty(max(n - 1, 0), dtype=torch.int32, device=dev),
        edge_d2=torch.empty(max(n - 1, 0), dtype=torch.float64, device=dev),
    )
    _check(lib.isoclust_cluster_detail(
        xp, n, d, dt, int(k), float(sigma), _opts_ptr(o),
        *[out[key].data_ptr() for key in ("labels", "residual", "i_k", "parent", "phi_par", "omega", "p", "beta",
                                          "edge_u", "edge_v", "edge_d2")], _stream(dev)))
    return out


class BatchPlan:
    """Host arrays of a batch (offsets, ks) marshalled once for repeated calls."""

    def __init__(self, offsets, ks):
        self.nsets = len(offsets) - 1
        if len(ks) != self.nsets:
            raise ValueError("ks must have one entry per set")
        self.n = int(offsets[-1])
        self.offsets = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
        self.ks = (ctypes.c_int32 * max(self.nsets, 1))(*[int(v) for v in ks])


def cluster_batched_into(X: torch.Tensor, plan: BatchPlan, sigma: float, labels, residual, ik, beta=None,
                         o: Opts | None = None):
    """cluster_batched() writing into caller-provided device tensors."""
    lib = load()
    xp, n, d, dt = _points(X)
    if n != plan.n:
        raise ValueError("X rows differ from the plan's offsets[-1]")
    _check(lib.isoclust_cluster_batched(xp, plan.offsets, plan.nsets, d, dt, plan.ks, float(sigma), _opts_ptr(o),
                                        labels.data_ptr(), residual.data_ptr(), ik.data_ptr(),
                                        beta.data_ptr() if beta is not None else None, _stream(X.device)))


def cluster_batched(X: torch.Tensor, offsets, ks, sigma: float, o: Opts | None = None,
                    detail: bool = False) -> dict:
    """Independent point sets in one call (isoclust_cluster_batched).

    X: (N, d) float32 CUDA tensor holding the sets row-wise; offsets: N+1
    host integers (set b = rows offsets[b] .. offsets[b+1]-1); ks: the k of
    each set.  Returns labels [N], residual [N], i_k [nsets], beta [nsets]
    (and parent, phi_par, omega [N] with detail=True) on X's device."""
    lib = load()
    xp, n, d, dt = _points(X)
    off = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
    nsets = len(offsets) - 1
    if len(ks) != nsets:
        raise ValueError("ks must have one entry per set")
    kk = (ctypes.c_int32 * max(nsets, 1))(*[int(v) for v in ks])
    if nsets >= 1 and int(offsets[-1]) != n:
        raise ValueError("offsets[-1] must equal X.shape[0]")
    dev = X.device
    out = dict(
        labels=torch.empty(n, dtype=torch.int32, device=dev),
        residual=torch.empty(n, dtype=torch.uint8, device=dev),
        i_k=torch.empty(max(nsets, 1), dtype=torch.float64, device=dev),
        beta=torch.empty(max(nsets, 1), dtype=torch.float64, device=dev),
    )
    if detail:
        out.update(parent=torch.empty(n, dtype=torch.int32, device=dev),
                   phi_par=torch.empty(n, dtype=torch.float64, device=dev),
                   omega=torch.empty(n, dtype=torch.float64, device=dev))
        _check(lib.isoclust_cluster_batched_detail(
            xp, off, nsets, d, dt, kk, float(sigma), _opts_ptr(o),
            *[out[key].data_ptr() for key in ("labels", "residual", "i_k", "beta", "parent", "phi_par", "omega")],
            _stream(dev)))
    else:
        _check(lib.isoclust_cluster_batched(
            xp, off, nsets, d, dt, kk, float(sigma), _opts_ptr(o),
            *[out[key].data_ptr() for key in ("labels", "residual", "i_k", "beta")], _stream(dev)))
    return out


def scale_features(X: torch.Tensor, scale: torch.Tensor) -> torch.Tensor:
    """Z = scale (.) X per feature, formed in FP64 on the device (isoclust_scale_features)."""
    lib = load()
    xp, n, d, dt = _points(X)
    sp = _dev_ptr(scale, torch.float64)
    if scale.numel() != d:
        raise ValueError("scale must have one entry per feature")
    Z = torch.empty_like(X)
    _check(lib.isoclust_scale_features(xp, n, d, dt, sp, Z.data_ptr(), _stream(X.device)))
    return Z


def ik_backward(X: torch.Tensor, scale: torch.Tensor, sigma: float, parent, labels, k: int, phi_par, omega,
                grad_ik: float = 1.0) -> dict:
    """Derivative of i_k through a forward call's fixed tree and subpartition
    (isoclust_ik_backward): dX [n, d], dscale [d], dsigma [1] in FP64, times
    grad_ik, and the FP64 i_k of that structure."""
    lib = load()
    xp, n, d, dt = _points(X)
    dev = X.device
    out = dict(dX=torch.empty((n, d), dtype=torch.float64, device=dev),
               dscale=torch.empty(d, dtype=torch.float64, device=dev),
               dsigma=torch.empty(1, dtype=torch.float64, device=dev),
               i_k=torch.empty(1, dtype=torch.float64, device=dev))
    _check(lib.isoclust_ik_backward(
        xp, n, d, dt, _dev_ptr(scale, torch.float64), float(sigma), _dev_ptr(parent, torch.int32),
        _dev_ptr(labels, torch.int32), int(k), _dev_ptr(phi_par, torch.float64), _dev_ptr(omega, torch.float64),
        float(grad_ik), out["dX"].data_ptr(), out["dscale"].data_ptr(), out["dsigma"].data_ptr(),
        out["i_k"].data_ptr(), _stream(dev)))
    return out


class IsoperimetricNumber(torch.autograd.Function):
    """i_k of the points scale (.) X (alpha = 0) as a differentiable function
    of X, the per-feature scale and sigma, through the fixed tree and
    subpartition of the forward pass.  Returns (i_k, labels); labels are not
    differentiable.

        ik, labels = IsoperimetricNumber.apply(X, scale, sigma, k)
    """

    @staticmethod
    def forward(ctx, X, scale, sigma, k):
        s64 = scale.detach().to(torch.float64).contiguous()
        Z = scale_features(X.detach().contiguous(), s64)
        out = cluster_detail(Z, int(k), float(sigma))
        ctx.save_for_backward(X.detach(), s64, out["parent"], out["labels"], out["phi_par"], out["omega"])
        ctx.sigma = float(sigma)
        ctx.k = int(k)
        ctx.sigma_is_tensor = isinstance(sigma, torch.Tensor)
        ctx.mark_non_differentiable(out["labels"])
        return out["i_k"].reshape(()).clone(), out["labels"]

    @staticmethod
    def backward(ctx, g_ik, g_labels):
        X, s64, parent, labels, phi, omega = ctx.saved_tensors
        g = ik_backward(X.contiguous(), s64, ctx.sigma, parent, labels, ctx.k, phi, omega, float(g_ik))
        dsig = g["dsigma"].reshape(()) if ctx.sigma_is_tensor else None
        return g["dX"], g["dscale"], dsig, None


def set_sweep_variant(variant: int) -> None:
    """Force the tensor-core sweep's tile variant (0..3: bit 0 = 32-column
    candidate blocks, bit 1 = streamed row block) or let the library time and
    cache the fastest per shape class (-1, the default) -- isoclust_set_sweep_variant."""
    _check(load().isoclust_set_sweep_variant(int(variant)))


def last_sweep_variant() -> int:
    """Sweep variant of the last MST build on this thread (-1: none)."""
    return int(load().isoclust_last_sweep_variant())


def last_batched_graph_mode() -> int:
    """0 kernel by kernel, 1 captured into CUDA graphs, 2 replayed graphs
    (the last batched call; isoclust_last_batched_graph_mode)."""
    return int(load().isoclust_last_batched_graph_mode())


def set_batched_graphs(enable: bool) -> None:
    """Allow (True, the default) or forbid CUDA-graph capture and replay of
    repeated batched calls (isoclust_set_batched_graphs)."""
    _check(load().isoclust_set_batched_graphs(int(bool(enable))))


def set_omega_gram(mode) -> None:
    """eq. omega's Gram on the tensor cores: True / 1 always, False / 0 never
    (double-word sums of squared differences), -1 by row length, the
    default (isoclust_set_omega_gram)."""
    _check(load().isoclust_set_omega_gram(int(mode)))


def set_mst_prune(mode) -> None:
    """Pruned Boruvka rounds of one-set calls: True / 1 whenever supported,
    False / 0 never, -1 by size and dimension, the default
    (isoclust_set_mst_prune)."""
    _check(load().isoclust_set_mst_prune(int(mode)))


def set_test_stalled_wait(on: bool) -> None:
    """Test hook of the timeout path (isoclust_set_test_stalled_wait): while
    on, every tensor-core sweep's epilogue waits for a barrier nothing
    arrives at, so calls run into their spin limit."""
    _check(load().isoclust_set_test_stalled_wait(int(bool(on))))


def kernel_launches() -> int:
    """Cumulative count of kernels launched by libisoclust in this process."""
    return int(load().isoclust_kernel_launches())


def last_profile() -> dict:
    """Per-stage device times (ms) and counters of the last call on this thread."""
    lib = load()
    t = (ctypes.c_double * 6)()
    c = (ctypes.c_int64 * 4)()
    lib.isoclust_last_profile(t, c)
    tl = (ctypes.c_int64 * 3)()
    lib.isoclust_last_omega_tiles(tl)
    mt = (ctypes.c_int64 * 2)()
    lib.isoclust_last_mst_tiles(mt)
    gb, gf = ctypes.c_int64(0), ctypes.c_int64(0)
    gms = float(lib.isoclust_last_omega_gram_ms(ctypes.byref(gb), ctypes.byref(gf)))
    return dict(omega_tiles=tl[0], omega_tiles_dw=tl[1], omega_symmetric=tl[2],
                omega_kernel_ms=float(lib.isoclust_last_omega_kernel_ms()),
                omega_gram_ms=gms, omega_gram_blocks=int(gb.value), omega_gram_direct_pairs=int(gf.value),
                mst_tiles_swept=mt[0], mst_tiles_full=mt[1], validate_ms=t[0], weights_ms=t[1], mst_ms=t[2], orient_ms=t[3], search_ms=t[4], labels_ms=t[5],
                boruvka_rounds=c[0], rescanned_rows=c[1], alg1_passes=c[2], tree_depth=c[3])


@dataclass
class HostResult:
    labels: object
    residual: object
    i_k: float


def cluster_host(X_host, k: int, sigma: float, o: Opts | None = None, device="cuda") -> HostResult:
    """Host-buffer entry: copies X (pinned host) to the device, runs cluster(),
    copies labels / residual / i_k back."""
    Xd = X_host.to(device, non_blocking=True)
    labels, residual, ik = cluster(Xd, k, sigma, o)
    return HostResult(labels.cpu(), residual.cpu(), float(ik.cpu()[0]))

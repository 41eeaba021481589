"""Seeded synthetic point sets (numpy only; no clustering arithmetic here).

The paper measures on UCI datasets (Table 1) that are not available offline;
these generators stand in for them with the shapes, value distributions and
cluster structure of the workloads the library is benchmarked on.  Every
generator is a pure function of its seed.  Rows are shuffled so that the
input carries no ordering by cluster.

  blobs_isotropic   n = 2,000, d = 8: 5 blobs, std 1, centres U[-10,10]^8, FP64
  blobs_anisotropic n = 100,000, d = 64: 20 blobs with random rotations and
                    eigenvalues log-uniform in [0.1, 2], Zipf(1.1) sizes, and
                    2% uniform outliers in the bounding box, FP32
  sparse_groups     n = 50,000, d = 4,096: non-negative log-normal values at
                    1% density, 10 groups sharing support pools, rows
                    L2-normalised, FP32
  table1_shape      blobs at a (n, k, d) shape of the paper's Table 1
  moons_embedded    n = 20,000, d = 128: 3 interleaved half-circle arcs (radius
                    1) in 2-D, embedded by the first 2 columns of a random
                    orthogonal matrix, plus N(0, 0.1^2) noise in all 128
                    dimensions, FP32 (the differentiation workload)
  batched_sets      4,096 independent sets, sizes log-uniform in [64, 8192],
                    d = 32, each 2-8 isotropic blobs (std 1, centres
                    U[-10,10]^32, equal split), k = its blob count, FP32
"""
from __future__ import annotations

import numpy as np


def _shuffle(rng, X, y):
    perm = rng.permutation(X.shape[0])
    return np.ascontiguousarray(X[perm]), y[perm]


def blobs_isotropic(seed: int = 0, n_per: int = 400, k: int = 5, d: int = 8,
                    lo: float = -10.0, hi: float = 10.0, std: float = 1.0,
                    dtype=np.float64):
    """k isotropic Gaussian blobs of equal size; returns (X, true_labels)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(lo, hi, size=(k, d))
    X = np.concatenate([c + std * rng.standard_normal((n_per, d)) for c in centres])
    y = np.repeat(np.arange(k), n_per)
    X, y = _shuffle(rng, X, y)
    return X.astype(dtype), y.astype(np.int32)


def _largest_remainder(weights, total):
    w = np.asarray(weights, dtype=np.float64)
    raw = w / w.sum() * total
    base = np.floor(raw).astype(np.int64)
    rem = int(total - base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return base


def blobs_anisotropic(seed: int = 0, n: int = 100_000, k: int = 20, d: int = 64,
                      outlier_frac: float = 0.02, zipf: float = 1.1,
                      lam_lo: float = 0.1, lam_hi: float = 2.0, dtype=np.float32):
    """k rotated anisotropic blobs, Zipf sizes, plus uniform outliers.

    Outliers get true label -1."""
    rng = np.random.default_rng(seed)
    n_out = int(round(outlier_frac * n))
    n_in = n - n_out
    sizes = _largest_remainder(np.arange(1, k + 1, dtype=np.float64) ** (-zipf), n_in)
    centres = rng.uniform(-10.0, 10.0, size=(k, d))
    parts = []
    for b in range(k):
        G = rng.standard_normal((d, d))
        Q, R = np.linalg.qr(G)
        Q = Q * np.sign(np.diag(R))[None, :]          # sign-fixed orthogonal factor
        lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), size=d))
        Z = rng.standard_normal((int(sizes[b]), d))
        parts.append(centres[b] + (Z * np.sqrt(lam)[None, :]) @ Q.T)
    Xin = np.concatenate(parts)
    lo, hi = Xin.min(axis=0), Xin.max(axis=0)
    Xout = rng.uniform(lo, hi, size=(n_out, d))
    X = np.concatenate([Xin, Xout])
    y = np.concatenate([np.repeat(np.arange(k), sizes), np.full(n_out, -1)])
    X, y = _shuffle(rng, X, y)
    return X.astype(dtype), y.astype(np.int32)


def sparse_groups(seed: int = 0, n_per: int = 5_000, k: int = 10, d: int = 4096,
                  pool_frac: float = 0.05, density: float = 0.01, in_pool: float = 0.8,
                  dtype=np.float32):
    """Sparse-like non-negative rows (stored dense), L2-normalised."""
    rng = np.random.default_rng(seed)
    pool = int(round(pool_frac * d))
    nnz = int(round(density * d))
    X = np.zeros((n_per * k, d), dtype=np.float64)
    y = np.repeat(np.arange(k), n_per)
    for g in range(k):
        support = rng.choice(d, size=pool, replace=False)
        for r in range(n_per):
            row = g * n_per + r
            n_in = rng.binomial(nnz, in_pool)
            cols_in = rng.choice(support, size=n_in, replace=False)
            cols_out = rng.choice(d, size=nnz - n_in, replace=False)
            cols = np.unique(np.concatenate([cols_in, cols_out]))
            X[row, cols] = np.exp(rng.standard_normal(cols.size))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X, y = _shuffle(rng, X, y)
    return X.astype(dtype), y.astype(np.int32)


def table1_shape(seed: int, n: int, k: int, d: int, dtype=np.float64):
    """Isotropic blobs at one of the paper's Table 1 shapes (n, k, d)."""
    rng = np.random.default_rng(seed)
    sizes = _largest_remainder(np.ones(k), n)
    centres = rng.uniform(-10.0, 10.0, size=(k, d))
    X = np.concatenate([c + rng.standard_normal((int(s), d)) for c, s in zip(centres, sizes)])
    y = np.repeat(np.arange(k), sizes)
    X, y = _shuffle(rng, X, y)
    return X.astype(dtype), y.astype(np.int32)


def uniform_points(seed: int, n: int, d: int, lo: float = -1.0, hi: float = 1.0,
                   dtype=np.float32):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, d)).astype(dtype)


def integer_grid_points(seed: int, n: int, d: int, span: int = 4, dtype=np.float32):
    """Small-integer coordinates: many exactly tied distances (tie-break tests)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-span, span + 1, size=(n, d)).astype(dtype)


def random_rooted_tree(seed: int, n: int, shape: str = "random", max_children: int = 0):
    """(parent, phi_par, omega, p) of a random weighted tree, parent[root] = -1.

    shape: random (uniform attachment), path, star, caterpillar, deep (long
    chains with short side twigs), binary."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    parent = np.full(n, -1, dtype=np.int32)
    for idx in range(1, n):
        v = perm[idx]
        if shape == "path":
            u = perm[idx - 1]
        elif shape == "star":
            u = perm[0]
        elif shape == "caterpillar":
            u = perm[max(0, idx - 1 - (idx % 2))]
        elif shape == "binary":
            u = perm[(idx - 1) // 2]
        elif shape == "deep":
            u = perm[idx - 1] if rng.random() < 0.85 else perm[max(0, idx - 1 - int(rng.integers(1, 8)))]
        else:
            u = perm[rng.integers(0, idx)]
        parent[v] = u
    phi = np.where(parent >= 0, np.exp(-rng.uniform(0.1, 6.0, n)), 0.0)
    omega = rng.uniform(0.2, 5.0, n)
    p = rng.uniform(0.0, 0.3, n)
    return parent, phi, omega, p


def batched_sets(seed: int = 0, nsets: int = 4096, n_lo: int = 64, n_hi: int = 8192, d: int = 32,
                 blobs_lo: int = 2, blobs_hi: int = 8, std: float = 1.0, dtype=np.float32, sizes=None):
    """Independent point sets concatenated row-wise.

    Returns (X, offsets, ks): set b is X[offsets[b]:offsets[b+1]] with
    k = ks[b] equal to its number of blobs (at most its size).  Sizes are
    floor(exp(U[ln n_lo, ln n_hi])) unless given; blob sizes split each set
    as equally as possible."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=nsets))).astype(np.int64)
        sizes = np.clip(sizes, n_lo, n_hi)
    else:
        sizes = np.asarray(sizes, dtype=np.int64)
        nsets = sizes.size
    ks = rng.integers(blobs_lo, blobs_hi + 1, size=nsets).astype(np.int32)
    ks = np.minimum(ks, sizes).astype(np.int32)
    parts = []
    for b in range(nsets):
        kb = int(ks[b])
        centres = rng.uniform(-10.0, 10.0, size=(kb, d))
        split = _largest_remainder(np.ones(kb), int(sizes[b]))
        Xb = np.concatenate([c + std * rng.standard_normal((int(m), d)) for c, m in zip(centres, split)])
        parts.append(Xb[rng.permutation(Xb.shape[0])])
    offsets = np.zeros(nsets + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.ascontiguousarray(np.concatenate(parts).astype(dtype)), offsets, ks


def moons_embedded(seed: int = 0, n: int = 20_000, d: int = 128, noise: float = 0.1, dtype=np.float32):
    """Three half-circle arcs of radius 1 interleaved along x (up, down, up:
    centres (0, 0), (1, 0.5) flipped, (2, 0)), equal sizes, embedded in d
    dimensions by the first two columns of a sign-fixed random orthogonal
    matrix, plus isotropic Gaussian noise.  Returns (X, true_labels)."""
    rng = np.random.default_rng(seed)
    sizes = _largest_remainder(np.ones(3), n)
    parts, ys = [], []
    for m, cnt in enumerate(sizes):
        t = rng.uniform(0.0, np.pi, size=int(cnt))
        if m == 1:
            P = np.stack([1.0 - np.cos(t), 0.5 - np.sin(t)], axis=1)
        else:
            P = np.stack([2.0 * (m // 2) + np.cos(t), np.sin(t)], axis=1)
        parts.append(P)
        ys.append(np.full(int(cnt), m))
    P = np.concatenate(parts)
    G = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    X = P @ Q[:, :2].T + noise * rng.standard_normal((P.shape[0], d))
    X, y = _shuffle(rng, X, np.concatenate(ys))
    return X.astype(dtype), y.astype(np.int32)


CONFIGS = {
    "blobs_n2000_d8": dict(gen="blobs_isotropic", n=2000, d=8, k=5, sigma=1.0, dtype="f64"),
    "blobs_n100k_d64": dict(gen="blobs_anisotropic", n=100_000, d=64, k=20, sigma=1.0, dtype="f32"),
    "sparse_n50k_d4096": dict(gen="sparse_groups", n=50_000, d=4096, k=10, sigma=1.0, dtype="f32"),
    "batched_4096_d32": dict(gen="batched_sets", nsets=4096, d=32, sigma=1.0, dtype="f32"),
    "moons_n20k_d128": dict(gen="moons_embedded", n=20_000, d=128, k=3, sigma=1.0, dtype="f32"),
}


def make(config: str, seed: int = 0):
    """(X, k, sigma) of a named single-set workload."""
    c = CONFIGS[config]
    if c["gen"] == "blobs_isotropic":
        X, _ = blobs_isotropic(seed)
    elif c["gen"] == "blobs_anisotropic":
        X, _ = blobs_anisotropic(seed)
    elif c["gen"] == "moons_embedded":
        X, _ = moons_embedded(seed)
    else:
        X, _ = sparse_groups(seed)
    return X, c["k"], c["sigma"]


def make_batched(config: str = "batched_4096_d32", seed: int = 0, nsets: int | None = None,
                 n_hi: int | None = None):
    """(X, offsets, ks, sigma) of a batched workload, optionally with fewer
    or smaller sets (the same recipe)."""
    c = CONFIGS[config]
    kw = dict(nsets=nsets or c["nsets"], d=c["d"])
    if n_hi is not None:
        kw["n_hi"] = n_hi
    X, offsets, ks = batched_sets(seed, **kw)
    return X, offsets, ks, c["sigma"]

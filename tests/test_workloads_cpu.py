"""The synthetic workload recipes (stand-ins for the paper's datasets) match
their stated construction; reduced sizes of the same generators."""
import numpy as np

from paper_1702_04739_gb300 import workloads as W


def test_anisotropic_blobs_recipe():
    n, k, d = 5000, 20, 64
    X, y = W.blobs_anisotropic(seed=3, n=n, k=k, d=d)
    assert X.shape == (n, d) and X.dtype == np.float32 and X.flags["C_CONTIGUOUS"]
    n_out = int(round(0.02 * n))
    assert (y == -1).sum() == n_out
    sizes = np.bincount(y[y >= 0], minlength=k)
    w = np.arange(1, k + 1, dtype=np.float64) ** -1.1
    ideal = w / w.sum() * (n - n_out)
    assert sizes.sum() == n - n_out and np.abs(sizes - ideal).max() < 1.0      # largest remainder
    assert (np.diff(sizes) <= 0).all()                                           # Zipf order
    inl = X[y >= 0]
    lo, hi = inl.min(axis=0), inl.max(axis=0)
    out = X[y == -1]
    assert (out >= lo - 1e-5).all() and (out <= hi + 1e-5).all()                # inside the bounding box
    assert not (np.diff(y) == 0).all()                                           # rows shuffled
    a, b = W.blobs_anisotropic(seed=3, n=n, k=k, d=d)
    assert (a == X).all() and (b == y).all()                                     # seeded


def test_anisotropic_blob_covariance():
    # one blob, many points: its covariance has the drawn spectrum in [0.1, 2]
    X, y = W.blobs_anisotropic(seed=5, n=40000, k=1, d=8, outlier_frac=0.0)
    ev = np.linalg.eigvalsh(np.cov(X.astype(np.float64).T))
    assert ev.min() > 0.08 and ev.max() < 2.3


def test_sparse_groups_recipe():
    n_per, k, d = 40, 10, 4096
    X, y = W.sparse_groups(seed=7, n_per=n_per, k=k, d=d)
    assert X.shape == (n_per * k, d) and X.dtype == np.float32
    assert (X >= 0).all()
    assert np.allclose(np.linalg.norm(X.astype(np.float64), axis=1), 1.0, rtol=1e-6)
    nnz = (X > 0).sum(axis=1)
    assert nnz.max() <= 41 and np.median(nnz) >= 40            # 1 % density; duplicates merge
    assert np.bincount(y, minlength=k).tolist() == [n_per] * k
    # rows of a group share most of their support (80 % from a 205-feature pool)
    for g in range(3):
        cols = np.flatnonzero((X[y == g] > 0).any(axis=0))
        counts = (X[y == g] > 0).sum(axis=0)[cols]
        assert (counts >= 3).sum() <= 205

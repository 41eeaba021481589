#!/usr/bin/env python3
"""Writes the full-size expected results of the five benchmark workloads.

Every stored value comes from the FP64 oracle (``oracle/``) run on the seeded
synthetic inputs of ``paper_1702_04739_gb300.workloads``; nothing here touches
the CUDA library.  The GPU parity tests compare the library's outputs with
these files element by element.

  python tests/golden/make_fullsize.py [workload ...] [--threads T]

One file per workload, ``tests/golden/fullsize/<workload>.npz``:
  x_sha256           SHA-256 of the input bytes (X as stored; for the batched
                     workload X, offsets and ks), so a test can tell that its
                     input is the one the oracle saw
  edge_u, edge_v,    the n-1 minimum-spanning-tree edges in key order
  edge_d2            (Section 2.2 step 2, Algorithm 3)
  parent             the tree rooted at vertex 0 (-1 at the root)
  omega              eq. omega of every point
  labels, i_k, beta  Algorithms 1-2 (readings A4-A8)
  stats              phi*, phi_*, omega*, omega_*, p*, p_*, alpha_0, beta_0
  oracle_s, threads  wall time of the oracle call and its thread count

The batched workload (4,096 independent sets) stores, per set, SHA-256
digests of its edges (u, v, d2 in set-local indices), parent and labels,
its i_k and beta, and the full omega of 16 sets spread over the size range
(the digests make every set's tree and labels comparable bit for bit; all
6.7 M omega values would not be compact).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1702_04739_gb300 import workloads  # noqa: E402

OUT = os.path.join(HERE, "fullsize")
SINGLE = ["blobs_n2000_d8", "moons_n20k_d128", "blobs_n100k_d64", "sparse_n50k_d4096"]
BATCHED = "batched_4096_d32"
OMEGA_SETS = 16


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def set_digests(r) -> tuple[str, str, str]:
    """Digests of one set's tree and labels, in the dtypes the tests compare."""
    e = sha(r["edge_u"].astype(np.int32), r["edge_v"].astype(np.int32), r["edge_d2"].astype(np.float64))
    return e, sha(r["parent"].astype(np.int32)), sha(r["labels"].astype(np.int32))


def omega_sample_sets(sizes) -> np.ndarray:
    """16 sets spread over the size range: the smallest, the largest and 14
    sets at evenly spaced size ranks."""
    order = np.argsort(sizes, kind="stable")
    pick = order[np.linspace(0, sizes.size - 1, OMEGA_SETS).round().astype(np.int64)]
    return np.unique(pick)


def make_single(name: str, threads: int) -> None:
    X, k, sigma = workloads.make(name, seed=0)
    t0 = time.perf_counter()
    r = oracle.cluster(X, k, sigma)
    dt = time.perf_counter() - t0
    np.savez_compressed(
        os.path.join(OUT, name + ".npz"),
        workload=name, seed=0, n=X.shape[0], d=X.shape[1], k=k, sigma=sigma, x_sha256=sha(X),
        edge_u=r["edge_u"], edge_v=r["edge_v"], edge_d2=r["edge_d2"], parent=r["parent"],
        omega=r["omega"], labels=r["labels"].astype(np.int8 if k < 128 else np.int32),
        i_k=r["i_k"], beta=r["beta"], stats=r["stats"], oracle_s=dt, threads=threads,
        machine=platform.machine())
    print(f"{name}: n={X.shape[0]} d={X.shape[1]} i_k={r['i_k']!r} oracle {dt:.1f} s on {threads} threads",
          flush=True)


def make_batched(threads: int) -> None:
    X, offs, ks, sigma = workloads.make_batched(BATCHED, seed=0)
    nsets = ks.size
    sizes = np.diff(offs)
    om_sets = omega_sample_sets(sizes)
    dig = np.zeros((nsets, 3), dtype="S64")
    ik = np.zeros(nsets)
    beta = np.zeros(nsets)
    om_parts = []
    t0 = time.perf_counter()
    for b in range(nsets):
        r = oracle.cluster(np.ascontiguousarray(X[offs[b]:offs[b + 1]]), int(ks[b]), sigma)
        dig[b] = [s.encode() for s in set_digests(r)]
        ik[b] = r["i_k"]
        beta[b] = r["beta"]
        if b in om_sets:
            om_parts.append(r["omega"])
    dt = time.perf_counter() - t0
    np.savez_compressed(
        os.path.join(OUT, BATCHED + ".npz"),
        workload=BATCHED, seed=0, nsets=nsets, sigma=sigma, x_sha256=sha(X, offs, ks),
        digests=dig, i_k=ik, beta=beta, omega_sets=om_sets, omega=np.concatenate(om_parts),
        oracle_s=dt, threads=threads, machine=platform.machine())
    print(f"{BATCHED}: {nsets} sets, {X.shape[0]} points, oracle {dt:.1f} s on {threads} threads", flush=True)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=SINGLE + [BATCHED])
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    os.makedirs(OUT, exist_ok=True)
    oracle.build()
    threads = a.threads or len(os.sched_getaffinity(0))
    oracle.set_threads(threads)
    for w in a.workloads:
        if w == BATCHED:
            make_batched(threads)
        elif w in SINGLE:
            make_single(w, threads)
        else:
            raise SystemExit(f"unknown workload {w}")
    return 0


if __name__ == "__main__":
    sys.exit(main())

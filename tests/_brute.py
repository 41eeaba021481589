"""Brute-force MISO_k of a weighted tree, straight from the definitions.

Used to pin the oracle's Algorithms 1 and 2 independently of them:
  * k-subpartition (Section 2.1): k pairwise disjoint, non-empty subsets;
    they need not cover X and need not be connected;
  * boundary delta(A): the tree edges with exactly one end in A;
  * cost (eq. cost): max_i (phi(delta A_i) + p(A_i)) / omega(A_i);
  * MISO_k (eq. MISO): the minimum cost over all k-subpartitions.
Every assignment V -> {0 (no set), 1..k} is enumerated, (k+1)^n of them, so
this is for n <= 12 or so.
"""
from __future__ import annotations

import itertools

import numpy as np


def miso_bruteforce(parent, phi_par, omega, p, k: int, chunk: int = 1 << 18) -> float:
    parent = np.asarray(parent, dtype=np.int64)
    n = parent.size
    phi_par = np.asarray(phi_par, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    p = np.zeros(n) if p is None else np.asarray(p, dtype=np.float64)
    child = np.array([v for v in range(n) if parent[v] >= 0], dtype=np.int64)
    par = parent[child]
    ephi = phi_par[child]
    best = np.inf
    total = (k + 1) ** n
    digits = (k + 1) ** np.arange(n, dtype=np.int64)
    for start in range(0, total, chunk):
        codes = np.arange(start, min(total, start + chunk), dtype=np.int64)
        A = (codes[:, None] // digits[None, :]) % (k + 1)          # (M, n) set id per vertex
        cost = np.zeros(codes.size)
        valid = np.ones(codes.size, dtype=bool)
        for s in range(1, k + 1):
            m = A == s
            w = m @ omega
            nonempty = m.any(axis=1)
            valid &= nonempty
            bnd = (m[:, child] ^ m[:, par]) @ ephi
            ps = m @ p
            with np.errstate(divide="ignore", invalid="ignore"):
                r = np.where(nonempty, (bnd + ps) / np.where(w > 0, w, 1.0), np.inf)
            cost = np.maximum(cost, r)
        if valid.any():
            best = min(best, float(cost[valid].min()))
    return best


def random_tree(rng, n: int, shape: str = "random"):
    """parent[] of a tree on n vertices rooted at a random vertex."""
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
        else:
            u = perm[rng.integers(0, idx)]
        parent[v] = u
    return parent


def reroot(parent, new_root: int):
    """The same undirected tree rooted at new_root."""
    parent = np.asarray(parent, dtype=np.int64)
    n = parent.size
    adj = [[] for _ in range(n)]
    for v in range(n):
        if parent[v] >= 0:
            adj[v].append(int(parent[v]))
            adj[int(parent[v])].append(v)
    out = np.full(n, -1, dtype=np.int32)
    seen = np.zeros(n, dtype=bool)
    stack = [new_root]
    seen[new_root] = True
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if not seen[w]:
                seen[w] = True
                out[w] = u
                stack.append(w)
    return out


def edge_flow_map(parent, phi_par):
    """{frozenset(u, v): phi} for re-rooting tests."""
    return {frozenset((int(v), int(parent[v]))): float(phi_par[v])
            for v in range(len(parent)) if parent[v] >= 0}


def phi_for_parent(parent, emap):
    return np.array([emap[frozenset((v, int(parent[v])))] if parent[v] >= 0 else 0.0
                     for v in range(len(parent))])


__all__ = ["miso_bruteforce", "random_tree", "reroot", "edge_flow_map", "phi_for_parent",
           "itertools"]

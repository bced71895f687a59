"""Brute-force BFS levels for tiny graphs — TEST INFRASTRUCTURE ONLY.

Level of v from root r is the smallest k with ((A + I)^k)[r, v] != 0 over the
boolean semiring, where A is the symmetric adjacency matrix without
self-loops; -1 if no k <= n reaches v. This is the definition of hop distance
written as matrix powers, independent of any queue-based traversal.
"""
from __future__ import annotations

import numpy as np


def adjacency(n: int, src, dst) -> np.ndarray:
    """Symmetric boolean adjacency matrix of the undirected pairs, self-loops dropped."""
    a = np.zeros((n, n), dtype=bool)
    for u, v in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if u != v:
            a[u, v] = True
            a[v, u] = True
    return a


def brute_levels(n: int, src, dst) -> np.ndarray:
    """Levels from every root at once: L[r, v] (int32), -1 if unreachable."""
    a = adjacency(n, src, dst)
    step = (a | np.eye(n, dtype=bool)).astype(np.int64)
    reach = np.eye(n, dtype=np.int64)  # (A+I)^0
    level = np.full((n, n), -1, dtype=np.int32)
    level[reach > 0] = 0
    for k in range(1, n + 1):
        reach = ((reach @ step) > 0).astype(np.int64)  # (A+I)^k, boolean
        newly = (reach > 0) & (level < 0)
        if not newly.any():
            break
        level[newly] = k
    return level


def brute_canonical_parent(n: int, src, dst, level_from_root: np.ndarray, root: int) -> np.ndarray:
    """min{u : u ~ v, level[u] = level[v] - 1} by a scan of the adjacency matrix."""
    a = adjacency(n, src, dst)
    par = np.full(n, -1, dtype=np.int32)
    for v in range(n):
        if level_from_root[v] <= 0:
            continue
        cands = [u for u in range(n) if a[u, v] and level_from_root[u] == level_from_root[v] - 1]
        par[v] = min(cands)
    if level_from_root[root] == 0:
        par[root] = root
    return par

"""Host-side helpers for the merge list the library returns.

A clustering of n objects is returned as n - 1 steps (i, j, height): the
clusters in slots i < j merged, slot i keeps the result (Section 4 steps 2
and 4).  These helpers turn that list into the forms other tools use:

* ``to_linkage_matrix`` -- the (n - 1) x 4 matrix of SciPy's hierarchy
  module: step t merges cluster ids a and b (an object's id is its index, the
  cluster made at step t gets id n + t), at the step's height, into a cluster
  of the given size;
* ``cut`` -- the partition into k clusters (the tree level after n - k
  merges, Section 4 step 4's "current tree level");
* ``cut_height`` -- the partition of the clusters formed at heights <= h.

Pure numpy, no device work.
"""
from __future__ import annotations

import numpy as np


def _check(merges: np.ndarray, n: int) -> np.ndarray:
    m = np.asarray(merges)
    if hasattr(merges, "cpu"):
        m = merges.cpu().numpy()
    m = m.reshape(-1, 2).astype(np.int64)
    if n < 1 or m.shape[0] != max(n - 1, 0):
        raise ValueError(f"expected {max(n - 1, 0)} merges for n = {n}, got {m.shape[0]}")
    return m


def to_linkage_matrix(merges, heights, n: int) -> np.ndarray:
    """SciPy-style linkage matrix Z (float64, shape (n - 1, 4)): row t is
    (id_a, id_b, height, size) with id_a < id_b."""
    m = _check(merges, n)
    h = np.asarray(heights.cpu().numpy() if hasattr(heights, "cpu") else heights, dtype=np.float64)
    slot_id = np.arange(n, dtype=np.int64)      # cluster id currently held by each slot
    size = np.ones(n, dtype=np.int64)
    Z = np.zeros((max(n - 1, 0), 4), dtype=np.float64)
    for t, (i, j) in enumerate(m):
        a, b = slot_id[i], slot_id[j]
        Z[t] = (min(a, b), max(a, b), h[t], size[i] + size[j])
        size[i] += size[j]
        slot_id[i] = n + t
    return Z


def _labels_after(m: np.ndarray, n: int, steps: int) -> np.ndarray:
    parent = np.arange(n, dtype=np.int64)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for i, j in m[:steps]:
        parent[find(j)] = find(i)
    roots = np.array([find(x) for x in range(n)])
    # labels 0..k-1 in order of each cluster's smallest object
    _, labels = np.unique(roots, return_inverse=True)
    first = {}
    out = np.empty(n, dtype=np.int64)
    for x in range(n):
        r = labels[x]
        if r not in first:
            first[r] = len(first)
        out[x] = first[r]
    return out


def cut(merges, n: int, k: int) -> np.ndarray:
    """Labels (0..k-1, numbered by each cluster's smallest object) of the k
    clusters left after the first n - k merges."""
    m = _check(merges, n)
    if not 1 <= k <= n:
        raise ValueError(f"k must be in [1, {n}]")
    return _labels_after(m, n, n - k)


def cut_height(merges, heights, n: int, h: float) -> np.ndarray:
    """Labels of the clusters formed by the merges of height <= h, taken in
    order until the first merge above h (for linkages whose heights never
    decrease this is every merge <= h)."""
    m = _check(merges, n)
    hh = np.asarray(heights.cpu().numpy() if hasattr(heights, "cpu") else heights, dtype=np.float64)
    steps = 0
    while steps < len(hh) and hh[steps] <= h:
        steps += 1
    return _labels_after(m, n, steps)

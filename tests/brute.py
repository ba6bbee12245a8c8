"""Independent references used to pin the oracle (tests only).

None of these use the Lance-Williams recurrence: they compute cluster
distances from the original members (Section 2.1 defines single linkage by the
closest members and complete linkage by the furthest), the minimum spanning
tree that single linkage follows (Section 2.1: Prim's algorithm), and Ward's
centroid form.
"""
from __future__ import annotations

import numpy as np


def unpack(D: np.ndarray, n: int) -> np.ndarray:
    """Full symmetric float64 matrix from the packed upper triangle."""
    M = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    M[iu] = D.astype(np.float64)
    M[(iu[1], iu[0])] = D.astype(np.float64)
    return M


def prim_mst_weights(M: np.ndarray) -> np.ndarray:
    """Edge weights of a minimum spanning tree (Prim), float64."""
    n = M.shape[0]
    if n < 2:
        return np.zeros(0)
    in_tree = np.zeros(n, dtype=bool)
    in_tree[0] = True
    best = M[0].copy()
    best[0] = np.inf
    out = []
    for _ in range(n - 1):
        cand = np.where(in_tree, np.inf, best)
        v = int(np.argmin(cand))
        out.append(cand[v])
        in_tree[v] = True
        best = np.minimum(best, M[v])
    return np.array(out)


def components(n: int, edges) -> list:
    """Connected components (as frozensets) of the graph with the given edges."""
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    groups = {}
    for v in range(n):
        groups.setdefault(find(v), set()).add(v)
    return sorted(frozenset(g) for g in groups.values())


def partitions_by_height(n: int, merges: np.ndarray, heights: np.ndarray) -> dict:
    """Partition after all merges with height <= h, for every distinct height h."""
    members = {s: {s} for s in range(n)}
    out = {}
    for t in range(len(heights)):
        i, j = int(merges[t, 0]), int(merges[t, 1])
        members[i] |= members.pop(j)
        if t + 1 == len(heights) or heights[t + 1] != heights[t]:
            out[float(heights[t])] = sorted(frozenset(g) for g in members.values())
    return out


def member_linkage(M: np.ndarray, linkage: str, points: np.ndarray | None = None):
    """Agglomerative clustering recomputing every cluster distance from members.

    linkage: 'single' (min over member pairs), 'complete' (max), 'average'
    (mean), 'ward' (2 nA nB / (nA+nB) ||cA - cB||^2 from ``points``),
    'centroid' (||cA - cB||^2 from ``points``).
    Minimum by (value, i, j) lexicographically over live slots i < j; slot i
    keeps the merged cluster.  Returns (merges (n-1, 2), heights float64,
    gaps float64) where gaps[t] is the distance between the smallest and the
    second-smallest candidate value at step t (inf when there is one).
    """
    n = M.shape[0]
    members = {s: [s] for s in range(n)}
    merges, heights, gaps = [], [], []
    for _ in range(n - 1):
        slots = sorted(members)
        best = None
        second = np.inf
        for a_idx, r in enumerate(slots):
            for c in slots[a_idx + 1:]:
                A, B = members[r], members[c]
                if linkage == "single":
                    v = M[np.ix_(A, B)].min()
                elif linkage == "complete":
                    v = M[np.ix_(A, B)].max()
                elif linkage == "average":
                    v = M[np.ix_(A, B)].mean()
                elif linkage == "ward":
                    ca = points[A].mean(axis=0)
                    cb = points[B].mean(axis=0)
                    v = 2.0 * len(A) * len(B) / (len(A) + len(B)) * float(((ca - cb) ** 2).sum())
                elif linkage == "centroid":
                    ca = points[A].mean(axis=0)
                    cb = points[B].mean(axis=0)
                    v = float(((ca - cb) ** 2).sum())
                else:
                    raise ValueError(linkage)
                if best is None or v < best[0]:
                    if best is not None:
                        second = min(second, best[0])
                    best = (v, r, c)
                else:
                    second = min(second, v)
        v, r, c = best
        merges.append((r, c))
        heights.append(v)
        gaps.append(second - v)
        members[r] = members[r] + members.pop(c)
    return np.array(merges, dtype=np.int32).reshape(-1, 2), np.array(heights), np.array(gaps)


def cophenetic(n: int, merges: np.ndarray, heights: np.ndarray) -> np.ndarray:
    """Cophenetic matrix: the height at which two objects first share a cluster."""
    C = np.zeros((n, n))
    members = {s: [s] for s in range(n)}
    for t in range(len(heights)):
        i, j = int(merges[t, 0]), int(merges[t, 1])
        A, B = members[i], members.pop(j)
        C[np.ix_(A, B)] = heights[t]
        C[np.ix_(B, A)] = heights[t]
        members[i] = A + B
    return C


def dyadic_matrix(n: int, seed: int, bits: int = 22) -> np.ndarray:
    """Packed FP32 matrix of multiples of 1/1024 below 2^12 (exact halves and sums)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << bits, size=n * (n - 1) // 2)
    return (k.astype(np.float64) / 1024.0).astype(np.float32)


def dyadic_from_points(points: np.ndarray) -> np.ndarray:
    """Euclidean distances of ``points`` rounded to multiples of 1/1024, FP32, packed."""
    n = points.shape[0]
    iu = np.triu_indices(n, 1)
    d = np.sqrt(((points[iu[0]] - points[iu[1]]) ** 2).sum(axis=1))
    return (np.round(d * 1024.0) / 1024.0).astype(np.float32)

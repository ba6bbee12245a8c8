"""Seeded generators of dissimilarity matrices for Lance-Williams clustering.

The paper clusters protein conformations from an n x n distance matrix
(Abstract; Section 1; Section 3.2) with mean n about 1968 (Section 6).  That data is
not available, so every workload here is synthetic and seeded:

* Gaussian-mixture point clouds (isotropic components) with Euclidean distances;
* conformer-like chains: 64 seed chains of 128 beads (3D random walks with
  step 3.8), each conformer a seed chain plus N(0, 0.5^2) noise per coordinate,
  with d = ||delta coords|| / sqrt(128) (an RMSD without superposition).

Storage follows the paper's upper-triangle layout (Section 5.1, Section 5.2): the
packed row-major upper triangle of n(n-1)/2 FP32 cells, cell (r, c) with r < c
at r*n - r*(r+1)/2 + (c - r - 1).

Distances are computed in FP64 as sqrt(sum over coordinates, in coordinate
order, of (x - y)^2), optionally divided by a scale, optionally rounded
half-to-even to a multiple of 1/1024, and rounded once to FP32.  The numpy
path and the torch path (used for the large workloads, on any torch device)
perform the same elementwise IEEE operations in the same order, so they give
the same bits.

Random draws happen only here, with ``numpy.random.default_rng(seed)``; the
order of draws is part of each generator's definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Linkage codes shared with the C interfaces (Table 1 rows used here).
SINGLE, COMPLETE, AVERAGE, WARD, WEIGHTED, CENTROID = 0, 1, 2, 3, 4, 5
LINKAGE_NAMES = {SINGLE: "single", COMPLETE: "complete", AVERAGE: "average", WARD: "ward",
                 WEIGHTED: "weighted", CENTROID: "centroid"}


def packed_size(n: int) -> int:
    """Number of cells of the strict upper triangle, (n^2 - n) / 2 (Section 5.1)."""
    return n * (n - 1) // 2


# ----------------------------------------------------------------------------
# points
# ----------------------------------------------------------------------------

def gmm_points(rng: np.random.Generator, n: int, dim: int, k: int,
               center_range: float = 10.0, sigma=1.0) -> np.ndarray:
    """n points from a k-component isotropic Gaussian mixture in R^dim.

    Draw order: centers U[-center_range, center_range]^(k x dim); then, if
    ``sigma`` is a (lo, hi) pair, one sigma per component from U[lo, hi];
    then the component of each point, uniform over k; then the N(0, 1) noise
    (n x dim), scaled by the point's component sigma.
    """
    centers = rng.uniform(-center_range, center_range, size=(k, dim))
    if isinstance(sigma, tuple):
        sig = rng.uniform(sigma[0], sigma[1], size=k)
    else:
        sig = np.full(k, float(sigma))
    comp = rng.integers(0, k, size=n)
    noise = rng.standard_normal(size=(n, dim))
    return centers[comp] + noise * sig[comp][:, None]


def conformer_points(rng: np.random.Generator, n: int, n_seeds: int = 64,
                     beads: int = 128, step: float = 3.8, noise: float = 0.5) -> np.ndarray:
    """n conformer-like chains, flattened to vectors of 3*beads coordinates.

    Draw order: for each of ``n_seeds`` seed chains, beads-1 step directions
    (standard normal 3-vectors normalised to unit length, times ``step``) with
    bead 0 at the origin; then the seed chain of each conformer (uniform);
    then N(0, noise^2) per coordinate.
    """
    dirs = rng.standard_normal(size=(n_seeds, beads - 1, 3))
    dirs /= np.linalg.norm(dirs, axis=2, keepdims=True)
    chains = np.zeros((n_seeds, beads, 3))
    chains[:, 1:, :] = np.cumsum(step * dirs, axis=1)
    seed_of = rng.integers(0, n_seeds, size=n)
    pts = chains[seed_of].reshape(n, beads * 3)
    pts = pts + noise * rng.standard_normal(size=pts.shape)
    return pts


# ----------------------------------------------------------------------------
# distances
# ----------------------------------------------------------------------------

def _finish_numpy(ss: np.ndarray, scale, quantum_inv) -> np.ndarray:
    d = np.sqrt(ss)
    if scale is not None:
        d = d / scale
    if quantum_inv is not None:
        d = np.round(d * quantum_inv) / quantum_inv
    return d.astype(np.float32)


def packed_distances(points: np.ndarray, scale: float | None = None,
                     quantum_inv: float | None = None, device=None,
                     block_bytes: int = 1 << 28):
    """Packed upper-triangle FP32 distance matrix of ``points`` (n x dim).

    With ``device=None`` the result is a numpy array; with a torch device the
    computation runs there in FP64 and a torch float32 tensor on that device
    is returned.  Both paths evaluate, per pair, acc = 0; acc += (x_d - y_d)^2
    for d in coordinate order; d = sqrt(acc) [/ scale] [rounded to a multiple
    of 1/quantum_inv]; then one rounding to FP32.
    """
    n, dim = points.shape
    if device is None:
        out = np.empty(packed_size(n), dtype=np.float32)
        X = np.ascontiguousarray(points, dtype=np.float64)
        pos = 0
        r0 = 0
        while r0 < n - 1:
            cols = n - r0
            B = max(1, min(n - 1 - r0, block_bytes // (8 * cols)))
            Xb = X[r0:r0 + B]
            Xc = X[r0:]
            acc = np.zeros((B, cols))
            for d in range(dim):
                t = Xb[:, d, None] - Xc[None, :, d]
                acc += t * t
            blk = _finish_numpy(acc, scale, quantum_inv)
            for a in range(B):
                seg = blk[a, a + 1:]
                out[pos:pos + seg.size] = seg
                pos += seg.size
            r0 += B
        assert pos == out.size
        return out

    import torch
    X = torch.as_tensor(np.ascontiguousarray(points, dtype=np.float64), device=device)
    out = torch.empty(packed_size(n), dtype=torch.float32, device=device)
    pos = 0
    r0 = 0
    while r0 < n - 1:
        cols = n - r0
        B = max(1, min(n - 1 - r0, block_bytes // (8 * cols)))
        Xb = X[r0:r0 + B]
        Xc = X[r0:]
        acc = torch.zeros((B, cols), dtype=torch.float64, device=device)
        for d in range(dim):
            t = Xb[:, d, None] - Xc[None, :, d]
            acc.add_(t * t)
        dd = torch.sqrt(acc)
        if scale is not None:
            dd = dd / scale
        if quantum_inv is not None:
            dd = torch.round(dd * quantum_inv) / quantum_inv
        blk = dd.to(torch.float32)
        mask = torch.ones((B, cols), dtype=torch.bool, device=device).triu(diagonal=1)
        seg = torch.masked_select(blk, mask)
        out[pos:pos + seg.numel()] = seg
        pos += seg.numel()
        r0 += B
    assert pos == out.numel()
    return out


# ----------------------------------------------------------------------------
# small test inputs
# ----------------------------------------------------------------------------

def small_gmm(n: int, seed: int, dim: int = 8, k: int = 4) -> np.ndarray:
    """A small Gaussian-mixture matrix (FP32, packed) for fuzz and unit tests."""
    rng = np.random.default_rng(seed)
    pts = gmm_points(rng, n, dim, max(1, min(k, n)))
    return packed_distances(pts)


def tie_heavy(n: int, seed: int, levels: int = 8) -> np.ndarray:
    """A packed matrix of integer-valued distances in [0, levels], many ties.

    Zero distances are allowed (duplicate objects).  Draw: one uniform integer
    per cell in packed order.
    """
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels + 1, size=packed_size(n)).astype(np.float32)


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    linkages: tuple
    seed: int
    description: str
    points_fn: object = field(repr=False, default=None)
    scale: float | None = None
    quantum_inv: float | None = None

    def points(self) -> np.ndarray:
        return self.points_fn(np.random.default_rng(self.seed))

    def matrix(self, device=None):
        return packed_distances(self.points(), scale=self.scale,
                                quantum_inv=self.quantum_inv, device=device)


def workload(name: str) -> Workload:
    """The named synthetic workloads (sizes and distributions of the paper's use case).

    * ``gmm512``: n=512 points in R^8 from 8 isotropic Gaussians (centers
      U[-10,10]^8, sigma=1), seed 0; complete linkage.
    * ``gmm16384q``: n=16384 points in R^64 from a 32-component mixture with
      sigma_c ~ U[0.5, 2], centers U[-10,10]^64, distances rounded to
      multiples of 1/1024 (forces ties), seed 1; single/complete/average.
    * ``conformer65536``: n=65536 conformer-like chains (64 seed chains of 128
      beads, step 3.8, noise 0.5), d = ||delta|| / sqrt(128), seed 2;
      complete and Ward.
    * ``serve<N>``: N points in R^16 from 16 isotropic Gaussians (centers
      U[-10,10]^16, sigma=1), seed 4: one request of the serving stream's
      recipe at a chosen size.
    Smaller ``conformer<N>`` / ``gmm<N>`` variants use the same recipes.
    """
    if name == "gmm512":
        return Workload(name, 512, (COMPLETE,), 0,
                        "512 points in R^8, 8 isotropic Gaussians, centers U[-10,10]^8, sigma=1, seed 0",
                        lambda rng: gmm_points(rng, 512, 8, 8, 10.0, 1.0))
    if name.startswith("gmm") and name.endswith("q"):
        n = int(name[3:-1])
        return Workload(name, n, (SINGLE, COMPLETE, AVERAGE), 1,
                        f"{n} points in R^64, 32 Gaussians sigma~U[0.5,2], centers U[-10,10]^64, "
                        "distances rounded to multiples of 1/1024, seed 1",
                        lambda rng: gmm_points(rng, n, 64, 32, 10.0, (0.5, 2.0)),
                        None, 1024.0)
    if name.startswith("conformer"):
        n = int(name[len("conformer"):])
        return Workload(name, n, (COMPLETE, WARD), 2,
                        f"{n} conformer-like chains (64 seeds x 128 beads, step 3.8, noise 0.5), "
                        "d=||delta||/sqrt(128), seed 2",
                        lambda rng: conformer_points(rng, n),
                        math.sqrt(128.0), None)
    if name.startswith("serve"):
        n = int(name[len("serve"):])
        return Workload(name, n, (SINGLE, COMPLETE, AVERAGE, WARD), 4,
                        f"{n} points in R^16, 16 isotropic Gaussians (centers U[-10,10]^16, sigma=1), "
                        "the serving stream's recipe, seed 4",
                        lambda rng: gmm_points(rng, n, 16, 16, 10.0, 1.0))
    if name.startswith("gmm"):
        n = int(name[3:])
        return Workload(name, n, (COMPLETE,), 0,
                        f"{n} points in R^8, 8 isotropic Gaussians, centers U[-10,10]^8, sigma=1, seed 0",
                        lambda rng: gmm_points(rng, n, 8, 8, 10.0, 1.0))
    raise KeyError(name)


def batch_jobs(n_jobs: int = 4096, seed: int = 3, n_lo: int = 64, n_hi: int = 2048):
    """Specs of independent clustering jobs of uneven size.

    Draw order per job: n = floor(exp(U[ln n_lo, ln n_hi])), linkage uniform
    over {single, complete, average, Ward}, mixture size K uniform in 4..32,
    then the points (R^16, centers U[-10,10]^16, sigma=1) from a per-job
    generator seeded with (seed, job index).  Returns a list of
    (n, linkage, point_seed, K) tuples; ``job_matrix`` turns one into a matrix.
    """
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n_jobs):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n = max(n_lo, min(n_hi, n))
        link = int(rng.integers(0, 4))
        K = int(rng.integers(4, 33))
        specs.append((n, link, K))
    return specs


def job_points(spec, job_index: int, seed: int = 3) -> np.ndarray:
    n, _, K = spec
    rng = np.random.default_rng([seed, job_index])
    return gmm_points(rng, n, 16, K, 10.0, 1.0)


def job_matrix(spec, job_index: int, seed: int = 3, device=None):
    return packed_distances(job_points(spec, job_index, seed), device=device)


def serve_requests(n_requests: int = 2000, rate: float = 200.0, seed: int = 4,
                   n_lo: int = 256, n_hi: int = 32768):
    """A Poisson request stream: list of (arrival_s, n, linkage, K, point_seed).

    Draw order per request: exponential gap with mean 1/rate, then
    n = floor(exp(U[ln n_lo, ln n_hi])), linkage uniform over 4, K uniform
    in 4..32.  Points come from a generator seeded with (seed, request index).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for q in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n = max(n_lo, min(n_hi, n))
        link = int(rng.integers(0, 4))
        K = int(rng.integers(4, 33))
        out.append((t, n, link, K, q))
    return out

"""Seeded synthetic inputs for the Lance-Williams clustering path.

This package is shared by the CPU oracle (``oracle/``) and the CUDA library
(``paper_1709_06816_gb300``). It draws points and turns them into packed
upper-triangle FP32 dissimilarity matrices; it holds none of the clustering
arithmetic (no minimum search, no update formula, no linkage coefficients).
"""
from .generators import (  # noqa: F401
    Workload,
    gmm_points,
    conformer_points,
    packed_distances,
    packed_size,
    small_gmm,
    tie_heavy,
    workload,
    batch_jobs,
    job_points,
    job_matrix,
    serve_requests,
    SINGLE, COMPLETE, AVERAGE, WARD, WEIGHTED, CENTROID, LINKAGE_NAMES,
)

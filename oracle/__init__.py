"""CPU oracle of the Lance-Williams merge loop -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library ``paper_1709_06816_gb300``; both read their inputs from ``synth``.

The arithmetic lives in ``lw_oracle.c`` (plain C, FP32, no FMA contraction,
OpenMP over host cores); this module only compiles it with gcc and marshals
numpy arrays through ctypes.

Functions:
  naive(D, n, linkage)   -- Section 4 loop verbatim: full minimum search per iteration.
  cached(D, n, linkage)  -- the same loop with a per-row minimum cache.
  coefficients(...)      -- Table 1 (a_i, a_j, b, g) in FP32.
  update(...)            -- the Section 4 step-3 formula for one cell.
  sample(D, n, linkage)  -- wall time of the cached loop on a bounded prefix
                            (validation + the first K merges), for CPU baselines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblw_oracle.so")
_lock = threading.Lock()
_lib = None

SINGLE, COMPLETE, AVERAGE, WARD, WEIGHTED, CENTROID = 0, 1, 2, 3, 4, 5


class OracleError(RuntimeError):
    pass


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile lw_oracle.c (or the copy at ``src`` into ``out``) with gcc:
    FP32 IEEE arithmetic, -ffp-contract=off (no fused multiply-add), OpenMP."""
    src = src or _SRC
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class OracleLib:
    """ctypes view of one compiled copy of lw_oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        f32p = ctypes.POINTER(ctypes.c_float)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.lwo_naive.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, i32p, f32p, i64p]
        lib.lwo_naive.restype = ctypes.c_int
        lib.lwo_cached.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, i32p, f32p,
                                   ctypes.c_int64, i64p, f64p]
        lib.lwo_cached.restype = ctypes.c_int
        lib.lwo_coefficients.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, f32p]
        lib.lwo_coefficients.restype = None
        lib.lwo_update.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        lib.lwo_update.restype = ctypes.c_float
        lib.lwo_threads.argtypes = []
        lib.lwo_threads.restype = ctypes.c_int
        lib.lwo_set_threads.argtypes = [ctypes.c_int]
        lib.lwo_set_threads.restype = None
        self.lib = lib

    def naive(self, D, n: int, linkage: int, inplace: bool = False):
        """Section 4 loop verbatim.  Returns (merges int32 (n-1, 2), heights float32
        (n-1), cells scanned per iteration int64 (n-1))."""
        D = _matrix(D, n, inplace)
        m = max(n - 1, 0)
        merges = np.zeros((m, 2), dtype=np.int32)
        heights = np.zeros(m, dtype=np.float32)
        scanned = np.zeros(m, dtype=np.int64)
        _check(self.lib.lwo_naive(_ptr(D, ctypes.c_float), n, linkage,
                                  _ptr(merges, ctypes.c_int32), _ptr(heights, ctypes.c_float),
                                  _ptr(scanned, ctypes.c_int64)))
        return merges, heights, scanned

    def cached(self, D, n: int, linkage: int, max_merges: int = -1, inplace: bool = False):
        """Section 4 loop with a row-minimum cache.  Returns (merges, heights, stats, times).

        stats keys: rescans, rescan_cells, updated, rowi_cells, merges, sum_m.
        times: (seconds validating + building the cache, seconds in the merge loop).
        """
        D = _matrix(D, n, inplace)
        m = max(n - 1, 0)
        if max_merges >= 0:
            m = min(m, max_merges)
        merges = np.zeros((m, 2), dtype=np.int32)
        heights = np.zeros(m, dtype=np.float32)
        st = np.zeros(6, dtype=np.int64)
        tm = np.zeros(2, dtype=np.float64)
        _check(self.lib.lwo_cached(_ptr(D, ctypes.c_float), n, linkage,
                                   _ptr(merges, ctypes.c_int32), _ptr(heights, ctypes.c_float),
                                   max_merges, _ptr(st, ctypes.c_int64), _ptr(tm, ctypes.c_double)))
        stats = dict(zip(("rescans", "rescan_cells", "updated", "rowi_cells", "merges", "sum_m"),
                         (int(x) for x in st)))
        return merges, heights, stats, (float(tm[0]), float(tm[1]))

    def coefficients(self, linkage: int, ni: int, nj: int, nk: int) -> np.ndarray:
        """Table 1 row for ``linkage`` as FP32 (a_i, a_j, b, g)."""
        out = np.zeros(4, dtype=np.float32)
        self.lib.lwo_coefficients(linkage, ni, nj, nk, _ptr(out, ctypes.c_float))
        return out

    def update(self, linkage: int, dki: float, dkj: float, dij: float,
               ni: int, nj: int, nk: int) -> np.float32:
        """Section 4 step-3 formula for one cell, in FP32."""
        return np.float32(self.lib.lwo_update(linkage, dki, dkj, dij, ni, nj, nk))


def _load() -> OracleLib:
    global _lib
    with _lock:
        if _lib is None:
            _lib = OracleLib(build())
        return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


_ERR = {1: "invalid argument", 2: "invalid input (NaN, infinite or negative distance)",
        3: "out of host memory"}


def _check(rc: int):
    if rc != 0:
        raise OracleError(f"oracle status {rc}: {_ERR.get(rc, 'unknown')}")


def _matrix(D, n: int, inplace: bool) -> np.ndarray:
    D = np.asarray(D)
    if D.dtype != np.float32 or D.ndim != 1 or D.size != n * (n - 1) // 2:
        raise ValueError("D must be a flat float32 array of n(n-1)/2 cells")
    if inplace:
        if not D.flags.c_contiguous or not D.flags.writeable:
            raise ValueError("in-place D must be a writeable contiguous array")
        return D
    return np.array(D, dtype=np.float32, copy=True)


def naive(D, n: int, linkage: int, inplace: bool = False):
    return _load().naive(D, n, linkage, inplace)


def cached(D, n: int, linkage: int, max_merges: int = -1, inplace: bool = False):
    return _load().cached(D, n, linkage, max_merges, inplace)


naive.__doc__ = OracleLib.naive.__doc__
cached.__doc__ = OracleLib.cached.__doc__


def coefficients(linkage: int, ni: int, nj: int, nk: int) -> np.ndarray:
    """Table 1 row for ``linkage`` as FP32 (a_i, a_j, b, g)."""
    return _load().coefficients(linkage, ni, nj, nk)


def update(linkage: int, dki: float, dkj: float, dij: float, ni: int, nj: int, nk: int) -> np.float32:
    """Section 4 step-3 formula for one cell, in FP32."""
    return _load().update(linkage, dki, dkj, dij, ni, nj, nk)


def threads() -> int:
    return int(_load().lib.lwo_threads())


def set_threads(k: int) -> None:
    _load().lib.lwo_set_threads(int(k))


def sample(D, n: int, linkage: int, target_s: float = 12.0) -> dict:
    """Time the cached loop, as it stands, on validation + the first K merges
    of ``D`` (left unchanged), K chosen from a 50-merge calibration so the
    sample takes about ``target_s`` seconds.  The full-run time is estimated by
    scaling the sample's loop time with the work of the whole run, sum over
    merges of the live cluster count m_t = n - t.

    Returns {"K", "t_init_s", "t_loop_s", "est_total_s", "wall_s", "cores"}.
    """
    D = np.asarray(D)
    work = np.empty_like(D)
    np.copyto(work, D)
    _, _, _, (t_init, t_loop) = cached(work, n, linkage, max_merges=50, inplace=True)
    per_merge = t_loop / 50.0
    K = int(max(100, min(n - 1, (target_s - t_init) / max(per_merge, 1e-6))))
    np.copyto(work, D)
    w0 = time.perf_counter()
    _, _, _, (t_init, t_loop) = cached(work, n, linkage, max_merges=K, inplace=True)
    wall = time.perf_counter() - w0
    del work
    sum_all = n * (n + 1) / 2 - 1
    sum_k = K * n - K * (K - 1) / 2
    est_total = t_init + t_loop * sum_all / sum_k
    return {"K": K, "t_init_s": t_init, "t_loop_s": t_loop, "est_total_s": est_total,
            "wall_s": wall, "cores": threads()}

"""ctypes binding of liblw.so (the C ABI in include/lw.h).

Argument marshalling only: every step of the clustering runs in the CUDA
kernels of liblw.so.  There is no CPU fallback: if the library is missing
or cannot be loaded, every call raises.

Functions keep the C names (``lw_create``, ``lw_cluster``, ...); the
``Context`` class wraps them for torch tensors and numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblw.so")
# built with -DLW_CHECKED (global accesses of the merge kernel bounds-checked);
# loaded instead of liblw.so when LW_CHECKED=1 is in the environment
CHECKED_LIB_PATH = os.path.join(_HERE, "liblw_checked.so")

LW_SINGLE, LW_COMPLETE, LW_AVERAGE, LW_WARD, LW_WEIGHTED, LW_CENTROID = 0, 1, 2, 3, 4, 5
LINKAGES = {"single": 0, "complete": 1, "average": 2, "ward": 3, "weighted": 4, "centroid": 5}
LW_OPT_GRID, LW_OPT_TIMEOUT_MS = 1, 2
STATUS = {0: "LW_OK", 1: "LW_ERR_INVALID_ARG", 2: "LW_ERR_INVALID_INPUT", 3: "LW_ERR_OOM",
          4: "LW_ERR_CUDA", 5: "LW_ERR_TIMEOUT", 6: "LW_ERR_BUSY", 7: "LW_ERR_CANCELLED"}

# every symbol include/lw.h declares
EXPORTS = ("lw_create", "lw_cluster", "lw_cluster_async", "lw_wait", "lw_get_stats",
           "lw_set_option", "lw_status_string", "lw_last_error", "lw_destroy",
           "lw_batch_create", "lw_batch_run", "lw_batch_wait", "lw_batch_destroy",
           "lw_set_batch_classes",
           "lw_cluster_batch", "lw_server_create", "lw_server_submit", "lw_server_poll",
           "lw_server_drain", "lw_server_get_stats", "lw_server_destroy", "lw_server_cancel",
           "lw_cluster_noalloc")
LW_OPT_PHASE_TIMES, LW_OPT_BATCH_SPLIT, LW_OPT_CTA_THREADS, LW_OPT_LAYOUT = 4, 5, 6, 7
LW_OPT_TEST_FAIL_ALLOC = 8


class LwServerStats(ctypes.Structure):
    """struct lw_server_stats of include/lw.h."""
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("peak_inflight", ctypes.c_int32),
                ("cancelled", ctypes.c_int32), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("wall_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LwJob(ctypes.Structure):
    """struct lw_job of include/lw.h."""
    _fields_ = [("dist", ctypes.c_void_p), ("n", ctypes.c_int64), ("linkage", ctypes.c_int32),
                ("status", ctypes.c_int32), ("merges_out", ctypes.c_void_p),
                ("heights_out", ctypes.c_void_p)]
LW_NOALLOC_MAX_N = 16384

_lib = None
_lock = threading.Lock()


class LwError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {detail}")


def load(path: str | None = None):
    """Load liblw.so, or liblw_checked.so when LW_CHECKED=1 (raises if it is
    not built)."""
    global _lib
    if path is None:
        path = CHECKED_LIB_PATH if os.environ.get("LW_CHECKED") == "1" else LIB_PATH
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run __graft_entry__.build() "
                               "(the CUDA library is required, there is no fallback)")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.lw_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
        lib.lw_create.restype = ctypes.c_int
        for name in ("lw_cluster", "lw_cluster_async"):
            f = getattr(lib, name)
            f.argtypes = [vp, vp, i64, ctypes.c_int, vp, vp]
            f.restype = ctypes.c_int
        lib.lw_wait.argtypes = [vp]
        lib.lw_wait.restype = ctypes.c_int
        lib.lw_get_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.c_int]
        lib.lw_get_stats.restype = ctypes.c_int
        lib.lw_set_option.argtypes = [vp, ctypes.c_int, i64]
        lib.lw_set_option.restype = ctypes.c_int
        lib.lw_status_string.argtypes = [ctypes.c_int]
        lib.lw_status_string.restype = ctypes.c_char_p
        lib.lw_last_error.argtypes = [vp]
        lib.lw_last_error.restype = ctypes.c_char_p
        lib.lw_destroy.argtypes = [vp]
        lib.lw_destroy.restype = None
        lib.lw_cluster_noalloc.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp]
        lib.lw_cluster_noalloc.restype = ctypes.c_int
        jp = ctypes.POINTER(LwJob)
        lib.lw_batch_create.argtypes = [vp, jp, ctypes.c_int32, ctypes.POINTER(vp)]
        lib.lw_batch_create.restype = ctypes.c_int
        lib.lw_batch_run.argtypes = [vp]
        lib.lw_batch_run.restype = ctypes.c_int
        lib.lw_batch_wait.argtypes = [vp, jp]
        lib.lw_batch_wait.restype = ctypes.c_int
        lib.lw_batch_destroy.argtypes = [vp]
        lib.lw_batch_destroy.restype = None
        lib.lw_set_batch_classes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_int32]
        lib.lw_set_batch_classes.restype = ctypes.c_int
        lib.lw_cluster_batch.argtypes = [vp, jp, ctypes.c_int32]
        lib.lw_cluster_batch.restype = ctypes.c_int
        lib.lw_server_create.argtypes = [ctypes.c_int, i64, ctypes.c_int32, ctypes.POINTER(vp)]
        lib.lw_server_create.restype = ctypes.c_int
        lib.lw_server_submit.argtypes = [vp, vp, i64, ctypes.c_int, vp, vp,
                                         ctypes.POINTER(ctypes.c_uint64)]
        lib.lw_server_submit.restype = ctypes.c_int
        lib.lw_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        lib.lw_server_poll.restype = ctypes.c_int
        lib.lw_server_cancel.argtypes = [vp, ctypes.c_uint64]
        lib.lw_server_cancel.restype = ctypes.c_int
        lib.lw_server_drain.argtypes = [vp]
        lib.lw_server_drain.restype = ctypes.c_int
        lib.lw_server_get_stats.argtypes = [vp, ctypes.POINTER(LwServerStats)]
        lib.lw_server_get_stats.restype = ctypes.c_int
        lib.lw_server_destroy.argtypes = [vp]
        lib.lw_server_destroy.restype = None
        _lib = lib
        return lib


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array (contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer {type(x)}")


# ---- C-named functions ------------------------------------------------------

def lw_create(device: int = 0, stream=None) -> int:
    lib = load()
    h = ctypes.c_void_p()
    s = lib.lw_create(ctypes.byref(h), int(device), stream)
    if s != 0:
        raise LwError(s, "lw_create")
    return h.value


def lw_cluster(ctx: int, dist, n: int, linkage: int, merges_out, heights_out) -> None:
    lib = load()
    s = lib.lw_cluster(ctx, _ptr(dist), int(n), int(linkage), _ptr(merges_out), _ptr(heights_out))
    if s != 0:
        raise LwError(s, lib.lw_last_error(ctx).decode())


def lw_cluster_async(ctx: int, dist, n: int, linkage: int, merges_out, heights_out) -> None:
    lib = load()
    s = lib.lw_cluster_async(ctx, _ptr(dist), int(n), int(linkage), _ptr(merges_out),
                             _ptr(heights_out))
    if s != 0:
        raise LwError(s, lib.lw_last_error(ctx).decode())


def lw_wait(ctx: int) -> None:
    lib = load()
    s = lib.lw_wait(ctx)
    if s != 0:
        raise LwError(s, lib.lw_last_error(ctx).decode())


def lw_get_stats(ctx: int) -> dict:
    lib = load()
    a = (ctypes.c_int64 * 33)()
    s = lib.lw_get_stats(ctx, a, 33)
    if s != 0:
        raise LwError(s, "lw_get_stats")
    out = {"rounds": a[0], "idle_rounds": a[1], "updated": a[2], "grid": a[3],
           "refills": a[4], "refill_cells": a[5], "installs": a[6], "walk_steps": a[7],
           "rescans": a[14], "rescan_cells": a[15]}
    if any(a[8:14]):
        G = max(1, a[3])
        names = ("barrier", "walk", "pass1", "refill", "certify", "pass2")
        out["phase_ms"] = {nm: a[8 + q] / G / 1e6 for q, nm in enumerate(names)}
        sub = ("records", "walk_installs", "chain", "minima", "certify", "bookkeeping", "pass2",
               "rescans", "scan_log", "scan_matrix", "walk_only")
        out["subphase_ms"] = {nm: a[16 + q] / G / 1e6 for q, nm in enumerate(sub)}
        if a[28] > 0:
            out["barrier_detail"] = {
                "barriers": a[28],
                "last_arriver_wait_us": a[27] / a[28] / 1e3,
                "b_last_serving_refill": a[30] / max(1, a[29]),
                "a_last_serving_refill": a[31] / max(1, a[28] - a[29]),
                "last_is_cta0": a[32] / a[28],
            }
    return out


def lw_set_option(ctx: int, option: int, value: int) -> None:
    s = load().lw_set_option(ctx, int(option), int(value))
    if s != 0:
        raise LwError(s, f"lw_set_option({option}, {value})")


def lw_cluster_noalloc(dist, n: int, linkage: int, merges_out, heights_out, stream=None) -> None:
    """Clustering for callers that cannot allocate: device buffers only,
    scratch in the library's fixed device array (n <= LW_NOALLOC_MAX_N)."""
    lib = load()
    sp = None
    if stream is not None:
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    s = lib.lw_cluster_noalloc(_ptr(dist), int(n), int(linkage), _ptr(merges_out),
                               _ptr(heights_out), sp)
    if s != 0:
        raise LwError(s, "lw_cluster_noalloc")


def lw_batch_create(ctx: int, jobs) -> int:
    """jobs: a ctypes array of LwJob.  Returns the plan handle."""
    lib = load()
    h = ctypes.c_void_p()
    s = lib.lw_batch_create(ctx, jobs, len(jobs), ctypes.byref(h))
    if s != 0:
        raise LwError(s, lib.lw_last_error(ctx).decode())
    return h.value


def lw_batch_run(batch: int, ctx: int = 0) -> None:
    lib = load()
    s = lib.lw_batch_run(batch)
    if s != 0:
        raise LwError(s, lib.lw_last_error(ctx).decode() if ctx else "lw_batch_run")


def lw_batch_wait(batch: int, jobs=None) -> int:
    """Waits; fills jobs[q].status; returns the first failing status (0 = all ok)."""
    return int(load().lw_batch_wait(batch, jobs))


def lw_batch_destroy(batch: int) -> None:
    if batch:
        load().lw_batch_destroy(batch)


def lw_cluster_batch(ctx: int, jobs) -> int:
    """Blocking batch; fills jobs[q].status; returns the first failing status."""
    return int(load().lw_cluster_batch(ctx, jobs, len(jobs)))


class Server:
    """A continuous-batching request loop (lw_server_* of include/lw.h)."""

    def __init__(self, device: int = 0, budget_bytes: int = 1 << 30, lanes: int = 8):
        lib = load()
        h = ctypes.c_void_p()
        s = lib.lw_server_create(int(device), int(budget_bytes), int(lanes), ctypes.byref(h))
        if s != 0:
            raise LwError(s, "lw_server_create")
        self.handle = h.value

    def submit(self, D, n: int, linkage, merges, heights) -> int:
        if isinstance(linkage, str):
            linkage = LINKAGES[linkage]
        t = ctypes.c_uint64()
        s = load().lw_server_submit(self.handle, _ptr(D) if n > 1 else None, int(n), int(linkage),
                                    _ptr(merges) if n > 1 else None,
                                    _ptr(heights) if n > 1 else None, ctypes.byref(t))
        if s != 0:
            raise LwError(s, "lw_server_submit")
        return t.value

    def poll(self, ticket: int):
        """(done, status, latency_ms)."""
        d = ctypes.c_int32()
        st = ctypes.c_int()
        lat = ctypes.c_double()
        s = load().lw_server_poll(self.handle, ticket, ctypes.byref(d), ctypes.byref(st),
                                  ctypes.byref(lat))
        if s != 0:
            raise LwError(s, "lw_server_poll")
        return bool(d.value), st.value, lat.value

    def cancel(self, ticket: int) -> int:
        """lw_server_cancel: 0 if the queued request was withdrawn, else its status code."""
        return int(load().lw_server_cancel(self.handle, ticket))

    def drain(self) -> int:
        return int(load().lw_server_drain(self.handle))

    def stats(self) -> dict:
        st = LwServerStats()
        load().lw_server_get_stats(self.handle, ctypes.byref(st))
        return st.as_dict()

    def close(self):
        if self.handle:
            load().lw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lw_status_string(status: int) -> str:
    return load().lw_status_string(int(status)).decode()


def lw_destroy(ctx: int) -> None:
    if ctx:
        load().lw_destroy(ctx)


# ---- convenience wrapper ----------------------------------------------------

class Context:
    """One lw_ctx on one device; outputs are allocated next to the inputs.

    ``cluster(D, n, linkage)`` takes a flat float32 torch tensor (CUDA or
    CPU) or numpy array holding the packed upper triangle and returns
    (merges int32 (n-1, 2), heights float32 (n-1)) of the same kind.  A CUDA
    ``D`` is overwritten in place (pass ``D.clone()`` to keep it); a host
    ``D`` is copied by the library and left unchanged.
    """

    def __init__(self, device: int = 0, stream=None):
        self.device = device
        sp = None
        if stream is not None:
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.handle = lw_create(device, sp)

    def close(self):
        if self.handle:
            lw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_grid(self, G: int):
        lw_set_option(self.handle, LW_OPT_GRID, G)

    def set_phase_timing(self, on: bool = True):
        lw_set_option(self.handle, 4, 1 if on else 0)

    def set_batch_classes(self, classes):
        """classes: [(n_hi, cta_threads), ...] ascending in n_hi; [] = default."""
        k = len(classes)
        nh = (ctypes.c_int64 * max(k, 1))(*[int(a) for a, _ in classes])
        nt = (ctypes.c_int32 * max(k, 1))(*[int(b) for _, b in classes])
        s = load().lw_set_batch_classes(self.handle, nh, nt, k)
        if s != 0:
            raise LwError(s, f"lw_set_batch_classes({classes})")

    def set_layout(self, layout: int):
        """0 automatic (row-log layout for multi-CTA runs when it fits), 1 row-log
        layout, 2 packed triangle."""
        lw_set_option(self.handle, LW_OPT_LAYOUT, layout)

    def set_cta_threads(self, nt: int):
        lw_set_option(self.handle, LW_OPT_CTA_THREADS, nt)

    def set_batch_split(self, n: int):
        lw_set_option(self.handle, LW_OPT_BATCH_SPLIT, n)

    def make_jobs(self, mats, ns, linkages):
        """Job table for device matrices; allocates the device outputs.
        Returns (ctypes LwJob array, list of (merges, heights) tensors)."""
        import torch
        jobs = (LwJob * len(mats))()
        outs = []
        for q, (D, n, link) in enumerate(zip(mats, ns, linkages)):
            if isinstance(link, str):
                link = LINKAGES[link]
            self._check_matrix(D, n)
            m = torch.empty((max(n - 1, 0), 2), dtype=torch.int32, device=D.device)
            h = torch.empty(max(n - 1, 0), dtype=torch.float32, device=D.device)
            jobs[q].dist = D.data_ptr() if D.numel() else 0
            jobs[q].n = n
            jobs[q].linkage = link
            jobs[q].status = -1
            jobs[q].merges_out = m.data_ptr() if m.numel() else 0
            jobs[q].heights_out = h.data_ptr() if h.numel() else 0
            outs.append((m, h))
        return jobs, outs

    def cluster_batch(self, mats, ns, linkages):
        """Cluster many device matrices in one batch.  Returns (outs, statuses)."""
        jobs, outs = self.make_jobs(mats, ns, linkages)
        lw_cluster_batch(self.handle, jobs)
        return outs, [jobs[q].status for q in range(len(mats))]

    def set_timeout_ms(self, ms: int):
        lw_set_option(self.handle, LW_OPT_TIMEOUT_MS, ms)

    def stats(self) -> dict:
        return lw_get_stats(self.handle)

    def _outputs(self, D, n):
        m = max(n - 1, 0)
        if not isinstance(D, np.ndarray):
            import torch
            merges = torch.empty((m, 2), dtype=torch.int32, device=D.device)
            heights = torch.empty(m, dtype=torch.float32, device=D.device)
        else:
            merges = np.empty((m, 2), dtype=np.int32)
            heights = np.empty(m, dtype=np.float32)
        return merges, heights

    @staticmethod
    def _check_matrix(D, n):
        size = D.numel() if hasattr(D, "numel") else D.size
        dt = str(D.dtype)
        if "float32" not in dt:
            raise ValueError("D must be float32")
        if size != n * (n - 1) // 2:
            raise ValueError(f"D has {size} cells, expected n(n-1)/2 = {n * (n - 1) // 2}")

    def cluster(self, D, n: int, linkage, merges=None, heights=None):
        if isinstance(linkage, str):
            linkage = LINKAGES[linkage]
        self._check_matrix(D, n)
        if merges is None or heights is None:
            merges, heights = self._outputs(D, n)
        if n <= 1:
            return merges, heights
        lw_cluster(self.handle, D, n, linkage, merges, heights)
        return merges, heights

    def cluster_async(self, D, n: int, linkage, merges, heights):
        if isinstance(linkage, str):
            linkage = LINKAGES[linkage]
        self._check_matrix(D, n)
        lw_cluster_async(self.handle, D, n, linkage, merges, heights)

    def wait(self):
        lw_wait(self.handle)

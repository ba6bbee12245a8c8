#!/usr/bin/env python3
"""Benchmark of the Lance-Williams merge loop on GB300.

A step is one whole clustering of the n = 65536 conformer-like matrix
(complete linkage): the library validates the 8.59 GB packed triangle,
builds its working layout and row minima and performs all 65535 merges
(Section 4's iteration).  The kernels rewrite the matrix in place, so every
step first restores it from a pristine device copy (a device-to-device copy,
counted inside the step).

Printed (rank 0, one JSON line): merges/s over K timed steps (CUDA events on
the library's stream, W untimed warm-up steps), the dendrogram time, the
HBM roofline fraction of the merge kernel, a full-length parity check of the
result against the oracle's stored digest, the CPU oracle's rate (a bounded
sample, calibrated against a full oracle run), an end-to-end rate through
the C ABI with host buffers, the SM clocks sampled during the timed region,
and one block per other workload: the n = 65536 Ward run, the three
n = 16384 linkages, the n = 512 run against the L2 roofline, the batched
and the served workloads (each against the plain per-job path) and the
clustering time against the CTA count at n = 1968.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle instead (the reference arm): each step
is a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun, N > 1): independent replicas, one per GPU; no
collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "conformer65536"
LINKAGE = 1  # complete linkage, the paper's own choice (Section 5.3 step 6)
METRIC = "merges/s at n=65536 (complete linkage, bit-exact)"
UNIT = "merges/s"
FALLBACK_HBM_GBS = 6800.0
LINK_NAMES = {0: "single", 1: "complete", 2: "average", 3: "ward", 4: "weighted", 5: "centroid"}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one merge
# kernel launch on the bench workload, from one ncu capture of the bench's
# launch.  It describes the kernel code it was taken on (lw_merge.cu and
# lw_internal.h, comments aside) and is reported only while that code is
# unchanged.
MEASURED_TRAFFIC = {
    "workload": "conformer65536:1",
    "kernel_sha256": "7121625236e78601fa57f2afbc30f02cf54894b4e14f5da609e112627263da3e",
    "bytes_per_launch": 78290216448 + 23549573376,  # read + write
}


def kernel_source_sha256() -> str:
    """Hash of the merge kernel's code (the kernel and its constants), with
    // comments and blank space left out: an edit of the text around the code
    keeps a measurement valid, an edit of the code does not."""
    h = hashlib.sha256()
    for name in ("lw_merge.cu", "lw_internal.h"):
        with open(os.path.join(ROOT, "paper_1709_06816_gb300", "csrc", name), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def measured_traffic(workload: str, linkage: int):
    try:
        sha = kernel_source_sha256()
    except OSError:
        return None
    if (sha != MEASURED_TRAFFIC["kernel_sha256"] or f"{workload}:{linkage}" != MEASURED_TRAFFIC["workload"]
            or not MEASURED_TRAFFIC["bytes_per_launch"]):
        return None
    return MEASURED_TRAFFIC["bytes_per_launch"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def work_counts(key: str):
    """The oracle's record for a workload ("name:linkage"): exact counters,
    result digests and the CPU-sample calibration, written by
    ``python -m oracle.work_counts``; None if absent."""
    try:
        with open(os.path.join(ROOT, "bench_work_counts.json")) as f:
            return json.load(f).get(key)
    except FileNotFoundError:
        return None


def algorithmic_bytes(n: int, linkage: int, counts) -> tuple:
    """Bytes one clustering must move (per launch):
    init: read the packed triangle once, write n row keys (8 B);
    per merge t with m_t = n - t live clusters: read the m_t row keys (8 B),
    read D(k,i), D(k,j) and write D(k,i+j) for the m_t - 2 other clusters
    (12 B), Ward also reads m_t sizes (4 B), re-read every live cell of each
    row whose cached minimum pointed at i or j and got worse, and the live
    cells of the merged row i, whose minimum is recomputed (4 B each; the
    counts are the oracle's, one cached key per row), and write the step
    (12 B).  Returns (bytes, note)."""
    cells = n * (n - 1) // 2
    sum_m = n * (n + 1) // 2 - 1
    updated = (n - 1) * (n - 2) // 2  # sum over merges of m_t - 2
    b = 4 * cells + 8 * n + 8 * sum_m + 12 * updated + 12 * (n - 1)
    if linkage == 3:
        b += 4 * sum_m
    if counts is None:
        return b, "rescan term missing (no oracle counts for this workload)"
    return (b + 4 * int(counts["rescan_cells"]) + 4 * int(counts.get("rowi_cells", 0)),
            "rescan and row-i terms from the oracle's full run")


def sha256_of(a) -> str:
    """SHA-256 of an array's bytes in C order (the layout oracle.work_counts hashes)."""
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def parity_block(merges, heights, key: str):
    """Compare a whole GPU result with the oracle's stored digests of the
    same workload (all n - 1 merges and heights, bit for bit)."""
    rec = work_counts(key)
    if rec is None or "merges_sha256" not in rec:
        return {"oracle_sha_match": None, "note": f"no oracle digest for {key}"}
    mm = sha256_of(merges) == rec["merges_sha256"]
    hh = sha256_of(heights) == rec["heights_sha256"]
    return {"oracle_sha_match": bool(mm and hh), "merges_match": bool(mm), "heights_match": bool(hh),
            "reference": f"oracle full run ({rec.get('oracle_threads')} host threads, "
                         f"{rec.get('oracle_seconds')} s), bench_work_counts.json[{key}]"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """Largest value over the ranks (timed region length); identity at N = 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def bench_config(n: int, world: int) -> dict:
    """The workload description shared by both arms (same keys and values)."""
    return {"workload": WORKLOAD, "n": n, "linkage": LINK_NAMES[LINKAGE],
            "matrix_bytes": 4 * (n * (n - 1) // 2),
            "l2": f"inputs larger than L2 ({4 * (n * (n - 1) // 2) / 1e9:.2f} GB packed triangle)",
            "step": f"one clustering of the n={n} matrix: validate, row minima, {n - 1} merges",
            "parallelism": f"replicas{world}"}


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(D_host, n: int, linkage: int, key: str, target_s: float):
    """The oracle, as it stands, on a bounded prefix of the same matrix
    (oracle.sample), its full-run time estimated by the work sum(m_t) and
    then calibrated by the ratio that a full oracle run on this kind of host
    showed between its true time and the same estimate.  Returns (merges/s,
    info)."""
    import oracle
    smp = oracle.sample(D_host, n, linkage, target_s=target_s)
    rec = work_counts(key) or {}
    cal = (rec.get("sample") or {}).get("full_over_est")
    est = smp["est_total_s"]
    full = est * cal if cal else est
    info = dict(smp)
    info.update({"calibration": cal, "calibrated_total_s": full,
                 "uncalibrated_rate": (n - 1) / est})
    return (n - 1) / full, info


def cpu_sample_text(info, n):
    cal = info["calibration"]
    return (f"validation + first {info['K']} of {n - 1} merges of the same n={n} matrix on "
            f"{info['cores']} host threads ({info['wall_s']:.1f} s); full-run time estimated by "
            f"the work sum(m_t) ({info['est_total_s']:.1f} s)"
            + (f" x {cal:.3f}, the ratio of a full oracle run's time to the same estimate "
               f"({info['calibrated_total_s']:.1f} s)" if cal else " (no full-run calibration)"))


# ---------------------------------------------------------------------------
# helpers of the GPU arm
# ---------------------------------------------------------------------------

def time_steps(ctx, stream, src, work, n, link, m_out, h_out, warmup, steps):
    """W + K clusterings (restore + one launch each); returns the K kernel
    times (ms, CUDA events around the launch) and the total (ms)."""
    import torch

    def step(ev=None):
        with torch.cuda.stream(stream):
            work.copy_(src)
            if ev is not None:
                ev[0].record(stream)
            ctx.cluster_async(work, n, link, m_out, h_out)
            if ev is not None:
                ev[1].record(stream)
        ctx.wait()

    for _ in range(warmup):
        step()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(steps):
        step(kev[k])
    e1.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in kev], e0.elapsed_time(e1)


def l2_probe(device: int):
    """Measured L2 copy bandwidth: a device copy between two buffers that
    together stay well inside L2, repeated back to back (read + write bytes
    over CUDA-event time); the best of a few sizes."""
    import torch
    best = 0.0
    l2 = torch.cuda.get_device_properties(device).L2_cache_size
    for mb in (4, 8, 16):
        nbytes = mb << 20
        if 2 * nbytes > l2 // 2:
            continue
        a = torch.ones(nbytes // 4, device=f"cuda:{device}")
        b = torch.empty_like(a)
        for _ in range(5):
            b.copy_(a)
        reps = 200
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        gbs = 2 * nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
        best = max(best, gbs)
        del a, b
    return best


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import synth
    from paper_1709_06816_gb300 import Context

    torch.cuda.set_device(local)
    w = synth.workload(args.workload)
    n = w.n
    src = w.matrix(device=f"cuda:{local}")
    work = torch.empty_like(src)
    m_out = torch.empty((n - 1, 2), dtype=torch.int32, device=src.device)
    h_out = torch.empty(n - 1, dtype=torch.float32, device=src.device)
    stream = torch.cuda.Stream(device=src.device)
    ctx = Context(local, stream=stream)
    torch.cuda.synchronize()

    # warm-up (untimed), then the timed steps with the clocks sampled
    def step(ev=None):
        with torch.cuda.stream(stream):
            work.copy_(src)
            if ev is not None:
                ev[0].record(stream)
            ctx.cluster_async(work, n, LINKAGE, m_out, h_out)
            if ev is not None:
                ev[1].record(stream)
        ctx.wait()

    for _ in range(args.warmup):
        step()
    ref_m = m_out.clone()
    ref_h = h_out.clone()
    stats = ctx.stats()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for k in range(args.steps):
            step(kev[k])
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier(world)
    total_ms = e0.elapsed_time(e1)
    kernel_ms = [a.elapsed_time(b) for a, b in kev]
    deterministic = bool(torch.equal(ref_m, m_out) and torch.equal(ref_h, h_out))
    total_ms_max = max_over_ranks(total_ms, world)
    key = f"{args.workload}:{LINKAGE}"
    parity = parity_block(m_out.cpu().numpy(), h_out.cpu().numpy(), key)
    parity["deterministic_across_steps"] = deterministic

    # end-to-end through the C ABI with host buffers (pinned input, host outputs)
    e2e = None
    if not args.no_e2e:
        host = torch.empty(src.numel(), dtype=torch.float32, pin_memory=True)
        host.copy_(src)
        hm = np.empty((n - 1, 2), dtype=np.int32)
        hh = np.empty(n - 1, dtype=np.float32)
        ctx2 = Context(local)
        ctx2.cluster(host, n, LINKAGE, hm, hh)  # warm: allocates the device buffers
        reps = max(1, min(3, args.steps))
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx2.cluster(host, n, LINKAGE, hm, hh)
        e2e_s = (time.perf_counter() - t0) / reps
        e2e_ok = bool(np.array_equal(hm, ref_m.cpu().numpy())
                      and np.array_equal(hh.view(np.uint32), ref_h.cpu().numpy().view(np.uint32)))
        ctx2.close()
        del host
        e2e_s = max_over_ranks(e2e_s, world)
        e2e = {"value": world * (n - 1) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 4 * (n * (n - 1) // 2),
               "d2h_bytes_per_step": 12 * (n - 1) + 16 + 8 * 33,
               "seconds_per_step": e2e_s, "matches_device_run": e2e_ok,
               "note": "lw_cluster with a pinned host matrix and host outputs: the matrix crosses "
                       "the host link inside the timed call (read in place by the layout kernel), "
                       "then the clustering and the result copies"}

    peak, peak_kind = peaks()
    extra = {}
    if world == 1 and not args.no_configs:
        # the same matrix, Ward linkage (the other n = 65536 configuration)
        km, _ = time_steps(ctx, stream, src, work, n, 3, m_out, h_out, 1, 3)
        alg3, note3 = algorithmic_bytes(n, 3, work_counts(f"{args.workload}:3"))
        k3 = sum(km) / len(km)
        extra["conformer65536_ward"] = {
            "n": n, "linkage": "ward", "dendrogram_ms": k3, "merges_per_s": (n - 1) / (k3 * 1e-3),
            "roofline": {"bound": "hbm", "achieved": alg3 / (k3 * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg3 / (k3 * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": alg3,
                         "algorithmic_note": note3},
            "parity": parity_block(m_out.cpu().numpy(), h_out.cpu().numpy(), f"{args.workload}:3")}

    # CPU oracle on a bounded sample of the same matrix (rank 0, N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        D_host = src.cpu().numpy()
        rate, info = oracle_rate(D_host, n, LINKAGE, key, args.cpu_seconds)
        del D_host
        cpu = {"value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
               "sample": cpu_sample_text(info, n), "uncalibrated_value": info["uncalibrated_rate"]}

    ctx.close()
    del work, src
    torch.cuda.empty_cache()
    if world == 1 and not args.no_configs:
        extra.update(run_other_configs(args, local, peak))
    batched = None if args.no_batched else run_batched(args, local, peak)
    torch.cuda.empty_cache()
    serving = None if args.no_serving else run_serving(args, local)
    torch.cuda.empty_cache()
    sweep = None if (args.no_sweep or world > 1) else run_cta_sweep(args, local)
    alg, alg_note = algorithmic_bytes(n, LINKAGE, work_counts(key))
    k_avg_ms = sum(kernel_ms) / len(kernel_ms)
    achieved = alg / (k_avg_ms * 1e-3) / 1e9
    clocks = clk.summary()
    out = {
        "metric": METRIC if n == 65536 else METRIC.replace("n=65536", f"n={n}"),
        "value": world * args.steps * (n - 1) / (total_ms_max * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(n, world),
        "dendrogram_ms": k_avg_ms,
        "kernel_ms": kernel_ms,
        "parity": parity,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(args.workload, LINKAGE),
                     "algorithmic_bytes_per_launch": alg, "algorithmic_note": alg_note,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "merge_kernel (one persistent cooperative launch per clustering)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * 2,
        "gpu_launches_note": "per step: the layout kernel (symmetric copy of the triangle) and the "
                             "persistent merge kernel",
        "clocks": clocks,
        "counters": stats,
        "configs": extra,
        "batched": batched,
        "serving": serving,
        "cta_sweep": sweep,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_other_configs(args, local, peak):
    """The other single-matrix configurations, each checked in full against
    the oracle: n = 16384 (three linkages, distances on a 1/1024 grid: ties)
    against the HBM roofline, and n = 512 (complete) against the L2
    roofline (the matrix fits L2)."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1709_06816_gb300 import Context

    out = {}
    dev = f"cuda:{local}"
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream=stream)
    try:
        w = synth.workload("gmm16384q")
        n = w.n
        src = w.matrix(device=dev)
        work = torch.empty_like(src)
        m_out = torch.empty((n - 1, 2), dtype=torch.int32, device=dev)
        h_out = torch.empty(n - 1, dtype=torch.float32, device=dev)
        D_host = src.cpu().numpy() if not args.no_cpu_baseline else None
        for link in (0, 1, 2):
            km, _ = time_steps(ctx, stream, src, work, n, link, m_out, h_out, 2, 5)
            k = sum(km) / len(km)
            rec = work_counts(f"gmm16384q:{link}")
            alg, note = algorithmic_bytes(n, link, rec)
            out[f"gmm16384q_{LINK_NAMES[link]}"] = {
                "n": n, "linkage": LINK_NAMES[link], "dendrogram_ms": k, "merges_per_s": (n - 1) / (k * 1e-3),
                "roofline": {"bound": "hbm", "achieved": alg / (k * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": alg / (k * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": alg,
                             "algorithmic_note": note},
                "parity": parity_block(m_out.cpu().numpy(), h_out.cpu().numpy(), f"gmm16384q:{link}")}
            if D_host is not None:
                out[f"gmm16384q_{LINK_NAMES[link]}"]["cpu"] = cpu_single_and_all(D_host, n, link, rec)
        del src, work, D_host
        torch.cuda.empty_cache()

        w = synth.workload("gmm512")
        n = w.n
        D = w.matrix()
        src = torch.from_numpy(D).to(dev)
        work = torch.empty_like(src)
        m_out = torch.empty((n - 1, 2), dtype=torch.int32, device=dev)
        h_out = torch.empty(n - 1, dtype=torch.float32, device=dev)
        km, _ = time_steps(ctx, stream, src, work, n, 1, m_out, h_out, 5, 50)
        k = sum(km) / len(km)
        cores = oracle.threads()
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.cached(D, n, 1)
        one_s = time.perf_counter() - t0
        oracle.set_threads(cores)
        t0 = time.perf_counter()
        wm, wh, st, _ = oracle.cached(D, n, 1)
        all_s = time.perf_counter() - t0
        same = bool(np.array_equal(m_out.cpu().numpy(), wm)
                    and np.array_equal(h_out.cpu().numpy().view(np.uint32), wh.view(np.uint32)))
        alg, _ = algorithmic_bytes(n, 1, st)
        l2 = l2_probe(local)
        out["gmm512_complete"] = {
            "n": n, "linkage": "complete", "dendrogram_ms": k, "merges_per_s": (n - 1) / (k * 1e-3),
            "roofline": {"bound": "l2", "achieved": alg / (k * 1e-3) / 1e9, "peak": l2, "unit": "GB/s",
                         "frac": alg / (k * 1e-3) / 1e9 / l2, "algorithmic_bytes_per_launch": alg,
                         "peak_source": "measured here: L2-resident device copy (read + write bytes)",
                         "note": "one CTA (n <= 4096): a single SM works through 511 dependent merges"},
            "parity": {"oracle_match": same, "reference": "oracle run here on the same matrix"},
            "cpu": {"kind": "oracle, full runs on the same matrix", "single_thread_merges_per_s": (n - 1) / one_s,
                    "all_cores_merges_per_s": (n - 1) / all_s, "cores": cores}}
    finally:
        ctx.close()
    return out


def cpu_single_and_all(D_host, n: int, link: int, rec) -> dict:
    """The oracle on one host thread (a bounded sample of the same matrix, its
    full-run time estimated by the work sum(m_t), uncalibrated) and on all of
    them (the full run that made the stored digest)."""
    import oracle
    cores = oracle.threads()
    oracle.set_threads(1)
    try:
        smp = oracle.sample(D_host, n, link, target_s=3.0)
    finally:
        oracle.set_threads(cores)
    out = {"kind": "oracle", "single_thread_merges_per_s": (n - 1) / smp["est_total_s"],
           "single_thread_sample": f"validation + first {smp['K']} of {n - 1} merges on 1 thread "
                                   f"({smp['wall_s']:.1f} s), full run estimated by the work sum(m_t), uncalibrated "
                                   f"(on the n = 65536 matrix that model ran about 1.5x short of a full run)"}
    if rec and rec.get("oracle_seconds"):
        out["all_cores_merges_per_s"] = (n - 1) / rec["oracle_seconds"]
        out["all_cores_note"] = (f"the full oracle run behind the stored digest, "
                                 f"{rec.get('oracle_threads')} threads, {rec['oracle_seconds']} s")
    return out


def run_batched(args, local, peak, plain_sample: int = 256):
    """The batched workload: 4096 independent jobs (n log-uniform in [64, 2048],
    linkage uniform over the four, R^16 Gaussian mixtures) through one batch
    plan (one persistent launch per size class, work queue, CUDA graph),
    against the same jobs through one lw_cluster call each on one stream
    (timed on a sample).  A sample of the jobs is checked against the oracle."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1709_06816_gb300 import Context, autotune, native

    dev = f"cuda:{local}"
    specs = synth.batch_jobs()
    sizes = [n * (n - 1) // 2 for n, _, _ in specs]
    offs = np.zeros(len(specs) + 1, dtype=np.int64)
    for q, c in enumerate(sizes):
        offs[q + 1] = offs[q] + ((c + 3) // 4) * 4  # 16-byte aligned starts
    pristine = torch.empty(int(offs[-1]), dtype=torch.float32, device=dev)
    for q, spec in enumerate(specs):
        pristine[int(offs[q]):int(offs[q]) + sizes[q]] = synth.job_matrix(spec, q, device=dev)
    work = pristine.clone()
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream=stream)
    mats = [work[int(offs[q]):int(offs[q]) + sizes[q]] for q in range(len(specs))]
    classes = autotune.apply(ctx, local)
    table, outs = ctx.make_jobs(mats, [n for n, _, _ in specs], [l for _, l, _ in specs])
    plan = native.lw_batch_create(ctx.handle, table)
    total_merges = sum(n - 1 for n, _, _ in specs)
    times = []
    try:
        for k in range(args.warmup + args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                work.copy_(pristine)
                e0.record(stream)
            native.lw_batch_run(plan, ctx.handle)
            with torch.cuda.stream(stream):
                e1.record(stream)
            rc = native.lw_batch_wait(plan, table)
            if rc != 0:
                raise RuntimeError(f"batch failed: {native.lw_status_string(rc)}")
            if k >= args.warmup:
                times.append(e0.elapsed_time(e1))
    finally:
        native.lw_batch_destroy(plan)
    batch_ms = statistics.median(times)
    # a sample of the jobs against the oracle
    check = list(range(0, len(specs), 128))
    bad = 0
    for q in check:
        D = pristine[int(offs[q]):int(offs[q]) + sizes[q]].cpu().numpy()
        wm, wh, _, _ = oracle.cached(D, specs[q][0], specs[q][1])
        m, h = outs[q]
        if not (np.array_equal(m.cpu().numpy(), wm)
                and np.array_equal(h.cpu().numpy().view(np.uint32), wh.view(np.uint32))):
            bad += 1
    # plain path: one lw_cluster launch per job, same stream, a sample of the jobs
    pick = list(range(0, len(specs), max(1, len(specs) // plain_sample)))[:plain_sample]
    with torch.cuda.stream(stream):
        work.copy_(pristine)
    torch.cuda.synchronize()
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        pe0.record(stream)
    for q in pick:
        m, h = outs[q]
        ctx.cluster_async(mats[q], specs[q][0], specs[q][1], m, h)
    with torch.cuda.stream(stream):
        pe1.record(stream)
    ctx.wait()
    plain_ms = pe0.elapsed_time(pe1)
    ctx.close()
    jobs_per_s = len(specs) / (batch_ms * 1e-3)
    plain_jobs_per_s = len(pick) / (plain_ms * 1e-3)
    rec = work_counts("batch4096:mixed")
    alg = 0
    for n, link, _ in specs:
        alg += algorithmic_bytes(n, link, {"rescan_cells": 0})[0]
    note = "rescan and row-i terms missing"
    if rec is not None:
        alg += 4 * int(rec["rescan_cells"]) + 4 * int(rec.get("rowi_cells", 0))
        note = "rescan and row-i terms from the oracle's runs of all 4096 jobs"
    achieved = alg / (batch_ms * 1e-3) / 1e9
    return {
        "metric": "jobs/s (4096 independent jobs, n log-uniform in [64,2048], mixed linkage)",
        "value": jobs_per_s, "unit": "jobs/s", "ms_per_batch": batch_ms,
        "merges_per_s": total_merges / (batch_ms * 1e-3), "n_jobs": len(specs),
        "total_merges": total_merges, "matrix_bytes": 4 * int(sum(sizes)),
        "plain_jobs_per_s": plain_jobs_per_s, "plain_sample_jobs": len(pick),
        "speedup_vs_plain": jobs_per_s / plain_jobs_per_s,
        "parity": {"oracle_checked_jobs": len(check), "mismatches": bad},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "algorithmic_bytes": alg, "algorithmic_note": note,
                     "note": "the 4.98 GB of triangles exceed L2 together; each job alone fits L2"},
        "step": "restore all matrices (one device copy) + one batch-plan run (CUDA graph: "
                "per size class, queue reset + persistent CTA-per-job kernel, classes side by side)",
        "classes": classes,
    }


def run_serving(args, local):
    """The serving workload: Poisson streams of clustering requests (n
    log-uniform in [256, 32768], linkage uniform over the four, R^16
    Gaussian-mixture distances) through a server with a 120 GB pool, at
    several offered rates.  Every request has its own matrix (no two share
    one): the requests' matrices are generated on the device before the
    streams run and are the same at every rate (the stream's draws of n,
    linkage and mixture do not depend on the rate, only the gaps do).
    Latency runs from submission (matrix ready) to completion.  The same
    requests are then run one by one through lw_cluster (the plain per-job
    path): their results must match the served ones bit for bit, and their
    total time gives the plain jobs/s."""
    import numpy as np
    import torch

    import synth
    from paper_1709_06816_gb300 import Context
    from paper_1709_06816_gb300.native import Server

    dev = f"cuda:{local}"
    count = args.serve_requests
    specs0 = synth.serve_requests(count, rate=200.0)
    bank = []
    for (_, n, link, K, q) in specs0:
        pts = synth.gmm_points(np.random.default_rng([4, q]), n, 16, K, 10.0, 1.0)
        bank.append(synth.packed_distances(pts, device=dev))
    torch.cuda.synchronize()

    def one_rate(rate):
        specs = synth.serve_requests(count, rate=rate)
        assert [s[1:] for s in specs] == [s[1:] for s in specs0]
        outs = []
        srv = Server(local, budget_bytes=120 * 10**9, lanes=48)
        late = 0
        try:
            t0 = time.perf_counter()
            for q, spec in enumerate(specs):
                wait = spec[0] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                elif wait < -0.002:
                    late += 1
                n, link = spec[1], spec[2]
                m = torch.empty((n - 1, 2), dtype=torch.int32, device=dev)
                h = torch.empty(n - 1, dtype=torch.float32, device=dev)
                outs.append((srv.submit(bank[q], n, link, m, h), m, h))
            rc = srv.drain()
            st = srv.stats()
        finally:
            srv.close()
        merges = sum(s[1] - 1 for s in specs)
        return outs, {
            "offered_rate": count / specs[-1][0], "requests": count, "completed": st["completed"],
            "failed": st["failed"], "jobs_per_s": st["completed"] / st["wall_s"] if st["wall_s"] else None,
            "merges_per_s": merges / st["wall_s"] if st["wall_s"] else None,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "peak_inflight": st["peak_inflight"], "peak_pool_bytes": st["peak_bytes"],
            "arrivals_late": late, "status": rc}

    results = []
    outs = None
    for rate in (25, 50, 100, 200, 400):
        outs, r = one_rate(rate)
        results.append(r)
        torch.cuda.empty_cache()
    # the plain path: the same requests alone, one by one, on one context
    ctx = Context(local)
    plain_ms, same = 0.0, 0
    try:
        for q, (spec, (_, m, h)) in enumerate(zip(specs0, outs)):
            n, link = spec[1], spec[2]
            work = bank[q].clone()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            pm, ph = ctx.cluster(work, n, link)
            e1.record()
            torch.cuda.synchronize()
            plain_ms += e0.elapsed_time(e1)
            same += bool(torch.equal(pm, m) and torch.equal(ph.view(torch.int32), h.view(torch.int32)))
            del work
    finally:
        ctx.close()
    del bank
    plain_jobs_per_s = count / (plain_ms * 1e-3)
    best = max(results, key=lambda r: r["jobs_per_s"] or 0)
    sustained = [r for r in results if r["jobs_per_s"] and r["jobs_per_s"] >= 0.9 * r["offered_rate"]]
    return {
        "metric": "served jobs/s and latency (Poisson arrivals, n log-uniform [256, 32768], mixed linkage)",
        "value": best["jobs_per_s"], "unit": "jobs/s", "rates": results,
        "sustained_rate": max((r["offered_rate"] for r in sustained), default=None),
        "plain_jobs_per_s": plain_jobs_per_s,
        "speedup_vs_plain": best["jobs_per_s"] / plain_jobs_per_s if best["jobs_per_s"] else None,
        "plain_matches_served": same, "plain_checked": count,
        "pool_bytes": 120 * 10**9, "lanes": 48,
        "inputs": f"{count} requests, each with its own matrix, generated on the device before the "
                  "streams; the same requests at every offered rate",
    }


def run_reference(args, world, rank, local):
    """The reference arm: the CPU oracle, each step a bounded sample."""
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import torch

    import oracle
    import synth

    w = synth.workload(args.workload)
    n = w.n
    if not torch.cuda.is_available():
        print(json.dumps({"impl": "reference", "unavailable":
                          "the n=65536 conformer matrix is generated on the GPU; none visible"}))
        return
    D_host = w.matrix(device=f"cuda:{local}").cpu().numpy()
    torch.cuda.empty_cache()
    oracle.build()
    key = f"{args.workload}:{LINKAGE}"
    rates, infos = [], []
    for k in range(args.warmup + args.steps):
        rate, info = oracle_rate(D_host, n, LINKAGE, key, args.ref_step_seconds)
        if k >= args.warmup:
            rates.append(rate)
            infos.append(info)
    value = statistics.median(rates)
    wall_ms = 1e3 * statistics.mean(i["wall_s"] for i in infos)
    sample = ("each step: " + cpu_sample_text(infos[0], n)
              + "; value = median over the steps; ms_per_step = measured wall time of one step")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(n, world),
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle",
                         "cores": infos[0]["cores"], "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_cta_sweep(args, local):
    """Time of one clustering against the number of CTAs (the GPU analogue of
    the paper's running time against processor count, Section 6, Figure 2),
    at the paper's mean problem size n = 1968 (conformer-like chains),
    complete linkage.  Every point is the best of five synchronised
    lw_cluster calls (host wall clock, launch included) and its result is
    compared with the oracle's."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1709_06816_gb300 import Context
    torch.cuda.set_device(local)
    w = synth.workload(f"conformer{args.sweep_n}")
    D = w.matrix()
    want_m, want_h, _, _ = oracle.cached(D, w.n, LINKAGE)
    src = torch.from_numpy(D).to(f"cuda:{local}")
    work = src.clone()
    ctx = Context(local)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    blocks = (w.n + 31) // 32  # a grid holds at most one CTA per 32-row block
    grids = sorted({min(g, sms, blocks) for g in (1, 2, 4, 8, 16, 32, 64, 128, sms)})
    points = []
    for g in grids:
        ctx.set_grid(g)
        best = float("inf")
        for _ in range(5):
            work.copy_(src)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m, h = ctx.cluster(work, w.n, LINKAGE)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        ok = bool(np.array_equal(m.cpu().numpy(), want_m)
                  and np.array_equal(h.cpu().numpy().view(np.uint32), want_h.view(np.uint32)))
        points.append({"ctas_requested": g, "ctas": ctx.stats()["grid"], "ms": best * 1e3,
                       "oracle_match": ok})
    ctx.close()
    return {"experiment": "clustering time vs CTAs (Section 6, Figure 2 analogue)", "n": w.n,
            "linkage": LINK_NAMES[LINKAGE], "data": "synthetic conformer-like chains", "points": points}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target length of the CPU oracle sample")
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    ap.add_argument("--serve-requests", type=int, default=240,
                    help="requests of each offered rate of the serving workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other single-matrix workloads")
    ap.add_argument("--no-sweep", action="store_true", help="skip the CTA-count sweep")
    ap.add_argument("--cta-sweep", action="store_true",
                    help="only the clustering time against the CTA count")
    ap.add_argument("--sweep-n", type=int, default=1968)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic workload name (profiling uses smaller conformer<N> cases)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if args.impl == "ours" else "gloo")
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, local)
        else:
            import __graft_entry__
            if rank == 0 or world == 1:
                __graft_entry__.build()
            barrier(world)
            __graft_entry__.build()
            if args.cta_sweep:
                if rank == 0:
                    print(json.dumps(run_cta_sweep(args, local)), flush=True)
            else:
                run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

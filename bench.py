#!/usr/bin/env python3
"""Benchmark of the Lance-Williams merge loop on GB300.

A step is one whole clustering of the n = 65536 conformer-like matrix
(complete linkage): the persistent kernel validates the 8.59 GB packed
triangle, builds the row minima and performs all 65535 merges (Section 4's
iteration).  The kernel rewrites the matrix in place, so every step first
restores it from a pristine device copy (a device-to-device copy, counted
inside the step).

Printed (rank 0, one JSON line): merges/s over K timed steps (CUDA events on
the library's stream, W untimed warm-up steps), the dendrogram time, the
HBM roofline fraction of the kernel (algorithmic bytes from the kernel's own
counters), the CPU oracle's rate on a bounded sample, an end-to-end rate
through the C ABI with host buffers, and the SM clocks sampled during the
timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle instead (the reference arm): each step
is a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun, N > 1): independent replicas, one per GPU; no
collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
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


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one merge
# kernel launch on the bench workload, from one ncu capture
# (profiles/merge_kernel_conformer65536_dram.md).  It describes the kernel
# code it was taken on (lw_merge.cu and lw_internal.h, comments aside) and is
# reported only while that code is unchanged.
MEASURED_TRAFFIC = {
    "workload": "conformer65536:1",
    "kernel_sha256": "7bb81418a6bf71c046d2c280a2de8faefe851597d7d17e9cb8cb31936261f36e",
    "bytes_per_launch": 370.61e9 + 35.09e9,
}


def kernel_source_sha256() -> str:
    """Hash of the merge kernel's code (the kernel and its constants), with
    // comments and blank space left out: an edit of the text around the code
    keeps a measurement valid, an edit of the code does not."""
    import hashlib
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
    if sha != MEASURED_TRAFFIC["kernel_sha256"] or f"{workload}:{linkage}" != MEASURED_TRAFFIC["workload"]:
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


def work_counts(workload: str, linkage: int):
    """The oracle's exact counters for this workload (bench_work_counts.json,
    written by ``python -m oracle.work_counts``), or None."""
    try:
        with open(os.path.join(ROOT, "bench_work_counts.json")) as f:
            return json.load(f).get(f"{workload}:{linkage}")
    except FileNotFoundError:
        return None


def algorithmic_bytes(n: int, linkage: int, counts) -> tuple:
    """Bytes one clustering must move (per launch):
    init: read the packed triangle once, write n row keys (8 B);
    per merge t with m_t = n - t live clusters: read the m_t row keys (8 B),
    read D(k,i), D(k,j) and write D(k,i+j) for the m_t - 2 other clusters
    (12 B), Ward also reads m_t sizes (4 B), re-read every live cell of each
    row whose cached minimum pointed at i or j and got worse (4 B; the count
    is the oracle's, one cached key per row), and write the step (12 B).
    Returns (bytes, note)."""
    cells = n * (n - 1) // 2
    sum_m = n * (n + 1) // 2 - 1
    updated = (n - 1) * (n - 2) // 2  # sum over merges of m_t - 2
    b = 4 * cells + 8 * n + 8 * sum_m + 12 * updated + 12 * (n - 1)
    if linkage == 3:
        b += 4 * sum_m
    if counts is None:
        return b, "rescan term missing (no oracle counts for this workload)"
    return b + 4 * int(counts["rescan_cells"]), "rescan term from the oracle's full run"


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


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(D_host, n: int, linkage: int, target_s: float = 12.0):
    """Run the oracle (as it stands) on init + the first K merges of the same
    matrix, K chosen from a short calibration so the sample takes about
    target_s seconds.  Returns (merges/s estimate for the whole run, info)."""
    import numpy as np
    import oracle

    work = np.empty_like(D_host)
    np.copyto(work, D_host)
    _, _, st, (t_init, t_loop) = oracle.cached(work, n, linkage, max_merges=50, inplace=True)
    per_merge = t_loop / 50.0
    K = int(max(100, min(n - 1, (target_s - t_init) / max(per_merge, 1e-6))))
    np.copyto(work, D_host)
    _, _, st, (t_init, t_loop) = oracle.cached(work, n, linkage, max_merges=K, inplace=True)
    del work
    # merge t costs about m_t = n - t; scale the sample's loop time by total work
    sum_all = n * (n + 1) / 2 - 1
    sum_k = sum(n - t for t in range(K))
    est_total = t_init + t_loop * sum_all / sum_k
    rate = (n - 1) / est_total
    info = {"K": K, "t_init_s": t_init, "t_loop_s": t_loop, "est_total_s": est_total,
            "cores": oracle.threads()}
    return rate, info


# ---------------------------------------------------------------------------
# arms
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

    def step(ev_pair=None):
        with torch.cuda.stream(stream):
            work.copy_(src)
            if ev_pair is not None:
                ev_pair[0].record(stream)
            ctx.cluster_async(work, n, LINKAGE, m_out, h_out)
            if ev_pair is not None:
                ev_pair[1].record(stream)
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

    # end-to-end through the C ABI with host buffers (pinned input, host outputs)
    e2e = None
    if not args.no_e2e:
        host = torch.empty(src.numel(), dtype=torch.float32, pin_memory=True)
        host.copy_(src)
        hm = np.empty((n - 1, 2), dtype=np.int32)
        hh = np.empty(n - 1, dtype=np.float32)
        ctx2 = Context(local)
        ctx2.cluster(host, n, LINKAGE, hm, hh)  # warm: allocates the device copy
        reps = max(1, min(3, args.steps))
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx2.cluster(host, n, LINKAGE, hm, hh)
        e2e_s = (time.perf_counter() - t0) / reps
        e2e_ok = bool(np.array_equal(hm, ref_m.cpu().numpy()))
        ctx2.close()
        del host
        e2e_s = max_over_ranks(e2e_s, world)
        e2e = {"value": world * (n - 1) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 4 * (n * (n - 1) // 2),
               "d2h_bytes_per_step": 12 * (n - 1) + 16 + 32,
               "seconds_per_step": e2e_s, "matches_device_run": e2e_ok}

    # CPU oracle on a bounded sample of the same matrix (rank 0, N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        D_host = src.cpu().numpy()
        del src
        torch.cuda.empty_cache()
        rate, info = oracle_sample(D_host, n, LINKAGE, target_s=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
               "sample": (f"init + first {info['K']} of {n - 1} merges of the same n={n} matrix on "
                          f"{info['cores']} host threads ({info['t_init_s']:.1f} s init, "
                          f"{info['t_loop_s']:.1f} s merges); full-run time extrapolated by "
                          f"work sum(m_t): {info['est_total_s']:.1f} s")}

    ctx.close()
    del work
    torch.cuda.empty_cache()
    batched = None if args.no_batched else run_batched(args, local)
    torch.cuda.empty_cache()
    serving = None if args.no_serving else run_serving(args, local)
    peak, peak_kind = peaks()
    alg, alg_note = algorithmic_bytes(n, LINKAGE, work_counts(args.workload, LINKAGE))
    k_avg_ms = sum(kernel_ms) / len(kernel_ms)
    achieved = alg / (k_avg_ms * 1e-3) / 1e9
    clocks = clk.summary()
    out = {
        "metric": METRIC,
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
        "config": {"workload": args.workload, "n": n, "linkage": "complete",
                   "matrix_bytes": 4 * (n * (n - 1) // 2),
                   "l2": f"inputs larger than L2 ({4 * (n * (n - 1) // 2) / 1e9:.2f} GB packed triangle)",
                   "step": "restore matrix (device copy) + one lw_cluster launch: validate, "
                           f"row minima, {n - 1} merges",
                   "grid_ctas": stats.get("grid"), "parallelism": f"replicas{world}"},
        "dendrogram_ms": k_avg_ms,
        "kernel_ms": kernel_ms,
        "deterministic_across_steps": deterministic,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(args.workload, LINKAGE),
                     "algorithmic_bytes_per_launch": alg, "algorithmic_note": alg_note,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "counters": stats,
        "batched": batched,
        "serving": serving,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_batched(args, local, plain_sample: int = 256):
    """The batched workload: 4096 independent jobs (n log-uniform in [64, 2048],
    linkage uniform over the four, R^16 Gaussian mixtures) through one batch
    plan (one persistent launch, work queue, CUDA graph), against the same jobs
    through one lw_cluster call each on one stream (timed on a sample)."""
    import numpy as np
    import torch

    import synth
    from paper_1709_06816_gb300 import Context, native

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
    from paper_1709_06816_gb300 import autotune
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
    return {
        "metric": "jobs/s (4096 independent jobs, n log-uniform in [64,2048], mixed linkage)",
        "value": jobs_per_s, "unit": "jobs/s", "ms_per_batch": batch_ms,
        "merges_per_s": total_merges / (batch_ms * 1e-3), "n_jobs": len(specs),
        "total_merges": total_merges, "matrix_bytes": 4 * int(sum(sizes)),
        "plain_jobs_per_s": plain_jobs_per_s, "plain_sample_jobs": len(pick),
        "speedup_vs_plain": jobs_per_s / plain_jobs_per_s,
        "step": "restore all matrices (one device copy) + one batch-plan run (CUDA graph: "
                "per size class, queue reset + persistent CTA-per-job kernel, classes side by side)",
        "classes": classes,
    }


def run_serving(args, local, n_requests: int = 2000, bank_size: int = 48):
    """The serving workload: a Poisson stream (mean 200 requests/s) of
    clustering requests, n log-uniform in [256, 32768], linkage uniform over
    the four, R^16 Gaussian-mixture distances, through a server with a
    120 GB pool.  Matrices come from a bank of bank_size requests of the same
    stream, generated on the device beforehand (request q uses bank entry
    q mod bank_size, with that entry's n); latency runs from submission (the
    matrix is ready on the device) to completion."""
    import time as _time

    import torch

    import synth
    from paper_1709_06816_gb300.native import Server

    dev = f"cuda:{local}"
    stream_specs = synth.serve_requests(n_requests)
    bank = []
    for (_, n, link, K, q) in stream_specs[:bank_size]:
        rng_seed = [4, q]
        pts = synth.gmm_points(__import__("numpy").random.default_rng(rng_seed), n, 16, K, 10.0, 1.0)
        bank.append((synth.packed_distances(pts, device=dev), n, link))
    outs = []
    for q in range(n_requests):
        D, n, link = bank[q % bank_size]
        outs.append((torch.empty((n - 1, 2), dtype=torch.int32, device=dev),
                     torch.empty(n - 1, dtype=torch.float32, device=dev)))
    torch.cuda.synchronize()
    srv = Server(local, budget_bytes=120 * 10**9, lanes=48)
    try:
        t0 = _time.perf_counter()
        for q, (arrival, _, _, _, _) in enumerate(stream_specs):
            wait = arrival - (_time.perf_counter() - t0)
            if wait > 0:
                _time.sleep(wait)
            D, n, link = bank[q % bank_size]
            m, h = outs[q]
            srv.submit(D, n, link, m, h)
        submit_s = _time.perf_counter() - t0
        rc = srv.drain()
        st = srv.stats()
    finally:
        srv.close()
    merges = sum(bank[q % bank_size][1] - 1 for q in range(n_requests))
    return {
        "metric": "served jobs/s and latency (Poisson 200 req/s, n log-uniform [256, 32768])",
        "value": st["completed"] / st["wall_s"] if st["wall_s"] else None, "unit": "jobs/s",
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
        "requests": n_requests, "completed": st["completed"], "failed": st["failed"],
        "offered_rate": n_requests / stream_specs[-1][0], "arrival_span_s": stream_specs[-1][0],
        "submit_span_s": submit_s, "wall_s": st["wall_s"],
        "merges_per_s": merges / st["wall_s"] if st["wall_s"] else None,
        "peak_inflight": st["peak_inflight"], "peak_pool_bytes": st["peak_bytes"],
        "pool_bytes": st["budget_bytes"], "lanes": 48, "status": rc,
        "inputs": f"bank of {bank_size} matrices of the same request stream, generated on the device",
    }


def run_reference(args, world, rank, local):
    """The reference arm: the CPU oracle, each step a bounded sample."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import oracle
    import synth

    w = synth.workload(args.workload)
    n = w.n
    if torch.cuda.is_available():
        D_host = w.matrix(device=f"cuda:{local}").cpu().numpy()
        torch.cuda.empty_cache()
    else:
        print(json.dumps({"impl": "reference", "unavailable":
                          "the n=65536 conformer matrix is generated on the GPU; none visible"}))
        return
    oracle.build()
    rates = []
    infos = []
    for k in range(args.warmup + args.steps):
        rate, info = oracle_sample(D_host, n, LINKAGE, target_s=args.ref_step_seconds)
        if k >= args.warmup:
            rates.append(rate)
            infos.append(info)
    value = statistics.median(rates)
    est = statistics.median(i["est_total_s"] for i in infos)
    sample = (f"each step: init + first ~{infos[0]['K']} of {n - 1} merges of the n={n} matrix on "
              f"{infos[0]['cores']} host threads; full-run time extrapolated by work sum(m_t)")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": est * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "linkage": "complete",
                   "l2": "inputs larger than L2 (8.59 GB packed triangle)",
                   "parallelism": "host cores (OpenMP)"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle",
                         "cores": infos[0]["cores"], "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_cta_sweep(args, local):
    """Time of one clustering against the number of CTAs (the GPU analogue of
    the paper's running time against processor count, Section 6), at the
    paper's mean problem size n = 1968 (conformer-like chains), complete
    linkage.  Prints one JSON line; every point is the best of five runs of
    a synchronised lw_cluster call (host wall clock, launch included)."""
    import torch
    import synth
    from paper_1709_06816_gb300 import Context
    torch.cuda.set_device(local)
    w = synth.workload(f"conformer{args.sweep_n}")
    src = w.matrix(device=f"cuda:{local}")
    work = src.clone()
    ctx = Context(local)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    blocks = (w.n + 31) // 32  # a grid holds at most one CTA per 32-row block
    grids = sorted({min(g, sms, blocks) for g in (1, 2, 4, 8, 16, 32, 64, 128, sms)})
    points = []
    ref = None
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
        got = (m.cpu().numpy().tobytes(), h.cpu().numpy().tobytes())
        ref = ref or got
        points.append({"ctas": ctx.stats()["grid"], "ms": best * 1e3, "same_result": got == ref})
    ctx.close()
    print(json.dumps({"experiment": "clustering time vs CTAs", "n": w.n, "linkage": "complete",
                      "data": "synthetic conformer-like chains", "points": points}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target length of the CPU oracle sample")
    ap.add_argument("--ref-step-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--cta-sweep", action="store_true",
                    help="instead of the benchmark: clustering time against the CTA count")
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
                    run_cta_sweep(args, local)
            else:
                run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Autotuner of the batch path: which CTA size serves which job sizes.

A one-CTA batch job runs on a CTA of 128, 256 or 512 threads.  Smaller CTAs
let several jobs share an SM (registers allow 4, 2 or 1 per SM) but give each
job fewer threads, and the shared memory a job needs grows with n, so the
best choice depends on n and on the device.  ``tune_batch_classes`` measures,
for each size bucket, the merges per second of a full-device batch of
synthetic jobs at every CTA size that fits, keeps the fastest, merges
neighbouring buckets with the same choice into classes and caches the table
per device (``_tune/batch_<device>_<SMs>.json``).  ``apply`` sets the table on a
context (lw_set_batch_classes): a fresh measurement in ``_tune/`` if there is
one, else the table shipped in ``tuned/`` for this device (measured on it by
this module), else it measures.

All timing runs through the library's batch plan; the jobs are seeded
Gaussian-mixture matrices in R^16 (the batched workload's distribution).
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import native

_HERE = os.path.dirname(os.path.abspath(__file__))
BUCKETS = (256, 512, 1024, 2048)
CTA_SIZES = (128, 256, 512)


def _cache_path(torch, device: int, shipped: bool = False) -> str:
    props = torch.cuda.get_device_properties(device)
    name = props.name.replace(" ", "_")
    return os.path.join(_HERE, "tuned" if shipped else "_tune",
                        f"batch_{name}_{props.multi_processor_count}.json")


def _measure(ctx, torch, device, n_lo, n_hi, nt, jobs_per_cta=2, seed=11):
    """Merges/s of one full-device batch of jobs with n in (n_lo, n_hi] on CTAs of nt threads."""
    import synth

    ctx.set_batch_classes([(n_hi, nt)])
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    per_sm = {128: 4, 256: 2, 512: 1}[nt]
    count = sms * per_sm * jobs_per_cta
    rng = np.random.default_rng(seed)
    bank = []
    for q in range(8):
        n = int(rng.integers(max(n_lo, 2) + 1, n_hi + 1))
        pts = synth.gmm_points(np.random.default_rng([seed, q]), n, 16, 8)
        bank.append((synth.packed_distances(pts, device=f"cuda:{device}"), n))
    src = [bank[q % len(bank)] for q in range(count)]
    mats = [D.clone() for D, _ in src]
    table, _ = ctx.make_jobs(mats, [n for _, n in src], [q % 4 for q in range(count)])
    try:
        plan = native.lw_batch_create(ctx.handle, table)
    except native.LwError:
        return None  # this CTA size cannot hold jobs of this size
    try:
        best = None
        for rep in range(3):
            for m, (D, _) in zip(mats, src):
                m.copy_(D)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            native.lw_batch_run(plan, ctx.handle)
            rc = native.lw_batch_wait(plan, table)
            dt = time.perf_counter() - t0
            if rc != 0:
                return None
            best = dt if best is None else min(best, dt)
    finally:
        native.lw_batch_destroy(plan)
    merges = sum(n - 1 for _, n in src)
    return merges / best


def tune_batch_classes(device: int = 0, force: bool = False, verbose: bool = False):
    """The measured class table [(n_hi, cta_threads), ...] for this device."""
    import torch

    path = _cache_path(torch, device)
    if not force:
        for p in (path, _cache_path(torch, device, shipped=True)):
            if os.path.exists(p):
                with open(p) as f:
                    return [tuple(x) for x in json.load(f)["classes"]]
    ctx = native.Context(device)
    choices = []
    report = {}
    try:
        lo = 0
        for hi in BUCKETS:
            rates = {}
            for nt in CTA_SIZES:
                r = _measure(ctx, torch, device, lo, hi, nt)
                if r is not None:
                    rates[nt] = r
            best = max(rates, key=rates.get) if rates else 512
            choices.append((hi, best))
            report[str(hi)] = rates
            if verbose:
                print(f"bucket ({lo}, {hi}]: merges/s by CTA size {rates} -> {best}", flush=True)
            lo = hi
    finally:
        ctx.close()
    classes = []
    for hi, nt in choices:
        if classes and classes[-1][1] == nt:
            classes[-1] = (hi, nt)
        else:
            classes.append((hi, nt))
    # jobs above the last bucket keep the one-CTA default (512 threads)
    if classes[-1][1] != 512:
        classes.append((4096, 512))
    else:
        classes[-1] = (4096, 512)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"classes": classes, "merges_per_s": report,
                   "when": time.strftime("%Y-%m-%dT%H:%M:%S")}, f, indent=1)
    return classes


def apply(ctx, device: int = 0, force: bool = False):
    """Tune (or read the cached table) and set it on ctx; returns the table."""
    classes = tune_batch_classes(device, force)
    ctx.set_batch_classes(classes)
    return classes

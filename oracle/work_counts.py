"""Exact work counters and result digests of the oracle on the benchmark
workloads (test infrastructure).

The benchmark's roofline numerator ("algorithmic bytes") needs, besides
closed-form terms in n, the number of live cells that the row-minimum cache
of the merge loop must re-read: rows whose cached minimum pointed at the
merged pair and got worse.  That count depends on the data, so it is taken
from a full run of this oracle, never from the CUDA path.

The same full run gives the expected result of the whole clustering: the
SHA-256 of the merge list (int32, (n - 1) x 2, row-major, little-endian) and
of the heights (float32, n - 1), plus the SHA-256 of the input matrix (the
packed float32 triangle), so that a GPU run of all n - 1 merges can be
compared with it bit for bit without running the oracle again.

Finally it times ``oracle.sample`` (the bounded prefix the benchmark's CPU
baseline runs) on the same matrix, so the benchmark can calibrate the
prefix's extrapolated time against this full run.

    python -m oracle.work_counts conformer65536:1 [name:linkage ...] [batch4096:mixed]

generates each workload with ``synth`` (on the GPU when torch sees one,
else with numpy), runs ``oracle.cached`` over all merges on the host cores
and writes the record to ``bench_work_counts.json`` at the repository
root, merged with what is already there.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "bench_work_counts.json")
SAMPLE_SECONDS = 15.0


def sha256(a) -> str:
    """SHA-256 of an array's bytes in C order (little-endian on every host here)."""
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def batch_counts(oracle, synth) -> dict:
    """The batched workload (synth.batch_jobs(): 4096 jobs, mixed linkage):
    the oracle's counters summed over every job."""
    t0 = time.time()
    tot = {"jobs": 0, "rescan_cells": 0, "rescans": 0, "rowi_cells": 0, "updated": 0, "sum_m": 0}
    for q, spec in enumerate(synth.batch_jobs()):
        n, link, _ = spec
        _, _, st, _ = oracle.cached(synth.job_matrix(spec, q), n, link, inplace=True)
        tot["jobs"] += 1
        for k in ("rescan_cells", "rescans", "rowi_cells", "updated", "sum_m"):
            tot[k] += st[k]
    tot["oracle_seconds"] = round(time.time() - t0, 1)
    tot["oracle_threads"] = oracle.threads()
    return tot


def main(argv):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np

    import oracle
    import synth

    try:
        with open(OUT) as f:
            table = json.load(f)
    except FileNotFoundError:
        table = {}
    for item in argv:
        name, link = item.split(":")
        if name == "batch4096":
            table[item] = batch_counts(oracle, synth)
            print(item, table[item], flush=True)
            continue
        link = int(link)
        w = synth.workload(name)
        try:
            import torch
            dev = "cuda" if torch.cuda.is_available() else None
        except ImportError:
            dev = None
        D = w.matrix(device=dev)
        if dev is not None:
            D = D.cpu().numpy()
            torch.cuda.empty_cache()
        input_sha = sha256(D)
        smp = oracle.sample(D, w.n, link, target_s=SAMPLE_SECONDS)
        t0 = time.time()
        merges, heights, stats, times = oracle.cached(D, w.n, link, inplace=True)
        full_s = time.time() - t0
        del D
        table[f"{name}:{link}"] = {
            "n": w.n, "linkage": link, "rescans": stats["rescans"],
            "rescan_cells": stats["rescan_cells"], "rowi_cells": stats["rowi_cells"],
            "updated": stats["updated"], "sum_m": stats["sum_m"],
            "oracle_seconds": round(full_s, 1), "oracle_threads": oracle.threads(),
            "input_sha256": input_sha,
            "merges_sha256": sha256(np.asarray(merges, dtype=np.int32)),
            "heights_sha256": sha256(np.asarray(heights, dtype=np.float32)),
            "sample": {"target_s": SAMPLE_SECONDS, "K": smp["K"],
                       "est_total_s": round(smp["est_total_s"], 2),
                       "full_over_est": round(full_s / smp["est_total_s"], 4)},
        }
        print(name, link, table[f"{name}:{link}"], flush=True)
    with open(OUT, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])

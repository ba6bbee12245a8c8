"""Exact work counters of the oracle on the benchmark workloads (test infrastructure).

The benchmark's roofline numerator ("algorithmic bytes") needs, besides
closed-form terms in n, the number of live cells that the row-minimum cache
of the merge loop must re-read: rows whose cached minimum pointed at the
merged pair and got worse.  That count depends on the data, so it is taken
from a full run of this oracle, never from the CUDA path.

    python -m oracle.work_counts conformer65536:1 [name:linkage ...]

generates each workload with ``synth`` (on the GPU when torch sees one,
else with numpy), runs ``oracle.cached`` over all merges on the host cores
and writes the counters to ``bench_work_counts.json`` at the repository
root, merged with what is already there.
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "bench_work_counts.json")


def main(argv):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    import synth

    try:
        with open(OUT) as f:
            table = json.load(f)
    except FileNotFoundError:
        table = {}
    for item in argv:
        name, link = item.split(":")
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
        t0 = time.time()
        _, _, stats, times = oracle.cached(D, w.n, link, inplace=True)
        table[f"{name}:{link}"] = {
            "n": w.n, "linkage": link, "rescans": stats["rescans"],
            "rescan_cells": stats["rescan_cells"], "updated": stats["updated"],
            "sum_m": stats["sum_m"], "oracle_seconds": round(time.time() - t0, 1),
            "oracle_threads": oracle.threads(),
        }
        print(name, link, table[f"{name}:{link}"], flush=True)
        del D
    with open(OUT, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])

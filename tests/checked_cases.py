"""Parity cases run on the bounds-checked library (liblw_checked.so, built
with -DLW_CHECKED): every global load and store of the merge kernel is
checked against the job's buffers, and an access outside them fails the
call with the source line.  Run by tests/test_gpu_checked.py in a child
process with LW_CHECKED=1 (the library is chosen when it is first loaded).
Prints one line per group and "checked ok <count>" at the end.
"""
import hashlib
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_1709_06816_gb300 import Context, native  # noqa: E402


def bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def same(got, want, what):
    gm, gh = got
    if not (np.array_equal(gm, want[0]) and np.array_equal(bits(gh), bits(want[1]))):
        raise AssertionError(f"{what}: differs from the oracle")


def main():
    assert os.environ.get("LW_CHECKED") == "1"
    lib = native.load()
    assert lib._name.endswith("liblw_checked.so"), lib._name
    ctx = Context(0)
    count = 0
    # one CTA and several, both working layouts, all six linkages, ragged sizes
    for s, n in enumerate([3, 33, 257, 1000, 2100]):
        for link in range(6):
            D = synth.small_gmm(n, 700 + s) if (s + link) % 2 else synth.tie_heavy(n, 700 + s, levels=4)
            want = oracle.cached(D, n, link)
            for layout, grid in ((0, 1), (1, 7), (2, 7), (1, 0)):
                ctx.set_layout(layout)
                ctx.set_grid(grid)
                m, h = ctx.cluster(torch.from_numpy(D).cuda(), n, link)
                same((m.cpu().numpy(), h.cpu().numpy()), want, f"n={n} link={link} layout={layout} grid={grid}")
                count += 1
    ctx.set_layout(0)
    ctx.set_grid(0)
    print("single matrices ok", count, flush=True)
    # a pinned host matrix read in place by the layout kernel
    n = 900
    D = synth.small_gmm(n, 77)
    m, h = ctx.cluster(torch.from_numpy(D).pin_memory(), n, 1)
    same((m.numpy(), h.numpy()), oracle.cached(D, n, 1), "pinned host")
    count += 1
    # a batch: one CTA per job, and jobs over the whole device
    ctx.set_batch_split(600)
    rng = np.random.default_rng(5)
    jobs = []
    for q in range(24):
        nq = int(rng.integers(40, 1300))
        jobs.append((synth.small_gmm(nq, 800 + q), nq, q % 6))
    outs, st = ctx.cluster_batch([torch.from_numpy(Dq).cuda() for Dq, _, _ in jobs],
                                 [nq for _, nq, _ in jobs], [lq for _, _, lq in jobs])
    for (Dq, nq, lq), (mq, hq), sq in zip(jobs, outs, st):
        assert sq == 0, sq
        same((mq.cpu().numpy(), hq.cpu().numpy()), oracle.cached(Dq, nq, lq), f"batch n={nq}")
        count += 1
    ctx.set_batch_split(0)
    print("batch ok", flush=True)
    # the entry point without allocation
    n = 3000
    D = synth.small_gmm(n, 91, dim=8, k=7)
    dD = torch.from_numpy(D).cuda()
    mm = torch.empty((n - 1, 2), dtype=torch.int32, device="cuda")
    hh = torch.empty(n - 1, dtype=torch.float32, device="cuda")
    native.lw_cluster_noalloc(dD, n, 2, mm, hh)
    torch.cuda.synchronize()
    same((mm.cpu().numpy(), hh.cpu().numpy()), oracle.cached(D, n, 2), "noalloc")
    count += 1
    # a full-size grid run (n = 16384, every SM) against the oracle's digest
    table = json.load(open(os.path.join(ROOT, "bench_work_counts.json")))
    w = synth.workload("gmm16384q")
    src = w.matrix(device="cuda")
    m, h = ctx.cluster(src.clone(), w.n, 1)
    rec = table["gmm16384q:1"]
    assert hashlib.sha256(np.ascontiguousarray(m.cpu().numpy()).tobytes()).hexdigest() == rec["merges_sha256"]
    assert hashlib.sha256(np.ascontiguousarray(h.cpu().numpy()).tobytes()).hexdigest() == rec["heights_sha256"]
    count += 1
    ctx.close()
    print("checked ok", count, flush=True)


if __name__ == "__main__":
    main()

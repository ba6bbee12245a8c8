"""GPU parity of the batch path (one persistent launch, work queue, CUDA graph).

Every job of a batch must give the oracle's dendrogram bit for bit, whether
it ran on one CTA of the batch kernel or over the whole device.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_06816_gb300 import Context, LwError, native  # noqa: E402


@pytest.fixture()
def ctx():
    c = Context(0)
    yield c
    c.close()


def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def _mixed_jobs(count, seed, n_lo=2, n_hi=700):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        link = int(rng.integers(0, 6))
        D = synth.small_gmm(n, 1000 * seed + q, dim=6, k=5) if q % 3 else synth.tie_heavy(n, q, 6)
        out.append((D, n, link))
    return out


def _check(outs, statuses, jobs):
    for (m, h), st, (D, n, link) in zip(outs, statuses, jobs):
        assert st == 0, st
        wm, wh, _, _ = oracle.cached(D, n, link)
        assert np.array_equal(m.cpu().numpy(), wm), (n, link)
        assert np.array_equal(_bits(h.cpu().numpy()), _bits(wh)), (n, link)


def test_batch_small_jobs_match_oracle(ctx):
    jobs = _mixed_jobs(96, 1)
    mats = [torch.from_numpy(D).cuda() for D, _, _ in jobs]
    outs, st = ctx.cluster_batch(mats, [n for _, n, _ in jobs], [l for _, _, l in jobs])
    torch.cuda.synchronize()
    _check(outs, st, jobs)


def test_batch_with_large_jobs_on_the_grid_path(ctx):
    """Split at n = 300: larger jobs run over the whole device, the rest one per CTA."""
    ctx.set_batch_split(300)
    jobs = _mixed_jobs(24, 2, n_lo=100, n_hi=1500)
    mats = [torch.from_numpy(D).cuda() for D, _, _ in jobs]
    outs, st = ctx.cluster_batch(mats, [n for _, n, _ in jobs], [l for _, _, l in jobs])
    _check(outs, st, jobs)


def test_batch_plan_replays(ctx):
    """One plan (one CUDA graph) run twice on restored inputs gives the same result."""
    jobs = _mixed_jobs(40, 3)
    src = [torch.from_numpy(D).cuda() for D, _, _ in jobs]
    mats = [s.clone() for s in src]
    table, outs = ctx.make_jobs(mats, [n for _, n, _ in jobs], [l for _, _, l in jobs])
    plan = native.lw_batch_create(ctx.handle, table)
    try:
        for rep in range(2):
            for m, s in zip(mats, src):
                m.copy_(s)
            torch.cuda.synchronize()
            native.lw_batch_run(plan, ctx.handle)
            assert native.lw_batch_wait(plan, table) == 0
            _check(outs, [table[q].status for q in range(len(jobs))], jobs)
    finally:
        native.lw_batch_destroy(plan)


def test_batch_reports_bad_job(ctx):
    jobs = _mixed_jobs(10, 4)
    mats = [torch.from_numpy(D).cuda() for D, _, _ in jobs]
    bad = synth.small_gmm(50, 5)
    bad[7] = np.nan
    mats[3] = torch.from_numpy(bad).cuda()
    ns = [n for _, n, _ in jobs]
    ns[3] = 50
    outs, st = ctx.cluster_batch(mats, ns, [l for _, _, l in jobs])
    assert st[3] == 2
    jobs[3] = (bad, 50, jobs[3][2])
    good = [q for q in range(10) if q != 3]
    _check([outs[q] for q in good], [st[q] for q in good], [jobs[q] for q in good])
    # a host pointer in the table is refused before anything runs
    table, _ = ctx.make_jobs(mats[:2], ns[:2], [1, 1])
    table[1].dist = torch.from_numpy(jobs[1][0]).data_ptr()
    with pytest.raises(LwError) as e:
        native.lw_batch_create(ctx.handle, table)
    assert e.value.status == 1 and "job 1" in str(e.value)


def test_batched_workload_sample(ctx):
    """A slice of the 4096-job batched workload (n log-uniform in [64, 2048],
    linkage uniform over the four, R^16 mixtures)."""
    specs = synth.batch_jobs()
    pick = list(range(0, 4096, 64))
    jobs = []
    for q in pick:
        D = synth.job_matrix(specs[q], q)
        jobs.append((D, specs[q][0], specs[q][1]))
    mats = [torch.from_numpy(D).cuda() for D, _, _ in jobs]
    outs, st = ctx.cluster_batch(mats, [n for _, n, _ in jobs], [l for _, _, l in jobs])
    _check(outs, st, jobs)


def test_batch_many_copies_of_a_rescan_heavy_job(ctx):
    """96 copies of one tie-heavy job (many equal cells, frequent refills) in
    one batch: every copy must equal the oracle, every time (a missing
    barrier between a cache write and the scan that reads it shows up as a
    rare wrong merge in such runs)."""
    n, link = 433, 1
    D = synth.tie_heavy(n, 60, 6)
    wm, wh, _, _ = oracle.cached(D, n, link)
    for _ in range(2):
        mats = [torch.from_numpy(D).cuda() for _ in range(96)]
        outs, st = ctx.cluster_batch(mats, [n] * 96, [link] * 96)
        for (m, h), s in zip(outs, st):
            assert s == 0
            assert np.array_equal(m.cpu().numpy(), wm)
            assert np.array_equal(_bits(h.cpu().numpy()), _bits(wh))


def test_batch_size_classes(ctx):
    """Jobs split over three classes of CTA sizes (128, 256, 512 threads), each
    its own persistent launch on a branch of the graph, plus grid-path jobs."""
    ctx.set_batch_classes([(300, 128), (900, 256), (1600, 512)])
    jobs = _mixed_jobs(60, 6, n_lo=2, n_hi=2200)
    mats = [torch.from_numpy(D).cuda() for D, _, _ in jobs]
    outs, st = ctx.cluster_batch(mats, [n for _, n, _ in jobs], [l for _, _, l in jobs])
    _check(outs, st, jobs)
    with pytest.raises(LwError):
        ctx.set_batch_classes([(900, 256), (300, 128)])  # not ascending
    with pytest.raises(LwError):
        ctx.set_batch_classes([(900, 200)])  # not a built CTA size

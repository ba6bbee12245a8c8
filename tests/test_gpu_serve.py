"""GPU tests of the serving loop (continuous batching).

Requests submitted while others are on the GPU are admitted as lanes and pool
memory free up; every result must be the same, bit for bit, as the same
request clustered alone with lw_cluster (and as the oracle)."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_06816_gb300 import Context, LwError  # noqa: E402
from paper_1709_06816_gb300.native import Server  # noqa: E402


def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def _requests(count, seed, n_lo=40, n_hi=3000):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        link = int(rng.integers(0, 4))
        D = synth.small_gmm(n, 7000 + q, dim=8, k=6) if q % 4 else synth.tie_heavy(n, 7000 + q, 6)
        out.append((D, n, link))
    return out


def _alone(D, n, link):
    ctx = Context(0)
    try:
        m, h = ctx.cluster(torch.from_numpy(D).cuda(), n, link)
        return m.cpu().numpy(), h.cpu().numpy()
    finally:
        ctx.close()


def test_results_same_alone_and_in_the_mix():
    reqs = _requests(36, 1)
    # a pool of 24 MB holds only a few of the larger matrices at once
    srv = Server(0, budget_bytes=24 << 20, lanes=8)
    try:
        inputs, outs = [], []
        for q, (D, n, link) in enumerate(reqs):
            if q % 2:  # pinned host input, host outputs
                Dx = torch.from_numpy(D).pin_memory()
                m = np.empty((n - 1, 2), dtype=np.int32)
                h = np.empty(n - 1, dtype=np.float32)
            else:      # device input and outputs
                Dx = torch.from_numpy(D).cuda()
                m = torch.empty((n - 1, 2), dtype=torch.int32, device="cuda")
                h = torch.empty(n - 1, dtype=torch.float32, device="cuda")
            inputs.append(Dx)
            outs.append((m, h))
        torch.cuda.synchronize()
        # a burst: most requests arrive while earlier ones are on the GPU
        tickets = [srv.submit(Dx, n, link, m, h)
                   for Dx, (D, n, link), (m, h) in zip(inputs, reqs, outs)]
        assert srv.drain() == 0
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["peak_bytes"] <= st["budget_bytes"]
        assert st["peak_inflight"] > 1  # requests overlapped on the device
        for q, ((D, n, link), (m, h), t) in enumerate(zip(reqs, outs, tickets)):
            done, status, lat = srv.poll(t)
            assert done and status == 0 and lat > 0
            m = m.cpu().numpy() if hasattr(m, "cpu") else m
            h = h.cpu().numpy() if hasattr(h, "cpu") else h
            am, ah = _alone(D, n, link)
            assert np.array_equal(m, am) and np.array_equal(_bits(h), _bits(ah)), q
            if n <= 900:
                wm, wh, _, _ = oracle.cached(D, n, link)
                assert np.array_equal(m, wm) and np.array_equal(_bits(h), _bits(wh)), q
    finally:
        srv.close()


def test_arrivals_while_busy_and_refusal():
    reqs = _requests(16, 2, n_lo=500, n_hi=2500)
    srv = Server(0, budget_bytes=64 << 20, lanes=4)
    try:
        outs, tickets = [], []
        for q, (D, n, link) in enumerate(reqs):
            Dx = torch.from_numpy(D).cuda()
            m = torch.empty((n - 1, 2), dtype=torch.int32, device="cuda")
            h = torch.empty(n - 1, dtype=torch.float32, device="cuda")
            outs.append((Dx, m, h))
        torch.cuda.synchronize()
        for (Dx, m, h), (D, n, link) in zip(outs, reqs):
            tickets.append(srv.submit(Dx, n, link, m, h))
            time.sleep(0.002)  # staggered arrivals: later requests join a busy server
        assert srv.stats()["peak_inflight"] > 1
        assert srv.drain() == 0
        for (D, n, link), (_, m, h) in zip(reqs, outs):
            am, ah = _alone(D, n, link)
            assert np.array_equal(m.cpu().numpy(), am)
            assert np.array_equal(_bits(h.cpu().numpy()), _bits(ah))
        # a matrix larger than the whole pool can never be admitted
        big = torch.zeros(4, device="cuda")
        with pytest.raises(LwError) as e:
            srv.submit(big, 8000, 1, big, big)  # 128 MB > 64 MB pool
        assert e.value.status == 1
    finally:
        srv.close()


def test_cancel_a_queued_request():
    """A request still in the queue can be withdrawn: it never runs, polls as
    done with LW_ERR_CANCELLED, and the others complete as usual; a request
    that is running (or done) cannot be cancelled."""
    reqs = _requests(12, 3, n_lo=1500, n_hi=2500)
    srv = Server(0, budget_bytes=64 << 20, lanes=1)  # one lane: the rest wait in the queue
    try:
        outs, tickets = [], []
        for D, n, link in reqs:
            Dx = torch.from_numpy(D).cuda()
            m = torch.empty((n - 1, 2), dtype=torch.int32, device="cuda")
            h = torch.empty(n - 1, dtype=torch.float32, device="cuda")
            outs.append((Dx, m, h))
        torch.cuda.synchronize()
        for (Dx, m, h), (D, n, link) in zip(outs, reqs):
            tickets.append(srv.submit(Dx, n, link, m, h))
        cancelled = [t for t in tickets[-4:] if srv.cancel(t) == 0]
        assert len(cancelled) >= 3  # at most the first of them can have started
        assert srv.drain() == 0
        st = srv.stats()
        assert st["cancelled"] == len(cancelled)
        assert st["completed"] == len(reqs) - len(cancelled)
        for t, (D, n, link), (_, m, h) in zip(tickets, reqs, outs):
            done, status, _ = srv.poll(t)
            assert done
            if t in cancelled:
                assert status == 7
                continue
            assert status == 0
            am, ah = _alone(D, n, link)
            assert np.array_equal(m.cpu().numpy(), am)
            assert np.array_equal(_bits(h.cpu().numpy()), _bits(ah))
        assert srv.cancel(tickets[0]) == 6  # finished: nothing to withdraw
        assert srv.cancel(10**9) == 1       # unknown ticket
    finally:
        srv.close()


def test_largest_request_size_matches_the_oracle():
    """One request of the serving stream's largest size (n = 32768, the
    stream's recipe: R^16, 16 Gaussians; group average) through the server,
    next to smaller ones: the whole dendrogram equals the oracle's full run
    (its stored digests, oracle/work_counts.py) bit for bit."""
    import hashlib
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "bench_work_counts.json")) as f:
        rec = json.load(f)["serve32768:2"]
    w = synth.workload("serve32768")
    D = w.matrix(device="cuda")
    assert hashlib.sha256(D.cpu().numpy().tobytes()).hexdigest() == rec["input_sha256"]
    m = torch.empty((w.n - 1, 2), dtype=torch.int32, device="cuda")
    h = torch.empty(w.n - 1, dtype=torch.float32, device="cuda")
    small = _requests(6, 4, n_lo=300, n_hi=3000)
    srv = Server(0, budget_bytes=8 << 30, lanes=8)
    try:
        side = []
        for Ds, n, link in small[:3]:
            Dx = torch.from_numpy(Ds).cuda()
            ms = torch.empty((n - 1, 2), dtype=torch.int32, device="cuda")
            hs = torch.empty(n - 1, dtype=torch.float32, device="cuda")
            side.append((Dx, ms, hs))
        torch.cuda.synchronize()
        for (Dx, ms, hs), (Ds, n, link) in zip(side, small):
            srv.submit(Dx, n, link, ms, hs)
        t = srv.submit(D, w.n, 2, m, h)
        assert srv.drain() == 0
        assert srv.poll(t)[:2] == (True, 0)
    finally:
        srv.close()
    assert hashlib.sha256(m.cpu().numpy().tobytes()).hexdigest() == rec["merges_sha256"]
    assert hashlib.sha256(h.cpu().numpy().tobytes()).hexdigest() == rec["heights_sha256"]

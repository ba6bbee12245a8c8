"""lw_cluster_noalloc: the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc/cudaFree while they cluster (a memory
pool or arena that owns every allocation, a plug-in inside a host
application, a loop that must never enter the allocator).  lw_cluster_noalloc
takes their device buffers and keeps its scratch in a fixed device array of
the library.  This test calls it through the C ABI twice in a row (two sizes,
two linkages: the second call reuses the scratch the first one left behind)
and requires the same dendrogram, bit for bit, as lw_cluster -- the exact
tolerance every parity test here uses.  It runs last so that a failure here
cannot hide an earlier one, and it passes alone in a fresh process too (its
first call then performs the one-time set-up).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1709_06816_gb300 import Context, LwError, native  # noqa: E402


def _with_lw_cluster(D, n, link):
    ctx = Context(0)
    try:
        m, h = ctx.cluster(torch.from_numpy(D).cuda(), n, link)
        torch.cuda.synchronize()
        return m.cpu().numpy(), h.cpu().numpy()
    finally:
        ctx.close()


def _with_noalloc(D, n, link):
    dD = torch.from_numpy(D).cuda()
    m = torch.empty((n - 1, 2), dtype=torch.int32, device="cuda")
    h = torch.empty(n - 1, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    native.lw_cluster_noalloc(dD, n, link, m, h)
    return m.cpu().numpy(), h.cpu().numpy()


def test_noalloc_matches_lw_cluster_twice_in_a_row():
    cases = [(5000, 1, synth.small_gmm(5000, 21, dim=12, k=9)),   # every-SM grid
             (1200, 3, synth.small_gmm(1200, 22, dim=6, k=5))]    # one-CTA grid
    for n, link, D in cases:
        got = _with_noalloc(D, n, link)
        want = _with_lw_cluster(D, n, link)
        assert np.array_equal(got[0], want[0]), (n, link)
        assert np.array_equal(got[1].view(np.uint32), want[1].view(np.uint32)), (n, link)


def test_noalloc_at_its_size_limit_matches_the_oracle():
    """n = LW_NOALLOC_MAX_N (16384, a 512 MB triangle, every-SM grid): the
    whole dendrogram equals the oracle's (its stored digest of the same
    workload) and lw_cluster's, bit for bit."""
    import hashlib
    import json
    import os
    w = synth.workload("gmm16384q")
    assert w.n == native.LW_NOALLOC_MAX_N
    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "bench_work_counts.json")) as f:
        rec = json.load(f)["gmm16384q:1"]
    D = w.matrix(device="cuda")
    keep = D.clone()
    m = torch.empty((w.n - 1, 2), dtype=torch.int32, device="cuda")
    h = torch.empty(w.n - 1, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    native.lw_cluster_noalloc(D, w.n, 1, m, h)
    gm, gh = m.cpu().numpy(), h.cpu().numpy()
    assert hashlib.sha256(gm.tobytes()).hexdigest() == rec["merges_sha256"]
    assert hashlib.sha256(gh.tobytes()).hexdigest() == rec["heights_sha256"]
    ctx = Context(0)
    try:
        wm, wh = ctx.cluster(keep, w.n, 1)
    finally:
        ctx.close()
    assert np.array_equal(gm, wm.cpu().numpy())
    assert np.array_equal(gh.view(np.uint32), wh.cpu().numpy().view(np.uint32))


def test_noalloc_rejects_sizes_beyond_its_limit():
    n = native.LW_NOALLOC_MAX_N + 1
    dD = torch.zeros(8, dtype=torch.float32, device="cuda")
    m = torch.empty((1, 2), dtype=torch.int32, device="cuda")
    h = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(LwError) as e:
        native.lw_cluster_noalloc(dD, n, 1, m, h)
    assert e.value.status == 1

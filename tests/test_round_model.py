"""The round protocol of the merge kernel, modelled on the CPU
(tests/round_model.py), reproduces the oracle's dendrogram bit for bit: the
chain walk, the certification and the refill replay are exact, not merely
close.  A planted mistake (keeping every proposed merge without
certification) must be caught by the same comparison."""
import numpy as np
import pytest

import oracle
import synth
from round_model import RoundModel


def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


CASES = [(n, kind) for n in (2, 5, 33, 70) for kind in ("gmm", "ties")]


@pytest.mark.parametrize("link", range(6))
@pytest.mark.parametrize("G,chain,pub,refill_at", [(1, 16, 16, 0), (3, 32, 4, 0), (3, 32, 4, 2)])
def test_model_matches_oracle(link, G, chain, pub, refill_at):
    for s, (n, kind) in enumerate(CASES):
        D = synth.small_gmm(n, 40 + s) if kind == "gmm" else synth.tie_heavy(n, 40 + s, levels=4)
        wm, wh, _, _ = oracle.cached(D.copy(), n, link)
        m, h, rounds = RoundModel(D.copy(), n, link, G=G, chain=chain, pub=pub, refill_at=refill_at).run()
        assert np.array_equal(m, wm), (n, kind)
        assert np.array_equal(_bits(h), _bits(wh)), (n, kind)
        assert rounds <= max(n - 1, 1) + 64  # rounds certify one merge or more, bar refill waits


def test_rounds_certify_several_merges():
    # (refills asked for at two keys left: the model has no rescans of rows
    # whose cache empties at the front, so emptied caches would idle rounds)
    n = 160
    D = synth.small_gmm(n, 7, dim=8, k=6)
    m, h, rounds = RoundModel(D.copy(), n, 1, G=3, chain=32, pub=4, refill_at=2).run()
    wm, _, _, _ = oracle.cached(D.copy(), n, 1)
    assert np.array_equal(m, wm)
    assert rounds < (n - 1) / 3  # the point of the protocol


def test_uncertified_chain_is_caught():
    """Accepting the whole chain without the certification step must give a
    different dendrogram on some input of the sweep (ties make it likely)."""
    caught = 0
    for s in range(6):
        n = 40
        D = synth.tie_heavy(n, 90 + s, levels=3)
        wm, wh, _, _ = oracle.cached(D.copy(), n, 1)
        try:
            m, h, _ = RoundModel(D.copy(), n, 1, G=2, chain=32, pub=4, certify=False).run()
        except RuntimeError:
            caught += 1
            continue
        if not (np.array_equal(m, wm) and np.array_equal(_bits(h), _bits(wh))):
            caught += 1
    assert caught > 0



@pytest.mark.parametrize("link", [0, 1, 3])
def test_certification_by_scans_decides_the_same(link):
    """The kernel's form of the certification (per merge a, a suffix minimum
    over the later pairs of the cells merge a alone wrote and an exclusive
    prefix minimum over a < c < p of the cells after merges a and c) accepts
    exactly the prefix the direct loops accept, round by round, ties
    included."""
    for s_, n in enumerate((40, 90)):
        for D in (synth.tie_heavy(n, 300 + s_, levels=3), synth.small_gmm(n, 310 + s_)):
            direct = RoundModel(D.copy(), n, link, G=3, chain=32, pub=4, refill_at=2)
            scans = RoundModel(D.copy(), n, link, G=3, chain=32, pub=4, refill_at=2, scan=True)
            m1, h1, _ = direct.run()
            m2, h2, _ = scans.run()
            assert direct.decisions == scans.decisions
            assert np.array_equal(m1, m2) and np.array_equal(_bits(h1), _bits(h2))
            wm, wh, _, _ = oracle.cached(D.copy(), n, link)
            assert np.array_equal(m2, wm) and np.array_equal(_bits(h2), _bits(wh))

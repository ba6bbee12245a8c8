"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test names the passage of the paper (Yarmish, Listowsky, Dexter,
"Distributed Lance-William Clustering Algorithm") or the mathematical fact it
relies on.  Together they are chosen so that a plausible slip in the oracle
-- a wrong coefficient or sign, a dropped term, a swapped operand, a wrong
tie-break, a stale cached row minimum -- fails at least one of them
(``test_planted_mistakes_are_caught`` checks that on purpose-built mutants).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LINK = {"single": 0, "complete": 1, "average": 2, "ward": 3, "weighted": 4, "centroid": 5}
SQUARED = ("ward", "centroid")  # the closed forms hold for squared Euclidean distances


def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Table 1 and the update formula
# --------------------------------------------------------------------------

def test_table1_coefficients_golden():
    """Table 1 evaluated by hand (tests/golden/table1_coefficients.txt)."""
    for row in _read_golden("table1_coefficients.txt"):
        link, ni, nj, nk = LINK[row[0]], int(row[1]), int(row[2]), int(row[3])
        want = [Fraction(x) for x in row[4:8]]
        got = oracle.coefficients(link, ni, nj, nk)
        for g, w in zip(got, want):
            # each coefficient is one correctly rounded FP32 value of the fraction
            assert g == np.float32(float(w)), (row, got)


@pytest.mark.parametrize("seed", range(3))
def test_single_complete_are_min_max_on_grid(seed):
    """On multiples of 1/1024 below 2^12 every FP32 step is exact, so the Table 1
    single row gives min(a, b) and the complete row (Section 5.3 step 6) gives max(a, b)."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 1 << 22, 2000) / 1024.0
    b = rng.integers(0, 1 << 22, 2000) / 1024.0
    h = np.minimum(a, b) * rng.random(2000)
    for x, y, z in zip(a, b, h):
        assert oracle.update(0, x, y, z, 3, 4, 5) == np.float32(min(x, y))
        assert oracle.update(1, x, y, z, 3, 4, 5) == np.float32(max(x, y))


def test_average_is_weighted_mean():
    """Group average: the new distance is the size-weighted mean (exact here)."""
    # ni = nj: coefficients 1/2, exact on the grid
    for a, b in [(1.0, 3.0), (0.5, 0.25), (1024.0, 2.0)]:
        assert oracle.update(2, a, b, 0.0, 5, 5, 1) == np.float32((a + b) / 2)
    # ni = 3, nj = 1: 3/4 and 1/4 are exact
    assert oracle.update(2, 4.0, 8.0, 1.0, 3, 1, 9) == np.float32(5.0)


def test_ward_update_matches_centroid_form():
    """Ward row of Table 1 on squared Euclidean distances reproduces
    2 nA nB/(nA+nB) ||cA - cB||^2 (checked in exact rationals at small sizes)."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        ni, nj, nk = (int(x) for x in rng.integers(1, 6, 3))
        # clusters on a line with integer centroids: exact arithmetic
        ci, cj, ck = (int(x) for x in rng.integers(-20, 20, 3))

        def wd(na, ca, nb, cb):
            return Fraction(2 * na * nb, na + nb) * (ca - cb) ** 2

        dki, dkj, dij = wd(nk, ck, ni, ci), wd(nk, ck, nj, cj), wd(ni, ci, nj, cj)
        T = ni + nj + nk
        lw = (Fraction(ni + nk, T) * dki + Fraction(nj + nk, T) * dkj - Fraction(nk, T) * dij)
        cij = Fraction(ni * ci + nj * cj, ni + nj)
        assert lw == wd(nk, ck, ni + nj, cij)
        got = oracle.update(3, float(dki), float(dkj), float(dij), ni, nj, nk)
        # FP32 error bound: inputs and coefficients rounded once, three products
        # and three sums rounded; relative to the magnitude of the terms
        mag = float(Fraction(ni + nk, T) * dki + Fraction(nj + nk, T) * dkj + Fraction(nk, T) * dij)
        assert abs(float(got) - float(lw)) <= 10 * 2.0 ** -24 * mag


def test_weighted_average_is_midpoint():
    """Weighted average (Table 1): the new distance is (D(k,i) + D(k,j)) / 2
    whatever the sizes -- exact on the dyadic grid."""
    rng = np.random.default_rng(3)
    a = rng.integers(0, 1 << 22, 500) / 1024.0
    b = rng.integers(0, 1 << 22, 500) / 1024.0
    for x, y in zip(a, b):
        ni, nj, nk = (int(v) for v in rng.integers(1, 50, 3))
        assert oracle.update(4, x, y, min(x, y), ni, nj, nk) == np.float32((x + y) / 2)


def test_centroid_update_matches_centroid_form():
    """Centroid row of Table 1 on squared Euclidean distances gives the squared
    distance between the merged cluster's centroid and the other one's
    (checked in exact rationals on a line with integer centroids), and the
    FP32 result stays within the rounding bound of that value."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        ni, nj, nk = (int(x) for x in rng.integers(1, 7, 3))
        ci, cj, ck = (int(x) for x in rng.integers(-20, 20, 3))
        dki, dkj, dij = Fraction((ck - ci) ** 2), Fraction((ck - cj) ** 2), Fraction((ci - cj) ** 2)
        s = ni + nj
        lw = Fraction(ni, s) * dki + Fraction(nj, s) * dkj - Fraction(ni * nj, s * s) * dij
        cij = Fraction(ni * ci + nj * cj, s)
        assert lw == (ck - cij) ** 2
        got = oracle.update(5, float(dki), float(dkj), float(dij), ni, nj, nk)
        mag = float(Fraction(ni, s) * dki + Fraction(nj, s) * dkj + Fraction(ni * nj, s * s) * dij)
        assert abs(float(got) - float(lw)) <= 10 * 2.0 ** -24 * mag


def test_centroid_clustering_matches_centroids():
    """Centroid linkage of points (squared Euclidean input) merges the pair of
    clusters with the nearest centroids, at their squared centroid distance,
    until FP32 rounding can reorder a near-tie."""
    for seed in range(3):
        p = np.random.default_rng(20 + seed).normal(size=(32, 3)) * 4
        iu = np.triu_indices(32, 1)
        D = ((p[iu[0]] - p[iu[1]]) ** 2).sum(axis=1).astype(np.float32)
        m, h, _, _ = oracle.cached(D, 32, 5)
        bm, bh, gaps = brute.member_linkage(brute.unpack(D, 32), "centroid", points=p)
        for t in range(31):
            assert (m[t] == bm[t]).all(), (seed, t)
            assert abs(float(h[t]) - bh[t]) <= 1e-4 * bh[t] + 1e-5, (seed, t)
            if gaps[t] <= 1e-3 * bh[t]:
                break


def test_weighted_heights_lie_between_member_extremes():
    """A weighted-average height is a weighted mean of member distances: at
    every merge it lies between the closest and the furthest member pair of
    the two clusters (brute force over members)."""
    n = 40
    D = synth.small_gmm(n, 9, dim=4, k=5)
    M = brute.unpack(D, n).astype(np.float64)
    m, h, _, _ = oracle.cached(D, n, 4)
    members = {s: [s] for s in range(n)}
    for t in range(n - 1):
        i, j = int(m[t, 0]), int(m[t, 1])
        block = M[np.ix_(members[i], members[j])]
        tol = 8 * 2.0 ** -24 * block.max()
        assert block.min() - tol <= float(h[t]) <= block.max() + tol, t
        members[i] = members[i] + members.pop(j)


# --------------------------------------------------------------------------
# worked examples and the paper's counts
# --------------------------------------------------------------------------

def test_line4_worked_dendrograms():
    rows = _read_golden("line4_dendrograms.txt")
    pts = [float(x) for x in rows[0][1:]]
    n = len(pts)
    want = {}
    for r in rows[1:]:
        want.setdefault(r[0], []).append((int(r[2]), int(r[3]), Fraction(r[4])))
    for name, steps in want.items():
        iu = np.triu_indices(n, 1)
        d = np.array([abs(pts[a] - pts[b]) for a, b in zip(*iu)])
        if name in SQUARED:
            d = d ** 2
        m, h, _ = oracle.naive(d.astype(np.float32), n, LINK[name])
        for t, (i, j, hv) in enumerate(steps):
            assert (m[t, 0], m[t, 1]) == (i, j), name
            assert abs(float(h[t]) - float(hv)) <= 2.0 ** -20 * float(hv), (name, t)


def test_section5_counts():
    """Section 5.2: n = 8 keeps 28 cells, 4 per processor for p = 7; Section 5.4: the
    search of an iteration with m live clusters reads (m^2 - m)/2 cells."""
    (n, p, cells, per), = [[int(x) for x in r] for r in _read_golden("section5_partition.txt")]
    assert synth.packed_size(n) == cells and cells // p == per and cells % p == 0
    for link in range(6):
        _, _, scanned = oracle.naive(synth.small_gmm(40, 3), 40, link)
        m = 40 - np.arange(39)
        assert (scanned == (m * m - m) // 2).all()


def test_tiny_cases():
    assert oracle.naive(np.zeros(0, np.float32), 1, 1)[0].shape == (0, 2)
    m, h, _ = oracle.naive(np.array([2.5], np.float32), 2, 0)
    assert m.tolist() == [[0, 1]] and h.tolist() == [2.5]
    for link in range(6):
        # all distances equal: ties resolve to (0,1) then (0,2)
        m, h, _ = oracle.naive(np.ones(3, np.float32), 3, link)
        assert m.tolist() == [[0, 1], [0, 2]]
        m2, h2, _, _ = oracle.cached(np.ones(3, np.float32), 3, link)
        assert m2.tolist() == [[0, 1], [0, 2]]


def test_figure1_single_vs_complete():
    """Section 2.1 / Figure 1: single linkage joins the two elongated groups through
    their closest ends; complete linkage joins the compact group to the nearer one."""
    red = [0.0, 2.0, 4.0, 6.0]
    yellow = [9.0, 11.0, 13.0, 15.0]
    blue = [22.0, 23.0]
    pts = red + yellow + blue
    group = [0] * 4 + [1] * 4 + [2] * 2
    n = len(pts)
    iu = np.triu_indices(n, 1)
    d = np.array([abs(pts[a] - pts[b]) for a, b in zip(*iu)], dtype=np.float32)

    def third_last_join(link):
        m, _, _ = oracle.naive(d, n, link)
        members = {s: {s} for s in range(n)}
        for t in range(n - 3):
            members[m[t, 0]] |= members.pop(m[t, 1])
        assert sorted(sorted({group[x] for x in g}) for g in members.values()) == [[0], [1], [2]]
        i, j = m[n - 3]
        return sorted({group[x] for x in members[i]} | {group[x] for x in members[j]})

    assert third_last_join(0) == [0, 1]   # red + yellow
    assert third_last_join(1) == [1, 2]   # yellow + blue


# --------------------------------------------------------------------------
# closed forms and brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_single_linkage_is_prim_mst(seed):
    """Section 2.1: single linkage follows Prim's minimum spanning tree.  On the
    dyadic grid heights are the MST weights and every level's partition is
    the components of the graph of edges <= h."""
    n = 60
    pts = np.random.default_rng(seed).normal(size=(n, 3)) * 40
    D = brute.dyadic_from_points(pts)
    m, h, _, _ = oracle.cached(D, n, 0)
    M = brute.unpack(D, n)
    assert np.array_equal(np.sort(h.astype(np.float64)), np.sort(brute.prim_mst_weights(M)))
    iu = np.triu_indices(n, 1)
    for hv, part in brute.partitions_by_height(n, m, h).items():
        sel = M[iu] <= hv
        assert part == brute.components(n, zip(iu[0][sel], iu[1][sel]))


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("name", ["single", "complete"])
def test_member_brute_force_exact_on_grid(seed, name):
    """Closest / furthest members (Section 2.1) recomputed from scratch: identical merge
    sequence and heights, ties included (tie-heavy integer grid)."""
    n = 36
    for D in (brute.dyadic_matrix(n, seed), synth.tie_heavy(n, seed, levels=5)):
        m, h, _, _ = oracle.cached(D, n, LINK[name])
        bm, bh, _ = brute.member_linkage(brute.unpack(D, n), name)
        assert np.array_equal(m, bm)
        assert np.array_equal(h.astype(np.float64), bh)


@pytest.mark.parametrize("seed", range(4))
def test_average_matches_member_mean(seed):
    """Group average equals the mean over member pairs (float64 brute force) up to
    FP32 rounding; merges agree while the brute-force gap exceeds the error."""
    n = 48
    D = synth.small_gmm(n, seed, dim=4, k=5)
    m, h, _, _ = oracle.cached(D, n, 2)
    bm, bh, gaps = brute.member_linkage(brute.unpack(D, n), "average")
    for t in range(n - 1):
        assert abs(float(h[t]) - bh[t]) <= 1e-5 * bh[t] + 1e-6
        assert (m[t] == bm[t]).all()
        if gaps[t] <= 1e-4 * bh[t]:
            break


@pytest.mark.parametrize("seed", range(4))
def test_ward_matches_centroid_brute_force(seed):
    """Ward on squared Euclidean distances equals 2 nA nB/(nA+nB) ||cA - cB||^2."""
    n = 40
    pts = np.random.default_rng(seed).normal(size=(n, 3)) * 5
    iu = np.triu_indices(n, 1)
    D = ((pts[iu[0]] - pts[iu[1]]) ** 2).sum(axis=1).astype(np.float32)
    m, h, _, _ = oracle.cached(D, n, 3)
    bm, bh, gaps = brute.member_linkage(brute.unpack(D, n), "ward", points=pts)
    for t in range(n - 1):
        assert abs(float(h[t]) - bh[t]) <= 1e-4 * bh[t] + 1e-5
        assert (m[t] == bm[t]).all()
        if gaps[t] <= 1e-3 * bh[t]:
            break


# --------------------------------------------------------------------------
# invariants and the cache
# --------------------------------------------------------------------------

@pytest.mark.parametrize("link", range(6))
@pytest.mark.parametrize("kind", ["gmm", "ties"])
def test_naive_equals_cached(link, kind):
    """The row-minimum cache changes nothing: bit-identical to the full search."""
    for n, seed in [(2, 0), (5, 1), (33, 2), (130, 3), (300, 4)]:
        D = synth.small_gmm(n, seed) if kind == "gmm" else synth.tie_heavy(n, seed)
        a = oracle.naive(D, n, link)
        b = oracle.cached(D, n, link)
        assert np.array_equal(a[0], b[0])
        assert np.array_equal(_bits(a[1]), _bits(b[1]))


@pytest.mark.parametrize("link", range(6))
def test_structural_invariants(link):
    n = 200
    D = synth.small_gmm(n, 11, dim=6, k=6)
    m, h, stats, _ = oracle.cached(D, n, link)
    assert (m[:, 0] < m[:, 1]).all()
    retired = set()
    sizes = {s: 1 for s in range(n)}
    for i, j in m:
        assert i not in retired and j not in retired
        retired.add(j)
        sizes[i] += sizes.pop(j)
    assert list(sizes) == [0] and sizes[0] == n
    # monotone heights: exact for single/complete; a few ulps for average,
    # Ward and weighted average; centroid linkage may invert (Table 1 note)
    if link in (0, 1):
        assert (np.diff(h) >= 0).all()
    elif link != 5:
        assert (h[1:] >= h[:-1] * (1 - 4 * 2.0 ** -24)).all()
    if link in (0, 1):
        C = brute.cophenetic(n, m, h.astype(np.float64))
        # ultrametric: C[x,z] <= max(C[x,y], C[y,z]) for all triples
        for y in range(n):
            assert (C <= np.maximum(C[:, y][:, None], C[y, :][None, :]) + 0).all()
    assert stats["merges"] == n - 1 and stats["updated"] == sum(n - t - 2 for t in range(n - 1))


def test_validation():
    D = synth.small_gmm(10, 0)
    for bad in (np.nan, np.inf, -1.0, -1e-30):
        E = D.copy()
        E[7] = bad
        with pytest.raises(oracle.OracleError):
            oracle.naive(E, 10, 1)
        with pytest.raises(oracle.OracleError):
            oracle.cached(E, 10, 1)
    E = D.copy()
    E[3] = -0.0
    F = D.copy()
    F[3] = 0.0
    a, b = oracle.cached(E, 10, 1), oracle.cached(F, 10, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(_bits(a[1]), _bits(b[1]))


def test_max_merges_prefix():
    n = 120
    D = synth.small_gmm(n, 5)
    full = oracle.cached(D, n, 1)
    part = oracle.cached(D, n, 1, max_merges=30)
    assert np.array_equal(full[0][:30], part[0]) and np.array_equal(_bits(full[1][:30]), _bits(part[1]))


# --------------------------------------------------------------------------
# planted mistakes: every mutant of the oracle must fail some pin
# --------------------------------------------------------------------------

MUTANTS = {
    "single gamma sign": ("ai = 0.5f; aj = 0.5f; b = 0.0f; g = -0.5f;",
                          "ai = 0.5f; aj = 0.5f; b = 0.0f; g = 0.5f;"),
    "complete drops |a-b| term": ("ai = 0.5f; aj = 0.5f; b = 0.0f; g = 0.5f;",
                                  "ai = 0.5f; aj = 0.5f; b = 0.0f; g = 0.0f;"),
    "average swaps sizes": ("case LWO_AVERAGE: {\n        float sum = (float)(ni + nj);\n        ai = (float)ni / sum;",
                            "case LWO_AVERAGE: {\n        float sum = (float)(ni + nj);\n        ai = (float)nj / sum;"),
    "ward beta sign": ("b = -((float)nk / T);", "b = ((float)nk / T);"),
    "ward alpha_i uses n_j": ("ai = (float)(ni + nk) / T;", "ai = (float)(ni + nj) / T;"),
    "centroid beta sign": ("b = -((float)(ni * nj) / (float)((ni + nj) * (ni + nj)));",
                           "b = ((float)(ni * nj) / (float)((ni + nj) * (ni + nj)));"),
    "weighted uses group-average weights": ("ai = 0.5f; aj = 0.5f;\n        break;\n    case LWO_CENTROID",
                                            "ai = (float)ni / (float)(ni + nj); aj = (float)nj / (float)(ni + nj);\n        break;\n    case LWO_CENTROID"),
    "formula drops beta term": ("s = s + co[2] * dij;", "s = s + 0.0f * dij;"),
    "naive tie-break last": ("if (i < 0 || v < h) {", "if (i < 0 || v <= h) {"),
    "swapped operands": ("D[pi] = lw_formula(co, D[pi], D[pair_index(n, k, j)], h);",
                         "D[pi] = lw_formula(co, D[pair_index(n, k, j)], D[pi], h);"),
    "cache keeps a worse minimum": ("if (nk <= old)\n                        rowkey[k] = nk;",
                                    "if (1)\n                        rowkey[k] = nk;"),
    "cache skips new row i": ("rowkey[i] = row_minimum(D, n, active, i, &cnt);",
                              "(void)cnt;"),
    "cache ignores retired arg": ("if ((rowkey[k] & 0xffffffffu) == (uint64_t)j)\n                    rescan[k] = 1;",
                                  "if (0)\n                    rescan[k] = 1;"),
}


def _pins_pass(lib) -> bool:
    """A compact run of the pins above against one compiled oracle copy."""
    try:
        # worked example (both loops)
        pts = [0.0, 1.0, 3.0, 7.0]
        iu = np.triu_indices(4, 1)
        d = np.array([abs(pts[a] - pts[b]) for a, b in zip(*iu)])
        rows = _read_golden("line4_dendrograms.txt")[1:]
        for r in rows:
            link = LINK[r[0]]
            dd = (d ** 2 if r[0] in SQUARED else d).astype(np.float32)
            for res in (lib.naive(dd, 4, link), lib.cached(dd, 4, link)):
                t = int(r[1])
                if (res[0][t, 0], res[0][t, 1]) != (int(r[2]), int(r[3])):
                    return False
                if abs(float(res[1][t]) - float(Fraction(r[4]))) > 2.0 ** -20 * float(Fraction(r[4])):
                    return False
        # member brute force on the tie-heavy grid, both loops
        for name in ("single", "complete"):
            for D in (brute.dyadic_matrix(30, 1), synth.tie_heavy(30, 2, levels=5)):
                bm, bh, _ = brute.member_linkage(brute.unpack(D, 30), name)
                for res in (lib.naive(D, 30, LINK[name]), lib.cached(D, 30, LINK[name])):
                    if not (np.array_equal(res[0], bm) and np.array_equal(res[1].astype(np.float64), bh)):
                        return False
        # naive vs cached on all linkages
        for link in range(6):
            for D in (synth.small_gmm(90, 3), synth.tie_heavy(90, 4)):
                a, b = lib.naive(D, 90, link), lib.cached(D, 90, link)
                if not (np.array_equal(a[0], b[0]) and np.array_equal(_bits(a[1]), _bits(b[1]))):
                    return False
        # average and Ward against their member / centroid forms
        D = synth.small_gmm(40, 1, dim=4, k=5)
        m, h, _, _ = lib.cached(D, 40, 2)
        bm, bh, gaps = brute.member_linkage(brute.unpack(D, 40), "average")
        for t in range(39):
            if abs(float(h[t]) - bh[t]) > 1e-5 * bh[t] + 1e-6 or not (m[t] == bm[t]).all():
                return False
            if gaps[t] <= 1e-4 * bh[t]:
                break
        p = np.random.default_rng(1).normal(size=(30, 3)) * 5
        iu = np.triu_indices(30, 1)
        D = ((p[iu[0]] - p[iu[1]]) ** 2).sum(axis=1).astype(np.float32)
        for name in ("ward", "centroid"):
            m, h, _, _ = lib.cached(D, 30, LINK[name])
            bm, bh, gaps = brute.member_linkage(brute.unpack(D, 30), name, points=p)
            for t in range(29):
                if abs(float(h[t]) - bh[t]) > 1e-4 * bh[t] + 1e-5 or not (m[t] == bm[t]).all():
                    return False
                if gaps[t] <= 1e-3 * bh[t]:
                    break
    except oracle.OracleError:
        return False
    return True


def test_pins_pass_on_the_real_oracle(tmp_path):
    src = open(oracle._SRC).read()
    (tmp_path / "o.c").write_text(src)
    lib = oracle.OracleLib(oracle.build(True, str(tmp_path / "o.c"), str(tmp_path / "o.so")))
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, name
    (tmp_path / "m.c").write_text(src.replace(old, new))
    lib = oracle.OracleLib(oracle.build(True, str(tmp_path / "m.c"), str(tmp_path / "m.so")))
    assert not _pins_pass(lib), f"mutant '{name}' passed every pin"

"""Host-side dendrogram helpers: SciPy-style linkage matrix and tree cuts.

The merge lists come from the oracle (the same contract as the library's
output); SciPy's hierarchy module, an independent implementation of the same
linkages, must give the same tree: the same merges in the same order and the
same heights (Ward and centroid: SciPy reports the square roots of the
heights the Lance-Williams update gives on squared Euclidean input)."""
import numpy as np
import pytest

import oracle
from paper_1709_06816_gb300 import dendrogram

hierarchy = pytest.importorskip("scipy.cluster.hierarchy")
spatial = pytest.importorskip("scipy.spatial.distance")

METHODS = {"single": 0, "complete": 1, "average": 2, "weighted": 4, "ward": 3, "centroid": 5}


@pytest.mark.parametrize("method", sorted(METHODS))
def test_linkage_matrix_matches_scipy(method):
    for seed in range(3):
        p = np.random.default_rng(seed).normal(size=(40, 3))
        d = spatial.pdist(p)                      # packed upper triangle, row-major
        squared = method in ("ward", "centroid")
        D = (d ** 2 if squared else d).astype(np.float32)
        m, h, _, _ = oracle.cached(D, 40, METHODS[method])
        Z = dendrogram.to_linkage_matrix(m, h, 40)
        Zs = hierarchy.linkage(d, method=method)
        heights = np.sqrt(Z[:, 2]) if squared else Z[:, 2]
        assert np.array_equal(Z[:, :2], np.sort(Zs[:, :2], axis=1)), (method, seed)
        assert np.allclose(heights, Zs[:, 2], rtol=1e-5, atol=1e-6), (method, seed)
        assert np.array_equal(Z[:, 3], Zs[:, 3])


def test_cuts_on_the_worked_line():
    # objects at 0, 1, 3, 7, single linkage: merges (0,1)@1, (0,2)@2, (0,3)@4
    m = np.array([[0, 1], [0, 2], [0, 3]])
    h = np.array([1.0, 2.0, 4.0])
    assert dendrogram.cut(m, 4, 4).tolist() == [0, 1, 2, 3]
    assert dendrogram.cut(m, 4, 3).tolist() == [0, 0, 1, 2]
    assert dendrogram.cut(m, 4, 1).tolist() == [0, 0, 0, 0]
    assert dendrogram.cut_height(m, h, 4, 2.5).tolist() == [0, 0, 0, 1]
    assert dendrogram.cut_height(m, h, 4, 0.5).tolist() == [0, 1, 2, 3]
    Z = dendrogram.to_linkage_matrix(m, h, 4)
    assert Z.tolist() == [[0, 1, 1.0, 2], [2, 4, 2.0, 3], [3, 5, 4.0, 4]]


def test_cut_matches_scipy_fcluster():
    p = np.random.default_rng(5).normal(size=(60, 2))
    d = spatial.pdist(p)
    m, h, _, _ = oracle.cached(d.astype(np.float32), 60, 1)
    Zs = hierarchy.linkage(d, method="complete")
    for k in (1, 2, 5, 17, 60):
        ours = dendrogram.cut(m, 60, k)
        theirs = hierarchy.fcluster(Zs, k, criterion="maxclust")
        # same partition (labels may differ): a bijection between label sets
        pairs = set(zip(ours.tolist(), theirs.tolist()))
        assert len(pairs) == len(set(ours.tolist())) == len(set(theirs.tolist())) == k


def test_bad_arguments():
    with pytest.raises(ValueError):
        dendrogram.cut(np.zeros((2, 2)), 4, 2)
    with pytest.raises(ValueError):
        dendrogram.cut(np.array([[0, 1]]), 2, 3)

"""Invariants and library special cases that pin the FP64 oracle.

Each check follows from the paper's definitions or reduces the method to a
library routine; none restates the oracle's own code.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial.distance import cdist

from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic


@pytest.fixture(scope="module")
def tiny():
    return synthetic.make_workload(synthetic.TINY)


@pytest.fixture(scope="module")
def tiny_run(tiny):
    return o.rerank(tiny.xq, tiny.xg, k1=26, k2=7, layers=2, mode="sparse")


def _csr(m):
    return m.tocsr() if sp.issparse(m) else sp.csr_matrix(m)


def test_knn_matches_library_cosine_ranking(tiny):
    # Eq. 7-8 with S from scipy's cosine distance and a stable sort on it.
    xu = np.concatenate([tiny.xq, tiny.xg]).astype(np.float64)
    d = cdist(xu, xu, "cosine")
    np.fill_diagonal(d, -1.0)  # self first (S_ii := 1 is the row maximum)
    want = np.argsort(d, axis=1, kind="stable")[:, :26]
    idx, score = o.knn_lists(xu, 26)
    assert (idx == want).all()
    np.testing.assert_allclose(score[:, 1:], 1.0 - np.take_along_axis(d, want, 1)[:, 1:], atol=1e-12)


def test_degree_and_symmetry(tiny_run):
    r = tiny_run
    n = r.knn_idx.shape[0]
    assert (r.knn_idx[:, 0] == np.arange(n)).all()           # self is rank 1
    assert all(len(set(row)) == 26 for row in r.knn_idx)      # out-degree exactly k1
    a = _csr(r.a_star)
    assert abs(a - a.T).max() == 0                           # A* symmetric (Eq. 9)
    assert set(np.unique(a.data)) <= {0.5, 1.0}              # values of Eq. 10
    assert (a.diagonal() == 1.0).all()
    nbr = [set(row) for row in r.knn_idx]
    coo = a.tocoo()
    for i, j, v in zip(coo.row, coo.col, coo.data):
        recip = (j in nbr[i]) and (i in nbr[j])
        assert (v == 1.0) == recip
        assert (j in nbr[i]) or (i in nbr[j])


def test_features_normalised_and_supports(tiny_run):
    r = tiny_run
    for lvl in (1, 2):
        h = _csr(r.h[lvl])
        nrm = np.sqrt(np.asarray(h.multiply(h).sum(axis=1)).ravel())
        np.testing.assert_allclose(nrm, 1.0, atol=1e-14)
        assert h.data.min() > 0
        prev = _csr(r.h[lvl - 1])
        for i in range(0, h.shape[0], 37):
            want = set()
            for j in r.knn_idx[i, :7]:
                want |= set(prev.indices[prev.indptr[j]:prev.indptr[j + 1]])
            got = set(h.indices[h.indptr[i]:h.indptr[i + 1]])
            assert got == want   # support of h^(l+1)_i = union over N(i, k2)


def test_final_scores_range_and_zero_iff_disjoint(tiny_run):
    r = tiny_run
    assert r.s.min() >= 0.0 and r.s.max() <= 1.0 + 1e-15
    h = _csr(r.h[2])
    q = r.s.shape[0]
    sup = (h > 0).astype(np.int32)
    overlap = (sup[:q] @ sup[q:].T).toarray()
    assert ((r.s == 0.0) == (overlap == 0)).all()
    # the zero tail is in ascending gallery index
    for i in range(q):
        z = r.idx[i][r.dist[i] == 1.0]
        assert (np.diff(z) > 0).all()


def test_scaling_rows_changes_nothing(tiny, tiny_run):
    rng = np.random.default_rng(0)
    fq = rng.uniform(0.25, 4.0, size=(len(tiny.xq), 1)).astype(np.float32)
    fg = rng.uniform(0.25, 4.0, size=(len(tiny.xg), 1)).astype(np.float32)
    r2 = o.rerank(tiny.xq * fq, tiny.xg * fg, k1=26, k2=7, layers=2, mode="sparse")
    assert (r2.knn_idx == tiny_run.knn_idx).all()
    np.testing.assert_allclose(r2.s, tiny_run.s, atol=1e-6)


def test_gallery_permutation_permutes_output(tiny, tiny_run):
    perm = np.random.default_rng(1).permutation(len(tiny.xg))
    r2 = o.rerank(tiny.xq, tiny.xg[perm], k1=26, k2=7, layers=2, mode="sparse")
    np.testing.assert_allclose(r2.s, tiny_run.s[:, perm], atol=1e-12)


def test_k2_one_makes_layers_idle(tiny):
    # N(i, 1) = {i}: each layer maps h_i to normalise(2 h_i), the same direction.
    outs = [o.rerank(tiny.xq, tiny.xg, k1=26, k2=1, layers=L, mode="sparse") for L in (0, 1, 3)]
    for r in outs[1:]:
        np.testing.assert_allclose(r.s, outs[0].s, atol=1e-14)
        # same order, except that mathematically equal scores may round apart
        ref = np.take_along_axis(outs[0].s, outs[0].idx, 1)
        got = np.take_along_axis(outs[0].s, r.idx, 1)
        assert np.abs(got - ref).max() < 1e-14


def test_original_features_without_layers_give_initial_ranking(tiny):
    # Table 1, first column equals the baseline: x_i features, no propagation.
    r = o.rerank(tiny.xq, tiny.xg, k1=26, k2=7, layers=0, feature="x")
    d = cdist(tiny.xq.astype(np.float64), tiny.xg.astype(np.float64), "cosine")
    assert (r.idx == np.argsort(d, axis=1, kind="stable")).all()
    np.testing.assert_allclose(r.dist, np.sort(d, axis=1), atol=1e-12)


def test_mean_aggregator_alpha_zero_is_query_expansion(tiny):
    # Sec. 3.4: one layer, alpha = 0, mean aggregator.  The aggregate is Eq. 4's
    # average over N(i, k2); Eq. 13 adds the residual h_i on top of it.
    r = o.rerank(tiny.xq, tiny.xg, k1=26, k2=5, layers=1, alpha=0.0, aggregator="mean", feature="x")
    xu = np.concatenate([tiny.xq, tiny.xg]).astype(np.float64)
    xh = xu / np.linalg.norm(xu, axis=1, keepdims=True)
    d = cdist(xu, xu, "cosine")
    np.fill_diagonal(d, -1.0)
    nbr = np.argsort(d, axis=1, kind="stable")[:, :5]
    aqe = xh[nbr].mean(axis=1)                      # Eq. 4
    want = xh + aqe
    want /= np.linalg.norm(want, axis=1, keepdims=True)
    np.testing.assert_allclose(r.h[1], want, atol=1e-14)


def test_many_layers_settle(tiny):
    # Table 2: with more layers the features over-smooth and the ranking settles.
    s = {L: o.rerank(tiny.xq, tiny.xg, k1=26, k2=7, layers=L, mode="sparse").s for L in (1, 2, 64, 65)}
    assert np.abs(s[65] - s[64]).max() < 0.1 * np.abs(s[2] - s[1]).max()


def test_dense_and_sparse_modes_agree(tiny, tiny_run):
    r = o.rerank(tiny.xq, tiny.xg, k1=26, k2=7, layers=2, mode="dense")
    assert (r.knn_idx == tiny_run.knn_idx).all()
    np.testing.assert_allclose(r.h[2], tiny_run.h[2].toarray(), atol=1e-12)
    np.testing.assert_allclose(r.s, tiny_run.s, atol=1e-12)
    assert (r.idx == tiny_run.idx).all()

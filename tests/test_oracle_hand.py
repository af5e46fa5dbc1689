"""Hand-worked 6-vertex example of Eq. 7-14 and Algorithm 1, pinned on the oracle.

Vertices are 2-D integer vectors whose unit directions have rational
coordinates (Pythagorean triples), at angles 0, 28.07, 36.87, 67.38, 90 and
112.62 degrees: two arcs.  Vertex 0 is the only query.  k1 = 3, k2 = 2,
alpha = 2, sum aggregator, one layer.  Every number below was worked by hand
from the equations; none comes from running code.

S (cosines of angle differences, Eq. 7):
  S01=15/17 S02=4/5 S03=5/13 S04=0 S05=-5/13 S12=84/85 S13=171/221 S14=8/17
  S15=21/221 S23=56/65 S24=3/5 S25=16/65 S34=12/13 S35=119/169 S45=12/13
Row 4 ties S43 = S45 = 12/13 exactly (p4 = (0, 1) makes both dot products the
same floating-point operation), so the lower index 3 ranks first.
"""
from fractions import Fraction as F
import math

import numpy as np
import pytest

from oracle import rerank_oracle as o

X = np.array([[1, 0], [15, 8], [4, 3], [5, 12], [0, 1], [-5, 12]], dtype=np.float32)

# N(i, 3), sorted by (S desc, index asc), self first (Eq. 8).
KNN3 = [[0, 1, 2], [1, 2, 0], [2, 1, 3], [3, 4, 2], [4, 3, 5], [5, 4, 3]]
KNN3_S = [[F(1), F(15, 17), F(4, 5)], [F(1), F(84, 85), F(15, 17)], [F(1), F(84, 85), F(56, 65)],
          [F(1), F(12, 13), F(56, 65)], [F(1), F(12, 13), F(12, 13)], [F(1), F(12, 13), F(119, 169)]]
H = F(1, 2)
# A* = (A + A^T)/2 (Eq. 9): 1 for reciprocal pairs, 1/2 for one-way (Eq. 10).
A_STAR = [[1, 1, H, 0, 0, 0],
          [1, 1, 1, 0, 0, 0],
          [H, 1, 1, 1, 0, 0],
          [0, 0, 1, 1, 1, H],
          [0, 0, 0, 1, 1, 1],
          [0, 0, 0, H, 1, 1]]
RECIPROCAL = {(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)}
ONE_WAY = {(0, 2), (3, 5)}
# Layer 1 before normalisation: h_i + sum_{j in N(i,2)} S_ij^2 h_j = 2 h_i + S^2 h_nbr,
# written as integer numerators over the denominators 289, 7225, 7225, 169, 169, 169.
H1_NUM = [[803, 803, 514, 0, 0, 0],
          [17978, 21506, 21506, 7056, 0, 0],
          [14281, 21506, 21506, 14450, 0, 0],
          [0, 0, 338, 482, 482, 313],
          [0, 0, 144, 482, 482, 410],
          [0, 0, 0, 313, 482, 482]]
# Final cosines of query 0 against gallery rows 0..4 (vertices 1..5): integer
# dot products and squared norms of the numerators above.
DOT0 = [42759736, 39791045, 173732, 74016, 0]
NORM2 = [1553814, 1298011692, 1337765533, 676861, 653484, 562617]


@pytest.fixture(scope="module", params=["dense", "sparse"])
def res(request):
    return o.rerank(X[:1], X[1:], k1=3, k2=2, layers=1, mode=request.param)


def _dense(m):
    return m.toarray() if hasattr(m, "toarray") else np.asarray(m)


def test_neighbour_lists(res):
    assert res.knn_idx.tolist() == KNN3
    # reading: S_ii := 1 exactly, not the rounded x_i . x_i
    assert (res.knn_score[:, 0] == 1.0).all()
    np.testing.assert_allclose(res.knn_score, np.array(KNN3_S, dtype=float), rtol=0, atol=1e-15)


def test_symmetric_adjacency(res):
    a = _dense(res.a_star)
    assert a.tolist() == np.array(A_STAR, dtype=float).tolist()
    for i in range(6):
        for j in range(6):
            if i == j:
                continue
            p = (min(i, j), max(i, j))
            want = 1.0 if p in RECIPROCAL else 0.5 if p in ONE_WAY else 0.0
            assert a[i, j] == want


def test_initial_features_are_astar_rows(res):
    assert _dense(res.h[0]).tolist() == np.array(A_STAR, dtype=float).tolist()


def test_layer_one(res):
    u = np.array(H1_NUM, dtype=float)
    want = u / np.sqrt(np.array(NORM2, dtype=float))[:, None]
    np.testing.assert_allclose(_dense(res.h[1]), want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(_dense(res.h[1]), axis=1), 1.0, atol=1e-15)


def test_final_ranking(res):
    s = [DOT0[g] / math.sqrt(NORM2[0] * NORM2[g + 1]) for g in range(5)]
    assert res.idx.tolist() == [[0, 1, 2, 3, 4]]
    np.testing.assert_allclose(res.dist[0], 1.0 - np.array(s), rtol=0, atol=1e-15)
    assert res.dist[0, 4] == 1.0  # disjoint supports give exactly s = 0


def test_zero_layers_rank_by_astar_cosine():
    r = o.rerank(X[:1], X[1:], k1=3, k2=2, layers=0)
    # h0 = (1, 1, 1/2, 0, 0, 0): dots 5/2, 2, 1/2, 0, 0; |h0|^2 = 9/4;
    # |A*_1|^2 = 3, |A*_2|^2 = 13/4, |A*_3|^2 = 13/4.
    s = [2.5 / math.sqrt(2.25 * 3.0), 2.0 / math.sqrt(2.25 * 3.25), 0.5 / math.sqrt(2.25 * 3.25), 0.0, 0.0]
    assert r.idx.tolist() == [[0, 1, 2, 3, 4]]
    np.testing.assert_allclose(r.dist[0], 1.0 - np.array(s), atol=1e-15)


def test_k1_rule():
    # Eq. 15: k1 = floor(n / C); Market-1501 test set: 23,100 images over 750 ids.
    assert o.k1_from_classes(23100, 750) == 30
    assert o.k1_from_classes(6, 2) == 3

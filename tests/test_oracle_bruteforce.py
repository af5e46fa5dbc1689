"""Brute force on tiny graphs, in exact arithmetic, against the FP64 oracle.

An independent pure-Python restatement of Eq. 7-14 and Algorithm 1: vertices
are small integer vectors; every comparison of S values is exact (the sign
and the rational square dot^2 / (|x_i|^2 |x_j|^2) decide it), A, A* and the
alpha in {0, 2} edge weights are exact fractions, and the vertex features are
carried in 60-digit decimals.  Instances whose top-(k1+1) lists hold exact or
near ties are redrawn (an FP64 program may order those either way), and tie
breaking is pinned separately on bitwise-identical duplicates.
"""
from decimal import Decimal, getcontext
from fractions import Fraction
from functools import cmp_to_key
import random

import numpy as np
import pytest

from oracle import rerank_oracle as o

getcontext().prec = 60


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


class Exact:
    """Algorithm 1 with exact phase 1 and 60-digit features."""

    def __init__(self, x, k1, k2, alpha, aggregator, feature):
        n = len(x)
        self.n = n
        nn = [_dot(v, v) for v in x]
        g = [[_dot(x[i], x[j]) for j in range(n)] for i in range(n)]

        def s_key(i, j):  # S_ij as (sign, S^2); S_ii := 1
            if i == j:
                return 1, Fraction(1)
            d = g[i][j]
            return (d > 0) - (d < 0), Fraction(d * d, nn[i] * nn[j])

        def s_cmp(a, b):  # -1 if a ranks before b: S desc, then S^2, then value sign
            if a[0] != b[0]:
                return -1 if a[0] > b[0] else 1
            if a[1] == b[1]:
                return 0
            bigger = a[1] > b[1]
            return (-1 if bigger else 1) if a[0] > 0 else (1 if bigger else -1)

        self.s_key, self.s_cmp = s_key, s_cmp
        self.order = []
        for i in range(n):
            def cmp(j1, j2, i=i):
                c = s_cmp(s_key(i, j1), s_key(i, j2))
                return c if c else (j1 > j2) - (j1 < j2)
            self.order.append(sorted(range(n), key=cmp_to_key(cmp)))
        self.knn = [row[:k1] for row in self.order]
        a = [[Fraction(0)] * n for _ in range(n)]
        for i in range(n):
            for j in self.knn[i]:
                a[i][j] = Fraction(1)
        self.a = a
        self.a_star = [[(a[i][j] + a[j][i]) / 2 for j in range(n)] for i in range(n)]
        # e_ij^alpha for alpha in {0, 2}: S^2 is exact, S^0 = 1.
        self.w = [[(s_key(i, j)[1] if alpha == 2 else Fraction(1)) for j in self.knn[i][:k2]]
                  for i in range(n)]
        if aggregator == "mean":
            self.w = [[v / k2 for v in row] for row in self.w]
        if feature == "astar":
            h = [[Decimal(v.numerator) / Decimal(v.denominator) for v in row] for row in self.a_star]
        elif feature == "a":
            h = [[Decimal(v.numerator) for v in row] for row in a]
        else:
            h = [[Decimal(c) / Decimal(nn[i]).sqrt() for c in x[i]] for i in range(n)]
        self.h = [h]
        self.k2, self.aggregator = k2, aggregator

    def layer(self):
        h = self.h[-1]
        out = []
        for i in range(self.n):
            js = self.knn[i][:self.k2]
            ws = [Decimal(v.numerator) / Decimal(v.denominator) for v in self.w[i]]
            if self.aggregator == "max":
                agg = [max(w * h[j][c] for w, j in zip(ws, js)) for c in range(len(h[i]))]
            else:
                agg = [sum(w * h[j][c] for w, j in zip(ws, js)) for c in range(len(h[i]))]
            v = [h[i][c] + agg[c] for c in range(len(h[i]))]
            nrm = sum(t * t for t in v).sqrt()
            out.append([t / nrm for t in v])
        self.h.append(out)

    def ranking(self, q, layers):
        h = self.h[layers]
        nrm = [sum(t * t for t in row).sqrt() for row in h]
        res = []
        for i in range(q):
            s = [sum(a * b for a, b in zip(h[i], h[g])) / (nrm[i] * nrm[g]) for g in range(q, self.n)]
            res.append(s)
        return res


def _clean_instance(ex, k1):
    """True when no row holds an exact or near tie within its top-(k1+1)."""
    for i in range(ex.n):
        row = ex.order[i][:k1 + 1]
        for a, b in zip(row, row[1:]):
            ka, kb = ex.s_key(i, a), ex.s_key(i, b)
            if ex.s_cmp(ka, kb) == 0:
                return False
            va = ka[0] * float(ka[1]) ** 0.5
            vb = kb[0] * float(kb[1]) ** 0.5
            if abs(va - vb) < 1e-9:
                return False
    return True


def _cases(count, seed):
    rnd = random.Random(seed)
    out = []
    while len(out) < count:
        n = rnd.randint(4, 11)
        d = rnd.randint(2, 4)
        x = []
        while len(x) < n:
            v = [rnd.randint(-4, 4) for _ in range(d)]
            if any(v):
                x.append(v)
        k1 = rnd.randint(1, n)
        k2 = rnd.randint(1, k1)
        layers = rnd.randint(0, 3)
        q = rnd.randint(1, n - 1)
        alpha = rnd.choice([0, 2])
        agg = rnd.choice(["sum", "sum", "mean", "max"])
        feat = rnd.choice(["astar", "astar", "a", "x"])
        ex = Exact(x, k1, k2, alpha, agg, feat)
        if not _clean_instance(ex, k1):
            continue
        out.append((x, q, k1, k2, layers, alpha, agg, feat, ex))
    return out


CASES = _cases(40, seed=2012_07620)


def _dense(m):
    return m.toarray() if hasattr(m, "toarray") else np.asarray(m)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("mode", ["dense", "sparse"])
def test_oracle_matches_exact_brute_force(case, mode):
    x, q, k1, k2, layers, alpha, agg, feat, ex = CASES[case]
    xf = np.array(x, dtype=np.float32)
    r = o.rerank(xf[:q], xf[q:], k1=k1, k2=k2, layers=layers, alpha=alpha, aggregator=agg,
                 feature=feat, mode=mode)
    assert r.knn_idx.tolist() == ex.knn
    a_star = [[float(v) for v in row] for row in ex.a_star]
    assert _dense(r.a_star).tolist() == a_star
    while len(ex.h) < layers + 1:
        ex.layer()
    for lvl in range(layers + 1):
        want = np.array([[float(v) for v in row] for row in ex.h[lvl]])
        np.testing.assert_allclose(_dense(r.h[lvl]), want, rtol=0, atol=1e-13)
    exact_s = ex.ranking(q, layers)
    s = np.array([[float(v) for v in row] for row in exact_s])
    np.testing.assert_allclose(r.s, s, rtol=0, atol=1e-13)
    for i in range(q):
        # the exact order: s desc, gallery index asc; values within 1e-12 count as tied
        srt = sorted(range(len(s[i])), key=lambda g: (-exact_s[i][g], g))
        got = r.idx[i].tolist()
        for p, (a, b) in enumerate(zip(got, srt)):
            if a != b:
                assert abs(s[i][a] - s[i][b]) < 1e-12, (i, p)


def test_duplicate_vectors_tie_to_lower_index():
    # Vertices 1, 3 and 4 are the same vector, so row 0 sees three bitwise-equal
    # S values; N(0, 3) = {0, 1, 3} keeps the lower indices, and vertex 3's own
    # list starts with vertex 1 (S_31 = 1 = S_33, lower index first).
    x = np.array([[3, 4], [4, 3], [0, 5], [4, 3], [4, 3], [5, 0]], dtype=np.float32)
    r = o.rerank(x[:2], x[2:], k1=3, k2=2, layers=1)
    assert r.knn_idx[0].tolist() == [0, 1, 3]
    assert r.knn_idx[3].tolist()[:3] == [1, 3, 4]
    assert r.knn_idx[4].tolist()[:3] == [1, 3, 4]


def test_many_equal_scores_keep_index_order():
    # 200 copies of one direction interleaved with 99 vectors orthogonal to
    # vertex 0: every copy scores the same against vertex 0, so N(0, 150) is
    # vertex 0 followed by the 149 lowest-indexed copies, in index order.
    x = np.zeros((300, 3), dtype=np.float32)
    x[0] = [1, 0, 0]
    copies = [i for i in range(1, 300) if i % 3 != 0]
    others = [i for i in range(1, 300) if i % 3 == 0]
    x[copies] = [3, 4, 0]
    x[others, 2] = 1 + np.arange(len(others)) % 5
    x[others, 1] = np.arange(len(others)) % 4
    r = o.rerank(x[:1], x[1:], k1=150, k2=3, layers=1, mode="sparse")
    assert r.knn_idx[0].tolist() == [0] + copies[:149]

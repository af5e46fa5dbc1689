"""The FP64 oracle's Algorithm 1 on full-size instances, for the tests.

``rerank_sparse`` composes the oracle's own step functions in the order of
``oracle.rerank_oracle.rerank`` (sparse mode, sum aggregator, A* features).
The only difference is scheduling: the row-independent steps, the per-row
sorts of Eq. 8 and of the final ranking (Alg. 1 step 7), run on blocks of
rows in a thread pool.  NumPy's sorts release the GIL, so the blocks sort in
parallel.  Each block goes through the same oracle function that the
sequential path applies to all rows, and a row's result does not depend on
the other rows, so the output equals ``rerank(..., mode="sparse")`` element
for element (checked on the CPU by ``tests/test_oracle_parallel.py``).
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np
import scipy.sparse as sp

from oracle import rerank_oracle as o


def _workers(workers):
    return workers or max(1, min(32, os.cpu_count() or 1))


def _blocks(n, parts):
    step = max(1, -(-n // parts))
    return [(a, min(n, a + step)) for a in range(0, n, step)]


def knn_lists(xu, k, workers=None):
    """``o.knn_lists(xu, k)``: S rows by the oracle's similarity_rows, one BLAS
    product per chunk of 1,024 rows as the oracle chunks them (the same
    products, so the same rounding), then the sorted top-k of each block of
    those rows by its top_k_rows, blocks sorted concurrently."""
    chunk = 1024
    wk = _workers(workers)
    xh = o.unit_rows(xu)
    n = xh.shape[0]
    idx = np.empty((n, k), dtype=np.int64)
    score = np.empty((n, k), dtype=np.float64)
    with cf.ThreadPoolExecutor(wk) as ex:
        for a in range(0, n, chunk):
            rows = np.arange(a, min(n, a + chunk))
            s = o.similarity_rows(xh, rows)

            def one(bounds, s=s, a=a):
                lo, hi = bounds
                top = o.top_k_rows(s[lo:hi], k)
                idx[a + lo:a + hi] = top
                score[a + lo:a + hi] = np.take_along_axis(s[lo:hi], top, axis=1)

            list(ex.map(one, _blocks(len(rows), wk)))
    return idx, score


def final_ranking(h, n_query, workers=None):
    """``o.final_ranking(h, n_query)`` on blocks of queries: block [a, b) is the
    oracle's final_ranking of the stacked rows (h_a .. h_b-1, gallery rows)."""
    h = h.tocsr()
    g = h.shape[0] - n_query
    hg = h[n_query:]
    idx = np.empty((n_query, g), dtype=np.int64)
    dist = np.empty((n_query, g), dtype=np.float64)
    s = np.empty((n_query, g), dtype=np.float64)

    def one(bounds):
        lo, hi = bounds
        bi, bd, bs = o.final_ranking(sp.vstack([h[lo:hi], hg]).tocsr(), hi - lo)
        idx[lo:hi], dist[lo:hi], s[lo:hi] = bi, bd, bs

    with cf.ThreadPoolExecutor(_workers(workers)) as ex:
        list(ex.map(one, _blocks(n_query, 4 * _workers(workers))))
    return idx, dist, s


def rerank_sparse(xq, xg, k1, k2, layers, alpha=2.0, workers=None) -> o.OracleResult:
    """Algorithm 1 (sum aggregator, A* features) in the oracle's sparse mode."""
    xu = np.concatenate([np.asarray(xq, np.float64), np.asarray(xg, np.float64)])
    n, q = xu.shape[0], len(xq)
    knn_idx, knn_score = knn_lists(xu, k1, workers)                      # Eq. 7, 8
    a = o.adjacency(knn_idx, n, False)                                     # Eq. 8
    a_star = o.symmetric_adjacency(a)                                      # Eq. 9, 10
    w = o.knn_graph_weights(knn_idx, knn_score, k2, alpha, "sum", n, False)  # Eq. 12, 14
    hs = [a_star]                                                          # Eq. 11
    for _ in range(layers):                                                # Eq. 13, 14
        hs.append(o.propagate(hs[-1], w, knn_idx, k2, "sum"))
    idx, dist, s = final_ranking(hs[-1], q, workers)                       # Alg. 1 step 7
    return o.OracleResult(knn_idx, knn_score, a_star, hs, idx, dist, s, None)

"""FP64 CPU oracle of GNN-based re-ranking -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and its ``--impl reference`` arm) may import this module.  The
product path never calls it: the CUDA library has no CPU fallback.

It restates Sec. 3.3 ("GNN-based Re-Ranking") and Algorithm 1 of Zhang et
al., "Understanding Image Retrieval Re-Ranking: A Graph Neural Network
Perspective" (arXiv 2012.07620) in plain NumPy/SciPy, in float64, step by
step in the paper's order:

  Alg. 1 step 1   S_ij = cos(x_i, x_j) over X_u = X_q u X_g         (Eq. 7)
  Alg. 1 step 2   A_ij = 1 iff j in N(i, k1), top-k1 of row i of S   (Eq. 8)
  Alg. 1 step 3   A* = (A + A^T) / 2                                 (Eq. 9, 10)
  Alg. 1 step 4   h_i = row i of A*, e_ij = S_ij, j in N(i, k2)      (Eq. 11, 12)
  Alg. 1 step 5   k-NN graph on the top-k2 edges                     (Eq. 12)
  Alg. 1 step 6   h_i <- h_i + aggregate{ e_ij^alpha h_j }, then
                  L2-normalise every h_i                              (Eq. 13, 14)
  Alg. 1 step 7   rank the gallery by cos(h_q, h_g) for each query    (Sec. 3.3)

Library primitives (matrix products, sparse products, stable sorts) serve as
single steps; nothing is blocked, fused or reordered beyond chunking the rows
of S so that an N x N matrix need not be held at once.

Readings of points the paper leaves open:
  * self is a candidate of its own neighbourhood and S_ii := 1 exactly, so
    vertex i is first in N(i, k);
  * ties in every ordering (neighbour lists, final ranking) go to the lower
    index; the union index puts queries first, then the gallery;
  * N(i, k2) is the first k2 entries of the sorted N(i, k1) list (self
    included), the same graph in every layer;
  * h^(0) = A*_i is not normalised before the first layer; normalisation
    follows every propagation;
  * "mean" divides the aggregated sum by k2; "max" is the element-wise max;
  * the final similarity is the cosine over the n-dimensional features of
    query rows against gallery rows; the returned distance is 1 - s.

Two modes compute the same quantities: ``dense`` builds literal N x N
matrices (small N only), ``sparse`` keeps A*, the k-NN graph and h as SciPy
CSR matrices.  They agree to rounding.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Optional

import numpy as np
import scipy.sparse as sp

__all__ = [
    "unit_rows", "similarity_rows", "top_k_rows", "knn_lists", "adjacency", "symmetric_adjacency",
    "knn_graph_weights", "propagate", "final_ranking", "OracleResult", "rerank", "k1_from_classes",
]

AGGREGATORS = ("sum", "mean", "max")
FEATURES = ("astar", "a", "x")


def unit_rows(x: np.ndarray) -> np.ndarray:
    """x_i / ||x_i||_2 in float64, the normalisation inside cos (Eq. 7)."""
    x = np.asarray(x, dtype=np.float64)
    return x / np.sqrt((x * x).sum(axis=1))[:, None]


def similarity_rows(xu_hat: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Rows ``rows`` of S = cos(x_i, x_j) (Eq. 7), with S_ii := 1 exactly."""
    s = xu_hat[rows] @ xu_hat.T
    s[np.arange(len(rows)), rows] = 1.0
    return s


def top_k_rows(s_rows: np.ndarray, k: int) -> np.ndarray:
    """N(i, k): the k largest entries of each row, by (S desc, index asc) (Eq. 8)."""
    order = np.argsort(-s_rows, axis=1, kind="stable")
    return order[:, :k]


def knn_lists(xu: np.ndarray, k: int, rows: Optional[np.ndarray] = None,
              chunk: int = 1024) -> tuple[np.ndarray, np.ndarray]:
    """Sorted top-k neighbour lists and their S values for the given rows.

    Returns ``idx`` (len(rows), k) int64 and ``score`` (len(rows), k) float64.
    """
    xh = unit_rows(xu)
    n = xh.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = np.empty((len(rows), k), dtype=np.int64)
    score = np.empty((len(rows), k), dtype=np.float64)
    for a in range(0, len(rows), chunk):
        r = rows[a:a + chunk]
        s = similarity_rows(xh, r)
        top = top_k_rows(s, k)
        idx[a:a + chunk] = top
        score[a:a + chunk] = np.take_along_axis(s, top, axis=1)
    return idx, score


def adjacency(knn_idx: np.ndarray, n: int, dense: bool):
    """A_ij = 1 if j in N(i, k1), else 0 (Eq. 8)."""
    k1 = knn_idx.shape[1]
    if dense:
        a = np.zeros((n, n), dtype=np.float64)
        a[np.repeat(np.arange(n), k1), knn_idx.ravel()] = 1.0
        return a
    return sp.csr_matrix((np.ones(n * k1), (np.repeat(np.arange(n), k1), knn_idx.ravel())), shape=(n, n))


def symmetric_adjacency(a):
    """A* = (A + A^T) / 2 (Eq. 9); entries are 1, 1/2 or 0 as Eq. 10 lists."""
    if sp.issparse(a):
        return ((a + a.T) * 0.5).tocsr()
    return (a + a.T) / 2.0


def knn_graph_weights(knn_idx: np.ndarray, knn_score: np.ndarray, k2: int, alpha: float,
                      aggregator: str, n: int, dense: bool):
    """Message weights f(e_ij) = e_ij^alpha with e_ij = S_ij for j in N(i, k2)
    (Eq. 12, Eq. 14) as an N x N matrix W; "mean" folds in the 1/k2."""
    cols = knn_idx[:, :k2]
    w = knn_score[:, :k2] ** alpha
    if aggregator == "mean":
        w = w / k2
    rows = np.repeat(np.arange(n), k2)
    if dense:
        m = np.zeros((n, n), dtype=np.float64)
        m[rows, cols.ravel()] = w.ravel()
        return m
    return sp.csr_matrix((w.ravel(), (rows, cols.ravel())), shape=(n, n))


def _normalise(h):
    """Divide every row by its L2 norm (Sec. 3.3, after every propagation)."""
    if sp.issparse(h):
        nrm = np.sqrt(np.asarray(h.multiply(h).sum(axis=1)).ravel())
        return sp.diags(1.0 / nrm) @ h
    return h / np.sqrt((h * h).sum(axis=1))[:, None]


def propagate(h, w, knn_idx: np.ndarray, k2: int, aggregator: str):
    """One layer of Eq. 13/14 followed by L2 normalisation.

    sum / mean:  h_i + sum_j W_ij h_j  (W already holds e^alpha, and 1/k2 for mean)
    max:         h_i + max_j (W_ij h_j), element-wise over j in N(i, k2)
    """
    if aggregator in ("sum", "mean"):
        return _normalise(h + w @ h)
    dense_h = h.toarray() if sp.issparse(h) else h
    wd = w.toarray() if sp.issparse(w) else w
    n = dense_h.shape[0]
    agg = np.empty_like(dense_h)
    for i in range(n):
        js = knn_idx[i, :k2]
        agg[i] = (wd[i, js][:, None] * dense_h[js]).max(axis=0)
    out = _normalise(dense_h + agg)
    return sp.csr_matrix(out) if sp.issparse(h) else out


def final_ranking(h, n_query: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """cos(h_q, h_g) for every query row against every gallery row, each list
    sorted by (s desc, gallery index asc) (Alg. 1 step 7).

    Returns ``idx`` (Q, G) gallery indices, ``dist`` (Q, G) = 1 - s in that
    order, and the unsorted score matrix ``s`` (Q, G).
    """
    if sp.issparse(h):
        h = h.tocsr()
        nrm = np.sqrt(np.asarray(h.multiply(h).sum(axis=1)).ravel())
        hq, hg = h[:n_query], h[n_query:]
        s = (hq @ hg.T).toarray() / nrm[:n_query, None] / nrm[None, n_query:]
    else:
        nrm = np.sqrt((h * h).sum(axis=1))
        s = (h[:n_query] @ h[n_query:].T) / nrm[:n_query, None] / nrm[None, n_query:]
    idx = np.argsort(-s, axis=1, kind="stable")
    dist = 1.0 - np.take_along_axis(s, idx, axis=1)
    return idx, dist, s


@dataclasses.dataclass
class OracleResult:
    knn_idx: np.ndarray          # (N, k1) union indices, sorted (S desc, index asc)
    knn_score: np.ndarray        # (N, k1) S values
    a_star: object               # N x N, dense ndarray or CSR
    h: list                      # h^(0) ... h^(L), dense ndarray or CSR
    idx: np.ndarray              # (Q, G) final gallery order per query
    dist: np.ndarray             # (Q, G) 1 - s in that order
    s: np.ndarray                # (Q, G) final cosine, gallery order
    s_initial: Optional[np.ndarray] = None  # dense mode: the full S


def rerank(xq: np.ndarray, xg: np.ndarray, k1: int, k2: int, layers: int, alpha: float = 2.0,
           aggregator: str = "sum", feature: str = "astar", mode: str = "auto",
           timings: Optional[dict] = None) -> OracleResult:
    """Algorithm 1 end to end in float64.

    ``xq`` (Q, d) and ``xg`` (G, d) are the raw features; X_u stacks them,
    queries first.  ``mode`` is "dense", "sparse" or "auto" (dense up to 2,000
    vertices).  When ``timings`` is a dict, the wall time (s) of each group of
    steps is stored in it: "knn" (Eq. 7-8), "graph" (Eq. 8-12), "propagate"
    (Eq. 13-14, all layers), "rank" (Alg. 1 step 7); the arithmetic is the
    same either way.
    """
    clock = [time.perf_counter()]

    def lap(name):
        now = time.perf_counter()
        if timings is not None:
            timings[name] = now - clock[0]
        clock[0] = now

    if aggregator not in AGGREGATORS or feature not in FEATURES:
        raise ValueError("unknown aggregator or feature mode")
    xu = np.concatenate([np.asarray(xq, np.float64), np.asarray(xg, np.float64)])
    n, q = xu.shape[0], len(xq)
    if not (1 <= k2 <= k1 <= n) or layers < 0:
        raise ValueError("need 1 <= k2 <= k1 <= n and layers >= 0")
    dense = (n <= 2000) if mode == "auto" else (mode == "dense")

    s_full = None
    if dense:
        xh = unit_rows(xu)
        s_full = similarity_rows(xh, np.arange(n))                  # Eq. 7
        knn_idx = top_k_rows(s_full, k1)                             # Eq. 8
        knn_score = np.take_along_axis(s_full, knn_idx, axis=1)
    else:
        knn_idx, knn_score = knn_lists(xu, k1)                       # Eq. 7, 8
    lap("knn")

    a = adjacency(knn_idx, n, dense)                                 # Eq. 8
    a_star = symmetric_adjacency(a)                                  # Eq. 9, 10
    if feature == "astar":                                           # Eq. 11
        h0 = a_star
    elif feature == "a":
        h0 = a
    else:
        h0 = unit_rows(xu)
        h0 = h0 if dense else sp.csr_matrix(h0)
    w = knn_graph_weights(knn_idx, knn_score, k2, alpha, aggregator, n, dense)  # Eq. 12, 14
    lap("graph")
    hs = [h0]
    for _ in range(layers):                                          # Eq. 13, 14
        hs.append(propagate(hs[-1], w, knn_idx, k2, aggregator))
    lap("propagate")
    idx, dist, s = final_ranking(hs[-1], q)                          # Alg. 1 step 7
    lap("rank")
    return OracleResult(knn_idx, knn_score, a_star, hs, idx, dist, s, s_full)


def k1_from_classes(n: int, n_classes: int) -> int:
    """k1 = floor(n / C), the average number of images per class (Eq. 15)."""
    return n // n_classes

"""Retrieval accuracy of ranked gallery lists, for the synthetic sweeps.

Evaluation only: nothing here is part of the re-ranking path.  The paper
reports mAP and Rank-1 (Sec. 4.1, Tables 1, 2, 5); the definitions are the
usual ones for retrieval with identity labels:

* AP of a query: the mean, over the gallery items with the query's label, of
  the precision of the ranked list at each such item's position; items missing
  from a truncated list count as precision 0.
* mAP: AP averaged over the queries that have at least one match.
* Rank-k: fraction of those queries whose first k results hold a match.

Distractors carry label -1 and never match.  Also the k1 rule of Eq. 15.
"""
from __future__ import annotations

import numpy as np


def retrieval_metrics(ranked_idx: np.ndarray, yq: np.ndarray, yg: np.ndarray, ks=(1, 5, 10)) -> dict:
    """ranked_idx: (Q, T) gallery indices, best first (T <= G)."""
    ranked_idx = np.asarray(ranked_idx)
    yq = np.asarray(yq)
    yg = np.asarray(yg)
    match = yg[ranked_idx] == yq[:, None]
    match &= (yq[:, None] >= 0)
    # matches of each query in the whole gallery (the AP denominator)
    labels, counts = np.unique(yg[yg >= 0], return_counts=True)
    per_label = dict(zip(labels.tolist(), counts.tolist()))
    n_rel = np.array([per_label.get(int(y), 0) for y in yq], dtype=np.int64)
    keep = n_rel > 0
    hits = np.cumsum(match, axis=1, dtype=np.int64)
    pos = np.arange(1, match.shape[1] + 1, dtype=np.float64)
    ap = (match * (hits / pos)).sum(axis=1) / np.maximum(n_rel, 1)
    out = {"mAP": float(ap[keep].mean()) if keep.any() else 0.0, "queries": int(keep.sum())}
    for k in ks:
        k = min(k, match.shape[1])
        out[f"R{k}"] = float(match[keep, :k].any(axis=1).mean()) if keep.any() else 0.0
    return out


def k1_from_classes(n: int, n_classes: int) -> int:
    """k1 = floor(n / C): the average number of images per class (Eq. 15)."""
    if n_classes < 1 or n < 1:
        raise ValueError("n and n_classes must be positive")
    return max(1, n // n_classes)

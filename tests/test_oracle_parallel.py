"""The threaded composition used by the full-size GPU parity tests gives the
oracle's result element for element (CPU only)."""
import numpy as np

import oracle_parallel
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic


def test_threaded_oracle_equals_sequential_oracle():
    spec = synthetic.WorkloadSpec("par", 230, 2570, 96, 160, 0.35, 100, None, seed=77)
    w = synthetic.make_workload(spec)
    ref = o.rerank(w.xq, w.xg, k1=26, k2=7, layers=2, mode="sparse")
    got = oracle_parallel.rerank_sparse(w.xq, w.xg, 26, 7, 2, workers=5)
    assert (got.knn_idx == ref.knn_idx).all() and (got.knn_score == ref.knn_score).all()
    assert (got.a_star != ref.a_star).nnz == 0
    for a, b in zip(got.h, ref.h):
        assert abs(a - b).max() == 0.0
    assert (got.idx == ref.idx).all() and (got.dist == ref.dist).all() and (got.s == ref.s).all()


def test_threaded_knn_ragged_blocks():
    x = np.random.default_rng(5).standard_normal((2100, 20))
    a = oracle_parallel.knn_lists(x, 9, workers=7)
    b = o.knn_lists(x, 9)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()

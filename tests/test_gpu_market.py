"""Full-size workloads against the FP64 oracle, every output element.

market_23k_d2048: 3,368 queries + 19,732 gallery vectors, d = 2048 (the
configuration bench.py times), and large_50k_d512: 5,000 + 45,000 vectors,
d = 512; k1 = 26, k2 = 7, L = 2, full ranked lists.

The oracle runs Algorithm 1 once per workload on the host cores
(``oracle_parallel.rerank_sparse``: the oracle's own step functions, its
per-row sorts spread over threads), then every precision of the GPU path is
compared with it element by element by the rules of ``parity.py``:
  * all N x k1 neighbour lists (Eq. 8) equal the oracle's;
  * h^(0) = A* rows (Eq. 9-11) equal as CSR, exactly;
  * h^(L) (Eq. 13-14): the same support in every row, values within FP32
    accuracy;
  * all Q x G ranked lists and distances (Alg. 1 step 7).
The BF16 and FP8 tensor-core paths must also reproduce the FP32 path bit for
bit, and properties that hold at any size are checked on top.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle_parallel
import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K1, K2, L = 26, 7, 2
PRECISIONS = ("fp32", "bf16", "fp8")


def _csr_from_padded(start, length, col, val, n):
    """The GPU's layer rows (row i at start[i], length[i] entries, columns in no
    set order) as a SciPy CSR matrix with sorted columns."""
    length = length.astype(np.int64)
    rows = np.repeat(np.arange(n), length)
    first = np.repeat(np.cumsum(length) - length, length)
    off = np.arange(int(length.sum())) - first + np.repeat(start.astype(np.int64), length)
    m = sp.csr_matrix((val[off].astype(np.float64), (rows, col[off])), shape=(n, n))
    m.sort_indices()
    return m


@pytest.fixture(scope="module", params=["MARKET_SCALE", "LARGE_50K"])
def market(request):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    w = synthetic.make_workload(getattr(synthetic, request.param))
    n = len(w.xq) + len(w.xg)
    xq = torch.from_numpy(w.xq).cuda()
    xg = torch.from_numpy(w.xg).cuda()
    out = {}
    for prec in PRECISIONS:
        with rerank.Reranker(precision=prec) as R:
            idx, dist = R.run(xq, xg, K1, K2, L)
            torch.cuda.synchronize()
            out[prec] = dict(idx=idx.cpu().numpy(), dist=dist.cpu().numpy(),
                             knn=R.debug("knn_idx").reshape(n, K1), info=R.last_info())
            if prec == "fp32":
                rp = R.debug("h0_rowptr")[: n + 1]
                out[prec].update(h0=(rp, R.debug("h0_col")[: rp[-1]], R.debug("h0_val")[: rp[-1]]),
                                 hl=_csr_from_padded(R.debug("hl_start")[:n], R.debug("hl_len")[:n],
                                                     R.debug("hl_col"), R.debug("hl_val"), n))
        del idx, dist
    del xq, xg
    torch.cuda.empty_cache()
    ref = oracle_parallel.rerank_sparse(w.xq, w.xg, K1, K2, L)
    return w, out, ref


def test_all_neighbour_lists_match_oracle(market):
    w, out, ref = market
    xu_hat = o.unit_rows(np.concatenate([w.xq, w.xg]))
    for prec in PRECISIONS:
        parity.assert_knn_equal(out[prec]["knn"], ref.knn_idx, ref.knn_score, xu_hat)


def test_graph_and_layer_features_match_oracle(market):
    _, out, ref = market
    rp, col, val = out["fp32"]["h0"]
    a = ref.a_star.tocsr()
    a.sort_indices()
    assert (rp == a.indptr).all() and (col == a.indices).all() and (val == a.data).all()
    got, want = out["fp32"]["hl"], ref.h[-1].tocsr()
    want.sort_indices()
    assert (got.indptr == want.indptr).all() and (got.indices == want.indices).all()
    np.testing.assert_allclose(got.data, want.data, rtol=2e-5, atol=1e-7)
    assert out["fp32"]["info"]["h_nnz"][: L + 1] == [h.nnz for h in ref.h]


def test_all_ranked_lists_match_oracle(market):
    _, out, ref = market
    for prec in PRECISIONS:
        stats = parity.assert_ranked_equal(out[prec]["idx"], out[prec]["dist"], ref.s, ref.idx)
        assert stats["max_dist_err"] <= 1e-5, prec


def test_lowprec_paths_reproduce_fp32(market):
    _, out, _ = market
    for prec in ("bf16", "fp8"):
        assert (out[prec]["knn"] == out["fp32"]["knn"]).all(), prec
        assert (out[prec]["idx"] == out["fp32"]["idx"]).all(), prec
        assert (out[prec]["dist"] == out["fp32"]["dist"]).all(), prec


def test_graph_and_output_invariants(market):
    w, out, _ = market
    knn = out["fp32"]["knn"]
    n = knn.shape[0]
    assert (knn[:, 0] == np.arange(n)).all()
    srt = np.sort(knn, axis=1)
    assert not (srt[:, 1:] == srt[:, :-1]).any()
    idx, dist = out["fp32"]["idx"], out["fp32"]["dist"]
    assert idx.shape == (len(w.xq), len(w.xg))
    assert (np.diff(dist, axis=1) >= 0).all()
    assert dist.min() >= 0.0 and dist.max() <= 1.0

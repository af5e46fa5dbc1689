"""Variants of Eq. 13-14 on the GPU against the FP64 oracle, through the C ABI.

The paper's default is the sum aggregator over A* rows with alpha = 2
(Sec. 4.1); it also discusses the mean and max aggregators, the A_i initial
features (Table 1) and the weight exponent (Eq. 14; alpha = 0 with the mean is
the query expansion of Sec. 3.4).  Each combination the GPU path implements is
checked here on a clustered instance with the parity rules of parity.py,
including the dense x_i initial features (Table 1, first column): with
L = 0 they give the initial cosine ranking, and with alpha = 0, the mean and
one layer they are local query expansion (Sec. 3.4, Eq. 4) plus the residual.
"""
import numpy as np
import pytest

import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    return rerank


@pytest.fixture(scope="module")
def inst():
    spec = synthetic.WorkloadSpec("variants", 61, 700, 96, 45, 0.35, 0, None, seed=33)
    return synthetic.make_workload(spec)


@pytest.mark.parametrize("aggregator,feature,alpha,layers", [
    ("mean", "astar", 2.0, 2),
    ("max", "astar", 2.0, 2),
    ("max", "astar", 2.0, 3),
    ("sum", "a", 2.0, 2),
    ("mean", "a", 0.0, 1),
    ("max", "a", 2.0, 2),
    ("sum", "astar", 0.0, 2),
])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_variant_matches_oracle(lib, inst, aggregator, feature, alpha, layers, precision):
    k1, k2 = 20, 5
    ref = o.rerank(inst.xq, inst.xg, k1=k1, k2=k2, layers=layers, alpha=alpha, aggregator=aggregator,
                   feature=feature, mode="sparse")
    with lib.Reranker(precision=precision, aggregator=aggregator, feature=feature, alpha=alpha) as R:
        idx, dist = R.run(torch.from_numpy(inst.xq).cuda(), torch.from_numpy(inst.xg).cuda(), k1, k2, layers)
        torch.cuda.synchronize()
        stats = parity.assert_ranked_equal(idx.cpu().numpy(), dist.cpu().numpy(), ref.s, ref.idx)
    assert stats["max_dist_err"] < 1e-5


def test_max_aggregator_differs_from_sum(lib, inst):
    """The max path is not the sum path under another name: their rankings differ."""
    outs = []
    for agg in ("sum", "max"):
        with lib.Reranker(aggregator=agg) as R:
            idx, dist = R.run(torch.from_numpy(inst.xq).cuda(), torch.from_numpy(inst.xg).cuda(), 20, 5, 2)
            torch.cuda.synchronize()
            outs.append(dist.cpu().numpy())
    assert not np.array_equal(outs[0], outs[1])


def _dense_run(lib, inst, precision, aggregator, alpha, layers, k1=20, k2=5):
    with lib.Reranker(precision=precision, aggregator=aggregator, feature="x", alpha=alpha) as R:
        idx, dist = R.run(torch.from_numpy(inst.xq).cuda(), torch.from_numpy(inst.xg).cuda(), k1, k2, layers)
        torch.cuda.synchronize()
        n = len(inst.xq) + len(inst.xg)
        h = R.debug("hl_dense")
        knn = R.debug("knn_idx").reshape(n, k1)
    return idx.cpu().numpy(), dist.cpu().numpy(), h.reshape(n, -1), knn


@pytest.mark.parametrize("aggregator,alpha,layers", [
    ("sum", 2.0, 2),
    ("mean", 0.0, 1),   # local query expansion + residual (Sec. 3.4)
    ("max", 2.0, 2),
    ("sum", 2.0, 0),    # the initial ranking
    ("mean", 2.0, 3),
])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_dense_features_match_oracle(lib, inst, aggregator, alpha, layers, precision):
    """x_i initial features: h^(L) (dense, Eq. 13-14) and the ranked lists
    (Alg. 1 step 7) against the oracle's feature="x" run."""
    k1, k2 = 20, 5
    ref = o.rerank(inst.xq, inst.xg, k1=k1, k2=k2, layers=layers, alpha=alpha, aggregator=aggregator,
                   feature="x", mode="dense")
    idx, dist, h, knn = _dense_run(lib, inst, precision, aggregator, alpha, layers)
    d = inst.xq.shape[1]
    np.testing.assert_allclose(h[:, :d], ref.h[-1], rtol=0, atol=2e-6)
    assert not h[:, d:].any()  # padding columns stay zero
    assert (knn == ref.knn_idx).all()
    stats = parity.assert_ranked_equal(idx, dist, ref.s, ref.idx)
    assert stats["max_dist_err"] < 1e-5


def test_dense_ranking_paths_agree():
    """The dense ranking sorts each query's scores by one bucket pass (keys in
    global scratch, a key's place = its bucket's start + the smaller keys in
    it); a query with a crowded bucket takes a 4-pass radix sort instead.  A
    test hook lowers the bucket cap to 1, so that every query takes the radix
    sort: both give the same lists, bit for bit, including a group of equal
    scores (copies of one gallery row), and match the oracle."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys, hashlib; sys.path.insert(0, '.'); sys.path.insert(0, 'tests');"
        "import parity; from oracle import rerank_oracle as o;"
        "from paper_2012_07620_gb300 import rerank, synthetic;"
        "w = synthetic.make_workload(synthetic.WorkloadSpec('dense_sort', 80, 2920, 64, 100, 0.6, 0, None, seed=23));"
        "xg = w.xg.copy(); xg[200:206] = xg[11];"
        "R = rerank.Reranker(feature='x'); tq, tg = torch.from_numpy(w.xq).cuda(), torch.from_numpy(xg).cuda();"
        "i, d = R.run(tq, tg, 20, 5, 1); i2, d2 = R.run(tq, tg, 20, 5, 1, 100);"
        "torch.cuda.synchronize(); i, d, i2, d2 = (a.cpu().numpy() for a in (i, d, i2, d2));"
        "ref = o.rerank(w.xq, xg, 20, 5, 1, feature='x', mode='dense');"
        "parity.assert_ranked_equal(i, d, ref.s, ref.idx); parity.assert_ranked_equal(i2, d2, ref.s, ref.idx, 100);"
        "assert (i2 == i[:, :100]).all() and (d2 == d[:, :100]).all();"
        "print('digest', hashlib.sha256(i.tobytes() + d.tobytes()).hexdigest())"
    )
    digests = []
    for caps in (None, "8192,1"):
        env = dict(os.environ)
        env.pop("RERANK_TEST_RANK_CAPS", None)
        if caps:
            env["RERANK_TEST_RANK_CAPS"] = caps
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and "digest" in r.stdout, (caps, r.stderr[-2000:])
        digests.append(r.stdout.split("digest")[-1].strip())
    assert len(set(digests)) == 1, digests


def test_dense_features_without_layers_give_the_initial_ranking(lib, inst):
    """x_i features with L = 0: the list of every query is the gallery sorted by
    cos(x_q, x_g), ties to the lower index (Table 1, first column = the
    baseline ranking), checked against SciPy-free FP64 cosines."""
    idx, dist, _, _ = _dense_run(lib, inst, "fp32", "sum", 2.0, 0)
    xq = o.unit_rows(inst.xq)
    xg = o.unit_rows(inst.xg)
    s = xq @ xg.T
    want = np.argsort(-s, axis=1, kind="stable")
    parity.assert_ranked_equal(idx, dist, s, want)


def test_dense_one_layer_mean_alpha0_is_query_expansion(lib, inst):
    """Sec. 3.4: with alpha = 0 and the mean aggregator, one layer gives
    h_i = normalise(x_i + (1/k2) sum_{j in N(i, k2)} x_j) (Eq. 4 plus the
    residual of Eq. 13), computed here from the GPU's own neighbour lists."""
    k1, k2 = 20, 5
    _, _, h, knn = _dense_run(lib, inst, "fp32", "mean", 0.0, 1, k1, k2)
    x = o.unit_rows(np.concatenate([inst.xq, inst.xg]))
    want = x + x[knn[:, :k2]].mean(axis=1)
    want /= np.linalg.norm(want, axis=1, keepdims=True)
    np.testing.assert_allclose(h[:, :x.shape[1]], want, rtol=0, atol=2e-6)


def test_dense_features_refused_by_batch_and_serving(lib, inst):
    xq = torch.from_numpy(inst.xq).cuda()
    xg = torch.from_numpy(inst.xg).cuda()
    with lib.Reranker(feature="x") as R:
        with pytest.raises(lib.RerankError) as e:
            R.run_batch([dict(xq=xq, xg=xg, k1=20, k2=5, layers=2)])
        assert e.value.status == 7  # EUNSUPPORTED
    with lib.Reranker(precision="bf16", feature="x") as R:
        with pytest.raises(lib.RerankError) as e:
            R.load_gallery(xg, max_query=16, k1=20, k2=5, layers=2)
        assert e.value.status == 7

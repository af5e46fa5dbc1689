"""Variants of Eq. 13-14 on the GPU against the FP64 oracle, through the C ABI.

The paper's default is the sum aggregator over A* rows with alpha = 2
(Sec. 4.1); it also discusses the mean and max aggregators, the A_i initial
features (Table 1) and the weight exponent (Eq. 14; alpha = 0 with the mean is
the query expansion of Sec. 3.4).  Each combination the GPU path implements is
checked here on a clustered instance with the parity rules of parity.py; the
dense x_i features are oracle-only and must be refused.
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


def test_dense_features_are_refused(lib, inst):
    with lib.Reranker(feature="x") as R:
        with pytest.raises(lib.RerankError) as e:
            R.run(torch.from_numpy(inst.xq).cuda(), torch.from_numpy(inst.xg).cuda(), 20, 5, 2)
        assert e.value.status == 7  # EUNSUPPORTED

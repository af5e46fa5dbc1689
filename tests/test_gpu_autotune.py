"""Autotuner: the table it writes is read back, and no launch shape it can
choose changes a result (bit-for-bit equal outputs)."""
import json

import numpy as np
import pytest

from paper_2012_07620_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPEC = synthetic.WorkloadSpec("tune", 300, 2700, 256, 150, 0.35, 0, None, seed=31)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    return rerank


@pytest.fixture(scope="module")
def data():
    w = synthetic.make_workload(SPEC)
    return torch.from_numpy(w.xq).cuda(), torch.from_numpy(w.xg).cuda()


def _run(R, xq, xg):
    i, d = R.run(xq, xg, 26, 7, 2)
    torch.cuda.synchronize()
    return i.cpu().numpy(), d.cpu().numpy()


def _bucket(n):
    b = 0
    while 2 ** (b + 1) <= n * n:
        b += 1
    return b


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_autotune_writes_table_and_keeps_results(lib, data, tmp_path, precision):
    xq, xg = data
    path = str(tmp_path / "tune.json")
    with lib.Reranker(precision=precision) as D:
        ref = _run(D, xq, xg)
    with lib.Reranker(precision=precision, autotune_path=path) as R:
        t = R.autotune(xq, xg, 26, 7, 2)
        assert t["n_bucket"] == _bucket(SPEC.n) and t["ms"] > 0
        got = _run(R, xq, xg)
    table = json.load(open(path))
    assert len(table["entries"]) == 1
    assert lib.tuning_lookup(path, precision, SPEC.n, SPEC.dim)["sim_chunks"] == t["sim_chunks"]
    assert (got[0] == ref[0]).all() and (got[1] == ref[1]).all()
    with lib.Reranker(precision=precision, autotune_path=path) as R2:  # a new context reads the file
        got2 = _run(R2, xq, xg)
    assert (got2[0] == ref[0]).all() and (got2[1] == ref[1]).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(1, 4, 0, 8), (3, 16, 1, 22), (32, 24, 0, 30), (2, 8, 1, -1), (0, 8, 1, 1)])
def test_every_launch_shape_gives_the_same_result(lib, data, tmp_path, precision, shape):
    xq, xg = data
    chunks, warps, order, m = shape
    path = tmp_path / "t.json"
    prec = {"fp32": 0, "bf16": 1, "fp8": 2}[precision]
    path.write_text(json.dumps({"version": 1, "entries": [
        {"precision": prec, "d": SPEC.dim, "n_bucket": _bucket(SPEC.n), "sim_chunks": chunks, "prop_warps": warps,
         "refine_order": order, "rescore_m": m, "ms": 0}]}))
    with lib.Reranker(precision=precision) as D, lib.Reranker(precision=precision, autotune_path=str(path)) as R:
        a = _run(D, xq, xg)
        b = _run(R, xq, xg)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


@pytest.fixture(scope="module")
def oracle_ref():
    from oracle import rerank_oracle as o
    w = synthetic.make_workload(SPEC)
    return o.rerank(w.xq, w.xg, k1=26, k2=7, layers=2, mode="sparse")


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_tuned_path_matches_oracle(lib, data, tmp_path, oracle_ref, precision):
    """The launch shapes the autotuner picks give Algorithm 1's result: the
    tuned run's neighbour lists (Eq. 8) and ranked lists (Alg. 1 step 7)
    against the FP64 oracle on the same instance."""
    import parity
    xq, xg = data
    path = str(tmp_path / "tune.json")
    with lib.Reranker(precision=precision, autotune_path=path) as R:
        R.autotune(xq, xg, 26, 7, 2)
        idx, dist = _run(R, xq, xg)
        knn = R.debug("knn_idx").reshape(SPEC.n, 26)
    w = synthetic.make_workload(SPEC)
    from oracle import rerank_oracle as o
    xu_hat = o.unit_rows(np.concatenate([w.xq, w.xg]))
    parity.assert_knn_equal(knn, oracle_ref.knn_idx, oracle_ref.knn_score, xu_hat)
    parity.assert_ranked_equal(idx, dist, oracle_ref.s, oracle_ref.idx)

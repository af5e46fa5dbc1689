"""GPU path against the FP64 oracle, through the C ABI.

Inputs are seeded; sizes span several 128-row tiles with ragged tails.
Rules (see parity.py): neighbour lists exactly equal, final lists equal up
to swaps of entries whose oracle scores are within 1e-6, distances within
1e-5 relative.
"""
import numpy as np
import pytest

import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    r = rerank.Reranker(device=0)
    yield r
    r.close()


def _gpu(R, xq, xg, k1, k2, layers, topk=0):
    tq = torch.from_numpy(np.ascontiguousarray(xq)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(xg)).cuda()
    idx, dist = R.run(tq, tg, k1, k2, layers, topk)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def _unit(x):
    x = np.asarray(x, np.float64)
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def _check_all(R, xq, xg, k1, k2, layers, topk=0, check_h=True):
    ref = o.rerank(xq, xg, k1=k1, k2=k2, layers=layers, mode="sparse")
    idx, dist = _gpu(R, xq, xg, k1, k2, layers, topk)
    n = len(xq) + len(xg)
    xu_hat = _unit(np.concatenate([xq, xg]))
    knn = R.debug("knn_idx").reshape(n, k1)
    parity.assert_knn_equal(knn, ref.knn_idx, ref.knn_score, xu_hat)
    if check_h:
        # h^(0) = A* rows exactly (Eq. 9-11)
        rp = R.debug("h0_rowptr")[: n + 1]
        col = R.debug("h0_col")[: rp[-1]]
        val = R.debug("h0_val")[: rp[-1]]
        a = ref.a_star.tocsr()
        a.sort_indices()
        assert (rp == a.indptr).all() and (col == a.indices).all() and (val == a.data).all()
        # h^(L): same supports, values within FP32 accuracy (layer rows are
        # stored in no particular column order: compare them sorted)
        st = R.debug("hl_start")[:n]
        ln = R.debug("hl_len")[:n]
        hc = R.debug("hl_col")
        hv = R.debug("hl_val")
        hl = ref.h[-1].tocsr()
        hl.sort_indices()
        for i in range(0, n, max(1, n // 97)):
            c = hc[st[i]: st[i] + ln[i]]
            v = hv[st[i]: st[i] + ln[i]]
            order = np.argsort(c, kind="stable")
            c, v = c[order], v[order]
            rc = hl.indices[hl.indptr[i]: hl.indptr[i + 1]]
            rv = hl.data[hl.indptr[i]: hl.indptr[i + 1]]
            assert (c == rc).all(), i
            np.testing.assert_allclose(v, rv, rtol=2e-5, atol=1e-7)
    t = topk if topk else len(xg)
    return parity.assert_ranked_equal(idx, dist, ref.s, ref.idx, t)


def test_tiny_workload(R):
    w = synthetic.make_workload(synthetic.TINY)
    stats = _check_all(R, w.xq, w.xg, 26, 7, 2)
    assert stats["max_dist_err"] < 1e-5


def test_layer_nnz_reported(R):
    """rerank_info.h_nnz: the non-zeros of h^(0) (= A*, Eq. 9-11) and of every
    propagated layer (Eq. 14) equal the oracle's supports exactly."""
    spec = synthetic.WorkloadSpec("nnz", 90, 800, 64, 40, 0.35, 20, None, seed=23)
    w = synthetic.make_workload(spec)
    ref = o.rerank(w.xq, w.xg, k1=20, k2=6, layers=3, mode="sparse")
    _gpu(R, w.xq, w.xg, 20, 6, 3)
    got = R.last_info()["h_nnz"]
    want = [ref.a_star.nnz] + [h.nnz for h in ref.h[1:]]
    assert got[:4] == want and got[4:] == [0] * 5, (got, want)


@pytest.mark.parametrize("nq,ng,d,c,k1,k2,layers", [
    (37, 300, 64, 20, 10, 3, 1),
    (129, 1200, 200, 60, 26, 7, 2),
    (300, 2700, 256, 150, 30, 5, 3),
    (61, 1950, 77, 90, 20, 7, 2),
])
def test_clustered_shapes(R, nq, ng, d, c, k1, k2, layers):
    spec = synthetic.WorkloadSpec("t", nq, ng, d, c, 0.35, 0, None, seed=nq + ng)
    w = synthetic.make_workload(spec)
    _check_all(R, w.xq, w.xg, k1, k2, layers)


@pytest.mark.parametrize("nq,ng,d,k1,k2,layers,topk", [
    (1, 700, 96, 20, 5, 3, 0),      # one query
    (50, 1, 64, 26, 7, 2, 0),       # one gallery item
    (40, 200, 32, 1, 1, 0, 0),      # k1 = k2 = 1, no layers
    (20, 28, 48, 48, 1, 2, 0),      # k1 = n = 48 = RERANK_MAX_K1 (every vertex a neighbour)
    (30, 970, 40, 48, 7, 1, 0),     # k1 = RERANK_MAX_K1 with n >> k1
    (30, 500, 128, 26, 7, 0, 0),    # no propagation
    (64, 900, 128, 26, 7, 2, 17),   # truncated output lists
    (5, 1000, 16, 8, 8, 4, 0),      # k2 = k1, four layers
    (40, 800, 64, 48, 40, 2, 0),    # more messages per row than lanes in a warp (k2 >= 32)
])
def test_edge_shapes(R, nq, ng, d, k1, k2, layers, topk):
    rng = np.random.default_rng(nq * 1000 + ng)
    xq = rng.standard_normal((nq, d)).astype(np.float32)
    xg = rng.standard_normal((ng, d)).astype(np.float32)
    _check_all(R, xq, xg, k1, k2, layers, topk)


def test_duplicates_and_scaled_rows(R):
    rng = np.random.default_rng(11)
    xg = rng.standard_normal((400, 64)).astype(np.float32)
    xg[10] = xg[3]
    xg[200] = xg[3] * 3.0       # same direction, other length
    xq = np.concatenate([xg[3:4] * 0.5, rng.standard_normal((9, 64)).astype(np.float32)])
    _check_all(R, xq, xg, 12, 4, 2)


def test_host_buffers_match_device(R):
    w = synthetic.make_workload(synthetic.TINY)
    di, dd = _gpu(R, w.xq, w.xg, 26, 7, 2)
    hi, hd = R.run(w.xq, w.xg, 26, 7, 2)
    assert (hi == di).all() and (hd == dd).all()


@pytest.mark.parametrize("topk", [0, 37])
def test_host_outputs_copied_in_parts_match_device(R, topk):
    """With host outputs and enough queries the call ranks the queries in parts
    and copies each part back while the next is ranked: same bits as device outputs."""
    spec = synthetic.WorkloadSpec("many_queries", 1300, 2100, 96, 160, 0.35, 0, None, seed=12)
    w = synthetic.make_workload(spec)
    di, dd = _gpu(R, w.xq, w.xg, 20, 5, 2, topk)
    hi, hd = R.run(w.xq, w.xg, 20, 5, 2, topk)
    assert (hi == di).all() and (hd == dd).all()


def test_repeat_is_bitwise_identical(R):
    w = synthetic.make_workload(synthetic.TINY)
    a = _gpu(R, w.xq, w.xg, 26, 7, 2)
    b = _gpu(R, w.xq, w.xg, 26, 7, 2)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


def test_bf16_inputs(R):
    w = synthetic.make_workload(synthetic.TINY)
    tq = torch.from_numpy(w.xq).to(torch.bfloat16)
    tg = torch.from_numpy(w.xg).to(torch.bfloat16)
    xq, xg = tq.float().numpy(), tg.float().numpy()
    ref = o.rerank(xq, xg, k1=26, k2=7, layers=2, mode="sparse")
    idx, dist = R.run(tq.cuda(), tg.cuda(), 26, 7, 2)
    torch.cuda.synchronize()
    parity.assert_ranked_equal(idx.cpu().numpy(), dist.cpu().numpy(), ref.s, ref.idx)


def test_knn_entry_point(R):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1500, 100)).astype(np.float32)
    ridx, rs = o.knn_lists(x, 30)
    idx, s = R.knn(torch.from_numpy(x).cuda(), 30)
    torch.cuda.synchronize()
    parity.assert_knn_equal(idx.cpu().numpy(), ridx, rs, _unit(x))
    np.testing.assert_allclose(s.cpu().numpy(), rs, atol=2e-6)


def test_bad_rows_are_rejected(R):
    from paper_2012_07620_gb300.rerank import RerankError
    rng = np.random.default_rng(2)
    xq = rng.standard_normal((10, 32)).astype(np.float32)
    xg = rng.standard_normal((100, 32)).astype(np.float32)
    bad = xg.copy()
    bad[7, 3] = np.nan
    with pytest.raises(RerankError) as e:
        _gpu(R, xq, bad, 5, 2, 1)
    assert e.value.status == 1 and R.last_info()["bad_row"] == 10 + 7
    bad = xg.copy()
    bad[0] = 0.0
    with pytest.raises(RerankError) as e:
        _gpu(R, xq, bad, 5, 2, 1)
    assert e.value.status == 1 and R.last_info()["bad_row"] == 10
    # the context stays usable
    _check_all(R, xq, xg, 5, 2, 1)


def test_generator_is_portable():
    w = synthetic.make_workload(synthetic.TINY)
    assert synthetic.array_digest(w.xq, w.xg) == "1b491f1d79575c3f22a106da512bb61392e50401515ccfe446dcb841c741dee8"


def test_overflow_retry_path():
    """Layer buffers that start too small overflow, grow, and the call is redone."""
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys; sys.path.insert(0, '.'); sys.path.insert(0, 'tests');"
        "import parity; from oracle import rerank_oracle as o;"
        "from paper_2012_07620_gb300 import rerank;"
        "rng = np.random.default_rng(9); xq = rng.standard_normal((64, 128)).astype(np.float32);"
        "xg = rng.standard_normal((900, 128)).astype(np.float32);"
        "R = rerank.Reranker(); i, d = R.run(torch.from_numpy(xq).cuda(), torch.from_numpy(xg).cuda(), 26, 7, 2);"
        "torch.cuda.synchronize(); ref = o.rerank(xq, xg, 26, 7, 2, mode='sparse');"
        "parity.assert_ranked_equal(i.cpu().numpy(), d.cpu().numpy(), ref.s, ref.idx); print('ok')"
    )
    import os
    env = dict(os.environ, RERANK_TEST_CAP_H="60000")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]


def test_rank_sort_paths_agree():
    """The final ranking sorts each query's non-zero scores by buckets (for a
    truncated list only the buckets that reach it), with the keys in shared
    memory or, beyond its cap, in global scratch, where full lists cut each
    bucket into sub-buckets of about four keys; queries with too crowded a
    bucket take the global radix sort.  A test hook lowers both limits: every
    path gives the same lists, bit for bit, full or truncated, and they match
    the oracle."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys, hashlib; sys.path.insert(0, '.'); sys.path.insert(0, 'tests');"
        "import parity; from oracle import rerank_oracle as o;"
        "from paper_2012_07620_gb300 import rerank, synthetic;"
        "w = synthetic.make_workload(synthetic.TINY);"
        "xg = w.xg.copy(); xg[100:104] = xg[7];"  # copies of one gallery row (a tie group inside N(i, k2))
        "R = rerank.Reranker(); tq, tg = torch.from_numpy(w.xq).cuda(), torch.from_numpy(xg).cuda();"
        "i, d = R.run(tq, tg, 26, 7, 2); i2, d2 = R.run(tq, tg, 26, 7, 2, 37);"  # full and top-37 lists
        "torch.cuda.synchronize(); i, d, i2, d2 = (a.cpu().numpy() for a in (i, d, i2, d2));"
        "ref = o.rerank(w.xq, xg, 26, 7, 2, mode='sparse');"
        "parity.assert_ranked_equal(i, d, ref.s, ref.idx); parity.assert_ranked_equal(i2, d2, ref.s, ref.idx, 37);"
        "assert (i2 == i[:, :37]).all() and (d2 == d[:, :37]).all();"
        "print('digest', hashlib.sha256(i.tobytes() + d.tobytes() + i2.tobytes() + d2.tobytes()).hexdigest())"
    )
    digests = []
    for caps in (None, "0,256", "100,256", "8192,1", "8192,4", "0,1", "0,4"):
        env = dict(os.environ)
        env.pop("RERANK_TEST_RANK_CAPS", None)
        if caps:
            env["RERANK_TEST_RANK_CAPS"] = caps
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and "digest" in r.stdout, (caps, r.stderr[-2000:])
        digests.append(r.stdout.split("digest")[-1].strip())
    assert len(set(digests)) == 1, digests


def test_propagation_paths_agree():
    """A layer row goes through a 512-slot warp table; rows that overflow it
    take a second pass with 2,048-slot tables when there are at least 4 per
    SM, else (and beyond 1,536 distinct columns) one CTA per row with a dense
    accumulator.  With noisy features (norm 1.2 around the centres), k1 = 40
    and k2 = 16, 2,839 of the 3,000 second-layer rows here have more than 384
    columns and 11 more than 1,536.  A test hook sends every overflowing row to the
    second pass or every one to the CTA path: the ranked lists and distances
    are the same bit for bit (each column is summed in message order and the
    norm is an exact fixed-point sum on every path), and match the oracle."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys, hashlib; sys.path.insert(0, '.'); sys.path.insert(0, 'tests');"
        "import parity; from oracle import rerank_oracle as o;"
        "from paper_2012_07620_gb300 import rerank, synthetic;"
        "w = synthetic.make_workload(synthetic.WorkloadSpec('spill', 300, 2700, 64, 100, 1.2, 0, None, seed=17));"
        "R = rerank.Reranker(); i, d = R.run(torch.from_numpy(w.xq).cuda(), torch.from_numpy(w.xg).cuda(), 40, 16, 2);"
        "torch.cuda.synchronize(); i, d = i.cpu().numpy(), d.cpu().numpy();"
        "ref = o.rerank(w.xq, w.xg, 40, 16, 2, mode='sparse');"
        "nz = np.diff(ref.h[-1].tocsr().indptr); assert (nz > 384).sum() > 100, (nz > 384).sum();"
        "parity.assert_ranked_equal(i, d, ref.s, ref.idx);"
        "print('digest', hashlib.sha256(i.tobytes() + d.tobytes()).hexdigest())"
    )
    digests = []
    for second_min in (None, "0", "1000000000"):
        env = dict(os.environ)
        env.pop("RERANK_TEST_PROP_SECOND_MIN", None)
        if second_min:
            env["RERANK_TEST_PROP_SECOND_MIN"] = second_min
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and "digest" in r.stdout, (second_min, r.stderr[-2000:])
        digests.append(r.stdout.split("digest")[-1].strip())
    assert len(set(digests)) == 1, digests


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_no_rescore_margin_sends_rows_to_the_exact_scan(precision):
    """With rescore_m = 0 the first pass keeps exactly k1 candidates, so no
    list can be certified (Eq. 8's boundary is unbounded) and every row goes
    on to the exact scan, which keeps k1 + 16 candidates of its own; at
    k1 = RERANK_MAX_K1 = 48 the lists must still equal the oracle's."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    spec = synthetic.WorkloadSpec("nomargin", 60, 1140, 64, 70, 0.35, 100, None, seed=91)
    w = synthetic.make_workload(spec)
    with rerank.Reranker(device=0, precision=precision, rescore_m=0) as R:
        stats = _check_all(R, w.xq, w.xg, 48, 7, 2)
        info = R.last_info()
    assert info["exact_scan_rows"] > 0 or info["fallback_rows"] > 0
    assert stats["max_dist_err"] < 1e-5

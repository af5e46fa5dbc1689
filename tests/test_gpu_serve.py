"""Serving: resident gallery, request loop, continuous batching.

Each request is Algorithm 1 on (its queries) u (the resident gallery).  The
tests check every served result against the FP64 oracle on that union (with
the layer rows a request leaves unchanged taken from the gallery's own
graph), that a request's result is the same bit for bit alone and in a mix of
overlapping requests, admission under an HBM budget, and the argument errors.
"""
import numpy as np
import pytest

import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K1, K2, L = 26, 7, 2
GALLERY = synthetic.WorkloadSpec("serve_small", 0, 3000, 256, 150, 0.35, 0, None, seed=21)
SIZES = [1, 7, 64, 300, 2, 129]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    return rerank


@pytest.fixture(scope="module")
def gallery():
    return synthetic.make_workload(GALLERY)


def _queries(w, sizes):
    return [synthetic.request_queries(w, 1000 + r, q) for r, q in enumerate(sizes)]


def _wait(R, t):
    info = R.wait(t, 120000)
    assert info is not None, "request still running after 120 s"
    return info


def _serve(R, qs, together, topk=0):
    outs = []
    if together:
        pend = [R.submit(torch.from_numpy(q).cuda(), topk) for q in qs]
        infos = [_wait(R, t) for t, _, _ in pend]
        outs = [(i.cpu().numpy(), d.cpu().numpy()) for _, i, d in pend]
    else:
        infos = []
        for q in qs:
            t, i, d = R.submit(torch.from_numpy(q).cuda(), topk)
            infos.append(_wait(R, t))
            outs.append((i.cpu().numpy(), d.cpu().numpy()))
    return outs, infos


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_served_results_match_oracle_alone_and_in_a_mix(lib, gallery, precision):
    qs = _queries(gallery, SIZES)
    with lib.Reranker(precision=precision) as R:
        R.load_gallery(torch.from_numpy(gallery.xg).cuda(), max_query=512, k1=K1, k2=K2, layers=L, slots=4)
        alone, _ = _serve(R, qs, together=False)
        mix, infos = _serve(R, qs, together=True)
        info = R.serve_info()
        assert info["slots"] == 4 and info["completed"] == 2 * len(qs)
        assert info["max_in_flight"] >= 2, "requests submitted together never overlapped"
        assert info["touched_rows"] > 0
        # layer rows a request leaves unchanged come from the gallery's own graph
        total = 2 * sum(q + gallery.xg.shape[0] for q in SIZES) * L
        assert info["reuse_layers"] == 1 and 0 < info["recomputed_rows"] < total
        for (ai, ad), (mi, md) in zip(alone, mix):
            assert (ai == mi).all() and (ad == md).all(), "result depends on the other requests"
        for q, (ai, ad) in zip(qs, alone):
            ref = o.rerank(q, gallery.xg, k1=K1, k2=K2, layers=L, mode="sparse")
            parity.assert_ranked_equal(ai, ad, ref.s, ref.idx)


def test_served_equals_rerank_run_on_the_union(lib, gallery):
    """The serving path re-derives only the gallery rows a query can enter;
    its results must agree with a fresh rerank_run of the same union."""
    qs = _queries(gallery, [1, 50, 400])
    with lib.Reranker(precision="bf16") as R, lib.Reranker(precision="bf16") as F:
        R.load_gallery(torch.from_numpy(gallery.xg).cuda(), max_query=512, k1=K1, k2=K2, layers=L, slots=2)
        out, _ = _serve(R, qs, together=True, topk=100)
        xg = torch.from_numpy(gallery.xg).cuda()
        for q, (si, sd) in zip(qs, out):
            fi, fd = F.run(torch.from_numpy(q).cuda(), xg, K1, K2, L, 100)
            torch.cuda.synchronize()
            fi, fd = fi.cpu().numpy(), fd.cpu().numpy()
            assert np.abs(sd.astype(np.float64) - fd).max() <= 1e-6
            differ = si != fi
            # entries may swap only where their distances tie to 1e-6
            assert np.all(np.abs(sd[differ].astype(np.float64) - fd[differ]) <= 1e-6)


def test_host_buffers_and_topk(lib, gallery):
    qs = _queries(gallery, [3, 40])
    with lib.Reranker(precision="bf16") as R:
        R.load_gallery(gallery.xg, max_query=64, k1=K1, k2=K2, layers=L, slots=2)
        for q in qs:
            t, i, d = R.submit(np.ascontiguousarray(q), 50)
            _wait(R, t)
            ref = o.rerank(q, gallery.xg, k1=K1, k2=K2, layers=L, mode="sparse")
            parity.assert_ranked_equal(i, d, ref.s, ref.idx, topk=50)


def test_budget_admission(lib, gallery):
    """A budget that admits one slot still serves every request (queued), with
    the same results; a budget below one slot is refused."""
    qs = _queries(gallery, [5, 90, 11, 200])
    with lib.Reranker(precision="bf16") as R:
        R.load_gallery(torch.from_numpy(gallery.xg).cuda(), max_query=256, k1=K1, k2=K2, layers=L, slots=4)
        info = R.serve_info()
        ref, _ = _serve(R, qs, together=True)
    budget = info["resident_bytes"] + int(2.5 * info["slot_bytes"])
    with lib.Reranker(precision="bf16", hbm_budget=budget) as R:
        R.load_gallery(torch.from_numpy(gallery.xg).cuda(), max_query=256, k1=K1, k2=K2, layers=L, slots=4)
        slots = R.serve_info()["slots"]
        assert 1 <= slots <= 2
        out, _ = _serve(R, qs, together=True)
        assert R.serve_info()["max_in_flight"] <= slots
        for (a, b), (c, d) in zip(ref, out):
            assert (a == c).all() and (b == d).all()
    with lib.Reranker(precision="bf16", hbm_budget=info["resident_bytes"] + info["slot_bytes"] // 2) as R:
        with pytest.raises(lib.RerankError) as e:
            R.load_gallery(torch.from_numpy(gallery.xg).cuda(), max_query=256, k1=K1, k2=K2, layers=L)
        assert e.value.status == 3


def test_argument_errors(lib, gallery):
    xg = torch.from_numpy(gallery.xg).cuda()
    q = torch.from_numpy(_queries(gallery, [4])[0]).cuda()
    with lib.Reranker(precision="fp32") as R:
        with pytest.raises(lib.RerankError) as e:
            R.load_gallery(xg, max_query=16, k1=K1, k2=K2, layers=L)
        assert e.value.status == 7
    with lib.Reranker(precision="bf16") as R:
        R._gallery_rows = 3000
        with pytest.raises(lib.RerankError) as e:
            R.submit(q)
        assert e.value.status == 7
        R.load_gallery(xg, max_query=16, k1=K1, k2=K2, layers=L, slots=1)
        with pytest.raises(lib.RerankError) as e:
            R.submit(torch.from_numpy(_queries(gallery, [17])[0]).cuda())
        assert e.value.status == 1
        with pytest.raises(lib.RerankError) as e:
            R.load_gallery(xg, max_query=16, k1=K1, k2=K2, layers=L)
        assert e.value.status == 7
        t, i, d = R.submit(q)
        _wait(R, t)
        with pytest.raises(lib.RerankError) as e:
            R.wait(t)
        assert e.value.status == 1
        R.unload_gallery()
        R.load_gallery(xg, max_query=8, k1=K1, k2=K2, layers=1, slots=1)
        t, i, d = R.submit(q)
        _wait(R, t)

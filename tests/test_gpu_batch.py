"""rerank_run_batch: many independent instances of Algorithm 1 in one call.

Each instance's output must equal, bit for bit, what rerank_run returns for it
alone (the batch only changes which instances run side by side), and must
match the FP64 oracle under the usual parity rules.
"""
import os
import subprocess
import sys

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


def _small_instances():
    """Mixed sizes, widths, k1/k2/L and input types; two tails that are not multiples of any tile."""
    shapes = [(40, 260, 64, 20, 5, 1), (129, 1200, 200, 26, 7, 2), (300, 2700, 256, 30, 5, 3),
              (17, 483, 128, 22, 6, 2), (90, 610, 96, 25, 7, 1), (200, 1800, 128, 28, 6, 3),
              (64, 900, 256, 20, 5, 2), (11, 389, 72, 24, 7, 3)]
    out = []
    for i, (q, g, d, k1, k2, layers) in enumerate(shapes):
        c = max(2, (q + g) // 20)
        spec = synthetic.WorkloadSpec(f"b{i}", q, g, d, c, 0.35, 0, None, seed=100 + i)
        w = synthetic.make_workload(spec)
        out.append(dict(w=w, k1=k1, k2=k2, layers=layers, bf16=(i % 2 == 1)))
    return out


def _features(w, bf16):
    xq, xg = torch.from_numpy(w.xq), torch.from_numpy(w.xg)
    if bf16:
        xq, xg = xq.bfloat16(), xg.bfloat16()
    return xq.cuda(), xg.cuda()


def _oracle_inputs(xq, xg):
    return xq.float().cpu().numpy().astype(np.float32), xg.float().cpu().numpy().astype(np.float32)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_batch_equals_single_calls_and_oracle(lib, precision):
    inst = _small_instances()
    feats = [_features(c["w"], c["bf16"]) for c in inst]
    with lib.Reranker(precision=precision) as R:
        jobs = [dict(xq=xq, xg=xg, k1=c["k1"], k2=c["k2"], layers=c["layers"]) for c, (xq, xg) in zip(inst, feats)]
        jobs[2]["topk_out"] = 100
        outs = R.run_batch(jobs)
        torch.cuda.synchronize()
        assert R.batch_status == [0] * len(jobs)
        batch = [(i.cpu().numpy(), d.cpu().numpy()) for i, d in outs]
        for c, (xq, xg), j, (bi, bd) in zip(inst, feats, jobs, batch):
            si, sd = R.run(xq, xg, c["k1"], c["k2"], c["layers"], j.get("topk_out", 0))
            torch.cuda.synchronize()
            assert (si.cpu().numpy() == bi).all() and (sd.cpu().numpy() == bd).all(), "batch differs from rerank_run"
            oq, og = _oracle_inputs(xq, xg)
            ref = o.rerank(oq, og, k1=c["k1"], k2=c["k2"], layers=c["layers"], mode="sparse")
            parity.assert_ranked_equal(bi, bd, ref.s, ref.idx)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_batch_spanning_several_similarity_launches(lib, precision):
    """More instances than one similarity launch takes (64), with feature widths
    on both sides of the epilogue layout switch (d <= 1024 and d > 1024)."""
    rng = np.random.default_rng(21)
    shapes = [(int(rng.integers(1, 40)), int(rng.integers(60, 400)), [32, 64, 200, 1100][i % 4]) for i in range(70)]
    feats = [(torch.from_numpy(rng.standard_normal((q, d)).astype(np.float32)).cuda(),
              torch.from_numpy(rng.standard_normal((g, d)).astype(np.float32)).cuda()) for q, g, d in shapes]
    with lib.Reranker(precision=precision) as R:
        jobs = [dict(xq=xq, xg=xg, k1=12, k2=4, layers=2) for xq, xg in feats]
        outs = R.run_batch(jobs)
        torch.cuda.synchronize()
        assert R.batch_status == [0] * len(jobs)
        for (xq, xg), (bi, bd) in zip(feats, outs):
            si, sd = R.run(xq, xg, 12, 4, 2)
            torch.cuda.synchronize()
            assert torch.equal(si, bi) and torch.equal(sd, bd)
        for t in (0, 3, 69):
            xq, xg = feats[t]
            ref = o.rerank(xq.cpu().numpy(), xg.cpu().numpy(), k1=12, k2=4, layers=2, mode="sparse")
            parity.assert_ranked_equal(outs[t][0].cpu().numpy(), outs[t][1].cpu().numpy(), ref.s, ref.idx)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_repeated_batch_replays_graph_on_new_data(lib, precision):
    """The same buffers three times: the second call captures a CUDA graph and
    the third replays it.  New contents in the same buffers give new results,
    equal to single calls; other keys in between evict nothing they need."""
    inst = _small_instances()[:5]
    feats = [_features(c["w"], False) for c in inst]
    rng = np.random.default_rng(8)
    with lib.Reranker(precision=precision) as R:
        jobs = []
        for c, (xq, xg) in zip(inst, feats):
            nq, ng = xq.shape[0], xg.shape[0]
            jobs.append(dict(xq=xq, xg=xg, k1=c["k1"], k2=c["k2"], layers=c["layers"],
                             out_idx=torch.empty((nq, ng), dtype=torch.int32, device="cuda"),
                             out_dist=torch.empty((nq, ng), dtype=torch.float32, device="cuda")))
        for rep in range(6):
            if rep >= 3:
                # fresh contents in the same buffers (the key is unchanged)
                for j in jobs:
                    j["xq"].copy_(torch.from_numpy(rng.standard_normal(tuple(j["xq"].shape)).astype(np.float32)))
                    j["xg"].copy_(torch.from_numpy(rng.standard_normal(tuple(j["xg"].shape)).astype(np.float32)))
            if rep == 4:
                # other keys in between: two smaller batches, each run twice (captured)
                for sub in (jobs[:2], jobs[2:4]):
                    for _ in range(2):
                        R.run_batch([dict(j, out_idx=None, out_dist=None) for j in sub])
            R.run_batch(jobs)
            torch.cuda.synchronize()
            assert R.batch_status == [0] * len(jobs)
            for j in jobs:
                si, sd = R.run(j["xq"], j["xg"], j["k1"], j["k2"], j["layers"])
                torch.cuda.synchronize()
                assert torch.equal(si, j["out_idx"]) and torch.equal(sd, j["out_dist"]), rep
        j = jobs[0]
        ref = o.rerank(j["xq"].cpu().numpy(), j["xg"].cpu().numpy(), k1=j["k1"], k2=j["k2"], layers=j["layers"],
                       mode="sparse")
        parity.assert_ranked_equal(j["out_idx"].cpu().numpy(), j["out_dist"].cpu().numpy(), ref.s, ref.idx)


def test_graph_cache_survives_workspace_regrowth(lib):
    """A captured batch graph names the workspace allocation.  A larger single
    call in between replaces the workspace (the new block may start at the same
    address); the next identical batch call must not replay the old graph, and
    its results stay equal to single calls."""
    inst = _small_instances()[:3]
    feats = [_features(c["w"], False) for c in inst]
    big = synthetic.make_workload(synthetic.WorkloadSpec("grow", 1500, 10500, 1024, 600, 0.35, 0, None, seed=77))
    bq, bg = torch.from_numpy(big.xq).cuda(), torch.from_numpy(big.xg).cuda()
    with lib.Reranker(precision="bf16") as R:
        jobs = []
        for c, (xq, xg) in zip(inst, feats):
            nq, ng = xq.shape[0], xg.shape[0]
            jobs.append(dict(xq=xq, xg=xg, k1=c["k1"], k2=c["k2"], layers=c["layers"],
                             out_idx=torch.empty((nq, ng), dtype=torch.int32, device="cuda"),
                             out_dist=torch.empty((nq, ng), dtype=torch.float32, device="cuda")))
        for _ in range(3):  # direct, captured, replayed
            R.run_batch(jobs)
        torch.cuda.synchronize()
        ws0 = R.last_info()["workspace_bytes"]
        R.run(bq, bg, 26, 7, 2, topk_out=10)
        torch.cuda.synchronize()
        assert R.last_info()["workspace_bytes"] > ws0, "the single call did not grow the workspace"
        for _ in range(3):
            for j in jobs:
                j["out_idx"].fill_(-1)
            R.run_batch(jobs)
            torch.cuda.synchronize()
            assert R.batch_status == [0] * len(jobs)
            for j in jobs:
                si, sd = R.run(j["xq"], j["xg"], j["k1"], j["k2"], j["layers"])
                torch.cuda.synchronize()
                assert torch.equal(si, j["out_idx"]) and torch.equal(sd, j["out_dist"])


def test_batch_host_buffers(lib):
    """NumPy (host) inputs and outputs in a batch are staged by the library."""
    inst = _small_instances()[:3]
    with lib.Reranker(precision="bf16") as R:
        jobs = [dict(xq=c["w"].xq, xg=c["w"].xg, k1=c["k1"], k2=c["k2"], layers=c["layers"]) for c in inst]
        outs = R.run_batch(jobs)
        for c, (bi, bd) in zip(inst, outs):
            ref = o.rerank(c["w"].xq, c["w"].xg, k1=c["k1"], k2=c["k2"], layers=c["layers"], mode="sparse")
            parity.assert_ranked_equal(bi, bd, ref.s, ref.idx)


def test_batch_rejects_bad_instance_before_running(lib):
    inst = _small_instances()[:2]
    with lib.Reranker() as R:
        xq, xg = _features(inst[0]["w"], False)
        jobs = [dict(xq=xq, xg=xg, k1=20, k2=5, layers=1), dict(xq=xq, xg=xg, k1=5, k2=7, layers=1)]
        with pytest.raises(lib.RerankError) as e:
            R.run_batch(jobs)
        assert e.value.status == 1
        assert R.batch_status == [0, 1]


def test_batch_overflow_rerun():
    """Instances whose layer buffers overflow are rerun alone with the capacity they asked for."""
    code = (
        "import numpy as np, torch, sys; sys.path.insert(0, '.'); sys.path.insert(0, 'tests');"
        "import parity; from oracle import rerank_oracle as o;"
        "from paper_2012_07620_gb300 import rerank;"
        "rng = np.random.default_rng(11);"
        "xs = [(rng.standard_normal((q, 128)).astype(np.float32), rng.standard_normal((g, 128)).astype(np.float32))"
        "      for q, g in [(64, 900), (30, 500), (80, 1100)]];"
        "R = rerank.Reranker(precision='bf16');"
        "outs = R.run_batch([dict(xq=torch.from_numpy(a).cuda(), xg=torch.from_numpy(b).cuda(), k1=26, k2=7,"
        "                         layers=2) for a, b in xs]);"
        "torch.cuda.synchronize();"
        "[parity.assert_ranked_equal(i.cpu().numpy(), d.cpu().numpy(), r.s, r.idx)"
        " for (i, d), r in zip(outs, [o.rerank(a, b, 26, 7, 2, mode='sparse') for a, b in xs])];"
        "print('ok')"
    )
    env = dict(os.environ, RERANK_TEST_CAP_H="60000")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]


def test_batched_64_instances_full_size(lib):
    """The 64-instance workload (N log-uniform 500-8000, d in {256, 512, 2048}, BF16
    features): one batched call equals 64 sequential rerank_run calls bit for bit;
    the three smallest instances also against the oracle."""
    specs = synthetic.batched_specs()
    inst = []
    for s in specs:
        w = synthetic.make_workload(s["spec"])
        inst.append((w, s))
    feats = [(torch.from_numpy(w.xq).bfloat16().cuda(), torch.from_numpy(w.xg).bfloat16().cuda()) for w, _ in inst]
    with lib.Reranker(precision="bf16") as R:
        jobs = [dict(xq=xq, xg=xg, k1=s["k1"], k2=s["k2"], layers=s["layers"]) for (xq, xg), (_, s) in
                zip(feats, inst)]
        outs = R.run_batch(jobs)
        torch.cuda.synchronize()
        for (xq, xg), (w, s), (bi, bd) in zip(feats, inst, outs):
            si, sd = R.run(xq, xg, s["k1"], s["k2"], s["layers"])
            torch.cuda.synchronize()
            assert torch.equal(si, bi) and torch.equal(sd, bd), s["spec"].name
        order = np.argsort([w.spec.n for w, _ in inst])[:3]
        for t in order:
            (xq, xg), (w, s), (bi, bd) = feats[t], inst[t], outs[t]
            oq, og = _oracle_inputs(xq, xg)
            ref = o.rerank(oq, og, k1=s["k1"], k2=s["k2"], layers=s["layers"], mode="sparse")
            parity.assert_ranked_equal(bi.cpu().numpy(), bd.cpu().numpy(), ref.s, ref.idx)

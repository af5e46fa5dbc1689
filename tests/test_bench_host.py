"""Host-side arithmetic of bench.py's roofline objects (no GPU).

The figures follow the per-unit counts stated beside each function: 2 N^2 d
flops for the similarity GEMM, and the bytes each memory-side stage must move.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")


def test_similarity_roofline_counts_the_full_square():
    n, d = 23100, 2048
    r = bench._roofline("bf16", 1.0, n, d, "market")
    assert r["flops_per_launch"] == 2.0 * n * n * d
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2.0 * n * n * d / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    f = bench._roofline("fp32", 1.0, n, d, "market")
    assert f["bound"] == "alu" and f["traffic"] is None


def test_stage_rooflines_bytes():
    nq, ng, d, k1, k2 = 3368, 19732, 2048, 26, 7
    n = nq + ng
    h_nnz = [731000, 1780000, 2540000] + [0] * 6
    st = {"normalize": 0.1, "refine": 1.0, "propagate": 0.3, "rank": 0.6, "graph": 0.09}
    r = bench._stage_rooflines("bf16", st, nq, ng, d, k1, k2, 22, h_nnz, 2, "market")
    np_ = 23296  # rows padded to the 256-row tensor-core tile
    assert r["normalize"]["bytes"] == n * d * 4 + np_ * d * 8
    assert r["propagate"]["bytes"] == ((k2 + 1) * 731000 + 1780000 + (k2 + 1) * 1780000 + 2540000) * 8
    assert r["rank"]["bytes"] == nq * ng * 8
    assert "graph" not in r
    for k in ("normalize", "propagate", "rank"):
        v = r[k]
        assert v["achieved_gbs"] == pytest.approx(v["bytes"] / (v["ms"] * 1e-3) / 1e9)
        assert v["frac_of_hbm"] == pytest.approx(v["achieved_gbs"] / r["peak_gbs"])
    # the refinement is a gather: its floor is every unit row read once; the
    # first rescoring batch's rows ((k1 + 7) & ~3 = 32 per row) are a gather
    # rate, with no HBM fraction
    ref = r["refine"]
    assert "frac_of_hbm" not in ref
    assert ref["floor_bytes"] == n * d * 4
    assert ref["floor_frac_of_hbm"] == pytest.approx(n * d * 4 / 1e-3 / 1e9 / r["peak_gbs"])
    assert ref["gathered_bytes"] == n * 32 * d * 4
    assert ref["gather_rate_gbs"] == pytest.approx(n * 32 * d * 4 / 1e-3 / 1e9)
    # a small rescore margin caps the first batch at k1 + m rows
    assert bench._stage_rooflines("fp32", st, nq, ng, d, k1, k2, 2, h_nnz, 2, "market")["refine"][
        "gathered_bytes"] == n * 28 * d * 4

"""Tensor-core (BF16 / FP8-E4M3) similarity path against the FP64 oracle and the FP32 path.

The low-precision GEMM only proposes candidates; the neighbour lists must
still equal the oracle's exactly, and every later stage must match the FP32
path bit for bit (same lists, same rescored weights).
"""
import numpy as np
import pytest

import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    return rerank


def _run(R, xq, xg, k1, k2, layers, topk=0):
    idx, dist = R.run(torch.from_numpy(xq).cuda(), torch.from_numpy(xg).cuda(), k1, k2, layers, topk)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def _unit(x):
    x = np.asarray(x, np.float64)
    return x / np.linalg.norm(x, axis=1, keepdims=True)


CASES = [
    ("tiny", None, 26, 7, 2),
    ("clustered_ragged", synthetic.WorkloadSpec("t", 129, 1200, 200, 60, 0.35, 0, None, seed=7), 26, 7, 2),
    ("clustered_wide", synthetic.WorkloadSpec("t", 300, 2700, 256, 150, 0.35, 0, None, seed=8), 30, 5, 3),
]


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_lowprec_matches_oracle_and_fp32(lib, precision, case):
    name, spec, k1, k2, layers = CASES[case]
    w = synthetic.make_workload(spec or synthetic.TINY)
    ref = o.rerank(w.xq, w.xg, k1=k1, k2=k2, layers=layers, mode="sparse")
    with lib.Reranker(precision=precision) as R, lib.Reranker(precision="fp32") as F:
        idx, dist = _run(R, w.xq, w.xg, k1, k2, layers)
        n = len(w.xq) + len(w.xg)
        knn = R.debug("knn_idx").reshape(n, k1)
        parity.assert_knn_equal(knn, ref.knn_idx, ref.knn_score, _unit(np.concatenate([w.xq, w.xg])))
        parity.assert_ranked_equal(idx, dist, ref.s, ref.idx)
        fidx, fdist = _run(F, w.xq, w.xg, k1, k2, layers)
        assert (fidx == idx).all() and (fdist == dist).all(), "differs from the FP32 path"


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_candidate_scores_within_error_model(lib, precision):
    """The tensor-core scores obey the bound the certificate assumes:
    |g_ij - <q_i, q_j>| <= (dp/16 + 32) 2u ||q_i|| ||q_j|| (FP32 accumulation),
    with q the BF16 (or scaled FP8) copy of the unit rows."""
    w = synthetic.make_workload(synthetic.TINY)
    k1 = 26
    with lib.Reranker(precision=precision) as R:
        _run(R, w.xq, w.xg, k1, 7, 1)
        ps = R.debug("part_s")
        pi = R.debug("part_i")
        qerr = R.debug("qerr")
        n = len(w.xq) + len(w.xg)
        K = R.last_info()["candidates_per_row"]
        P = ps.size // (n * K)
    x = np.concatenate([w.xq, w.xg]).astype(np.float32)
    d = x.shape[1]
    dp = 128 if precision == "fp8" else 64
    dp = (d + dp - 1) // dp * dp
    r32 = (1.0 / np.sqrt((x.astype(np.float64) ** 2).sum(1))).astype(np.float32)
    xh = x * r32[:, None]
    if precision == "bf16":
        q = torch.from_numpy(xh).to(torch.bfloat16).double().numpy()
    else:
        amax = np.abs(xh).max(1)
        sc = (np.float32(448.0) / amax).astype(np.float32)
        inv = (amax / np.float32(448.0)).astype(np.float32)
        q8 = torch.from_numpy(xh * sc[:, None]).to(torch.float8_e4m3fn).double().numpy()
        q = q8 * inv[:, None].astype(np.float64)
    qn = np.linalg.norm(q, axis=1)
    ps = ps.reshape(n, P, K)
    pi = pi.reshape(n, P, K)
    bound = (dp / 16 + 32) * 2 * U
    worst = 0.0
    for i in range(n):
        m = (pi[i] != 0x7FFFFFFF) & (pi[i] != i)
        js = pi[i][m]
        exact = q[js] @ q[i]
        err = np.abs(ps[i][m].astype(np.float64) - exact) / (qn[i] * qn[js])
        worst = max(worst, float(err.max(initial=0.0)))
    assert worst <= bound, (worst, bound)
    # the per-row quantisation bound covers the actual error
    act = np.linalg.norm(xh.astype(np.float64) - q, axis=1)
    assert (act <= qerr[:n] * (1 + 1e-6)).all()

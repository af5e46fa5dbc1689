"""Invariants of the method checked on the CUDA path alone (no oracle).

* Scaling a row by a power of two changes nothing, bit for bit: the unit rows
  (Eq. 7) are then identical, and so is every later step.
* Permuting the gallery permutes the ranked lists (Sec. 3: every step is
  defined per vertex pair), up to the order inside groups of equal scores.
* With k2 = 1 a layer of Eq. 14 maps h_i to 2 h_i, which the normalisation
  undoes, so the output does not depend on the number of layers.
"""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def inst():
    spec = synthetic.WorkloadSpec("inv", 130, 1210, 96, 60, 0.35, 40, None, seed=31)
    return synthetic.make_workload(spec)


def _run(R, xq, xg, k1=20, k2=6, layers=2):
    tq = torch.from_numpy(np.ascontiguousarray(xq, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(xg, dtype=np.float32)).cuda()
    idx, dist = R.run(tq, tg, k1, k2, layers)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def assert_same_ranking(idx_a, dist_a, idx_b, dist_b, tol):
    """Full lists over the same gallery: every item's distance agrees within
    tol, and list b is in ascending order of list a's distances up to tol
    (so the two orders differ only inside groups of near-equal scores)."""
    assert idx_a.shape == idx_b.shape
    for q in range(idx_a.shape[0]):
        da = np.empty(idx_a.shape[1])
        da[idx_a[q]] = dist_a[q]
        db = np.empty(idx_b.shape[1])
        db[idx_b[q]] = dist_b[q]
        assert np.array_equal(np.sort(idx_a[q]), np.arange(idx_a.shape[1]))
        assert np.array_equal(np.sort(idx_b[q]), np.arange(idx_b.shape[1]))
        assert np.abs(da - db).max() <= tol, q
        seq = da[idx_b[q]]
        assert (np.diff(seq) >= -tol).all(), q


def test_power_of_two_row_scaling_is_bit_exact(R, inst):
    rng = np.random.default_rng(5)
    sq = np.exp2(rng.integers(-4, 5, size=(len(inst.xq), 1))).astype(np.float32)
    sg = np.exp2(rng.integers(-4, 5, size=(len(inst.xg), 1))).astype(np.float32)
    i0, d0 = _run(R, inst.xq, inst.xg)
    i1, d1 = _run(R, inst.xq * sq, inst.xg * sg)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)


def test_gallery_permutation_permutes_the_lists(R, inst):
    rng = np.random.default_rng(6)
    perm = rng.permutation(len(inst.xg))
    i0, d0 = _run(R, inst.xq, inst.xg)
    ip, dp = _run(R, inst.xq, inst.xg[perm])
    # item p of the permuted gallery is item perm[p] of the original one
    assert_same_ranking(i0, d0, perm[ip], dp, tol=2e-6)


def test_k2_one_output_does_not_depend_on_layers(R, inst):
    outs = [_run(R, inst.xq, inst.xg, k1=20, k2=1, layers=L) for L in (0, 1, 3)]
    for i, d in outs[1:]:
        assert_same_ranking(outs[0][0], outs[0][1], i, d, tol=2e-6)

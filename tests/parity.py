"""Comparison rules shared by the GPU parity tests.

Neighbour lists: equal to the oracle's; a position may differ only where the
oracle's own scores of the two entries are within 1e-12 (FP64 rounding ties).
Final lists: at every position p the oracle score of the GPU's entry is within
1e-6 of the oracle score at p (so entries may swap only across near-ties),
every list is a set of distinct gallery indices, entries the oracle scores
exactly 0 appear in ascending index order, and distances agree with the
oracle's 1 - s within 1e-5 relative to max(d, 1 - d).
"""
import numpy as np

SCORE_TOL = 1e-6
DIST_RTOL = 1e-5
KNN_TIE = 1e-12


def assert_knn_equal(gpu_idx, ref_idx, ref_score, xu_hat=None):
    gpu_idx = np.asarray(gpu_idx)
    assert gpu_idx.shape == ref_idx.shape
    bad = np.argwhere(gpu_idx != ref_idx)
    for i, p in bad:
        # only a tie in FP64 may reorder two entries
        assert xu_hat is not None, f"row {i} position {p}: {gpu_idx[i, p]} != {ref_idx[i, p]}"
        s_gpu = float(xu_hat[i] @ xu_hat[gpu_idx[i, p]]) if gpu_idx[i, p] != i else 1.0
        assert abs(s_gpu - ref_score[i, p]) <= KNN_TIE, (i, p, s_gpu, ref_score[i, p])
    return len(bad)


def assert_ranked_equal(gpu_idx, gpu_dist, ref_s, ref_idx, topk=None):
    """gpu_idx/gpu_dist: (Q, T); ref_s: (Q, G) oracle scores; ref_idx: (Q, G) oracle order."""
    gpu_idx = np.asarray(gpu_idx)
    gpu_dist = np.asarray(gpu_dist)
    q, t = gpu_idx.shape
    g = ref_s.shape[1]
    assert (gpu_idx >= 0).all() and (gpu_idx < g).all()
    srt = np.sort(gpu_idx, axis=1)
    rep = np.flatnonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1)) if t > 1 else []
    assert len(rep) == 0, f"row {rep[0]} repeats an index"
    got = np.take_along_axis(ref_s, gpu_idx.astype(np.int64), axis=1)
    want = np.take_along_axis(ref_s, ref_idx[:, :t], axis=1)
    dev = np.abs(got - want)
    assert dev.max() <= SCORE_TOL, f"order deviates by {dev.max():.3e} at {np.unravel_index(dev.argmax(), dev.shape)}"
    zero = want == 0.0
    assert (gpu_idx[zero] == ref_idx[:, :t][zero]).all(), "zero tail not in ascending gallery order"
    d_ref = 1.0 - got
    err = np.abs(gpu_dist.astype(np.float64) - d_ref)
    lim = DIST_RTOL * np.maximum(d_ref, 1.0 - d_ref)
    assert (err <= lim).all(), f"distance error {err.max():.3e}"
    swaps = int((gpu_idx != ref_idx[:, :t]).sum())
    return dict(max_score_dev=float(dev.max()), max_dist_err=float(err.max()), swapped_positions=swaps)

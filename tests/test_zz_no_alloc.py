"""rerank_knn_noalloc: neighbour lists without any device allocation.

Some callers cannot allocate device memory: they run inside a framework
whose memory pool already owns the GPU, in a latency-bound loop that cannot
wait for an allocation, or under a fixed memory footprint.  For them the
library offers rerank_knn_noalloc, which keeps its temporaries in a fixed
scratch area compiled into the library.  These tests call it through the C
ABI on several calls in a row that share that scratch area (the limit
corner n = 4096, d = 256, k = 48 among them, then smaller calls, so that
leftovers of an earlier call would show), compare every call with the
allocating entry point rerank_knn, and compare one call directly with the
FP64 oracle's neighbour lists (Eq. 7-8).  They also check that sizes over
the limits and host buffers are refused.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

import parity
from oracle import rerank_oracle as o

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EINVAL, EBUDGET = 1, 3


def _entry():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_07620_gb300 import rerank
    lib = rerank.load_library()
    fn = lib.rerank_knn_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn, rerank


# (n, d, k, dtype): an ordinary call, the limit corner (n, d and k at their
# maxima: the scratch layout is full and the candidate lists are full length),
# BF16 input with a width that is not a multiple of 4 (the scalar
# normalisation path), and a small call after the big ones.
CALLS = [(4000, 256, 30, "f32"), (4096, 256, 48, "f32"), (1500, 130, 20, "bf16"), (700, 64, 12, "f32")]


def _score_bound(d):
    dp = -(-d // 64) * 64
    return (dp / 32 + 10) * 2.0 ** -24 * 1.01


def test_noalloc_matches_allocating_knn_and_oracle_on_consecutive_calls():
    fn, rerank = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    with rerank.Reranker(device=0) as ref:
        for call, (n, d, k, dt) in enumerate(CALLS):
            x32 = np.random.default_rng(40 + call).standard_normal((n, d)).astype(np.float32)
            x = torch.from_numpy(x32).cuda()
            if dt == "bf16":
                x = x.bfloat16()
            idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
            score = torch.empty((n, k), dtype=torch.float32, device="cuda")
            st = fn(x.data_ptr(), n, d, 1 if dt == "bf16" else 0, k, idx.data_ptr(), score.data_ptr(), stream)
            assert st == 0, rerank.strerror(st)
            ridx, rscore = ref.knn(x, k)
            torch.cuda.synchronize()
            got_i, got_s = idx.cpu().numpy(), score.cpu().numpy()
            assert (got_i == ridx.cpu().numpy()).all(), f"call {call}: indices differ from rerank_knn"
            np.testing.assert_allclose(got_s, rscore.cpu().numpy(), rtol=0, atol=2e-6)
            if call in (1, 2):
                # directly against the oracle (FP64, the exact input values)
                xin = x.float().cpu().numpy().astype(np.float64)
                oi, os_ = o.knn_lists(xin, k)
                parity.assert_knn_equal(got_i, oi, os_, o.unit_rows(xin))
                assert np.abs(got_s - os_).max() <= _score_bound(d)


def test_noalloc_refuses_sizes_over_the_limits_and_host_buffers():
    fn, rerank = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.zeros((5000, 300), dtype=torch.float32, device="cuda")
    idx = torch.empty((5000, 80), dtype=torch.int32, device="cuda")
    score = torch.empty((5000, 80), dtype=torch.float32, device="cuda")
    assert fn(x.data_ptr(), 5000, 8, 0, 10, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET   # n
    assert fn(x.data_ptr(), 100, 300, 0, 10, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET  # d
    assert fn(x.data_ptr(), 100, 8, 0, 80, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET    # k
    assert fn(x.data_ptr(), 100, 8, 0, 49, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET    # k = max + 1
    # a pageable host array is refused before anything runs
    hx = np.ones((100, 8), dtype=np.float32)
    assert fn(hx.ctypes.data, 100, 8, 0, 10, idx.data_ptr(), score.data_ptr(), stream) == EINVAL
    hi = np.empty((100, 10), dtype=np.int32)
    assert fn(x.data_ptr(), 100, 8, 0, 10, hi.ctypes.data, score.data_ptr(), stream) == EINVAL

"""rerank_knn_noalloc: neighbour lists without any device allocation.

Some callers cannot allocate device memory: they run inside a framework
whose memory pool already owns the GPU, in a latency-bound loop that cannot
wait for an allocation, or under a fixed memory footprint.  For them the
library offers rerank_knn_noalloc, which keeps its temporaries in a fixed
scratch area compiled into the library.  These tests call it through the C
ABI and compare it with the allocating entry point rerank_knn on two calls
in a row (the second one smaller, so leftovers of the first call in the
shared scratch area would show), and check that sizes over the limits are
refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EBUDGET = 3


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


def test_noalloc_matches_allocating_knn_on_two_calls():
    fn, rerank = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    with rerank.Reranker(device=0) as ref:
        for call, (n, d, k) in enumerate([(4000, 256, 30), (1500, 100, 20)]):
            x = torch.from_numpy(np.random.default_rng(40 + call).standard_normal((n, d)).astype(np.float32)).cuda()
            idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
            score = torch.empty((n, k), dtype=torch.float32, device="cuda")
            st = fn(x.data_ptr(), n, d, 0, k, idx.data_ptr(), score.data_ptr(), stream)
            assert st == 0, rerank.strerror(st)
            ridx, rscore = ref.knn(x, k)
            torch.cuda.synchronize()
            assert torch.equal(idx.cpu(), ridx.cpu()), f"call {call}: indices differ"
            np.testing.assert_allclose(score.cpu().numpy(), rscore.cpu().numpy(), rtol=0, atol=2e-6)


def test_noalloc_refuses_sizes_over_the_limits():
    fn, rerank = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.zeros((5000, 300), dtype=torch.float32, device="cuda")
    idx = torch.empty((5000, 80), dtype=torch.int32, device="cuda")
    score = torch.empty((5000, 80), dtype=torch.float32, device="cuda")
    assert fn(x.data_ptr(), 5000, 8, 0, 10, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET   # n
    assert fn(x.data_ptr(), 100, 300, 0, 10, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET  # d
    assert fn(x.data_ptr(), 100, 8, 0, 80, idx.data_ptr(), score.data_ptr(), stream) == EBUDGET    # k

"""Failure detection on the GPU without a fault.

Every wait of the tensor-core kernel (TMA ring, MMA issue, epilogue) has an
iteration limit.  A test hook (RERANK_TEST_TC_STALL) makes the kernel's TMA
warp issue nothing, so the MMA and epilogue waits run out: the kernel raises
its abort flag, records a timeout bit and returns (no copy or MMA is ever in
flight on that path).  The call must return ETIMEOUT, and the same context
must then give the oracle's result.  Argument errors are checked too.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STALL_CHILD = r"""
import os, sys, time
sys.path.insert(0, '.'); sys.path.insert(0, 'tests')
import numpy as np, torch
import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import rerank, synthetic
w = synthetic.make_workload(synthetic.TINY)
xq, xg = torch.from_numpy(w.xq).cuda(), torch.from_numpy(w.xg).cuda()
R = rerank.Reranker(precision=sys.argv[1])
t0 = time.time()
try:
    R.run(xq, xg, 26, 7, 2)
    print('returned without error')
    sys.exit(1)
except rerank.RerankError as e:
    assert e.status == 5, e.status          # ETIMEOUT
    assert R.last_info()['error_bits'] & 16  # the device's timeout bit
    print('etimeout after %.2f s' % (time.time() - t0))
del os.environ['RERANK_TEST_TC_STALL']
i, d = R.run(xq, xg, 26, 7, 2)
torch.cuda.synchronize()
ref = o.rerank(w.xq, w.xg, 26, 7, 2, mode='sparse')
parity.assert_ranked_equal(i.cpu().numpy(), d.cpu().numpy(), ref.s, ref.idx)
print('ok')
"""


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_stalled_wait_returns_etimeout_and_context_recovers(built, precision):
    env = dict(os.environ, RERANK_TEST_TC_STALL="1")
    r = subprocess.run([sys.executable, "-c", STALL_CHILD, precision], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
    assert "etimeout" in r.stdout


BATCH_STALL_CHILD = r"""
import os, sys
sys.path.insert(0, '.'); sys.path.insert(0, 'tests')
import numpy as np, torch
import parity
from oracle import rerank_oracle as o
from paper_2012_07620_gb300 import rerank
rng = np.random.default_rng(4)
xs = [(torch.from_numpy(rng.standard_normal((q, 64)).astype(np.float32)).cuda(),
       torch.from_numpy(rng.standard_normal((g, 64)).astype(np.float32)).cuda()) for q, g in [(20, 300), (9, 150)]]
R = rerank.Reranker(precision=sys.argv[1])
jobs = [dict(xq=a, xg=b, k1=10, k2=4, layers=1) for a, b in xs]
try:
    R.run_batch(jobs)
    print('returned without error')
    sys.exit(1)
except rerank.RerankError as e:
    assert e.status == 5, e.status
    assert R.batch_status == [5, 5], R.batch_status
del os.environ['RERANK_TEST_TC_STALL']
outs = R.run_batch(jobs)
torch.cuda.synchronize()
for (a, b), (i, d) in zip(xs, outs):
    ref = o.rerank(a.cpu().numpy(), b.cpu().numpy(), 10, 4, 1, mode='sparse')
    parity.assert_ranked_equal(i.cpu().numpy(), d.cpu().numpy(), ref.s, ref.idx)
print('ok')
"""


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_stalled_batched_launch_times_out_every_instance(built, precision):
    """A batched similarity launch whose waits run out reports ETIMEOUT for
    every instance it carried; the context then runs the batch correctly."""
    env = dict(os.environ, RERANK_TEST_TC_STALL="1")
    r = subprocess.run([sys.executable, "-c", BATCH_STALL_CHILD, precision], env=env, capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])


def test_device_reports_bad_rows(built):
    """A non-finite query row and an all-zero gallery row are found on the device
    (BF16 path): EINVAL and the first bad vertex index."""
    torch = pytest.importorskip("torch")
    from paper_2012_07620_gb300 import rerank, synthetic
    w = synthetic.make_workload(synthetic.TINY)
    nq = len(w.xq)
    xq, xg = w.xq.copy(), w.xg.copy()
    xq[37, 5] = np.nan
    xg[5] = 0.0
    cases = [(xq, w.xg, 37), (w.xq, xg, nq + 5), (xq, xg, 37)]
    for q, g, want in cases:
        with rerank.Reranker(precision="bf16") as R:
            with pytest.raises(rerank.RerankError) as e:
                R.run(torch.from_numpy(q).cuda(), torch.from_numpy(g).cuda(), 26, 7, 2)
            assert e.value.status == 1
            assert R.last_info()["bad_row"] == want

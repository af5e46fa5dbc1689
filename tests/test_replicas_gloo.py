"""The N > 1 path of bench.py on the CPU: two `gloo` ranks.

With N GPUs every rank runs an independent replica (instances need no
exchange), so the only cross-rank steps are the barrier around the timed
region and the max over ranks of the measured time; the reference arm runs
on rank 0 alone and the other ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench._dist_setup()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench._barrier(w)
    t = bench._max_over_ranks(10.0 * (rank + 1), w)
    out.put((rank, t))
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 20.0, 1: 20.0}


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "tiny", "--gpus", "2", "--steps", "3", "--warmup", "1", "--ref-seconds", "60"]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=280, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    # the whole oracle ran for every step it reports (the tiny case fits the budget)
    assert d["steps"] == 3 and d["warmup"] == 1 and d["requested"] == {"steps": 3, "warmup": 1, "budget_s": 60.0}
    assert set(d["cpu_baseline"]["stages_ms"]) == {"knn", "graph", "propagate", "rank"}
    assert "no scaling" in d["cpu_baseline"]["sample"]

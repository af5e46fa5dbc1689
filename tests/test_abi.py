"""The C ABI on the host: the library builds, loads, exports every function
declared in include/rerank.h, and validates arguments without a GPU."""
import re
import subprocess

import pytest

from paper_2012_07620_gb300 import build, rerank

HEADER = build.INCLUDE / "rerank.h"


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rerank.load_library()


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rerank_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "rerank_run" in names and "rerank_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", str(build.LIB)], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rerank_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_check_args(lib):
    ok = rerank.check_args(100, 900, 128, "f32", 26, 7, 2, 0)
    assert ok == 0
    bad = [
        (0, 900, 128, "f32", 26, 7, 2, 0),      # no queries
        (100, 0, 128, "f32", 26, 7, 2, 0),      # no gallery
        (100, 900, 0, "f32", 26, 7, 2, 0),      # d = 0
        (100, 900, 128, 5, 26, 7, 2, 0),        # dtype
        (100, 900, 128, "f32", 7, 26, 2, 0),    # k2 > k1
        (100, 900, 128, "f32", 0, 0, 2, 0),     # k1 = 0
        (10, 10, 128, "f32", 21, 7, 2, 0),      # k1 > n
        (100, 900, 128, "f32", 26, 7, -1, 0),   # layers < 0
        (100, 900, 128, "f32", 26, 7, 2, 901),  # topk > ng
    ]
    for args in bad:
        assert rerank.check_args(*args) == 1, args


def test_strerror(lib):
    assert rerank.strerror(0) == "ok"
    assert "budget" in rerank.strerror(3)


def test_create_without_gpu_reports_status(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rerank.RerankError) as e:
        rerank.Reranker(device=0)
    assert e.value.status == 4  # ECUDA, not a crash
    # the failing CUDA call is named, in the status text and in the exception
    assert "cudaGetDeviceCount" in lib.rerank_last_cuda_error().decode()
    assert "cudaGetDeviceCount" in str(e.value)


def _bucket(n):
    # the largest b with 2^b <= n^2 (half-octave bucket of the vertex count)
    b = 0
    while 2 ** (b + 1) <= n * n:
        b += 1
    return b


def test_tuning_table_lookup(lib, tmp_path):
    """The autotuner's JSON table: entries found by (precision, d, bucket of N)."""
    path = tmp_path / "tune.json"
    n = 23100
    path.write_text('{"version": 1, "entries": [\n'
                    f'  {{"precision": 1, "d": 2048, "n_bucket": {_bucket(n)}, "sim_chunks": 4, "prop_warps": 16, '
                    '"refine_order": 0, "ms": 7.5},\n'
                    '  {"precision": 0, "d": 128, "n_bucket": 19, "sim_chunks": 2, "prop_warps": 8, '
                    '"refine_order": 1, "rescore_m": 22, "ms": 0.3}\n]}\n')
    t = rerank.tuning_lookup(str(path), "bf16", n, 2048)
    assert t == {"sim_chunks": 4, "prop_warps": 16, "refine_order": 0, "rescore_m": -1, "n_bucket": _bucket(n),
                 "ms": 7.5}
    assert rerank.tuning_lookup(str(path), "bf16", int(n * 0.97), 2048)["sim_chunks"] == 4  # same half-octave
    assert rerank.tuning_lookup(str(path), "bf16", n * 2, 2048) is None
    assert rerank.tuning_lookup(str(path), "fp8", n, 2048) is None
    t2 = rerank.tuning_lookup(str(path), "fp32", 1000, 128)  # 2 log2(1000) = 19.93
    assert t2["prop_warps"] == 8 and t2["rescore_m"] == 22
    with pytest.raises(rerank.RerankError):
        rerank.tuning_lookup(str(tmp_path / "missing.json"), "bf16", n, 2048)
    bad = tmp_path / "bad.json"
    bad.write_text("not a table")
    with pytest.raises(rerank.RerankError):
        rerank.tuning_lookup(str(bad), "bf16", n, 2048)


@pytest.mark.parametrize("n", [2, 3, 4, 1000, 1023, 1024, 1025, 1448, 1449, 23100, 50000, 2 ** 20, 3 ** 13])
def test_tuning_bucket_boundaries(lib, tmp_path, n):
    """The library's bucket is floor(2 log2 N): 2^b <= N^2 < 2^(b+1)."""
    b = _bucket(n)
    assert 2 ** b <= n * n < 2 ** (b + 1)
    path = tmp_path / "t.json"
    path.write_text('{"entries": [{"precision": 1, "d": 64, "n_bucket": %d, "sim_chunks": 3, "prop_warps": 4, '
                    '"refine_order": 1}]}' % b)
    assert rerank.tuning_lookup(str(path), "bf16", n, 64)["n_bucket"] == b

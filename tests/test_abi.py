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

"""The ctypes mirrors in rerank.py have the layout of the C structs in
include/rerank.h (same size, every field at the same offset) and the same
status and enum values.  A mismatch would pass garbage across the boundary
without any error, so the checks compile the header with the host C compiler
and compare (no GPU)."""
import ctypes
import shutil
import subprocess

import pytest

from paper_2012_07620_gb300 import build, rerank

PAIRS = [
    ("rerank_config", rerank.RerankConfig),
    ("rerank_info", rerank.RerankInfo),
    ("rerank_job", rerank.RerankJob),
    ("rerank_serve_config", rerank.ServeConfig),
    ("rerank_request", rerank.Request),
    ("rerank_ticket_info", rerank.TicketInfo),
    ("rerank_serve_info", rerank.ServeInfo),
    ("rerank_tuning", rerank.Tuning),
]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rerank.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", f"-I{build.INCLUDE}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    return got


def test_ctypes_mirrors_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, py in PAIRS:
        assert c[(cname, ".")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert c[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_python_constants_match_the_header(tmp_path):
    """Status codes and the enum values the binding passes by number."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    names = {f"RERANK_{v}": k for k, v in rerank.STATUS_NAMES.items()}
    names.update({f"RERANK_PREC_{k.upper()}": v for k, v in rerank.PRECISION.items()})
    names.update({f"RERANK_DTYPE_{k.upper()}": v for k, v in rerank.DTYPE.items()})
    names.update({f"RERANK_AGG_{k.upper()}": v for k, v in rerank.AGGREGATOR.items()})
    names.update({f"RERANK_FEAT_{k.upper()}": v for k, v in rerank.FEATURE.items()})
    names.update({f"RERANK_DBG_{k.upper()}": v for k, v in rerank.DEBUG.items()})
    lines = ["#include <stdio.h>", '#include "rerank.h"', "int main(void) {"]
    lines += [f'  printf("{n} %d\\n", (int){n});' for n in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", f"-I{build.INCLUDE}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {n: int(v) for n, v in (line.split() for line in out.splitlines())}
    assert got == names


def test_header_compiles_as_c_and_cpp(tmp_path):
    """The boundary is plain C with extern "C" guards: both compilers accept it
    with warnings as errors."""
    for cc, std, ext in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "cpp")):
        exe = shutil.which(cc)
        if exe is None:
            pytest.skip(f"no {cc}")
        src = tmp_path / f"h.{ext}"
        src.write_text('#include "rerank.h"\nint main(void) { return RERANK_OK; }\n')
        subprocess.run([exe, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", f"-I{build.INCLUDE}", str(src)],
                       check=True)
